"""Python-side objects over the libnif C ABI: device buffers come from torch
(caching allocator, streams), every computation runs in libnif's kernels.

* ``BVH``        -- bvh_build / bvh_cast_shadow / bvh_cast_closest / bvh_cast_pairs
* ``NifModel``   -- model description, grids and weights; frontend, encode,
                    infer_queries, infer
* ``Trainer``    -- FP32 master state and Adam moments; nif_train_step
* ``NifQueryFn`` -- torch.autograd.Function whose forward is nif_fwd_train and
                    whose backward is nif_mlp_bwd + nif_grid_bwd
* ``NifLossFn``  -- torch.autograd.Function around nif_loss
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L

_DT = {L.NIF_F32: torch.float32, L.NIF_F16: torch.float16, L.NIF_BF16: torch.bfloat16,
       L.NIF_E4M3: torch.float8_e4m3fn}


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def bits_to_bool(bits: torch.Tensor, n: int) -> torch.Tensor:
    """Unpack a uint32 occlusion bitmask (bit i%32 of word i/32) into bool[n]."""
    w = bits.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    sh = torch.arange(32, device=bits.device, dtype=torch.int64)
    return (((w[:, None] >> sh[None, :]) & 1).reshape(-1)[:n]).bool()


def light_cdf(weight: torch.Tensor, stream=None) -> torch.Tensor:
    """Light selection table from per-light weights (nif_light_cdf)."""
    w = weight.float().contiguous()
    cdf = torch.empty_like(w)
    L.call("nif_light_cdf", _ptr(w), int(w.numel()), _ptr(cdf), _stream(stream))
    return cdf


def light_samples(camera, t, prim, verts, tris, lights, cdf, u, spp: int, tmin: float = 1e-3,
                  albedo: float = 0.8, stream=None):
    """Shadow rays [n*spp, 8] towards sampled points of quad lights and the
    samples' values without visibility [n*spp] (nif_light_samples)."""
    n = int(camera.shape[0])
    out = torch.empty((n * spp, 8), dtype=torch.float32, device=camera.device)
    f = torch.empty(n * spp, dtype=torch.float32, device=camera.device)
    L.call("nif_light_samples", _ptr(camera), _ptr(t), _ptr(prim), _ptr(verts), _ptr(tris), n, spp,
           _ptr(lights), _ptr(cdf), int(lights.shape[0]), _ptr(u), tmin, albedo, _ptr(out), _ptr(f),
           _stream(stream))
    return out, f


def shade(f, bits, n: int, spp: int, out=None, stream=None) -> torch.Tensor:
    """Pixel radiance from sample values and their occlusion bits (nif_shade)."""
    out = out if out is not None else torch.empty(n, dtype=torch.float32, device=f.device)
    L.call("nif_shade", _ptr(f), _ptr(bits), n, spp, _ptr(out), _stream(stream))
    return out


def clear_bits(bits: torch.Tensor, n: int, stream=None) -> torch.Tensor:
    """Zero an occlusion mask of n rays on the stream (nif_bits_clear)."""
    L.call("nif_bits_clear", _ptr(bits), n, _stream(stream))
    return bits


def empty_bits(n: int, device="cuda") -> torch.Tensor:
    return torch.zeros((n + 31) // 32, dtype=torch.int32, device=device)


class BVH:
    """Exact shadow-ray visibility over a triangle soup (or object boxes)."""

    def __init__(self, verts: torch.Tensor, tris: torch.Tensor, tags: torch.Tensor | None = None,
                 boxes: bool = False, stream=None, builder: str = "lbvh"):
        """builder: "lbvh" (bvh_build, Morton-code splits) or "ploc"
        (bvh_build_ploc, locally-ordered clustering: a lower surface-area
        cost)."""
        self.n = int(tris.shape[0])
        self.builder = builder
        nb = L.lib.bvh_build_size(self.n)
        nw = (L.lib.bvh_build_ploc_workspace_size(self.n) if builder == "ploc"
              else L.lib.bvh_build_workspace_size(self.n))
        dev = verts.device
        self.buf = torch.empty(nb, dtype=torch.uint8, device=dev)
        ws = torch.empty(max(nw, 256), dtype=torch.uint8, device=dev)
        if boxes:
            L.call("bvh_build_boxes_ploc" if builder == "ploc" else "bvh_build_boxes", _ptr(verts), self.n,
                   _ptr(self.buf), nb, _ptr(ws), ws.numel(), _stream(stream))
        else:
            self._inputs = (verts, tris, tags)
            L.call("bvh_build_ploc" if builder == "ploc" else "bvh_build", _ptr(verts), int(verts.shape[0]),
                   _ptr(tris), self.n, _ptr(tags), _ptr(self.buf), nb, _ptr(ws), ws.numel(), _stream(stream))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        del ws
        self._inputs = None
        self.check(stream)

    def stats(self, rays: torch.Tensor | None = None, stream=None):
        """bvh_stats: the tree's surface-area cost and, over `rays` cast
        any-hit, the mean nodes visited and triangles tested per ray."""
        n = int(rays.shape[0]) if rays is not None else 0
        sums = torch.zeros(2, dtype=torch.int64, device=self.buf.device)
        sah, nv, nt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        L.call("bvh_stats", _ptr(self.buf), _ptr(rays) if n else None, n, ctypes.byref(sah), ctypes.byref(nv),
               ctypes.byref(nt), _ptr(sums), _stream(stream))
        return {"sah_cost": sah.value, "nodes_per_ray": nv.value, "tris_per_ray": nt.value}

    def check(self, stream=None):
        """Raise NifError if the build or any traversal through this buffer
        recorded a failure (bvh_check: a tree deeper than the traversal
        stack, a stack overflow or the node-visit bound)."""
        L.call("bvh_check", _ptr(self.buf), _stream(stream))

    @classmethod
    def from_boxes(cls, boxes: torch.Tensor, stream=None, builder: str = "lbvh") -> "BVH":
        """The top level over object boxes [n][6] (bvh_build_boxes, or
        bvh_build_boxes_ploc with builder="ploc")."""
        return cls(boxes.contiguous(), boxes, boxes=True, stream=stream, builder=builder)

    def info(self):
        nn, npr, dep = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        L.call("bvh_info", _ptr(self.buf), ctypes.byref(nn), ctypes.byref(npr), ctypes.byref(dep),
               _stream())
        return {"nodes": nn.value, "prims": npr.value, "depth": dep.value}

    def cast_shadow(self, rays: torch.Tensor, out: torch.Tensor | None = None, stream=None,
                    or_into: bool = False):
        """Any-hit cast into an occlusion mask; or_into ORs the bits into
        `out` (which may be written concurrently) instead of overwriting."""
        n = int(rays.shape[0])
        bits = out if out is not None else empty_bits(n, rays.device)
        L.call("bvh_cast_shadow_or" if or_into else "bvh_cast_shadow", _ptr(self.buf), _ptr(rays), n,
               _ptr(bits), _stream(stream))
        return bits

    def cast_closest(self, rays: torch.Tensor, stream=None):
        n = int(rays.shape[0])
        t = torch.empty(n, dtype=torch.float32, device=rays.device)
        prim = torch.empty(n, dtype=torch.int32, device=rays.device)
        L.call("bvh_cast_closest", _ptr(self.buf), _ptr(rays), n, _ptr(t), _ptr(prim), _stream(stream))
        return t, prim

    def cast_pairs(self, rays, ray_id, obj, stream=None):
        nq = int(ray_id.shape[0])
        hit = torch.empty(nq, dtype=torch.uint8, device=rays.device)
        L.call("bvh_cast_pairs", _ptr(self.buf), _ptr(rays), _ptr(ray_id), _ptr(obj), nq, _ptr(hit),
               _stream(stream))
        return hit

    def cast_pairs_closest(self, rays, ray_id, obj, stream=None):
        """Per pair: the nearest hit t of the pair's object (+inf) and the
        triangle (-1)."""
        nq = int(ray_id.shape[0])
        t = torch.empty(nq, dtype=torch.float32, device=rays.device)
        prim = torch.empty(nq, dtype=torch.int32, device=rays.device)
        L.call("bvh_cast_pairs_closest", _ptr(self.buf), _ptr(rays), _ptr(ray_id), _ptr(obj), nq,
               _ptr(t), _ptr(prim), _stream(stream))
        return t, prim


def shadow_rays(camera: torch.Tensor, t: torch.Tensor, light: torch.Tensor, spp: int = 1,
                per_ray: bool = False, tmin: float = 1e-3, stream=None) -> torch.Tensor:
    n = int(camera.shape[0])
    out = torch.empty((n * spp, 8), dtype=torch.float32, device=camera.device)
    L.call("nif_shadow_rays", _ptr(camera), _ptr(t), n, spp, _ptr(light), int(per_ray), tmin,
           _ptr(out), _stream(stream))
    return out


@dataclass
class NifConfig:
    res: list
    n_features: int = 2
    log2_table: int = 19
    grid_dtype: int = L.NIF_F32
    n_hidden: int = 3
    width: int = 64
    act: int = L.NIF_ACT_RELU
    leaky_slope: float = 0.01
    mlp_dtype: int = L.NIF_F32
    net_mode: int = L.NIF_NETS_SINGLE
    tile_m: int = 0
    ctas_per_sm: int = 0
    schedule: int = L.NIF_SCHED_AUTO
    # the paper's own encoding (NIF_ENC_SPHERICAL_OUTER / _INNER): res = [R]
    # for the 2D grids, n_features = N; inner pairs add res_1d x n_features_1d
    encoding: int = L.NIF_ENC_MULTIRES
    res_1d: int = 0
    n_features_1d: int = 0
    # output rows: 1 = the occupancy logit; 5 = the primary-ray outputs
    # [z | normal | delta] (Sec. 3.2, Sec. 6.1)
    n_outputs: int = 1
    # the pair nif_infer queries first per ray (NIF_ROUND1_*)
    round1: int = L.NIF_ROUND1_NEAREST

    @property
    def n_levels(self):
        return len(self.res)

    @property
    def K(self):
        if self.encoding == L.NIF_ENC_SPHERICAL_OUTER:
            return 2 * self.n_features
        if self.encoding == L.NIF_ENC_SPHERICAL_INNER:
            return 2 * self.n_features + self.n_features_1d
        return 3 * len(self.res) * self.n_features

    def fill(self, d: "L.ModelDesc") -> "L.ModelDesc":
        """Write the shape fields of this configuration into a descriptor."""
        d.n_levels = len(self.res)
        d.n_features = self.n_features
        d.log2_table = self.log2_table
        for i, r in enumerate(self.res):
            d.res[i] = int(r)
        d.n_hidden = self.n_hidden
        d.width = self.width
        d.encoding = self.encoding
        d.res_1d = self.res_1d
        d.n_features_1d = self.n_features_1d
        d.n_outputs = self.n_outputs
        d.round1 = self.round1
        return d


class NifModel:
    """A NIF model: per-object grids and per-network weights on the device."""

    def __init__(self, cfg: NifConfig, obj_aabb: torch.Tensor, grids: torch.Tensor,
                 weights: torch.Tensor, scales: torch.Tensor | None = None):
        self.cfg = cfg
        self.obj_aabb = obj_aabb.contiguous()
        self.grids = grids
        self.weights = weights
        self.scales = scales
        self.n_obj = int(obj_aabb.shape[0])
        if cfg.net_mode == L.NIF_NETS_CLASS:
            self.n_nets = 2
        elif cfg.net_mode == L.NIF_NETS_OBJECT:
            self.n_nets = self.n_obj
        else:
            self.n_nets = 1
        self._ws = None

    def desc(self) -> L.ModelDesc:
        c = self.cfg
        d = c.fill(L.ModelDesc())
        d.grid_dtype = c.grid_dtype
        d.n_objects = self.n_obj
        d.d_obj_aabb = self.obj_aabb.data_ptr()
        d.d_grids = self.grids.data_ptr()
        d.act = c.act
        d.leaky_slope = c.leaky_slope
        d.mlp_dtype = c.mlp_dtype
        d.net_mode = c.net_mode
        d.n_nets = self.n_nets
        d.d_weights = self.weights.data_ptr()
        d.d_scales = self.scales.data_ptr() if self.scales is not None else None
        d.tile_m = c.tile_m
        d.ctas_per_sm = c.ctas_per_sm
        d.schedule = c.schedule
        return d

    @staticmethod
    def grid_vertices(cfg: NifConfig) -> int:
        """Vertices V of one grid (multi-resolution: grids are [obj][2][V][F]),
        or the elements G of one object's block (spherical: [obj][G])."""
        v = L.lib.nif_grid_vertices(ctypes.byref(cfg.fill(L.ModelDesc())))
        if v < 0:
            raise L.NifError(L.NIF_ERR_ARG, "bad grid configuration")
        return int(v)

    @staticmethod
    def weight_count(cfg: NifConfig) -> int:
        return int(L.lib.nif_weight_count(ctypes.byref(cfg.fill(L.ModelDesc()))))

    def workspace(self, max_q: int, max_rays: int = 0) -> torch.Tensor:
        d = self.desc()
        need = L.lib.nif_workspace_size(ctypes.byref(d), max_rays, max_q)
        if need == 0:
            raise L.NifError(L.NIF_ERR_ARG, L.last_error())
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.zeros(need, dtype=torch.uint8, device=self.obj_aabb.device)
        return self._ws

    def check(self, ws: torch.Tensor | None = None, stream=None):
        ws = ws if ws is not None else self._ws
        det = ctypes.c_int64()
        L.call("nif_check", _ptr(ws), ctypes.byref(det), _stream(stream))

    def frontend(self, rays: torch.Tensor, tlas: BVH | None = None, max_q: int | None = None,
                 stream=None):
        n = int(rays.shape[0])
        max_q = max_q if max_q is not None else 4 * n + 1024
        dev = rays.device
        ray_id = torch.empty(max_q, dtype=torch.int32, device=dev)
        qobj = torch.empty(max_q, dtype=torch.int32, device=dev)
        goff = torch.empty(self.n_nets + 1, dtype=torch.int64, device=dev)
        count = torch.empty(1, dtype=torch.int64, device=dev)
        ws = self.workspace(0, n)
        d = self.desc()
        L.call("nif_frontend", ctypes.byref(d), _ptr(tlas.buf) if tlas else None, _ptr(rays), n,
               _ptr(ray_id), _ptr(qobj), max_q, _ptr(goff), _ptr(count), _ptr(ws), ws.numel(),
               _stream(stream))
        return ray_id, qobj, goff, count

    def encode(self, rays, ray_id, qobj, nq: int, dtype=L.NIF_F32, stream=None):
        out = torch.empty((nq, self.cfg.K), dtype=_DT[dtype], device=rays.device)
        d = self.desc()
        L.call("nif_encode", ctypes.byref(d), _ptr(rays), _ptr(ray_id), _ptr(qobj), nq, _ptr(out),
               dtype, _stream(stream))
        return out

    def infer_queries(self, rays, ray_id, qobj, goff, nq_max: int, bits=None, logits=True,
                      stream=None):
        """Outputs of a grouped query list: logits [nq_max] (or [nq_max, O]
        with O > 1 outputs), occlusion bits OR-ed into `bits`."""
        O = self.cfg.n_outputs
        shape = (max(nq_max, 1),) if O == 1 else (max(nq_max, 1), O)
        z = torch.empty(shape, dtype=torch.float32, device=rays.device) if logits else None
        ws = self.workspace(0)
        d = self.desc()
        L.call("nif_infer_queries", ctypes.byref(d), _ptr(rays), int(rays.shape[0]), _ptr(ray_id),
               _ptr(qobj), _ptr(goff), nq_max, _ptr(bits), _ptr(z), _ptr(ws), ws.numel(),
               _stream(stream))
        return z

    def infer(self, rays, bits, tlas: BVH | None = None, max_q: int | None = None, stream=None):
        n = int(rays.shape[0])
        ws = self.workspace(max_q if max_q is not None else 4 * n + 1024, n)
        d = self.desc()
        L.call("nif_infer", ctypes.byref(d), _ptr(tlas.buf) if tlas else None, _ptr(rays), n,
               _ptr(bits), _ptr(ws), ws.numel(), _stream(stream))
        return bits

    def infer_query_counts(self, n_rays: int, stream=None) -> torch.Tensor:
        """Pairs the last infer() queried: [round 1, both rounds] (device int64)."""
        out = torch.empty(2, dtype=torch.int64, device=self.obj_aabb.device)
        d = self.desc()
        L.call("nif_infer_query_counts", ctypes.byref(d), _ptr(self._ws), self._ws.numel(), n_rays,
               _ptr(out), _stream(stream))
        return out


class Trainer:
    """Adam state for a NifModel (Sec. 5 'Training'): FP32 masters, FP32
    gradients and moments; nif_train_step refreshes the model's copies.

    half_precision: forward and MLP backward on the tensor cores with the
    model's 16-bit copies (FP32 accumulation, masters and moments FP32).
    dynamic_scale: the loss scale lives on the device, starts at loss_scale,
    halves after a step whose scaled gradients overflow the 16-bit type (the
    step is skipped) and doubles after scale_window clean steps."""

    def __init__(self, model: NifModel, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-15,
                 loss_scale=1.0, w_master: torch.Tensor | None = None,
                 g_master: torch.Tensor | None = None, deterministic: bool = False,
                 half_precision: bool = False, dynamic_scale: bool = False, scale_window: int = 2000):
        self.model = model
        dev = model.obj_aabb.device
        self.w_master = (w_master if w_master is not None else model.weights.float()).clone().contiguous()
        self.g_master = (g_master if g_master is not None else model.grids.float()).clone().contiguous()
        self.w_grad = torch.zeros_like(self.w_master)
        self.w_m = torch.zeros_like(self.w_master)
        self.w_v = torch.zeros_like(self.w_master)
        self.g_grad = torch.zeros_like(self.g_master)
        self.g_m = torch.zeros_like(self.g_master)
        self.g_v = torch.zeros_like(self.g_master)
        self.o = L.OptimDesc()
        self.o.lr, self.o.beta1, self.o.beta2, self.o.eps = lr, beta1, beta2, eps
        self.o.loss_scale = loss_scale
        self.o.step = 0
        self.o.deterministic = int(deterministic)
        self._det_ws = None
        for name in ("w_master", "w_grad", "w_m", "w_v", "g_master", "g_grad", "g_m", "g_v"):
            setattr(self.o, "d_" + name, getattr(self, name).data_ptr())
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self._ws = None
        self.o.half_precision = int(half_precision)
        self.scale = self.scale_state = None
        if dynamic_scale:
            self.scale = torch.full((1,), float(loss_scale), dtype=torch.float32, device=dev)
            self.scale_state = torch.zeros(2, dtype=torch.int32, device=dev)
            self.o.d_loss_scale = self.scale.data_ptr()
            self.o.d_scale_state = self.scale_state.data_ptr()
            self.o.scale_window = int(scale_window)

    def state_bytes(self, stream=None) -> np.ndarray:
        """The optimiser state (nif_state_save): FP32 masters, Adam moments and
        the step count in one host buffer, complete when this returns."""
        d = self.model.desc()
        buf = np.empty(int(L.lib.nif_state_size(ctypes.byref(d))), dtype=np.uint8)
        L.call("nif_state_save", ctypes.byref(d), ctypes.byref(self.o), buf.ctypes.data_as(ctypes.c_void_p),
               buf.nbytes, _stream(stream))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return buf

    def load_state_bytes(self, buf: np.ndarray, stream=None):
        """Resume from nif_state_save's buffer (nif_state_load): masters,
        moments and step restored, gradients zeroed, the model's copies
        refreshed."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        d = self.model.desc()
        L.call("nif_state_load", ctypes.byref(d), ctypes.byref(self.o), buf.ctypes.data_as(ctypes.c_void_p),
               buf.nbytes, _stream(stream))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def save(self, path: str):
        self.state_bytes().tofile(path)

    def load(self, path: str):
        self.load_state_bytes(np.fromfile(path, dtype=np.uint8))

    def _workspace(self, d, nq: int, device):
        need = L.lib.nif_train_workspace_size(ctypes.byref(d), nq)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.zeros(need, dtype=torch.uint8, device=device)
        return self._ws

    def grads(self, rays, ray_id, qobj, goff, label, nq: int, stream=None):
        """nif_train_grads: the step's forward, loss and backward into
        w_grad / g_grad (gradients of the scaled loss), without the update."""
        d = self.model.desc()
        ws = self._workspace(d, nq, rays.device)
        L.call("nif_train_grads", ctypes.byref(d), ctypes.byref(self.o), _ptr(rays), _ptr(ray_id), _ptr(qobj),
               _ptr(goff), _ptr(label), nq, _ptr(self.loss), _ptr(ws), ws.numel(), _stream(stream))
        return self.loss

    def step(self, rays, ray_id, qobj, goff, label, nq: int, stream=None, aux=None):
        """One nif_train_step (or nif_train_step_aux with the targets aux
        [nq, O-1] of an O-output network)."""
        d = self.model.desc()
        self._workspace(d, nq, rays.device)
        if self.o.deterministic:
            dn = L.lib.nif_deterministic_workspace_size(ctypes.byref(d), nq)
            if self._det_ws is None or self._det_ws.numel() < dn:
                self._det_ws = torch.empty(dn, dtype=torch.uint8, device=rays.device)
            self.o.d_det_ws = self._det_ws.data_ptr()
            self.o.det_ws_bytes = self._det_ws.numel()
        if aux is None:
            L.call("nif_train_step", ctypes.byref(d), ctypes.byref(self.o), _ptr(rays), _ptr(ray_id),
                   _ptr(qobj), _ptr(goff), _ptr(label), nq, _ptr(self.loss), _ptr(self._ws),
                   self._ws.numel(), _stream(stream))
        else:
            L.call("nif_train_step_aux", ctypes.byref(d), ctypes.byref(self.o), _ptr(rays), _ptr(ray_id),
                   _ptr(qobj), _ptr(goff), _ptr(label), _ptr(aux), nq, _ptr(self.loss), _ptr(self._ws),
                   self._ws.numel(), _stream(stream))
        return self.loss


def primary_resolve(model: NifModel, rays, ray_id, qobj, goff, nq_max: int, out, t=None, normal=None,
                    winner=None, key=None, stream=None):
    """Closest NIF hit per ray from the O >= 5 outputs `out` [nq_max, O] of a
    grouped query list (nif_primary_resolve).  t (in/out, +inf when None)
    holds the exact cast's t of the other geometry; where a NIF hit is
    nearer, t, normal [n, 3] and winner (query index) are written."""
    n = int(rays.shape[0])
    dev = rays.device
    t = t if t is not None else torch.full((n,), float("inf"), dtype=torch.float32, device=dev)
    normal = normal if normal is not None else torch.zeros((n, 3), dtype=torch.float32, device=dev)
    winner = winner if winner is not None else torch.full((n,), -1, dtype=torch.int32, device=dev)
    key = key if key is not None else torch.empty(n, dtype=torch.int64, device=dev)
    d = model.desc()
    L.call("nif_primary_resolve", ctypes.byref(d), _ptr(rays), n, _ptr(ray_id), _ptr(qobj), _ptr(goff),
           nq_max, _ptr(out), _ptr(key), _ptr(t), _ptr(normal), _ptr(winner), _stream(stream))
    return t, normal, winner


def _f32_view(model: NifModel, grids: torch.Tensor, weights: torch.Tensor) -> NifModel:
    cfg = NifConfig(**{**model.cfg.__dict__, "grid_dtype": L.NIF_F32, "mlp_dtype": L.NIF_F32})
    return NifModel(cfg, model.obj_aabb, grids, weights)


class NifQueryFn(torch.autograd.Function):
    """z = NIF(grids, weights; rays, queries): forward by nif_fwd_train, backward
    by nif_mlp_bwd (weights) and nif_grid_bwd (grid latents), all FP32."""

    @staticmethod
    def forward(ctx, grids, weights, model, rays, ray_id, qobj, goff, nq):
        m = _f32_view(model, grids, weights)
        d = m.desc()
        z = torch.empty(nq, dtype=torch.float32, device=rays.device)
        saved = torch.empty(L.lib.nif_saved_size(ctypes.byref(d), nq) // 4, dtype=torch.float32,
                            device=rays.device)
        L.call("nif_fwd_train", ctypes.byref(d), _ptr(rays), _ptr(ray_id), _ptr(qobj), _ptr(goff), nq,
               _ptr(z), _ptr(saved), _stream())
        ctx.m = m
        ctx.nq = nq
        ctx.save_for_backward(rays, ray_id, qobj, goff, saved)
        return z

    @staticmethod
    def backward(ctx, gz):
        rays, ray_id, qobj, goff, saved = ctx.saved_tensors
        m, nq = ctx.m, ctx.nq
        d = m.desc()
        gz = gz.contiguous().float()
        gw = torch.zeros_like(m.weights)
        gg = torch.zeros_like(m.grids)
        dx = torch.empty(m.cfg.K * nq, dtype=torch.float32, device=rays.device)
        L.call("nif_mlp_bwd", ctypes.byref(d), _ptr(qobj), _ptr(goff), nq, _ptr(saved), _ptr(gz),
               _ptr(gw), _ptr(dx), _stream())
        L.call("nif_grid_bwd", ctypes.byref(d), _ptr(rays), _ptr(ray_id), _ptr(qobj), nq, _ptr(dx),
               _ptr(gg), _stream())
        return gg, gw, None, None, None, None, None, None


class NifLossFn(torch.autograd.Function):
    """L = mean (sigmoid(z) - y)^2 (Sec. 5 'Training', L2 loss) by nif_loss."""

    @staticmethod
    def forward(ctx, z, label):
        nq = int(z.shape[0])
        dz = torch.empty_like(z)
        loss = torch.zeros(1, dtype=torch.float32, device=z.device)
        L.call("nif_loss", _ptr(z), _ptr(label), nq, 1.0, _ptr(dz), _ptr(loss), _stream())
        ctx.save_for_backward(dz)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (dz,) = ctx.saved_tensors
        return dz * g, None


def adam_(master, grad, m1, m2, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-15,
          grad_scale=1.0, copy: torch.Tensor | None = None, copy_dtype: int = L.NIF_F32, stream=None):
    L.call("nif_adam", _ptr(master), _ptr(grad), _ptr(m1), _ptr(m2), master.numel(), lr, beta1, beta2,
           eps, grad_scale, step, _ptr(copy), copy_dtype, _stream(stream))


E4M3_MAX = 448.0


def quantize_e4m3(weights_f32: torch.Tensor, cfg: NifConfig, n_nets: int, act_amax):
    """Per-tensor FP8-E4M3 quantisation of every network's layers: weight
    scale = amax(|W_l|) / 448, activation scale = act_amax[g][l] / 448 for the
    input of layer l (l = 0..n_hidden-1; the output layer's input stays FP32).
    Returns (e4m3 weights [n_nets*P], scales [n_nets][n_hidden+1][2] FP32)."""
    P = NifModel.weight_count(cfg)
    W, K, H = cfg.width, cfg.K, cfg.n_hidden
    w = weights_f32.detach().float().reshape(n_nets, P)
    q = torch.empty_like(w)
    scales = torch.ones((n_nets, H + 1, 2), dtype=torch.float32, device=w.device)
    for g in range(n_nets):
        off, fan_in = 0, K
        for l in range(H + 1):
            n = (W * fan_in) if l < H else fan_in
            blk = w[g, off:off + n]
            sw = float(blk.abs().max().clamp_min(1e-30)) / E4M3_MAX
            q[g, off:off + n] = blk / sw
            scales[g, l, 1] = sw
            if l < H:
                scales[g, l, 0] = max(float(act_amax[g][l]), 1e-30) / E4M3_MAX
            off += n
            fan_in = W
    return q.reshape(-1).to(torch.float8_e4m3fn).contiguous(), scales.contiguous()


# (schedule, CTAs per SM) pairs the autotuner times: the serial schedule at
# 4, 3 or 2 CTAs per SM (more CTAs trade gathers in flight per thread for more
# warps) and the pipelined schedule (its own occupancy).  A later candidate
# replaces the choice only when it is faster by more than TUNE_MARGIN, so that
# timing noise between near-equal candidates does not flip the choice.
SCHEDULE_CANDIDATES = ((L.NIF_SCHED_SERIAL, 4), (L.NIF_SCHED_PIPELINED, 0), (L.NIF_SCHED_SERIAL, 3),
                       (L.NIF_SCHED_SERIAL, 2), (L.NIF_SCHED_SERIAL, 2, 256))
TUNE_MARGIN = 0.02


def autotune(model: NifModel, run, key_extra=(), candidates=SCHEDULE_CANDIDATES, reps: int = 5,
             cache_path: str | None = None, also=()):
    """Pick the tensor-core forward's (schedule, CTAs per SM, tile M) by
    timing `run()` (the caller's own query, e.g. nif_infer on its rays): the
    median of `reps` runs per candidate, each after an L2 flush.  A candidate
    is (schedule, ctas) or (schedule, ctas, tile_m) (tile_m 128 when left
    out; 256 runs tiles of two 128-row blocks); one the library refuses for
    this model is skipped.  The choice is written into model.cfg (and the cfg
    of every model in `also`, other networks the same run() queries) and
    cached per (model shape, key_extra, GPU) in a JSON file.  Returns
    (schedule, ctas_per_sm, {candidate: ms})."""
    import hashlib
    import json
    import os
    c = model.cfg
    cfgs = [c] + [m.cfg for m in also]

    def apply(sched, ctas, tile_m=128):
        for cf in cfgs:
            cf.schedule, cf.ctas_per_sm, cf.tile_m = int(sched), int(ctas), int(tile_m)

    cands = [tuple(x) for x in candidates]
    key = hashlib.sha1(json.dumps([list(c.res), c.n_features, c.log2_table, c.grid_dtype, c.n_hidden,
                                   c.width, c.mlp_dtype, c.net_mode, c.encoding, model.n_obj,
                                   list(key_extra), cands, torch.cuda.get_device_name()]).encode()
                       ).hexdigest()[:16]
    cache_path = cache_path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        apply(*cache[key]["choice"])
        return c.schedule, c.ctas_per_sm, cache[key]["ms"]
    label = {L.NIF_SCHED_SERIAL: "serial", L.NIF_SCHED_PIPELINED: "pipelined", L.NIF_SCHED_AUTO: "auto"}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=model.obj_aabb.device)  # > L2
    timings = {}
    for cand in cands:
        apply(*cand)
        try:
            run()
        except L.NifError:
            continue  # not offered for this model
        torch.cuda.synchronize()
        got = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            got.append(e0.elapsed_time(e1))
        timings[cand] = sorted(got)[len(got) // 2]
    del flush
    tried = [k for k in cands if k in timings]
    choice = tried[0]
    for k in tried[1:]:
        if timings[k] < timings[choice] * (1.0 - TUNE_MARGIN):
            choice = k
    apply(*choice)
    ms = {f"{label[k[0]]}/{k[1]}" + (f"/m{k[2]}" if len(k) > 2 else ""): v for k, v in timings.items()}
    cache[key] = {"choice": list(choice), "ms": ms}
    try:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return choice[0], choice[1], ms
