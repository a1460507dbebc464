"""The room workload end to end on one GPU: scene, exact BVHs, primary hits,
shadow rays, per-pair BVH labels, online training (Sec. 4.2) and the two
shadow-ray queries that are compared (Sec. 6.6): the learned one (top-level
front end + fused NIF networks) and the exact one (full BVH traversal).

Everything runs in libnif; torch only holds device buffers and streams."""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from . import nif, synth, workloads

GRID_SEED = workloads.GRID_SEED
ROUND1_NAME = {L.NIF_ROUND1_NEAREST: "nearest", L.NIF_ROUND1_OUTER: "outer"}
GRID_SCALE = workloads.GRID_SCALE  # latent init U(-1e-4, 1e-4), Sec. 5 "Initialization"
_ROOM = workloads.ROOM_FRAME
_FULL = workloads.FULL_FRAME


class BatchDraw:
    """Training batches drawn without replacement: a seeded permutation of
    the pool per epoch, cut into consecutive batches of pool indices."""

    def __init__(self, n: int, seed: int):
        self.n = n
        self.rng = np.random.default_rng(seed)
        self.perm = self.rng.permutation(n)
        self.pos = 0

    def __call__(self, b: int) -> np.ndarray:
        if self.pos + b > self.n:
            self.perm = self.rng.permutation(self.n)
            self.pos = 0
        sel = self.perm[self.pos:self.pos + b]
        self.pos += b
        return sel


@dataclass
class RoomConfig:
    n_obj: int = _ROOM.n_obj
    n: int = _ROOM.n            # icosphere frequency: 20 n^2 triangles
    width: int = _ROOM.width
    height: int = _ROOM.height
    seed: int = _ROOM.seed
    res: tuple = _ROOM.res
    n_features: int = _ROOM.n_features
    log2_table: int = _ROOM.log2_table
    grid_dtype: int = L.NIF_F16
    mlp_dtype: int = L.NIF_F16
    n_hidden: int = _ROOM.n_hidden
    width_mlp: int = _ROOM.width_mlp
    train_spp: int = 4          # jittered samples per pixel collected for training
    train_steps: int = 64
    batch: int = 262144
    lr: float = 1e-2
    tmin: float = _ROOM.tmin
    ctas_per_sm: int = 0
    schedule: int = 0  # NIF_SCHED_* of the tensor-core forward (0: library choice)
    layout: str = "random"      # "random" | "single" | "lattice" | "mixed" (see workloads.room_scene)
    nif_min_tris: int = 0       # objects with at most this many triangles stay in the exact BVH
    # exact cast of the non-NIF geometry: "first" (its bits let the NIF front
    # end skip rays), "after" (skipping rays NIF occluded) or "overlap" (on a
    # second stream beside the NIF query)
    exact_cast: str = "first"
    tlas_builder: str = "lbvh"  # top level over the object boxes: "lbvh" or "ploc"
    n_lights: int = 1           # point lights (one shadow ray per light per pixel)
    area_light: bool = False    # 4 x 4 ceiling quad light instead of point lights
    samples: int = 1            # shadow rays per pixel (area-light samples)
    max_pairs_per_ray: int = 6  # capacity of the front end's pair lists
    pairs_per_spp: int = 0      # training pairs kept per jittered sample (0 = all)
    # training precision: FP32 on the CUDA cores over the FP32 masters, or
    # the model's 16-bit copies on the tensor cores with a dynamic loss scale
    half_precision_train: bool = False
    loss_scale: float = 65536.0
    scale_window: int = 2000


def small_object_precision_config() -> RoomConfig:
    """The small-configuration object and network (8 dense FP32 levels, R = 4..64,
    3x64) in the room, 4 point lights -> 8,294,400 shadow rays."""
    return RoomConfig(layout="single", n_obj=1, res=tuple(workloads.TINY_RES), log2_table=19,
                      grid_dtype=L.NIF_F32, mlp_dtype=L.NIF_F32, n_lights=4, samples=4,
                      train_spp=1)


def mixed_scene_config() -> RoomConfig:
    """A mixed scene (Sec. 6.6: NIF only for objects above 100K triangles,
    the exact BVH for the rest): 32 displaced icospheres with 10K-500K
    triangles (log-uniform) in the room, one point light -> 2,073,600 shadow
    rays; the room's hashed FP16 grids and 3x64 FP16 networks for the NIF
    objects.  The exact cast of the small objects and the room runs on a
    second stream beside the NIF query (0.71 ms per step against 0.76 ms
    cast first on one GB300)."""
    return RoomConfig(layout="mixed", n_obj=32, nif_min_tris=100_000, exact_cast="overlap")


def full_scale_config() -> RoomConfig:
    """480 displaced icospheres of 62,720 triangles (30.1M) on a jittered
    lattice in the room, a 4 x 4 area light, 4 samples per pixel -> 8,294,400
    shadow rays; dense 8-level FP16 grids per object, FP16 networks, trained on
    16 jittered samples x 4 light samples = 64 shadow samples per pixel.  The
    exact cast of the 12 room triangles follows the NIF query and skips the
    rays it occluded (3.045 ms per step against 3.079 ms with the cast first
    on one GB300)."""
    return RoomConfig(layout=_FULL.layout, n_obj=_FULL.n_obj, n=_FULL.n, res=_FULL.res,
                      log2_table=_FULL.log2_table, grid_dtype=L.NIF_F16, mlp_dtype=L.NIF_F16,
                      area_light=_FULL.area_light, samples=_FULL.samples, train_spp=16,
                      pairs_per_spp=1 << 20, max_pairs_per_ray=8, exact_cast="after")


class RoomPipeline:
    n_outputs = 1  # network output rows (the occupancy logit)

    def __init__(self, cfg: RoomConfig, device="cuda", log=print):
        self.cfg = cfg
        self.log = log
        t0 = time.time()
        ws = workloads.room_scene(cfg.n_obj, cfg.n, cfg.width, cfg.height, cfg.seed,
                                  layout=cfg.layout, n_lights=cfg.n_lights)
        self.ws = ws
        sc = ws.scene
        dev = torch.device(device)
        self.dev = dev
        self.verts = torch.from_numpy(sc.verts).to(dev)
        self.tris = torch.from_numpy(sc.tris).to(dev)
        tri_obj, obj_aabb = sc.tri_obj, sc.obj_aabb
        if cfg.nif_min_tris > 0:
            # objects at or below the threshold join the room in the exact
            # cast; the NIF objects are renumbered 0 .. n_obj - 1
            keep = sc.obj_tri_range[:, 1] > cfg.nif_min_tris
            new_id = np.full(len(keep), -1, dtype=np.int32)
            new_id[keep] = np.arange(int(keep.sum()), dtype=np.int32)
            tri_obj = np.full_like(sc.tri_obj, -1)
            on = sc.tri_obj >= 0
            tri_obj[on] = new_id[sc.tri_obj[on]]
            obj_aabb = np.ascontiguousarray(sc.obj_aabb[keep])
        self.n_obj = int(obj_aabb.shape[0])
        self.tags = torch.from_numpy(tri_obj).to(dev)
        self.obj_aabb = torch.from_numpy(obj_aabb).to(dev)
        self.n_tris = int(sc.tris.shape[0])
        self.n_tris_nif = int((tri_obj >= 0).sum())
        # exact structures: all triangles (comparison + labels), non-NIF
        # geometry alone (the room), object boxes (top level of the NIF query)
        self.bvh = nif.BVH(self.verts, self.tris, self.tags)
        room = tri_obj < 0
        self.room_bvh = nif.BVH(self.verts, torch.from_numpy(sc.tris[room]).to(dev))
        self.tlas = nif.BVH.from_boxes(self.obj_aabb, builder=cfg.tlas_builder)
        self.light = torch.from_numpy(ws.light.astype(np.float32).reshape(-1)).to(dev)
        # evaluation frame: pixel-centre camera rays -> primary hits -> shadow rays
        self.rays = self._eval_rays(torch.from_numpy(ws.camera).to(dev))
        self.n_rays = int(self.rays.shape[0])
        n_grid = self._build_model()
        torch.cuda.synchronize()
        self.log(f"room scene ready: {self.n_tris} triangles ({self.n_tris_nif} in {self.n_obj} NIF objects), "
                 f"{self.n_rays} rays, "
                 f"{n_grid / 1e9:.3f}G grid latents ({time.time() - t0:.1f}s)")

    def _build_model(self) -> int:
        """The multi-resolution model (shared outer/inner networks over
        per-object grids); returns the number of grid latents."""
        c, dev = self.cfg, self.dev
        ncfg = nif.NifConfig(res=list(c.res), n_features=c.n_features, log2_table=c.log2_table,
                             grid_dtype=c.grid_dtype, n_hidden=c.n_hidden, width=c.width_mlp,
                             mlp_dtype=c.mlp_dtype, net_mode=L.NIF_NETS_CLASS,
                             ctas_per_sm=c.ctas_per_sm, schedule=c.schedule, n_outputs=self.n_outputs)
        self.V = nif.NifModel.grid_vertices(ncfg)
        self.P = nif.NifModel.weight_count(ncfg)
        n_grid = self.n_obj * 2 * self.V * c.n_features
        self.g_master = torch.empty(n_grid, dtype=torch.float32, device=dev)
        L.call("nif_fill_uniform", ctypes.c_void_p(self.g_master.data_ptr()), n_grid, GRID_SEED,
               GRID_SCALE, nif._stream())
        wr = np.random.default_rng(c.seed + 101)
        flat = np.concatenate([synth.flatten_mlp(synth.mlp_init(wr, ncfg.K, c.width_mlp, c.n_hidden,
                                                                n_out=self.n_outputs))
                               for _ in range(2)])
        self.w_master = torch.from_numpy(flat).to(dev)
        gdt = {L.NIF_F16: torch.float16, L.NIF_F32: torch.float32}[c.grid_dtype]
        mdt = {L.NIF_F16: torch.float16, L.NIF_BF16: torch.bfloat16, L.NIF_F32: torch.float32}[c.mlp_dtype]
        self.model = nif.NifModel(ncfg, self.obj_aabb, self.g_master.to(gdt), self.w_master.to(mdt))
        self.init_weights = self.model.weights.clone()
        self.init_grids = self.model.grids.clone()
        return n_grid

    # ------------------------------------------------------------ inputs
    def _eval_rays(self, camera: torch.Tensor) -> torch.Tensor:
        """The rays of the evaluation frame: shadow rays from the primary hits."""
        return self._shadow_rays(camera, light_seed=workloads.EVAL_LIGHT_SEED)

    def _shadow_rays(self, camera: torch.Tensor, light_seed: int) -> torch.Tensor:
        """Shadow rays from the primary hits of `camera`: one per point light,
        or cfg.samples uniform samples of the area light per pixel."""
        c = self.cfg
        t, _ = self.bvh.cast_closest(camera)
        n = int(camera.shape[0])
        if c.area_light:
            pts = workloads.area_light_samples(np.random.default_rng(light_seed), n, c.samples)
            return nif.shadow_rays(camera, t, torch.from_numpy(pts).to(self.dev), spp=c.samples,
                                   per_ray=True, tmin=c.tmin)
        if c.n_lights > 1:
            pts = self.light.reshape(1, c.n_lights, 3).expand(n, c.n_lights, 3).contiguous()
            return nif.shadow_rays(camera, t, pts, spp=c.n_lights, per_ray=True, tmin=c.tmin)
        return nif.shadow_rays(camera, t, self.light, tmin=c.tmin)

    def training_pairs(self, spp: int | None = None, seed: int = 1234):
        """Shadow rays from jittered primary samples (the first spp of the
        frame, Sec. 4.2), their (ray, object) pairs and per-pair BVH labels
        (1 = visible, Sec. 6.4)."""
        c = self.cfg
        spp = spp or c.train_spp
        rays, rids, qobjs, labels = [], [], [], []
        base = 0
        for s in range(spp):
            jit = np.random.default_rng(seed + s).uniform(size=(c.width * c.height, 2))
            cam = synth.camera_rays(c.width, c.height, (0.0, 0.0, 19.0), (0.0, 0.0, 0.0), 60.0, jitter=jit)
            r = self._shadow_rays(torch.from_numpy(cam).to(self.dev), light_seed=5000 + s)
            rid, qo, goff, count = self.model.frontend(r, tlas=self.tlas,
                                                       max_q=c.max_pairs_per_ray * r.shape[0] + 1024)
            torch.cuda.synchronize()
            self.model.check()
            nq = int(count.item())
            rid, qo = rid[:nq], qo[:nq]
            if c.pairs_per_spp and nq > c.pairs_per_spp:
                keep = torch.randperm(nq, device=self.dev,
                                      generator=torch.Generator(device=self.dev).manual_seed(seed + s))
                keep = keep[:c.pairs_per_spp].sort().values
                rid, qo = rid[keep].contiguous(), qo[keep].contiguous()
            hit = self.bvh.cast_pairs(r, rid, qo)
            rays.append(r)
            rids.append(rid.to(torch.int64) + base)
            qobjs.append(qo)
            labels.append(1 - hit)
            base += r.shape[0]
        rays = torch.cat(rays)
        rid = torch.cat(rids)
        qo = torch.cat(qobjs)
        lab = torch.cat(labels)
        # group by network (outer = 0, inner = 1), stable
        inner = ((qo.to(torch.int64) >> 31) & 1)
        order = torch.argsort(inner, stable=True)
        return rays, rid[order].to(torch.int32), qo[order].contiguous(), lab[order].contiguous(), \
            int((inner == 0).sum().item())

    def calibrate_e4m3(self, pairs, n_cal: int = 65536, seed: int = 7):
        """Per-tensor FP8-E4M3 scales from the FP32 trained network: the amax
        of every layer's input over n_cal training pairs (per network), and
        of every weight matrix.  Returns (e4m3 weights, scales)."""
        rays, rid, qo, lab, n_outer = pairs
        npool = int(rid.shape[0])
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(npool, min(n_cal, npool), replace=False))
        k = int(np.searchsorted(idx, n_outer))
        nq = len(idx)
        it = torch.from_numpy(idx).to(self.dev)
        ray_id, qobj = rid[it].contiguous(), qo[it].contiguous()
        goff = torch.tensor([0, k, nq], dtype=torch.int64, device=self.dev)
        c = self.cfg
        f32cfg = nif.NifConfig(**{**self.model.cfg.__dict__, "grid_dtype": L.NIF_F32, "mlp_dtype": L.NIF_F32})
        m32 = nif.NifModel(f32cfg, self.obj_aabb, self.trainer.g_master, self.trainer.w_master)
        d = m32.desc()
        z = torch.empty(nq, dtype=torch.float32, device=self.dev)
        saved = torch.empty(L.lib.nif_saved_size(ctypes.byref(d), nq) // 4, dtype=torch.float32,
                            device=self.dev)
        L.call("nif_fwd_train", ctypes.byref(d), nif._ptr(rays), nif._ptr(ray_id), nif._ptr(qobj),
               nif._ptr(goff), nq, nif._ptr(z), nif._ptr(saved), nif._stream())
        K, W = f32cfg.K, c.width_mlp
        sv = saved.reshape(K + c.n_hidden * W, nq)
        bounds = [(0, K)] + [(K + l * W, K + (l + 1) * W) for l in range(c.n_hidden - 1)]
        amax = []
        for g, (a, b) in enumerate(((0, k), (k, nq))):
            amax.append([float(sv[r0:r1, a:b].abs().max()) if b > a else 1.0 for r0, r1 in bounds])
        return nif.quantize_e4m3(self.trainer.w_master, f32cfg, 2, amax)

    def train(self, steps: int | None = None, seed: int = 99, pairs=None):
        c = self.cfg
        steps = steps if steps is not None else c.train_steps
        pairs = pairs if pairs is not None else self.training_pairs()
        rays, rid, qo, lab, n_outer = pairs[:5]
        aux = pairs[5] if len(pairs) > 5 else None  # regression targets (several outputs)
        self.pairs = pairs
        npool = int(rid.shape[0])
        hp = bool(c.half_precision_train)
        self.trainer = nif.Trainer(self.model, lr=c.lr, w_master=self.w_master, g_master=self.g_master,
                                   half_precision=hp, dynamic_scale=hp,
                                   loss_scale=c.loss_scale if hp else 1.0, scale_window=c.scale_window)
        draw = BatchDraw(npool, seed)
        losses = []
        step_ev = []
        t0 = time.time()
        B = min(c.batch, npool)
        for s in range(steps):
            idx = draw(B)
            # outer pairs first, then inner ones (the pool is ordered that way)
            inner = idx >= n_outer
            k = int(B - np.count_nonzero(inner))
            idx = np.concatenate([idx[~inner], idx[inner]])
            goff = torch.tensor([0, k, B], dtype=torch.int64, device=self.dev)
            it = torch.from_numpy(idx).to(self.dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            loss = self.trainer.step(rays, rid[it].contiguous(), qo[it].contiguous(), goff,
                                     lab[it].contiguous(), B,
                                     aux=aux[it].contiguous() if aux is not None else None)
            e1.record()
            step_ev.append((e0, e1))
            losses.append(loss.clone())
        torch.cuda.synchronize()
        dt = time.time() - t0
        # device time of nif_train_step alone (forward, loss, backward, grid
        # scatter, Adam), without the host-side batch draw
        self.train_step_ms = [a.elapsed_time(b) for a, b in step_ev]
        self.model.check(self.trainer._ws)
        self.losses = [float(x.item()) for x in losses]
        self.log(f"trained {steps} steps of {B} pairs from a pool of {npool} in {dt:.2f}s; "
                 f"loss {self.losses[0]:.4f} -> {self.losses[-1]:.4f}")
        return dt

    def release_training_state(self):
        """Drop FP32 masters, Adam moments and the initial copies once
        training and the ablations are done (inference keeps the FP16 copies)."""
        self.trainer = None
        self.pairs = None
        self.g_master = None
        self.w_master = None
        self.init_grids = None
        self.init_weights = None

    # ------------------------------------------------------------ queries
    def front_model(self) -> nif.NifModel:
        """The model whose descriptor drives the front end (class bucketing)."""
        return self.model

    def forward_models(self):
        """(model, first group) pairs the forward runs on each round's pairs."""
        return [(self.model, 0)]

    def _query_buffers(self):
        if getattr(self, "_qb", None) is None:
            n = self.n_rays
            mq = self.cfg.max_pairs_per_ray * n + 1024
            fe = self.front_model()
            self._qb = {
                "max_q": mq,
                "ray_id": torch.empty(mq, dtype=torch.int32, device=self.dev),
                "qobj": torch.empty(mq, dtype=torch.int32, device=self.dev),
                "goff1": torch.empty(fe.n_nets + 1, dtype=torch.int64, device=self.dev),
                "goff2": torch.empty(fe.n_nets + 1, dtype=torch.int64, device=self.dev),
                "count": torch.zeros(2, dtype=torch.int64, device=self.dev),
                "ws": fe.workspace(mq, n),
            }
        return self._qb

    def _exact_begin(self, bits: torch.Tensor, rays: torch.Tensor, stream=None):
        """The part of the exact cast of the non-NIF geometry that precedes
        the NIF query (Sec. 4.1 combines both answers by OR).
        "first": overwrite the mask; the front end then skips occluded rays.
        "after": zero the mask; the cast follows the NIF query (_exact_end).
        "overlap": zero the mask and cast on a second stream, OR-ing into the
        mask while the NIF query runs on `stream`; returns the join event."""
        stream = stream if stream is not None else torch.cuda.current_stream()
        n = int(rays.shape[0])
        mode = self.cfg.exact_cast
        if mode == "first":
            self.room_bvh.cast_shadow(rays, out=bits, stream=stream)
            return None
        nif.clear_bits(bits, n, stream=stream)
        if mode == "after":
            return None
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=self.dev)
            self._fork, self._join = torch.cuda.Event(), torch.cuda.Event()
        self._fork.record(stream)
        self._side.wait_event(self._fork)
        self.room_bvh.cast_shadow(rays, out=bits, stream=self._side, or_into=True)
        self._join.record(self._side)
        return self._join

    def _exact_end(self, join, bits: torch.Tensor, rays: torch.Tensor, stream=None):
        stream = stream if stream is not None else torch.cuda.current_stream()
        if self.cfg.exact_cast == "after":
            self.room_bvh.cast_shadow(rays, out=bits, stream=stream, or_into=True)
        elif join is not None:
            stream.wait_event(join)

    def query_step(self, bits: torch.Tensor, rays: torch.Tensor | None = None, ev=None):
        """The calls of one two-round visibility query, with optional CUDA
        events ev[0..3] (and ev[4]) recorded between them: the non-NIF cast
        (or its start, see _exact_begin), then nif_frontend_nearest, the
        forward of round 1, nif_frontend_rest, the forward of round 2 and the
        end of the non-NIF cast (what nif_infer does for one model)."""
        rays = self.rays if rays is None else rays
        b = self._query_buffers()
        vp, sp, n = ctypes.c_void_p, nif._stream(), int(rays.shape[0])
        stream = torch.cuda.current_stream()
        join = self._exact_begin(bits, rays, stream)
        d = self.front_model().desc()
        ws = b["ws"]
        common = (ctypes.byref(d), vp(self.tlas.buf.data_ptr()), vp(rays.data_ptr()), n, vp(bits.data_ptr()),
                  vp(b["ray_id"].data_ptr()), vp(b["qobj"].data_ptr()), b["max_q"])

        def forward(goff):
            for m, g0 in self.forward_models():
                md = m.desc()
                L.call("nif_infer_queries", ctypes.byref(md), vp(rays.data_ptr()), n, vp(b["ray_id"].data_ptr()),
                       vp(b["qobj"].data_ptr()), vp(goff.data_ptr() + 8 * g0), b["max_q"], vp(bits.data_ptr()),
                       None, vp(ws.data_ptr()), ws.numel(), sp)

        if ev is not None:
            ev[0].record(stream)
        L.call("nif_frontend_nearest", *common, vp(b["goff1"].data_ptr()), vp(b["count"].data_ptr()),
               vp(ws.data_ptr()), ws.numel(), sp)
        if ev is not None:
            ev[1].record(stream)
        forward(b["goff1"])
        if ev is not None:
            ev[2].record(stream)
        L.call("nif_frontend_rest", *common, vp(b["count"].data_ptr()), vp(b["goff2"].data_ptr()),
               vp(b["count"].data_ptr() + 8), vp(ws.data_ptr()), ws.numel(), sp)
        if ev is not None:
            ev[3].record(stream)
        forward(b["goff2"])
        if ev is not None and len(ev) > 4:
            ev[4].record(stream)
        self._exact_end(join, bits, rays, stream)
        return bits

    def tune_round1(self):
        """Pick the round-1 rule (NIF_ROUND1_NEAREST or _OUTER) that queries
        fewer pairs on this frame; the mask is the same either way.  Returns
        {rule name: pairs queried}."""
        bits = nif.empty_bits(self.n_rays)
        cfg = self.front_model().cfg
        pairs = {}
        for rule in (L.NIF_ROUND1_NEAREST, L.NIF_ROUND1_OUTER):
            cfg.round1 = rule
            self.query_step(bits)
            torch.cuda.synchronize()
            pairs[rule] = self.last_query_counts()[1]
        cfg.round1 = min(pairs, key=lambda r: (pairs[r], r))
        return {ROUND1_NAME[r]: v for r, v in pairs.items()}

    def query_cost(self):
        """Algorithmic grid-tap bytes and MLP flops of one queried pair."""
        c = self.cfg
        esz = 2 if c.grid_dtype == L.NIF_F16 else 4
        L_ = len(c.res)
        K = 3 * L_ * c.n_features
        W = c.width_mlp
        return 3 * L_ * 8 * c.n_features * esz, 2 * (K * W + (c.n_hidden - 1) * W * W + W)

    def param_count(self) -> int:
        return int(self.g_master.numel() + self.w_master.numel())

    def last_query_counts(self):
        """Pairs the last query_step queried: (round 1, both rounds)."""
        c = self._query_buffers()["count"].tolist()
        return int(c[0]), int(c[1])

    def check(self):
        self.front_model().check(self._query_buffers()["ws"])
        for b in (self.bvh, self.room_bvh, self.tlas):
            b.check()

    def nif_query(self, bits: torch.Tensor, rays: torch.Tensor | None = None, stream=None):
        """NIF visibility: exact cast of the non-NIF geometry (the room), then
        the top-level front end and the fused networks OR-ed into the mask."""
        rays = self.rays if rays is None else rays
        join = self._exact_begin(bits, rays, stream)
        self.model.infer(rays, bits, tlas=self.tlas, stream=stream,
                         max_q=self.cfg.max_pairs_per_ray * int(rays.shape[0]) + 1024)
        self._exact_end(join, bits, rays, stream)
        return bits

    def bvh_query(self, bits: torch.Tensor, rays: torch.Tensor | None = None, stream=None):
        rays = self.rays if rays is None else rays
        return self.bvh.cast_shadow(rays, out=bits, stream=stream)

    def nif_query_host(self, host_rays: torch.Tensor, host_bits: torch.Tensor, dev_rays: torch.Tensor,
                       bits: torch.Tensor, n_chunks: int = 4) -> torch.Tensor:
        """NIF visibility of rays in pinned host memory into a pinned host
        mask.  The rays go up and the mask comes back in n_chunks pieces on a
        copy stream, so each piece's copies overlap the queries of the others
        (pieces are multiples of 32 rays: whole mask words).  dev_rays and
        bits are device buffers of the full size."""
        n = int(host_rays.shape[0])
        step = (-(-n // max(1, n_chunks)) + 31) // 32 * 32
        main = torch.cuda.current_stream()
        if getattr(self, "_copy", None) is None:
            self._copy = torch.cuda.Stream(device=self.dev)
        cp = self._copy
        cp.wait_stream(main)  # earlier work on these buffers comes first
        bounds = [(a, min(n, a + step)) for a in range(0, n, step)]
        ready = []
        for a, b in bounds:
            with torch.cuda.stream(cp):
                dev_rays[a:b].copy_(host_rays[a:b], non_blocking=True)
            e = torch.cuda.Event()
            e.record(cp)
            ready.append(e)
        for (a, b), e in zip(bounds, ready):
            main.wait_event(e)
            w0, w1 = a // 32, (b + 31) // 32
            self.nif_query(bits[w0:w1], dev_rays[a:b])
            done = torch.cuda.Event()
            done.record(main)
            cp.wait_event(done)
            with torch.cuda.stream(cp):
                host_bits[w0:w1].copy_(bits[w0:w1], non_blocking=True)
        main.wait_stream(cp)
        return host_bits

    def nif_query_host_frames(self, frames, dev_rays, bits, on_frame=None):
        """NIF visibility of a sequence of frames in pinned host memory:
        frames is a list of (host_rays [n, 8] float32, host_bits int32 mask)
        pairs, all of this pipeline's ray count.  Two frames are in flight:
        frame k + 1's rays go up on a copy stream while frame k is queried,
        and frame k's mask comes back while frame k + 1 is queried.  dev_rays
        and bits are two device buffers each (alternate frames use them).
        on_frame(k), if given, runs on the host just before frame k's query
        is enqueued on the current stream."""
        K = len(frames)
        main = torch.cuda.current_stream()
        if getattr(self, "_copy", None) is None:
            self._copy = torch.cuda.Stream(device=self.dev)
        cp = self._copy
        cp.wait_stream(main)  # earlier work on these buffers comes first
        up = [None] * K
        queried = [None] * K

        def upload(k):
            j = k % 2
            with torch.cuda.stream(cp):
                if k >= 2:
                    cp.wait_event(queried[k - 2])  # frame k - 2 is done with this buffer
                dev_rays[j].copy_(frames[k][0], non_blocking=True)
            up[k] = torch.cuda.Event()
            up[k].record(cp)

        if K:
            upload(0)
        for k in range(K):
            j = k % 2
            if k + 1 < K:
                upload(k + 1)
            main.wait_event(up[k])  # also orders after frame k - 2's mask copy on cp
            if on_frame is not None:
                on_frame(k)
            self.nif_query(bits[j], dev_rays[j])
            queried[k] = torch.cuda.Event()
            queried[k].record(main)
            with torch.cuda.stream(cp):
                cp.wait_event(queried[k])
                frames[k][1].copy_(bits[j], non_blocking=True)
        main.wait_stream(cp)
        return [f[1] for f in frames]

    def disagreement(self):
        """Fraction of shadow rays where NIF and the BVH disagree, over all rays
        and over rays with at least one NIF query."""
        a = nif.empty_bits(self.n_rays)
        b = nif.empty_bits(self.n_rays)
        self.nif_query(a)
        self.bvh_query(b)
        rid, qo, goff, count = self.model.frontend(self.rays, tlas=self.tlas,
                                                   max_q=self.cfg.max_pairs_per_ray * self.n_rays + 1024)
        torch.cuda.synchronize()
        self.model.check()
        nq = int(count.item())
        has = torch.zeros(self.n_rays, dtype=torch.bool, device=self.dev)
        has[rid[:nq].long()] = True
        va = nif.bits_to_bool(a, self.n_rays)
        vb = nif.bits_to_bool(b, self.n_rays)
        diff = va != vb
        return {
            "all": float(diff.float().mean().item()),
            "queried": float(diff[has].float().mean().item()) if bool(has.any()) else 0.0,
            "occluded_bvh": float(vb.float().mean().item()),
            "queries": nq,
            "rays_with_query": int(has.sum().item()),
        }

    def ablations(self):
        """What the learned part gains: the same rays answered by the AABB alone
        (occluded iff the ray meets any object box) and by the untrained net."""
        b = nif.empty_bits(self.n_rays)
        self.bvh_query(b)
        vb = nif.bits_to_bool(b, self.n_rays)
        rid, qo, goff, count = self.model.frontend(self.rays, tlas=self.tlas,
                                                   max_q=self.cfg.max_pairs_per_ray * self.n_rays + 1024)
        torch.cuda.synchronize()
        self.model.check()
        nq = int(count.item())
        aabb_only = torch.zeros(self.n_rays, dtype=torch.bool, device=self.dev)
        aabb_only[rid[:nq].long()] = True
        w, g = self.model.weights, self.model.grids
        self.model.weights, self.model.grids = self.init_weights, self.init_grids
        a = nif.empty_bits(self.n_rays)
        self.nif_query(a)
        untrained = nif.bits_to_bool(a, self.n_rays)
        self.model.weights, self.model.grids = w, g
        return {"aabb_only": float((aabb_only != vb).float().mean().item()),
                "untrained": float((untrained != vb).float().mean().item())}


# --------------------------------------------------------------------------
# The paper's own encoding on the same scene (Sec. 3.1, Sec. 3.2, Table 1,
# Sec. 5 'Architecture'): an outer and an inner network with their own
# spherical grids per object.

@dataclass
class PaperEncodingConfig(RoomConfig):
    outer_res: int = 256        # Table 1: outer 2D grids R = 256, N = 3
    outer_features: int = 3
    outer_hidden: int = 2       # Sec. 5: outer 2 x 64, inner 3 x 48, leaky ReLU
    outer_width: int = 64
    inner_res: int = 128        # Table 1: inner 2D grids R = 128, N = 5; 1D R = 128, N = 3
    inner_features: int = 5
    inner_res_1d: int = 128
    inner_features_1d: int = 3
    inner_hidden: int = 3
    inner_width: int = 48
    lr: float = 5e-3            # Sec. 5 'Training'


def _pad_width(flat: torch.Tensor, K: int, W: int, H: int, Wp: int) -> torch.Tensor:
    """The same bias-free network with Wp >= W hidden units: the extra units
    get zero weights in and out, so they stay at zero (ReLU and leaky ReLU map
    0 to 0) and the output is unchanged."""
    out, off, fan, fanp = [], 0, K, K
    for _ in range(H):
        m = flat[off:off + W * fan].view(W, fan)
        mp = torch.zeros(Wp, fanp, dtype=flat.dtype, device=flat.device)
        mp[:W, :fan] = m
        out.append(mp.reshape(-1))
        off += W * fan
        fan, fanp = W, Wp
    wo = torch.zeros(Wp, dtype=flat.dtype, device=flat.device)
    wo[:W] = flat[off:off + W]
    out.append(wo)
    return torch.cat(out).contiguous()


class PaperEncodingPipeline(RoomPipeline):
    """The room workload with the paper's encoding and its two networks.
    Outer pairs go to the outer model, inner pairs to the inner one; one
    class-mode front end bins them.  The inner network (48 wide) is trained in
    FP32 and queried on the tensor cores as the same network padded to 64."""

    def _build_model(self) -> int:
        c, dev = self.cfg, self.dev
        total = 0
        self.cls = {}
        for k, (name, enc, R, N, R1, N1, H, W) in enumerate((
                ("outer", L.NIF_ENC_SPHERICAL_OUTER, c.outer_res, c.outer_features, 0, 0, c.outer_hidden,
                 c.outer_width),
                ("inner", L.NIF_ENC_SPHERICAL_INNER, c.inner_res, c.inner_features, c.inner_res_1d,
                 c.inner_features_1d, c.inner_hidden, c.inner_width))):
            ncfg = nif.NifConfig(res=[R], n_features=N, grid_dtype=L.NIF_F16, n_hidden=H, width=W,
                                 act=L.NIF_ACT_LEAKY, mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_SINGLE,
                                 encoding=enc, res_1d=R1, n_features_1d=N1,
                                 ctas_per_sm=c.ctas_per_sm, schedule=c.schedule)
            n_grid = self.n_obj * nif.NifModel.grid_vertices(ncfg)
            g = torch.empty(n_grid, dtype=torch.float32, device=dev)
            L.call("nif_fill_uniform", ctypes.c_void_p(g.data_ptr()), n_grid, GRID_SEED + 17 * (k + 1),
                   GRID_SCALE, nif._stream())
            wr = np.random.default_rng(c.seed + 101 + k)
            w = torch.from_numpy(synth.flatten_mlp(synth.mlp_init(wr, ncfg.K, W, H))).to(dev)
            model = nif.NifModel(ncfg, self.obj_aabb, g.half(), w.half())
            self.cls[name] = {"model": model, "g_master": g, "w_master": w,
                              "init_grids": model.grids.clone(), "init_weights": model.weights.clone()}
            total += n_grid
        self._make_inference_models(init=True)
        oc = self.cls["outer"]["model"]
        fe_cfg = nif.NifConfig(**{**oc.cfg.__dict__, "net_mode": L.NIF_NETS_CLASS})
        self.model = nif.NifModel(fe_cfg, self.obj_aabb, oc.grids, torch.cat([oc.weights, oc.weights]))
        self.g_master = self.w_master = None
        return total

    def _make_inference_models(self, init: bool = False):
        """Tensor-core copies: the outer model as is, the inner one padded to a
        width the tensor cores take."""
        inner = self.cls["inner"]["model"]
        c = inner.cfg
        Wp = 64 if c.width <= 64 else 128
        src = self.cls["inner"]["init_weights"] if init else self.cls["inner"]["w_master"]
        wp = _pad_width(src.float(), c.K, c.width, c.n_hidden, Wp).half()
        icfg = nif.NifConfig(**{**c.__dict__, "width": Wp})
        self.inner_inf = nif.NifModel(icfg, self.obj_aabb, inner.grids, wp)
        if init:
            self.inner_inf_init_weights = wp.clone()

    def front_model(self) -> nif.NifModel:
        return self.model

    def forward_models(self):
        return [(self.cls["outer"]["model"], 0), (self.inner_inf, 1)]

    def param_count(self) -> int:
        return int(sum(cl["model"].grids.numel() + cl["model"].weights.numel() for cl in self.cls.values()))

    def query_cost(self):
        """Per queried pair, averaged over the class mix of the last query:
        grid-tap bytes (4 bilinear taps per 2D lookup, 2 linear taps of the
        distance grid, FP16) and MLP flops of the unpadded networks."""
        b = self._query_buffers()
        n_cls = [0, 0]
        for g in (b["goff1"].tolist(), b["goff2"].tolist()):
            n_cls[0] += g[1] - g[0]
            n_cls[1] += g[2] - g[1]
        cost = []
        for name in ("outer", "inner"):
            c = self.cls[name]["model"].cfg
            taps = 2 * 4 * c.n_features + 2 * c.n_features_1d
            W, H, K = c.width, c.n_hidden, c.K
            cost.append((taps * 2, 2 * (K * W + (H - 1) * W * W + W)))
        tot = max(1, sum(n_cls))
        return (sum(n * c[0] for n, c in zip(n_cls, cost)) / tot,
                sum(n * c[1] for n, c in zip(n_cls, cost)) / tot)

    def nif_query(self, bits: torch.Tensor, rays: torch.Tensor | None = None, stream=None):
        return self.query_step(bits, rays)

    def train(self, steps: int | None = None, seed: int = 99, pairs=None):
        c = self.cfg
        steps = steps if steps is not None else c.train_steps
        rays, rid, qo, lab, n_outer = pairs if pairs is not None else self.training_pairs()
        self.pairs = (rays, rid, qo, lab, n_outer)
        npool = int(rid.shape[0])
        parts = {"outer": (0, n_outer), "inner": (n_outer, npool)}
        trainers = {}
        for name in ("outer", "inner"):
            cl = self.cls[name]
            trainers[name] = nif.Trainer(cl["model"], lr=c.lr, w_master=cl["w_master"], g_master=cl["g_master"])
        self.trainers = trainers
        draws = {name: BatchDraw(b - a, seed + k) for k, (name, (a, b)) in enumerate(parts.items())}
        B = min(c.batch, npool)
        losses, step_ev = [], []
        t0 = time.time()
        for s in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step_loss = []
            for name, (a, b) in parts.items():
                nb = int(round(B * (b - a) / npool))
                if nb == 0:
                    continue
                idx = draws[name](nb) + a
                it = torch.from_numpy(idx).to(self.dev)
                goff = torch.tensor([0, nb], dtype=torch.int64, device=self.dev)
                loss = trainers[name].step(rays, rid[it].contiguous(), qo[it].contiguous(), goff,
                                           lab[it].contiguous(), nb)
                step_loss.append((loss.clone(), nb))
            e1.record()
            step_ev.append((e0, e1))
            losses.append(step_loss)
        torch.cuda.synchronize()
        dt = time.time() - t0
        self.train_step_ms = [a.elapsed_time(b) for a, b in step_ev]
        for name in ("outer", "inner"):
            self.cls[name]["model"].check(trainers[name]._ws)
            self.cls[name]["w_master"] = trainers[name].w_master
        self._make_inference_models()
        tot = [sum(float(l.item()) * nb for l, nb in st) / max(1, sum(nb for _, nb in st)) for st in losses]
        self.losses = tot
        self.log(f"trained outer + inner networks for {steps} steps of {B} pairs from a pool of {npool} "
                 f"({n_outer} outer) in {dt:.2f}s; loss {tot[0]:.4f} -> {tot[-1]:.4f}")
        return dt

    def ablations(self):
        b = nif.empty_bits(self.n_rays)
        self.bvh_query(b)
        vb = nif.bits_to_bool(b, self.n_rays)
        rid, qo, goff, count = self.model.frontend(self.rays, tlas=self.tlas,
                                                   max_q=self.cfg.max_pairs_per_ray * self.n_rays + 1024)
        torch.cuda.synchronize()
        self.model.check()
        nq = int(count.item())
        aabb_only = torch.zeros(self.n_rays, dtype=torch.bool, device=self.dev)
        aabb_only[rid[:nq].long()] = True
        om, inf = self.cls["outer"]["model"], self.inner_inf
        saved = (om.weights, om.grids, inf.weights, inf.grids)
        om.weights, om.grids = self.cls["outer"]["init_weights"], self.cls["outer"]["init_grids"]
        inf.weights, inf.grids = self.inner_inf_init_weights, self.cls["inner"]["init_grids"]
        a = nif.empty_bits(self.n_rays)
        self.nif_query(a)
        untrained = nif.bits_to_bool(a, self.n_rays)
        om.weights, om.grids, inf.weights, inf.grids = saved
        return {"aabb_only": float((aabb_only != vb).float().mean().item()),
                "untrained": float((untrained != vb).float().mean().item())}

    def release_training_state(self):
        self.trainers = None
        self.pairs = None
        for cl in self.cls.values():
            cl["g_master"] = cl["w_master"] = None
            cl["init_grids"] = cl["init_weights"] = None
        self.inner_inf_init_weights = None


# ---------------------------------------------------------------------------
# NIF for primary rays (Sec. 3.2, Sec. 6.1 with Fig. 5)
# ---------------------------------------------------------------------------
def primary_config() -> RoomConfig:
    """The room scene seen directly by the camera: 2,073,600 pixel-centre
    primary rays; per object the room's hashed FP16 grids, outer/inner 3x64
    FP16 networks with five outputs (occupancy, normal, depth in the box),
    trained on 4 jittered samples per pixel."""
    return RoomConfig(schedule=L.NIF_SCHED_SERIAL)


def face_normals(verts: torch.Tensor, tris: torch.Tensor, prim: torch.Tensor, d: torch.Tensor) -> torch.Tensor:
    """Unit geometric normals of triangles prim (>= 0) facing against the
    ray directions d: the regression targets and the truth of the normal."""
    t = tris[prim.long()].long()
    v0, v1, v2 = verts[t[:, 0]], verts[t[:, 1]], verts[t[:, 2]]
    n = torch.linalg.cross(v1 - v0, v2 - v0)
    n = n / n.norm(dim=1, keepdim=True).clamp_min(1e-30)
    flip = (n * d).sum(dim=1, keepdim=True) > 0
    return torch.where(flip, -n, n)


def slab_params(rays: torch.Tensor, boxes: torch.Tensor):
    """FP32 t_in, t_out of ray segments against their boxes (one box per
    ray), as the front end computes them: IEEE divisions, an axis with
    d == 0 inside its slab passes."""
    o, d = rays[:, 0:3], rays[:, 4:7]
    lo, hi = boxes[:, 0:3], boxes[:, 3:6]
    par = d == 0
    dd = torch.where(par, torch.ones_like(d), d)
    t0, t1 = (lo - o) / dd, (hi - o) / dd
    near = torch.where(par, torch.full_like(d, -float("inf")), torch.minimum(t0, t1))
    far = torch.where(par, torch.full_like(d, float("inf")), torch.maximum(t0, t1))
    # a parallel axis with the origin outside its slab misses the box
    blocked = (par & ~((lo <= o) & (o <= hi))).any(dim=1)
    inf = torch.full_like(rays[:, 3], float("inf"))
    entry = torch.where(blocked, inf, near.max(dim=1).values)
    exitv = torch.where(blocked, -inf, far.min(dim=1).values)
    tin = torch.maximum(rays[:, 3], entry)
    tout = torch.minimum(rays[:, 7], exitv)
    return tin, tout


class PrimaryPipeline(RoomPipeline):
    """Primary visibility with NIF: per pixel the nearest hit, its depth and
    its shading normal (Sec. 6.1, Fig. 5).  One step: the exact closest-hit
    cast of the non-NIF geometry (the room), the front end over the object
    boxes (every pair: a closest hit needs them all), the fused network with
    five outputs, and the closest-hit resolution.  The comparison is the
    exact closest-hit cast over every triangle."""
    n_outputs = 5
    # two rounds (nearest pair first, then only pairs entered before the
    # nearest hit) query 16% fewer pairs on the room frame, but the second
    # front end and resolution cost more than the fused time they save
    # (0.744 vs 0.722 ms per step), so one round is the default
    two_rounds = False

    def _eval_rays(self, camera: torch.Tensor) -> torch.Tensor:
        return camera.contiguous()

    def training_pairs(self, spp: int | None = None, seed: int = 1234):
        """Jittered camera rays (the first spp of the frame, Sec. 4.2), their
        (ray, object) pairs, the per-pair labels (1 = the ray misses the
        object) and targets [normal | delta] from the exact closest hit of
        the pair's own object."""
        c = self.cfg
        spp = spp or c.train_spp
        rays, rids, qobjs, labels, auxs = [], [], [], [], []
        base = 0
        for s in range(spp):
            jit = np.random.default_rng(seed + s).uniform(size=(c.width * c.height, 2))
            cam = synth.camera_rays(c.width, c.height, (0.0, 0.0, 19.0), (0.0, 0.0, 0.0), 60.0, jitter=jit)
            r = torch.from_numpy(cam).to(self.dev)
            rid, qo, goff, count = self.model.frontend(r, tlas=self.tlas,
                                                       max_q=c.max_pairs_per_ray * r.shape[0] + 1024)
            torch.cuda.synchronize()
            self.model.check()
            nq = int(count.item())
            rid, qo = rid[:nq].contiguous(), qo[:nq].contiguous()
            t_hit, prim = self.bvh.cast_pairs_closest(r, rid, qo)
            hit = prim >= 0
            rr = r[rid.long()]
            obj = (qo.to(torch.int64) & 0x7FFFFFFF)
            tin, tout = slab_params(rr, self.obj_aabb[obj])
            aux = torch.zeros((nq, 4), dtype=torch.float32, device=self.dev)
            h = hit.nonzero().squeeze(1)
            aux[h, 0:3] = face_normals(self.verts, self.tris, prim[h], rr[h, 4:7])
            span = (tout[h] - tin[h]).clamp_min(1e-30)
            aux[h, 3] = ((t_hit[h] - tin[h]) / span).clamp(0.0, 1.0)
            rays.append(r)
            rids.append(rid.to(torch.int64) + base)
            qobjs.append(qo)
            labels.append((~hit).to(torch.uint8))
            auxs.append(aux)
            base += r.shape[0]
        rays = torch.cat(rays)
        rid = torch.cat(rids)
        qo = torch.cat(qobjs)
        lab = torch.cat(labels)
        aux = torch.cat(auxs)
        inner = ((qo.to(torch.int64) >> 31) & 1)
        order = torch.argsort(inner, stable=True)
        return (rays, rid[order].to(torch.int32), qo[order].contiguous(), lab[order].contiguous(),
                int((inner == 0).sum().item()), aux[order].contiguous())

    # ------------------------------------------------------------ queries
    def _primary_buffers(self):
        if getattr(self, "_pb", None) is None:
            n = self.n_rays
            mq = self.cfg.max_pairs_per_ray * n + 1024
            dev = self.dev
            self._pb = {
                "max_q": mq,
                "ray_id": torch.empty(mq, dtype=torch.int32, device=dev),
                "qobj": torch.empty(mq, dtype=torch.int32, device=dev),
                "goff": torch.empty(self.model.n_nets + 1, dtype=torch.int64, device=dev),
                "goff2": torch.empty(self.model.n_nets + 1, dtype=torch.int64, device=dev),
                "count": torch.zeros(2, dtype=torch.int64, device=dev),
                "clear": nif.empty_bits(n, dev),
                "ws": self.model.workspace(mq, n),
                "out": torch.empty((mq, self.n_outputs), dtype=torch.float32, device=dev),
                "key": torch.empty(n, dtype=torch.int64, device=dev),
                "t": torch.empty(n, dtype=torch.float32, device=dev),
                "prim": torch.empty(n, dtype=torch.int32, device=dev),
                "normal": torch.empty((n, 3), dtype=torch.float32, device=dev),
                "winner": torch.empty(n, dtype=torch.int32, device=dev),
            }
        return self._pb

    def primary_step(self, rays: torch.Tensor | None = None, winner: bool = False, ev=None,
                     two_rounds: bool | None = None):
        """One primary-visibility query; returns (t, normal, winner or None).
        Two rounds: each ray's nearest pair first, resolved
        into the exact cast's t, then only the other pairs whose box the ray
        enters before its nearest hit so far (nif_frontend_rest_nearer); one
        round (the default): every pair at once.  ev (optional CUDA events) are recorded
        after the start, the exact cast, the (first) front end and the (first)
        fused forward; with two rounds also after the second front end and
        the second fused forward (6 events)."""
        rays = self.rays if rays is None else rays
        two_rounds = self.two_rounds if two_rounds is None else two_rounds
        b = self._primary_buffers()
        vp, sp, n = ctypes.c_void_p, nif._stream(), int(rays.shape[0])
        stream = torch.cuda.current_stream()
        d = self.model.desc()
        ws = b["ws"]
        pw = vp(b["winner"].data_ptr()) if winner else None
        if ev is not None:
            ev[0].record(stream)
        L.call("bvh_cast_closest", vp(self.room_bvh.buf.data_ptr()), vp(rays.data_ptr()), n,
               vp(b["t"].data_ptr()), vp(b["prim"].data_ptr()), sp)
        if ev is not None:
            ev[1].record(stream)
        common = (ctypes.byref(d), vp(self.tlas.buf.data_ptr()), vp(rays.data_ptr()), n)
        if two_rounds:
            L.call("nif_frontend_nearest", *common, vp(b["clear"].data_ptr()), vp(b["ray_id"].data_ptr()),
                   vp(b["qobj"].data_ptr()), b["max_q"], vp(b["goff"].data_ptr()), vp(b["count"].data_ptr()),
                   vp(ws.data_ptr()), ws.numel(), sp)
        else:
            L.call("nif_frontend", *common, vp(b["ray_id"].data_ptr()), vp(b["qobj"].data_ptr()), b["max_q"],
                   vp(b["goff"].data_ptr()), vp(b["count"].data_ptr()), vp(ws.data_ptr()), ws.numel(), sp)
        if ev is not None:
            ev[2].record(stream)

        def forward_and_resolve(goff, ev_mid=None):
            L.call("nif_infer_queries", ctypes.byref(d), vp(rays.data_ptr()), n, vp(b["ray_id"].data_ptr()),
                   vp(b["qobj"].data_ptr()), vp(goff.data_ptr()), b["max_q"], None, vp(b["out"].data_ptr()),
                   vp(ws.data_ptr()), ws.numel(), sp)
            if ev_mid is not None:
                ev_mid.record(stream)
            L.call("nif_primary_resolve", ctypes.byref(d), vp(rays.data_ptr()), n, vp(b["ray_id"].data_ptr()),
                   vp(b["qobj"].data_ptr()), vp(goff.data_ptr()), b["max_q"], vp(b["out"].data_ptr()),
                   vp(b["key"].data_ptr()), vp(b["t"].data_ptr()), vp(b["normal"].data_ptr()), pw, sp)

        if winner:
            b["winner"].fill_(-1)
        forward_and_resolve(b["goff"], ev[3] if ev is not None else None)
        if two_rounds:
            L.call("nif_frontend_rest_nearer", *common, vp(b["t"].data_ptr()), vp(b["ray_id"].data_ptr()),
                   vp(b["qobj"].data_ptr()), b["max_q"], vp(b["count"].data_ptr()), vp(b["goff2"].data_ptr()),
                   vp(b["count"].data_ptr() + 8), vp(ws.data_ptr()), ws.numel(), sp)
            if ev is not None:
                ev[4].record(stream)
            forward_and_resolve(b["goff2"], ev[5] if ev is not None else None)
        return b["t"], b["normal"], b["winner"] if winner else None

    def bvh_step(self, rays: torch.Tensor | None = None):
        """The exact closest-hit cast over every triangle (the comparison)."""
        rays = self.rays if rays is None else rays
        b = self._primary_buffers()
        vp = ctypes.c_void_p
        L.call("bvh_cast_closest", vp(self.bvh.buf.data_ptr()), vp(rays.data_ptr()), int(rays.shape[0]),
               vp(b["t"].data_ptr()), vp(b["prim"].data_ptr()), nif._stream())
        return b["t"], b["prim"]

    def query_cost(self):
        c = self.cfg
        esz = 2 if c.grid_dtype == L.NIF_F16 else 4
        K = 3 * len(c.res) * c.n_features
        W = c.width_mlp
        return 3 * len(c.res) * 8 * c.n_features * esz, 2 * (K * W + (c.n_hidden - 1) * W * W + self.n_outputs * W)

    def check(self):
        self.model.check(self._primary_buffers()["ws"])
        for b in (self.bvh, self.room_bvh, self.tlas):
            b.check()

    def disagreement(self):
        """Accuracy against the exact closest-hit cast over every triangle:
        pixels whose hit is a NIF object for one and not the other; over the
        pixels where both see a NIF object, the relative depth error and the
        angle between the normals; and the PSNR of the normal image
        ((n + 1) / 2) and of the depth image (t over the frame's depth range)
        over the pixels that see an object, as Fig. 5 compares them."""
        t_b, prim_b = (x.clone() for x in self.bvh_step())
        t_n, n_n, win = (x.clone() for x in self.primary_step(winner=True))
        torch.cuda.synchronize()
        self.check()
        tags = self.tags
        obj_b = torch.where(prim_b >= 0, tags[prim_b.clamp_min(0).long()], torch.full_like(prim_b, -1))
        nif_b = obj_b >= 0
        nif_n = win >= 0
        both = nif_b & nif_n
        d = self.rays[:, 4:7]
        n_true = torch.zeros_like(n_n)
        n_true[nif_b] = face_normals(self.verts, self.tris, prim_b[nif_b], d[nif_b])
        rel = ((t_n - t_b).abs() / t_b)[both]
        cosang = (n_n[both] * n_true[both]).sum(dim=1).clamp(-1.0, 1.0)
        ang = torch.rad2deg(torch.arccos(cosang))
        either = nif_b | nif_n
        img_n = torch.where(nif_n[:, None], (n_n + 1) * 0.5, torch.zeros_like(n_n))
        img_b = torch.where(nif_b[:, None], (n_true + 1) * 0.5, torch.zeros_like(n_n))
        mse_n = float(((img_n - img_b)[either] ** 2).mean())
        tmax = float(t_b[nif_b].max())
        dep_n = torch.where(nif_n, t_n / tmax, torch.zeros_like(t_n))
        dep_b = torch.where(nif_b, t_b / tmax, torch.zeros_like(t_b))
        mse_d = float(((dep_n - dep_b)[either] ** 2).mean())
        return {
            "hit_disagreement": float((nif_b != nif_n).float().mean()),
            "hit_disagreement_on_object_pixels": float((nif_b != nif_n)[either].float().mean()),
            "object_pixels": int(nif_b.sum()),
            "depth_rel_err_mean": float(rel.mean()), "depth_rel_err_median": float(rel.median()),
            "normal_err_deg_mean": float(ang.mean()), "normal_err_deg_median": float(ang.median()),
            "psnr_normal_db": 10.0 * float(np.log10(1.0 / max(mse_n, 1e-30))),
            "psnr_depth_db": 10.0 * float(np.log10(1.0 / max(mse_d, 1e-30))),
            "queries": int(self._primary_buffers()["count"][1 if self.two_rounds else 0].item()),
        }

    def ablations(self):
        """The untrained network's hit disagreement and normal error."""
        w, g = self.model.weights, self.model.grids
        self.model.weights, self.model.grids = self.init_weights, self.init_grids
        r = self.disagreement()
        self.model.weights, self.model.grids = w, g
        return {"untrained_hit_disagreement": r["hit_disagreement"],
                "untrained_normal_err_deg_mean": r["normal_err_deg_mean"]}


# ---------------------------------------------------------------------------
# Direct lighting with importance-sampled lights (Sec. 5 'Training', Sec. 6.2)
# ---------------------------------------------------------------------------
def ceiling_lights() -> np.ndarray:
    """Eight one-sided quad lights under the room's ceiling (y = 19.9),
    emitting downwards, with radiant fluxes spread over two orders of
    magnitude: [K, 10] = corner, edge e1, edge e2, radiance."""
    rows = []
    spec = [(-16, -12, 4, 4, 6.0), (-6, -14, 2, 2, 24.0), (4, -12, 3, 5, 2.0), (12, -6, 2, 6, 0.5),
            (-14, 6, 5, 3, 0.25), (-4, 8, 1, 1, 60.0), (6, 4, 4, 2, 1.0), (12, 10, 6, 4, 0.02)]
    for x, z, a, b, Le in spec:
        # e1 along +x, e2 along +z: e1 x e2 points down (-y)
        rows.append([x, 19.9, z, a, 0, 0, 0, 0, b, Le])
    return np.asarray(rows, np.float32)


@dataclass
class RenderConfig(PaperEncodingConfig):
    sampling: str = "importance"  # light selection of the training rays: "importance" (flux) or "uniform"
    render_spp: int = 4           # light samples per pixel of the rendered frame (importance)
    albedo: float = 0.8
    train_spp: int = 4


def render_config(sampling: str = "importance", train_spp: int = 4) -> RenderConfig:
    return RenderConfig(sampling=sampling, train_spp=train_spp, max_pairs_per_ray=8)


class RenderPipeline(PaperEncodingPipeline):
    """The paper-encoding pipeline inside a direct-lighting renderer: the
    shadow rays of the rendered frame are render_spp light samples per pixel,
    lights picked by flux from a tabulated CDF (Sec. 5); the training rays are
    one light sample per jittered camera sample, picked by flux or uniformly
    (the comparison of Sec. 6.2).  A frame is light sampling, the shadow
    query and shading; the exact frame uses the BVH cast instead of NIF."""

    def _light_setup(self):
        if getattr(self, "_lt", None) is None:
            lights = ceiling_lights()
            A = np.linalg.norm(np.cross(lights[:, 3:6], lights[:, 6:9]), axis=1)
            power = np.pi * lights[:, 9] * A
            self._lt = torch.from_numpy(lights).to(self.dev)
            self._cdf = {"importance": nif.light_cdf(torch.from_numpy(power.astype(np.float32)).to(self.dev)),
                         "uniform": nif.light_cdf(torch.ones(len(lights), device=self.dev))}
        return self._lt

    def _light_rays(self, camera: torch.Tensor, seed: int, spp: int, sampling: str):
        lights = self._light_setup()
        n = int(camera.shape[0])
        t, prim = self.bvh.cast_closest(camera)
        u = torch.from_numpy(np.random.default_rng(seed).random((n * spp, 3), dtype=np.float32)).to(self.dev)
        return nif.light_samples(camera, t, prim, self.verts, self.tris, lights, self._cdf[sampling], u, spp,
                                 self.cfg.tmin, self.cfg.albedo)

    def _eval_rays(self, camera: torch.Tensor) -> torch.Tensor:
        self.n_pix = int(camera.shape[0])
        self.eval_camera = camera
        self.eval_u = torch.from_numpy(np.random.default_rng(4321).random(
            (self.n_pix * self.cfg.render_spp, 3), dtype=np.float32)).to(self.dev)
        rays, self.eval_f = self._light_rays(camera, 4321, self.cfg.render_spp, "importance")
        return rays

    def _shadow_rays(self, camera: torch.Tensor, light_seed: int) -> torch.Tensor:
        rays, _ = self._light_rays(camera, light_seed, 1, self.cfg.sampling)
        return rays

    def render(self, visibility: str = "nif") -> torch.Tensor:
        """Pixel radiance of the frame with NIF or exact (BVH) visibility."""
        bits = nif.empty_bits(self.n_rays)
        (self.nif_query if visibility == "nif" else self.bvh_query)(bits)
        return nif.shade(self.eval_f, bits, self.n_pix, self.cfg.render_spp)

    def psnr(self) -> float:
        """PSNR (dB) of the NIF frame against the exact frame, both scaled by
        the exact frame's 99.5th percentile and clamped to [0, 1]."""
        ref = self.render("bvh")
        img = self.render("nif")
        torch.cuda.synchronize()
        s = float(torch.quantile(ref[ref > 0][::max(1, int((ref > 0).sum()) // 1_000_000)].float(), 0.995))
        a = (ref / s).clamp(0, 1)
        b = (img / s).clamp(0, 1)
        mse = float(((a - b) ** 2).mean())
        return 10.0 * float(np.log10(1.0 / max(mse, 1e-30)))
