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

GRID_SEED = 0x5EED0001
GRID_SCALE = 1e-4  # latent init U(-1e-4, 1e-4), Sec. 5 "Initialization"


@dataclass
class RoomConfig:
    n_obj: int = 64
    n: int = 28                 # icosphere frequency: 20 n^2 triangles
    width: int = 1920
    height: int = 1080
    seed: int = 7
    res: tuple = tuple(workloads.ROOM_RES)
    n_features: int = 2
    log2_table: int = 19
    grid_dtype: int = L.NIF_F16
    mlp_dtype: int = L.NIF_F16
    n_hidden: int = 3
    width_mlp: int = 64
    train_spp: int = 4          # jittered samples per pixel collected for training
    train_steps: int = 64
    batch: int = 262144
    lr: float = 1e-2
    tmin: float = 1e-3
    ctas_per_sm: int = 0


class RoomPipeline:
    def __init__(self, cfg: RoomConfig, device="cuda", log=print):
        self.cfg = cfg
        self.log = log
        t0 = time.time()
        ws = workloads.room_scene(cfg.n_obj, cfg.n, cfg.width, cfg.height, cfg.seed)
        self.ws = ws
        sc = ws.scene
        dev = torch.device(device)
        self.dev = dev
        self.verts = torch.from_numpy(sc.verts).to(dev)
        self.tris = torch.from_numpy(sc.tris).to(dev)
        self.tags = torch.from_numpy(sc.tri_obj).to(dev)
        self.obj_aabb = torch.from_numpy(sc.obj_aabb).to(dev)
        self.n_tris = int(sc.tris.shape[0])
        # exact structures: all triangles (comparison + labels), non-NIF
        # geometry alone (the room), object boxes (top level of the NIF query)
        self.bvh = nif.BVH(self.verts, self.tris, self.tags)
        room = sc.tri_obj < 0
        self.room_bvh = nif.BVH(self.verts, torch.from_numpy(sc.tris[room]).to(dev))
        self.tlas = nif.BVH.from_boxes(self.obj_aabb)
        self.light = torch.from_numpy(ws.light.astype(np.float32)).to(dev)
        # evaluation frame: pixel-centre camera rays -> primary hits -> shadow rays
        self.rays = self._shadow_rays(torch.from_numpy(ws.camera).to(dev))
        self.n_rays = int(self.rays.shape[0])
        # model
        c = cfg
        ncfg = nif.NifConfig(res=list(c.res), n_features=c.n_features, log2_table=c.log2_table,
                             grid_dtype=c.grid_dtype, n_hidden=c.n_hidden, width=c.width_mlp,
                             mlp_dtype=c.mlp_dtype, net_mode=L.NIF_NETS_CLASS,
                             ctas_per_sm=c.ctas_per_sm)
        self.V = nif.NifModel.grid_vertices(ncfg)
        self.P = nif.NifModel.weight_count(ncfg)
        n_grid = c.n_obj * 2 * self.V * c.n_features
        self.g_master = torch.empty(n_grid, dtype=torch.float32, device=dev)
        L.call("nif_fill_uniform", ctypes.c_void_p(self.g_master.data_ptr()), n_grid, GRID_SEED,
               GRID_SCALE, nif._stream())
        wr = np.random.default_rng(c.seed + 101)
        flat = np.concatenate([synth.flatten_mlp(synth.mlp_init(wr, ncfg.K, c.width_mlp, c.n_hidden))
                               for _ in range(2)])
        self.w_master = torch.from_numpy(flat).to(dev)
        gdt = {L.NIF_F16: torch.float16, L.NIF_F32: torch.float32}[c.grid_dtype]
        mdt = {L.NIF_F16: torch.float16, L.NIF_BF16: torch.bfloat16, L.NIF_F32: torch.float32}[c.mlp_dtype]
        self.model = nif.NifModel(ncfg, self.obj_aabb, self.g_master.to(gdt), self.w_master.to(mdt))
        self.init_weights = self.model.weights.clone()
        self.init_grids = self.model.grids.clone()
        torch.cuda.synchronize()
        self.log(f"room scene ready: {self.n_tris} triangles, {self.n_rays} shadow rays, "
                 f"{n_grid / 1e9:.3f}G grid latents ({time.time() - t0:.1f}s)")

    # ------------------------------------------------------------ inputs
    def _shadow_rays(self, camera: torch.Tensor) -> torch.Tensor:
        t, _ = self.bvh.cast_closest(camera)
        return nif.shadow_rays(camera, t, self.light, tmin=self.cfg.tmin)

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
            r = self._shadow_rays(torch.from_numpy(cam).to(self.dev))
            rid, qo, goff, count = self.model.frontend(r, tlas=self.tlas)
            torch.cuda.synchronize()
            nq = int(count.item())
            rid, qo = rid[:nq], qo[:nq]
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

    def train(self, steps: int | None = None, seed: int = 99, pairs=None):
        c = self.cfg
        steps = steps if steps is not None else c.train_steps
        rays, rid, qo, lab, n_outer = pairs if pairs is not None else self.training_pairs()
        npool = int(rid.shape[0])
        self.trainer = nif.Trainer(self.model, lr=c.lr, w_master=self.w_master, g_master=self.g_master)
        rng = np.random.default_rng(seed)
        losses = []
        t0 = time.time()
        B = min(c.batch, npool)
        for s in range(steps):
            idx = np.sort(rng.choice(npool, B, replace=False))
            k = int(np.searchsorted(idx, n_outer))
            goff = torch.tensor([0, k, B], dtype=torch.int64, device=self.dev)
            it = torch.from_numpy(idx).to(self.dev)
            loss = self.trainer.step(rays, rid[it].contiguous(), qo[it].contiguous(), goff,
                                     lab[it].contiguous(), B)
            losses.append(loss.clone())
        torch.cuda.synchronize()
        dt = time.time() - t0
        self.model.check(self.trainer._ws)
        self.losses = [float(x.item()) for x in losses]
        self.log(f"trained {steps} steps of {B} pairs from a pool of {npool} in {dt:.2f}s; "
                 f"loss {self.losses[0]:.4f} -> {self.losses[-1]:.4f}")
        return dt

    def release_training_state(self):
        """Drop FP32 masters, Adam moments and the initial copies once
        training and the ablations are done (inference keeps the FP16 copies)."""
        self.trainer = None
        self.g_master = None
        self.w_master = None
        self.init_grids = None
        self.init_weights = None

    # ------------------------------------------------------------ queries
    def nif_query(self, bits: torch.Tensor, rays: torch.Tensor | None = None, stream=None):
        """NIF visibility: exact cast of the non-NIF geometry (the room), then
        the top-level front end and the fused networks OR-ed into the mask."""
        rays = self.rays if rays is None else rays
        self.room_bvh.cast_shadow(rays, out=bits, stream=stream)
        self.model.infer(rays, bits, tlas=self.tlas, stream=stream)
        return bits

    def bvh_query(self, bits: torch.Tensor, rays: torch.Tensor | None = None, stream=None):
        rays = self.rays if rays is None else rays
        return self.bvh.cast_shadow(rays, out=bits, stream=stream)

    def disagreement(self):
        """Fraction of shadow rays where NIF and the BVH disagree, over all rays
        and over rays with at least one NIF query."""
        a = nif.empty_bits(self.n_rays)
        b = nif.empty_bits(self.n_rays)
        self.nif_query(a)
        self.bvh_query(b)
        rid, qo, goff, count = self.model.frontend(self.rays, tlas=self.tlas)
        torch.cuda.synchronize()
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
        rid, qo, goff, count = self.model.frontend(self.rays, tlas=self.tlas)
        torch.cuda.synchronize()
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
