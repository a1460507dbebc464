"""The CPU oracle's own evaluation frames and its timed visibility query.

TEST INFRASTRUCTURE ONLY: only the tests and the CPU legs of ``bench.py`` may
import this module.  It imports nothing from the CUDA library's package: the
scene, camera rays and light points come in as arrays from the seeded input
generators, and the oracle derives everything else itself.

* ``shadow_rays``: shadow segments from primary hits towards light points
  (FP32, one rounding per operation, in the written order): p = o + t d,
  v = light - p, |v| = sqrt(vx^2 + vy^2 + vz^2) summed left to right,
  d' = v / |v|, segment (tmin, |v|).  A primary miss gives an empty segment
  (tmin = tmax = 0) along the camera ray.
* ``frame_rays``: primary hits of camera rays with the oracle's own BVH,
  then ``shadow_rays``.
* ``timed_query``: the FP64 NIF visibility query (query selection, encoding,
  MLP, threshold; ``oracle.nif``) of a set of shadow rays, split into chunks
  over a pool of worker processes on the host's cores, and timed.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

from . import OracleBVH
from . import nif as onif


def shadow_rays(camera: np.ndarray, t: np.ndarray, light_pts: np.ndarray, tmin: float,
                spp: int = 1) -> np.ndarray:
    """Shadow rays [n * spp, 8] float32 from the primary hits at parameter t of
    `camera` rays (float32 [n, 8]; t = inf for a miss) towards light points:
    one shared point (float32 [3]) or one per shadow ray (float32 [n * spp, 3],
    pixel-major)."""
    cam = np.repeat(np.asarray(camera, np.float32), spp, axis=0)
    th = np.repeat(np.asarray(t, np.float32), spp)
    lp = np.asarray(light_pts, np.float32)
    lp = np.broadcast_to(lp.reshape(-1, 3), (cam.shape[0], 3)) if lp.size == 3 else lp.reshape(-1, 3)
    hit = np.isfinite(th)
    tt = np.where(hit, th, np.float32(0.0)).astype(np.float32)
    p = np.stack([cam[:, k] + tt * cam[:, 4 + k] for k in range(3)], 1).astype(np.float32)
    v = (lp - p).astype(np.float32)
    ss = v[:, 0] * v[:, 0]
    ss = ss + v[:, 1] * v[:, 1]
    ss = ss + v[:, 2] * v[:, 2]
    ln = np.sqrt(ss).astype(np.float32)
    safe = np.where(hit, ln, np.float32(1.0)).astype(np.float32)
    out = np.zeros((cam.shape[0], 8), np.float32)
    out[:, 0:3] = np.where(hit[:, None], p, cam[:, 0:3])
    out[:, 3] = np.where(hit, np.float32(tmin), np.float32(0.0))
    out[:, 4:7] = np.where(hit[:, None], v / safe[:, None], cam[:, 4:7])
    out[:, 7] = np.where(hit, ln, np.float32(0.0))
    return out


def frame_rays(bvh: OracleBVH, camera: np.ndarray, light_pts: np.ndarray, tmin: float,
               spp: int = 1) -> np.ndarray:
    """Shadow rays of `camera` rays: their closest hits with the oracle's
    BVH (t = inf for a miss), then shadow_rays."""
    _, t, _ = bvh.cast(camera, closest=True)
    occ_t = np.where(np.isfinite(t), t, np.inf).astype(np.float32)
    return shadow_rays(camera, occ_t, light_pts, tmin, spp)


# ------------------------------------------------------- timed FP64 query
_MODEL = None


def _init_worker(model):
    global _MODEL
    _MODEL = model


def query_occlusion(m: onif.Model, rays: np.ndarray):
    """FP64 NIF visibility of shadow rays: every (ray, object) pair whose
    segment overlaps the object's box, its logit, and the ray's occlusion
    (any pair with z < 0).  Returns (occluded bool [n], pairs)."""
    rid, obj, inner = onif.queries(rays, m.obj_aabb)
    z = onif.forward(m, rays, rid, obj, inner)
    return onif.ray_occlusion(rays.shape[0], rid, z), len(rid)


def _work(rays):
    occ, nq = query_occlusion(_MODEL, rays)
    return int(occ.sum()), nq


def cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class QueryPool:
    """Worker processes (started with `spawn`, one BLAS thread each) that
    hold one oracle model and answer chunks of shadow rays."""

    def __init__(self, model: onif.Model, processes: int | None = None):
        self.processes = processes or cores()
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.processes, initializer=_init_worker, initargs=(model,))
        # every worker loads numpy and the model before the first timed call
        self.pool.map(_work, [np.zeros((1, 8), np.float32)] * self.processes)

    def timed_query(self, rays: np.ndarray, chunk: int | None = None):
        """Answer all rays in chunks (by default one per process: the oracle's
        encoding loops over the objects of a chunk, so large chunks amortise
        it); returns (rays per second, seconds, pairs, occluded rays)."""
        chunk = chunk or -(-rays.shape[0] // self.processes)
        parts = [rays[a:a + chunk] for a in range(0, rays.shape[0], chunk)]
        t0 = time.perf_counter()
        res = self.pool.map(_work, parts, chunksize=1)
        dt = time.perf_counter() - t0
        return rays.shape[0] / dt, dt, sum(r[1] for r in res), sum(r[0] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()
