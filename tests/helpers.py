"""Shared test scaffolding: builds the same seeded inputs for the CUDA path and
the oracle (inputs only; no expected value is computed here)."""
from __future__ import annotations

import numpy as np

from paper_2306_07191_gb300 import synth


def to_dtype_values(a: np.ndarray, dtype: str) -> np.ndarray:
    """Round float32 values to the storage type the GPU will hold and return
    them as float64 (what the oracle consumes)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    if dtype == "f16":
        t = t.half()
    elif dtype == "bf16":
        t = t.bfloat16()
    elif dtype == "e4m3":
        t = t.to(torch.float8_e4m3fn)
    return t.double().numpy()


def oracle_model(onif, res, F, log2, aabb, grids64, nets64, net_mode="single", act="relu"):
    return onif.Model(res=list(res), F=F, log2_table=log2, obj_aabb=np.asarray(aabb, np.float32),
                      grids=np.asarray(grids64, np.float64), nets=nets64, net_mode=net_mode, act=act)


def pairs_key(ray_id, obj):
    return np.asarray(ray_id, np.int64) * 65536 + np.asarray(obj, np.int64)


def random_boxes_scene(rng, n_obj=6, extent=3.0):
    """Overlapping object boxes with rays from inside and outside them."""
    lo = rng.uniform(-extent, extent - 1.0, size=(n_obj, 3))
    size = rng.uniform(0.5, 2.0, size=(n_obj, 3))
    return np.concatenate([lo, lo + size], axis=1).astype(np.float32)
