"""The measured workloads, built from the seeded generators in ``synth``.

Each workload is described by what it is and its sizes:

* ``tiny_object``   -- one displaced level-5 icosphere (20,480 triangles)
  scaled to the unit box, 65,536 rays from a radius-1.5 shell in uniform
  directions (or aimed at the box), 8-level x 2-feature dense FP32 grids at
  resolutions 4..64, MLP 3x64 ReLU with Xavier weights.
* ``room_scene``    -- 64 displaced icospheres (15,680 triangles each, 1.0M
  in total) with centres uniform in [-10,10]^3 inside a 12-triangle room
  [-20,20]^3, a pinhole camera at (0,0,19) looking at the origin (vfov 60),
  a point light outside every object; hashed 16-level x 2-feature FP16 grids
  (2^19 entries per level, resolutions 16..1024) per object, shared outer
  and inner 3x64 networks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth

TINY_RES = [4, 5, 8, 13, 19, 28, 43, 64]
ROOM_RES = [16, 21, 27, 36, 48, 64, 84, 111, 147, 194, 256, 337, 445, 588, 776, 1024]


@dataclass
class TinyObject:
    verts: np.ndarray
    tris: np.ndarray
    aabb: np.ndarray  # [1, 6]
    rays: np.ndarray
    res: list
    weights: list     # Xavier matrices
    grid_values: np.ndarray  # [1, 2, V*F]


def tiny_object(seed: int = 1, n_rays: int = 65536, aimed: bool = False,
                grid_scale: float = 1e-4, V: int | None = None) -> TinyObject:
    """One mesh n=32 in the unit box, shell rays, dense 8-level grids."""
    rng = np.random.default_rng(seed)
    v, t = synth.displaced_icosphere(32, rng)
    v = synth.fit_to_box(v).astype(np.float32)
    aabb = np.concatenate([v.min(axis=0), v.max(axis=0)])[None, :].astype(np.float32)
    rr = np.random.default_rng(seed + 1000)
    rays = synth.aimed_rays(rr, n_rays, aabb[0], 1.5) if aimed else synth.shell_rays(rr, n_rays)
    res = list(TINY_RES)
    if V is None:
        V = sum(synth.level_sizes(res, 19))
    wr = np.random.default_rng(seed + 2000)
    mats = synth.mlp_init(wr, 3 * len(res) * 2, 64, 3)
    grid = synth.grid_init(np.random.default_rng(seed + 3000), 2 * V * 2, scale=grid_scale)
    return TinyObject(v, t, aabb, rays, res, mats, grid.reshape(1, 2, V * 2))


@dataclass
class RoomScene:
    scene: synth.Scene
    camera: np.ndarray  # [W*H, 8] camera rays
    light: np.ndarray   # [3]
    width: int
    height: int


def room_scene(n_obj: int = 64, n: int = 28, width: int = 1920, height: int = 1080,
               seed: int = 7, jitter_seed: int | None = None) -> RoomScene:
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-10.0, 10.0, size=(n_obj, 3))
    meshes = [synth.displaced_icosphere(n, rng, centre=c) for c in centres]
    sc = synth.build_scene(meshes, extra_geometry=synth.room_box(20.0))
    light = synth.outside_point(rng, sc.obj_aabb, -15.0, 15.0)
    jitter = None
    if jitter_seed is not None:
        jitter = np.random.default_rng(jitter_seed).uniform(size=(width * height, 2))
    cam = synth.camera_rays(width, height, (0.0, 0.0, 19.0), (0.0, 0.0, 0.0), 60.0, jitter=jitter)
    return RoomScene(sc, cam, light, width, height)
