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

GRID_SEED = 0x5EED0001  # SplitMix64 seed of the grid latents
GRID_SCALE = 1e-4       # latent initialisation U(-1e-4, 1e-4), Sec. 5 "Initialization"
EVAL_LIGHT_SEED = 4321  # area-light samples of the evaluation frame


@dataclass(frozen=True)
class FrameSpec:
    """The evaluation frame of a room-style workload and its network, as
    plain numbers: what the GPU pipeline and the CPU oracle both build from.

    n_obj objects of icosphere frequency n in the given layout, a width x
    height pixel-centre frame, shadow rays to one point light or `samples`
    area-light points per pixel, segments starting at tmin; per object a
    position and a direction grid of len(res) levels x n_features, 2^log2_table
    entries per hashed level; outer and inner networks of n_hidden x width."""
    name: str
    n_obj: int
    n: int
    layout: str
    res: tuple
    n_features: int = 2
    log2_table: int = 19
    n_hidden: int = 3
    width_mlp: int = 64
    width: int = 1920
    height: int = 1080
    seed: int = 7
    tmin: float = 1e-3
    area_light: bool = False
    samples: int = 1

    @property
    def K(self) -> int:
        return 3 * len(self.res) * self.n_features


ROOM_FRAME = FrameSpec("room", n_obj=64, n=28, layout="random", res=tuple(ROOM_RES))
FULL_FRAME = FrameSpec("full", n_obj=480, n=56, layout="lattice", res=tuple(TINY_RES),
                       area_light=True, samples=4)
FRAMES = {"room": ROOM_FRAME, "full": FULL_FRAME}


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
               seed: int = 7, jitter_seed: int | None = None, layout: str = "random",
               n_lights: int = 1, tri_min: int = 10_000, tri_max: int = 500_000) -> RoomScene:
    """Objects in a 12-triangle room [-20,20]^3 seen by a pinhole camera at
    (0,0,19) looking at the origin.

    layout "random":  n_obj displaced icospheres (frequency n), centres uniform
                      in [-10,10]^3; n_lights point lights outside every box.
    layout "single":  the small-configuration object (frequency 32, 20,480
                      triangles) scaled to the box [-4,4]^3 at the origin.
    layout "lattice": a jittered 10 x 6 x 8 lattice (spacing 4) of displaced
                      icospheres of frequency n (480 objects for n_obj=480).
    layout "mixed":   n_obj displaced icospheres of radius 1.5 with triangle
                      counts log-uniform in [tri_min, tri_max] (frequency
                      round(sqrt(T / 20))), centres uniform in [-10,10]^3.
    Point lights are drawn outside every object box; area-light samples are
    drawn separately (area_light_samples)."""
    rng = np.random.default_rng(seed)
    if layout == "single":
        v, t = synth.displaced_icosphere(32, rng)
        v = synth.fit_to_box(v, -4.0, 4.0)
        meshes = [(v, t)]
    elif layout == "lattice":
        gx, gy, gz = 10, 6, 8
        cells = np.stack(np.meshgrid(np.arange(gx), np.arange(gy), np.arange(gz), indexing="ij"), -1)
        cells = cells.reshape(-1, 3)[:n_obj].astype(np.float64)
        centres = (cells - (np.array([gx, gy, gz]) - 1) / 2.0) * 4.0
        centres += rng.uniform(-0.6, 0.6, size=centres.shape)
        meshes = [synth.displaced_icosphere(n, rng, centre=c) for c in centres]
    elif layout == "mixed":
        tris = np.exp(rng.uniform(np.log(tri_min), np.log(tri_max), size=n_obj))
        freqs = np.maximum(1, np.round(np.sqrt(tris / 20.0))).astype(int)
        centres = rng.uniform(-10.0, 10.0, size=(n_obj, 3))
        meshes = [synth.displaced_icosphere(int(f), rng, radius=1.5, centre=c) for f, c in zip(freqs, centres)]
    else:
        centres = rng.uniform(-10.0, 10.0, size=(n_obj, 3))
        meshes = [synth.displaced_icosphere(n, rng, centre=c) for c in centres]
    sc = synth.build_scene(meshes, extra_geometry=synth.room_box(20.0))
    lights = [synth.outside_point(rng, sc.obj_aabb, -15.0, 15.0) for _ in range(n_lights)]
    light = lights[0] if n_lights == 1 else np.stack(lights)
    jitter = None
    if jitter_seed is not None:
        jitter = np.random.default_rng(jitter_seed).uniform(size=(width * height, 2))
    cam = synth.camera_rays(width, height, (0.0, 0.0, 19.0), (0.0, 0.0, 0.0), 60.0, jitter=jitter)
    return RoomScene(sc, cam, light, width, height)


AREA_LIGHT = ((-2.0, 19.9, -2.0), (4.0, 0.0, 0.0), (0.0, 0.0, 4.0))  # corner, edge u, edge v


def area_light_samples(rng: np.random.Generator, n_pixels: int, spp: int) -> np.ndarray:
    """Uniform points on the 4 x 4 ceiling quad light, spp per pixel:
    float32 [n_pixels * spp, 3]."""
    c, eu, ev = (np.asarray(x) for x in AREA_LIGHT)
    a = rng.uniform(size=(n_pixels * spp, 1))
    b = rng.uniform(size=(n_pixels * spp, 1))
    return (c[None, :] + a * eu[None, :] + b * ev[None, :]).astype(np.float32)


@dataclass
class GroupedObjects:
    scene: synth.Scene
    rays: np.ndarray    # [N, 8], rays of object k are contiguous
    counts: np.ndarray  # pairs (= rays) per object, int64 [n_obj]


def grouped_objects(n_obj: int = 32, total_rays: int = 8_000_000, seed: int = 11,
                    tri_min: int = 10_000, tri_max: int = 500_000, alpha: float = 1.5,
                    spacing: float = 8.0) -> GroupedObjects:
    """n_obj displaced icospheres with triangle counts log-uniform in
    [tri_min, tri_max] (frequency n = round(sqrt(T / 20))), placed on a line
    `spacing` apart; object k (1-based) gets round(total * k^-alpha / sum_j
    j^-alpha) rays (the remainder goes to k = 1), each from a sphere of 1.5x the
    box half-diagonal around its box, aimed at a uniform point in the box."""
    rng = np.random.default_rng(seed)
    tris = np.exp(rng.uniform(np.log(tri_min), np.log(tri_max), size=n_obj))
    freqs = np.maximum(1, np.round(np.sqrt(tris / 20.0))).astype(int)
    meshes = [synth.displaced_icosphere(int(f), rng, centre=(k * spacing, 0.0, 0.0))
              for k, f in enumerate(freqs)]
    sc = synth.build_scene(meshes)
    w = np.arange(1, n_obj + 1, dtype=np.float64) ** (-alpha)
    counts = np.round(total_rays * w / w.sum()).astype(np.int64)
    counts[0] += total_rays - counts.sum()
    rays = []
    for k in range(n_obj):
        box = sc.obj_aabb[k]
        half_diag = 0.5 * float(np.linalg.norm(box[3:] - box[:3]))
        rays.append(synth.aimed_rays(rng, int(counts[k]), box, 1.5 * half_diag))
    return GroupedObjects(sc, np.ascontiguousarray(np.concatenate(rays)), counts)
