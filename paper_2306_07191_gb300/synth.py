"""Seeded synthetic inputs for the Neural Intersection Function shadow-ray path.

This module only *draws* inputs: procedural meshes, rays, camera rays, light
samples, network and grid initial values, training-batch permutations.  It holds
none of the method's arithmetic (no ray/triangle or ray/box test, no encoding,
no network evaluation), so the CUDA path and the CPU oracle can both consume
what it produces without sharing any computation.

The paper's scenes (Stanford models, Centaur, Bistro; Sec. 6, Table 2) are not
available, so frequency-n geodesic icospheres with smooth seeded radial noise
stand in for them at the paper's scale (0.5M-53M triangles, ~1M shadow rays per
1920x1080 frame, Table 2).  Every random draw goes through numpy's PCG64 with a
seed stated in the workload description.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RAY_FLOATS = 8  # ox, oy, oz, tmin, dx, dy, dz, tmax (32 bytes)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
_PHI = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array(
    [(-1, _PHI, 0), (1, _PHI, 0), (-1, -_PHI, 0), (1, -_PHI, 0),
     (0, -1, _PHI), (0, 1, _PHI), (0, -1, -_PHI), (0, 1, -_PHI),
     (_PHI, 0, -1), (_PHI, 0, 1), (-_PHI, 0, -1), (-_PHI, 0, 1)], dtype=np.float64)
_ICO_F = np.array(
    [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
     (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
     (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)

_SPHERE_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def geodesic_sphere(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit geodesic sphere of frequency n: 20*n^2 triangles, 10*n^2+2 vertices.

    Each icosahedron face is split into n^2 triangles on a barycentric lattice,
    the lattice points are projected to the unit sphere and shared points on
    face edges are merged so the mesh is watertight.
    Returns (vertices float64 [V,3], triangles int32 [T,3]).
    """
    if n in _SPHERE_CACHE:
        v, t = _SPHERE_CACHE[n]
        return v.copy(), t.copy()
    ii, jj = [], []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            ii.append(i)
            jj.append(j)
    ii = np.array(ii)
    jj = np.array(jj)
    lat = {(a, b): k for k, (a, b) in enumerate(zip(ii.tolist(), jj.tolist()))}
    tri_local = []
    for i in range(n):
        for j in range(n - i):
            tri_local.append((lat[(i, j)], lat[(i + 1, j)], lat[(i, j + 1)]))
            if i + j < n - 1:
                tri_local.append((lat[(i + 1, j)], lat[(i + 1, j + 1)], lat[(i, j + 1)]))
    tri_local = np.array(tri_local, dtype=np.int64)
    npts = len(ii)
    a = _ICO_V[_ICO_F[:, 0]][:, None, :]
    b = _ICO_V[_ICO_F[:, 1]][:, None, :]
    c = _ICO_V[_ICO_F[:, 2]][:, None, :]
    pts = a + (b - a) * (ii[None, :, None] / n) + (c - a) * (jj[None, :, None] / n)
    pts = pts.reshape(-1, 3)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    key = np.round(pts * 1e9).astype(np.int64)
    _, first, inverse = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inverse = inverse.reshape(-1)
    verts = pts[first]
    tris = (tri_local[None, :, :] + (np.arange(20) * npts)[:, None, None]).reshape(-1, 3)
    tris = inverse[tris].astype(np.int32)
    _SPHERE_CACHE[n] = (verts, tris)
    return verts.copy(), tris.copy()


def radial_noise(unit_dirs: np.ndarray, rng: np.random.Generator, waves: int = 8) -> np.ndarray:
    """Sum of `waves` plane-wave sinusoids (frequencies 1..waves, seeded unit axes
    and phases) evaluated on unit vectors, normalised to [-1, 1] over the given set."""
    axes = rng.normal(size=(waves, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=waves)
    freqs = np.arange(1, waves + 1, dtype=np.float64)
    s = np.sin((unit_dirs @ axes.T) * freqs[None, :] + phases[None, :]).sum(axis=1)
    return s / np.max(np.abs(s))


def displaced_icosphere(n: int, rng: np.random.Generator, amplitude: float = 0.2,
                        radius: float = 1.0, centre=(0.0, 0.0, 0.0)) -> tuple[np.ndarray, np.ndarray]:
    """Frequency-n geodesic sphere with radius r = radius*(1 + amplitude*noise(v))."""
    v, t = geodesic_sphere(n)
    r = radius * (1.0 + amplitude * radial_noise(v, rng))
    v = v * r[:, None] + np.asarray(centre, dtype=np.float64)[None, :]
    return v, t


def fit_to_box(v: np.ndarray, lo=-0.5, hi=0.5) -> np.ndarray:
    """Per-axis affine map of vertices so their bounding box becomes [lo, hi]^3."""
    vmin = v.min(axis=0)
    vmax = v.max(axis=0)
    return lo + (v - vmin) / (vmax - vmin) * (hi - lo)


def room_box(half: float = 20.0) -> tuple[np.ndarray, np.ndarray]:
    """Closed axis-aligned box [-half, half]^3 as 12 triangles."""
    h = half
    v = np.array([[x, y, z] for x in (-h, h) for y in (-h, h) for z in (-h, h)], dtype=np.float64)
    # vertex index = 4*ix + 2*iy + iz
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    t = []
    for a, b, c, d in quads:
        t.append((a, b, c))
        t.append((a, c, d))
    return v, np.array(t, dtype=np.int32)


@dataclass
class Scene:
    """Triangle soup of several objects plus per-object bookkeeping.

    verts float32 [V,3]; tris int32 [T,3]; tri_obj int32 [T] (object id, -1 for
    non-NIF geometry such as the room); obj_aabb float32 [n_obj, 6] =
    (min xyz, max xyz) of each object's float32 vertices.
    """
    verts: np.ndarray
    tris: np.ndarray
    tri_obj: np.ndarray
    obj_aabb: np.ndarray
    obj_tri_range: np.ndarray  # int64 [n_obj, 2] first triangle, count
    light: np.ndarray | None = None  # point light, float32 [3]
    extra: dict = field(default_factory=dict)

    @property
    def n_obj(self) -> int:
        return int(self.obj_aabb.shape[0])

    def object_mesh(self, k: int) -> tuple[np.ndarray, np.ndarray]:
        s, c = self.obj_tri_range[k]
        tri = self.tris[s:s + c]
        return self.verts, tri


def build_scene(meshes: list[tuple[np.ndarray, np.ndarray]], extra_geometry=None) -> Scene:
    verts, tris, tri_obj, aabbs, ranges = [], [], [], [], []
    voff = 0
    toff = 0
    for k, (v, t) in enumerate(meshes):
        v32 = np.asarray(v, dtype=np.float32)
        verts.append(v32)
        tris.append(t.astype(np.int64) + voff)
        tri_obj.append(np.full(len(t), k, dtype=np.int32))
        aabbs.append(np.concatenate([v32.min(axis=0), v32.max(axis=0)]))
        ranges.append((toff, len(t)))
        voff += len(v32)
        toff += len(t)
    if extra_geometry is not None:
        v, t = extra_geometry
        verts.append(np.asarray(v, dtype=np.float32))
        tris.append(t.astype(np.int64) + voff)
        tri_obj.append(np.full(len(t), -1, dtype=np.int32))
        voff += len(v)
    return Scene(
        verts=np.ascontiguousarray(np.concatenate(verts), dtype=np.float32),
        tris=np.ascontiguousarray(np.concatenate(tris), dtype=np.int32),
        tri_obj=np.concatenate(tri_obj),
        obj_aabb=np.ascontiguousarray(np.stack(aabbs), dtype=np.float32),
        obj_tri_range=np.array(ranges, dtype=np.int64),
    )


# --------------------------------------------------------------------------
# rays
# --------------------------------------------------------------------------
def unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def pack_rays(o: np.ndarray, d: np.ndarray, tmin, tmax) -> np.ndarray:
    n = o.shape[0]
    r = np.empty((n, RAY_FLOATS), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


def shell_rays(rng: np.random.Generator, n: int, radius: float = 1.5,
               centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Origins uniform on a sphere of `radius`, directions uniform on S^2,
    segment [0, +inf)."""
    o = unit_vectors(rng, n) * radius + np.asarray(centre)
    d = unit_vectors(rng, n)
    return pack_rays(o, d, 0.0, np.inf)


def aimed_rays(rng: np.random.Generator, n: int, aabb: np.ndarray, shell_radius: float) -> np.ndarray:
    """Origins uniform on a sphere around the box centre, each ray aimed at a
    uniform point inside the box; segment [0, +inf)."""
    lo = aabb[:3].astype(np.float64)
    hi = aabb[3:].astype(np.float64)
    c = 0.5 * (lo + hi)
    o = c + unit_vectors(rng, n) * shell_radius
    tgt = lo + rng.uniform(size=(n, 3)) * (hi - lo)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return pack_rays(o, d, 0.0, np.inf)


def camera_rays(width: int, height: int, eye, target, vfov_deg: float,
                up=(0.0, 1.0, 0.0), jitter: np.ndarray | None = None) -> np.ndarray:
    """Pinhole camera rays, row-major over pixels, through pixel centres or
    through pixel + jitter (jitter float [H*W, 2] in [0,1)); segment [0, +inf)."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    h = math.tan(math.radians(vfov_deg) * 0.5)
    aspect = width / height
    py, px = np.meshgrid(np.arange(height, dtype=np.float64), np.arange(width, dtype=np.float64),
                         indexing="ij")
    px = px.reshape(-1)
    py = py.reshape(-1)
    if jitter is None:
        sx = px + 0.5
        sy = py + 0.5
    else:
        sx = px + jitter[:, 0]
        sy = py + jitter[:, 1]
    x = (2.0 * sx / width - 1.0) * aspect * h
    y = (1.0 - 2.0 * sy / height) * h
    d = fwd[None, :] + x[:, None] * right[None, :] + y[:, None] * upv[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(eye, d.shape)
    return pack_rays(o, d, 0.0, np.inf)


def surface_points(rng: np.random.Generator, scene: Scene, n: int, objects=None) -> tuple[np.ndarray, np.ndarray]:
    """Area-uniform points on the triangles of the given objects (all objects if
    None). Returns (points float32 [n,3], object id int32 [n])."""
    v = scene.verts.astype(np.float64)
    sel = np.ones(len(scene.tris), dtype=bool) if objects is None else np.isin(scene.tri_obj, objects)
    sel &= scene.tri_obj >= 0
    idx = np.nonzero(sel)[0]
    t = scene.tris[idx]
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cdf = np.cumsum(area)
    pick = np.searchsorted(cdf, rng.uniform(0, cdf[-1], size=n), side="right")
    pick = np.minimum(pick, len(idx) - 1)
    r1 = rng.uniform(size=n)
    r2 = rng.uniform(size=n)
    s = np.sqrt(r1)
    p = (1 - s)[:, None] * a[pick] + (s * (1 - r2))[:, None] * b[pick] + (s * r2)[:, None] * c[pick]
    return p.astype(np.float32), scene.tri_obj[idx[pick]].astype(np.int32)


def point_to_light_rays(points: np.ndarray, light: np.ndarray, tmin: float = 1e-3) -> np.ndarray:
    """Shadow rays from surface points to a point light: unit direction, segment
    [tmin, |light - p|). Built in float64 then stored as float32 (an input recipe
    for tests; the camera pipeline builds its own rays on the device)."""
    p = points.astype(np.float64)
    dv = np.asarray(light, dtype=np.float64)[None, :] - p
    ln = np.linalg.norm(dv, axis=1)
    d = dv / ln[:, None]
    return pack_rays(p, d, tmin, ln)


def outside_point(rng: np.random.Generator, aabbs: np.ndarray, lo: float, hi: float,
                  margin: float = 0.25) -> np.ndarray:
    """A uniform point in [lo,hi]^3 that lies outside every box grown by margin."""
    for _ in range(100000):
        p = rng.uniform(lo, hi, size=3)
        inside = np.all((p[None, :] >= aabbs[:, :3] - margin) & (p[None, :] <= aabbs[:, 3:] + margin), axis=1)
        if not inside.any():
            return p.astype(np.float32)
    raise RuntimeError("no free light position")


# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------
def resolution_ladder(n_levels: int, n_min: int, n_max: int) -> list[int]:
    """Geometric per-level grid resolutions R_l = floor(n_min * b^l + 1e-9),
    b = (n_max / n_min)^(1/(L-1)); R counts cells per axis."""
    if n_levels == 1:
        return [n_min]
    b = (n_max / n_min) ** (1.0 / (n_levels - 1))
    return [int(math.floor(n_min * b ** l + 1e-9)) for l in range(n_levels)]


def level_sizes(res: list[int], log2_table: int) -> list[int]:
    """Vertices stored per level: (R+1)^3 when that fits in T = 2^log2_table,
    else T (hashed)."""
    t = 1 << log2_table
    return [min((r + 1) ** 3, t) for r in res]


def xavier_uniform(rng: np.random.Generator, fan_out: int, fan_in: int) -> np.ndarray:
    """Glorot-uniform matrix [fan_out, fan_in] (Sec. 5 'Initialization')."""
    a = math.sqrt(6.0 / (fan_in + fan_out))
    return rng.uniform(-a, a, size=(fan_out, fan_in)).astype(np.float32)


def mlp_init(rng: np.random.Generator, n_in: int, width: int, n_hidden: int,
             n_out: int = 1) -> list[np.ndarray]:
    """Bias-free MLP n_in -> width (x n_hidden) -> n_out, Xavier-uniform."""
    mats = []
    fan_in = n_in
    for _ in range(n_hidden):
        mats.append(xavier_uniform(rng, width, fan_in))
        fan_in = width
    mats.append(xavier_uniform(rng, n_out, fan_in))
    return mats


def grid_init(rng: np.random.Generator, n_params: int, scale: float = 1e-4) -> np.ndarray:
    """Latent grid values drawn from U(-1e-4, 1e-4) (Sec. 5 'Initialization')."""
    return rng.uniform(-scale, scale, size=n_params).astype(np.float32)


def flatten_mlp(mats: list[np.ndarray]) -> np.ndarray:
    return np.concatenate([m.reshape(-1) for m in mats]).astype(np.float32)


def unflatten_mlp(flat: np.ndarray, n_in: int, width: int, n_hidden: int,
                  n_out: int = 1) -> list[np.ndarray]:
    mats, off, fan_in = [], 0, n_in
    for _ in range(n_hidden):
        mats.append(flat[off:off + width * fan_in].reshape(width, fan_in))
        off += width * fan_in
        fan_in = width
    mats.append(flat[off:off + n_out * fan_in].reshape(n_out, fan_in))
    return mats


def mlp_param_count(n_in: int, width: int, n_hidden: int) -> int:
    return n_in * width + (n_hidden - 1) * width * width + width if n_hidden > 0 else n_in


def splitmix_uniform(index: np.ndarray, seed: int, scale: float) -> np.ndarray:
    """Counter-based U(-scale, scale) values of table entries `index`:
    scale * (2u - 1) with u the top 24 bits of SplitMix64 (Steele, Lea & Flood
    2014) of seed + (i + 1) * 0x9E3779B97F4A7C15, rounded once to float32.
    The device fill (nif_fill_uniform) draws the same values."""
    i = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (i + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(40)).astype(np.float32) * np.float32(1.0 / 16777216.0)
    s = np.float32(2.0) * u - np.float32(1.0)
    return (s * np.float32(scale)).astype(np.float32)


class SplitMixTable:
    """Read-only view of a table whose entry e is splitmix_uniform(base + e):
    indexing with an integer array returns float64 values on demand, so a
    1.5G-entry grid initialisation never has to exist on the host."""

    def __init__(self, base: int, seed: int, scale: float):
        self.base, self.seed, self.scale = int(base), int(seed), float(scale)

    def __getitem__(self, idx):
        return splitmix_uniform(np.asarray(idx, dtype=np.int64) + self.base, self.seed,
                                self.scale).astype(np.float64)


class SplitMixGrids:
    """grids[k, g] -> SplitMixTable of object k's grid g in a [n_obj][2][V*F]
    table filled by nif_fill_uniform(seed, scale)."""

    def __init__(self, grid_elems: int, seed: int, scale: float):
        self.n, self.seed, self.scale = int(grid_elems), int(seed), float(scale)

    def __getitem__(self, kg):
        k, g = kg
        return SplitMixTable((int(k) * 2 + int(g)) * self.n, self.seed, self.scale)
