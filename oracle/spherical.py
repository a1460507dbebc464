"""CPU oracle for the paper's own encoding of a NIF query (FP64).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and imports nothing from the product package.

What it computes (Sec. 3.1, Sec. 3.2, Table 1, Sec. 5 'Architecture'):

* Outer pairs (origin outside the object's AABB): the ray is represented by its
  entry point p on the AABB and its direction d.  Both are converted from 3D to
  2D spherical coordinates, p' from p - c (c the box centre; the box is convex,
  so this is a bijection from its surface onto the sphere) and d' from d.  Each
  indexes its own 2D latent grid (R x R cells of N features), bilinearly
  interpolated; x = [v_p | v_d], K = 2N.
* Inner pairs (origin inside): the hit point p is the segment start o + tmin d;
  p' and d' as above, plus the distance r' = |p - c| / (half diagonal) in
  [0, 1] into a 1D grid (R1 cells of N1 features), linearly interpolated;
  x = [v_p | v_d | v_r], K = 2N + N1.
* One network per class (the paper: outer 2 x 64, inner 3 x 48 hidden units,
  leaky ReLU), bias-free, one output logit; visible iff z >= 0.

Readings where the paper is silent (also listed in the design notes):

* Spherical coordinates: theta = atan2(sqrt(x^2 + y^2), z) in [0, pi] and
  phi = atan2(y, x) in [-pi, pi]; (u, v) = (theta / pi, (phi + pi) / (2 pi)).
  (atan2 for theta stays well conditioned at the poles, where acos is not.)
* A grid of resolution R has R cells per dimension, each holding a latent at
  its centre; bilinear interpolation between the four nearest centres:
  s = u R - 1/2, i = clamp(floor(s), 0, R - 2), f = clamp(s - i, 0, 1) along
  theta (values beyond the first/last centre are the edge values), and along
  phi j0 = floor(s) mod R, j1 = (j0 + 1) mod R, g = s - floor(s) (phi wraps
  around).  The 1D grid interpolates like the theta axis.
* Table layout per object: [position R x R x N | direction R x R x N |
  distance R1 x N1 (inner only)], cell (i, j) at (i R + j) N.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import nif as onif


@dataclass
class SphericalModel:
    """One class network with its per-object grids.

    kind: 'outer' or 'inner'; R, N: the 2D grids' resolution and latent size;
    R1, N1: the inner 1D grid's; grids: float64 [n_obj, G] in the layout
    above; net: [W_1 (w x K), ..., W_H (w x w), w_out (1 x w)]."""
    kind: str
    R: int
    N: int
    obj_aabb: np.ndarray
    grids: np.ndarray
    net: list
    R1: int = 0
    N1: int = 0
    act: str = "leaky"
    slope: float = 0.01

    @property
    def K(self) -> int:
        return 2 * self.N + (self.N1 if self.kind == "inner" else 0)

    @property
    def table_sizes(self):
        """Elements of the position, direction and distance tables."""
        t2 = self.R * self.R * self.N
        return t2, t2, (self.R1 * self.N1 if self.kind == "inner" else 0)

    @property
    def G(self) -> int:
        return sum(self.table_sizes)


def spherical_uv(v: np.ndarray) -> np.ndarray:
    """(theta / pi, (phi + pi) / (2 pi)) of vectors v [n, 3] (float64)."""
    v = np.asarray(v, dtype=np.float64)
    theta = np.arctan2(np.hypot(v[:, 0], v[:, 1]), v[:, 2])
    phi = np.arctan2(v[:, 1], v[:, 0])
    return np.stack([theta / np.pi, (phi + np.pi) / (2.0 * np.pi)], axis=1)


def query_points(kind: str, rays: np.ndarray, box: np.ndarray):
    """p - c (float64 [n, 3]) for the pairs of one box, the direction, and for
    inner pairs r' = |p - c| / half diagonal (else None)."""
    r = np.asarray(rays, dtype=np.float64)
    b = np.asarray(box, dtype=np.float64)
    lo, hi = b[0:3], b[3:6]
    c, ext = 0.5 * (lo + hi), hi - lo
    d = r[:, 4:7]
    if kind == "outer":
        p_in, _, _ = onif.entry_exit(rays, box)  # normalised, on its face
        v = (p_in - 0.5) * ext[None, :]
        return v, d, None
    p = r[:, 0:3] + r[:, 3:4] * d
    v = p - c[None, :]
    rr = np.linalg.norm(v, axis=1) / (0.5 * np.linalg.norm(ext))
    return v, d, np.clip(rr, 0.0, 1.0)


def lookup_2d(table: np.ndarray, R: int, N: int, uv: np.ndarray):
    """Bilinear lookup of points uv [n, 2] in one R x R x N table.  Returns
    (features [n, N], cell indices [n, 4], weights [n, 4])."""
    s = uv[:, 0] * R - 0.5
    i0 = np.clip(np.floor(s), 0, R - 2).astype(np.int64)
    f = np.clip(s - i0, 0.0, 1.0)
    t = uv[:, 1] * R - 0.5
    jf = np.floor(t)
    g = t - jf
    j0 = np.mod(jf.astype(np.int64), R)
    j1 = np.mod(j0 + 1, R)
    cells = np.stack([i0 * R + j0, (i0 + 1) * R + j0, i0 * R + j1, (i0 + 1) * R + j1], axis=1)
    w = np.stack([(1 - f) * (1 - g), f * (1 - g), (1 - f) * g, f * g], axis=1)
    feat = np.zeros((uv.shape[0], N))
    for k in range(4):
        for n in range(N):
            feat[:, n] += w[:, k] * table[cells[:, k] * N + n]
    return feat, cells, w


def lookup_1d(table: np.ndarray, R1: int, N1: int, r: np.ndarray):
    """Linear lookup of r [n] in [0, 1] in one R1 x N1 table.  Returns
    (features [n, N1], cell indices [n, 2], weights [n, 2])."""
    s = r * R1 - 0.5
    i0 = np.clip(np.floor(s), 0, R1 - 2).astype(np.int64)
    f = np.clip(s - i0, 0.0, 1.0)
    cells = np.stack([i0, i0 + 1], axis=1)
    w = np.stack([1 - f, f], axis=1)
    feat = np.zeros((r.shape[0], N1))
    for k in range(2):
        for n in range(N1):
            feat[:, n] += w[:, k] * table[cells[:, k] * N1 + n]
    return feat, cells, w


def encode(m: SphericalModel, rays: np.ndarray, ray_id, obj, want_taps: bool = False):
    """Input vectors x [nq, K] of the queried pairs.  With want_taps, also the
    taps: a list of (element offset [nq, T] into the object's grid block,
    weight [nq, T], column of x) per latent component."""
    nq = len(ray_id)
    x = np.zeros((nq, m.K))
    t_pos, t_dir, _ = m.table_sizes
    taps = []  # (sel, element index [n, T], weight [n, T], x column)
    for k in np.unique(obj):
        sel = np.nonzero(np.asarray(obj) == k)[0]
        v, d, rr = query_points(m.kind, rays[np.asarray(ray_id)[sel]], m.obj_aabb[k])
        blk = m.grids[k]
        fp, cp, wp = lookup_2d(blk[:t_pos], m.R, m.N, spherical_uv(v))
        fd, cd, wd = lookup_2d(blk[t_pos:t_pos + t_dir], m.R, m.N, spherical_uv(d))
        x[sel, 0:m.N] = fp
        x[sel, m.N:2 * m.N] = fd
        for n in range(m.N):
            taps.append((sel, cp * m.N + n, wp, n))
            taps.append((sel, t_pos + cd * m.N + n, wd, m.N + n))
        if m.kind == "inner":
            fr, cr, wr = lookup_1d(blk[t_pos + t_dir:], m.R1, m.N1, rr)
            x[sel, 2 * m.N:] = fr
            for n in range(m.N1):
                taps.append((sel, t_pos + t_dir + cr * m.N1 + n, wr, 2 * m.N + n))
    if want_taps:
        return x, taps
    return x


def forward(m: SphericalModel, rays, ray_id, obj):
    """Logits z of the queried pairs."""
    return onif.mlp_forward(encode(m, rays, ray_id, obj), m.net, m.act, m.slope)[0]


def loss_and_grads(m: SphericalModel, rays, ray_id, obj, label):
    """L = (1/B) sum (sigmoid(z) - y)^2 and its gradients w.r.t. the network
    weights and every grid latent (same structures as m.net and m.grids)."""
    B = len(ray_id)
    y = np.asarray(label, dtype=np.float64)
    x, taps = encode(m, rays, ray_id, obj, want_taps=True)
    z, pre, post = onif.mlp_forward(x, m.net, m.act, m.slope)
    s = onif.sigmoid(z)
    L = float(np.sum((s - y) ** 2)) / B
    dz = (2.0 / B) * (s - y) * s * (1.0 - s)
    dnet = [np.zeros_like(np.asarray(W, dtype=np.float64)) for W in m.net]
    dnet[-1] += (dz[:, None] * post[-1]).sum(axis=0)[None, :]
    dh = dz[:, None] * np.asarray(m.net[-1], dtype=np.float64)
    for li in range(len(m.net) - 2, -1, -1):
        da = dh * onif.activation_grad(pre[li], m.act, m.slope)
        dnet[li] += da.T @ post[li]
        dh = da @ np.asarray(m.net[li], dtype=np.float64)
    dgrids = np.zeros_like(m.grids, dtype=np.float64)
    obj = np.asarray(obj)
    for sel, idx, w, col in taps:
        for t in range(idx.shape[1]):
            np.add.at(dgrids, (obj[sel], idx[:, t]), w[:, t] * dh[sel, col])
    return L, dnet, dgrids
