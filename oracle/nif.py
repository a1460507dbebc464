"""CPU oracle for the Neural Intersection Function shadow-ray path (FP64).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and imports nothing from the product package.

What it computes, in the paper's order:

1. Query selection and AABB parameterisation (Sec. 3.1, Eq. 2; Sec. 3.2): a
   (ray, object) pair is queried when the ray segment overlaps the object's
   AABB (FP32 slab test, the same decision the GPU takes in FP32); the pair is
   "inner" when the origin is inside the box, else "outer".  The origin is moved
   to the entry point so aliased rays on one line share an input (Sec. 2,
   Sec. 3.1); entry and exit points are normalised to [0,1]^3 inside the box and
   the direction is mapped to (d+1)/2.  These continuous values are recomputed
   in FP64.
2. Grid encoding (Sec. 3.1, Table 1): trainable latent grids indexed by the
   normalised coordinates with multi-linear interpolation; the multi-resolution
   3D form used here stacks L levels of F features, dense when a level's
   (R+1)^3 vertices fit in T entries, otherwise addressed by the spatial hash of
   Teschner et al. 2003 with the primes used by Mueller et al. 2022.
3. MLP (Sec. 5 'Architecture'): bias-free hidden layers with ReLU (or leaky
   ReLU), a single output logit z; the visible probability is sigmoid(z).
4. Visibility (Sec. 5): a pair is occluded when sigmoid(z) < 0.5, i.e. z < 0;
   a ray is occluded when any of its pairs is.
5. Training (Sec. 4.2, Sec. 5 'Training'): L2 loss on sigmoid(z) against the
   BVH label, back-propagation into the weights and the grid latents, Adam.

Readings where the paper is silent are listed in the design notes; the ones
that shape this file: mean-reduced loss; z >= 0 is visible; R counts cells so
a level has R+1 vertices per axis; s = u*R, i = clamp(floor(s), 0, R-1),
f = s - i; the lookup order of the input vector is
[entry levels | exit levels | direction levels], level-major, F per level.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

HASH_PI = (1, 2654435761, 805459861)


# ---------------------------------------------------------------- step 1
def slab_fp32(rays: np.ndarray, box: np.ndarray):
    """FP32 slab test of ray segments (rays float32 [n,8]) against one box
    (float32 [6]).  Returns (hit bool[n], tin f32[n], tout f32[n], entry f32[n])
    with entry = max_k near_k, tin = max(tmin, entry), tout = min(tmax, min_k far_k);
    an axis with d_k == 0 passes iff lo_k <= o_k <= hi_k."""
    rays = np.asarray(rays, dtype=np.float32)
    box = np.asarray(box, dtype=np.float32)
    n = rays.shape[0]
    entry = np.full(n, -np.inf, dtype=np.float32)
    exitv = np.full(n, np.inf, dtype=np.float32)
    blocked = np.zeros(n, dtype=bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for k in range(3):
            o = rays[:, k]
            d = rays[:, 4 + k]
            par = d == 0
            t0 = (box[k] - o) / d
            t1 = (box[3 + k] - o) / d
            near = np.minimum(t0, t1)
            far = np.maximum(t0, t1)
            entry = np.where(par, entry, np.maximum(entry, near))
            exitv = np.where(par, exitv, np.minimum(exitv, far))
            blocked |= par & ~((box[k] <= o) & (o <= box[3 + k]))
    entry = np.where(blocked, np.float32(np.inf), entry)
    exitv = np.where(blocked, np.float32(-np.inf), exitv)
    tin = np.maximum(rays[:, 3], entry)
    tout = np.minimum(rays[:, 7], exitv)
    return tin <= tout, tin, tout, entry


def queries(rays: np.ndarray, obj_aabb: np.ndarray):
    """All (ray, object) pairs whose segment overlaps the object's AABB.
    Returns (ray_id int64, obj int64, inner bool), sorted by (ray, obj)."""
    rid, oid, inn = [], [], []
    for k in range(obj_aabb.shape[0]):
        hit, _, _, entry = slab_fp32(rays, obj_aabb[k])
        idx = np.nonzero(hit)[0]
        rid.append(idx)
        oid.append(np.full(len(idx), k, dtype=np.int64))
        inn.append(entry[idx] <= rays[idx, 3])
    rid = np.concatenate(rid) if rid else np.zeros(0, np.int64)
    oid = np.concatenate(oid) if oid else np.zeros(0, np.int64)
    inn = np.concatenate(inn) if inn else np.zeros(0, bool)
    order = np.lexsort((oid, rid))
    return rid[order].astype(np.int64), oid[order].astype(np.int64), inn[order]


def entry_exit(rays: np.ndarray, box: np.ndarray):
    """FP64 normalised entry point, exit point and direction of ray segments
    clipped to one box (Eq. 2 with the origin moved onto the box, Sec. 3.1).
    Returns three float64 [n,3] arrays in [0,1]^3.

    A segment that enters (leaves) the box through a face has its entry (exit)
    point on that face, so the coordinate across the face is exactly 0 (the
    low face) or 1 (the high face): it is set so, not left to o + t d, whose
    rounding would put the point a hair off the face.  The face is the slab
    whose near (far) parameter is the segment's t_in (t_out)."""
    r = np.asarray(rays, dtype=np.float64)
    b = np.asarray(box, dtype=np.float64)
    o, d = r[:, 0:3], r[:, 4:7]
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (b[None, 0:3] - o) / d
        t1 = (b[None, 3:6] - o) / d
    par = d == 0
    near = np.where(par, -np.inf, np.minimum(t0, t1))
    far = np.where(par, np.inf, np.maximum(t0, t1))
    tin = np.maximum(r[:, 3], near.max(axis=1))
    tout = np.minimum(r[:, 7], far.min(axis=1))
    lo, ext = b[None, 0:3], (b[3:6] - b[0:3])[None, :]
    p_in = np.clip((o + tin[:, None] * d - lo) / ext, 0.0, 1.0)
    p_out = np.clip((o + tout[:, None] * d - lo) / ext, 0.0, 1.0)
    # moving +: enter through the low face, leave through the high one
    on_in = ~par & (near == tin[:, None])
    on_out = ~par & (far == tout[:, None])
    p_in = np.where(on_in, np.where(d > 0, 0.0, 1.0), p_in)
    p_out = np.where(on_out, np.where(d > 0, 1.0, 0.0), p_out)
    u_dir = (d + 1.0) * 0.5
    return p_in, p_out, u_dir


# ---------------------------------------------------------------- step 2
def level_layout(res, log2_table: int):
    """Per level: (vertex count stored, hashed?) and the level offsets."""
    T = 1 << log2_table
    sizes, hashed = [], []
    for R in res:
        full = (R + 1) ** 3
        hashed.append(full > T)
        sizes.append(T if full > T else full)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return sizes, hashed, offsets


def corner_index(ix, iy, iz, R: int, hashed: bool, log2_table: int):
    """Vertex index of integer lattice coordinates at one level."""
    ix = np.asarray(ix, dtype=np.uint64)
    iy = np.asarray(iy, dtype=np.uint64)
    iz = np.asarray(iz, dtype=np.uint64)
    if not hashed:
        n = np.uint64(R + 1)
        return (ix + n * (iy + n * iz)).astype(np.int64)
    m32 = np.uint64(0xFFFFFFFF)
    h = ((ix * np.uint64(HASH_PI[0])) & m32) ^ ((iy * np.uint64(HASH_PI[1])) & m32) \
        ^ ((iz * np.uint64(HASH_PI[2])) & m32)
    return (h & np.uint64((1 << log2_table) - 1)).astype(np.int64)


def lookup_weights(u: np.ndarray, R: int):
    """Cell and corner weights of points u (float64 [n,3] in [0,1]) at
    resolution R.  Returns (i int64 [n,3], corners list of 8 (offset [3],
    weight float64 [n])) with corner c = cx + 2cy + 4cz."""
    s = u * R
    i = np.clip(np.floor(s), 0, R - 1).astype(np.int64)
    f = s - i
    out = []
    for c in range(8):
        bits = np.array([(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1])
        w = np.ones(u.shape[0])
        for k in range(3):
            w = w * (f[:, k] if bits[k] else (1.0 - f[:, k]))
        out.append((bits, w))
    return i, out


def grid_lookup(table: np.ndarray, u: np.ndarray, res, F: int, log2_table: int,
                want_taps: bool = False):
    """Multi-resolution trilinear lookup into one grid table (float64
    [V*F]) for points u [n,3]. Returns features [n, L*F] (level-major) and,
    if asked, the taps (entry index [n, L, 8], weight [n, L, 8])."""
    sizes, hashed, offsets = level_layout(res, log2_table)
    n = u.shape[0]
    L = len(res)
    feat = np.zeros((n, L * F))
    tap_idx = np.zeros((n, L, 8), dtype=np.int64)
    tap_w = np.zeros((n, L, 8))
    for l, R in enumerate(res):
        i, corners = lookup_weights(u, R)
        for c, (bits, w) in enumerate(corners):
            v = corner_index(i[:, 0] + bits[0], i[:, 1] + bits[1], i[:, 2] + bits[2], R,
                             hashed[l], log2_table)
            e = offsets[l] + v
            tap_idx[:, l, c] = e
            tap_w[:, l, c] = w
            for fi in range(F):
                feat[:, l * F + fi] += w * table[e * F + fi]
    if want_taps:
        return feat, tap_idx, tap_w
    return feat


@dataclass
class Model:
    """Everything the oracle needs about one NIF model.

    grids: float64 [n_obj, 2, V*F]; grid 0 is the position grid (entry and exit
    points), grid 1 the direction grid.  nets: list of per-network weight lists
    [W_1 (w x K), ..., W_H (w x w), w_out (1 x w)].  net_mode: 'class' (net 0 for
    outer pairs, net 1 for inner pairs), 'object' (net = object id) or 'single'.
    """
    res: list
    F: int
    log2_table: int
    obj_aabb: np.ndarray
    grids: np.ndarray
    nets: list
    net_mode: str = "class"
    act: str = "relu"
    slope: float = 0.01

    @property
    def K(self) -> int:
        return 3 * len(self.res) * self.F

    def net_of(self, obj, inner):
        if self.net_mode == "class":
            return np.where(inner, 1, 0)
        if self.net_mode == "object":
            return np.asarray(obj)
        return np.zeros(len(obj), dtype=np.int64)


def encode(m: Model, rays: np.ndarray, ray_id, obj, want_taps: bool = False):
    """Input vectors x [nq, 3*L*F] of the queried pairs (step 2)."""
    nq = len(ray_id)
    x = np.zeros((nq, m.K))
    LF = len(m.res) * m.F
    all_idx = np.zeros((nq, 3, len(m.res), 8), dtype=np.int64)
    all_w = np.zeros((nq, 3, len(m.res), 8))
    for k in np.unique(obj):
        sel = np.nonzero(obj == k)[0]
        p_in, p_out, u_dir = entry_exit(rays[ray_id[sel]], m.obj_aabb[k])
        for j, (u, g) in enumerate(((p_in, 0), (p_out, 0), (u_dir, 1))):
            f, ti, tw = grid_lookup(m.grids[k, g], u, m.res, m.F, m.log2_table, want_taps=True)
            x[sel, j * LF:(j + 1) * LF] = f
            all_idx[sel, j] = ti
            all_w[sel, j] = tw
    if want_taps:
        return x, all_idx, all_w
    return x


# ---------------------------------------------------------------- step 3
def activation(a, act: str, slope: float):
    return np.maximum(a, 0.0) if act == "relu" else np.where(a > 0, a, slope * a)


def activation_grad(a, act: str, slope: float):
    return (a > 0).astype(np.float64) if act == "relu" else np.where(a > 0, 1.0, slope)


def mlp_forward(x: np.ndarray, mats, act: str = "relu", slope: float = 0.01):
    """Bias-free MLP: h_0 = x, a_l = h_{l-1} W_l^T, h_l = act(a_l), z = h_H w_out^T.
    Returns z [n] and the lists of pre-activations a_l and activations h_l."""
    h = np.asarray(x, dtype=np.float64)
    pre, post = [], [h]
    for W in mats[:-1]:
        a = h @ np.asarray(W, dtype=np.float64).T
        h = activation(a, act, slope)
        pre.append(a)
        post.append(h)
    z = (h @ np.asarray(mats[-1], dtype=np.float64).T)[:, 0]
    return z, pre, post


def forward(m: Model, rays, ray_id, obj, inner):
    """Logits z of the queried pairs."""
    x = encode(m, rays, ray_id, obj)
    net = m.net_of(obj, inner)
    z = np.zeros(len(ray_id))
    for g in np.unique(net):
        sel = net == g
        z[sel] = mlp_forward(x[sel], m.nets[g], m.act, m.slope)[0]
    return z


# ---------------------------------------------------------------- step 4
def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def l2_sigmoid_terms(z, y):
    """e = sigmoid(z) - y and sigmoid'(z) = sigmoid(z) (1 - sigmoid(z)) of the
    L2 loss on the sigmoid, with 1 - sigmoid(z) taken as sigmoid(-z) (the
    same number, without the cancellation that loses it for large z); for a
    label y = 1, e = -sigmoid(-z) likewise."""
    z = np.asarray(z, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    sp, sm = sigmoid(z), sigmoid(-z)
    e = np.where(y == 1.0, -sm, sp - y)
    return e, sp * sm


def ray_occlusion(n_rays: int, ray_id, z) -> np.ndarray:
    """Ray occluded (1) when any of its pairs has sigmoid(z) < 0.5 <=> z < 0."""
    occ = np.zeros(n_rays, dtype=bool)
    occ[np.asarray(ray_id)[np.asarray(z) < 0]] = True
    return occ


# ---------------------------------------------------------------- step 5
def loss_and_grads(m: Model, rays, ray_id, obj, inner, label, sparse_grids: bool = False, z_at=None):
    """L = (1/B) sum (sigmoid(z) - y)^2 with y = 1 for visible pairs, and its
    gradients w.r.t. every network weight and every grid latent.
    Returns (L, dnets (same structure as m.nets), dgrids (same shape as m.grids)).
    With sparse_grids the grid gradient is returned as (flat index, value)
    over the latents the pairs tap (flat index ((obj * 2 + grid) * V + vertex)
    * F + feature), for grids too large to hold densely; the arithmetic is
    the same sum of weight x dL/dx per tap.
    z_at (one logit per pair, optional): dL/dz is taken at these logits
    instead of the forward's own, and carried back through the network and
    the grids at the FP64 activations (the chain rule's J^T dL/dz with dL/dz
    from elsewhere); L stays the forward's own.  It checks a backward pass
    apart from the forward whose logits it was given."""
    B = len(ray_id)
    y = np.asarray(label, dtype=np.float64)
    x, tap_idx, tap_w = encode(m, rays, ray_id, obj, want_taps=True)
    net = m.net_of(obj, inner)
    dnets = [[np.zeros_like(np.asarray(W, dtype=np.float64)) for W in ws] for ws in m.nets]
    dx = np.zeros_like(x)
    L = 0.0
    for g in np.unique(net):
        sel = np.nonzero(net == g)[0]
        mats = m.nets[g]
        z, pre, post = mlp_forward(x[sel], mats, m.act, m.slope)
        e, ds = l2_sigmoid_terms(z, y[sel])
        L += float(np.sum(e ** 2)) / B
        if z_at is not None:
            e, ds = l2_sigmoid_terms(np.asarray(z_at, dtype=np.float64)[sel], y[sel])
        dz = (2.0 / B) * e * ds
        dnets[g][-1] += (dz[:, None] * post[-1]).sum(axis=0)[None, :]
        dh = dz[:, None] * np.asarray(mats[-1], dtype=np.float64)
        for li in range(len(mats) - 2, -1, -1):
            da = dh * activation_grad(pre[li], m.act, m.slope)
            dnets[g][li] += da.T @ post[li]
            dh = da @ np.asarray(mats[li], dtype=np.float64)
        dx[sel] = dh
    L_F = len(m.res) * m.F
    obj = np.asarray(obj)
    if sparse_grids:
        GF = int(level_layout(m.res, m.log2_table)[2][-1]) * m.F
        keys, vals = [], []
        for j in range(3):
            g = 0 if j < 2 else 1
            for l in range(len(m.res)):
                for c in range(8):
                    for fi in range(m.F):
                        keys.append((obj * 2 + g) * GF + tap_idx[:, j, l, c] * m.F + fi)
                        vals.append(tap_w[:, j, l, c] * dx[:, j * L_F + l * m.F + fi])
        uk, inv = np.unique(np.concatenate(keys), return_inverse=True)
        acc = np.zeros(len(uk))
        np.add.at(acc, inv, np.concatenate(vals))
        return L, dnets, (uk, acc)
    dgrids = np.zeros_like(m.grids, dtype=np.float64)
    for j in range(3):
        g = 0 if j < 2 else 1
        for l in range(len(m.res)):
            for c in range(8):
                for fi in range(m.F):
                    np.add.at(dgrids, (obj, g, tap_idx[:, j, l, c] * m.F + fi),
                              tap_w[:, j, l, c] * dx[:, j * L_F + l * m.F + fi])
    return L, dnets, dgrids


def adam_step(theta, grad, m1, m2, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam update with bias correction (Kingma & Ba), applied to every
    entry, zero-gradient entries included.  Returns (theta, m1, m2)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)
    m1 = beta1 * np.asarray(m1, dtype=np.float64) + (1.0 - beta1) * g
    m2 = beta2 * np.asarray(m2, dtype=np.float64) + (1.0 - beta2) * g * g
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2
