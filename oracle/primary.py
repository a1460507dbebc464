"""CPU oracle for NIF on primary rays: the network also outputs the shading
normal and the depth at the hit (FP64).

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and imports nothing from the product package.

What it computes (Sec. 3.2, last paragraph: the network may output surface
properties at the hit point besides the occupancy; Sec. 6.1 with Fig. 5: for
primary rays the outputs are the shading normal and the depth from the
camera).  The encoding and hidden layers are those of ``oracle.nif``; the
output layer has O >= 5 rows instead of one.

Readings where the paper is silent (also listed in the design notes):

* Outputs z = [z_0 | z_1 z_2 z_3 | z_4]: z_0 the occupancy logit (the pair is a
  hit iff z_0 < 0, as for shadow rays), (z_1, z_2, z_3) the unit normal of the
  hit surface facing the ray (n . d <= 0), z_4 = delta, the hit's position
  inside the pair's AABB segment: t_hit = t_in + delta (t_out - t_in).  The
  depth is kept relative to the box so that it is a property of the pair, like
  every other input of the network; the depth from the camera follows from
  the slab parameters.
* Loss: L = (1/B) sum_q [(sigmoid(z_0) - y)^2 + (1 - y) sum_{k=1..O-1} (z_k - a_k)^2]
  with y = 1 for a pair whose segment misses the object's triangles (the
  shadow-ray label) and a the pair's normal and delta targets: the regression
  terms count on hit pairs only.
* Resolution per ray (closest hit): among its pairs with z_0 < 0, the smallest
  t = t_in + clamp(delta, 0, 1) (t_out - t_in) computed in FP32 from the FP32
  slab parameters with each operation rounded on its own (difference,
  product, sum), ties to the smallest query index; the ray's normal is
  (z_1, z_2, z_3) normalised.  Rays without a hit pair report t = +inf and
  winner -1.
"""
from __future__ import annotations

import numpy as np

from . import nif as onif


def mlp_outputs(x: np.ndarray, mats, act: str = "relu", slope: float = 0.01):
    """Bias-free MLP with an O-row output layer: h_0 = x, h_l = act(h_{l-1} W_l^T),
    Z = h_H W_out^T.  Returns Z [n, O] and the pre-activations / activations."""
    h = np.asarray(x, dtype=np.float64)
    pre, post = [], [h]
    for W in mats[:-1]:
        a = h @ np.asarray(W, dtype=np.float64).T
        h = onif.activation(a, act, slope)
        pre.append(a)
        post.append(h)
    return h @ np.asarray(mats[-1], dtype=np.float64).T, pre, post


def outputs(m: onif.Model, rays, ray_id, obj, inner):
    """Outputs Z [nq, O] of the queried pairs."""
    x = onif.encode(m, rays, np.asarray(ray_id), np.asarray(obj))
    net = m.net_of(obj, inner)
    O = np.asarray(m.nets[0][-1]).shape[0]
    Z = np.zeros((len(ray_id), O))
    for g in np.unique(net):
        sel = net == g
        Z[sel] = mlp_outputs(x[sel], m.nets[g], m.act, m.slope)[0]
    return Z


def loss_and_grads(m: onif.Model, rays, ray_id, obj, inner, label, aux):
    """The loss above and its gradients w.r.t. every network weight and grid
    latent.  label [B] (1 = miss), aux [B, O-1] targets (read on hit pairs).
    Returns (L, dnets like m.nets, dgrids like m.grids)."""
    B = len(ray_id)
    y = np.asarray(label, dtype=np.float64)
    a = np.asarray(aux, dtype=np.float64)
    obj = np.asarray(obj)
    x, tap_idx, tap_w = onif.encode(m, rays, np.asarray(ray_id), obj, want_taps=True)
    net = m.net_of(obj, inner)
    dnets = [[np.zeros_like(np.asarray(W, dtype=np.float64)) for W in ws] for ws in m.nets]
    dx = np.zeros_like(x)
    L = 0.0
    for g in np.unique(net):
        sel = np.nonzero(net == g)[0]
        mats = m.nets[g]
        Z, pre, post = mlp_outputs(x[sel], mats, m.act, m.slope)
        e, ds = onif.l2_sigmoid_terms(Z[:, 0], y[sel])
        hit = 1.0 - y[sel]
        r = Z[:, 1:] - a[sel]
        L += float(np.sum(e ** 2) + np.sum(hit[:, None] * r * r)) / B
        dZ = np.zeros_like(Z)
        dZ[:, 0] = (2.0 / B) * e * ds
        dZ[:, 1:] = (2.0 / B) * hit[:, None] * r
        dnets[g][-1] += dZ.T @ post[-1]
        dh = dZ @ np.asarray(mats[-1], dtype=np.float64)
        for li in range(len(mats) - 2, -1, -1):
            da = dh * onif.activation_grad(pre[li], m.act, m.slope)
            dnets[g][li] += da.T @ post[li]
            dh = da @ np.asarray(mats[li], dtype=np.float64)
        dx[sel] = dh
    dgrids = np.zeros_like(m.grids, dtype=np.float64)
    LF = len(m.res) * m.F
    for j in range(3):
        gi = 0 if j < 2 else 1
        for l in range(len(m.res)):
            for c in range(8):
                for fi in range(m.F):
                    np.add.at(dgrids, (obj, gi, tap_idx[:, j, l, c] * m.F + fi),
                              tap_w[:, j, l, c] * dx[:, j * LF + l * m.F + fi])
    return L, dnets, dgrids


def hit_parameter(rays, ray_id, obj, obj_aabb, delta):
    """FP32 t = t_in + clamp(delta, 0, 1) (t_out - t_in) of each pair, with
    t_in, t_out from the FP32 slab test and each operation rounded alone."""
    rays = np.asarray(rays, dtype=np.float32)
    rid = np.asarray(ray_id)
    obj = np.asarray(obj)
    t = np.zeros(len(rid), dtype=np.float32)
    dc = np.clip(np.asarray(delta, dtype=np.float32), np.float32(0), np.float32(1))
    for k in np.unique(obj):
        sel = np.nonzero(obj == k)[0]
        _, tin, tout, _ = onif.slab_fp32(rays[rid[sel]], obj_aabb[k])
        span = (tout - tin).astype(np.float32)
        prod = (dc[sel] * span).astype(np.float32)
        t[sel] = (tin + prod).astype(np.float32)
    return t


def resolve(n_rays: int, rays, ray_id, obj, obj_aabb, Z):
    """Closest NIF hit per ray.  Z [nq, >= 5] float32 outputs of the pairs.
    Returns (t float32 [n_rays], normal float64 [n_rays, 3], winner int64
    [n_rays]); rays without a hit pair have t = inf, normal 0, winner -1."""
    Z = np.asarray(Z, dtype=np.float32)
    t_pair = hit_parameter(rays, ray_id, obj, obj_aabb, Z[:, 4])
    t = np.full(n_rays, np.inf, dtype=np.float32)
    win = np.full(n_rays, -1, dtype=np.int64)
    for q in range(len(ray_id)):  # ascending q: a tie keeps the first
        if not Z[q, 0] < 0:
            continue
        r = int(ray_id[q])
        if t_pair[q] < t[r]:
            t[r] = t_pair[q]
            win[r] = q
    nrm = np.zeros((n_rays, 3))
    has = win >= 0
    v = Z[win[has], 1:4].astype(np.float64)
    ln = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[has] = np.where(ln > 0, v / np.where(ln > 0, ln, 1.0), 0.0)
    return t, nrm, win
