"""Pins for the primary-ray oracle (``oracle/primary.py``: the network also
outputs the normal and the depth at the hit, Sec. 3.2 and Sec. 6.1): the
output layer against the single-output network, the loss against the
shadow-ray loss it reduces to, gradients against central finite differences,
closest-hit resolution on a hand-worked case, and the per-pair closest hit
against the brute-force cast of the object alone.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import nif as onif
from oracle import primary as opr
from paper_2306_07191_gb300 import synth


def _tiny(seed=0, O=5, res=(2, 3), width=6, n_hidden=2, act="leaky"):
    rng = np.random.default_rng(seed)
    boxes = np.array([[-1, -1, -1, 1, 1, 1], [1.5, -0.5, -0.5, 3.0, 1.0, 0.5]], np.float32)
    sizes, hashed, off = onif.level_layout(list(res), 4)
    V = int(off[-1])
    F = 2
    grids = rng.uniform(-1, 1, size=(2, 2, V * F))
    K = 3 * len(res) * F
    mats = [np.asarray(w, np.float64) for w in synth.mlp_init(rng, K, width, n_hidden)]
    mats[-1] = rng.uniform(-0.5, 0.5, size=(O, width))
    m = onif.Model(res=list(res), F=F, log2_table=4, obj_aabb=boxes, grids=grids, nets=[mats],
                   net_mode="single", act=act)
    return m, rng


def _pairs(m, rng, n=40):
    k = rng.integers(0, 2, n)
    rays = np.concatenate([synth.aimed_rays(rng, 1, m.obj_aabb[i], 4.0) for i in k])
    return rays, np.arange(n), k, np.zeros(n, bool)


def test_each_output_is_the_single_output_network_with_that_row():
    m, rng = _tiny()
    rays, rid, obj, inn = _pairs(m, rng)
    Z = opr.outputs(m, rays, rid, obj, inn)
    for o in range(Z.shape[1]):
        m1 = onif.Model(**{**m.__dict__, "nets": [m.nets[0][:-1] + [m.nets[0][-1][o:o + 1]]]})
        np.testing.assert_allclose(Z[:, o], onif.forward(m1, rays, rid, obj, inn), rtol=0, atol=1e-14)


def test_loss_reduces_to_the_shadow_loss_when_every_pair_misses():
    """y = 1 everywhere: the regression terms vanish, so L and every gradient
    equal the shadow-ray loss of the network with output row 0 alone."""
    m, rng = _tiny(seed=2)
    rays, rid, obj, inn = _pairs(m, rng)
    y = np.ones(len(rid))
    aux = rng.normal(size=(len(rid), 4))
    L, dn, dg = opr.loss_and_grads(m, rays, rid, obj, inn, y, aux)
    m1 = onif.Model(**{**m.__dict__, "nets": [m.nets[0][:-1] + [m.nets[0][-1][0:1]]]})
    L1, dn1, dg1 = onif.loss_and_grads(m1, rays, rid, obj, inn, y)
    assert abs(L - L1) < 1e-15
    np.testing.assert_allclose(dg, dg1, rtol=0, atol=1e-15)
    for a, b in zip(dn[0][:-1], dn1[0][:-1]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)
    np.testing.assert_allclose(dn[0][-1][0:1], dn1[0][-1], rtol=0, atol=1e-15)
    assert not dn[0][-1][1:].any()


def test_regression_terms_count_on_hit_pairs_only():
    m, rng = _tiny(seed=3)
    rays, rid, obj, inn = _pairs(m, rng)
    y = (np.arange(len(rid)) % 3 == 0).astype(np.float64)
    aux = rng.normal(size=(len(rid), 4))
    L0 = opr.loss_and_grads(m, rays, rid, obj, inn, y, aux)[0]
    moved = aux.copy()
    moved[y == 1] += 5.0  # targets of miss pairs are never read
    assert opr.loss_and_grads(m, rays, rid, obj, inn, y, moved)[0] == L0
    # one hit pair's delta target moved by h changes L by ((z-a-h)^2 - (z-a)^2)/B
    q = int(np.nonzero(y == 0)[0][0])
    Z = opr.outputs(m, rays, rid, obj, inn)
    h = 0.75
    moved = aux.copy()
    moved[q, 3] += h
    r = Z[q, 4] - aux[q, 3]
    want = L0 + ((r - h) ** 2 - r ** 2) / len(rid)
    assert abs(opr.loss_and_grads(m, rays, rid, obj, inn, y, moved)[0] - want) < 1e-13


def test_gradients_match_central_finite_differences():
    m, rng = _tiny(seed=4)
    rays, rid, obj, inn = _pairs(m, rng, 30)
    y = (rng.uniform(size=len(rid)) < 0.5).astype(np.float64)
    aux = rng.normal(size=(len(rid), 4))

    def loss():
        return opr.loss_and_grads(m, rays, rid, obj, inn, y, aux)[0]

    _, dn, dg = opr.loss_and_grads(m, rays, rid, obj, inn, y, aux)
    touched = np.argwhere(np.abs(dg) > 0)
    assert len(touched) > 10
    for idx in touched[rng.choice(len(touched), 10, replace=False)]:
        idx = tuple(idx)
        h = 1e-6 * max(1.0, abs(m.grids[idx]))
        m.grids[idx] += h
        lp = loss()
        m.grids[idx] -= 2 * h
        lm = loss()
        m.grids[idx] += h
        fd = (lp - lm) / (2 * h)
        assert abs(fd - dg[idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10
    for li, W in enumerate(m.nets[0]):
        for (a, b) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, 1)]:
            h = 1e-6 * max(1.0, abs(W[a, b]))
            W[a, b] += h
            lp = loss()
            W[a, b] -= 2 * h
            lm = loss()
            W[a, b] += h
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dn[0][li][a, b]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (li, a, b)


def test_resolution_of_the_closest_hit_worked_case():
    """Rays along +x from x = -10 through box A = [0,2] (t 10..12) and box B =
    [4,6] (t 14..16): the answers follow from t = t_in + clamp(delta) (t_out - t_in)."""
    boxes = np.array([[0, -1, -1, 2, 1, 1], [4, -1, -1, 6, 1, 1]], np.float32)
    o = np.array([[-10.0, 0, 0]] * 5)
    d = np.array([[1.0, 0, 0]] * 5)
    rays = synth.pack_rays(o, d, 0.0, np.inf)
    #           ray obj  z0    n                 delta
    rows = [(0, 0, +1.0, (1, 0, 0), 0.5),     # ray 0: A misses,
            (0, 1, -1.0, (0, 0, -2), 0.5),    #        B hits at 15, normal (0,0,-1)
            (1, 0, -0.5, (-3, 4, 0), 0.25),   # ray 1: A hits at 10.5
            (1, 1, -2.0, (1, 0, 0), 0.0),     #        B at 14: A wins
            (2, 1, -1.0, (0, 1, 0), 1.7),     # ray 2: delta clamped to 1 -> t_out = 16
            (3, 0, -1.0, (0, 1, 0), 0.5),     # ray 3: the same pair twice at 11;
            (3, 0, -1.0, (0, 0, 1), 0.5),     #        the first query wins the tie
            (4, 1, 0.0, (0, 1, 0), 0.5)]      # ray 4: z0 = 0 is a miss
    rid = np.array([r[0] for r in rows])
    obj = np.array([r[1] for r in rows])
    Z = np.array([[r[2], *r[3], r[4]] for r in rows], np.float32)
    t, nrm, win = opr.resolve(6, rays, rid, obj, boxes, Z)
    np.testing.assert_array_equal(t, np.array([15, 10.5, 16, 11, np.inf, np.inf], np.float32))
    np.testing.assert_array_equal(win, [1, 2, 4, 5, -1, -1])
    np.testing.assert_allclose(nrm[:4], [[0, 0, -1], [-0.6, 0.8, 0], [0, 1, 0], [0, 1, 0]], atol=1e-15)
    assert not nrm[4:].any()


def test_pair_closest_hit_equals_the_brute_force_cast_of_the_object_alone():
    rng = np.random.default_rng(8)
    meshes = [synth.displaced_icosphere(4, rng, centre=c) for c in ((0, 0, 0), (2.5, 0.3, 0), (5, 0, 0.2))]
    sc = synth.build_scene(meshes)
    n = 600
    rays = np.concatenate([synth.aimed_rays(rng, n // 3, sc.obj_aabb[k], 4.0) for k in range(3)])
    rid = np.repeat(np.arange(n), 3)
    obj = np.tile(np.arange(3), n)
    first, count = sc.obj_tri_range[:, 0], sc.obj_tri_range[:, 1]
    t, prim = oracle.brute_pairs_closest(sc.verts, sc.tris, first, count, rays, rid, obj)
    for k in range(3):
        sel = obj == k
        tris_k = sc.tris[first[k]:first[k] + count[k]]
        _, tk, pk = oracle.brute_cast(sc.verts, tris_k, rays)
        np.testing.assert_array_equal(t[sel], tk)
        np.testing.assert_array_equal(prim[sel], np.where(pk >= 0, pk + first[k], -1))
    hit = oracle.brute_pairs(sc.verts, sc.tris, first, count, rays, rid, obj)
    np.testing.assert_array_equal(hit == 1, prim >= 0)
    assert 0.2 < (prim >= 0).mean() < 0.9
