"""Pins for the oracle of the paper's own encoding (Sec. 3.1, Sec. 3.2,
Table 1): spherical coordinates, bilinear 2D grids with phi wrap-around, the
1D distance grid, the outer/inner query points and the gradients, each checked
against closed forms or finite differences.  CPU only."""
import numpy as np
import pytest

from oracle import nif as onif
from oracle import spherical as osph
from paper_2306_07191_gb300 import synth

BOX = np.array([-1, -2, -0.5, 3, 2, 1.5], np.float32)  # centre (1, 0, 0.5)


def test_spherical_coordinates_closed_forms():
    v = np.array([[0, 0, 2.0], [0, 0, -1.0], [3.0, 0, 0], [-1.0, 0, 0], [0, 5.0, 0], [0, -1.0, 0],
                  [1.0, 1.0, np.sqrt(2.0)]])
    uv = osph.spherical_uv(v)
    want = np.array([[0, 0.5], [1, 0.5], [0.5, 0.5], [0.5, 1.0], [0.5, 0.75], [0.5, 0.25],
                     [0.25, 0.625]])
    np.testing.assert_allclose(uv, want, atol=1e-15)


def test_spherical_coordinates_are_a_bijection_on_directions():
    rng = np.random.default_rng(3)
    d = synth.unit_vectors(rng, 2000).astype(np.float64)
    uv = osph.spherical_uv(3.7 * d)  # scale does not matter
    th, ph = uv[:, 0] * np.pi, uv[:, 1] * 2 * np.pi - np.pi
    back = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    np.testing.assert_allclose(back, d, atol=1e-12)


def test_outer_point_is_the_entry_point_relative_to_the_centre():
    # along +x through y = 0.3, z = 0.5: enters the face x = -1 at (-1, 0.3, 0.5)
    r = synth.pack_rays(np.array([[-6.0, 0.3, 0.5]]), np.array([[1.0, 0, 0]]), 0.0, np.inf)
    v, d, rr = osph.query_points("outer", r, BOX)
    np.testing.assert_allclose(v[0], [-2.0, 0.3, 0.0], atol=1e-7)
    assert rr is None and np.allclose(d[0], [1, 0, 0])
    uv = osph.spherical_uv(v)[0]
    np.testing.assert_allclose(uv, [0.5, (np.arctan2(0.3, -2.0) + np.pi) / (2 * np.pi)], atol=1e-12)


def test_inner_point_and_normalised_distance():
    # origin at the centre: r' = 0; at a corner (inside by a hair): r' -> 1
    half_diag = 0.5 * np.linalg.norm([4.0, 4.0, 2.0])
    r = synth.pack_rays(np.array([[1.0, 0.0, 0.5], [2.9, 1.9, 1.4]]), np.array([[0, 0, 1.0], [1.0, 0, 0]]),
                        0.0, 10.0)
    v, d, rr = osph.query_points("inner", r, BOX)
    np.testing.assert_allclose(v[0], [0, 0, 0], atol=1e-15)
    assert rr[0] == 0.0
    assert abs(rr[1] - np.linalg.norm([1.9, 1.9, 0.9]) / half_diag) < 1e-6
    # the segment start moves with tmin along d
    r2 = synth.pack_rays(np.array([[1.0, 0.0, 0.5]]), np.array([[0, 0, 1.0]]), 0.25, 10.0)
    v2, _, rr2 = osph.query_points("inner", r2, BOX)
    np.testing.assert_allclose(v2[0], [0, 0, 0.25], atol=1e-15)
    assert abs(rr2[0] - 0.25 / half_diag) < 1e-15


def test_bilinear_lookup_partition_one_hot_and_affine():
    R, N = 6, 2
    rng = np.random.default_rng(5)
    uv = rng.uniform(0, 1, size=(500, 2))
    table = rng.uniform(-1, 1, size=R * R * N)
    _, cells, w = osph.lookup_2d(table, R, N, uv)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-15)
    assert (w >= 0).all()
    # cell centres are one-hot
    i, j = 2, 4
    c = np.array([[(i + 0.5) / R, (j + 0.5) / R]])
    f, _, _ = osph.lookup_2d(table, R, N, c)
    np.testing.assert_allclose(f[0], table[(i * R + j) * N:(i * R + j) * N + N], atol=1e-14)
    # a table affine in the theta index reproduces the affine function of s
    # between the first and last centre (theta is clamped, not wrapped)
    ii, jj = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    aff = np.repeat((3.0 * ii + 0.25).ravel(), N)
    pts = np.stack([rng.uniform(0.5 / R, 1 - 0.5 / R, 200), rng.uniform(0, 1, 200)], 1)
    f, _, _ = osph.lookup_2d(aff, R, N, pts)
    np.testing.assert_allclose(f[:, 0], 3.0 * (pts[:, 0] * R - 0.5) + 0.25, atol=1e-12)


def test_bilinear_lookup_wraps_around_in_phi_and_clamps_theta():
    R, N = 8, 1
    ii, jj = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    table = np.cos(2 * np.pi * jj / R).ravel().astype(np.float64)
    # between the last column centre (R - 1/2)/R and the first one, wrapped
    for v in (0.999, 0.01):
        t = v * R - 0.5
        g = t - np.floor(t)
        j0, j1 = int(np.floor(t)) % R, (int(np.floor(t)) + 1) % R
        f, _, _ = osph.lookup_2d(table, R, N, np.array([[0.5, v]]))
        want = (1 - g) * np.cos(2 * np.pi * j0 / R) + g * np.cos(2 * np.pi * j1 / R)
        assert abs(f[0, 0] - want) < 1e-14
    # theta beyond the first / last centre takes the edge row
    rows = np.repeat(np.arange(R, dtype=np.float64), R)
    f, _, _ = osph.lookup_2d(rows, R, 1, np.array([[0.0, 0.3], [1.0, 0.3], [0.02, 0.7]]))
    np.testing.assert_allclose(f[:, 0], [0.0, R - 1.0, 0.0], atol=1e-15)


def test_linear_1d_lookup_closed_form():
    R1, N1 = 5, 3
    table = np.arange(R1 * N1, dtype=np.float64)  # cell i, feature n -> 3 i + n
    r = np.array([0.0, 0.1, 0.5, 0.75, 1.0])
    f, _, w = osph.lookup_1d(table, R1, N1, r)
    s = np.clip(r * R1 - 0.5, 0, R1 - 1)
    for n in range(N1):
        np.testing.assert_allclose(f[:, n], 3 * s + n, atol=1e-12)
    np.testing.assert_allclose(w.sum(1), 1.0)


def _tiny(kind, seed=0, n_obj=2, R=4, N=2, R1=3, N1=2, width=6, n_hidden=2):
    rng = np.random.default_rng(seed)
    boxes = np.array([[-1, -1, -1, 1, 1, 1], [1.5, -0.5, -0.5, 3.0, 1.0, 0.5]], np.float32)[:n_obj]
    G = 2 * R * R * N + (R1 * N1 if kind == "inner" else 0)
    K = 2 * N + (N1 if kind == "inner" else 0)
    grids = rng.uniform(-1, 1, size=(n_obj, G))
    net = [np.asarray(w, np.float64) for w in synth.mlp_init(rng, K, width, n_hidden)]
    return osph.SphericalModel(kind=kind, R=R, N=N, R1=R1, N1=N1, obj_aabb=boxes, grids=grids, net=net)


def _pairs(kind, m, rng, n=60):
    if kind == "outer":
        k = rng.integers(0, len(m.obj_aabb), n)
        rays = np.concatenate([synth.aimed_rays(rng, 1, m.obj_aabb[i], 5.0) for i in k])
    else:
        k = rng.integers(0, len(m.obj_aabb), n)
        lo, hi = m.obj_aabb[k, :3], m.obj_aabb[k, 3:]
        o = lo + rng.uniform(0.1, 0.9, size=(n, 3)) * (hi - lo)
        rays = synth.pack_rays(o, synth.unit_vectors(rng, n), 1e-3, 10.0)
    return rays, np.arange(n), k


@pytest.mark.parametrize("kind", ["outer", "inner"])
def test_spherical_gradients_match_central_finite_differences(kind):
    m = _tiny(kind, seed=1)
    rng = np.random.default_rng(2)
    rays, rid, obj = _pairs(kind, m, rng)
    label = rng.integers(0, 2, len(rid)).astype(np.float64)
    L0, dnet, dgrids = osph.loss_and_grads(m, rays, rid, obj, label)
    def loss():
        return osph.loss_and_grads(m, rays, rid, obj, label)[0]
    # a sample of weights and every latent the pairs touch
    touched = np.argwhere(np.abs(dgrids) > 0)
    assert len(touched) > 10
    for (k, e) in touched[rng.choice(len(touched), 12, replace=False)]:
        h = 1e-6 * max(1.0, abs(m.grids[k, e]))
        m.grids[k, e] += h
        lp = loss()
        m.grids[k, e] -= 2 * h
        lm = loss()
        m.grids[k, e] += h
        fd = (lp - lm) / (2 * h)
        assert abs(fd - dgrids[k, e]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10, (fd, dgrids[k, e])
    for li in range(len(m.net)):
        W = m.net[li]
        for (a, b) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1)]:
            h = 1e-6 * max(1.0, abs(W[a, b]))
            W[a, b] += h
            lp = loss()
            W[a, b] -= 2 * h
            lm = loss()
            W[a, b] += h
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dnet[li][a, b]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-10


def test_outer_encoding_of_aliased_rays_is_identical():
    """Sec. 3.1: rays on one line from outside the box share an input."""
    m = _tiny("outer", seed=4)
    rng = np.random.default_rng(6)
    rays, rid, obj = _pairs("outer", m, rng, 40)
    moved = rays.copy()
    s = rng.uniform(0.5, 2.0, size=40).astype(np.float32)
    moved[:, 0:3] = rays[:, 0:3] - s[:, None] * rays[:, 4:7]
    np.testing.assert_allclose(osph.encode(m, rays, rid, obj), osph.encode(m, moved, rid, obj), atol=1e-5)


def test_network_sizes_match_the_papers_figures():
    """Sec. 5 'Memory Footprint' gives 18 kB for the outer network and 21 kB
    for the inner one.  With the inputs of this encoding (K = 2N outer,
    2N + N1 inner; Table 1: N = 3, N = 5 and N1 = 3) and the architectures of
    Sec. 5 (2 x 64, 3 x 48), the bias-free weight counts in 4-byte floats come
    to 18.2 kB and 21.1 kB."""
    def count(K, W, H):
        return K * W + (H - 1) * W * W + W
    outer = osph.SphericalModel(kind="outer", R=256, N=3, obj_aabb=BOX[None], grids=np.zeros((1, 1)), net=[])
    inner = osph.SphericalModel(kind="inner", R=128, N=5, R1=128, N1=3, obj_aabb=BOX[None],
                                grids=np.zeros((1, 1)), net=[])
    assert outer.K == 6 and inner.K == 13
    assert round(count(outer.K, 64, 2) * 4 / 1000, 1) == 18.2
    assert round(count(inner.K, 48, 3) * 4 / 1000, 1) == 21.1
