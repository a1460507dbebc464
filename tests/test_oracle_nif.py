"""Pins for the FP64 NIF oracle: AABB parameterisation, grid encoding, MLP,
loss gradients and Adam, each checked against closed forms, hand-derived
values, invariants or finite differences rather than against itself.  CPU only."""
import os

import numpy as np
import pytest

from oracle import nif as onif
from paper_2306_07191_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BOX = np.array([-1, -2, -0.5, 3, 2, 1.5], np.float32)


def _model(res, F, log2_table, n_obj=1, n_hidden=2, width=8, seed=0, net_mode="single",
           n_nets=1, act="relu", aabb=None):
    rng = np.random.default_rng(seed)
    sizes, _, off = onif.level_layout(res, log2_table)
    V = int(off[-1])
    grids = rng.uniform(-1, 1, size=(n_obj, 2, V * F))
    K = 3 * len(res) * F
    nets = [[np.asarray(w, np.float64) for w in synth.mlp_init(rng, K, width, n_hidden)]
            for _ in range(n_nets)]
    if aabb is None:
        aabb = np.tile(BOX, (n_obj, 1))
    return onif.Model(res=list(res), F=F, log2_table=log2_table, obj_aabb=aabb, grids=grids,
                      nets=nets, net_mode=net_mode, act=act)


# ------------------------------------------------------------ parameterisation
def test_entry_exit_closed_forms():
    # ray along +x through the box centre (1, 0, 0.5): entry face x = -1, exit x = 3
    r = synth.pack_rays(np.array([[-5.0, 0.0, 0.5]]), np.array([[1.0, 0, 0]]), 0.0, np.inf)
    p_in, p_out, u_dir = onif.entry_exit(r, BOX)
    np.testing.assert_allclose(p_in[0], [0.0, 0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(p_out[0], [1.0, 0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(u_dir[0], [1.0, 0.5, 0.5], atol=1e-15)
    # origin inside (inner pair): entry is the origin itself, exit at tmax
    r = synth.pack_rays(np.array([[0.0, 0.0, 0.0]]), np.array([[0.0, -1.0, 0]]), 0.0, 1.0)
    p_in, p_out, u_dir = onif.entry_exit(r, BOX)
    np.testing.assert_allclose(p_in[0], [0.25, 0.5, 0.25], atol=1e-7)
    np.testing.assert_allclose(p_out[0], [0.25, 0.25, 0.25], atol=1e-7)
    np.testing.assert_allclose(u_dir[0], [0.5, 0.0, 0.5], atol=1e-15)


def test_entry_and_exit_points_lie_exactly_on_their_faces():
    """Eq. 2: the entry point of an outside origin is on the face it enters,
    the exit point on the face it leaves (the coordinate across the face is
    exactly 0 or 1, low or high face by the direction's sign); the other two
    coordinates are the closed form o + t d for t from that face's plane."""
    box = np.array([0.0, 0.0, 0.0, 1.0, 2.0, 4.0], np.float32)
    o = np.array([[-0.3, 0.37, 0.91], [1.7, 1.13, 2.2], [0.41, 0.5, 5.3]])
    d = np.array([[0.93, 0.27, 0.25], [-0.8, 0.1, -0.59], [0.05, 0.11, -0.99]])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = synth.pack_rays(o, d, 0.0, np.inf)
    p_in, p_out, _ = onif.entry_exit(r, box)
    rf = r.astype(np.float64)
    o, d = rf[:, 0:3], rf[:, 4:7]
    lo, ext = box[:3].astype(np.float64), (box[3:] - box[:3]).astype(np.float64)
    # slab parameters by hand: ray 0 enters x = 0 (t 0.32/|d|) before y and z
    # and leaves x = 1 (t 1.40) before y = 2 (6.0) and z = 4 (12.4); ray 1
    # enters x = 1 (0.875) and leaves x = 0 (2.125) before z = 0 (3.73); ray 2
    # enters z = 4 (1.31) and leaves z = 0 (5.35) before x = 1 (11.8)
    faces_in = [(0, 0.0, 0.0), (0, 1.0, 1.0), (2, 4.0, 1.0)]
    faces_out = [(0, 1.0, 1.0), (0, 0.0, 0.0), (2, 0.0, 0.0)]
    for i, ((ki, pi, ui), (ko, po, uo)) in enumerate(zip(faces_in, faces_out)):
        assert p_in[i, ki] == ui and p_out[i, ko] == uo
        t_in = (pi - o[i, ki]) / d[i, ki]
        t_out = (po - o[i, ko]) / d[i, ko]
        for k in range(3):
            if k != ki:
                assert abs(p_in[i, k] - (o[i, k] + t_in * d[i, k] - lo[k]) / ext[k]) < 1e-12
            if k != ko:
                assert abs(p_out[i, k] - (o[i, k] + t_out * d[i, k] - lo[k]) / ext[k]) < 1e-12
    # every outer pair of random aimed rays has an entry coordinate of exactly 0 or 1
    rays = synth.aimed_rays(np.random.default_rng(8), 500, BOX, 6.0)
    p_in, p_out, _ = onif.entry_exit(rays, BOX)
    assert np.all(np.any((p_in == 0.0) | (p_in == 1.0), axis=1))
    assert np.all(np.any((p_out == 0.0) | (p_out == 1.0), axis=1))


def test_aliased_rays_share_an_input():
    """Sec. 2 / Sec. 3.1: moving an outside origin along its direction leaves
    the encoder input unchanged."""
    rng = np.random.default_rng(4)
    m = _model([2, 4, 7], 2, 19, seed=1)
    rays = synth.aimed_rays(rng, 400, BOX, 6.0)
    moved = rays.copy()
    s = rng.uniform(0.5, 3.0, size=400).astype(np.float32)
    moved[:, 0:3] = rays[:, 0:3] - s[:, None] * rays[:, 4:7]
    rid = np.arange(400)
    obj = np.zeros(400, np.int64)
    x0 = onif.encode(m, rays, rid, obj)
    x1 = onif.encode(m, moved, rid, obj)
    np.testing.assert_allclose(x0, x1, atol=1e-5)


def test_queries_and_inner_classification():
    boxes = np.array([[-1, -1, -1, 1, 1, 1], [2, -1, -1, 4, 1, 1]], np.float32)
    o = np.array([[-3, 0, 0], [0, 0, 0], [3, 0, 0], [0, 5, 0]], np.float64)
    d = np.array([[1, 0, 0], [1, 0, 0], [-1, 0, 0], [1, 0, 0]], np.float64)
    rays = synth.pack_rays(o, d, 0.001, np.inf)
    rid, obj, inner = onif.queries(rays, boxes)
    got = set(zip(rid.tolist(), obj.tolist(), inner.tolist()))
    assert got == {(0, 0, False), (0, 1, False), (1, 0, True), (1, 1, False),
                   (2, 1, True), (2, 0, False)}


# ------------------------------------------------------------ grid encoding
def test_corner_weights_partition_of_unity_and_one_hot():
    rng = np.random.default_rng(0)
    u = rng.uniform(size=(500, 3))
    for R in (1, 3, 16, 1024):
        _, corners = onif.lookup_weights(u, R)
        w = np.stack([c[1] for c in corners])
        np.testing.assert_allclose(w.sum(axis=0), 1.0, atol=1e-14)
        assert (w >= 0).all()
    # at lattice vertices exactly one weight is 1
    R = 4
    ijk = rng.integers(0, R + 1, size=(50, 3))
    i, corners = onif.lookup_weights(ijk / R, R)
    w = np.stack([c[1] for c in corners])
    assert np.all(np.sort(w, axis=0)[-1] == 1.0) and np.all(np.sort(w, axis=0)[:-1] == 0.0)
    # u = 1 lands in the last cell with f = 1
    i, corners = onif.lookup_weights(np.ones((1, 3)), R)
    assert (i == R - 1).all()
    assert corners[7][1][0] == 1.0


def test_trilinear_textbook_form_single_level_r1():
    """R = 1, one level: the lookup equals nested linear interpolation of the
    eight corner values of the unit cube."""
    rng = np.random.default_rng(2)
    c = rng.normal(size=8)  # c[x + 2y + 4z]
    table = c.copy()
    u = rng.uniform(size=(200, 3))
    got = onif.grid_lookup(table, u, [1], 1, 19)[:, 0]
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    lerp = lambda a, b, t: a + (b - a) * t
    c00 = lerp(c[0], c[1], x)
    c10 = lerp(c[2], c[3], x)
    c01 = lerp(c[4], c[5], x)
    c11 = lerp(c[6], c[7], x)
    want = lerp(lerp(c00, c10, y), lerp(c01, c11, y), z)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_affine_table_is_reproduced_exactly_on_dense_levels():
    """A dense table filled with a.(vertex/R) + b interpolates to a.u + b."""
    res = [3, 5, 16, 64]
    F = 2
    sizes, hashed, off = onif.level_layout(res, 19)
    assert not any(hashed)
    a = np.array([[0.3, -1.2, 2.0], [1.5, 0.25, -0.75]])
    b = np.array([0.1, -0.4])
    table = np.zeros(int(off[-1]) * F)
    for l, R in enumerate(res):
        n = R + 1
        iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        idx = onif.corner_index(ix.ravel(), iy.ravel(), iz.ravel(), R, False, 19)
        pos = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) / R
        for f in range(F):
            table[(off[l] + idx) * F + f] = pos @ a[f] + b[f]
    u = np.random.default_rng(3).uniform(size=(300, 3))
    u[:5] = [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.5, 1, 0], [0.999999, 0.000001, 1]]
    feat = onif.grid_lookup(table, u, res, F, 19)
    for l in range(len(res)):
        for f in range(F):
            np.testing.assert_allclose(feat[:, l * F + f], u @ a[f] + b[f], atol=1e-12)


def test_dense_index_is_x_fastest():
    # R = 2: vertex (ix, iy, iz) -> ix + 3 iy + 9 iz
    assert onif.corner_index(1, 0, 0, 2, False, 19) == 1
    assert onif.corner_index(0, 1, 0, 2, False, 19) == 3
    assert onif.corner_index(0, 0, 1, 2, False, 19) == 9
    assert onif.corner_index(2, 2, 2, 2, False, 19) == 26


def test_spatial_hash_golden_values():
    rows = []
    with open(os.path.join(GOLDEN, "spatial_hash.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    for ix, iy, iz, h in rows:
        for log2 in (32, 19, 4):
            want = h & ((1 << log2) - 1) if log2 < 32 else h
            got = onif.corner_index(ix, iy, iz, 10 ** 6, True, min(log2, 32))
            assert int(got) == want


def test_hashed_level_lookup_matches_brute_force_dictionary():
    """A 3-cell level (64 vertices) hashed into T = 16 entries: build the table
    by walking every vertex and remembering which entry it maps to, then
    check interpolation through that dictionary."""
    R, log2 = 3, 4
    sizes, hashed, off = onif.level_layout([R], log2)
    assert hashed == [True] and sizes == [16]
    rng = np.random.default_rng(8)
    table = rng.normal(size=16)
    vertex_value = {}
    for ix in range(R + 1):
        for iy in range(R + 1):
            for iz in range(R + 1):
                e = int(onif.corner_index(ix, iy, iz, R, True, log2))
                vertex_value[(ix, iy, iz)] = table[e]
    # collisions exist: 64 vertices share 16 entries
    assert len(set(vertex_value.values())) <= 16
    u = rng.uniform(size=(100, 3))
    got = onif.grid_lookup(table, u, [R], 1, log2)[:, 0]
    for n in range(100):
        s = u[n] * R
        i = np.minimum(np.floor(s).astype(int), R - 1)
        f = s - i
        acc = 0.0
        for cx in (0, 1):
            for cy in (0, 1):
                for cz in (0, 1):
                    w = (f[0] if cx else 1 - f[0]) * (f[1] if cy else 1 - f[1]) * (f[2] if cz else 1 - f[2])
                    acc += w * vertex_value[(i[0] + cx, i[1] + cy, i[2] + cz)]
        assert abs(acc - got[n]) < 1e-12


def test_level_offsets_and_input_order():
    """Each level filled with its own constant, the direction grid with another:
    x must read [entry levels | exit levels | direction levels]."""
    res = [2, 3, 70]
    F = 2
    sizes, hashed, off = onif.level_layout(res, 12)
    assert hashed == [False, False, True] and sizes == [27, 64, 4096]
    m = _model(res, F, 12)
    for l in range(3):
        m.grids[0, 0, off[l] * F:off[l + 1] * F] = 10 * (l + 1) + np.tile([0, 1], sizes[l])
        m.grids[0, 1, off[l] * F:off[l + 1] * F] = -(10 * (l + 1)) - np.tile([0, 1], sizes[l])
    rays = synth.aimed_rays(np.random.default_rng(1), 10, BOX, 6.0)
    x = onif.encode(m, rays, np.arange(10), np.zeros(10, np.int64))
    level_vals = [10, 11, 20, 21, 30, 31]
    np.testing.assert_allclose(x[:, 0:6], np.tile(level_vals, (10, 1)), atol=1e-12)
    np.testing.assert_allclose(x[:, 6:12], np.tile(level_vals, (10, 1)), atol=1e-12)
    np.testing.assert_allclose(x[:, 12:18], -np.tile(level_vals, (10, 1)), atol=1e-12)


def test_entry_and_exit_use_their_own_points():
    """With an affine position table, the entry block equals a.u_in + b and the
    exit block a.u_out + b for the closed-form entry/exit of an axis ray."""
    res = [4]
    m = _model(res, 1, 19)
    R = 4
    n = R + 1
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    idx = onif.corner_index(ix.ravel(), iy.ravel(), iz.ravel(), R, False, 19)
    m.grids[0, 0, idx] = ix.ravel() / R + 2 * iy.ravel() / R + 4 * iz.ravel() / R
    r = synth.pack_rays(np.array([[-5.0, 0.0, 0.5]]), np.array([[1.0, 0, 0]]), 0.0, np.inf)
    x = onif.encode(m, r, np.array([0]), np.array([0]))
    assert abs(x[0, 0] - (0 + 2 * 0.5 + 4 * 0.5)) < 1e-12
    assert abs(x[0, 1] - (1 + 2 * 0.5 + 4 * 0.5)) < 1e-12


# ------------------------------------------------------------ MLP
def test_mlp_without_hidden_layers_is_a_dot_product():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(20, 6))
    w = rng.normal(size=(1, 6))
    z, _, _ = onif.mlp_forward(x, [w])
    np.testing.assert_allclose(z, [sum(x[i, k] * w[0, k] for k in range(6)) for i in range(20)],
                               atol=1e-13)


def test_relu_of_positive_path_collapses_to_linear_map():
    """Positive inputs and weights keep every unit active: z = x W1^T W2^T w^T."""
    rng = np.random.default_rng(1)
    x = rng.uniform(0.1, 1, size=(10, 4))
    W1 = rng.uniform(0.1, 1, size=(5, 4))
    W2 = rng.uniform(0.1, 1, size=(3, 5))
    w = rng.uniform(0.1, 1, size=(1, 3))
    z, _, _ = onif.mlp_forward(x, [W1, W2, w])
    prod = np.einsum("ik,jk->ij", np.einsum("ik,jk->ij", x, W1), W2)
    np.testing.assert_allclose(z, prod @ w[0], rtol=1e-13)


def test_relu_splits_positive_and_negative_parts():
    """W1 = [I; -I], w = [1 ... 1, -1 ... -1]: relu(x) - relu(-x) = x, so z = sum x;
    leaky ReLU with slope s gives (1 + s) sum x."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(30, 3))
    W1 = np.vstack([np.eye(3), -np.eye(3)])
    w = np.array([[1, 1, 1, -1, -1, -1.0]])
    z, _, _ = onif.mlp_forward(x, [W1, w], act="relu")
    np.testing.assert_allclose(z, x.sum(axis=1), atol=1e-14)
    z, _, _ = onif.mlp_forward(x, [W1, w], act="leaky", slope=0.01)
    np.testing.assert_allclose(z, 1.01 * x.sum(axis=1), atol=1e-13)


def test_visibility_threshold_tie_is_visible():
    occ = onif.ray_occlusion(4, np.array([0, 1, 2, 2]), np.array([0.0, -1e-300, 3.0, -2.0]))
    assert occ.tolist() == [False, True, True, False]
    assert onif.sigmoid(np.array([0.0]))[0] == 0.5


# ------------------------------------------------------------ gradients
def _loss_only(m, rays, rid, obj, inner, y):
    x = onif.encode(m, rays, rid, obj)
    net = m.net_of(obj, inner)
    z = np.zeros(len(rid))
    for g in np.unique(net):
        z[net == g] = onif.mlp_forward(x[net == g], m.nets[g], m.act, m.slope)[0]
    return float(np.mean((onif.sigmoid(z) - y) ** 2))


@pytest.mark.parametrize("act,n_hidden,res", [("relu", 1, [2]), ("relu", 2, [2, 4]),
                                               ("leaky", 2, [3, 4])])
def test_gradients_match_central_finite_differences(act, n_hidden, res):
    rng = np.random.default_rng(12)
    boxes = np.array([[-1, -1, -1, 1, 1, 1], [0.5, -1, -1, 2.5, 1, 1]], np.float32)
    m = _model(res, 2, 19, n_obj=2, n_hidden=n_hidden, width=6, seed=3, net_mode="class",
               n_nets=2, act=act, aabb=boxes)
    for nets in m.nets:
        for W in nets:
            W *= 3.0  # larger logits so sigmoid' is not tiny
    m.grids *= 2.0
    o = rng.uniform(-1.5, 3.0, size=(90, 3))
    d = synth.unit_vectors(rng, 90)
    rays = synth.pack_rays(o, d, 0.001, np.inf)
    rid, obj, inner = onif.queries(rays, boxes)
    assert len(rid) > 20 and inner.any() and (~inner).any()
    y = rng.integers(0, 2, size=len(rid)).astype(np.float64)
    L, dnets, dgrids = onif.loss_and_grads(m, rays, rid, obj, inner, y)
    assert abs(L - _loss_only(m, rays, rid, obj, inner, y)) < 1e-14
    # the sparse form holds the same sums at the tapped latents, nothing else
    _, _, (keys, vals) = onif.loss_and_grads(m, rays, rid, obj, inner, y, sparse_grids=True)
    dense = np.zeros(dgrids.size)
    dense[keys] = vals
    np.testing.assert_allclose(dense, dgrids.reshape(-1), rtol=1e-13, atol=1e-16)
    assert np.all(dgrids.reshape(-1)[np.setdiff1d(np.arange(dgrids.size), keys)] == 0)

    def fd(get, set_):
        th = get()
        h = 1e-6 * max(1.0, abs(th))
        set_(th + h)
        lp = _loss_only(m, rays, rid, obj, inner, y)
        set_(th - h)
        lm = _loss_only(m, rays, rid, obj, inner, y)
        set_(th)
        return (lp - lm) / (2 * h)

    checked = 0
    for g in range(2):
        for li, W in enumerate(m.nets[g]):
            for idx in list(np.ndindex(W.shape))[::3]:
                num = fd(lambda: W[idx], lambda v: W.__setitem__(idx, v))
                ana = dnets[g][li][idx]
                assert abs(num - ana) <= 1e-6 * max(abs(num), abs(ana)) + 1e-10, (g, li, idx)
                checked += 1
    flat = m.grids.reshape(-1)
    dflat = dgrids.reshape(-1)
    touched = np.nonzero(dflat)[0]
    assert len(touched) > 20
    for e in touched[::max(1, len(touched) // 150)]:
        num = fd(lambda: flat[e], lambda v: flat.__setitem__(e, v))
        assert abs(num - dflat[e]) <= 1e-6 * max(abs(num), abs(dflat[e])) + 1e-10, e
        checked += 1
    # untouched latents have exactly zero gradient
    assert checked > 100


def test_single_layer_gradient_closed_form():
    """No hidden layer: dL/dw = (2/B) sum (s - y) s (1 - s) x."""
    rng = np.random.default_rng(5)
    res = [3]
    m = _model(res, 2, 19, n_hidden=0, seed=9)
    m.nets[0][0] = rng.normal(size=(1, m.K)) * 5
    rays = synth.aimed_rays(rng, 30, BOX, 6.0)
    rid = np.arange(30)
    obj = np.zeros(30, np.int64)
    inner = np.zeros(30, bool)
    y = rng.integers(0, 2, size=30).astype(float)
    L, dnets, _ = onif.loss_and_grads(m, rays, rid, obj, inner, y)
    x = onif.encode(m, rays, rid, obj)
    z = x @ m.nets[0][0][0]
    s = 1 / (1 + np.exp(-z))
    want = (2 / 30) * ((s - y) * s * (1 - s)) @ x
    np.testing.assert_allclose(dnets[0][0][0], want, rtol=1e-12)


def test_sigmoid_loss_terms_against_50_digit_arithmetic():
    """sigmoid(z) - y and sigmoid(z)(1 - sigmoid(z)) of the L2 loss keep full
    relative precision for confident logits (|z| up to 40, where forming
    1 - sigmoid(z) by subtraction loses every digit), checked against the
    same formulas in 50-digit arithmetic; a single-layer weight gradient at
    such logits likewise."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    zs = np.array([-40.0, -25.0, -5.0, -0.5, 0.0, 0.5, 5.0, 25.0, 40.0])
    for y in (0.0, 1.0):
        e, ds = onif.l2_sigmoid_terms(zs, np.full(zs.shape, y))
        for k, z in enumerate(zs):
            s = 1 / (1 + mp.exp(-mp.mpf(z)))
            e_want, ds_want = s - y, s * (1 - s)
            assert abs(e[k] - float(e_want)) <= 1e-14 * abs(float(e_want)) + 1e-300, (z, y)
            assert abs(ds[k] - float(ds_want)) <= 1e-14 * float(ds_want), (z, y)
    rng = np.random.default_rng(31)
    m = _model([3], 2, 19, n_hidden=0, seed=9)
    m.nets[0][0] = rng.normal(size=(1, m.K)) * 60
    rays = synth.aimed_rays(rng, 12, BOX, 6.0)
    rid, obj, inner = np.arange(12), np.zeros(12, np.int64), np.zeros(12, bool)
    y = np.ones(12)
    _, dnets, _ = onif.loss_and_grads(m, rays, rid, obj, inner, y)
    x = onif.encode(m, rays, rid, obj)
    z = x @ m.nets[0][0][0]
    assert np.abs(z).max() > 20
    dz = [2 / mp.mpf(12) * (1 / (1 + mp.exp(-mp.mpf(v))) - 1) * (1 / (1 + mp.exp(-mp.mpf(v))))
          * (1 - 1 / (1 + mp.exp(-mp.mpf(v)))) for v in z]
    want = np.array([float(sum(dz[q] * mp.mpf(x[q, k]) for q in range(12))) for k in range(m.K)])
    np.testing.assert_allclose(dnets[0][0][0], want, rtol=1e-12, atol=1e-300)


def test_gradient_at_given_logits_closed_form_and_linearity():
    """dL/dz taken at given logits z_at: with no hidden layer the weight
    gradient is (2/B) sum (s(z_at) - y) s(z_at) (1 - s(z_at)) x, written out
    here; with hidden layers each pair's contribution scales with its dL/dz
    (the backward is linear in it), so one pair's gradient at z_at is its
    gradient at its own logit times dL/dz(z_at) / dL/dz(z); L stays the
    forward's own."""
    rng = np.random.default_rng(21)
    m = _model([3], 2, 19, n_hidden=0, seed=9)
    m.nets[0][0] = rng.normal(size=(1, m.K)) * 5
    rays = synth.aimed_rays(rng, 30, BOX, 6.0)
    rid = np.arange(30)
    obj = np.zeros(30, np.int64)
    inner = np.zeros(30, bool)
    y = rng.integers(0, 2, size=30).astype(float)
    x = onif.encode(m, rays, rid, obj)
    z = x @ m.nets[0][0][0]
    za = z + rng.normal(scale=0.3, size=30)
    L, dnets, _ = onif.loss_and_grads(m, rays, rid, obj, inner, y, z_at=za)
    s0 = 1 / (1 + np.exp(-z))
    assert abs(L - np.mean((s0 - y) ** 2)) < 1e-14
    s = 1 / (1 + np.exp(-za))
    np.testing.assert_allclose(dnets[0][0][0], (2 / 30) * ((s - y) * s * (1 - s)) @ x, rtol=1e-12)
    # hidden layers: one pair, the gradient scales with dL/dz
    m2 = _model([2, 4], 2, 19, n_hidden=2, width=6, seed=3)
    for W in m2.nets[0]:
        W *= 3.0
    m2.grids *= 2.0
    r1 = synth.aimed_rays(rng, 1, BOX, 6.0)
    one = (np.arange(1), np.zeros(1, np.int64), np.zeros(1, bool), np.ones(1))
    _, dn, dg = onif.loss_and_grads(m2, r1, *one)
    z1 = onif.mlp_forward(onif.encode(m2, r1, one[0], one[1]), m2.nets[0], m2.act, m2.slope)[0]
    za1 = z1 - 0.7

    def dz(v):
        sv = 1 / (1 + np.exp(-v))
        return 2 * (sv - 1) * sv * (1 - sv)
    ratio = float(dz(za1)[0] / dz(z1)[0])
    _, dn_a, dg_a = onif.loss_and_grads(m2, r1, *one, z_at=za1)
    for a, b in zip(dn_a[0], dn[0]):
        np.testing.assert_allclose(a, ratio * b, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(dg_a, ratio * dg, rtol=1e-12, atol=1e-300)
    assert np.abs(dg).max() > 0 and abs(ratio - 1) > 0.1


# ------------------------------------------------------------ Adam
def test_adam_first_step_closed_form():
    """Step 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    th = rng.normal(size=100)
    g = rng.normal(size=100)
    g[:10] = 0.0
    lr = 1e-2
    new, m1, m2 = onif.adam_step(th, g, np.zeros(100), np.zeros(100), 1, lr)
    np.testing.assert_allclose(new, th - lr * g / (np.abs(g) + 1e-15), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(new[10:] - th[10:], -lr * np.sign(g[10:]), rtol=1e-9)
    assert np.all(new[:10] == th[:10])


def test_adam_second_step_closed_form_constant_gradient():
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step."""
    th = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m1 = np.zeros(2)
    m2 = np.zeros(2)
    for step in (1, 2, 3):
        th_new, m1, m2 = onif.adam_step(th, g, m1, m2, step, 0.1)
        np.testing.assert_allclose(th_new - th, -0.1 * np.sign(g), rtol=1e-12)
        th = th_new
    # zero gradient after momentum: the entry still moves (dense update)
    th2, _, _ = onif.adam_step(th, np.zeros(2), m1, m2, 4, 0.1)
    assert np.all(th2 != th)
