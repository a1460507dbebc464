"""GPU NIF path (nif_frontend, nif_encode, nif_infer_queries, nif_infer)
against the FP64 oracle: query sets bit-exact, encodings and logits within
the stated tolerances (FP32 1e-4 abs, FP16 2e-2 abs, BF16 6e-2 abs)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import nif as onif  # noqa: E402
from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth, workloads  # noqa: E402
from helpers import oracle_model, pairs_key, random_boxes_scene, to_dtype_values  # noqa: E402

DT = {"f32": L.NIF_F32, "f16": L.NIF_F16, "bf16": L.NIF_BF16}
TORCH_DT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


def _build(res, F, log2, aabb, grid_vals, mats_list, grid_dt="f32", mlp_dt="f32",
           net_mode=L.NIF_NETS_SINGLE, act=L.NIF_ACT_RELU, ctas_per_sm=0,
           schedule=L.NIF_SCHED_AUTO):
    """GPU model and the matching oracle model from the same float32 inputs
    (rounded to the GPU storage types)."""
    n_hidden = len(mats_list[0]) - 1
    width = mats_list[0][0].shape[0]
    cfg = nif.NifConfig(res=list(res), n_features=F, log2_table=log2, grid_dtype=DT[grid_dt],
                        n_hidden=n_hidden, width=width, act=act, mlp_dtype=DT[mlp_dt],
                        net_mode=net_mode, ctas_per_sm=ctas_per_sm, schedule=schedule)
    flat = np.concatenate([synth.flatten_mlp(m) for m in mats_list])
    g = torch.from_numpy(np.ascontiguousarray(grid_vals, np.float32)).to(TORCH_DT[grid_dt]).cuda()
    w = torch.from_numpy(flat).to(TORCH_DT[mlp_dt]).cuda()
    model = nif.NifModel(cfg, torch.from_numpy(aabb).cuda(), g, w)
    K = 3 * len(res) * F
    nets64 = []
    for m in mats_list:
        f = to_dtype_values(synth.flatten_mlp(m), mlp_dt)
        nets64.append(synth.unflatten_mlp(f, K, width, n_hidden))
    om = oracle_model(onif, res, F, log2, aabb, to_dtype_values(grid_vals, grid_dt), nets64,
                      net_mode={L.NIF_NETS_SINGLE: "single", L.NIF_NETS_CLASS: "class",
                                L.NIF_NETS_OBJECT: "object"}[net_mode],
                      act="relu" if act == L.NIF_ACT_RELU else "leaky")
    return model, om


def _gpu_queries(model, rays_t, tlas=None):
    ray_id, qobj, goff, count = model.frontend(rays_t, tlas=tlas)
    torch.cuda.synchronize()
    nq = int(count.item())
    return ray_id, qobj, goff, nq


def _query_arrays(ray_id, qobj, nq):
    r = ray_id[:nq].cpu().numpy().astype(np.int64)
    q = qobj[:nq].cpu().numpy().view(np.uint32)
    return r, (q & 0x7FFFFFFF).astype(np.int64), (q >> 31).astype(bool)


@pytest.mark.parametrize("use_tlas", [False, True, "ploc"])
def test_frontend_query_set_bit_exact(use_tlas):
    rng = np.random.default_rng(21)
    boxes = random_boxes_scene(rng, n_obj=9)
    o = rng.uniform(-4, 4, size=(20000, 3))
    d = synth.unit_vectors(rng, 20000)
    rays = synth.pack_rays(o, d, 1e-3, np.inf)
    rays[::4, 7] = rng.uniform(0.5, 3.0, size=len(rays[::4]))
    rays[::7, 4:7] = [1.0, 0.0, 0.0]
    for mode, nn in ((L.NIF_NETS_CLASS, 2), (L.NIF_NETS_OBJECT, 9), (L.NIF_NETS_SINGLE, 1)):
        cfg = nif.NifConfig(res=[2], n_features=1, net_mode=mode)
        model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.zeros(9 * 2 * 27).cuda(),
                             torch.zeros(nn * nif.NifModel.weight_count(cfg)).cuda())
        tlas = (nif.BVH.from_boxes(torch.from_numpy(boxes).cuda(), builder="ploc" if use_tlas == "ploc" else "lbvh")
                if use_tlas else None)
        ray_id, qobj, goff, nq = _gpu_queries(model, torch.from_numpy(rays).cuda(), tlas)
        r, ob, inn = _query_arrays(ray_id, qobj, nq)
        rr, oo, ii = onif.queries(rays, boxes)
        assert nq == len(rr)
        got = sorted(zip(r.tolist(), ob.tolist(), inn.tolist()))
        want = sorted(zip(rr.tolist(), oo.tolist(), ii.tolist()))
        assert got == want
        # grouping: group g holds exactly the pairs of network g, objects ascending
        go = goff.cpu().numpy()
        assert go[0] == 0 and go[-1] == nq and np.all(np.diff(go) >= 0)
        for g in range(nn):
            s, e = go[g], go[g + 1]
            if mode == L.NIF_NETS_CLASS:
                assert np.all(inn[s:e] == bool(g))
            if mode == L.NIF_NETS_OBJECT:
                assert np.all(ob[s:e] == g)
            assert np.all(np.diff(ob[s:e]) >= 0)


def _tiny(grid_scale=1.0, aimed=True, n_rays=4000):
    w = workloads.tiny_object(n_rays=n_rays, aimed=aimed, grid_scale=grid_scale)
    return w


def test_encode_fp32_matches_oracle():
    w = _tiny()
    model, om = _build(w.res, 2, 19, w.aabb, w.grid_values, [w.weights])
    rays_t = torch.from_numpy(w.rays).cuda()
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t)
    x = model.encode(rays_t, ray_id, qobj, nq).cpu().numpy()
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    xo = onif.encode(om, w.rays, r, ob)
    assert nq > 3000
    np.testing.assert_allclose(x, xo, atol=2e-5, rtol=0)
    x16 = model.encode(rays_t, ray_id, qobj, nq, dtype=L.NIF_F16).float().cpu().numpy()
    np.testing.assert_allclose(x16, xo, atol=2e-3, rtol=0)


SER, PIPE = L.NIF_SCHED_SERIAL, L.NIF_SCHED_PIPELINED


@pytest.mark.parametrize("mlp_dt,grid_dt,tol,ctas,sched", [
    ("f32", "f32", 1e-4, 0, 0), ("f16", "f32", 2e-2, 0, 0), ("f16", "f16", 2e-2, 0, 0),
    ("bf16", "f32", 6e-2, 0, 0), ("f16", "f16", 2e-2, 3, SER), ("bf16", "f16", 6e-2, 3, SER),
    ("f16", "f16", 2e-2, 4, SER), ("bf16", "f32", 6e-2, 4, SER), ("f16", "f16", 2e-2, 0, PIPE),
    ("bf16", "f32", 6e-2, 0, PIPE)])
def test_logits_match_oracle(mlp_dt, grid_dt, tol, ctas, sched):
    w = _tiny(n_rays=6000)
    model, om = _build(w.res, 2, 19, w.aabb, w.grid_values, [w.weights], grid_dt=grid_dt, mlp_dt=mlp_dt,
                       ctas_per_sm=ctas, schedule=sched)
    rays_t = torch.from_numpy(w.rays).cuda()
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t)
    bits = nif.empty_bits(len(w.rays))
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq, bits=bits)
    model.check()
    torch.cuda.synchronize()
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    zo = onif.forward(om, w.rays, r, ob, inn)
    zg = z[:nq].cpu().numpy()
    err = np.abs(zg - zo)
    assert nq > 4000 and nq % 128 != 0  # several tiles and a ragged tail
    assert np.abs(zo).max() > 0.05      # logits are not trivially small
    assert err.max() <= tol, (err.max(), np.abs(zo).max())
    occ = nif.bits_to_bool(bits, len(w.rays)).cpu().numpy()
    want = onif.ray_occlusion(len(w.rays), r, zg)
    assert np.array_equal(occ, want)
    # decisions agree with the oracle wherever the oracle logit is not within tol of 0
    firm = np.abs(zo) > tol
    assert np.array_equal(zg[firm] < 0, zo[firm] < 0)


@pytest.mark.parametrize("mlp_dt,tol", [("f32", 1e-4), ("f16", 2e-2)])
def test_class_networks_hashed_grids_multi_object(mlp_dt, tol):
    """Two networks (outer / inner), several objects, hashed fine levels."""
    rng = np.random.default_rng(31)
    boxes = random_boxes_scene(rng, n_obj=5)
    res = [3, 6, 12, 40]
    log2 = 11
    sizes, hashed, off = onif.level_layout(res, log2)
    assert hashed == [False, False, True, True]
    V = int(off[-1])
    grid = rng.uniform(-1, 1, size=(5, 2, V * 2)).astype(np.float32)
    mats = [synth.mlp_init(rng, 24, 64, 2), synth.mlp_init(rng, 24, 64, 2)]
    model, om = _build(res, 2, log2, boxes, grid, mats, grid_dt="f16", mlp_dt=mlp_dt,
                       net_mode=L.NIF_NETS_CLASS)
    o = rng.uniform(-4, 4, size=(6000, 3))
    rays = synth.pack_rays(o, synth.unit_vectors(rng, 6000), 1e-3, np.inf)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t)
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq)
    model.check()
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    assert inn.any() and (~inn).any()
    zo = onif.forward(om, rays, r, ob, inn)
    err = np.abs(z[:nq].cpu().numpy() - zo)
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("mlp_dt", ["f32", "f16"])
def test_infer_end_to_end_equals_queries_path(mlp_dt):
    w = _tiny(n_rays=5000, aimed=False)
    model, om = _build(w.res, 2, 19, w.aabb, w.grid_values, [w.weights], mlp_dt=mlp_dt)
    rays_t = torch.from_numpy(w.rays).cuda()
    bits = nif.empty_bits(len(w.rays))
    model.infer(rays_t, bits)
    model.check()
    occ = nif.bits_to_bool(bits, len(w.rays)).cpu().numpy()
    rr, oo, ii = onif.queries(w.rays, w.aabb)
    zo = onif.forward(om, w.rays, rr, oo, ii)
    want = onif.ray_occlusion(len(w.rays), rr, zo)
    tol = 1e-4 if mlp_dt == "f32" else 2e-2
    firm = np.ones(len(w.rays), bool)
    firm[rr[np.abs(zo) <= tol]] = False
    assert np.array_equal(occ[firm], want[firm])
    # no ray without a query is ever occluded
    noq = np.ones(len(w.rays), bool)
    noq[rr] = False
    assert not occ[noq].any()


def test_zero_rays_and_zero_queries():
    w = _tiny(n_rays=64)
    model, _ = _build(w.res, 2, 19, w.aabb, w.grid_values, [w.weights], mlp_dt="f16")
    empty = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
    bits = nif.empty_bits(0)
    model.infer(empty, bits)
    # rays that miss the box entirely: no queries, nothing occluded
    far = synth.pack_rays(np.full((100, 3), 10.0), np.tile([[1.0, 0, 0]], (100, 1)), 0.0, np.inf)
    bits = nif.empty_bits(100)
    model.infer(torch.from_numpy(far).cuda(), bits)
    model.check()
    assert not nif.bits_to_bool(bits, 100).any()


def test_fp8_e4m3_logits_within_reported_bound():
    """FP8-E4M3 weights and activations with per-tensor scales (amax / 448,
    activations calibrated on the oracle's FP64 forward of the same queries),
    FP32 accumulation: logits within 0.25 abs of FP64 on dequantised weights."""
    w = _tiny(n_rays=6000)
    flat = np.concatenate([synth.flatten_mlp(w.weights)]).astype(np.float32)
    K = 48
    # calibration: the oracle's activations at each layer input
    om32 = oracle_model(onif, w.res, 2, 19, w.aabb, w.grid_values.astype(np.float64),
                        [[np.asarray(m, np.float64) for m in w.weights]])
    rr, oo, ii = onif.queries(w.rays, w.aabb)
    x = onif.encode(om32, w.rays, rr, oo)
    _, pre, post = onif.mlp_forward(x, om32.nets[0])
    amax = [[float(np.abs(post[l]).max()) for l in range(3)]]
    cfg = nif.NifConfig(res=w.res, n_features=2, log2_table=19, grid_dtype=L.NIF_F32, n_hidden=3,
                        width=64, mlp_dtype=L.NIF_E4M3)
    q, sc = nif.quantize_e4m3(torch.from_numpy(flat).cuda(), cfg, 1, amax)
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(), torch.from_numpy(w.grid_values.reshape(-1)).cuda(),
                         q, scales=sc)
    # oracle on the dequantised weights
    deq = (q.float().reshape(-1).cpu().numpy().astype(np.float64))
    scn = sc.cpu().numpy()
    mats, off, fan_in = [], 0, K
    for l in range(4):
        n = 64 * fan_in if l < 3 else fan_in
        mats.append(deq[off:off + n].reshape(64 if l < 3 else 1, fan_in) * scn[0, l, 1])
        off += n
        fan_in = 64
    om = oracle_model(onif, w.res, 2, 19, w.aabb, w.grid_values.astype(np.float64), [mats])
    rays_t = torch.from_numpy(w.rays).cuda()
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t)
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq)
    model.check()
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    zo = onif.forward(om, w.rays, r, ob, inn)
    err = np.abs(z[:nq].cpu().numpy() - zo)
    assert np.abs(zo).max() > 0.05
    assert err.max() <= 0.25, err.max()
    assert err.mean() <= 0.05, err.mean()


@pytest.mark.parametrize("use_tlas", [False, True, "ploc"])
def test_frontend_many_pairs_per_ray(use_tlas):
    """Rays crossing 16 boxes in a row: more pairs per ray than the front end
    keeps per ray in its single-traversal slots."""
    lo = np.stack([np.arange(16) * 1.5, np.zeros(16), np.zeros(16)], 1)
    boxes = np.concatenate([lo, lo + 1.0], axis=1).astype(np.float32)
    rng = np.random.default_rng(2)
    n = 3000
    o = np.stack([np.full(n, -5.0), rng.uniform(0.05, 0.95, n), rng.uniform(0.05, 0.95, n)], 1)
    d = np.tile([[1.0, 0.0, 0.0]], (n, 1))
    d[n // 2:] = synth.unit_vectors(rng, n - n // 2)
    rays = synth.pack_rays(o, d, 1e-3, np.inf)
    cfg = nif.NifConfig(res=[2], n_features=1, net_mode=L.NIF_NETS_CLASS)
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.zeros(16 * 2 * 27).cuda(),
                         torch.zeros(2 * nif.NifModel.weight_count(cfg)).cuda())
    tlas = (nif.BVH.from_boxes(torch.from_numpy(boxes).cuda(), builder="ploc" if use_tlas == "ploc" else "lbvh")
            if use_tlas else None)
    ray_id, qobj, goff, count = model.frontend(torch.from_numpy(rays).cuda(), tlas=tlas, max_q=20 * n)
    model.check()
    nq = int(count.item())
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    rr, oo, ii = onif.queries(rays, boxes)
    assert np.bincount(rr).max() == 16
    assert sorted(zip(r.tolist(), ob.tolist(), inn.tolist())) == sorted(zip(rr.tolist(), oo.tolist(), ii.tolist()))


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("mlp_dt,tol", [("f16", 2e-2), ("bf16", 6e-2)])
def test_per_object_networks_grouped_launch(mlp_dt, tol, tile_m):
    """One network per object (Sec. 6.3) in one persistent grouped launch:
    uneven group sizes, each group's weights loaded when the tile's group
    changes; logits against the oracle with every object's own network, for
    tiles of 128 and of 256 queries (two 128-row blocks in TMEM)."""
    gw = workloads.grouped_objects(n_obj=6, total_rays=20000, tri_min=500, tri_max=5000, seed=3)
    rng = np.random.default_rng(9)
    res = [4, 8, 16, 32]
    cfg_v = onif.level_layout(res, 19)[2][-1]
    grid = rng.uniform(-1, 1, size=(6, 2, int(cfg_v) * 2)).astype(np.float32)
    mats = [synth.mlp_init(rng, 24, 64, 3) for _ in range(6)]
    model, om = _build(res, 2, 19, gw.scene.obj_aabb, grid, mats, grid_dt="f16", mlp_dt=mlp_dt,
                       net_mode=L.NIF_NETS_OBJECT, schedule=SER)
    model.cfg.tile_m = tile_m
    n = len(gw.rays)
    obj = np.repeat(np.arange(6), gw.counts)
    rays_t = torch.from_numpy(gw.rays).cuda()
    ray_id = torch.arange(n, dtype=torch.int32, device="cuda")
    qobj = torch.from_numpy(obj.astype(np.int32)).cuda()
    goff = torch.from_numpy(np.concatenate([[0], np.cumsum(gw.counts)]).astype(np.int64)).cuda()
    z = model.infer_queries(rays_t, ray_id, qobj, goff, n)
    model.check()
    # every ray is aimed at its object's box, so every pair is a query
    hit = np.zeros(n, bool)
    for k in range(6):
        sel = obj == k
        hit[sel] = onif.slab_fp32(gw.rays[sel], gw.scene.obj_aabb[k])[0]
    assert hit.all()
    zo = onif.forward(om, gw.rays, np.arange(n), obj, np.zeros(n, bool))
    err = np.abs(z.cpu().numpy()[:n] - zo)
    assert (gw.counts % tile_m != 0).any() and gw.counts.max() > tile_m  # ragged, multi-tile groups
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("sched", [SER, PIPE, "serial/256"])
@pytest.mark.parametrize("mlp_dt,tol", [("f16", 2e-2), ("bf16", 6e-2)])
def test_sixteen_level_input_both_schedules(sched, mlp_dt, tol):
    """K = 96 (16 levels x 2 features x 3 points), hashed fine levels and two
    networks: the pipelined schedule's wide form (two 48-column TMEM buffers,
    16 encode warps) and the serial one give the oracle's logits."""
    rng = np.random.default_rng(57)
    boxes = random_boxes_scene(rng, n_obj=3)
    res = [4, 5, 6, 8, 10, 12, 15, 19, 24, 30, 38, 48, 60, 76, 96, 120]
    log2 = 14
    sizes, hashed, off = onif.level_layout(res, log2)
    assert any(hashed) and not all(hashed)
    V = int(off[-1])
    grid = rng.uniform(-1, 1, size=(3, 2, V * 2)).astype(np.float32)
    mats = [synth.mlp_init(rng, 96, 64, 3), synth.mlp_init(rng, 96, 64, 3)]
    model, om = _build(res, 2, log2, boxes, grid, mats, grid_dt="f16", mlp_dt=mlp_dt,
                       net_mode=L.NIF_NETS_CLASS, schedule=SER if sched == "serial/256" else sched)
    if sched == "serial/256":  # tiles of 256 queries
        model.cfg.tile_m = 256
    # rays aimed at a uniform point of a random box, from inside and outside
    n = 7000
    o = rng.uniform(-3, 3, size=(n, 3))
    k = rng.integers(0, 3, size=n)
    tgt = boxes[k, :3] + rng.uniform(size=(n, 3)) * (boxes[k, 3:] - boxes[k, :3])
    d = tgt - o
    rays = synth.pack_rays(o, d / np.linalg.norm(d, axis=1, keepdims=True), 1e-3, np.inf)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t)
    bits = nif.empty_bits(len(rays))
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq, bits=bits)
    model.check()
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    assert nq > 2000 and nq % 128 != 0 and inn.any() and (~inn).any()
    zo = onif.forward(om, rays, r, ob, inn)
    zg = z[:nq].cpu().numpy()
    assert np.abs(zo).max() > 0.05
    err = np.abs(zg - zo)
    assert err.max() <= tol, err.max()
    occ = nif.bits_to_bool(bits, len(rays)).cpu().numpy()
    assert np.array_equal(occ, onif.ray_occlusion(len(rays), r, zg))


@pytest.mark.parametrize("mlp_dt", ["f16", "bf16"])
def test_schedules_agree_on_grouped_networks(mlp_dt):
    """The serial and pipelined schedules on one grouped launch of per-object
    networks: the same query rows give logits within FP32 summation-order
    differences (the two sum the output layer in different orders)."""
    gw = workloads.grouped_objects(n_obj=5, total_rays=30000, tri_min=500, tri_max=5000, seed=5)
    rng = np.random.default_rng(13)
    res = [4, 8, 16, 32]
    V = int(onif.level_layout(res, 19)[2][-1])
    grid = rng.uniform(-1, 1, size=(5, 2, V * 2)).astype(np.float32)
    mats = [synth.mlp_init(rng, 24, 64, 3) for _ in range(5)]
    n = len(gw.rays)
    rays_t = torch.from_numpy(gw.rays).cuda()
    ray_id = torch.arange(n, dtype=torch.int32, device="cuda")
    obj = np.repeat(np.arange(5), gw.counts)
    qobj = torch.from_numpy(obj.astype(np.int32)).cuda()
    goff = torch.from_numpy(np.concatenate([[0], np.cumsum(gw.counts)]).astype(np.int64)).cuda()
    out = {}
    for sched in (SER, PIPE):
        model, _ = _build(res, 2, 19, gw.scene.obj_aabb, grid, mats, grid_dt="f16", mlp_dt=mlp_dt,
                          net_mode=L.NIF_NETS_OBJECT, schedule=sched)
        out[sched] = model.infer_queries(rays_t, ray_id, qobj, goff, n).cpu().numpy()[:n]
        model.check()
    scale = np.abs(out[SER]).max()
    assert scale > 0.05
    assert np.abs(out[SER] - out[PIPE]).max() <= 1e-5 * max(1.0, scale)


@pytest.mark.parametrize("mlp_dt,sched", [("f32", 0), ("f16", SER), ("f16", PIPE), ("bf16", 0)])
def test_two_round_infer_equals_all_pairs(mlp_dt, sched):
    """nif_infer's early-out (one pair per ray first, then the other pairs of
    rays still unoccluded) leaves exactly the bits of querying every pair;
    rays already occluded on entry are not queried at all."""
    rng = np.random.default_rng(71)
    boxes = random_boxes_scene(rng, n_obj=12, extent=3.0)
    res = [4, 8, 16, 32]
    V = int(onif.level_layout(res, 12)[2][-1])
    grid = rng.uniform(-1, 1, size=(12, 2, V * 2)).astype(np.float32)
    mats = [synth.mlp_init(rng, 24, 64, 3), synth.mlp_init(rng, 24, 64, 3)]
    model, om = _build(res, 2, 12, boxes, grid, mats, grid_dt="f16", mlp_dt=mlp_dt,
                       net_mode=L.NIF_NETS_CLASS, schedule=sched)
    n = 20000
    o = rng.uniform(-4, 4, size=(n, 3))
    rays = synth.pack_rays(o, synth.unit_vectors(rng, n), 1e-3, np.inf)
    rays_t = torch.from_numpy(rays).cuda()
    tlas = nif.BVH.from_boxes(torch.from_numpy(boxes).cuda())
    # every pair at once
    ray_id, qobj, goff, nq = _gpu_queries(model, rays_t, tlas=tlas)
    all_bits = nif.empty_bits(n)
    model.infer_queries(rays_t, ray_id, qobj, goff, nq, bits=all_bits)
    model.check()
    # two rounds, from zero and from a pre-set mask
    two = nif.empty_bits(n)
    model.infer(rays_t, two, tlas=tlas)
    model.check()
    counts = model.infer_query_counts(n).cpu().numpy()
    va = nif.bits_to_bool(all_bits, n).cpu().numpy()
    vt = nif.bits_to_bool(two, n).cpu().numpy()
    assert np.array_equal(va, vt)
    model.cfg.round1 = L.NIF_ROUND1_OUTER
    two_o = nif.empty_bits(n)
    model.infer(rays_t, two_o, tlas=tlas)
    model.check()
    assert torch.equal(two_o, two)
    model.cfg.round1 = L.NIF_ROUND1_NEAREST
    r = ray_id[:nq].cpu().numpy()
    with_pair = np.unique(r)
    assert counts[0] == len(with_pair)            # one round-1 pair per ray with a pair
    assert counts[0] < counts[1] < nq             # round 2 skipped pairs of occluded rays
    assert va.any() and (~va[with_pair]).any()
    pre = rng.uniform(size=n) < 0.3
    pre_bits = torch.from_numpy(np.packbits(pre, bitorder="little").view(np.uint8)).cuda()
    words = torch.zeros((n + 31) // 32 * 4, dtype=torch.uint8, device="cuda")
    words[:pre_bits.numel()] = pre_bits
    bits_pre = words.view(torch.int32).clone()
    model.infer(rays_t, bits_pre, tlas=tlas)
    model.check()
    vp = nif.bits_to_bool(bits_pre, n).cpu().numpy()
    assert np.array_equal(vp, va | pre)
    c2 = model.infer_query_counts(n).cpu().numpy()
    assert c2[0] == len(np.setdiff1d(with_pair, np.nonzero(pre)[0]))


@pytest.mark.parametrize("rule", [L.NIF_ROUND1_NEAREST, L.NIF_ROUND1_OUTER])
def test_round_one_choice(rule):
    """nif_frontend_nearest lists one pair per ray: its nearest pair
    (NIF_ROUND1_NEAREST), or its nearest outer pair, else one of its inner
    pairs (NIF_ROUND1_OUTER); the choice is checked against the oracle's
    query set and FP32 slab entries."""
    import ctypes
    rng = np.random.default_rng(75)
    boxes = random_boxes_scene(rng, n_obj=10, extent=3.0)
    n = 20000
    o = rng.uniform(-4, 4, size=(n, 3))
    ki = rng.integers(0, 10, n // 2)
    o[: n // 2] = boxes[ki, :3] + rng.uniform(0.05, 0.95, size=(n // 2, 3)) * (boxes[ki, 3:] - boxes[ki, :3])
    rays = synth.pack_rays(o, synth.unit_vectors(rng, n), 1e-3, np.inf)
    cfg = nif.NifConfig(res=[2], n_features=1, net_mode=L.NIF_NETS_CLASS, round1=rule)
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.zeros(10 * 2 * 27).cuda(),
                         torch.zeros(2 * nif.NifModel.weight_count(cfg)).cuda())
    rays_t = torch.from_numpy(rays).cuda()
    tlas = nif.BVH.from_boxes(torch.from_numpy(boxes).cuda())
    max_q = 8 * n
    ray_id = torch.empty(max_q, dtype=torch.int32, device="cuda")
    qobj = torch.empty(max_q, dtype=torch.int32, device="cuda")
    goff = torch.empty(3, dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    bits = nif.empty_bits(n)
    ws = model.workspace(max_q, n)
    d = model.desc()
    vp = ctypes.c_void_p
    L.call("nif_frontend_nearest", ctypes.byref(d), vp(tlas.buf.data_ptr()), vp(rays_t.data_ptr()), n,
           vp(bits.data_ptr()), vp(ray_id.data_ptr()), vp(qobj.data_ptr()), max_q, vp(goff.data_ptr()),
           vp(count.data_ptr()), vp(ws.data_ptr()), ws.numel(), nif._stream())
    torch.cuda.synchronize()
    model.check(ws)
    nq = int(count.item())
    r, ob, inn = _query_arrays(ray_id, qobj, nq)
    rr, oo, ii = onif.queries(rays, boxes)
    assert nq == len(np.unique(rr)) and len(np.unique(r)) == nq
    chosen = {int(a): (int(b), bool(c)) for a, b, c in zip(r, ob, inn)}
    entry = np.full(len(rr), np.inf)
    for k in range(len(boxes)):
        sel = np.nonzero(oo == k)[0]
        entry[sel] = onif.slab_fp32(rays[rr[sel]], boxes[k])[1]
    n_outer_first = 0
    for ray in np.unique(rr):
        sel = np.nonzero(rr == ray)[0]
        obj, inner = chosen[int(ray)]
        outer = sel[~ii[sel]]
        if rule == L.NIF_ROUND1_NEAREST:
            got = entry[sel[(oo[sel] == obj) & (ii[sel] == inner)]][0]
            assert got <= entry[sel].min() * (1 + 1e-5) + 1e-6, (ray, got)
            n_outer_first += int(inner and len(outer) > 0)
        elif len(outer):
            assert not inner, ray
            best = entry[outer].min()
            got = entry[sel[(oo[sel] == obj) & ~ii[sel]]][0]
            assert got <= best * (1 + 1e-5) + 1e-6, (ray, got, best)
            n_outer_first += int(ii[sel].any())
        else:  # only inner pairs (the origin inside overlapping boxes): one of them
            assert inner and obj in set(oo[sel].tolist())
    assert n_outer_first > 1000  # rays with both kinds: the inner (nearest) or the outer pair
