"""GPU path of NIF on primary rays (five outputs: occupancy logit, normal,
depth in the box; Sec. 3.2, Sec. 6.1) against the FP64 oracle in
``oracle/primary.py``: the outputs at FP32 and FP16 (tolerances 1e-4 and
2e-2 abs, as for the logit), the loss and gradients with the regression
terms, the closest-hit resolution bit for bit on seeded outputs, and the
per-pair closest hit of the exact cast against brute force."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import nif as onif  # noqa: E402
from oracle import primary as opr  # noqa: E402
from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth  # noqa: E402
from helpers import random_boxes_scene, to_dtype_values  # noqa: E402

DT = {"f32": L.NIF_F32, "f16": L.NIF_F16}
TDT = {"f32": torch.float32, "f16": torch.float16}
O = 5


def _setup(seed=51, n_obj=5, res=(4, 9, 20, 40), log2=12, width=64, n_hidden=2, n_rays=12000,
           grid_dt="f32", mlp_dt="f32", net_mode=L.NIF_NETS_CLASS, schedule=L.NIF_SCHED_AUTO):
    rng = np.random.default_rng(seed)
    boxes = random_boxes_scene(rng, n_obj=n_obj)
    sizes, hashed, off = onif.level_layout(list(res), log2)
    V, F = int(off[-1]), 2
    grid = rng.uniform(-1, 1, size=(n_obj, 2, V * F)).astype(np.float32)
    K = 3 * len(res) * F
    n_nets = 2 if net_mode == L.NIF_NETS_CLASS else 1
    mats = [synth.mlp_init(rng, K, width, n_hidden, n_out=O) for _ in range(n_nets)]
    flat = np.concatenate([synth.flatten_mlp(m) for m in mats]).astype(np.float32)
    # rays aimed at a point of a random box; a quarter start inside a box
    o = rng.uniform(-4.5, 4.5, size=(n_rays, 3))
    k = rng.integers(0, n_obj, n_rays)
    tgt = boxes[k, :3] + rng.uniform(size=(n_rays, 3)) * (boxes[k, 3:] - boxes[k, :3])
    ki = rng.integers(0, n_obj, n_rays // 4)
    o[: n_rays // 4] = boxes[ki, :3] + rng.uniform(0.05, 0.95, size=(n_rays // 4, 3)) * (boxes[ki, 3:] - boxes[ki, :3])
    d = tgt - o
    rays = synth.pack_rays(o, d / np.linalg.norm(d, axis=1, keepdims=True), 1e-3, np.inf)
    cfg = nif.NifConfig(res=list(res), n_features=F, log2_table=log2, grid_dtype=DT[grid_dt],
                        n_hidden=n_hidden, width=width, act=L.NIF_ACT_LEAKY, mlp_dtype=DT[mlp_dt],
                        net_mode=net_mode, n_outputs=O, schedule=schedule)
    assert nif.NifModel.weight_count(cfg) == len(flat) // n_nets
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(),
                         torch.from_numpy(grid.reshape(-1)).to(TDT[grid_dt]).cuda(),
                         torch.from_numpy(flat).to(TDT[mlp_dt]).cuda())
    nets64 = []
    per = len(flat) // n_nets
    for g in range(n_nets):
        f = to_dtype_values(flat[g * per:(g + 1) * per], mlp_dt)
        nets64.append(synth.unflatten_mlp(f, K, width, n_hidden, n_out=O))
    om = onif.Model(res=list(res), F=F, log2_table=log2, obj_aabb=boxes,
                    grids=to_dtype_values(grid, grid_dt),
                    nets=nets64, net_mode="class" if n_nets == 2 else "single", act="leaky")
    return model, om, rays, grid, flat


def _pairs(model, rays, boxes):
    """The oracle's query set (every overlapping (ray, object) pair), grouped
    by network as the calls expect: outer pairs, then inner ones."""
    r, ob, inn = onif.queries(rays, boxes)
    if model.n_nets == 2:
        order = np.argsort(inn, kind="stable")
        r, ob, inn = r[order], ob[order], inn[order]
        goff = [0, int((~inn).sum()), len(r)]
    else:
        goff = [0, len(r)]
    qo = (ob.astype(np.uint32) | (inn.astype(np.uint32) << 31)).view(np.int32)
    return (torch.from_numpy(r.astype(np.int32)).cuda(), torch.from_numpy(qo).cuda(),
            torch.tensor(goff, dtype=torch.int64, device="cuda"), len(r), r, ob, inn)


@pytest.mark.parametrize("dt,tol", [("f32", 1e-4), ("f16", 2e-2)])
def test_primary_outputs_match_oracle(dt, tol):
    model, om, rays, _, _ = _setup(grid_dt=dt, mlp_dt=dt, schedule=L.NIF_SCHED_SERIAL)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _pairs(model, rays, om.obj_aabb)
    assert nq > 3000 and nq % 128 != 0 and inn.any() and (~inn).any()
    bits = nif.empty_bits(len(rays))
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq, bits=bits)
    model.check()
    z = z[:nq].cpu().numpy()
    assert z.shape == (nq, O)
    zo = opr.outputs(om, rays, r, ob, inn)
    assert np.abs(zo).max() > 0.1
    err = np.abs(z - zo).max(axis=0)
    assert (err <= tol).all(), err
    # occupancy from output 0, exactly as for shadow rays
    occ = nif.bits_to_bool(bits, len(rays)).cpu().numpy()
    assert np.array_equal(occ, onif.ray_occlusion(len(rays), r, z[:, 0]))


def test_primary_loss_and_gradients_match_oracle():
    model, om, rays, grid, flat = _setup(seed=53, width=32, n_rays=16000)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _pairs(model, rays, om.obj_aabb)
    rng = np.random.default_rng(7)
    y = (rng.uniform(size=nq) < 0.4).astype(np.uint8)
    aux = rng.normal(size=(nq, O - 1)).astype(np.float32)
    d = model.desc()
    z = torch.empty((nq, O), dtype=torch.float32, device="cuda")
    saved = torch.empty(L.lib.nif_saved_size(ctypes.byref(d), nq) // 4, dtype=torch.float32, device="cuda")
    vp = ctypes.c_void_p
    sp = nif._stream()
    L.call("nif_fwd_train", ctypes.byref(d), vp(rays_t.data_ptr()), vp(ray_id.data_ptr()),
           vp(qobj.data_ptr()), vp(goff.data_ptr()), nq, vp(z.data_ptr()), vp(saved.data_ptr()), sp)
    lab = torch.from_numpy(y).cuda()
    aux_t = torch.from_numpy(aux).cuda()
    dz = torch.empty_like(z)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    L.call("nif_loss_aux", vp(z.data_ptr()), vp(lab.data_ptr()), vp(aux_t.data_ptr()), nq, O, 1.0,
           vp(dz.data_ptr()), vp(loss.data_ptr()), sp)
    wg = torch.zeros(len(flat), dtype=torch.float32, device="cuda")
    dx = torch.empty((om.K, nq), dtype=torch.float32, device="cuda")
    L.call("nif_mlp_bwd", ctypes.byref(d), vp(qobj.data_ptr()), vp(goff.data_ptr()), nq, vp(saved.data_ptr()),
           vp(dz.data_ptr()), vp(wg.data_ptr()), vp(dx.data_ptr()), sp)
    gg = torch.zeros(grid.size, dtype=torch.float32, device="cuda")
    L.call("nif_grid_bwd", ctypes.byref(d), vp(rays_t.data_ptr()), vp(ray_id.data_ptr()), vp(qobj.data_ptr()),
           nq, vp(dx.data_ptr()), vp(gg.data_ptr()), sp)
    torch.cuda.synchronize()
    Lo, dnets, dgrids = opr.loss_and_grads(om, rays, r, ob, inn, y.astype(np.float64), aux.astype(np.float64))
    assert abs(float(loss.item()) - Lo) <= 1e-5 * max(1.0, Lo)
    np.testing.assert_allclose(z.cpu().numpy(), opr.outputs(om, rays, r, ob, inn), rtol=0, atol=1e-4)
    want_w = np.concatenate([np.concatenate([m.reshape(-1) for m in net]) for net in dnets])
    got_w = wg.cpu().numpy()
    assert np.linalg.norm(got_w - want_w) <= 1e-3 * np.linalg.norm(want_w)
    got_g = gg.cpu().numpy().reshape(dgrids.shape)
    assert np.linalg.norm(got_g - dgrids) <= 1e-3 * np.linalg.norm(dgrids)
    # the output rows' gradients of both networks are all exercised
    assert all(np.abs(net[-1]).min() > 0 for net in dnets)


def test_train_step_needs_targets_for_several_outputs():
    model, om, rays, grid, flat = _setup(seed=55, n_rays=4000)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _pairs(model, rays, om.obj_aabb)
    tr = nif.Trainer(model, lr=1e-3)
    lab = torch.ones(nq, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.NifError):
        tr.step(rays_t, ray_id, qobj, goff, lab, nq)
    aux = torch.zeros((nq, O - 1), dtype=torch.float32, device="cuda")
    loss = tr.step(rays_t, ray_id, qobj, goff, lab, nq, aux=aux)
    model.check(tr._ws)
    assert np.isfinite(float(loss.item()))
    # several outputs: the pipelined schedule is refused, not run
    pm = nif.NifModel(nif.NifConfig(**{**model.cfg.__dict__, "grid_dtype": L.NIF_F16, "mlp_dtype": L.NIF_F16,
                                       "schedule": L.NIF_SCHED_PIPELINED}),
                      model.obj_aabb, model.grids.half(), model.weights.half())
    with pytest.raises(L.NifError) as e:
        pm.infer_queries(rays_t, ray_id, qobj, goff, nq)
    assert e.value.code == L.NIF_ERR_UNSUPPORTED


def test_closest_hit_resolution_is_bit_exact_on_seeded_outputs():
    """Outputs are seeded inputs here (not a network's), so the discrete
    choice of each ray's nearest hit can be compared bit for bit."""
    rng = np.random.default_rng(61)
    boxes = random_boxes_scene(rng, n_obj=7)
    n_rays = 20000
    o = rng.uniform(-4.5, 4.5, size=(n_rays, 3))
    k = rng.integers(0, 7, n_rays)
    tgt = boxes[k, :3] + rng.uniform(size=(n_rays, 3)) * (boxes[k, 3:] - boxes[k, :3])
    d = tgt - o
    rays = synth.pack_rays(o, d / np.linalg.norm(d, axis=1, keepdims=True), 1e-3, np.inf)
    cfg = nif.NifConfig(res=[2], n_features=2, n_hidden=1, width=8, net_mode=L.NIF_NETS_CLASS, n_outputs=O)
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.zeros(7 * 2 * 27 * 2).cuda(),
                         torch.zeros(2 * nif.NifModel.weight_count(cfg)).cuda())
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _pairs(model, rays, boxes)
    assert nq > 20000
    Z = np.empty((nq, O), np.float32)
    Z[:, 0] = rng.uniform(-1, 1, nq)
    Z[:, 1:4] = rng.normal(size=(nq, 3))
    Z[:, 4] = rng.uniform(-0.2, 1.2, nq)        # clamped at both ends
    Z[::97, 1:4] = 0.0                          # zero normals stay zero
    # ties: a ray's pairs with the same box entry and delta 0 meet at t_in
    Z[1::50, 4] = 0.0
    t_exact = np.full(n_rays, np.inf, np.float32)
    t_exact[::3] = rng.uniform(0.5, 8.0, len(t_exact[::3])).astype(np.float32)
    t = torch.from_numpy(t_exact.copy()).cuda()
    normal = torch.full((n_rays, 3), 7.0, device="cuda")
    win = torch.full((n_rays,), -2, dtype=torch.int32, device="cuda")
    nif.primary_resolve(model, rays_t, ray_id, qobj, goff, nq, torch.from_numpy(Z).cuda(), t=t, normal=normal,
                        winner=win)
    torch.cuda.synchronize()
    to, no, wo = opr.resolve(n_rays, rays, r, ob, boxes, Z)
    nearer = to < t_exact
    want_t = np.where(nearer, to, t_exact)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), want_t.view(np.uint32))
    w = win.cpu().numpy()
    assert np.array_equal(w[nearer], wo[nearer]) and (w[~nearer] == -2).all()
    n_ = normal.cpu().numpy()
    np.testing.assert_allclose(n_[nearer], no[nearer], rtol=0, atol=1e-6)
    assert (n_[~nearer] == 7.0).all()
    assert nearer.sum() > 1000 and (~nearer & (wo >= 0)).sum() > 100


def test_pair_closest_hit_matches_brute_force():
    rng = np.random.default_rng(63)
    meshes = [synth.displaced_icosphere(6, rng, centre=c) for c in ((0, 0, 0), (1.5, 0.4, 0), (3.5, 0, -0.3))]
    sc = synth.build_scene(meshes)
    n = 9000
    rays = np.concatenate([synth.aimed_rays(rng, n // 3, sc.obj_aabb[k], 3.0) for k in range(3)])
    rays[::5, 3] = 0.8  # some segments start past the first surface
    bvh = nif.BVH(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda(),
                  torch.from_numpy(sc.tri_obj).cuda())
    rid = np.repeat(np.arange(n), 3).astype(np.int32)
    obj = np.tile(np.arange(3), n).astype(np.int32)
    obj_q = obj.astype(np.uint32).copy()
    obj_q[::4] |= np.uint32(0x80000000)  # the class bit is ignored
    t, prim = bvh.cast_pairs_closest(torch.from_numpy(rays).cuda(), torch.from_numpy(rid).cuda(),
                                     torch.from_numpy(obj_q.view(np.int32)).cuda())
    torch.cuda.synchronize()
    to, po = oracle.brute_pairs_closest(sc.verts, sc.tris, sc.obj_tri_range[:, 0], sc.obj_tri_range[:, 1],
                                        rays, rid, obj)
    assert np.array_equal(t.cpu().numpy().view(np.uint32), to.view(np.uint32))
    assert np.array_equal(prim.cpu().numpy(), po)
    assert 0.2 < (po >= 0).mean() < 0.95


def test_resolution_of_empty_lists_leaves_the_exact_answer():
    rng = np.random.default_rng(65)
    boxes = random_boxes_scene(rng, n_obj=3)
    cfg = nif.NifConfig(res=[2], n_features=2, n_hidden=1, width=8, n_outputs=O)
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.zeros(3 * 2 * 27 * 2).cuda(),
                         torch.zeros(nif.NifModel.weight_count(cfg)).cuda())
    rays = torch.from_numpy(synth.pack_rays(rng.uniform(-3, 3, (100, 3)), synth.unit_vectors(rng, 100),
                                            0.0, np.inf)).cuda()
    t0 = torch.rand(100, device="cuda")
    t = t0.clone()
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    goff = torch.zeros(2, dtype=torch.int64, device="cuda")
    nif.primary_resolve(model, rays, e, e, goff, 0, torch.empty((0, O), device="cuda"), t=t)
    torch.cuda.synchronize()
    assert torch.equal(t, t0)
    # the shadow-ray descriptor (one output) is refused by the resolution
    m1 = nif.NifModel(nif.NifConfig(res=[2], n_features=2, n_hidden=1, width=8), model.obj_aabb,
                      model.grids, torch.zeros(nif.NifModel.weight_count(nif.NifConfig(res=[2], n_hidden=1,
                                                                                         width=8))).cuda())
    with pytest.raises(L.NifError):
        nif.primary_resolve(m1, rays, e, e, goff, 0, torch.empty((0, O), device="cuda"))
