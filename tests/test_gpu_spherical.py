"""GPU path of the paper's own encoding (NIF_ENC_SPHERICAL_OUTER / _INNER:
spherical 2D position and direction grids, the inner 1D distance grid, one
network per class) against the FP64 oracle in ``oracle/spherical.py``:
features, logits at every precision, gradients, and the class routing of the
front end.  Tolerances: FP32 1e-4 abs, FP16 2e-2 abs, BF16 6e-2 abs.

The mapping has singular points: the azimuth is undefined on the polar axis,
and both angles of an inner point at the box centre.  Near them an FP32 and an
FP64 evaluation may pick different cells, so the comparisons keep the pairs
the oracle finds away from them (sin(theta) > 0.05 for the point and the
direction; inner points farther than 5% of the half diagonal from the centre)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import nif as onif  # noqa: E402
from oracle import spherical as osph  # noqa: E402
from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth  # noqa: E402
from helpers import random_boxes_scene, to_dtype_values  # noqa: E402

DT = {"f32": L.NIF_F32, "f16": L.NIF_F16, "bf16": L.NIF_BF16}
TDT = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
ENC = {"outer": L.NIF_ENC_SPHERICAL_OUTER, "inner": L.NIF_ENC_SPHERICAL_INNER}


def _scene(seed=21, n_obj=5, n_rays=12000):
    rng = np.random.default_rng(seed)
    boxes = random_boxes_scene(rng, n_obj=n_obj)
    # rays aimed at a point of a random box, half of them from inside a box
    o = rng.uniform(-3.5, 3.5, size=(n_rays, 3))
    ki = rng.integers(0, n_obj, n_rays // 2)
    o[: n_rays // 2] = boxes[ki, :3] + rng.uniform(0.02, 0.98, size=(n_rays // 2, 3)) * (boxes[ki, 3:] - boxes[ki, :3])
    k = rng.integers(0, n_obj, n_rays)
    tgt = boxes[k, :3] + rng.uniform(size=(n_rays, 3)) * (boxes[k, 3:] - boxes[k, :3])
    d = tgt - o
    rays = synth.pack_rays(o, d / np.linalg.norm(d, axis=1, keepdims=True), 1e-3, 20.0)
    return rng, boxes, rays


def _model(kind, rng, boxes, R=16, N=3, R1=8, N1=3, width=64, n_hidden=2, grid_dt="f32",
           mlp_dt="f32", net_mode=L.NIF_NETS_SINGLE):
    inner = kind == "inner"
    G = 2 * R * R * N + (R1 * N1 if inner else 0)
    grids = rng.uniform(-1, 1, size=(len(boxes), G)).astype(np.float32)
    K = 2 * N + (N1 if inner else 0)
    mats = synth.mlp_init(rng, K, width, n_hidden)
    flat = synth.flatten_mlp(mats)
    cfg = nif.NifConfig(res=[R], n_features=N, grid_dtype=DT[grid_dt], n_hidden=n_hidden, width=width,
                        act=L.NIF_ACT_LEAKY, mlp_dtype=DT[mlp_dt], net_mode=net_mode,
                        encoding=ENC[kind], res_1d=R1 if inner else 0, n_features_1d=N1 if inner else 0)
    assert nif.NifModel.grid_vertices(cfg) == G
    assert nif.NifModel.weight_count(cfg) == len(flat)
    n_nets = 2 if net_mode == L.NIF_NETS_CLASS else 1
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(),
                         torch.from_numpy(grids.reshape(-1)).to(TDT[grid_dt]).cuda(),
                         torch.from_numpy(np.tile(flat, n_nets)).to(TDT[mlp_dt]).cuda())
    net64 = synth.unflatten_mlp(to_dtype_values(flat, mlp_dt), K, width, n_hidden)
    om = osph.SphericalModel(kind=kind, R=R, N=N, R1=R1 if inner else 0, N1=N1 if inner else 0,
                             obj_aabb=boxes, grids=to_dtype_values(grids, grid_dt), net=net64)
    return model, om


def _conditioned(kind, rays, boxes, r, ob):
    """Pairs away from the mapping's singular points (see the module notes)."""
    keep = np.ones(len(r), bool)
    for k in np.unique(ob):
        sel = np.nonzero(ob == k)[0]
        v, d, rr = osph.query_points(kind, rays[r[sel]], boxes[k])
        for a in (v, d):
            keep[sel] &= np.hypot(a[:, 0], a[:, 1]) > 0.05 * np.linalg.norm(a, axis=1)
        if kind == "inner":
            keep[sel] &= rr > 0.05
    return keep


def _class_pairs(kind, rays, boxes):
    r, ob, inn = onif.queries(rays, boxes)
    sel = inn if kind == "inner" else ~inn
    r, ob, inn = r[sel], ob[sel], inn[sel]
    keep = _conditioned(kind, rays, boxes, r, ob)
    r, ob, inn = r[keep], ob[keep], inn[keep]
    qobj = (ob.astype(np.uint32) | (inn.astype(np.uint32) << 31)).view(np.int32)
    return r, ob, torch.from_numpy(r.astype(np.int32)).cuda(), torch.from_numpy(qobj).cuda()


@pytest.mark.parametrize("kind", ["outer", "inner"])
def test_spherical_features_match_oracle(kind):
    rng, boxes, rays = _scene()
    model, om = _model(kind, rng, boxes)
    r, ob, rid_t, qobj_t = _class_pairs(kind, rays, boxes)
    assert len(r) > 1500 and len(r) % 128 != 0
    rays_t = torch.from_numpy(rays).cuda()
    x = model.encode(rays_t, rid_t, qobj_t, len(r)).cpu().numpy()
    xo = osph.encode(om, rays, r, ob)
    assert x.shape == xo.shape == (len(r), om.K)
    np.testing.assert_allclose(x, xo, atol=1e-4, rtol=0)


@pytest.mark.parametrize("kind", ["outer", "inner"])
@pytest.mark.parametrize("mlp_dt,tol", [("f32", 1e-4), ("f16", 2e-2), ("bf16", 6e-2)])
def test_spherical_logits_match_oracle(kind, mlp_dt, tol):
    rng, boxes, rays = _scene(seed=23)
    model, om = _model(kind, rng, boxes, mlp_dt=mlp_dt, grid_dt="f16" if mlp_dt != "f32" else "f32")
    r, ob, rid_t, qobj_t = _class_pairs(kind, rays, boxes)
    rays_t = torch.from_numpy(rays).cuda()
    goff = torch.tensor([0, len(r)], dtype=torch.int64, device="cuda")
    bits = nif.empty_bits(len(rays))
    z = model.infer_queries(rays_t, rid_t, qobj_t, goff, len(r), bits=bits)[:len(r)].cpu().numpy()
    model.check()
    zo = osph.forward(om, rays, r, ob)
    assert np.abs(zo).max() > 0.05
    assert np.abs(z - zo).max() <= tol, np.abs(z - zo).max()
    occ = nif.bits_to_bool(bits, len(rays)).cpu().numpy()
    assert np.array_equal(occ, onif.ray_occlusion(len(rays), r, z))


@pytest.mark.parametrize("kind", ["outer", "inner"])
def test_spherical_gradients_match_oracle(kind):
    rng, boxes, rays = _scene(seed=29, n_rays=20000)
    model, om = _model(kind, rng, boxes, width=32, n_hidden=2)
    r, ob, rid_t, qobj_t = _class_pairs(kind, rays, boxes)
    nq = len(r)
    y = (np.arange(nq) * 2654435761 >> 7) & 1
    rays_t = torch.from_numpy(rays).cuda()
    goff = torch.tensor([0, nq], dtype=torch.int64, device="cuda")
    g = model.grids.clone().requires_grad_(True)
    w = model.weights.clone().requires_grad_(True)
    z = nif.NifQueryFn.apply(g, w, model, rays_t, rid_t, qobj_t, goff, nq)
    loss = nif.NifLossFn.apply(z, torch.from_numpy(y.astype(np.uint8)).cuda())
    loss.backward()
    Lo, dnet, dgrids = osph.loss_and_grads(om, rays, r, ob, y.astype(np.float64))
    assert abs(float(loss.item()) - Lo) <= 1e-5 * max(1.0, Lo)
    gw = w.grad.cpu().numpy()
    want_w = np.concatenate([m.reshape(-1) for m in dnet])
    assert np.linalg.norm(gw - want_w) <= 1e-3 * np.linalg.norm(want_w)
    gg = g.grad.cpu().numpy().reshape(dgrids.shape)
    assert np.linalg.norm(gg - dgrids) <= 1e-3 * np.linalg.norm(dgrids)


def test_front_end_routes_classes_to_their_networks():
    """One class-mode front end bins every pair into outer and inner; each
    range goes to its own network (outer 2 x 64, inner 3 x 64 here) with its
    own encoding, and both match the oracle."""
    rng, boxes, rays = _scene(seed=31)
    outer, oo = _model("outer", rng, boxes, R=32, N=3, width=64, n_hidden=2, grid_dt="f16", mlp_dt="f16")
    inner, oi = _model("inner", rng, boxes, R=16, N=5, R1=16, N1=3, width=64, n_hidden=3, grid_dt="f16",
                       mlp_dt="f16")
    fe = nif.NifModel(nif.NifConfig(**{**outer.cfg.__dict__, "net_mode": L.NIF_NETS_CLASS}),
                      outer.obj_aabb, outer.grids, torch.cat([outer.weights, outer.weights]))
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, count = fe.frontend(rays_t)
    torch.cuda.synchronize()
    nq = int(count.item())
    g = goff.cpu().numpy()
    z_out = outer.infer_queries(rays_t, ray_id, qobj, goff, nq)
    z_in = inner.infer_queries(rays_t, ray_id, qobj, goff[1:], nq)
    outer.check()
    inner.check()
    r = ray_id[:nq].cpu().numpy().astype(np.int64)
    q = qobj[:nq].cpu().numpy().view(np.uint32)
    ob, inn = (q & 0x7FFFFFFF).astype(np.int64), (q >> 31).astype(bool)
    assert not inn[g[0]:g[1]].any() and inn[g[1]:g[2]].all() and g[1] > 500 and g[2] - g[1] > 500
    for zg, om, kind, a, b in ((z_out, oo, "outer", g[0], g[1]), (z_in, oi, "inner", g[1], g[2])):
        rr, oo_ = r[a:b], ob[a:b]
        keep = _conditioned(kind, rays, boxes, rr, oo_)
        assert keep.mean() > 0.8
        zo = osph.forward(om, rays, rr[keep], oo_[keep])
        assert np.abs(zg[a:b].cpu().numpy()[keep] - zo).max() <= 2e-2
    # the forward refuses a class-mode descriptor for a spherical encoding
    with pytest.raises(L.NifError):
        fe.infer_queries(rays_t, ray_id, qobj, goff, nq)
