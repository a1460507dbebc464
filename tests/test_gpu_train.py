"""GPU training path (nif_fwd_train, nif_loss, nif_mlp_bwd, nif_grid_bwd,
nif_adam, nif_train_step and the torch.autograd.Function around them) against
the FP64 oracle's gradients and Adam, plus what training gains."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import nif as onif  # noqa: E402
from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth  # noqa: E402
from helpers import random_boxes_scene  # noqa: E402


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _labels_for(ray_id, obj):
    """A fixed pseudo-random 0/1 label per (ray, object) pair (an input)."""
    k = (np.asarray(ray_id, np.uint64) * np.uint64(2654435761) + np.asarray(obj, np.uint64) * np.uint64(97))
    return ((k >> np.uint64(7)) & np.uint64(1)).astype(np.uint8)


def _setup(seed=41, n_obj=4, res=(4, 9, 20, 70), log2=12, n_rays=24000, width=64, n_hidden=3,
           act=L.NIF_ACT_RELU):
    rng = np.random.default_rng(seed)
    boxes = random_boxes_scene(rng, n_obj=n_obj)
    sizes, hashed, off = onif.level_layout(list(res), log2)
    V = int(off[-1])
    F = 2
    grid = rng.uniform(-1, 1, size=(n_obj, 2, V * F)).astype(np.float32)
    K = 3 * len(res) * F
    mats = [synth.mlp_init(rng, K, width, n_hidden) for _ in range(2)]
    flat = np.concatenate([synth.flatten_mlp(m) for m in mats]).astype(np.float32)
    o = rng.uniform(-4, 4, size=(n_rays, 3))
    rays = synth.pack_rays(o, synth.unit_vectors(rng, n_rays), 1e-3, np.inf)
    cfg = nif.NifConfig(res=list(res), n_features=F, log2_table=log2, grid_dtype=L.NIF_F32,
                        n_hidden=n_hidden, width=width, act=act, mlp_dtype=L.NIF_F32,
                        net_mode=L.NIF_NETS_CLASS)
    model = nif.NifModel(cfg, torch.from_numpy(boxes).cuda(), torch.from_numpy(grid.reshape(-1)).cuda(),
                         torch.from_numpy(flat).cuda())
    om = onif.Model(res=list(res), F=F, log2_table=log2, obj_aabb=boxes,
                    grids=grid.astype(np.float64),
                    nets=[[np.asarray(w, np.float64) for w in m] for m in mats], net_mode="class",
                    act="relu" if act == L.NIF_ACT_RELU else "leaky")
    return model, om, rays, flat, grid


def _frontend(model, rays_t):
    ray_id, qobj, goff, count = model.frontend(rays_t)
    torch.cuda.synchronize()
    nq = int(count.item())
    r = ray_id[:nq].cpu().numpy().astype(np.int64)
    q = qobj[:nq].cpu().numpy().view(np.uint32)
    return ray_id[:nq].contiguous(), qobj[:nq].contiguous(), goff, nq, r, (q & 0x7FFFFFFF).astype(np.int64), (q >> 31).astype(bool)


def _well_conditioned(om, rays, r, ob, inn):
    """Pairs whose FP64 gradient is defined to FP32 resolution: the entry and
    exit points move < 1e-4 under a 1e-6 relative perturbation of the ray (a
    segment grazing a box face is ill-conditioned), and no hidden
    pre-activation lies within 1e-3 of its layer's RMS of a ReLU kink."""
    keep = np.ones(len(r), bool)
    rng = np.random.default_rng(0)
    for k in np.unique(ob):
        sel = np.nonzero(ob == k)[0]
        a = onif.entry_exit(rays[r[sel]], om.obj_aabb[k])
        pr = rays[r[sel]].astype(np.float64).copy()
        pr[:, 0:3] *= 1 + 1e-6 * rng.standard_normal((len(sel), 3))
        pr[:, 4:7] *= 1 + 1e-6 * rng.standard_normal((len(sel), 3))
        b = onif.entry_exit(pr, om.obj_aabb[k])
        dev = np.maximum(np.abs(a[0] - b[0]).max(1), np.abs(a[1] - b[1]).max(1))
        keep[sel] &= dev < 1e-4
    x = onif.encode(om, rays, r, ob)
    net = om.net_of(ob, inn)
    for g in np.unique(net):
        sel = np.nonzero(net == g)[0]
        _, pre, _ = onif.mlp_forward(x[sel], om.nets[g], om.act, om.slope)
        for a in pre:
            rms = np.sqrt(np.mean(a * a))
            keep[sel] &= np.abs(a).min(axis=1) > 1e-3 * rms
    return keep


@pytest.mark.parametrize("act", [L.NIF_ACT_RELU, L.NIF_ACT_LEAKY])
def test_gradients_match_oracle(act):
    model, om, rays, flat, grid = _setup(act=act, n_rays=60000)
    # the oracle's own pairs, restricted to well-conditioned ones, grouped by network
    r, ob, inn = onif.queries(rays, om.obj_aabb)
    keep = _well_conditioned(om, rays, r, ob, inn)
    r, ob, inn = r[keep], ob[keep], inn[keep]
    order = np.argsort(inn, kind="stable")
    r, ob, inn = r[order], ob[order], inn[order]
    nq = len(r)
    assert nq > 2000 and inn.any() and (~inn).any()
    y = _labels_for(r, ob)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id = torch.from_numpy(r.astype(np.int32)).cuda()
    qobj = torch.from_numpy((ob.astype(np.uint32) | (inn.astype(np.uint32) << 31)).view(np.int32)).cuda()
    n_out = int((~inn).sum())
    goff = torch.tensor([0, n_out, nq], dtype=torch.int64, device="cuda")
    g = model.grids.clone().requires_grad_(True)
    w = model.weights.clone().requires_grad_(True)
    z = nif.NifQueryFn.apply(g, w, model, rays_t, ray_id, qobj, goff, nq)
    loss = nif.NifLossFn.apply(z, torch.from_numpy(y).cuda())
    loss.backward()
    Lo, dnets, dgrids = onif.loss_and_grads(om, rays, r, ob, inn, y.astype(np.float64))
    assert abs(float(loss.item()) - Lo) <= 1e-5 * max(1.0, Lo)
    gw = w.grad.cpu().numpy()
    want_w = np.concatenate([np.concatenate([m.reshape(-1) for m in net]) for net in dnets])
    assert _rel_l2(gw, want_w) <= 1e-3
    gg = g.grad.cpu().numpy().reshape(dgrids.shape)
    assert _rel_l2(gg, dgrids) <= 1e-3
    # latents the FP64 oracle leaves at exactly zero (no tap, or a point exactly
    # on a cell face, whose far-side weight is 0 in FP64 and an ulp in FP32)
    # get at most rounding-level values
    assert np.abs(gg[dgrids == 0]).max() <= 1e-4 * np.abs(dgrids).max()


def test_adam_matches_oracle_step_by_step():
    rng = np.random.default_rng(3)
    n = 100003
    th = rng.normal(size=n).astype(np.float32)
    grads = [rng.normal(size=n).astype(np.float32) * s for s in (1.0, 0.1, 0.0)]
    grads[1][:50] = 0
    t_th = torch.from_numpy(th).cuda()
    m1 = torch.zeros_like(t_th)
    m2 = torch.zeros_like(t_th)
    copy = torch.empty(n, dtype=torch.float16, device="cuda")
    oth, om1, om2 = th.astype(np.float64), np.zeros(n), np.zeros(n)
    for step, gr in enumerate(grads, start=1):
        t_g = torch.from_numpy(gr).cuda()
        nif.adam_(t_th, t_g, m1, m2, step, 1e-2, copy=copy, copy_dtype=L.NIF_F16)
        oth, om1, om2 = onif.adam_step(oth, gr, om1, om2, step, 1e-2)
        torch.cuda.synchronize()
        assert float(t_g.abs().max()) == 0.0  # gradient zeroed after use
        np.testing.assert_allclose(t_th.cpu().numpy(), oth, rtol=0, atol=1e-5)
        np.testing.assert_allclose(copy.float().cpu().numpy(), oth, rtol=1e-3, atol=1e-3)


def test_train_step_reduces_loss_and_beats_untrained_net():
    model, om, rays, flat, grid = _setup(n_rays=20000, seed=5)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _frontend(model, rays_t)
    y = _labels_for(r, ob)
    # make the labels learnable: a label that depends on the ray direction only
    d = rays[r, 4:7]
    y = (d[:, 0] + 0.3 * d[:, 1] > 0).astype(np.uint8)
    lab = torch.from_numpy(y).cuda()
    tr = nif.Trainer(model, lr=1e-2)
    losses = []
    for _ in range(40):
        losses.append(float(tr.step(rays_t, ray_id, qobj, goff, lab, nq).item()))
    model.check(tr._ws)
    assert losses[-1] < 0.5 * losses[0], losses[::5]
    z = model.infer_queries(rays_t, ray_id, qobj, goff, nq)
    acc = float(((z[:nq] >= 0).cpu().numpy() == (y == 1)).mean())
    assert acc > 0.9, acc
    # the trained master weights were copied into the model
    assert torch.equal(model.weights, tr.w_master)


def test_checkpoint_resume_restores_state_and_continues():
    """nif_state_save / nif_state_load: a fresh trainer loaded from a
    checkpoint holds the same masters, moments and step and the same model
    copies, and the next steps of both runs agree (to FP32 atomic-order
    rounding of the gradient sums)."""
    model, om, rays, flat, grid = _setup(n_rays=8000, seed=7)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _frontend(model, rays_t)
    lab = torch.from_numpy(_labels_for(r, ob)).cuda()
    tr = nif.Trainer(model, lr=1e-2)
    for _ in range(5):
        tr.step(rays_t, ray_id, qobj, goff, lab, nq)
    buf = tr.state_bytes()
    # a second model and trainer from the initial values
    model2 = nif.NifModel(model.cfg, model.obj_aabb, torch.from_numpy(grid.reshape(-1)).cuda(),
                          torch.from_numpy(flat).cuda())
    tr2 = nif.Trainer(model2, lr=1e-2)
    tr2.load_state_bytes(buf)
    assert tr2.o.step == tr.o.step == 5
    for name in ("w_master", "w_m", "w_v", "g_master", "g_m", "g_v"):
        assert torch.equal(getattr(tr, name), getattr(tr2, name)), name
    assert torch.equal(model.weights, model2.weights) and torch.equal(model.grids, model2.grids)
    assert float(tr2.w_grad.abs().max()) == 0.0 and float(tr2.g_grad.abs().max()) == 0.0
    for _ in range(3):
        tr.step(rays_t, ray_id, qobj, goff, lab, nq)
        tr2.step(rays_t, ray_id, qobj, goff, lab, nq)
    torch.cuda.synchronize()
    for name in ("w_master", "g_master"):
        a, b = getattr(tr, name), getattr(tr2, name)
        assert float((a - b).abs().max()) <= 1e-5 * max(1.0, float(a.abs().max())), name
    # a model of another shape refuses the checkpoint
    other = nif.NifModel(nif.NifConfig(**{**model.cfg.__dict__, "width": 32}), model.obj_aabb, model.grids,
                         torch.zeros(nif.NifModel.weight_count(nif.NifConfig(**{**model.cfg.__dict__, "width": 32})) * 2,
                                     device="cuda"))
    tr3 = nif.Trainer(other, lr=1e-2)
    with pytest.raises(L.NifError):
        tr3.load_state_bytes(buf)


def test_deterministic_steps_repeat_and_resume_bit_for_bit():
    """With deterministic gradients (tile-ordered weight sums, per-latent sums
    in pair order after a stable sort) two runs from the same state give the
    same bits, a run resumed from a checkpoint continues bit for bit, and the
    gradients equal the atomic path's up to summation order."""
    model, om, rays, flat, grid = _setup(n_rays=8000, seed=9)
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _frontend(model, rays_t)
    lab = torch.from_numpy(_labels_for(r, ob)).cuda()

    def fresh(det=True):
        m = nif.NifModel(model.cfg, model.obj_aabb, torch.from_numpy(grid.reshape(-1)).cuda(),
                         torch.from_numpy(flat).cuda())
        return nif.Trainer(m, lr=1e-2, deterministic=det)

    def same(a, b):
        return all(torch.equal(getattr(a, k), getattr(b, k))
                   for k in ("w_master", "w_m", "w_v", "g_master", "g_m", "g_v"))

    t1, t2 = fresh(), fresh()
    for _ in range(4):
        t1.step(rays_t, ray_id, qobj, goff, lab, nq)
        t2.step(rays_t, ray_id, qobj, goff, lab, nq)
    torch.cuda.synchronize()
    assert same(t1, t2)
    buf = t1.state_bytes()
    for _ in range(3):
        t1.step(rays_t, ray_id, qobj, goff, lab, nq)
    t3 = fresh()
    t3.load_state_bytes(buf)
    for _ in range(3):
        t3.step(rays_t, ray_id, qobj, goff, lab, nq)
    torch.cuda.synchronize()
    t1.model.check(t1._ws)
    assert same(t1, t3)
    assert torch.equal(t1.model.weights, t3.model.weights) and torch.equal(t1.model.grids, t3.model.grids)
    # one step each way from the same state: the same update up to summation order
    ta, tb = fresh(True), fresh(False)
    ta.step(rays_t, ray_id, qobj, goff, lab, nq)
    tb.step(rays_t, ray_id, qobj, goff, lab, nq)
    torch.cuda.synchronize()
    for k in ("w_m", "g_m"):
        a, b = getattr(ta, k), getattr(tb, k)
        assert float((a - b).abs().max()) <= 1e-6 * max(1e-12, float(b.abs().max())) + 1e-12, k
    assert float(ta.g_m.abs().max()) > 0 and float(ta.w_m.abs().max()) > 0
