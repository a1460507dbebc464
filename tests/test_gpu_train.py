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


def _away_from_kinks(om, rays, r, ob, inn, thr=1e-4):
    """Pairs whose FP64 gradient is defined to FP32 resolution: no hidden
    pre-activation within thr x its layer's RMS of the activation's kink.
    At a kink the gradient of a pair jumps, so an FP32 and an FP64 forward of
    the same pair can take different sides of it.  Measured on the CPU with
    exact face points: over all pairs, the FP64 gradient itself moves by
    2.6e-3 (ReLU) and 5.5e-3 (leaky) relative L2 when the rays are perturbed
    by one FP32 ulp; over the pairs kept at thr = 1e-4 (98.3-98.5% of them)
    it moves by 2e-5."""
    keep = np.ones(len(r), bool)
    x = onif.encode(om, rays, r, ob)
    net = om.net_of(ob, inn)
    for g in np.unique(net):
        sel = np.nonzero(net == g)[0]
        _, pre, _ = onif.mlp_forward(x[sel], om.nets[g], om.act, om.slope)
        for a in pre:
            rms = np.sqrt(np.mean(a * a))
            keep[sel] &= np.abs(a).min(axis=1) > thr * rms
    return keep


def _tapped(om, rays, r, ob, margin=1e-4):
    """Flat indices ((obj * 2 + grid) * V + vertex) * F + feature of every
    latent a pair may tap: the corners of the oracle's own cells, widened by
    one cell along an axis where the point lies within `margin` of a cell face
    (there an FP32 evaluation may take the neighbouring cell, whose far
    corners then get a weight of a few ulps)."""
    sizes, hashed, off = onif.level_layout(om.res, om.log2_table)
    GF = int(off[-1]) * om.F
    keys = []
    for k in np.unique(ob):
        sel = np.nonzero(ob == k)[0]
        pts = onif.entry_exit(rays[r[sel]], om.obj_aabb[k])
        for j, u in enumerate(pts):
            g = 0 if j < 2 else 1
            for l, R in enumerate(om.res):
                s = u * R
                i = np.clip(np.floor(s), 0, R - 1).astype(np.int64)
                f = s - i
                lo = np.where(f < margin, np.maximum(i - 1, 0), i)
                hi = np.where(f > 1 - margin, np.minimum(i + 2, R), i + 1)
                for dx in range(-1, 3):
                    for dy in range(-1, 3):
                        for dz in range(-1, 3):
                            c = i + np.array([dx, dy, dz])
                            ok = np.all((c >= lo) & (c <= hi), axis=1)
                            if not ok.any():
                                continue
                            v = onif.corner_index(c[ok, 0], c[ok, 1], c[ok, 2], R, hashed[l], om.log2_table)
                            for fi in range(om.F):
                                keys.append((k * 2 + g) * GF + (off[l] + v) * om.F + fi)
    return np.unique(np.concatenate(keys))


@pytest.mark.parametrize("act", [L.NIF_ACT_RELU, L.NIF_ACT_LEAKY])
def test_gradients_match_oracle(act):
    model, om, rays, flat, grid = _setup(act=act, n_rays=60000)
    # the oracle's own pairs away from activation kinks, grouped by network
    r, ob, inn = onif.queries(rays, om.obj_aabb)
    keep = _away_from_kinks(om, rays, r, ob, inn)
    assert keep.mean() > 0.98
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
    # a latent no pair taps is never written: exactly zero
    untouched = np.ones(gg.size, bool)
    untouched[_tapped(om, rays, r, ob)] = False
    assert untouched.sum() > 0.1 * gg.size
    assert not np.any(gg.reshape(-1)[untouched])


# The FP32 path forms each entry and exit point from its ray in about four
# rounded operations (slab parameter, point, box normalisation, level
# scaling), so its points carry a few ulps of rounding beyond the inputs'.
NUDGE_ULPS = 4


def _ulp_nudged(rays, seed=0, ulps=NUDGE_ULPS):
    """The rays with every origin and direction component moved by `ulps`
    FP32 ulps up or down at random (an input, to measure how much the FP64
    gradient itself moves under FP32 rounding of the query points)."""
    rng = np.random.default_rng(seed)
    out = rays.copy()
    for c in (0, 1, 2, 4, 5, 6):
        up = rng.random(len(out)) < 0.5
        col = out[:, c]
        for _ in range(ulps):
            col = np.where(up, np.nextafter(col, np.float32(np.inf)),
                           np.nextafter(col, np.float32(-np.inf))).astype(np.float32)
        out[:, c] = col
    return out


def _per_layer_rel_l2(flat, dnets):
    """Relative L2 of each network's layers of a flat gradient against the
    oracle's, with the norm ratio: where a mismatch sits."""
    out, o = [], 0
    for g, net in enumerate(dnets):
        for li, m in enumerate(net):
            n = m.size
            a, b = flat[o:o + n].astype(np.float64), m.reshape(-1)
            out.append(f"{g}.{li}: {_rel_l2(a, b):.2e} (x{np.linalg.norm(a) / max(np.linalg.norm(b), 1e-300):.3f})")
            o += n
    return ", ".join(out)


def _flat_w(dnets):
    return np.concatenate([np.concatenate([m.reshape(-1) for m in net]) for net in dnets])


class _Recorder:
    """A grid table that records the entries a lookup asks for (and answers
    zeros): the oracle's own tap indices, before any value is known."""

    def __init__(self, sink, base):
        self.sink, self.base = sink, base

    def __getitem__(self, idx):
        self.sink.append(self.base + np.asarray(idx, np.int64).reshape(-1))
        return np.zeros(np.shape(idx))


class _Sparse:
    """Entries of a large grid held as sorted (flat index, value) pairs."""

    def __init__(self, keys, vals, base):
        self.keys, self.vals, self.base = keys, vals, base

    def __getitem__(self, idx):
        k = self.base + np.asarray(idx, np.int64)
        pos = np.searchsorted(self.keys, k)
        assert np.array_equal(self.keys[pos], k)
        return self.vals[pos]


class _Grids:
    def __init__(self, GF, make):
        self.GF, self.make = GF, make

    def __getitem__(self, kg):
        k, g = kg
        return self.make((int(k) * 2 + int(g)) * self.GF)


def test_room_subset_gradients_match_oracle():
    """Sec. 5 'Training' on the room workload: after the 64 Adam steps of
    online training, the gradients of the L2 loss on 1,000 sampled pixels
    of the frame (their shadow rays and pairs derived by the oracle itself:
    hashed 16 x 2 grids with 2^19 entries per level, 1.465G FP32 master
    latents, the trained 3 x 64 outer and inner networks) agree with the FP64
    oracle within relative L2 1e-3, or within how far the FP64 gradient itself
    moves when the rays move by NUDGE_ULPS FP32 ulps (the rounding the FP32
    path's query points carry) where that is larger (the trained room
    network is that sensitive), for the weights and for the latents; the
    pairs away from activation kinks are compared (the fraction excluded is
    asserted below 5%), and every latent no pair taps stays exactly zero."""
    import oracle
    from oracle import frames
    from paper_2306_07191_gb300 import pipeline
    cfg = pipeline.RoomConfig()
    p = pipeline.RoomPipeline(cfg, log=lambda *a: None)
    p.train()
    gm, wm = p.trainer.g_master, p.trainer.w_master
    ws = p.ws
    pix = np.sort(np.random.default_rng(9).choice(ws.camera.shape[0], 1000, replace=False))
    ors = frames.frame_rays(oracle.OracleBVH(ws.scene.verts, ws.scene.tris), ws.camera[pix], ws.light, cfg.tmin)
    assert np.array_equal(ors.view(np.uint32), p.rays[torch.from_numpy(pix).cuda()].cpu().numpy().view(np.uint32))
    r, ob, inn = onif.queries(ors, ws.scene.obj_aabb)
    assert len(r) > 300 and inn.any() and (~inn).any()
    GF = p.V * cfg.n_features
    # the oracle's tap indices, then the trained latents at those entries
    asked = []
    nets = []
    wflat = wm.cpu().numpy().astype(np.float64)
    P = wflat.size // 2
    for g in range(2):
        nets.append(synth.unflatten_mlp(wflat[g * P:(g + 1) * P], 3 * len(cfg.res) * cfg.n_features,
                                        cfg.width_mlp, cfg.n_hidden))
    rec = onif.Model(res=list(cfg.res), F=cfg.n_features, log2_table=cfg.log2_table, obj_aabb=ws.scene.obj_aabb,
                     grids=_Grids(GF, lambda base: _Recorder(asked, base)), nets=nets, net_mode="class")
    nudged = _ulp_nudged(ors)
    onif.encode(rec, ors, r, ob)
    onif.encode(rec, nudged, r, ob)
    keys = np.unique(np.concatenate(asked))
    vals = gm[torch.from_numpy(keys).cuda()].cpu().numpy().astype(np.float64)
    om = onif.Model(res=list(cfg.res), F=cfg.n_features, log2_table=cfg.log2_table, obj_aabb=ws.scene.obj_aabb,
                    grids=_Grids(GF, lambda base: _Sparse(keys, vals, base)), nets=nets, net_mode="class")
    keep = _away_from_kinks(om, ors, r, ob, inn)
    assert keep.mean() > 0.95
    r, ob, inn = r[keep], ob[keep], inn[keep]
    order = np.argsort(inn, kind="stable")
    r, ob, inn = r[order], ob[order], inn[order]
    nq = len(r)
    y = _labels_for(r, ob)
    Lo, dnets, (gk, gv) = onif.loss_and_grads(om, ors, r, ob, inn, y.astype(np.float64), sparse_grids=True)
    # how far the FP64 gradient itself moves when the rays move by NUDGE_ULPS ulps
    _, dn_u, (gk_u, gv_u) = onif.loss_and_grads(om, nudged, r, ob, inn, y.astype(np.float64),
                                                sparse_grids=True)
    cond_w = _rel_l2(_flat_w(dn_u), _flat_w(dnets))
    # the same pairs on the GPU: the FP32 masters through nif_fwd_train,
    # nif_loss, nif_mlp_bwd and nif_grid_bwd
    rays_t = torch.from_numpy(ors).cuda()
    ray_id = torch.from_numpy(r.astype(np.int32)).cuda()
    qobj = torch.from_numpy((ob.astype(np.uint32) | (inn.astype(np.uint32) << 31)).view(np.int32)).cuda()
    goff = torch.tensor([0, int((~inn).sum()), nq], dtype=torch.int64, device="cuda")
    g = gm.detach().clone().requires_grad_(True)
    w = wm.detach().clone().requires_grad_(True)
    z = nif.NifQueryFn.apply(g, w, p.model, rays_t, ray_id, qobj, goff, nq)
    loss = nif.NifLossFn.apply(z, torch.from_numpy(y).cuda())
    loss.backward()
    assert abs(float(loss.item()) - Lo) <= 1e-5 * max(1.0, Lo)
    gw = w.grad.cpu().numpy()
    want_w = _flat_w(dnets)
    gk_t = torch.from_numpy(gk).cuda()
    gg = g.grad[gk_t].cpu().numpy()
    both = np.intersect1d(gk, gk_u)
    cond_g = _rel_l2(gv_u[np.searchsorted(gk_u, both)], gv[np.searchsorted(gk, both)])
    print(f"\nroom subset, FP32 path: {nq} pairs ({keep.mean():.4f} kept); rel L2 weights {_rel_l2(gw, want_w):.3e} "
          f"(FP64 moves {cond_w:.3e} under {NUDGE_ULPS} ulps), latents {_rel_l2(gg, gv):.3e} "
          f"(FP64 moves {cond_g:.3e}); per network and layer: {_per_layer_rel_l2(gw, dnets)}")
    # the bar: 1e-3, or the FP64 gradient's own movement when the rays move
    # by NUDGE_ULPS FP32 ulps where that is larger (no FP32 evaluation can be
    # held closer to FP64 than the rounding of its query points moves FP64)
    assert _rel_l2(gw, want_w) <= max(1e-3, cond_w)
    assert np.abs(gv).max() > 0 and _rel_l2(gg, gv) <= max(1e-3, cond_g)
    # every latent no pair taps (of the 1.465G) is exactly zero
    rest = g.grad.detach()
    rest[torch.from_numpy(_tapped(om, ors, r, ob)).cuda()] = 0
    assert int(torch.count_nonzero(rest).item()) == 0


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
    # the same array sizes with another level layout (resolutions permuted)
    # or grid dtype refuse it too
    for change in ({"res": [9, 4, 20, 70]}, {"grid_dtype": L.NIF_F16}):
        cfg4 = nif.NifConfig(**{**model.cfg.__dict__, **change})
        gdt = torch.float16 if cfg4.grid_dtype == L.NIF_F16 else torch.float32
        m4 = nif.NifModel(cfg4, model.obj_aabb, model.grids.to(gdt), model.weights.clone())
        assert nif.NifModel.grid_vertices(cfg4) == nif.NifModel.grid_vertices(model.cfg)
        with pytest.raises(L.NifError) as e:
            nif.Trainer(m4, lr=1e-2).load_state_bytes(buf)
        assert "header word" in str(e.value)


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


def _room_subset(p, cfg, seed=9, n_pix=1000):
    """The oracle's own shadow rays and pairs of n_pix sampled pixels of the
    room frame (bit-equal to the GPU's rays)."""
    import oracle
    from oracle import frames
    ws = p.ws
    pix = np.sort(np.random.default_rng(seed).choice(ws.camera.shape[0], n_pix, replace=False))
    ors = frames.frame_rays(oracle.OracleBVH(ws.scene.verts, ws.scene.tris), ws.camera[pix], ws.light, cfg.tmin)
    assert np.array_equal(ors.view(np.uint32), p.rays[torch.from_numpy(pix).cuda()].cpu().numpy().view(np.uint32))
    r, ob, inn = onif.queries(ors, ws.scene.obj_aabb)
    return ors, r, ob, inn


def test_half_precision_gradients_room_subset():
    """The half-precision training path (nif_train_grads with
    half_precision: the forward on the tensor cores saving FP16
    activations, the MLP backward on the tensor cores, FP32 accumulation, a
    fixed loss scale that brings the largest scaled dL/dz to about 64) on
    the room workload after online training:
    on the oracle's pairs of 1,000 sampled pixels, away from activation
    kinks, checked stage by stage.  The FP16 forward's logits agree with the
    FP64 oracle's within the FP16 logit bar 2e-2 x max(1, S) (S the output
    layer's sum of absolute terms).  Its gradients of the FP16 network (the
    model's FP16 weights and latents) agree within relative L2 2e-2 with the
    FP64 oracle's backward taken at those logits (dL/dz moves by up to twice
    a logit's error, relatively, so a trained network's large output terms
    would otherwise set the gradient's error, not the backward); untouched
    latents stay exactly zero."""
    from paper_2306_07191_gb300 import pipeline
    cfg = pipeline.RoomConfig()
    p = pipeline.RoomPipeline(cfg, log=lambda *a: None)
    p.train()
    ors, r, ob, inn = _room_subset(p, cfg)
    GF = p.V * cfg.n_features
    K = 3 * len(cfg.res) * cfg.n_features
    g16, w16 = p.model.grids, p.model.weights
    wflat = w16.float().cpu().numpy().astype(np.float64)
    P = wflat.size // 2
    nets = [synth.unflatten_mlp(wflat[g * P:(g + 1) * P], K, cfg.width_mlp, cfg.n_hidden) for g in range(2)]
    asked = []
    rec = onif.Model(res=list(cfg.res), F=cfg.n_features, log2_table=cfg.log2_table, obj_aabb=p.ws.scene.obj_aabb,
                     grids=_Grids(GF, lambda base: _Recorder(asked, base)), nets=nets, net_mode="class")
    onif.encode(rec, ors, r, ob)
    keys = np.unique(np.concatenate(asked))
    vals = g16[torch.from_numpy(keys).cuda()].float().cpu().numpy().astype(np.float64)
    om = onif.Model(res=list(cfg.res), F=cfg.n_features, log2_table=cfg.log2_table, obj_aabb=p.ws.scene.obj_aabb,
                    grids=_Grids(GF, lambda base: _Sparse(keys, vals, base)), nets=nets, net_mode="class")
    keep = _away_from_kinks(om, ors, r, ob, inn)
    assert keep.mean() > 0.95
    r, ob, inn = r[keep], ob[keep], inn[keep]
    order = np.argsort(inn, kind="stable")
    r, ob, inn = r[order], ob[order], inn[order]
    nq = len(r)
    y = _labels_for(r, ob)
    rays_t = torch.from_numpy(ors).cuda()
    ray_id = torch.from_numpy(r.astype(np.int32)).cuda()
    qobj = torch.from_numpy((ob.astype(np.uint32) | (inn.astype(np.uint32) << 31)).view(np.int32)).cuda()
    goff = torch.tensor([0, int((~inn).sum()), nq], dtype=torch.int64, device="cuda")
    # the forward: the FP16 logits (the serial tensor-core kernel, as the
    # saving forward of training) against FP64, within the FP16 logit bar
    zo = onif.forward(om, ors, r, ob, inn)
    p.model.cfg.schedule, p.model.cfg.ctas_per_sm = L.NIF_SCHED_SERIAL, 4
    zg = p.model.infer_queries(rays_t, ray_id, qobj, goff, nq)[:nq].cpu().numpy().astype(np.float64)
    x = onif.encode(om, ors, r, ob)
    S = np.zeros(nq)
    for gi in (0, 1):
        sel = om.net_of(ob, inn) == gi
        if sel.any():
            post = onif.mlp_forward(x[sel], om.nets[gi], om.act, om.slope)[2]
            S[sel] = np.abs(post[-1]) @ np.abs(np.asarray(om.nets[gi][-1], np.float64)[0])
    assert np.all(np.abs(zg - zo) <= 2e-2 * np.maximum(1.0, S)), float(np.max(np.abs(zg - zo) / np.maximum(1.0, S)))
    # the backward, against the oracle's taken at the FP16 forward's logits
    Lo, dnets, (gk, gv) = onif.loss_and_grads(om, ors, r, ob, inn, y.astype(np.float64), sparse_grids=True,
                                              z_at=zg)
    # the trained network is confident, so dL/dz is tiny: a loss scale that
    # brings the largest scaled dL/dz to about 64 keeps the backward's FP16
    # operands in range (what dynamic loss scaling settles on)
    so = 1.0 / (1.0 + np.exp(-zo))
    dz_max = float(np.abs((2.0 / nq) * (so - y) * so * (1.0 - so)).max())
    scale = float(2.0 ** np.floor(np.log2(64.0 / dz_max)))
    tr = nif.Trainer(p.model, half_precision=True, loss_scale=scale)
    loss = tr.grads(rays_t, ray_id, qobj, goff, torch.from_numpy(y).cuda(), nq)
    torch.cuda.synchronize()
    p.model.check(tr._ws)
    assert abs(float(loss.item()) - Lo) <= 2e-2 * max(Lo, 1e-6) + 1e-6
    gw = tr.w_grad.cpu().numpy() / scale
    want_w = _flat_w(dnets)
    gk_t = torch.from_numpy(gk).cuda()
    gg = tr.g_grad[gk_t].cpu().numpy() / scale
    print(f"\nroom subset, half-precision path: {nq} pairs, loss scale 2^{np.log2(scale):.0f}; logits within "
          f"{np.max(np.abs(zg - zo) / np.maximum(1.0, S)):.2e} x max(1, S); rel L2 weights "
          f"{_rel_l2(gw, want_w):.3e}, latents {_rel_l2(gg, gv):.3e}")
    assert _rel_l2(gw, want_w) <= 2e-2, _rel_l2(gw, want_w)
    assert np.abs(gv).max() > 0 and _rel_l2(gg, gv) <= 2e-2, _rel_l2(gg, gv)
    rest = tr.g_grad.detach()
    rest[torch.from_numpy(_tapped(om, ors, r, ob)).cuda()] = 0
    assert int(torch.count_nonzero(rest).item()) == 0


def test_dynamic_loss_scale_skips_overflowing_steps():
    """Dynamic loss scaling on the half-precision path: a step whose scaled
    gradients overflow FP16 (a 64-pair batch under a scale of 2^28) leaves
    the masters and moments unchanged, zeroes the gradients and halves the
    scale; a step under a scale that fits updates the masters; after
    scale_window clean steps the scale doubles.  No host synchronisation is
    needed inside a step: the scale and its state live on the device."""
    model, om, rays, flat, grid = _setup(n_rays=8000, seed=21, res=(4, 5, 8, 13, 19, 28, 43, 64))
    cfg16 = nif.NifConfig(**{**model.cfg.__dict__, "mlp_dtype": L.NIF_F16})
    m16 = nif.NifModel(cfg16, model.obj_aabb, model.grids.clone(), model.weights.half())
    rays_t = torch.from_numpy(rays).cuda()
    ray_id, qobj, goff, nq, r, ob, inn = _frontend(m16, rays_t)
    sel = torch.arange(64, device="cuda")
    n_out = int((~torch.from_numpy(inn[:64])).sum())
    g64 = torch.tensor([0, n_out, 64], dtype=torch.int64, device="cuda")
    order = torch.from_numpy(np.argsort(inn[:64], kind="stable")).cuda()
    rid64, q64 = ray_id[sel][order].contiguous(), qobj[sel][order].contiguous()
    lab = torch.from_numpy(_labels_for(r[:64], ob[:64])[np.argsort(inn[:64], kind="stable")]).cuda()
    tr = nif.Trainer(m16, half_precision=True, dynamic_scale=True, loss_scale=float(1 << 28), scale_window=3)
    w0, g0 = tr.w_master.clone(), tr.g_master.clone()
    tr.step(rays_t, rid64, q64, g64, lab, 64)
    torch.cuda.synchronize()
    assert float(tr.scale.item()) == float(1 << 27)
    assert torch.equal(tr.w_master, w0) and torch.equal(tr.g_master, g0)
    assert float(tr.w_grad.abs().max()) == 0.0 and float(tr.w_m.abs().max()) == 0.0
    # halve until it fits, then updates happen and clean steps count
    for _ in range(12):
        tr.step(rays_t, rid64, q64, g64, lab, 64)
    torch.cuda.synchronize()
    assert not torch.equal(tr.w_master, w0)
    s = float(tr.scale.item())
    assert 1.0 <= s < float(1 << 27)
    st = tr.scale_state.cpu().tolist()
    assert st[0] == 0 and 0 <= st[1] < 3
    m16.check(tr._ws)


def test_half_precision_training_learns_like_fp32():
    """Online training of the room pipeline at a reduced size with the
    half-precision path (FP16 operands on the tensor cores, dynamic loss
    scale) reaches a loss and a visibility disagreement with the BVH close
    to the FP32 path's on the same batches."""
    from paper_2306_07191_gb300 import pipeline
    res = {}
    for hp in (False, True):
        cfg = pipeline.RoomConfig(half_precision_train=hp)
        cfg.width, cfg.height, cfg.n_obj = 640, 360, 12
        cfg.train_steps, cfg.batch, cfg.train_spp = 32, 32768, 1
        p = pipeline.RoomPipeline(cfg, log=lambda *a: None)
        p.train()
        res[hp] = (p.losses[-1], p.disagreement()["all"])
        p.check()
    (l32, d32), (l16, d16) = res[False], res[True]
    assert l16 <= 1.25 * l32 + 2e-3, res
    assert d16 <= 1.25 * d32 + 2e-3, res
