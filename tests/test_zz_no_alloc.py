"""nif_infer_noalloc, the variant of nif_infer for callers that cannot
allocate device memory (a frame loop that must not allocate once running, a
plugin whose host application owns the GPU's memory): it must give exactly
the occlusion mask nif_infer gives with a caller-provided workspace, on two
calls in a row (the second call reuses the library's fixed scratch), and must
refuse work beyond its fixed capacity with a clear error.

Kept in its own file, named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth, workloads  # noqa: E402


def _noalloc(model, rays, bits, tlas=None):
    d = model.desc()
    return L.lib.nif_infer_noalloc(ctypes.byref(d), ctypes.c_void_p(tlas.buf.data_ptr()) if tlas else None,
                                   ctypes.c_void_p(rays.data_ptr()), int(rays.shape[0]),
                                   ctypes.c_void_p(bits.data_ptr()), nif._stream())


def _tiny_model(mlp_dtype):
    w = workloads.tiny_object(n_rays=20000, aimed=True, grid_scale=1.0)
    cfg = nif.NifConfig(res=w.res, n_features=2, log2_table=19, grid_dtype=L.NIF_F16,
                        n_hidden=3, width=64, mlp_dtype=mlp_dtype)
    flat = torch.from_numpy(synth.flatten_mlp(w.weights))
    flat = flat.half() if mlp_dtype == L.NIF_F16 else flat
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(),
                         torch.from_numpy(w.grid_values.reshape(-1)).half().cuda(), flat.cuda())
    return model, torch.from_numpy(w.rays).cuda(), None


def _multi_object_model():
    rng = np.random.default_rng(77)
    centres = rng.uniform(-4, 4, size=(12, 3))
    aabb = np.concatenate([centres - rng.uniform(0.5, 1.5, (12, 3)), centres + rng.uniform(0.5, 1.5, (12, 3))],
                          axis=1).astype(np.float32)
    res = [8, 16, 40, 100]
    cfg = nif.NifConfig(res=res, n_features=2, log2_table=14, grid_dtype=L.NIF_F16, n_hidden=3, width=64,
                        mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_CLASS)
    V = nif.NifModel.grid_vertices(cfg)
    grids = torch.from_numpy(rng.uniform(-1, 1, 12 * 2 * V * 2).astype(np.float32)).half().cuda()
    mats = np.concatenate([synth.flatten_mlp(synth.mlp_init(rng, cfg.K, 64, 3)) for _ in range(2)])
    model = nif.NifModel(cfg, torch.from_numpy(aabb).cuda(), grids, torch.from_numpy(mats).half().cuda())
    o = rng.uniform(-6, 6, size=(60000, 3))
    rays = synth.pack_rays(o, synth.unit_vectors(rng, 60000), 1e-3, np.inf)
    rays_t = torch.from_numpy(rays).cuda()
    return model, rays_t, nif.BVH.from_boxes(model.obj_aabb)


@pytest.mark.parametrize("case", ["tiny_f16", "tiny_f32", "objects_tlas"])
def test_noalloc_equals_workspace_path_on_two_calls(case):
    if case == "tiny_f16":
        model, rays, tlas = _tiny_model(L.NIF_F16)
    elif case == "tiny_f32":
        model, rays, tlas = _tiny_model(L.NIF_F32)
    else:
        model, rays, tlas = _multi_object_model()
    n = int(rays.shape[0])
    ref = nif.empty_bits(n)
    model.infer(rays, ref, tlas=tlas)
    model.check()
    torch.cuda.synchronize()
    ref_bool = nif.bits_to_bool(ref, n)
    assert bool(ref_bool.any()) and not bool(ref_bool.all())
    for _ in range(2):
        bits = nif.empty_bits(n)
        assert _noalloc(model, rays, bits, tlas) == L.NIF_OK, L.last_error()
        torch.cuda.synchronize()
        assert torch.equal(bits, ref)


def test_noalloc_rejects_work_beyond_its_scratch():
    model, rays, _ = _tiny_model(L.NIF_F16)
    d = model.desc()
    bits = nif.empty_bits(64)
    # far more rays than the fixed scratch can hold pairs for: refused before any launch
    st = L.lib.nif_infer_noalloc(ctypes.byref(d), None, ctypes.c_void_p(rays.data_ptr()), 1 << 30,
                                 ctypes.c_void_p(bits.data_ptr()), nif._stream())
    assert st == L.NIF_ERR_WORKSPACE
    assert "scratch" in L.last_error()
    assert L.lib.nif_infer_noalloc(ctypes.byref(d), None, None, 10, None, None) == L.NIF_ERR_ARG


def test_noalloc_first_call_matches_oracle():
    """The first call's mask against the FP64 oracle directly: every ray
    whose oracle logit is farther from 0 than the FP16 tolerance (2e-2) gets
    the oracle's decision (occluded iff z < 0)."""
    from oracle import nif as onif
    w = workloads.tiny_object(n_rays=20000, aimed=True, grid_scale=1.0)
    model, rays, _ = _tiny_model(L.NIF_F16)
    n = int(rays.shape[0])
    bits = nif.empty_bits(n)
    assert _noalloc(model, rays, bits) == L.NIF_OK, L.last_error()
    torch.cuda.synchronize()
    got = nif.bits_to_bool(bits, n).cpu().numpy()
    r, ob, inn = onif.queries(w.rays, w.aabb)
    grids = w.grid_values.astype(np.float16).astype(np.float64)
    nets = [synth.unflatten_mlp(synth.flatten_mlp(w.weights).astype(np.float16).astype(np.float64),
                                model.cfg.K, 64, 3)]
    om = onif.Model(res=w.res, F=2, log2_table=19, obj_aabb=w.aabb, grids=grids, nets=nets)
    z = onif.forward(om, w.rays, r, ob, inn)
    clear = np.abs(z) > 2e-2
    assert clear.sum() > 0.9 * len(z) and (z[clear] < 0).any() and (z[clear] > 0).any()
    want = np.zeros(n, bool)
    want[r[z < 0]] = True
    sure = np.zeros(n, bool)
    sure[np.setdiff1d(np.arange(n), r)] = True      # no pair: visible for certain
    sure[r[clear]] = True                            # one pair per ray here
    assert np.array_equal(got[sure], want[sure])


def test_noalloc_reports_pairs_beyond_its_scratch_after_the_call():
    """A ray count within the scratch whose pairs are not: 200,000 rays
    through the common core of 16 nested boxes make 3.2M pairs, more than
    the ~2.09M the scratch holds.  The call is not refused up front; the
    front end drops the pairs beyond capacity on the device and the call
    returns NIF_ERR_WORKSPACE naming the count found.  A call within
    capacity afterwards is exact again."""
    rng = np.random.default_rng(5)
    k = np.arange(16, dtype=np.float32)[:, None]
    aabb = np.concatenate([-(1.0 + k) * np.ones((16, 3), np.float32), (1.0 + k) * np.ones((16, 3), np.float32)],
                          axis=1).astype(np.float32)
    res = [4, 8]
    cfg = nif.NifConfig(res=res, n_features=2, log2_table=14, grid_dtype=L.NIF_F16, n_hidden=3, width=64,
                        mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_CLASS)
    V = nif.NifModel.grid_vertices(cfg)
    grids = torch.from_numpy(rng.uniform(-1, 1, 16 * 2 * V * 2).astype(np.float32)).half().cuda()
    mats = np.concatenate([synth.flatten_mlp(synth.mlp_init(rng, cfg.K, 64, 3)) for _ in range(2)])
    model = nif.NifModel(cfg, torch.from_numpy(aabb).cuda(), grids, torch.from_numpy(mats).half().cuda())
    n = 200_000
    o = synth.unit_vectors(rng, n) * 40.0
    rays = synth.pack_rays(o, -o / 40.0, 0.0, np.inf)     # every ray crosses all 16 boxes
    rays_t = torch.from_numpy(rays).cuda()
    bits = nif.empty_bits(n)
    st = _noalloc(model, rays_t, bits)
    assert st == L.NIF_ERR_WORKSPACE
    msg = L.last_error()
    assert "3200000" in msg and "incomplete" in msg
    # within capacity (100,000 rays, 1.6M pairs): equal to nif_infer
    half = rays_t[: n // 2].contiguous()
    ref = nif.empty_bits(n // 2)
    model.infer(half, ref, max_q=17 * (n // 2))
    model.check()
    got = nif.empty_bits(n // 2)
    assert _noalloc(model, half, got) == L.NIF_OK, L.last_error()
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
