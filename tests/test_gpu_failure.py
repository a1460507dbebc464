"""Failure detection without faulting the GPU: a bounded wait on a barrier
nothing arrives on expires, the kernel records NIF_ERR_TIMEOUT, the host reads
it with nif_check, and the context keeps working afterwards; device-side
capacity overflow is reported the same way."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth, workloads  # noqa: E402


def _check(ws):
    det = ctypes.c_int64()
    st = L.lib.nif_check(ctypes.c_void_p(ws.data_ptr()), ctypes.byref(det), nif._stream())
    return st, det.value


def test_bounded_wait_expires_and_reports_timeout():
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    assert _check(ws) == (L.NIF_OK, 0)
    # ~1 ms at 2 GHz: the wait gives up, records the timeout and returns
    st = L.lib.nif_wait_selftest(ctypes.c_void_p(ws.data_ptr()), 256, 2_000_000, nif._stream())
    assert st == L.NIF_OK
    torch.cuda.synchronize()
    assert _check(ws) == (L.NIF_ERR_TIMEOUT, 42)
    # nif_check cleared the error word
    assert _check(ws) == (L.NIF_OK, 0)
    # the context is still usable: a normal query afterwards works
    w = workloads.tiny_object(n_rays=512, aimed=True)
    bvh = nif.BVH(torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.tris).cuda())
    bits = bvh.cast_shadow(torch.from_numpy(w.rays).cuda())
    torch.cuda.synchronize()
    assert bool(nif.bits_to_bool(bits, 512).any())
    assert L.lib.nif_wait_selftest(ctypes.c_void_p(ws.data_ptr()), 256, -1, nif._stream()) == L.NIF_ERR_ARG


def test_pair_capacity_overflow_is_reported():
    w = workloads.tiny_object(n_rays=4000, aimed=True)
    cfg = nif.NifConfig(res=w.res, n_features=2, mlp_dtype=L.NIF_F16)
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(),
                         torch.from_numpy(w.grid_values.reshape(-1)).cuda(),
                         torch.from_numpy(synth.flatten_mlp(w.weights)).half().cuda())
    rays = torch.from_numpy(w.rays).cuda()
    # every aimed ray makes one pair: room for only 100 of them
    ray_id, qobj, goff, count = model.frontend(rays, max_q=100)
    torch.cuda.synchronize()
    with pytest.raises(L.NifError) as e:
        model.check()
    assert e.value.code == L.NIF_ERR_WORKSPACE
    assert int(count.item()) == 4000  # pairs found
    assert int(goff[-1].item()) == 100  # pairs kept


def _tiny_model(mlp_dt, schedule, n_rays=4000):
    w = workloads.tiny_object(n_rays=n_rays, aimed=True, grid_scale=0.5)
    half = mlp_dt == L.NIF_F16
    cfg = nif.NifConfig(res=w.res, n_features=2, mlp_dtype=mlp_dt, schedule=schedule,
                        grid_dtype=L.NIF_F16 if half else L.NIF_F32)
    tdt = torch.float16 if half else torch.float32
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(),
                         torch.from_numpy(w.grid_values.reshape(-1)).to(tdt).cuda(),
                         torch.from_numpy(synth.flatten_mlp(w.weights)).to(tdt).cuda())
    return model, torch.from_numpy(w.rays).cuda()


@pytest.mark.parametrize("mlp_dt,schedule", [(L.NIF_F32, L.NIF_SCHED_AUTO), (L.NIF_F16, L.NIF_SCHED_SERIAL),
                                             (L.NIF_F16, L.NIF_SCHED_PIPELINED)])
def test_out_of_range_queries_are_skipped_and_reported(mlp_dt, schedule):
    """A query naming an object id >= n_obj or a ray id >= n_rays is skipped
    before it touches memory: NIF_ERR_BOUNDS with its index, logit 0, no bit;
    every other query gives the logit and bit it gives without them."""
    model, rays = _tiny_model(mlp_dt, schedule)
    n = int(rays.shape[0])
    ray_id, qobj, goff, count = model.frontend(rays)
    torch.cuda.synchronize()
    nq = int(count.item())
    assert nq > 3000
    z_ref = model.infer_queries(rays, ray_id, qobj, goff, nq)[:nq].clone()
    model.check()
    bad_obj, bad_ray = 1234, 2345
    qobj[bad_obj] = 7                 # one object in the scene
    ray_id[bad_ray] = n + 100
    bits = nif.empty_bits(n)
    z = model.infer_queries(rays, ray_id, qobj, goff, nq, bits=bits)[:nq]
    torch.cuda.synchronize()
    with pytest.raises(L.NifError) as e:
        model.check()
    assert e.value.code == L.NIF_ERR_BOUNDS
    model.check()  # the error word was cleared
    keep = torch.ones(nq, dtype=torch.bool, device="cuda")
    keep[[bad_obj, bad_ray]] = False
    assert torch.equal(z[keep], z_ref[keep])
    assert float(z[bad_obj]) == 0.0 and float(z[bad_ray]) == 0.0
    rid = ray_id[:nq].long()
    want = torch.zeros(n, dtype=torch.bool, device="cuda")
    want[rid[keep & (z_ref < 0)]] = True
    assert torch.equal(nif.bits_to_bool(bits, n), want)
    assert bool(want.any())


def test_non_finite_parameter_after_adam_is_reported():
    """A NaN planted on the host in one grid master (as a diverging run would
    leave it) makes the Adam update non-finite: the train step records
    NIF_ERR_NUMERIC with the parameter's index instead of passing silently."""
    w = workloads.tiny_object(n_rays=4000, aimed=True, grid_scale=0.5)
    cfg = nif.NifConfig(res=w.res, n_features=2, mlp_dtype=L.NIF_F32)
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(), torch.from_numpy(w.grid_values.reshape(-1)).cuda(),
                         torch.from_numpy(synth.flatten_mlp(w.weights)).cuda())
    rays = torch.from_numpy(w.rays).cuda()
    ray_id, qobj, goff, count = model.frontend(rays)
    torch.cuda.synchronize()
    nq = int(count.item())
    lab = (torch.arange(nq, device="cuda") % 2).to(torch.uint8)
    tr = nif.Trainer(model, lr=1e-3)
    tr.step(rays, ray_id[:nq], qobj[:nq], goff, lab, nq)
    model.check(tr._ws)
    tr.g_master[12345] = float("nan")
    tr.step(rays, ray_id[:nq], qobj[:nq], goff, lab, nq)
    torch.cuda.synchronize()
    det = ctypes.c_int64()
    st = L.lib.nif_check(ctypes.c_void_p(tr._ws.data_ptr()), ctypes.byref(det), nif._stream())
    assert st == L.NIF_ERR_NUMERIC and det.value == 12345
