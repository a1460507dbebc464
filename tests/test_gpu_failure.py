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
