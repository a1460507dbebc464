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


# ------------------------------------------------------------ BVH status
def _box_nodes_buffer(bvh, both_children_hit):
    """A copy of a built BVH buffer whose root node is rewritten into a cycle
    (host-side fault injection): child 0 is the root itself with the box
    [-10, 10]^3; child 1 is the root too (both_children_hit: every visit
    pushes, so the 96-entry stack fills) or a leaf behind a box no ray meets
    (the walk loops on child 0 until the node-visit bound).  Every read stays
    inside the root node."""
    buf = bvh.buf.cpu().numpy().copy()
    off = int(buf[32:40].view(np.int64)[0])
    buf[24:28] = np.array([0], np.int32).view(np.uint8)             # root = node 0
    node = buf[off:off + 64]
    f = node[0:48].view(np.float32)
    d = node[48:64].view(np.int32)
    big = [-10.0, 10.0]
    f[0:4] = big + big                                                # child 0: x, y
    f[8:10] = big                                                     # child 0: z
    if both_children_hit:
        f[4:8] = big + big
        f[10:12] = big
        d[0:2] = [0, 0]
    else:
        f[4:8] = [1e30, 2e30, 1e30, 2e30]
        f[10:12] = [1e30, 2e30]
        d[0:2] = [0, ~((0 << 3) | 0)]
    out = torch.from_numpy(buf).cuda()
    b2 = nif.BVH.__new__(nif.BVH)
    b2.buf, b2.n, b2._inputs = out, bvh.n, None
    return b2


@pytest.mark.parametrize("both,code", [(True, L.NIF_ERR_BOUNDS), (False, L.NIF_ERR_TIMEOUT)])
def test_bvh_traversal_failures_are_reported(both, code):
    """A cast through a cyclic tree (planted on the host) does not return a
    silent "no hit": the overflowing stack or the exhausted visit bound is
    recorded in the buffer's status and bvh_check reports it; a cast through
    a sound tree stays clean."""
    w = workloads.tiny_object(n_rays=64, aimed=True)
    v, t = torch.from_numpy(w.verts).cuda(), torch.from_numpy(w.tris).cuda()
    good = nif.BVH(v, t)
    rays = synth.pack_rays(np.array([[0.0, 0.0, -15.0]] * 32), np.array([[0.0, 0.0, 1.0]] * 32), 0.0, 30.0)
    r = torch.from_numpy(rays).cuda()
    good.cast_shadow(r)
    good.check()
    bad = _box_nodes_buffer(good, both)
    bad.check()                       # nothing recorded before a cast
    bad.cast_shadow(r)
    torch.cuda.synchronize()
    with pytest.raises(L.NifError) as e:
        bad.check()
    assert e.value.code == code
    # sticky until rebuilt; the sound tree and the context are unaffected
    with pytest.raises(L.NifError):
        bad.check()
    bits = good.cast_shadow(torch.from_numpy(w.rays).cuda())
    torch.cuda.synchronize()
    good.check()
    assert bool(nif.bits_to_bool(bits, 64).any())


def test_front_end_top_level_failure_is_reported():
    """The NIF front end's top-level walk through a cyclic tree records
    NIF_ERR_TIMEOUT in the call's error word instead of dropping pairs."""
    w = workloads.tiny_object(n_rays=256, aimed=True)
    cfg = nif.NifConfig(res=w.res, n_features=2, mlp_dtype=L.NIF_F16)
    boxes = torch.from_numpy(np.concatenate([w.aabb, w.aabb + 3.0])).cuda()
    model = nif.NifModel(cfg, boxes, torch.from_numpy(np.tile(w.grid_values.reshape(-1), 2)).cuda(),
                         torch.from_numpy(synth.flatten_mlp(w.weights)).half().cuda())
    tlas = nif.BVH.from_boxes(boxes)
    bad = _box_nodes_buffer(tlas, False)
    rays = synth.pack_rays(np.array([[0.0, 0.0, -15.0]] * 32), np.array([[0.0, 0.0, 1.0]] * 32), 0.0, 30.0)
    model.frontend(torch.from_numpy(rays).cuda(), tlas=bad)
    torch.cuda.synchronize()
    with pytest.raises(L.NifError) as e:
        model.check()
    assert e.value.code == L.NIF_ERR_TIMEOUT
