"""nif_mlp_infer, the inference stage alone (the network over encoded
inputs, the paper's separate "Inference" kernel), against the FP64 oracle's
MLP: FP16 and BF16 operands, one network and class networks, ragged tails;
and the two-kernel path (nif_encode, then nif_mlp_infer) against the fused
query on the same pairs."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import nif as onif  # noqa: E402
from paper_2306_07191_gb300 import _lib as L  # noqa: E402
from paper_2306_07191_gb300 import nif, synth, workloads  # noqa: E402

TOL = {L.NIF_F16: 2e-2, L.NIF_BF16: 6e-2}
TDT = {L.NIF_F16: torch.float16, L.NIF_BF16: torch.bfloat16}


def _mlp_infer(model, x, goff, nq):
    z = torch.full((nq,), float("nan"), dtype=torch.float32, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    d = model.desc()
    L.call("nif_mlp_infer", ctypes.byref(d), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(goff.data_ptr()), nq,
           ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(), nif._stream())
    torch.cuda.synchronize()
    model.check(ws)
    return z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("dt", [L.NIF_F16, L.NIF_BF16])
@pytest.mark.parametrize("levels,n_nets,nq", [(8, 1, 5003), (16, 2, 9001), (4, 2, 300), (16, 2, 70001)])
def test_mlp_infer_matches_oracle(dt, levels, n_nets, nq, tile_m):
    """Both tile shapes: 128-row tiles (rows as the MMA's M) and 256-row
    tiles (rows as its N, features as its M); group boundaries inside tiles,
    ragged tails, and enough tiles for every CTA to run several."""
    rng = np.random.default_rng(levels * 10 + n_nets)
    res = list(workloads.ROOM_RES[:levels]) if levels > 8 else list(workloads.TINY_RES[:levels])
    cfg = nif.NifConfig(res=res, n_features=2, log2_table=19, grid_dtype=L.NIF_F16, n_hidden=3, width=64,
                        mlp_dtype=dt, net_mode=L.NIF_NETS_CLASS if n_nets == 2 else L.NIF_NETS_SINGLE,
                        tile_m=tile_m)
    K = cfg.K
    mats = [synth.mlp_init(rng, K, 64, 3) for _ in range(n_nets)]
    flat = torch.from_numpy(np.concatenate([synth.flatten_mlp(m) for m in mats])).to(TDT[dt]).cuda()
    V = nif.NifModel.grid_vertices(cfg)
    model = nif.NifModel(cfg, torch.zeros((1, 6), device="cuda"),
                         torch.zeros(2 * V * 2, dtype=torch.float16, device="cuda"), flat)
    x = torch.from_numpy(rng.uniform(-1, 1, size=(nq, K)).astype(np.float32)).to(TDT[dt]).cuda()
    split = nq // 3 if n_nets == 2 else nq
    goff = torch.tensor([0, split, nq][: n_nets + 1], dtype=torch.int64, device="cuda")
    z = _mlp_infer(model, x, goff, nq)
    x64 = x.float().cpu().numpy().astype(np.float64)
    wq = flat.float().cpu().numpy().astype(np.float64)
    P = wq.size // n_nets
    want = np.empty(nq)
    bounds = [0, split, nq] if n_nets == 2 else [0, nq]
    for g in range(n_nets):
        net = synth.unflatten_mlp(wq[g * P:(g + 1) * P], K, 64, 3)
        a, b = bounds[g], bounds[g + 1]
        want[a:b] = onif.mlp_forward(x64[a:b], net)[0]
    assert np.isfinite(z).all()
    assert np.abs(want).max() > 0.1
    assert np.abs(z - want).max() <= TOL[dt], np.abs(z - want).max()


def test_encode_then_mlp_equals_fused_query():
    """The paper's two-stage form (Grid kernel writing FP16 inputs, then the
    Inference kernel) against the fused kernel on the same pairs: the inputs
    are FP16 values interpolated in FP32 (Grid) or in FP16 (fused), so the
    logits agree within the FP16 rounding of the inputs."""
    w = workloads.tiny_object(n_rays=20000, aimed=True, grid_scale=1.0)
    cfg = nif.NifConfig(res=w.res, n_features=2, log2_table=19, grid_dtype=L.NIF_F16, n_hidden=3, width=64,
                        mlp_dtype=L.NIF_F16)
    model = nif.NifModel(cfg, torch.from_numpy(w.aabb).cuda(),
                         torch.from_numpy(w.grid_values.reshape(-1)).half().cuda(),
                         torch.from_numpy(synth.flatten_mlp(w.weights)).half().cuda())
    rays = torch.from_numpy(w.rays).cuda()
    ray_id, qobj, goff, count = model.frontend(rays)
    torch.cuda.synchronize()
    nq = int(count.item())
    fused = model.infer_queries(rays, ray_id, qobj, goff, nq)[:nq].cpu().numpy()
    x = model.encode(rays, ray_id, qobj, nq, dtype=L.NIF_F16)
    two = _mlp_infer(model, x, goff, nq)
    assert nq > 10000
    assert np.abs(two - fused).max() <= 1e-2, np.abs(two - fused).max()


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("n_hidden", [1, 2, 4])
def test_mlp_infer_leaky_depths(n_hidden, tile_m):
    """Leaky ReLU (the paper's activation for its own encoding, Sec. 5) at
    1, 2 and 4 hidden layers, K = 24 (padded to 32 inside the kernel), two
    networks whose boundary falls inside a tile."""
    rng = np.random.default_rng(100 + n_hidden)
    nq = 12345
    res = list(workloads.TINY_RES[:4])
    slope = 0.05
    cfg = nif.NifConfig(res=res, n_features=2, log2_table=19, grid_dtype=L.NIF_F16, n_hidden=n_hidden, width=64,
                        mlp_dtype=L.NIF_F16, net_mode=L.NIF_NETS_CLASS, act=L.NIF_ACT_LEAKY, leaky_slope=slope,
                        tile_m=tile_m)
    K = cfg.K
    assert K == 24
    mats = [synth.mlp_init(rng, K, 64, n_hidden) for _ in range(2)]
    flat = torch.from_numpy(np.concatenate([synth.flatten_mlp(m) for m in mats])).half().cuda()
    V = nif.NifModel.grid_vertices(cfg)
    model = nif.NifModel(cfg, torch.zeros((1, 6), device="cuda"),
                         torch.zeros(2 * V * 2, dtype=torch.float16, device="cuda"), flat)
    x = torch.from_numpy(rng.uniform(-1, 1, size=(nq, K)).astype(np.float32)).half().cuda()
    split = 4999
    goff = torch.tensor([0, split, nq], dtype=torch.int64, device="cuda")
    z = _mlp_infer(model, x, goff, nq)
    x64 = x.float().cpu().numpy().astype(np.float64)
    wq = flat.float().cpu().numpy().astype(np.float64)
    P = wq.size // 2
    want = np.empty(nq)
    for g, (a, b) in enumerate(((0, split), (split, nq))):
        net = synth.unflatten_mlp(wq[g * P:(g + 1) * P], K, 64, n_hidden)
        want[a:b] = onif.mlp_forward(x64[a:b], net, "leaky", slope)[0]
    assert np.isfinite(z).all()
    assert np.abs(want).max() > 0.1
    assert np.abs(z - want).max() <= TOL[L.NIF_F16], np.abs(z - want).max()


def test_tc_mma_rate_measures_every_shape():
    """nif_tc_mma_rate (the tensor-core instruction-rate measurement behind
    the MLP kernels' tile shapes) runs on every SM, with one or two CTAs per
    SM, at the shapes the kernels issue and reports a plausible number of
    cycles per MMA: at least the cycles the product needs at the nominal
    4,096 FP16 FMAs per cycle per SM, and no wait timed out; a shape too wide
    for two CTAs per SM is refused."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    cyc = torch.zeros(2 * n_sm, dtype=torch.int64, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    for m, n, a_tmem, per_sm in ((128, 64, 0, 1), (128, 64, 1, 1), (64, 256, 0, 1), (128, 256, 0, 1),
                                 (128, 64, 1, 2)):
        nc = per_sm * n_sm
        L.call("nif_tc_mma_rate", m, n, a_tmem, 16, 8, nc, ctypes.c_void_p(cyc.data_ptr()),
               ctypes.c_void_p(ws.data_ptr()), ws.numel(), nif._stream())
        torch.cuda.synchronize()
        per = cyc[:nc].double().cpu().numpy() / (16 * 8)
        assert (per > 0).all()
        assert per.min() >= m * n * 16 / 4096 * 0.9, per.min()
        assert np.median(per) < 10000
    det = ctypes.c_int64()
    L.call("nif_check", ctypes.c_void_p(ws.data_ptr()), ctypes.byref(det), nif._stream())
    with pytest.raises(L.NifError):
        L.call("nif_tc_mma_rate", 96, 64, 0, 16, 8, 1, ctypes.c_void_p(cyc.data_ptr()),
               ctypes.c_void_p(ws.data_ptr()), ws.numel(), nif._stream())
    with pytest.raises(L.NifError):
        L.call("nif_tc_mma_rate", 128, 256, 0, 16, 8, 2 * n_sm, ctypes.c_void_p(cyc.data_ptr()),
               ctypes.c_void_p(ws.data_ptr()), ws.numel(), nif._stream())
