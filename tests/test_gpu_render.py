"""GPU direct-lighting helpers around the shadow query (nif_light_cdf,
nif_light_samples, nif_shade; Sec. 5 'Training' and Sec. 6.2) against the
oracle in ``oracle/render.py``, bit for bit: the selection table, the light
choice, the shadow segments and sample values (each side from its own exact
closest-hit cast), and the shaded pixels from each side's own exact
visibility."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import render as ore  # noqa: E402
from paper_2306_07191_gb300 import nif, synth  # noqa: E402


def _scene(seed=71):
    rng = np.random.default_rng(seed)
    meshes = [synth.displaced_icosphere(5, rng, centre=c) for c in ((-2.5, -1.0, 0), (0.5, -1.5, 1.0), (2.0, 0.5, -1.0))]
    sc = synth.build_scene(meshes, extra_geometry=synth.room_box(6.0))
    lights = np.array([[-3, 5.9, -3, 2, 0, 0, 0, 0, 2, 12.0],     # bright
                       [2, 5.9, 1, 1, 0, 0, 0, 0, 0.5, 2.0],
                       [0, 5.9, -4, 0.25, 0, 0, 0, 0, 0.25, 40.0],  # small and hot
                       [-5, 3.0, 5.9, 1, 0, 0, 0, 1, 0, 1.0]], np.float32)  # wall light
    for L in lights:  # emit into the room
        n = np.cross(L[3:6], L[6:9])
        if n[1] > 0 or (L[2] > 5 and n[2] > 0):
            L[3:6], L[6:9] = L[6:9].copy(), L[3:6].copy()
    cam = synth.camera_rays(96, 64, (0.0, 0.0, 5.5), (0.0, -0.5, 0.0), 70.0)
    return sc, lights, cam, rng


@pytest.mark.parametrize("spp,importance", [(4, True), (3, False)])
def test_samples_and_shading_match_oracle_bit_for_bit(spp, importance):
    sc, lights, cam, rng = _scene()
    n = cam.shape[0]
    u = rng.uniform(size=(n * spp, 3)).astype(np.float32)
    w = ore.light_power(lights) if importance else np.ones(len(lights))
    dev = "cuda"
    verts, tris = torch.from_numpy(sc.verts).to(dev), torch.from_numpy(sc.tris).to(dev)
    bvh = nif.BVH(verts, tris)
    cam_t = torch.from_numpy(cam).to(dev)
    t, prim = bvh.cast_closest(cam_t)
    cdf = nif.light_cdf(torch.from_numpy(w.astype(np.float32)).to(dev))
    rays, f = nif.light_samples(cam_t, t, prim, verts, tris, torch.from_numpy(lights).to(dev), cdf,
                                torch.from_numpy(u).to(dev), spp, 1e-3, 0.8)
    bits = bvh.cast_shadow(rays)
    L = nif.shade(f, bits, n, spp)
    torch.cuda.synchronize()
    # the oracle from its own brute-force casts
    ocdf = ore.light_cdf(w)
    assert np.array_equal(cdf.cpu().numpy().view(np.uint32), ocdf.view(np.uint32))
    _, ot, oprim = oracle.brute_cast(sc.verts, sc.tris, cam)
    orays, of, ok = ore.light_samples(cam, ot, oprim, sc.verts, sc.tris, lights, ocdf, u, spp, 1e-3, 0.8)
    assert np.array_equal(rays.cpu().numpy().view(np.uint32), orays.view(np.uint32))
    assert np.array_equal(f.cpu().numpy().view(np.uint32), of.view(np.uint32))
    occ, _, _ = oracle.brute_cast(sc.verts, sc.tris, orays)
    oL = ore.shade(of, occ, n, spp)
    assert np.array_equal(L.cpu().numpy().view(np.uint32), oL.view(np.uint32))
    # the case is not degenerate: lit, shadowed and unlit samples, every light picked
    assert (of > 0).mean() > 0.3 and (occ[of > 0] == 1).mean() > 0.02 and (of == 0).any()
    assert len(np.unique(ok)) == len(lights)


def test_empty_calls_and_or_cast():
    """Zero-sized calls queue nothing; the OR-ing cast leaves set bits set,
    skips those rays and ORs the rest, so it equals the overwriting cast OR
    the mask it started from."""
    from paper_2306_07191_gb300 import _lib as L
    sc, lights, cam, rng = _scene(seed=73)
    dev = "cuda"
    verts, tris = torch.from_numpy(sc.verts).to(dev), torch.from_numpy(sc.tris).to(dev)
    bvh = nif.BVH(verts, tris)
    z = torch.empty(0, device=dev)
    zi = torch.empty(0, dtype=torch.int32, device=dev)
    lt = torch.from_numpy(lights).to(dev)
    cdf = nif.light_cdf(torch.ones(len(lights), device=dev))
    rays0, f0 = nif.light_samples(torch.empty((0, 8), device=dev), z, zi, verts, tris, lt, cdf,
                                  torch.empty((0, 3), device=dev), 2)
    assert rays0.shape == (0, 8) and f0.shape == (0,)
    nif.shade(f0, torch.zeros(1, dtype=torch.int32, device=dev), 0, 2)
    nif.clear_bits(torch.zeros(1, dtype=torch.int32, device=dev), 0)
    with pytest.raises(L.NifError):
        nif.light_cdf(torch.empty(0, device=dev))
    # OR cast against the overwriting cast
    n = cam.shape[0]
    r_np = synth.pack_rays(cam[:, 0:3], cam[:, 4:7], 0.0, np.inf)
    r_np[:, 7] = rng.uniform(1.0, 9.0, n)  # some segments end before any surface
    rays = torch.from_numpy(r_np).to(dev)
    start = torch.from_numpy(rng.integers(0, 2**31, size=(n + 31) // 32, dtype=np.int64).astype(np.int32)).to(dev)
    ored = start.clone()
    bvh.cast_shadow(rays, out=ored, or_into=True)
    plain = bvh.cast_shadow(rays)
    torch.cuda.synchronize()
    a = nif.bits_to_bool(ored, n)
    b = nif.bits_to_bool(plain, n) | nif.bits_to_bool(start, n)
    hit = nif.bits_to_bool(plain, n)
    assert torch.equal(a, b) and 0.05 < float(hit.float().mean()) < 0.95
