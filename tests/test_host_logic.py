"""Host-side logic of the pipelines, on the CPU: batch drawing without
replacement, the training-target helpers of the primary-ray pipeline against
the oracle's slab test and a plain cross product, and the renderer's lights."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nif as onif  # noqa: E402
from oracle import render as ore  # noqa: E402
from paper_2306_07191_gb300 import pipeline, synth  # noqa: E402


def test_batches_cover_every_pair_once_per_epoch():
    draw = pipeline.BatchDraw(1000, seed=5)
    seen = np.concatenate([draw(100) for _ in range(10)])
    assert np.array_equal(np.sort(seen), np.arange(1000))
    # the next epoch is a fresh permutation; a batch never straddles two epochs
    nxt = np.concatenate([draw(300) for _ in range(3)])
    assert len(np.unique(nxt)) == 900
    last = draw(300)
    assert len(np.unique(last)) == 300
    assert not np.array_equal(seen[:100], nxt[:100])


def test_slab_parameters_equal_the_oracle_fp32_slab():
    rng = np.random.default_rng(3)
    n = 4000
    boxes = np.concatenate([rng.uniform(-2, 0, (n, 3)), rng.uniform(0.1, 2, (n, 3))], 1).astype(np.float32)
    boxes[:, 3:] += boxes[:, :3]
    o = rng.uniform(-6, 6, (n, 3))
    d = synth.unit_vectors(rng, n)
    d[::11, 1] = 0.0  # directions parallel to a slab
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = synth.pack_rays(o, d, 1e-3, np.inf)
    rays[::5, 7] = 4.0
    tin, tout = pipeline.slab_params(torch.from_numpy(rays), torch.from_numpy(boxes))
    hit = (tin <= tout).numpy()
    for i in range(0, n, 7):
        h, ti, to, _ = onif.slab_fp32(rays[i:i + 1], boxes[i])
        assert bool(h[0]) == bool(hit[i])
        if h[0]:
            assert ti[0] == tin[i].item() and to[0] == tout[i].item()


def test_face_normals_are_unit_and_face_the_ray():
    rng = np.random.default_rng(4)
    v, t = synth.displaced_icosphere(6, rng)
    verts = torch.from_numpy(v.astype(np.float32))
    tris = torch.from_numpy(t.astype(np.int32))
    prim = torch.from_numpy(rng.integers(0, len(t), 500).astype(np.int32))
    d = torch.from_numpy(synth.unit_vectors(rng, 500).astype(np.float32))
    nrm = pipeline.face_normals(verts, tris, prim, d).numpy()
    tri = t[prim.numpy()]
    ref = np.cross(v[tri[:, 1]] - v[tri[:, 0]], v[tri[:, 2]] - v[tri[:, 0]])
    ref /= np.linalg.norm(ref, axis=1, keepdims=True)
    ref = np.where((np.sum(ref * d.numpy(), 1) > 0)[:, None], -ref, ref)
    np.testing.assert_allclose(nrm, ref, atol=1e-5)
    assert (np.sum(nrm * d.numpy(), 1) <= 1e-6).all()


def test_ceiling_lights_emit_into_the_room_with_spread_fluxes():
    L = pipeline.ceiling_lights()
    n = np.cross(L[:, 3:6], L[:, 6:9])
    assert (n[:, 1] < 0).all() and np.allclose(n[:, [0, 2]], 0)    # all face down
    assert (np.abs(L[:, 0:3] + L[:, 3:6] + L[:, 6:9]) <= 20).all()   # inside the room
    power = ore.light_power(L)
    assert power.max() / power.min() > 100
    cdf = ore.light_cdf(power)
    assert cdf[-1] == np.float32(1)
