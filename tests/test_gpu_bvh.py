"""GPU BVH (bvh_build, bvh_cast_shadow, bvh_cast_closest, bvh_cast_pairs,
nif_shadow_rays) against the CPU oracle: hit/miss and closest hit bit-exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2306_07191_gb300 import nif, synth, workloads  # noqa: E402


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _gpu_cast(verts, tris, rays, tags=None):
    bvh = nif.BVH(_cuda(verts), _cuda(tris), _cuda(tags) if tags is not None else None)
    r = _cuda(rays)
    bits = bvh.cast_shadow(r)
    t, p = bvh.cast_closest(r)
    torch.cuda.synchronize()
    occ = nif.bits_to_bool(bits, len(rays)).cpu().numpy()
    return bvh, occ, t.cpu().numpy(), p.cpu().numpy()


def test_tiny_object_all_rays_bit_exact():
    w = workloads.tiny_object()
    aimed = synth.aimed_rays(np.random.default_rng(5), 16384, w.aabb[0], 1.5)
    rays = np.concatenate([w.rays, aimed])
    occ_ref, t_ref, p_ref = oracle.brute_cast(w.verts, w.tris, rays)
    bvh, occ, t, p = _gpu_cast(w.verts, w.tris, rays)
    assert np.array_equal(occ.astype(np.uint8), occ_ref)
    assert np.array_equal(t.view(np.uint32), t_ref.view(np.uint32))
    assert np.array_equal(p, p_ref)
    info = bvh.info()
    assert info["prims"] == len(w.tris) and 0 < info["depth"] <= 96


def test_ragged_and_degenerate_ray_sets():
    rng = np.random.default_rng(3)
    v, t = synth.geodesic_sphere(5)
    v = v.astype(np.float32)
    for n in (1, 31, 33, 1000, 4097):
        rays = synth.shell_rays(rng, n, radius=2.0)
        rays[::3, 7] = 0.0        # empty segments
        rays[::5, 4:7] = [0, 0, 1]  # axis-parallel directions
        occ_ref, t_ref, p_ref = oracle.brute_cast(v, t, rays)
        _, occ, tt, pp = _gpu_cast(v, t, rays)
        assert np.array_equal(occ.astype(np.uint8), occ_ref)
        assert np.array_equal(tt.view(np.uint32), t_ref.view(np.uint32))
        assert np.array_equal(pp, p_ref)


def test_tiny_scenes_and_zero_rays():
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    idx = np.array([[0, 1, 2]], np.int32)
    rays = synth.pack_rays(np.array([[0.25, 0.25, 1.0], [2.0, 2.0, 1.0]]),
                           np.array([[0, 0, -1.0], [0, 0, -1.0]]), 0.0, np.inf)
    _, occ, t, p = _gpu_cast(tri, idx, rays)
    assert occ.tolist() == [True, False] and t[0] == 1.0 and p.tolist() == [0, -1]
    bvh = nif.BVH(_cuda(tri), _cuda(idx))
    bits = bvh.cast_shadow(_cuda(rays[:0].reshape(0, 8)))
    torch.cuda.synchronize()
    assert bits.numel() == 0
    # an empty scene is fully visible
    empty = nif.BVH(_cuda(tri), _cuda(np.zeros((0, 3), np.int32)))
    bits = empty.cast_shadow(_cuda(rays))
    assert not nif.bits_to_bool(bits, 2).any()


def test_pairs_labels_equal_per_object_brute_force():
    rng = np.random.default_rng(11)
    meshes = [synth.displaced_icosphere(8, rng, centre=c) for c in ((0, 0, 0), (1.6, 0, 0), (0.8, 1.2, 0))]
    sc = synth.build_scene(meshes)
    box = np.concatenate([sc.obj_aabb[:, :3].min(0), sc.obj_aabb[:, 3:].max(0)]).astype(np.float32)
    rays = synth.aimed_rays(rng, 3000, box, 4.0)
    rid = np.repeat(np.arange(3000), 3).astype(np.int32)
    obj = np.tile([0, 1, 2], 3000).astype(np.int32)
    ref = oracle.brute_pairs(sc.verts, sc.tris, sc.obj_tri_range[:, 0], sc.obj_tri_range[:, 1],
                             rays, rid, obj)
    bvh = nif.BVH(_cuda(sc.verts), _cuda(sc.tris), _cuda(sc.tri_obj))
    hit = bvh.cast_pairs(_cuda(rays), _cuda(rid), _cuda(obj)).cpu().numpy()
    assert np.array_equal(hit, ref)
    assert 0.05 < ref.mean() < 0.9


def test_room_scene_full_size_sampled():
    """Full-size room workload (1.0M triangles, 2,073,600 shadow rays): the GPU
    primary hits and shadow rays equal the oracle's on sampled pixels bit for
    bit, and so does shadow visibility."""
    ws = workloads.room_scene()
    sc = ws.scene
    verts, tris = _cuda(sc.verts), _cuda(sc.tris)
    bvh = nif.BVH(verts, tris, _cuda(sc.tri_obj))
    cam = _cuda(ws.camera)
    t, prim = bvh.cast_closest(cam)
    light = _cuda(ws.light)
    srays = nif.shadow_rays(cam, t, light, tmin=1e-3)
    bits = bvh.cast_shadow(srays)
    torch.cuda.synchronize()
    n = ws.camera.shape[0]
    assert n == 1920 * 1080
    occ = nif.bits_to_bool(bits, n).cpu().numpy()
    sample = np.random.default_rng(0).choice(n, 4000, replace=False)
    ob = oracle.OracleBVH(sc.verts, sc.tris)
    o_occ, o_t, o_p = ob.cast(ws.camera[sample], closest=True)
    assert np.array_equal(o_t.view(np.uint32), t.cpu().numpy()[sample].view(np.uint32))
    assert np.array_equal(o_p, prim.cpu().numpy()[sample])
    # shadow rays from the oracle's own hits, same FP32 operation order
    c = ws.camera[sample].astype(np.float32)
    tt = o_t.astype(np.float32)
    p = np.stack([c[:, k] + tt * c[:, 4 + k] for k in range(3)], 1).astype(np.float32)
    v = (ws.light[None, :].astype(np.float32) - p).astype(np.float32)
    ss = v[:, 0] * v[:, 0]
    ss = ss + v[:, 1] * v[:, 1]
    ss = ss + v[:, 2] * v[:, 2]
    ln = np.sqrt(ss).astype(np.float32)
    ors = np.zeros((len(sample), 8), np.float32)
    ors[:, 0:3] = p
    ors[:, 3] = np.float32(1e-3)
    ors[:, 4:7] = v / ln[:, None]
    ors[:, 7] = ln
    assert np.array_equal(ors.view(np.uint32), srays.cpu().numpy()[sample].view(np.uint32))
    s_occ, _, _ = ob.cast(ors, closest=False)
    assert np.array_equal(s_occ.astype(bool), occ[sample])
    assert 0.05 < occ.mean() < 0.95


def test_degenerate_triangle_sets_build_shallow_exact_trees():
    """Inputs that are hard on a Morton-code builder: 4,096 copies of one
    triangle spun about a shared centroid (every key equal), and a chain of
    triangles at x = 2^-k clustered exponentially towards the origin (keys
    sharing ever longer prefixes).  The trees stay within the traversal
    stack, bvh_check is clean after the casts, and the casts equal brute
    force bit for bit."""
    rng = np.random.default_rng(8)
    base = np.array([[1.0, 0.0, 0.0], [-0.5, 0.8660254, 0.0], [-0.5, -0.8660254, 0.0]])
    axes = synth.unit_vectors(rng, 4096)
    ang = rng.uniform(0, 2 * np.pi, 4096)
    spun = []
    for a, th in zip(axes, ang):
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        R = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
        spun.append(base @ R.T)
    chain = [base * 2.0 ** -k * 0.25 + np.array([2.0 ** -k, 0.0, 0.0]) for k in range(100)]
    for tris3 in (spun, chain):
        v = np.concatenate(tris3).astype(np.float32)
        t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
        rays = synth.shell_rays(rng, 4096, radius=2.0)
        occ_ref, t_ref, p_ref = oracle.brute_cast(v, t, rays)
        bvh, occ, tt, pp = _gpu_cast(v, t, rays)
        bvh.check()
        assert 0 < bvh.info()["depth"] <= 96
        assert occ_ref.any()
        assert np.array_equal(occ.astype(np.uint8), occ_ref)
        assert np.array_equal(tt.view(np.uint32), t_ref.view(np.uint32))
        assert np.array_equal(pp, p_ref)


@pytest.mark.parametrize("case", ["tiny", "spun", "tags"])
def test_ploc_tree_casts_equal_brute_force(case):
    """bvh_build_ploc (locally-ordered clustering, Meister & Bittner 2018):
    any-hit, closest-hit and per-pair casts through its tree equal brute
    force bit for bit, like the LBVH's; its surface-area cost is below the
    LBVH's, and bvh_stats reports the work per ray of both."""
    rng = np.random.default_rng(21)
    tags = None
    if case == "tiny":
        w = workloads.tiny_object()
        v, t = w.verts, w.tris
        rays = np.concatenate([w.rays[:20000], synth.aimed_rays(rng, 12000, w.aabb[0], 1.5)])
    elif case == "spun":
        base = np.array([[1.0, 0.0, 0.0], [-0.5, 0.8660254, 0.0], [-0.5, -0.8660254, 0.0]])
        tri3 = []
        for a, th in zip(synth.unit_vectors(rng, 3000), rng.uniform(0, 2 * np.pi, 3000)):
            K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            tri3.append(base @ (np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K).T)
        v = np.concatenate(tri3).astype(np.float32)
        t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
        rays = synth.shell_rays(rng, 4097, radius=2.0)
    else:
        sc = workloads.room_scene(6, 10, 64, 48, seed=3).scene
        v, t, tags = sc.verts, sc.tris, sc.tri_obj
        rays = synth.shell_rays(rng, 6000, radius=12.0)
        rays[:, 0:3] *= 0.5
    occ_ref, t_ref, p_ref = oracle.brute_cast(v, t, rays)
    vt, tt = _cuda(v), _cuda(t)
    ploc = nif.BVH(vt, tt, _cuda(tags) if tags is not None else None, builder="ploc")
    lbvh = nif.BVH(vt, tt, _cuda(tags) if tags is not None else None)
    r = _cuda(rays)
    bits = ploc.cast_shadow(r)
    th, pr = ploc.cast_closest(r)
    torch.cuda.synchronize()
    ploc.check()
    assert np.array_equal(nif.bits_to_bool(bits, len(rays)).cpu().numpy().astype(np.uint8), occ_ref)
    assert np.array_equal(th.cpu().numpy().view(np.uint32), t_ref.view(np.uint32))
    assert np.array_equal(pr.cpu().numpy(), p_ref)
    assert 0 < ploc.info()["depth"] <= 96 and ploc.info()["prims"] == len(t)
    if tags is not None:
        # per-pair labels through the clustered tree
        obj = rng.integers(0, 6, size=len(rays)).astype(np.int32)
        hit = ploc.cast_pairs(r, torch.arange(len(rays), dtype=torch.int32, device="cuda"), _cuda(obj))
        first = np.array([np.nonzero(tags == k)[0][0] for k in range(6)])
        count = np.array([np.count_nonzero(tags == k) for k in range(6)])
        ref = oracle.brute_pairs(v, t, first, count, rays, np.arange(len(rays)), obj)
        assert np.array_equal(hit.cpu().numpy(), ref)
    sp, sl = ploc.stats(r), lbvh.stats(r)
    print(f"\n{case}: SAH cost PLOC {sp['sah_cost']:.2f} LBVH {sl['sah_cost']:.2f}; nodes/ray "
          f"{sp['nodes_per_ray']:.1f} vs {sl['nodes_per_ray']:.1f}; triangles/ray {sp['tris_per_ray']:.1f} vs "
          f"{sl['tris_per_ray']:.1f}")
    assert sp["nodes_per_ray"] > 0 and sp["sah_cost"] > 0
    if case == "tiny":
        assert sp["sah_cost"] < sl["sah_cost"]
