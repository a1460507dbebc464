"""Pins for the oracle's FP32 geometry: Moller-Trumbore, brute force, own BVH,
slab test.  CPU only."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import nif as onif
from paper_2306_07191_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TRI = [np.array(v, np.float32) for v in ((0, 0, 0), (1, 0, 0), (0, 1, 0))]


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_mt_hand_derived_cases():
    rows = _golden_rows("moller_trumbore_cases.txt")
    assert len(rows) >= 15
    for r in rows:
        ray = np.array(r[:8], np.float32)
        hit, t = oracle.mt_hit(ray, *TRI)
        assert hit == bool(r[8]), r
        if hit:
            assert abs(t - r[9]) <= 1e-6 * max(1.0, abs(r[9])), (r, t)


def _exact_mt(ray, v0, v1, v2):
    """Exact rational solution of o + t d = v0 + u e1 + v e2 by Cramer's rule
    on the float32 inputs (exactly representable as fractions)."""
    F = [[Fraction(float(x)) for x in v] for v in (v0, v1, v2)]
    o = [Fraction(float(x)) for x in ray[0:3]]
    d = [Fraction(float(x)) for x in ray[4:7]]
    e1 = [F[1][k] - F[0][k] for k in range(3)]
    e2 = [F[2][k] - F[0][k] for k in range(3)]
    T = [o[k] - F[0][k] for k in range(3)]
    # [-d e1 e2] [t u v]^T = T
    cols = [[-d[k] for k in range(3)], e1, e2]

    def det3(c0, c1, c2):
        return (c0[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (c0[1] * c2[2] - c0[2] * c2[1])
                + c2[0] * (c0[1] * c1[2] - c0[2] * c1[1]))
    D = det3(*cols)
    if D == 0:
        return None
    t = det3(T, cols[1], cols[2]) / D
    u = det3(cols[0], T, cols[2]) / D
    v = det3(cols[0], cols[1], T) / D
    return t, u, v


def test_mt_against_exact_rational_arithmetic():
    """Away from the decision boundaries the FP32 test must agree with the exact
    answer computed in rational arithmetic."""
    rng = np.random.default_rng(7)
    checked = 0
    for _ in range(3000):
        v = rng.uniform(-1, 1, size=(3, 3)).astype(np.float32)
        o = rng.uniform(-2, 2, size=3)
        tgt = v.mean(axis=0) + rng.normal(scale=0.6, size=3)
        d = (tgt - o) / np.linalg.norm(tgt - o)
        ray = np.array([*o, 0.0, *d, 1e30], np.float32)
        ex = _exact_mt(ray, *v)
        hit, t = oracle.mt_hit(ray, v[0], v[1], v[2])
        if ex is None:
            continue
        te, ue, ve = (float(x) for x in ex)
        margin = min(abs(ue), abs(ve), abs(1 - ue - ve), abs(te))
        if margin < 1e-3:
            continue
        exact_hit = ue >= 0 and ve >= 0 and ue + ve <= 1 and te > 0
        assert hit == exact_hit
        if hit:
            assert abs(t - te) <= 1e-4 * max(1.0, abs(te))
        checked += 1
    assert checked > 2500


def test_brute_force_closest_is_min_over_triangles():
    rng = np.random.default_rng(3)
    v, t = synth.geodesic_sphere(3)
    rays = synth.shell_rays(rng, 200, radius=2.0)
    occ, th, pr = oracle.brute_cast(v, t, rays)
    for i in range(0, 200, 7):
        best = np.inf
        for k in range(len(t)):
            h, tt = oracle.mt_hit(rays[i], v[t[k, 0]], v[t[k, 1]], v[t[k, 2]])
            if h:
                best = min(best, tt)
        assert (best < np.inf) == bool(occ[i])
        if occ[i]:
            assert th[i] == np.float32(best)


def test_closed_sphere_blocks_rays_from_outside_through_centre():
    """Every ray aimed at the centre of a closed mesh around the origin is
    occluded; every ray aimed away is not."""
    rng = np.random.default_rng(11)
    v, t = synth.geodesic_sphere(6)
    o = synth.unit_vectors(rng, 500) * 3.0
    toward = synth.pack_rays(o, -o / 3.0, 0.0, np.inf)
    away = synth.pack_rays(o, o / 3.0, 0.0, np.inf)
    occ, th, _ = oracle.brute_cast(v, t, toward)
    assert occ.all()
    # the first hit lies between the inscribed radius of the mesh and 1
    assert np.all(th >= 3.0 - 1.0 - 1e-5) and np.all(th <= 3.0 - 0.97)
    occ2, _, _ = oracle.brute_cast(v, t, away)
    assert not occ2.any()


def test_oracle_bvh_equals_brute_force_on_tiny_scene_workload():
    """Own BVH (conservative culling) == brute force, bit for bit, on every ray
    of the 20,480-triangle single-object workload (65,536 shell rays)."""
    rng = np.random.default_rng(1)
    v, t = synth.displaced_icosphere(32, rng)
    v = synth.fit_to_box(v).astype(np.float32)
    rays = synth.shell_rays(np.random.default_rng(2), 65536)
    # a second set aimed at the box so most rays do real work
    aimed = synth.aimed_rays(np.random.default_rng(3), 16384,
                             np.array([-.5, -.5, -.5, .5, .5, .5], np.float32), 1.5)
    allr = np.concatenate([rays, aimed])
    occ_b, th_b, pr_b = oracle.brute_cast(v, t, allr)
    bvh = oracle.OracleBVH(v, t)
    occ_h, th_h, pr_h = bvh.cast(allr, closest=False)
    assert np.array_equal(occ_b, occ_h)
    occ_c, th_c, pr_c = bvh.cast(allr, closest=True)
    assert np.array_equal(occ_b, occ_c)
    assert np.array_equal(th_b.view(np.uint32), th_c.view(np.uint32))
    assert np.array_equal(pr_b, pr_c)
    assert 0.02 < occ_b[:65536].mean() < 0.1
    assert occ_b[65536:].mean() > 0.5


def test_brute_pairs_matches_per_object_brute_force():
    rng = np.random.default_rng(5)
    meshes = [synth.displaced_icosphere(4, rng, centre=c) for c in ((0, 0, 0), (1.5, 0, 0))]
    sc = synth.build_scene(meshes)
    rays = synth.shell_rays(rng, 300, radius=4.0)
    rid = np.repeat(np.arange(300), 2)
    obj = np.tile([0, 1], 300)
    hit = oracle.brute_pairs(sc.verts, sc.tris, sc.obj_tri_range[:, 0], sc.obj_tri_range[:, 1],
                             rays, rid, obj)
    for k in range(2):
        s, c = sc.obj_tri_range[k]
        occ, _, _ = oracle.brute_cast(sc.verts, sc.tris[s:s + c], rays)
        assert np.array_equal(occ, hit[obj == k])


BOX = np.array([-1, -1, -1, 1, 1, 1], np.float32)


def test_slab_special_cases():
    # through the centre along +x from x = -3: enters at t = 2, leaves at t = 4
    h, tin, tout, entry = oracle.slab(np.array([-3, 0, 0, 0, 1, 0, 0, np.inf], np.float32), BOX)
    assert h and tin == 2 and tout == 4 and entry == 2
    # origin inside: entry <= tmin (inner), tin = tmin
    h, tin, tout, entry = oracle.slab(np.array([0.5, 0, 0, 0.001, 1, 0, 0, np.inf], np.float32), BOX)
    assert h and entry <= 0.001 and tin == np.float32(0.001) and tout == np.float32(0.5)
    # parallel to x-planes and outside in y: miss; inside in y: hit
    assert not oracle.slab(np.array([-3, 2, 0, 0, 1, 0, 0, np.inf], np.float32), BOX)[0]
    assert oracle.slab(np.array([-3, 0.5, 0, 0, 1, 0, 0, np.inf], np.float32), BOX)[0]
    # segment ends before the box
    assert not oracle.slab(np.array([-3, 0, 0, 0, 1, 0, 0, 1.5], np.float32), BOX)[0]
    # pointing away
    assert not oracle.slab(np.array([-3, 0, 0, 0, -1, 0, 0, np.inf], np.float32), BOX)[0]
    # grazing a face plane counts (tin == tout)
    h, tin, tout, _ = oracle.slab(np.array([-3, 1, 0, 0, 1, 0, 0, np.inf], np.float32), BOX)
    assert h


def test_numpy_slab_equals_scalar_slab_bitwise():
    rng = np.random.default_rng(9)
    o = rng.uniform(-3, 3, size=(3000, 3))
    d = synth.unit_vectors(rng, 3000)
    d[::17, 1] = 0.0  # axis-parallel components
    rays = synth.pack_rays(o, d, 0.0, np.inf)
    rays[::5, 3] = 0.001
    rays[::7, 7] = 2.0
    box = np.array([-0.7, -1.1, -0.3, 0.9, 0.4, 1.2], np.float32)
    hit, tin, tout, entry = onif.slab_fp32(rays, box)
    for i in range(3000):
        h, a, b, e = oracle.slab(rays[i], box)
        assert h == hit[i]
        if h:
            assert a.view(np.uint32) == tin[i].view(np.uint32)
            assert b.view(np.uint32) == tout[i].view(np.uint32)
            assert e.view(np.uint32) == entry[i].view(np.uint32)


def test_geometry_oracle_is_clean_under_host_sanitizers(tmp_path):
    """AddressSanitizer and UndefinedBehaviorSanitizer over every entry point
    of the C oracle (oracle/sanitize_check.cpp drives them on a random soup,
    empty scenes and zero rays, and checks the BVH against brute force)."""
    import os
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    src = os.path.join(os.path.dirname(oracle.__file__), "sanitize_check.cpp")
    exe = str(tmp_path / "sanitize_check")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-g", "-ffp-contract=off", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-pthread", src, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr.splitlines()[-1])
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "OK", run.stdout + run.stderr
    assert "runtime error" not in run.stderr
