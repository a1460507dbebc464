"""Pins for the oracle's frame derivation (shadow segments from primary hits)
and its multi-process timed query: closed forms of hand-placed cases, and the
pooled query against the single-process oracle.  CPU only."""
import numpy as np

import oracle
from oracle import frames
from oracle import nif as onif
from paper_2306_07191_gb300 import synth


def test_shadow_segment_closed_forms():
    # camera ray along +z hits at t = 2: the point (0, 0, 2); the light 3
    # units above it gives direction +y and the segment (tmin, 3)
    cam = synth.pack_rays(np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]),
                          np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), 0.0, np.inf)
    t = np.array([2.0, np.inf], np.float32)
    r = frames.shadow_rays(cam, t, np.array([0.0, 3.0, 2.0], np.float32), tmin=1e-3)
    np.testing.assert_array_equal(r[0], np.float32([0, 0, 2, 1e-3, 0, 1, 0, 3]))
    # a primary miss: an empty segment (0, 0) along the camera ray
    np.testing.assert_array_equal(r[1], np.float32([1, 1, 1, 0, 1, 0, 0, 0]))


def test_per_ray_light_points_are_pixel_major():
    cam = synth.pack_rays(np.zeros((2, 3)), np.array([[0.0, 0.0, 1.0]] * 2), 0.0, np.inf)
    t = np.array([1.0, 1.0], np.float32)
    # pixel 0's samples at +x and +y, pixel 1's at -x and -y (distance 2 each)
    lp = np.array([[2, 0, 1], [0, 2, 1], [-2, 0, 1], [0, -2, 1]], np.float32)
    r = frames.shadow_rays(cam, t, lp, tmin=0.0, spp=2)
    np.testing.assert_array_equal(r[:, 4:7], np.float32([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]]))
    np.testing.assert_array_equal(r[:, 7], np.float32([2, 2, 2, 2]))
    np.testing.assert_array_equal(r[:, 0:3], np.float32([[0, 0, 1]] * 4))


def test_frame_rays_start_on_the_closest_hit():
    # two parallel triangles across the z axis at z = 1 and z = 3
    v = np.array([[-1, -1, 1], [1, -1, 1], [0, 1, 1], [-1, -1, 3], [1, -1, 3], [0, 1, 3]], np.float32)
    tr = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    cam = synth.pack_rays(np.array([[0.0, 0.0, 0.0], [5.0, 5.0, 0.0]]),
                          np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]]), 0.0, np.inf)
    r = frames.frame_rays(oracle.OracleBVH(v, tr), cam, np.array([0.0, 0.0, -4.0], np.float32), tmin=1e-3)
    np.testing.assert_array_equal(r[0], np.float32([0, 0, 1, 1e-3, 0, 0, -1, 5]))
    assert r[1, 3] == 0 and r[1, 7] == 0


def test_pooled_query_equals_single_process():
    rng = np.random.default_rng(4)
    boxes = np.array([[-1, -1, -1, 1, 1, 1], [0.5, -0.5, -0.5, 2.5, 1.5, 0.5]], np.float32)
    res, F, log2 = [2, 3], 2, 6
    _, _, off = onif.level_layout(res, log2)
    V = int(off[-1])
    nets = [[np.asarray(w, np.float64) for w in synth.mlp_init(rng, 3 * len(res) * F, 8, 2)] for _ in range(2)]
    m = onif.Model(res=res, F=F, log2_table=log2, obj_aabb=boxes,
                   grids=rng.uniform(-1, 1, size=(2, 2, V * F)), nets=nets, net_mode="class")
    o = rng.uniform(-3, 3, size=(3000, 3))
    d = synth.unit_vectors(rng, 3000)
    rays = synth.pack_rays(o, d, 0.0, 6.0)
    occ, nq = frames.query_occlusion(m, rays)
    assert nq > 500 and 0 < occ.sum() < 3000
    pool = frames.QueryPool(m, processes=2)
    try:
        _, _, nq2, n_occ = pool.timed_query(rays, chunk=700)
    finally:
        pool.close()
    assert nq2 == nq and n_occ == int(occ.sum())
