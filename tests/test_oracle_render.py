"""Pins for the renderer oracle (``oracle/render.py``: light importance
sampling by radiant flux from a tabulated CDF, Sec. 5 and Sec. 6.2, and the
direct-illumination estimator): the table and its bisection against a linear
scan, selection frequencies against the flux shares, and the estimator's mean
against the closed-form irradiance of a rectangular source, for importance
and uniform selection alike.  CPU only."""
import numpy as np

from oracle import render as ore
from paper_2306_07191_gb300 import synth


def test_table_and_bisection_against_a_linear_scan():
    w = np.array([3.0, 0.5, 0.0, 7.25, 1.0], np.float32)
    cdf = ore.light_cdf(w)
    assert cdf[-1] == np.float32(1) and (np.diff(cdf) >= 0).all()
    rng = np.random.default_rng(0)
    u = np.concatenate([rng.uniform(size=5000).astype(np.float32), cdf[:-1], [np.float32(0)],
                        np.nextafter(cdf[:-1], np.float32(0))])
    k = ore.pick_light(cdf, u)
    for uu, kk in zip(u, k):
        first = next(j for j in range(len(cdf)) if uu < cdf[j])
        assert kk == first
    assert not (k == 2).any()  # a light of weight 0 is never picked


def test_selection_frequencies_follow_the_flux():
    lights = np.zeros((4, 10), np.float32)
    lights[:, 3] = [1, 2, 0.5, 1]          # e1 along x
    lights[:, 8] = [1, 1, 1, 3]            # e2 along z
    lights[:, 9] = [1, 1, 8, 0.25]         # radiance
    power = ore.light_power(lights)
    np.testing.assert_allclose(power, np.pi * np.array([1, 2, 4, 0.75]))
    cdf = ore.light_cdf(power)
    u = np.random.default_rng(1).uniform(size=400000).astype(np.float32)
    freq = np.bincount(ore.pick_light(cdf, u), minlength=4) / len(u)
    p = power / power.sum()
    assert (np.abs(freq - p) < 4 * np.sqrt(p * (1 - p) / len(u))).all()


def _floor_scene(h=2.0):
    """A floor quad at y = 0 and a camera ray straight down onto (0, 0, 0)."""
    verts = np.array([[-50, 0, -50], [50, 0, -50], [50, 0, 50], [-50, 0, 50]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    cam = synth.pack_rays(np.array([[0.0, 5.0, 0.0]]), np.array([[0.0, -1.0, 0.0]]), 0.0, np.inf)
    return verts, tris, cam, np.array([5.0], np.float32), np.array([0], np.int32)


def _quad_above_corner(a, b, h, L_e, sx=1, sz=1):
    """A light a x b at height h, facing down, with a corner above the origin
    (extending towards sign sx along x and sz along z)."""
    c = np.array([0, h, 0], np.float32)
    e1 = np.array([sx * a, 0, 0], np.float32)
    e2 = np.array([0, 0, sz * b], np.float32)
    if np.cross(e1, e2)[1] > 0:  # emit downwards
        e1, e2 = e2, e1
    return np.concatenate([c, e1, e2, [L_e]]).astype(np.float32)


def test_estimator_mean_equals_the_closed_form_irradiance():
    """Two lights with a corner above the shading point: the mean of f over
    many samples is albedo/pi times the sum of their closed-form irradiances,
    with importance and with uniform selection."""
    verts, tris, cam, t, prim = _floor_scene()
    lights = np.stack([_quad_above_corner(1.0, 2.0, 2.0, 5.0), _quad_above_corner(0.5, 0.5, 1.0, 1.0, -1, -1)])
    albedo = 0.7
    E = ore.rect_irradiance_under_corner(5.0, 1.0, 2.0, 2.0) + ore.rect_irradiance_under_corner(1.0, 0.5, 0.5, 1.0)
    want = albedo / np.pi * E
    spp = 400000
    rng = np.random.default_rng(2)
    for weights in (ore.light_power(lights), np.ones(2)):
        u = rng.uniform(size=(spp, 3)).astype(np.float32)
        rays, f, k = ore.light_samples(cam, t, prim, verts, tris, lights, ore.light_cdf(weights), u, spp,
                                       1e-3, albedo)
        est = f.astype(np.float64).mean()
        sem = f.astype(np.float64).std() / np.sqrt(spp)
        assert abs(est - want) < 4 * sem and abs(est - want) < 0.01 * want, (est, want, sem)
        # every segment starts at the shading point and ends on its light
        assert np.allclose(rays[:, 1], 0) and (rays[:, 3] == np.float32(1e-3)).all()
        yl = rays[:, 0:3] + rays[:, 7:8] * rays[:, 4:7]
        np.testing.assert_allclose(yl[:, 1], lights[k, 1], atol=1e-5)


def test_samples_facing_away_are_empty():
    verts, tris, cam, t, prim = _floor_scene()
    below = _quad_above_corner(1.0, 1.0, -1.0, 1.0)        # under the floor
    up = below.copy()
    up[1] = 2.0                                             # above, but facing up
    up[3:6], up[6:9] = below[6:9].copy(), below[3:6].copy()
    for light in (below, up):
        L = light[None]
        u = np.random.default_rng(3).uniform(size=(64, 3)).astype(np.float32)
        rays, f, k = ore.light_samples(cam, t, prim, verts, tris, L, ore.light_cdf([1.0]), u, 64, 1e-3, 0.5)
        assert (f == 0).all() and (rays[:, 3] == 0).all() and (rays[:, 7] == 0).all()
    # a camera ray without a hit gives empty samples too
    rays, f, k = ore.light_samples(cam, np.array([np.inf], np.float32), np.array([-1]), verts, tris,
                                   _quad_above_corner(1, 1, 2, 1)[None], ore.light_cdf([1.0]),
                                   np.full((4, 3), 0.5, np.float32), 4, 1e-3, 0.5)
    assert (f == 0).all() and (rays[:, 7] == 0).all()


def test_shade_is_the_mean_of_visible_samples():
    f = np.array([1, 2, 3, 4, 0.5, 0.25], np.float32)
    occ = np.array([0, 1, 0, 0, 1, 1], bool)
    np.testing.assert_array_equal(ore.shade(f, occ, 2, 3), np.array([4 / 3, 4 / 3], np.float32))
