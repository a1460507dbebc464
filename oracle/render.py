"""CPU oracle for the direct-lighting renderer around the NIF shadow query:
light importance sampling by radiant flux and the direct-illumination
estimator.

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and imports nothing from the product package.

What it computes (Sec. 5 'Training': training rays sampled by light importance
according to radiant flux, from a tabulated CDF searched by bisection; Sec. 6.2
compares it with uniform sampling; Sec. 4 renders direct illumination with
shadow rays from the primary hits):

* Lights are one-sided Lambertian quads: corner c, edges e1, e2, normal
  n_l = (e1 x e2) / |e1 x e2| (they emit on that side), area A = |e1 x e2| and
  radiance L_e, so the radiant flux is pi L_e A.
* The table: cum_k = w_0 + ... + w_k summed in order in FP32, cdf_k = cum_k /
  cum_{K-1}; importance sampling takes w = flux, uniform sampling w = 1.
  A sample u0 picks the first k with u0 < cdf_k (bisection), probability
  p_k = cdf_k - cdf_{k-1}.
* The shading point x = o + t d of the camera ray's closest hit (triangle
  normal n, turned to face the camera), the light point y = c + u1 e1 + u2 e2,
  w = y - x, r = |w|, omega = w / r; the shadow segment is (x, omega,
  (tmin, r)).  The sample's value (without visibility) is
      f = (albedo / pi) L_e cos_x cos_y / r^2 * A / p_k,
  cos_x = n . omega, cos_y = -n_l . omega; a sample with cos_x <= 0 or
  cos_y <= 0 has f = 0 and an empty segment (tmin = tmax = 0).
* A pixel's radiance is the mean over its spp samples of f times the
  sample's visibility.

Every quantity above is computed here in FP32, one rounding per operation, in
the order written (no fused multiply-add), as the library's kernels do; the
estimator itself is pinned against the closed-form irradiance of a
rectangular source (tests/test_oracle_render.py).
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def _dot(a, b):
    """FP32 dot products of rows, summed x + y + z in order."""
    s = (a[:, 0] * b[:, 0]).astype(f32)
    s = (s + (a[:, 1] * b[:, 1]).astype(f32)).astype(f32)
    return (s + (a[:, 2] * b[:, 2]).astype(f32)).astype(f32)


def _cross(a, b):
    x = (a[:, 1] * b[:, 2]).astype(f32) - (a[:, 2] * b[:, 1]).astype(f32)
    y = (a[:, 2] * b[:, 0]).astype(f32) - (a[:, 0] * b[:, 2]).astype(f32)
    z = (a[:, 0] * b[:, 1]).astype(f32) - (a[:, 1] * b[:, 0]).astype(f32)
    return np.stack([x, y, z], axis=1).astype(f32)


def light_cdf(weight) -> np.ndarray:
    """The tabulated CDF of light selection (FP32 [K], last entry 1)."""
    w = np.asarray(weight, dtype=f32)
    cum = np.empty_like(w)
    c = f32(0)
    for k in range(len(w)):
        c = f32(c + w[k])
        cum[k] = c
    return (cum / cum[-1]).astype(f32)


def pick_light(cdf, u0) -> np.ndarray:
    """The first k with u0 < cdf_k (bisection over the table)."""
    k = np.searchsorted(np.asarray(cdf, f32), np.asarray(u0, f32), side="right")
    return np.minimum(k, len(cdf) - 1).astype(np.int64)


def light_power(lights) -> np.ndarray:
    """Radiant flux pi L_e A of each quad light [K, 10] (float64)."""
    L = np.asarray(lights, dtype=np.float64)
    A = np.linalg.norm(np.cross(L[:, 3:6], L[:, 6:9]), axis=1)
    return np.pi * L[:, 9] * A


def light_samples(cam, t, prim, verts, tris, lights, cdf, u, spp: int, tmin: float, albedo: float):
    """Shadow rays float32 [n*spp, 8], sample values f float32 [n*spp] and
    the chosen lights int64 [n*spp] for camera rays cam [n, 8] with closest
    hits (t, prim) (t = inf: no hit); u float32 [n*spp, 3] in [0, 1)."""
    cam = np.asarray(cam, f32)
    n = cam.shape[0]
    i = np.repeat(np.arange(n), spp)
    c = cam[i]
    th = np.asarray(t, f32)[i]
    pr = np.asarray(prim)[i]
    u = np.asarray(u, f32).reshape(n * spp, 3)
    lights = np.asarray(lights, f32)
    cdf = np.asarray(cdf, f32)
    hit = (th < np.inf) & (pr >= 0)
    k = pick_light(cdf, u[:, 0])
    p_k = np.where(k > 0, (cdf[k] - cdf[np.maximum(k - 1, 0)]).astype(f32), cdf[k]).astype(f32)
    Lk = lights[k]
    # shading point and its normal, facing the camera
    tt = np.where(hit, th, f32(0))
    x = (c[:, 0:3] + (tt[:, None] * c[:, 4:7]).astype(f32)).astype(f32)
    tri = np.asarray(tris)[np.where(hit, pr, 0)]
    v0 = np.asarray(verts, f32)[tri[:, 0]]
    e1 = (np.asarray(verts, f32)[tri[:, 1]] - v0).astype(f32)
    e2 = (np.asarray(verts, f32)[tri[:, 2]] - v0).astype(f32)
    nx = _cross(e1, e2)
    nlen = np.sqrt(_dot(nx, nx)).astype(f32)
    nx = (nx / np.where(nlen > 0, nlen, f32(1))[:, None]).astype(f32)
    nx = np.where((_dot(nx, c[:, 4:7]) > 0)[:, None], -nx, nx).astype(f32)
    # light point, direction, distance
    y = (Lk[:, 0:3] + (u[:, 1:2] * Lk[:, 3:6]).astype(f32)).astype(f32)
    y = (y + (u[:, 2:3] * Lk[:, 6:9]).astype(f32)).astype(f32)
    w = (y - x).astype(f32)
    r2 = _dot(w, w)
    r = np.sqrt(r2).astype(f32)
    om = (w / np.where(r > 0, r, f32(1))[:, None]).astype(f32)
    nl = _cross(Lk[:, 3:6], Lk[:, 6:9])
    A = np.sqrt(_dot(nl, nl)).astype(f32)
    nl = (nl / A[:, None]).astype(f32)
    cos_x = _dot(nx, om)
    cos_y = (-_dot(nl, om)).astype(f32)
    live = hit & (cos_x > 0) & (cos_y > 0) & (r > 0)
    # f = (albedo/pi) L_e cos_x cos_y / r^2 * A / p_k, left to right
    f = (f32(f32(albedo) / f32(np.pi)) * Lk[:, 9]).astype(f32)
    f = (f * cos_x).astype(f32)
    f = (f * cos_y).astype(f32)
    f = (f / r2).astype(f32)
    f = (f * A).astype(f32)
    f = (f / p_k).astype(f32)
    f = np.where(live, f, f32(0)).astype(f32)
    rays = np.zeros((n * spp, 8), f32)
    rays[:, 0:3] = np.where(live[:, None], x, c[:, 0:3])
    rays[:, 4:7] = np.where(live[:, None], om, c[:, 4:7])
    rays[:, 3] = np.where(live, f32(tmin), f32(0))
    rays[:, 7] = np.where(live, r, f32(0))
    return rays, f, k


def shade(f, occluded, n: int, spp: int) -> np.ndarray:
    """Pixel radiance float32 [n]: (sum_j f_j [sample j visible]) / spp, the
    sum taken in sample order in FP32."""
    v = np.where(np.asarray(occluded, bool), f32(0), np.asarray(f, f32)).reshape(n, spp)
    s = np.zeros(n, f32)
    for j in range(spp):
        s = (s + v[:, j]).astype(f32)
    return (s / f32(spp)).astype(f32)


def rect_irradiance_under_corner(L_e: float, a: float, b: float, h: float) -> float:
    """Closed-form irradiance at a point facing a parallel Lambertian
    rectangle a x b at height h, the point below one of its corners:
    E = L_e * pi * F, with the differential-area-to-rectangle form factor
    F = (1 / 2 pi) [A/sqrt(1+A^2) atan(B/sqrt(1+A^2)) + B/sqrt(1+B^2) atan(A/sqrt(1+B^2))],
    A = a / h, B = b / h (Howell's catalogue of configuration factors)."""
    A, B = a / h, b / h
    F = (A / np.sqrt(1 + A * A) * np.arctan(B / np.sqrt(1 + A * A))
         + B / np.sqrt(1 + B * B) * np.arctan(A / np.sqrt(1 + B * B))) / (2 * np.pi)
    return L_e * np.pi * F
