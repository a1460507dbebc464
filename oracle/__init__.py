"""CPU oracle for the Neural Intersection Function shadow-ray path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2306_07191_gb300``)
and imports nothing from it.

* ``oracle/geom.cpp`` (built into ``oracle/_geom.so``): FP32 ray/triangle and
  ray/box tests with a fixed operation order, brute force and an own BVH.
* ``oracle/nif.py``: FP64 AABB parameterisation, grid encoding, MLP, loss,
  gradients and Adam.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_geom.so")
_SRC = os.path.join(_HERE, "geom.cpp")
_lib = None


def build(force: bool = False) -> str:
    """Compile geom.cpp with gcc; FMA contraction off so every product and sum
    is rounded separately."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.oracle_mt_hit.argtypes = [P, P, P, P, P]
        L.oracle_mt_hit.restype = ctypes.c_int
        L.oracle_brute_cast.argtypes = [P, P, i64, P, i64, P, P, P, ctypes.c_int]
        L.oracle_brute_pairs.argtypes = [P, P, P, P, P, P, P, i64, P, ctypes.c_int]
        L.oracle_brute_pairs_closest.argtypes = [P, P, P, P, P, P, P, i64, P, P, ctypes.c_int]
        L.oracle_bvh_build.argtypes = [P, P, i64]
        L.oracle_bvh_build.restype = P
        L.oracle_bvh_free.argtypes = [P]
        L.oracle_bvh_node_count.argtypes = [P]
        L.oracle_bvh_node_count.restype = i64
        L.oracle_bvh_cast.argtypes = [P, P, P, P, i64, ctypes.c_int, P, P, P, ctypes.c_int]
        L.oracle_slab.argtypes = [P, P, P, P, P]
        L.oracle_slab.restype = ctypes.c_int
        _lib = L
    return _lib


def threads() -> int:
    return max(1, os.cpu_count() or 1)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def mt_hit(ray, v0, v1, v2):
    """Single Moller-Trumbore test -> (hit, t)."""
    r = np.ascontiguousarray(ray, dtype=np.float32)
    a = [np.ascontiguousarray(v, dtype=np.float32) for v in (v0, v1, v2)]
    t = np.zeros(1, dtype=np.float32)
    h = lib().oracle_mt_hit(_p(r), _p(a[0]), _p(a[1]), _p(a[2]), _p(t))
    return bool(h), float(t[0])


def brute_cast(verts, tris, rays, nthreads=None):
    """Brute-force cast of every ray against every triangle.
    Returns (occluded uint8 [n], t_hit float32 [n] (closest), prim int32 [n])."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    r = np.ascontiguousarray(rays, dtype=np.float32)
    n = r.shape[0]
    occ = np.zeros(n, np.uint8)
    th = np.zeros(n, np.float32)
    pr = np.zeros(n, np.int32)
    lib().oracle_brute_cast(_p(v), _p(t), t.shape[0], _p(r), n, _p(occ), _p(th), _p(pr),
                            nthreads or threads())
    return occ, th, pr


def brute_pairs(verts, tris, obj_first, obj_count, rays, ray_id, obj, nthreads=None):
    """Per (ray, object) pair: 1 when a triangle of that object is hit inside the
    ray's segment (the label of Sec. 6.4's per-pair training samples)."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    of = np.ascontiguousarray(obj_first, dtype=np.int64)
    oc = np.ascontiguousarray(obj_count, dtype=np.int64)
    r = np.ascontiguousarray(rays, dtype=np.float32)
    rid = np.ascontiguousarray(ray_id, dtype=np.int32)
    ob = np.ascontiguousarray(obj, dtype=np.int32)
    hit = np.zeros(len(rid), np.uint8)
    lib().oracle_brute_pairs(_p(v), _p(t), _p(of), _p(oc), _p(r), _p(rid), _p(ob), len(rid),
                             _p(hit), nthreads or threads())
    return hit


def brute_pairs_closest(verts, tris, obj_first, obj_count, rays, ray_id, obj, nthreads=None):
    """Per (ray, object) pair: the closest hit of that object's triangles
    inside the ray's segment.  Returns (t float32 [nq] (+inf if none), prim
    int32 [nq] (-1 if none))."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    of = np.ascontiguousarray(obj_first, dtype=np.int64)
    oc = np.ascontiguousarray(obj_count, dtype=np.int64)
    r = np.ascontiguousarray(rays, dtype=np.float32)
    rid = np.ascontiguousarray(ray_id, dtype=np.int32)
    ob = np.ascontiguousarray(obj, dtype=np.int32)
    th = np.zeros(len(rid), np.float32)
    pr = np.zeros(len(rid), np.int32)
    lib().oracle_brute_pairs_closest(_p(v), _p(t), _p(of), _p(oc), _p(r), _p(rid), _p(ob), len(rid),
                                     _p(th), _p(pr), nthreads or threads())
    return th, pr


class OracleBVH:
    """The oracle's own median-split BVH over a triangle soup."""

    def __init__(self, verts, tris):
        self.v = np.ascontiguousarray(verts, dtype=np.float32)
        self.t = np.ascontiguousarray(tris, dtype=np.int32)
        self.h = lib().oracle_bvh_build(_p(self.v), _p(self.t), self.t.shape[0])

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_bvh_free(self.h)
            self.h = None

    @property
    def n_nodes(self) -> int:
        return int(lib().oracle_bvh_node_count(self.h))

    def cast(self, rays, closest=False, nthreads=None):
        r = np.ascontiguousarray(rays, dtype=np.float32)
        n = r.shape[0]
        occ = np.zeros(n, np.uint8)
        th = np.zeros(n, np.float32)
        pr = np.zeros(n, np.int32)
        lib().oracle_bvh_cast(self.h, _p(self.v), _p(self.t), _p(r), n, int(closest), _p(occ),
                              _p(th), _p(pr), nthreads or threads())
        return occ, th, pr


def slab(ray, box):
    """Scalar FP32 slab test -> (hit, tin, tout, entry)."""
    r = np.ascontiguousarray(ray, dtype=np.float32)
    b = np.ascontiguousarray(box, dtype=np.float32)
    out = np.zeros(3, dtype=np.float32)
    h = lib().oracle_slab(_p(r), _p(b), _p(out[0:1]), _p(out[1:2]), _p(out[2:3]))
    return bool(h), out[0], out[1], out[2]
