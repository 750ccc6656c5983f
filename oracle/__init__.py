"""CPU FP64 oracle — TEST INFRASTRUCTURE ONLY.

Python marshalling for ``liboracle.so`` (built from ``oracle.cpp`` with g++).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg and reference arm may import this package. It never imports the CUDA package and
the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PIXEL_DTYPE = np.dtype([
    ("rgb", "<f8", 3), ("t", "<f8"), ("n", "<f8", 3), ("refl_t", "<f8"),
    ("inst", "<i4"), ("geom", "<i4"), ("prim", "<i4"),
    ("refl_inst", "<i4"), ("refl_geom", "<i4"), ("refl_prim", "<i4"),
    ("flags", "<u4"), ("rays", "<u4")])
assert PIXEL_DTYPE.itemsize == 96

F_HIT, F_SHADOW_CAST, F_LIT, F_REFL_CAST, F_REFL_HIT, F_SBT_ERROR = 1, 2, 4, 8, 16, 32


def build(force: bool = False) -> str:
    """Compile liboracle.so (IEEE FP, no contraction so FP32 steps round like the spec)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
            cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-pthread", "-o", _LIB + ".tmp", _SRC]
            subprocess.run(cmd, check=True)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_prims", "n_geoms", "n_blas", "n_inst", "n_hit_groups", "n_materials",
        "n_records", "n_ray_types", "sbt_stride_m")] + [
        ("aabbs", ctypes.c_void_p), ("params", ctypes.c_void_p),
        ("geom_prim_begin", ctypes.c_void_p), ("geom_prim_count", ctypes.c_void_p),
        ("blas_geom_begin", ctypes.c_void_p), ("blas_geom_count", ctypes.c_void_p),
        ("inst_xform", ctypes.c_void_p), ("inst_blas", ctypes.c_void_p),
        ("inst_id", ctypes.c_void_p), ("inst_sbt_offset", ctypes.c_void_p),
        ("inst_mask", ctypes.c_void_p), ("hit_groups", ctypes.c_void_p),
        ("materials", ctypes.c_void_p), ("sbt", ctypes.c_void_p), ("ray_types", ctypes.c_void_p),
        ("geom_type", ctypes.c_void_p), ("n_vertices", ctypes.c_uint32), ("n_triangles", ctypes.c_uint32),
        ("vertices", ctypes.c_void_p), ("indices", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("look_at", ctypes.c_double * 3),
                ("up", ctypes.c_double * 3), ("vfov_deg", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("max_depth", ctypes.c_uint32), ("max_steps", ctypes.c_uint32),
                ("light_pos", ctypes.c_double * 3), ("light_intensity", ctypes.c_double),
                ("eps_rel", ctypes.c_double), ("ambient", ctypes.c_double),
                ("background", ctypes.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def load(path: str):
    """Load an oracle library built from oracle.cpp (the one above, or a copy with
    a planted mistake that the pin tests must catch) and declare its signatures."""
    L = ctypes.CDLL(path)
    vp, u32, i64, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int64, ctypes.c_double
    L.or_render.argtypes = [vp, vp, vp, vp, i64, vp, ctypes.c_int]
    L.or_render.restype = ctypes.c_int
    L.or_world_bounds.argtypes = [vp, vp, vp]
    L.or_intersect.argtypes = [u32, u32, vp, vp, vp, dbl, dbl, dbl, u32, vp, vp, vp]
    L.or_intersect.restype = ctypes.c_int
    L.or_de.argtypes = [u32, vp, vp]
    L.or_de.restype = dbl
    L.or_triplex_pow.argtypes = [vp, dbl, vp]
    L.or_instance_boxes_f32.argtypes = [vp, vp]
    L.or_lbvh_f32.argtypes = [vp, u32, vp, vp, vp, vp, vp]
    L.or_ploc_f32.argtypes = [vp, u32, u32, vp, vp, vp, vp, vp]
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _SceneRef:
    """Keeps the contiguous arrays alive for as long as the ctypes struct is used."""

    def __init__(self, sc):
        c = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        self.arrays = dict(
            aabbs=c(sc.aabbs, np.float32), params=c(sc.params, np.float32),
            geom_prim_begin=c(sc.geom_prim_begin, np.uint32), geom_prim_count=c(sc.geom_prim_count, np.uint32),
            blas_geom_begin=c(sc.blas_geom_begin, np.uint32), blas_geom_count=c(sc.blas_geom_count, np.uint32),
            inst_xform=c(sc.inst_xform, np.float32), inst_blas=c(sc.inst_blas, np.uint32),
            inst_id=c(sc.inst_id, np.uint32), inst_sbt_offset=c(sc.inst_sbt_offset, np.uint32),
            inst_mask=c(sc.inst_mask, np.uint32), hit_groups=c(sc.hit_groups, np.uint32),
            materials=c(sc.materials, np.float32), sbt=c(sc.sbt, np.uint32), ray_types=c(sc.ray_types, np.uint32))
        s = _Scene()
        s.n_prims = len(self.arrays["aabbs"])
        s.n_geoms = len(self.arrays["geom_prim_begin"])
        s.n_blas = len(self.arrays["blas_geom_begin"])
        s.n_inst = len(self.arrays["inst_blas"])
        s.n_hit_groups = len(self.arrays["hit_groups"])
        s.n_materials = len(self.arrays["materials"])
        s.n_records = len(self.arrays["sbt"])
        s.n_ray_types = len(self.arrays["ray_types"])
        s.sbt_stride_m = int(sc.sbt_stride_m)
        for k, a in self.arrays.items():
            setattr(s, k, a.ctypes.data)
        gt = getattr(sc, "geom_type", None)
        self.tri = dict(vertices=c(getattr(sc, "vertices", np.zeros((0, 3))), np.float32).reshape(-1, 3),
                        indices=c(getattr(sc, "indices", np.zeros((0, 3))), np.uint32).reshape(-1, 3))
        if gt is not None:
            self.tri["geom_type"] = c(gt, np.uint32)
            s.geom_type = self.tri["geom_type"].ctypes.data
        s.n_vertices, s.n_triangles = len(self.tri["vertices"]), len(self.tri["indices"])
        s.vertices = self.tri["vertices"].ctypes.data if s.n_vertices else None
        s.indices = self.tri["indices"].ctypes.data if s.n_triangles else None
        self.struct = s


def _camera(cam) -> _Camera:
    c = _Camera()
    c.eye[:] = [float(v) for v in cam.eye]
    c.look_at[:] = [float(v) for v in cam.look_at]
    c.up[:] = [float(v) for v in cam.up]
    c.vfov_deg = float(np.float32(cam.vfov_deg))
    return c


def _params(tp) -> _Params:
    p = _Params()
    p.width, p.height, p.max_depth, p.max_steps = tp.width, tp.height, tp.max_depth, tp.max_steps
    p.light_pos[:] = [float(v) for v in np.asarray(tp.light_pos, np.float32)]
    p.light_intensity = float(np.float32(tp.light_intensity))
    p.eps_rel = float(np.float32(tp.eps_rel))
    p.ambient = float(np.float32(tp.ambient))
    p.background[:] = [float(v) for v in np.asarray(tp.background, np.float32)]
    return p


def render(workload, pixels=None, threads: int = 0) -> np.ndarray:
    """Render a Workload (scene, camera, params); pixels = linear indices or None for all."""
    L = lib()
    ref = _SceneRef(workload.scene)
    cam, prm = _camera(workload.camera), _params(workload.params)
    if pixels is None:
        n = workload.params.width * workload.params.height
        pix_ptr = None
    else:
        pixels = np.ascontiguousarray(pixels, np.int64)
        n = len(pixels)
        pix_ptr = _ptr(pixels)
    out = np.zeros(n, PIXEL_DTYPE)
    rc = L.or_render(ctypes.byref(ref.struct), ctypes.byref(cam), ctypes.byref(prm), pix_ptr, n, _ptr(out), threads)
    if rc != 0:
        raise RuntimeError(f"or_render failed ({rc})")
    return out


def world_bounds(scene):
    ref = _SceneRef(scene)
    lo, hi = np.zeros(3), np.zeros(3)
    lib().or_world_bounds(ctypes.byref(ref.struct), _ptr(lo), _ptr(hi))
    return lo, hi


def intersect(is_id, params, o, d, t_lo, t_hi=np.inf, eps=1e-4, max_steps=256, ahs_id=0xFFFFFFFF):
    """One object-space primitive (optionally with an any-hit shader). Returns (t, normal, steps) or None."""
    prm = np.zeros(16, np.float32)
    prm[: len(params)] = params
    o, d = np.asarray(o, np.float64), np.asarray(d, np.float64)
    t, n, st = ctypes.c_double(), np.zeros(3), ctypes.c_uint32()
    hit = lib().or_intersect(is_id, ahs_id, _ptr(prm), _ptr(o), _ptr(d), float(t_lo), float(t_hi), float(eps),
                             max_steps, ctypes.byref(t), _ptr(n), ctypes.byref(st))
    return (t.value, n, st.value) if hit else None


def de(is_id, params, p) -> float:
    prm = np.zeros(16, np.float32)
    prm[: len(params)] = params
    p = np.asarray(p, np.float64)
    return lib().or_de(is_id, _ptr(prm), _ptr(p))


def triplex_pow(z, n=8.0) -> np.ndarray:
    z = np.asarray(z, np.float64)
    out = np.zeros(3)
    lib().or_triplex_pow(_ptr(z), float(n), _ptr(out))
    return out


def instance_boxes_f32(scene) -> np.ndarray:
    ref = _SceneRef(scene)
    out = np.zeros((len(scene.inst_blas), 6), np.float32)
    lib().or_instance_boxes_f32(ctypes.byref(ref.struct), _ptr(out))
    return out


def lbvh_f32(boxes: np.ndarray):
    """Reference LBVH over [n,6] float32 boxes -> dict(perm, codes, child, cbox, root)."""
    boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    n = len(boxes)
    perm = np.zeros(n, np.uint32)
    codes = np.zeros(n, np.uint32)
    child = np.zeros((max(n - 1, 0), 2), np.int32)
    cbox = np.zeros((max(n - 1, 0), 12), np.float32)
    root = np.zeros(6, np.float32)
    if n:
        lib().or_lbvh_f32(_ptr(boxes), n, _ptr(perm), _ptr(codes), _ptr(child), _ptr(cbox), _ptr(root))
    return dict(perm=perm, codes=codes, child=child, cbox=cbox, root=root)


def ploc_f32(boxes: np.ndarray, radius: int = 16):
    """Reference PLOC tree over [n,6] float32 boxes (same Morton order and output
    layout as lbvh_f32) -> dict(perm, codes, child, cbox, root)."""
    boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    n = len(boxes)
    perm = np.zeros(n, np.uint32)
    codes = np.zeros(n, np.uint32)
    child = np.zeros((max(n - 1, 0), 2), np.int32)
    cbox = np.zeros((max(n - 1, 0), 12), np.float32)
    root = np.zeros(6, np.float32)
    if n:
        rc = lib().or_ploc_f32(_ptr(boxes), n, radius, _ptr(perm), _ptr(codes), _ptr(child), _ptr(cbox), _ptr(root))
        if rc:
            raise ValueError(f"or_ploc_f32 failed ({rc})")
    return dict(perm=perm, codes=codes, child=child, cbox=cbox, root=root)


def blas_leaf_boxes(scene, b: int) -> np.ndarray:
    """Object-space boxes of BLAS b's primitives in geometry-major order (the BLAS's
    leaf input): AABBs as given, triangles' vertex bounds."""
    g0, gn = int(scene.blas_geom_begin[b]), int(scene.blas_geom_count[b])
    gt = getattr(scene, "geom_type", None)
    rows = []
    for g in range(g0, g0 + gn):
        p0, pn = int(scene.geom_prim_begin[g]), int(scene.geom_prim_count[g])
        if gt is not None and int(gt[g]) == 1:
            tv = np.asarray(scene.vertices, np.float32)[np.asarray(scene.indices)[p0:p0 + pn]]   # [n,3,3]
            rows.append(np.concatenate([tv.min(1), tv.max(1)], 1))
        else:
            rows.append(scene.aabbs[p0:p0 + pn])
    return np.concatenate(rows).astype(np.float32)
