"""B300-native procedural-primitive ray tracer (Proceduray's hot path in CUDA).

Thin ctypes binding over the C ABI in ``include/proceduray.h``: argument
marshalling only. Every step of the path (BVH build, traversal, intersection,
shading) runs in the kernels of ``libproceduray.so``. PyTorch supplies device
memory and streams. There is no CPU fallback: importing this package fails if
the library is missing, and tracing needs a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libproceduray.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2012_10357_b300/build.py` "
                      "(the CUDA library is required; there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

# ---- constants mirrored from proceduray.h -------------------------------------
PR_OK, PR_ERR_INVALID_ARG, PR_ERR_OUT_OF_MEMORY, PR_ERR_CUDA = 0, 1, 2, 3
PR_ERR_SBT_INDEX, PR_ERR_STACK_OVERFLOW, PR_ERR_TIMEOUT, PR_ERR_NOT_BUILT, PR_ERR_BUDGET = 4, 5, 6, 7, 8
PR_NONE = 0xFFFFFFFF
PR_TRACE_WRITE_AOV = 1
PR_TRACE_TLAS_BVH2 = 2
PR_TRACE_OUTPUT_RGB = 4
PR_BUILD_TLAS_PLOC = 1
PR_BUILD_TLAS_PARITY4 = 2
PR_BUILD_TLAS_BVH8 = 4
PR_BUILD_TLAS_BVH8_F32 = 8
ERR_WORD_SBT = 1 << PR_ERR_SBT_INDEX
ERR_WORD_STACK = 1 << PR_ERR_STACK_OVERFLOW
PR_IS_COUNT = 10
WORK_FIELDS = (["tlas_nodes", "blas_nodes", "instances", "leaves", "sbt_lookups"] +
               [f"is_calls_{i}" for i in range(PR_IS_COUNT)] + [f"de_evals_{i}" for i in range(PR_IS_COUNT)] +
               ["julia_iters", "mandelbulb_iters", "shaded", "rays", "tlas_nodes4", "tlas_nodes8",
                                                                  "tlas_nodes8q"])

AOV_DTYPE = np.dtype([("t", "<f4"), ("inst", "<u4"), ("geom", "<u4"), ("prim", "<u4"), ("n", "<f4", 3),
                      ("flags", "<u4"), ("refl_t", "<f4"), ("refl_inst", "<u4"), ("refl_geom", "<u4"),
                      ("refl_prim", "<u4")])
assert AOV_DTYPE.itemsize == 48


class PrError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.pr_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


class _SceneDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "struct_size", "n_prims", "n_geoms", "n_blas", "n_inst", "n_hit_groups", "n_materials",
        "n_records", "n_ray_types", "sbt_stride_m")] + [
        (n, ctypes.c_void_p) for n in (
            "aabbs", "params", "geom_prim_begin", "geom_prim_count", "blas_geom_begin", "blas_geom_count",
            "inst_xform", "inst_blas", "inst_id", "inst_sbt_offset", "inst_mask", "hit_groups", "materials",
            "sbt", "ray_types", "geom_type")] + [
        ("n_vertices", ctypes.c_uint32), ("n_triangles", ctypes.c_uint32),
        ("vertices", ctypes.c_void_p), ("indices", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("look_at", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("vfov_deg", ctypes.c_float)]


class _TraceParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("struct_size", "width", "height", "max_depth", "max_steps", "flags")] + [
        ("light_pos", ctypes.c_float * 3), ("light_intensity", ctypes.c_float), ("eps_rel", ctypes.c_float),
        ("ambient", ctypes.c_float), ("background", ctypes.c_float * 3)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_vp, _u32, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
_sig("pr_version", _u32)
_sig("pr_last_error", ctypes.c_char_p)
_sig("pr_scene_validate", _i32, _vp)
_sig("pr_sbt_index", _i32, _u32, _u32, _u32, _u32, _u32, _vp)
_sig("pr_scene_create", _i32, _vp, _vp, _vp)
_sig("pr_scene_upload", _i32, _vp, _vp, _vp)
_sig("pr_build_bvh", _i32, _vp, _vp)
_sig("pr_build_bvh_many", _i32, _vp, _u32, _vp)
_sig("pr_build_bvh_ex", _i32, _vp, _u32, _vp)
_sig("pr_build_bvh_many_ex", _i32, _vp, _u32, _u32, _vp)
_sig("pr_trace", _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("pr_trace_frames", _i32, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp)
_sig("pr_trace_work", _i32, _vp, _vp, _u32, _vp, _vp, _vp, _vp)
_sig("pr_scene_error", _i32, _vp, _vp, _vp)
_sig("pr_scene_bounds", _i32, _vp, _vp, _vp)
_sig("pr_scene_read_bvh", _i32, _vp, _u32, _vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp)
_sig("pr_scene_device_bytes", ctypes.c_size_t, _vp)
_sig("pr_scene_kernel_launches", _i32, _vp, _vp, _vp)
_sig("pr_lbvh_build", _i32, _vp, _u32, _vp, _vp, _vp, _vp, _vp)
_sig("pr_lbvh_build_noalloc", _i32, _vp, _u32, _vp, _vp, _vp, _vp, _vp)
_sig("pr_batch_create", _i32, _u32, ctypes.c_uint64, _vp)
_sig("pr_batch_set_tuning", _i32, _vp, _vp)
_sig("pr_batch_get_tuning", _i32, _vp, _vp)
_sig("pr_trace_batch", _i32, _vp, _u32, _vp, _vp, _vp)
_sig("pr_trace_batch_graph", _i32, _vp, _u32, _vp, _vp, _vp)
_sig("pr_batch_autotune", _i32, _vp, _u32, _vp, _vp, _vp, _vp)
_sig("pr_batch_device_bytes", ctypes.c_size_t, _vp)
_sig("pr_batch_destroy", None, _vp)
_sig("pr_server_create", _i32, _vp, _vp)
_sig("pr_server_submit", _i32, _vp, _vp, _vp)
_sig("pr_server_poll", _i32, _vp, ctypes.c_uint64, _vp, _vp)
_sig("pr_server_drain", _i32, _vp, ctypes.c_double)
_sig("pr_server_get_stats", _i32, _vp, _vp)
_sig("pr_server_destroy", None, _vp)
_sig("pr_scene_destroy", None, _vp)
_sig("pr_fma_peak_probe", _i32, _u32, _vp, _vp, _vp)

EXPORTED = ["pr_version", "pr_last_error", "pr_scene_validate", "pr_sbt_index", "pr_scene_create",
            "pr_scene_upload", "pr_build_bvh", "pr_build_bvh_many", "pr_build_bvh_ex", "pr_build_bvh_many_ex", "pr_trace", "pr_trace_frames", "pr_trace_work", "pr_scene_error",
            "pr_scene_bounds", "pr_scene_read_bvh", "pr_scene_device_bytes", "pr_scene_kernel_launches",
            "pr_scene_destroy", "pr_lbvh_build", "pr_lbvh_build_noalloc", "pr_batch_create", "pr_batch_set_tuning", "pr_batch_get_tuning", "pr_trace_batch",
            "pr_trace_batch_graph", "pr_batch_autotune", "pr_batch_device_bytes", "pr_batch_destroy",
            "pr_server_create", "pr_server_submit", "pr_server_poll", "pr_server_drain", "pr_server_get_stats",
            "pr_server_destroy", "pr_fma_peak_probe"]
PR_SERVE_CONTINUOUS, PR_SERVE_PLAIN = 0, 1


def _check(status: int, where: str):
    if status != PR_OK:
        raise PrError(status, where)


def build_bvh_many(scenes, stream=None, flags: int = 0):
    """pr_build_bvh_many(_ex): the BVHs of many scenes, built concurrently on internal
    streams ordered after (and joined back into) `stream`; flags: PR_BUILD_*."""
    arr = (ctypes.c_void_p * len(scenes))(*[sc._h.value for sc in scenes])
    if flags:
        _check(_lib.pr_build_bvh_many_ex(arr, len(scenes), flags, _stream_handle(stream)), "pr_build_bvh_many_ex")
    else:
        _check(_lib.pr_build_bvh_many(arr, len(scenes), _stream_handle(stream)), "pr_build_bvh_many")


def version() -> int:
    return int(_lib.pr_version())


def sbt_index(r: int, m: int, g: int, i: int, n_records: int) -> Optional[int]:
    """Eq. 1 on the host; None when the index falls outside the table."""
    out = ctypes.c_uint32()
    st = _lib.pr_sbt_index(r, m, g, i, n_records, ctypes.byref(out))
    return None if st == PR_ERR_SBT_INDEX else (_check(st, "pr_sbt_index") or int(out.value))


class _DescRef:
    """Contiguous copies of a description's arrays plus the ctypes struct pointing at them."""

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
        d = _SceneDesc()
        d.struct_size = ctypes.sizeof(_SceneDesc)
        a = self.arrays
        d.n_prims, d.n_geoms, d.n_blas = len(a["aabbs"]), len(a["geom_prim_begin"]), len(a["blas_geom_begin"])
        d.n_inst, d.n_hit_groups, d.n_materials = len(a["inst_blas"]), len(a["hit_groups"]), len(a["materials"])
        d.n_records, d.n_ray_types, d.sbt_stride_m = len(a["sbt"]), len(a["ray_types"]), int(sc.sbt_stride_m)
        for k, v in a.items():
            setattr(d, k, v.ctypes.data if v.size else None)
        gt = getattr(sc, "geom_type", None)
        tri = dict(vertices=c(getattr(sc, "vertices", np.zeros((0, 3))), np.float32).reshape(-1, 3),
                   indices=c(getattr(sc, "indices", np.zeros((0, 3))), np.uint32).reshape(-1, 3))
        if gt is not None:
            tri["geom_type"] = c(gt, np.uint32)
            d.geom_type = tri["geom_type"].ctypes.data
        d.n_vertices, d.n_triangles = len(tri["vertices"]), len(tri["indices"])
        d.vertices = tri["vertices"].ctypes.data if d.n_vertices else None
        d.indices = tri["indices"].ctypes.data if d.n_triangles else None
        self.arrays.update(tri)
        self.struct = d
        self.nbytes = int(sum(v.nbytes for v in self.arrays.values()))


def validate(desc) -> None:
    ref = _DescRef(desc)
    _check(_lib.pr_scene_validate(ctypes.byref(ref.struct)), "pr_scene_validate")


def _camera(cam) -> _Camera:
    c = _Camera()
    c.eye[:] = [float(v) for v in cam.eye]
    c.look_at[:] = [float(v) for v in cam.look_at]
    c.up[:] = [float(v) for v in cam.up]
    c.vfov_deg = float(cam.vfov_deg)
    return c


def trace_params(tp, aov: bool = False, extra_flags: int = 0) -> _TraceParams:
    p = _TraceParams()
    p.struct_size = ctypes.sizeof(_TraceParams)
    p.width, p.height, p.max_depth, p.max_steps = tp.width, tp.height, tp.max_depth, tp.max_steps
    p.flags = (PR_TRACE_WRITE_AOV if aov else 0) | extra_flags
    p.light_pos[:] = [float(v) for v in tp.light_pos]
    p.light_intensity, p.eps_rel, p.ambient = float(tp.light_intensity), float(tp.eps_rel), float(tp.ambient)
    p.background[:] = [float(v) for v in tp.background]
    return p


def _check_image(out, lead: tuple, rgb: bool):
    """The output tensor: contiguous float32 on the GPU, lead dims + 3 or 4 channels."""
    import torch
    want = tuple(lead) + (3 if rgb else 4,)
    if (tuple(out.shape) != want or out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous()):
        raise ValueError(f"output image must be a contiguous float32 CUDA tensor of shape {want}")


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _dptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class CameraArray:
    """Cameras marshalled once into a C array (reuse it across launches)."""

    def __init__(self, cameras: Sequence):
        self.n = len(cameras)
        self.array = (_Camera * self.n)(*[_camera(c) for c in cameras])

    def __len__(self):
        return self.n


class Scene:
    """A scene on the device: inputs, BVH, shader binding table (pr_scene)."""

    def __init__(self, desc, stream=None, build: bool = True, build_flags: int = 0):
        self._h = ctypes.c_void_p()
        ref = _DescRef(desc)
        self.n_inst = len(ref.arrays["inst_blas"])
        self.n_blas = len(ref.arrays["blas_geom_begin"])
        _check(_lib.pr_scene_create(ctypes.byref(ref.struct), _stream_handle(stream), ctypes.byref(self._h)),
               "pr_scene_create")
        self.desc_bytes = ref.nbytes
        if build:
            self.build_bvh(stream, build_flags)

    def upload(self, desc, stream=None):
        ref = _DescRef(desc)
        _check(_lib.pr_scene_upload(self._h, ctypes.byref(ref.struct), _stream_handle(stream)), "pr_scene_upload")

    def build_bvh(self, stream=None, flags: int = 0):
        """pr_build_bvh, or pr_build_bvh_ex with PR_BUILD_* flags."""
        if flags:
            _check(_lib.pr_build_bvh_ex(self._h, flags, _stream_handle(stream)), "pr_build_bvh_ex")
        else:
            _check(_lib.pr_build_bvh(self._h, _stream_handle(stream)), "pr_build_bvh")

    def trace(self, camera, params, out=None, aov=None, ray_counter=None, stream=None, want_aov: bool = False,
              binary_tlas: bool = False, rgb: bool = False):
        """Render one frame. Returns the float32 [H, W, 4] device tensor ([H, W, 3]
        with rgb, or when out has 3 channels) and the uint8 [H, W, 48] AOV tensor
        when want_aov or aov is given. binary_tlas traverses the binary TLAS
        instead of its 4-wide collapse."""
        import torch
        W, H = params.width, params.height
        rgb = rgb or (out is not None and out.shape[-1] == 3)
        if out is None:
            out = torch.empty((H, W, 3 if rgb else 4), dtype=torch.float32, device="cuda")
        _check_image(out, (H, W), rgb)
        if want_aov and aov is None:
            aov = torch.empty((H, W, AOV_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        cam = _camera(camera)
        tp = trace_params(params, aov is not None,
                          (PR_TRACE_TLAS_BVH2 if binary_tlas else 0) | (PR_TRACE_OUTPUT_RGB if rgb else 0))
        _check(_lib.pr_trace(self._h, ctypes.byref(cam), ctypes.byref(tp), _dptr(out), _dptr(aov), _dptr(ray_counter),
                             _stream_handle(stream)), "pr_trace")
        return (out, aov) if aov is not None else out

    def trace_frames(self, cameras: Sequence, params, out=None, aov=None, ray_counter=None, stream=None,
                     want_aov: bool = False, binary_tlas: bool = False, rgb: bool = False):
        import torch
        n = len(cameras)
        W, H = params.width, params.height
        rgb = rgb or (out is not None and out.shape[-1] == 3)
        if out is None:
            out = torch.empty((n, H, W, 3 if rgb else 4), dtype=torch.float32, device="cuda")
        _check_image(out, (n, H, W), rgb)
        if want_aov and aov is None:
            aov = torch.empty((n, H, W, AOV_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        cams = cameras.array if isinstance(cameras, CameraArray) else CameraArray(cameras).array
        tp = trace_params(params, aov is not None,
                          (PR_TRACE_TLAS_BVH2 if binary_tlas else 0) | (PR_TRACE_OUTPUT_RGB if rgb else 0))
        _check(_lib.pr_trace_frames(self._h, cams, n, ctypes.byref(tp), _dptr(out), _dptr(aov), _dptr(ray_counter),
                                    _stream_handle(stream)), "pr_trace_frames")
        return (out, aov) if aov is not None else out

    def trace_work(self, camera, params, out=None, stream=None, cameras=None, binary_tlas: bool = False) -> dict:
        """Instrumented trace (one camera, or a list of cameras for a multi-frame
        launch): returns the work counters (see PR_WORK_COUNTERS)."""
        import torch
        if cameras is None:
            cameras = [camera]
        ca = cameras if isinstance(cameras, CameraArray) else CameraArray(cameras)
        if out is None:
            out = torch.empty((len(ca), params.height, params.width, 4), dtype=torch.float32, device="cuda")
        _check_image(out, (len(ca), params.height, params.width), False)
        work = torch.zeros(len(WORK_FIELDS), dtype=torch.int64, device="cuda")
        arr = ca.array
        cams = ca
        tp = trace_params(params, False, PR_TRACE_TLAS_BVH2 if binary_tlas else 0)
        _check(_lib.pr_trace_work(self._h, arr, len(cams), ctypes.byref(tp), _dptr(out), _dptr(work),
                                  _stream_handle(stream)), "pr_trace_work")
        torch.cuda.synchronize()          # the launch stream may not be torch's current stream
        vals = work.cpu().tolist()
        return dict(zip(WORK_FIELDS, vals))

    def error_word(self, stream=None) -> int:
        w = ctypes.c_uint32()
        _check(_lib.pr_scene_error(self._h, _stream_handle(stream), ctypes.byref(w)), "pr_scene_error")
        return int(w.value)

    def bounds(self, stream=None) -> np.ndarray:
        b = np.zeros(6, np.float32)
        _check(_lib.pr_scene_bounds(self._h, _stream_handle(stream), b.ctypes.data), "pr_scene_bounds")
        return b

    def read_bvh(self, level: int = PR_NONE, stream=None):
        """One built BVH level (PR_NONE = TLAS) as host arrays: perm, codes, child, cbox, root."""
        n = ctypes.c_uint32()
        h = _stream_handle(stream)
        _check(_lib.pr_scene_read_bvh(self._h, level, h, 0, ctypes.byref(n), None, None, None, None, None),
               "pr_scene_read_bvh(size)")
        k = int(n.value)
        perm = np.zeros(max(k, 1), np.uint32)
        codes = np.zeros(max(k, 1), np.uint32)
        child = np.zeros((max(k - 1, 1), 2), np.int32)
        cbox = np.zeros((max(k - 1, 1), 12), np.float32)
        root = np.zeros(6, np.float32)
        _check(_lib.pr_scene_read_bvh(self._h, level, h, k, ctypes.byref(n), perm.ctypes.data, codes.ctypes.data,
                                      child.ctypes.data, cbox.ctypes.data, root.ctypes.data), "pr_scene_read_bvh")
        return dict(perm=perm[:k], codes=codes[:k], child=child[:max(k - 1, 0)], cbox=cbox[:max(k - 1, 0)], root=root)

    def kernel_launches(self):
        """(build, trace) kernels enqueued by the most recent build and trace calls."""
        b, t = ctypes.c_uint32(), ctypes.c_uint32()
        _check(_lib.pr_scene_kernel_launches(self._h, ctypes.byref(b), ctypes.byref(t)), "pr_scene_kernel_launches")
        return int(b.value), int(t.value)

    def device_bytes(self) -> int:
        return int(_lib.pr_scene_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.pr_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbvh_build(boxes, stream=None) -> dict:
    """LBVH over a float32 [n, 6] device tensor of boxes (pr_lbvh_build).
    Returns device tensors: nodes [n-1, 16] float32, perm, codes [n] int32 views
    of uint32, root [8] float32."""
    import torch
    n = int(boxes.shape[0])
    assert boxes.is_cuda and boxes.dtype == torch.float32 and boxes.is_contiguous()
    nodes = torch.empty((max(n - 1, 1), 16), dtype=torch.float32, device=boxes.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=boxes.device)
    codes = torch.empty(max(n, 1), dtype=torch.int32, device=boxes.device)
    root = torch.zeros(8, dtype=torch.float32, device=boxes.device)
    _check(_lib.pr_lbvh_build(_dptr(boxes), n, _dptr(nodes), _dptr(perm), _dptr(codes), _dptr(root),
                              _stream_handle(stream)), "pr_lbvh_build")
    return dict(nodes=nodes[:max(n - 1, 0)], perm=perm[:n], codes=codes[:n], root=root)


def fma_peak_probe(iters: int = 16384, stream=None) -> tuple:
    """Measured FP32 FMA throughput of the current GPU (pr_fma_peak_probe):
    returns (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_float(), ctypes.c_float()
    _check(_lib.pr_fma_peak_probe(int(iters), ctypes.byref(tf), ctypes.byref(ms), _stream_handle(stream)),
           "pr_fma_peak_probe")
    return float(tf.value), float(ms.value)


def lbvh_to_host(res) -> dict:
    """Device LBVH tensors -> host arrays in the layout of Scene.read_bvh."""
    nodes = res["nodes"].cpu().numpy()
    child = nodes[:, 12:14].copy().view(np.int32)
    root = res["root"].cpu().numpy()
    return dict(perm=res["perm"].cpu().numpy().view(np.uint32), codes=res["codes"].cpu().numpy().view(np.uint32),
                child=child, cbox=nodes[:, :12].copy(), root=np.concatenate([root[0:3], root[4:7]]))


class _Request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("camera", _Camera), ("params", _TraceParams), ("out_rgba", ctypes.c_void_p),
                ("row_begin", ctypes.c_uint32), ("row_count", ctypes.c_uint32)]


class _BatchTuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("struct_size", "ctas_per_sm", "tile_w", "tile_h", "queue_chunk",
                                               "megakernel")]


class Batch:
    """Batched wavefront renderer (pr_batch): many requests, one set of persistent kernels."""

    def __init__(self, max_requests: int, max_pixels: int):
        self._h = ctypes.c_void_p()
        _check(_lib.pr_batch_create(max_requests, max_pixels, ctypes.byref(self._h)), "pr_batch_create")
        self._keep = None

    @staticmethod
    def _requests(items):
        """items: sequence of (Scene, camera, params, out_tensor[, row_begin, row_count])."""
        arr = (_Request * len(items))()
        for k, it in enumerate(items):
            sc, cam, tp, out = it[:4]
            arr[k].scene = sc._h.value
            arr[k].camera = _camera(cam)
            rgb = out.shape[-1] == 3
            _check_image(out, (tp.height, tp.width), rgb)
            arr[k].params = trace_params(tp, False, PR_TRACE_OUTPUT_RGB if rgb else 0)
            arr[k].out_rgba = out.data_ptr()
            if len(it) > 4:
                arr[k].row_begin, arr[k].row_count = int(it[4]), int(it[5])
        return arr

    def prepare(self, items):
        """Marshal a request list once, for repeated trace(prepared=...) calls."""
        return self._requests(items)

    def trace(self, items=None, ray_counter=None, stream=None, graph: bool = False, prepared=None):
        arr = prepared if prepared is not None else self._requests(items)
        items = arr
        self._keep = arr
        fn = _lib.pr_trace_batch_graph if graph else _lib.pr_trace_batch
        _check(fn(self._h, len(items), arr, _dptr(ray_counter), _stream_handle(stream)),
               "pr_trace_batch_graph" if graph else "pr_trace_batch")

    def autotune(self, items, stream=None):
        arr = self._requests(items)
        best = _BatchTuning()
        ms = ctypes.c_float()
        _check(_lib.pr_batch_autotune(self._h, len(items), arr, _stream_handle(stream), ctypes.byref(best),
                                      ctypes.byref(ms)), "pr_batch_autotune")
        return dict(ctas_per_sm=best.ctas_per_sm, tile_w=best.tile_w, tile_h=best.tile_h,
                    queue_chunk=best.queue_chunk, megakernel=best.megakernel), float(ms.value)

    def set_tuning(self, ctas_per_sm, tile_w, tile_h, queue_chunk, megakernel=0):
        t = _BatchTuning(ctypes.sizeof(_BatchTuning), ctas_per_sm, tile_w, tile_h, queue_chunk, megakernel)
        _check(_lib.pr_batch_set_tuning(self._h, ctypes.byref(t)), "pr_batch_set_tuning")

    def tuning(self) -> dict:
        t = _BatchTuning()
        _check(_lib.pr_batch_get_tuning(self._h, ctypes.byref(t)), "pr_batch_get_tuning")
        return dict(ctas_per_sm=t.ctas_per_sm, tile_w=t.tile_w, tile_h=t.tile_h, queue_chunk=t.queue_chunk,
                    megakernel=t.megakernel)

    def device_bytes(self) -> int:
        return int(_lib.pr_batch_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.pr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ServerConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("max_active", ctypes.c_uint32),
                ("solo_max_waiting", ctypes.c_uint32), ("mem_budget_bytes", ctypes.c_uint64),
                ("max_batch_pixels", ctypes.c_uint64), ("tuning", _BatchTuning)]


class _ServerRequest(ctypes.Structure):
    _fields_ = [("scene_key", ctypes.c_uint64), ("desc", ctypes.c_void_p), ("camera", _Camera),
                ("params", _TraceParams), ("out_rgba", ctypes.c_void_p)]


class _RequestStats(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_first_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_uint32), ("cache_hit", ctypes.c_uint32),
                ("t_load_start", ctypes.c_double), ("t_load_end", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("reserved", ctypes.c_uint32)] + [
        (n, ctypes.c_uint64) for n in ("submitted", "completed", "rays", "iterations", "cache_hits", "cache_misses",
                                       "evictions", "cache_bytes", "batch_bytes", "scene_loads")]


class Server:
    """Serving loop (pr_server): admission by memory budget, scene cache, continuous batching."""

    def __init__(self, mode=PR_SERVE_CONTINUOUS, max_active=64, mem_budget_bytes=100 << 30,
                 max_batch_pixels=16 << 20, tuning: Optional[dict] = None, solo_max_waiting: int = 0):
        cfg = _ServerConfig()
        cfg.struct_size = ctypes.sizeof(_ServerConfig)
        cfg.mode, cfg.max_active, cfg.solo_max_waiting = mode, max_active, solo_max_waiting
        cfg.mem_budget_bytes, cfg.max_batch_pixels = mem_budget_bytes, max_batch_pixels
        if tuning:
            cfg.tuning = _BatchTuning(ctypes.sizeof(_BatchTuning), tuning["ctas_per_sm"], tuning["tile_w"],
                                      tuning["tile_h"], tuning["queue_chunk"], tuning.get("megakernel", 0))
        self._h = ctypes.c_void_p()
        _check(_lib.pr_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "pr_server_create")

    def submit(self, key: int, desc, camera, params, out) -> int:
        """desc: a scene description object (or None if the key is resident)."""
        r = _ServerRequest()
        r.scene_key = key
        ref = _DescRef(desc) if desc is not None else None
        r.desc = ctypes.addressof(ref.struct) if ref is not None else None
        r.camera = _camera(camera)
        rgb = out.shape[-1] == 3
        _check_image(out, (params.height, params.width), rgb)
        r.params = trace_params(params, False, PR_TRACE_OUTPUT_RGB if rgb else 0)
        r.out_rgba = out.data_ptr()
        t = ctypes.c_uint64()
        _check(_lib.pr_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "pr_server_submit")
        return int(t.value)

    def poll(self, ticket: int):
        done = ctypes.c_int()
        st = _RequestStats()
        _check(_lib.pr_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(st)), "pr_server_poll")
        return bool(done.value), {k: getattr(st, k) for k, _ in _RequestStats._fields_}

    def drain(self, timeout_s: float = 600.0):
        _check(_lib.pr_server_drain(self._h, timeout_s), "pr_server_drain")

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_lib.pr_server_get_stats(self._h, ctypes.byref(st)), "pr_server_get_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_ if k not in ("struct_size", "reserved")}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.pr_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aov_to_numpy(aov_tensor) -> np.ndarray:
    """Device AOV bytes -> structured numpy array with AOV_DTYPE."""
    a = aov_tensor.detach().cpu().numpy()
    return a.reshape(-1).view(AOV_DTYPE).reshape(a.shape[:-1])
