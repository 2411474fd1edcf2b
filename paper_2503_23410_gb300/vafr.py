"""Thin ctypes binding of libvafr.so (include/vafr.h): argument marshalling only.

Every function named ``vafr_*`` here calls the C entry point of the same name.
Buffers may be torch tensors (device memory; ``data_ptr()`` is passed) or
numpy arrays (host memory).  Streams default to torch's current CUDA stream.
There is no fallback: if libvafr.so is missing or fails to load, importing the
binding raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvafr.so")

FMT_RGBA32F = 0
FMT_RGBA16F = 1
MAX_PIVOTS = 9
MAX_BATCH = 128

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_BUDGET = -5
ERR_DEVICE = -6
ERR_UNSUPPORTED = -7


class VafrError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str):
        super().__init__(f"vafr error {code} ({what}): {detail}")
        self.code = code


class vafr_acuity(ctypes.Structure):
    _fields_ = [("n_pivots", ctypes.c_int32),
                ("pivot_ecc_deg", ctypes.c_double * MAX_PIVOTS),
                ("pivot_cpd", ctypes.c_double * MAX_PIVOTS),
                ("e_max_deg", ctypes.c_double),
                ("anisotropic", ctypes.c_int32),
                ("pivot_delta", ctypes.c_double * MAX_PIVOTS)]


class vafr_session_desc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fov_v_deg", ctypes.c_double), ("n_eyes", ctypes.c_int32),
                ("eye_pose", (ctypes.c_double * 12) * 2),
                ("lp_format", ctypes.c_int32), ("display_format", ctypes.c_int32),
                ("acuity", vafr_acuity), ("lp_fxaa", ctypes.c_int32)]


class vafr_frame_desc(ctypes.Structure):
    _fields_ = [("session", ctypes.c_void_p), ("eye", ctypes.c_int32),
                ("lp", ctypes.c_void_p), ("display", ctypes.c_void_p),
                ("lp_aa", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PROTOS = {
    "vafr_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "vafr_last_error_message": (ctypes.c_char_p, []),
    "vafr_version": (_I32, []),
    "vafr_kernel_launch_count": (_I64, []),
    "vafr_acuity_default": (None, [_P]),
    "vafr_acuity_anisotropic": (None, [_P]),
    "vafr_acuity_display_limited": (ctypes.c_int, [_P, ctypes.c_double]),
    "vafr_build_scene": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P]),
    "vafr_scene_destroy": (ctypes.c_int, [_P]),
    "vafr_scene_info": (ctypes.c_int, [_P, _P, _P]),
    "vafr_scene_export_lbvh": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "vafr_scene_check": (ctypes.c_int, [_P, _P]),
    "vafr_scene_inject_fault": (ctypes.c_int, [_P, ctypes.c_int32]),
    "vafr_debug_fail_host_alloc": (ctypes.c_int, [ctypes.c_int32]),
    "vafr_scene_export_tree4": (ctypes.c_int, [_P, _P, _P, _P]),
    "vafr_session_create": (ctypes.c_int, [_P, _P]),
    "vafr_session_destroy": (ctypes.c_int, [_P]),
    "vafr_lp_layout": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "vafr_session_sizes": (ctypes.c_int, [_P, _P, _P]),
    "vafr_session_tuning": (ctypes.c_int, [_P, _I32, _P]),
    "vafr_set_gaze": (ctypes.c_int, [_P, _I32, ctypes.c_double, ctypes.c_double]),
    "vafr_session_check": (ctypes.c_int, [_P, _P]),
    "vafr_render_lp": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "vafr_reconstruct": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "vafr_fxaa_lp": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "vafr_render_lp_pt": (ctypes.c_int, [_P, _P, _I32, _P, ctypes.c_uint64, _I32, _P, _P]),
    "vafr_render_full_gt_pt": (ctypes.c_int, [_P, _P, _I32, _P, ctypes.c_uint64, _I32, _P]),
    "vafr_render_lp_rep": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "vafr_scene_set_point_lights": (ctypes.c_int, [_P, _I32, _P, _P]),
    "vafr_render_vbuffer": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "vafr_vbuffer_stats": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "vafr_shade_lp_deferred": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "vafr_shade_full_deferred": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "vafr_reproject_lp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "vafr_rep_hole_count": (ctypes.c_int, [_P, _P, _P]),
    "vafr_render_full_gt": (ctypes.c_int, [_P, _P, _I32, _P, _P, _P]),
    "vafr_render_frame": (ctypes.c_int, [_P, _P, _P, _P]),
    "vafr_traversal_stats": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "vafr_measure_fp32_peak": (ctypes.c_int, [_P, _P]),
    "vafr_session_autotune": (ctypes.c_int, [_P, _P, _P, _P, _I32, _I32, _P, _P]),
    "vafr_batch_create": (ctypes.c_int, [_P, _I32, _P]),
    "vafr_batch_destroy": (ctypes.c_int, [_P]),
    "vafr_batch_render": (ctypes.c_int, [_P, _P, _I32, _P]),
    "vafr_batch_capture": (ctypes.c_int, [_P, _P, _I32, _P]),
    "vafr_batch_replay": (ctypes.c_int, [_P, _P]),
    "vafr_batch_autotune": (ctypes.c_int, [_P, _P, _I32, _P, _I32]),
    "vafr_batch_tuning": (ctypes.c_int, [_P, _I32, _P]),
    "vafr_tuning_space": (ctypes.c_int, [_P, _P]),
    "vafr_morton_sort_noalloc": (ctypes.c_int, [_P, _I64, _P, _P, _P, ctypes.c_char_p, _I32]),
}

NOALLOC_MAX_TRIS = 524288

_lib = None


def load(path: str = LIB_PATH):
    """Load libvafr.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing; build it with paper_2503_23410_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int) -> None:
    if rc != OK:
        L = load()
        raise VafrError(rc, L.vafr_error_string(rc).decode(), L.vafr_last_error_message().decode())


def ptr(x) -> Optional[int]:
    """Address of a torch tensor, numpy array or raw int (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_ptr(stream=None) -> Optional[int]:
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# one Python function per C entry point


def vafr_error_string(code: int) -> str:
    return load().vafr_error_string(code).decode()


def vafr_last_error_message() -> str:
    return load().vafr_last_error_message().decode()


def vafr_version() -> int:
    return int(load().vafr_version())


def vafr_kernel_launch_count() -> int:
    return int(load().vafr_kernel_launch_count())


def vafr_acuity_default() -> vafr_acuity:
    a = vafr_acuity()
    load().vafr_acuity_default(ctypes.byref(a))
    return a


def vafr_acuity_anisotropic() -> vafr_acuity:
    a = vafr_acuity()
    load().vafr_acuity_anisotropic(ctypes.byref(a))
    return a


def vafr_acuity_display_limited(max_cpd: float) -> vafr_acuity:
    a = vafr_acuity()
    _check(load().vafr_acuity_display_limited(ctypes.byref(a), float(max_cpd)))
    return a


def make_acuity(pivots_deg: Sequence[float], pivots_cpd: Sequence[float],
                e_max_deg: float = 60.0, delta: Optional[Sequence[float]] = None) -> vafr_acuity:
    a = vafr_acuity()
    a.n_pivots = len(pivots_deg)
    for k, (e, f) in enumerate(zip(pivots_deg, pivots_cpd)):
        a.pivot_ecc_deg[k] = float(e)
        a.pivot_cpd[k] = float(f)
        a.pivot_delta[k] = 1.0
    a.e_max_deg = float(e_max_deg)
    if delta is not None:
        a.anisotropic = 1
        for k, d in enumerate(delta):
            a.pivot_delta[k] = float(d)
    return a


def _require_f32(x, name):
    if x is None:
        return
    dt = str(getattr(x, "dtype", ""))
    if dt not in ("float32", "torch.float32"):
        raise TypeError(f"{name} must be float32, got {dt}")


def vafr_build_scene(tri_xyz, albedo_rgb, light_dir, stream=None) -> int:
    n = int(tri_xyz.shape[0]) if tri_xyz is not None else 0
    _require_f32(tri_xyz, "tri_xyz")
    _require_f32(albedo_rgb, "albedo_rgb")
    L = (ctypes.c_float * 3)(*[float(v) for v in np.asarray(light_dir).reshape(3)])
    out = ctypes.c_void_p()
    _check(load().vafr_build_scene(ptr(tri_xyz) if n else None, ptr(albedo_rgb), n,
                                   ctypes.cast(L, ctypes.c_void_p), stream_ptr(stream),
                                   ctypes.byref(out)))
    return out.value


def vafr_scene_destroy(scene: int) -> None:
    _check(load().vafr_scene_destroy(scene))


def vafr_scene_info(scene: int):
    n, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().vafr_scene_info(scene, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def vafr_scene_export_lbvh(scene: int):
    n, _ = vafr_scene_info(scene)
    codes = np.zeros(n, np.uint32)
    ids = np.zeros(n, np.int32)
    ni = max(n - 1, 0)
    child = np.zeros((max(ni, 1), 2), np.int32)
    nb = np.zeros((max(ni, 1), 6), np.float32)
    lb = np.zeros((max(n, 1), 6), np.float32)
    _check(load().vafr_scene_export_lbvh(scene, ptr(codes), ptr(ids), ptr(child), ptr(nb), ptr(lb)))
    return codes, ids, child[:ni], nb[:ni], lb[:n]


def vafr_scene_export_tree4(scene: int):
    """(nodes (n_nodes, 32) float32, leaves (n_tris, 12) float32) of the traversal tree."""
    n, _ = vafr_scene_info(scene)
    cnt = ctypes.c_int64()
    _check(load().vafr_scene_export_tree4(scene, ctypes.byref(cnt), None, None))
    nodes = np.zeros((max(cnt.value, 1), 32), np.float32)
    leaves = np.zeros((max(n, 1), 12), np.float32)
    _check(load().vafr_scene_export_tree4(scene, ctypes.byref(cnt), ptr(nodes), ptr(leaves)))
    return nodes[:cnt.value], leaves[:n]


def vafr_scene_check(scene: int, stream=None) -> int:
    return int(load().vafr_scene_check(scene, stream_ptr(stream)))


INJECT_NONE, INJECT_BAD_CHILD, INJECT_LOOP, INJECT_STACK = 0, 1, 2, 3


def vafr_scene_inject_fault(scene: int, kind: int) -> None:
    _check(load().vafr_scene_inject_fault(scene, int(kind)))


def vafr_debug_fail_host_alloc(countdown: int) -> None:
    _check(load().vafr_debug_fail_host_alloc(int(countdown)))


def vafr_session_create(desc: vafr_session_desc) -> int:
    out = ctypes.c_void_p()
    _check(load().vafr_session_create(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def make_session_desc(width, height, fov_v_deg, poses, lp_format=FMT_RGBA32F,
                      display_format=FMT_RGBA32F, acuity: Optional[vafr_acuity] = None,
                      lp_fxaa: bool = False):
    d = vafr_session_desc()
    d.width, d.height, d.fov_v_deg = int(width), int(height), float(fov_v_deg)
    d.n_eyes = len(poses)
    for e, P in enumerate(poses):
        flat = np.asarray(P, np.float64).reshape(12)
        for k in range(12):
            d.eye_pose[e][k] = float(flat[k])
    d.lp_format, d.display_format = int(lp_format), int(display_format)
    d.acuity = acuity if acuity is not None else vafr_acuity_default()
    d.lp_fxaa = 1 if lp_fxaa else 0
    return d


def vafr_session_destroy(session: int) -> None:
    _check(load().vafr_session_destroy(session))


def vafr_lp_layout(session: int):
    nc, nt = ctypes.c_int32(), ctypes.c_int64()
    _check(load().vafr_lp_layout(session, ctypes.byref(nc), ctypes.byref(nt), None, None, None))
    counts = np.zeros(nc.value, np.int32)
    offs = np.zeros(nc.value, np.int64)
    ecc = np.zeros(nc.value, np.float32)
    _check(load().vafr_lp_layout(session, None, None, ptr(counts), ptr(offs), ptr(ecc)))
    return counts, offs, ecc, nt.value


def vafr_session_sizes(session: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().vafr_session_sizes(session, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def vafr_session_tuning(session: int, cfg: Optional[Sequence[int]] = None):
    c = (ctypes.c_int32 * 2)(*(cfg if cfg is not None else (0, 0)))
    _check(load().vafr_session_tuning(session, 1 if cfg is not None else 0,
                                      ctypes.cast(c, ctypes.c_void_p)))
    return int(c[0]), int(c[1])


def vafr_session_autotune(scene: int, session: int, lp, display, warm: int = 3, iters: int = 5,
                          stream=None):
    """Times every render and reconstruct variant on whole frames at the
    current gaze, keeps the fastest pair and returns it."""
    c = (ctypes.c_int32 * 2)(0, 0)
    _check(load().vafr_session_autotune(scene, session, ptr(lp), ptr(display), int(warm), int(iters),
                                        ctypes.cast(c, ctypes.c_void_p), stream_ptr(stream)))
    return int(c[0]), int(c[1])


def vafr_set_gaze(session: int, eye: int, x0: float, y0: float) -> None:
    _check(load().vafr_set_gaze(session, int(eye), float(x0), float(y0)))


def vafr_session_check(session: int, stream=None) -> int:
    return int(load().vafr_session_check(session, stream_ptr(stream)))


def vafr_render_lp(scene: int, session: int, eye_mask: int, lp_out, hit_ids_out=None,
                   stream=None) -> None:
    _check(load().vafr_render_lp(scene, session, int(eye_mask), ptr(lp_out), ptr(hit_ids_out),
                                 stream_ptr(stream)))


def vafr_reconstruct(session: int, eye: int, lp, display_out, stream=None) -> None:
    _check(load().vafr_reconstruct(session, int(eye), ptr(lp), ptr(display_out), stream_ptr(stream)))


def vafr_render_lp_pt(scene: int, session: int, eye_mask: int, lp_out, seed: int,
                      max_diffuse: int = 3, path_sig_out=None, stream=None) -> None:
    _check(load().vafr_render_lp_pt(scene, session, int(eye_mask), ptr(lp_out),
                                    int(seed) & (2 ** 64 - 1), int(max_diffuse),
                                    ptr(path_sig_out), stream_ptr(stream)))


def vafr_render_full_gt_pt(scene: int, session: int, eye: int, display_out, seed: int,
                           max_diffuse: int = 3, stream=None) -> None:
    _check(load().vafr_render_full_gt_pt(scene, session, int(eye), ptr(display_out),
                                         int(seed) & (2 ** 64 - 1), int(max_diffuse), stream_ptr(stream)))


def vafr_scene_set_point_lights(scene: int, positions, rgb) -> None:
    pos = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
    col = np.ascontiguousarray(rgb, np.float32).reshape(-1, 3)
    if pos.shape != col.shape:
        raise ValueError("positions and colours differ in shape")
    _check(load().vafr_scene_set_point_lights(scene, pos.shape[0], pos.ctypes.data, col.ctypes.data))


def vafr_render_vbuffer(scene: int, session: int, eye: int, vbuf_out, stream=None) -> None:
    _check(load().vafr_render_vbuffer(scene, session, int(eye), ptr(vbuf_out), stream_ptr(stream)))


def vafr_vbuffer_stats(scene: int, session: int, eye: int, vbuf_out, stream=None):
    out = np.zeros(4, np.int64)
    _check(load().vafr_vbuffer_stats(scene, session, int(eye), ptr(vbuf_out), ptr(out), stream_ptr(stream)))
    return {"prefilter": int(out[0]), "filtered": int(out[1]), "tests": int(out[2]), "atomics": int(out[3])}


def vafr_shade_lp_deferred(scene: int, session: int, eye: int, vbuf, lp_out, stream=None) -> None:
    _check(load().vafr_shade_lp_deferred(scene, session, int(eye), ptr(vbuf), ptr(lp_out), stream_ptr(stream)))


def vafr_shade_full_deferred(scene: int, session: int, eye: int, vbuf, display_out, stream=None) -> None:
    _check(load().vafr_shade_full_deferred(scene, session, int(eye), ptr(vbuf), ptr(display_out),
                                           stream_ptr(stream)))


def vafr_render_lp_rep(scene: int, session: int, lp_out, right_tri_out=None, stream=None) -> None:
    _check(load().vafr_render_lp_rep(scene, session, ptr(lp_out), ptr(right_tri_out), stream_ptr(stream)))


def vafr_reproject_lp(session: int, left_lp, left_depth, right_lp_out, right_tri_out=None,
                      stream=None) -> None:
    _check(load().vafr_reproject_lp(session, ptr(left_lp), ptr(left_depth), ptr(right_lp_out),
                                    ptr(right_tri_out), stream_ptr(stream)))


def vafr_rep_hole_count(session: int, stream=None) -> int:
    out = ctypes.c_int64()
    _check(load().vafr_rep_hole_count(session, ctypes.byref(out), stream_ptr(stream)))
    return int(out.value)


def vafr_fxaa_lp(session: int, eye: int, lp, lp_out, stream=None) -> None:
    _check(load().vafr_fxaa_lp(session, int(eye), ptr(lp), ptr(lp_out), stream_ptr(stream)))


def vafr_render_full_gt(scene: int, session: int, eye: int, display_out, hit_ids_out=None,
                        stream=None) -> None:
    _check(load().vafr_render_full_gt(scene, session, int(eye), ptr(display_out),
                                      ptr(hit_ids_out), stream_ptr(stream)))


def vafr_render_frame(scene: int, session: int, display_out, stream=None) -> None:
    _check(load().vafr_render_frame(scene, session, ptr(display_out), stream_ptr(stream)))


def vafr_measure_fp32_peak(stream=None):
    """(scalar FFMA, paired FFMA2) FMAs per second of the current device."""
    out = np.zeros(2, np.float64)
    _check(load().vafr_measure_fp32_peak(ptr(out), stream_ptr(stream)))
    return float(out[0]), float(out[1])


def vafr_traversal_stats(scene: int, session: int, eye: int = 0, stream=None):
    out = np.zeros(6, np.int64)
    _check(load().vafr_traversal_stats(scene, session, int(eye), ptr(out), stream_ptr(stream)))
    return {"rays": int(out[0]), "nodes": int(out[1]), "box_tests": int(out[2]),
            "tri_tests": int(out[3]), "hits": int(out[4]), "max_nodes": int(out[5])}


def _frames(frames):
    """frames: (session, eye, lp, display) or (session, eye, lp, display, lp_aa)."""
    arr = (vafr_frame_desc * len(frames))()
    for i, fr in enumerate(frames):
        sess, eye, lp, disp = fr[:4]
        arr[i].session = sess
        arr[i].eye = int(eye)
        arr[i].lp = ptr(lp)
        arr[i].display = ptr(disp)
        arr[i].lp_aa = ptr(fr[4]) if len(fr) > 4 else None
    return arr


def vafr_batch_create(scene: int, max_frames: int = MAX_BATCH) -> int:
    out = ctypes.c_void_p()
    _check(load().vafr_batch_create(scene, int(max_frames), ctypes.byref(out)))
    return out.value


def vafr_batch_destroy(batch: int) -> None:
    _check(load().vafr_batch_destroy(batch))


def vafr_batch_render(batch: int, frames, stream=None) -> None:
    arr = _frames(frames)
    _check(load().vafr_batch_render(batch, ctypes.cast(arr, ctypes.c_void_p), len(frames),
                                    stream_ptr(stream)))


def vafr_batch_capture(batch: int, frames, stream=None) -> None:
    arr = _frames(frames)
    _check(load().vafr_batch_capture(batch, ctypes.cast(arr, ctypes.c_void_p), len(frames),
                                     stream_ptr(stream)))


def vafr_batch_replay(batch: int, stream=None) -> None:
    _check(load().vafr_batch_replay(batch, stream_ptr(stream)))


def vafr_batch_autotune(batch: int, frames, stream=None, iters: int = 3) -> None:
    arr = _frames(frames)
    _check(load().vafr_batch_autotune(batch, ctypes.cast(arr, ctypes.c_void_p), len(frames),
                                      stream_ptr(stream), int(iters)))


def vafr_batch_tuning(batch: int, cfg: Optional[Sequence[int]] = None):
    c = (ctypes.c_int32 * 2)(*(cfg if cfg is not None else (0, 0)))
    _check(load().vafr_batch_tuning(batch, 1 if cfg is not None else 0,
                                    ctypes.cast(c, ctypes.c_void_p)))
    return int(c[0]), int(c[1])


def vafr_tuning_space():
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().vafr_tuning_space(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _noalloc_n(tri_xyz, codes_out, sorted_ids_out) -> int:
    """Triangle count of vafr_morton_sort_noalloc's arguments, checked here
    because the C entry point cannot see buffer sizes: tri_xyz is (n, 9) (or
    flat with 9 n floats) FP32, both outputs hold at least n 32-bit integers."""
    _require_f32(tri_xyz, "tri_xyz")
    shape = tuple(tri_xyz.shape)
    if len(shape) == 2 and shape[1] == 9:
        n = int(shape[0])
    elif len(shape) == 1 and shape[0] % 9 == 0:
        n = int(shape[0]) // 9
    else:
        raise ValueError(f"tri_xyz must be (n, 9) or flat with 9 n floats, got shape {shape}")
    for name, buf in (("codes_out", codes_out), ("sorted_ids_out", sorted_ids_out)):
        dt = str(buf.dtype)
        if not any(dt.endswith(t) for t in ("int32", "uint32")):
            raise ValueError(f"{name} must hold 32-bit integers, got {dt}")
        count = int(buf.numel()) if hasattr(buf, "numel") else int(buf.size)
        if count < n:
            raise ValueError(f"{name} holds {count} elements, fewer than the {n} triangles")
    return n


def vafr_morton_sort_noalloc(tri_xyz, codes_out, sorted_ids_out, stream=None) -> None:
    """Morton codes + stable (code, id) order without any allocation (device buffers)."""
    n = _noalloc_n(tri_xyz, codes_out, sorted_ids_out)
    msg = ctypes.create_string_buffer(256)
    rc = load().vafr_morton_sort_noalloc(ptr(tri_xyz), n, ptr(codes_out), ptr(sorted_ids_out),
                                         stream_ptr(stream), msg, len(msg))
    if rc != OK:
        raise VafrError(rc, vafr_error_string(rc), msg.value.decode())
