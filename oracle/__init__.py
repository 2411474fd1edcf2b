"""FP64 CPU oracle of the VaFR ray-casting hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product path (the CUDA library in
``paper_2503_23410_gb300``) never does, and the two share no code.

All arithmetic lives in ``vafr_oracle.c`` (plain C, FP64, OpenMP); this module
only marshals numpy arrays.  Function-level citations are in the C file.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against values the paper prints (tests/golden/paper_constants.json), closed
forms, invariants, textbook special cases or brute force.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vafr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

PAPER_PIVOTS_DEG = (0.0, 10.0, 20.0, 30.0, 60.0)
PAPER_PIVOTS_CPD = (40.0, 10.0, 6.0, 5.0, 4.0)
PAPER_E_MAX = 60.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.or_acuity_init.argtypes = [P, P, P, ctypes.c_int]
        L.or_acuity_init.restype = ctypes.c_int
        L.or_acuity_set_delta.argtypes = [P, P]
        L.or_acuity_set_delta.restype = ctypes.c_int
        L.or_sizeof_acuity.restype = i64
        L.or_eval.argtypes = [P, ctypes.c_int, P, P, i64]
        L.or_acuity_get.argtypes = [P, P, P, P]
        L.or_lp_layout.argtypes = [P, ctypes.c_double, ctypes.c_int, P, P, P, P]
        L.or_lp_layout.restype = ctypes.c_int
        L.or_lp_rays.argtypes = [P, P, P, P, ctypes.c_int, P, i64, P, P, P]
        L.or_pixel_rays.argtypes = [P, P, i64, P, P]
        L.or_cast_brute.argtypes = [P, i64, P, P, i64, P, P]
        L.or_ray_tri_t.argtypes = [P, P, P, P, i64, P]
        L.or_edge_margin.argtypes = [P, P, P]
        L.or_edge_margin.restype = ctypes.c_double
        L.or_bvh_build.argtypes = [P, i64]
        L.or_bvh_build.restype = P
        L.or_bvh_free.argtypes = [P]
        L.or_cast_bvh.argtypes = [P, P, P, i64, P, P]
        L.or_shade.argtypes = [P, P, P, P, P, i64, P]
        L.or_grazing.argtypes = [P, P, P, i64, P]
        L.or_reconstruct_points.argtypes = [P, ctypes.c_double, P, P, P, ctypes.c_int,
                                            P, ctypes.c_int, P, i64, P]
        L.or_morton.argtypes = [P, i64, P]
        L.or_fxaa_lp.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P]
        L.or_shade_points.argtypes = [P, P, P, P, P, P, i64, ctypes.c_int, P, P, P]
        L.or_reproject_lp.argtypes = [P, ctypes.c_double, P, P, P, ctypes.c_int, i64, P, P, P, P, P, P]
        L.or_rep_probe.argtypes = [P, ctypes.c_double, P, P, P, ctypes.c_int, i64, P, P, P, i64, P, P, P]
        L.or_path_trace.argtypes = [P, P, P, P, P, P, i64, ctypes.c_uint64, ctypes.c_int, P, P, P]
        L.or_pt_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
        L.or_pt_uniform.restype = ctypes.c_double
        L.or_lp_neighbor.argtypes = [P, P, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, i64, P]
        L.or_lbvh.argtypes = [P, i64, P, P, P, P, P, P]
        L.or_lbvh.restype = ctypes.c_int
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# acuity model and mapping


class Acuity:
    """Segmented acuity model (Eq. 12) built from pivots (E_k deg, f_k cpd)."""

    def __init__(self, pivots_deg: Sequence[float] = PAPER_PIVOTS_DEG,
                 pivots_cpd: Sequence[float] = PAPER_PIVOTS_CPD,
                 delta: Optional[Sequence[float]] = None):
        """`delta`: tangential/radial shading-rate ratio at the pivots (Sec. 9,
        Eq. 19), or None for the isotropic mapping."""
        self.E = _c(pivots_deg, np.float64)
        self.f = _c(pivots_cpd, np.float64)
        self._buf = ctypes.create_string_buffer(int(lib().or_sizeof_acuity()))
        rc = lib().or_acuity_init(self._buf, _p(self.E), _p(self.f), len(self.E))
        if rc != 0:
            raise ValueError("bad pivots")
        self.delta = None
        if delta is not None:
            self.delta = _c(delta, np.float64)
            if self.delta.size != self.E.size or lib().or_acuity_set_delta(self._buf, _p(self.delta)) != 0:
                raise ValueError("bad delta")
        n = len(self.E) - 1
        self.m = np.zeros(n)
        self.w0 = np.zeros(n)
        self.c = np.zeros(n)
        lib().or_acuity_get(self._buf, _p(self.m), _p(self.w0), _p(self.c))

    @property
    def ptr(self):
        return ctypes.cast(self._buf, ctypes.c_void_p)

    def _eval(self, what: int, x) -> np.ndarray:
        x = np.atleast_1d(_c(x, np.float64))
        out = np.empty_like(x)
        lib().or_eval(self.ptr, what, _p(x), _p(out), x.size)
        return out

    def u_of_e(self, e):
        return self._eval(0, e)

    def e_of_u(self, u):
        return self._eval(1, u)

    def l_of_e(self, e):
        return self._eval(2, e)

    def f_of_e(self, e):
        return self._eval(3, e)

    def delta_of_e(self, e):
        return self._eval(4, e)


@dataclass
class Layout:
    e_col: np.ndarray    # (C,) float64 eccentricity of column centres (deg)
    n_col: np.ndarray    # (C,) int32 texels per column
    off_col: np.ndarray  # (C,) int64 first texel of each column
    total: int

    @property
    def n_cols(self) -> int:
        return int(self.e_col.size)


def lp_layout(acuity: Optional[Acuity] = None, e_max: float = PAPER_E_MAX) -> Layout:
    a = acuity or Acuity()
    cap = 1 << 16
    e = np.zeros(cap)
    n = np.zeros(cap, np.int32)
    off = np.zeros(cap, np.int64)
    tot = np.zeros(1, np.int64)
    C = lib().or_lp_layout(a.ptr, float(e_max), cap, _p(e), _p(n), _p(off), _p(tot))
    if C < 0:
        raise ValueError("layout too large")
    return Layout(e[:C].copy(), n[:C].copy(), off[:C].copy(), int(tot[0]))


class _View(ctypes.Structure):
    _fields_ = [("width", ctypes.c_double), ("height", ctypes.c_double),
                ("fov_v_deg", ctypes.c_double), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("pose", ctypes.c_double * 12)]


def _view(width, height, fov_v_deg, gaze, pose) -> _View:
    v = _View()
    v.width, v.height, v.fov_v_deg = float(width), float(height), float(fov_v_deg)
    v.x0, v.y0 = float(gaze[0]), float(gaze[1])
    P = np.asarray(pose, np.float64).reshape(12)
    for k in range(12):
        v.pose[k] = float(P[k])
    return v


def lp_rays(layout: Layout, width, height, fov_v_deg, gaze, pose, texels=None):
    """Origins, directions and screen points of LP texels (Eqs. 3, 10, 11)."""
    if texels is None:
        texels = np.arange(layout.total, dtype=np.int64)
    t = _c(texels, np.int64)
    n = t.size
    o = np.empty((n, 3))
    d = np.empty((n, 3))
    xy = np.empty((n, 2))
    v = _view(width, height, fov_v_deg, gaze, pose)
    lib().or_lp_rays(ctypes.byref(v), _p(layout.e_col), _p(layout.n_col), _p(layout.off_col),
                     layout.n_cols, _p(t), n, _p(o), _p(d), _p(xy))
    return o, d, xy


def pixel_rays(width, height, fov_v_deg, pose, pixels=None):
    if pixels is None:
        pixels = np.arange(int(width) * int(height), dtype=np.int64)
    p = _c(pixels, np.int64)
    o = np.empty((p.size, 3))
    d = np.empty((p.size, 3))
    v = _view(width, height, fov_v_deg, (0.0, 0.0), pose)
    lib().or_pixel_rays(ctypes.byref(v), _p(p), p.size, _p(o), _p(d))
    return o, d


def cast_brute(tris, orig, dirs):
    tr = _c(tris, np.float32)
    o = _c(orig, np.float64)
    d = _c(dirs, np.float64)
    n = o.shape[0]
    ids = np.empty(n, np.int32)
    t = np.empty(n)
    lib().or_cast_brute(_p(tr), tr.shape[0], _p(o), _p(d), n, _p(ids), _p(t))
    return ids, t


class CpuBVH:
    def __init__(self, tris):
        self.tris = _c(tris, np.float32)
        self.h = lib().or_bvh_build(_p(self.tris), self.tris.shape[0])

    def cast(self, orig, dirs):
        o = _c(orig, np.float64)
        d = _c(dirs, np.float64)
        n = o.shape[0]
        ids = np.empty(n, np.int32)
        t = np.empty(n)
        lib().or_cast_bvh(self.h, _p(o), _p(d), n, _p(ids), _p(t))
        return ids, t

    def __del__(self):
        try:
            if self.h:
                lib().or_bvh_free(self.h)
                self.h = None
        except Exception:
            pass


def ray_tri_t(tris, ids, orig, dirs):
    tr = _c(tris, np.float32)
    i = _c(ids, np.int32)
    o = _c(orig, np.float64)
    d = _c(dirs, np.float64)
    out = np.empty(i.size)
    lib().or_ray_tri_t(_p(tr), _p(i), _p(o), _p(d), i.size, _p(out))
    return out


def edge_margin(tri, o, d) -> float:
    tr = _c(tri, np.float32).reshape(9)
    return float(lib().or_edge_margin(_p(_c(o, np.float64)), _p(_c(d, np.float64)), _p(tr)))


def shade(tris, albedo, light_dir, dirs, hit_ids, point_lights=None, orig=None, hit_t=None):
    """Lambert + ambient + directional light, sky on a miss; `point_lights` =
    (positions (k, 3), rgb (k, 3)) adds unshadowed inverse-square point lights
    (needs the ray origins and hit distances)."""
    tr = _c(tris, np.float32)
    al = _c(albedo, np.float32)
    L = _c(light_dir, np.float64)
    d = _c(dirs, np.float64)
    h = _c(hit_ids, np.int32)
    out = np.empty((h.size, 4))
    lib().or_shade(_p(tr), _p(al), _p(L), _p(d), _p(h), h.size, _p(out))
    if point_lights is not None and len(point_lights[0]):
        pos = _c(point_lights[0], np.float64).reshape(-1, 3)
        rgb = _c(point_lights[1], np.float64).reshape(-1, 3)
        o = _c(orig, np.float64)
        t = _c(np.where(h >= 0, hit_t, 0.0), np.float64)
        lib().or_shade_points(_p(tr), _p(al), _p(o), _p(d), _p(h), _p(t), h.size, pos.shape[0],
                              _p(pos), _p(rgb), _p(out))
    return out


def grazing(tris, dirs, hit_ids):
    tr = _c(tris, np.float32)
    d = _c(dirs, np.float64)
    h = _c(hit_ids, np.int32)
    out = np.empty(h.size)
    lib().or_grazing(_p(tr), _p(d), _p(h), h.size, _p(out))
    return out


def reconstruct_points(lp, layout: Layout, width, height, fov_v_deg, gaze, pts,
                       acuity: Optional[Acuity] = None, e_max: float = PAPER_E_MAX):
    """Bilinear inverse-mapping filter at arbitrary display points (x, y)."""
    a = acuity or Acuity()
    lpa = _c(lp, np.float64)
    nch = lpa.shape[1] if lpa.ndim == 2 else 1
    P = _c(pts, np.float64).reshape(-1, 2)
    out = np.empty((P.shape[0], nch))
    v = _view(width, height, fov_v_deg, gaze, np.eye(3, 4))
    lib().or_reconstruct_points(a.ptr, float(e_max), ctypes.byref(v), _p(layout.n_col),
                                _p(layout.off_col), layout.n_cols, _p(lpa), nch, _p(P),
                                P.shape[0], _p(out))
    return out


def pixel_centres(width, height, pixels=None):
    if pixels is None:
        pixels = np.arange(int(width) * int(height), dtype=np.int64)
    p = np.asarray(pixels, np.int64)
    return np.stack([(p % width) + 0.5, (p // width) + 0.5], 1).astype(np.float64)


def reconstruct(lp, layout, width, height, fov_v_deg, gaze, pixels=None, **kw):
    return reconstruct_points(lp, layout, width, height, fov_v_deg, gaze,
                              pixel_centres(width, height, pixels), **kw)


def fxaa_lp(lp, layout: Layout) -> np.ndarray:
    """FXAA inside the LP buffer (Sec. 3.4, Sec. 7) on texels in layout order;
    `layout` may be any (n_col, off_col) grid."""
    lpa = _c(lp, np.float64)
    nch = lpa.shape[1] if lpa.ndim == 2 else 1
    out = np.empty_like(lpa)
    n = _c(layout.n_col, np.int32)
    off = _c(layout.off_col, np.int64)
    lib().or_fxaa_lp(_p(n), _p(off), int(n.size), _p(lpa), nch, _p(out))
    return out


def lp_neighbor(layout: Layout, c: int, j: int, c2: int, dj: int) -> int:
    """Index of the texel of column c2 at the angle of (c, j), moved dj rows."""
    out = np.zeros(1, np.int64)
    n = _c(layout.n_col, np.int32)
    off = _c(layout.off_col, np.int64)
    lib().or_lp_neighbor(_p(n), _p(off), int(n.size), int(c), int(j), int(c2), int(dj), _p(out))
    return int(out[0])


def uniform_layout(n_cols: int, n_rows: int) -> Layout:
    """A rectangular LP grid (every column n_rows texels) for closed-form tests."""
    return Layout(np.zeros(n_cols), np.full(n_cols, n_rows, np.int32),
                  np.arange(n_cols, dtype=np.int64) * n_rows, n_cols * n_rows)


def morton(tris):
    tr = _c(tris, np.float32)
    out = np.empty(tr.shape[0], np.uint32)
    lib().or_morton(_p(tr), tr.shape[0], _p(out))
    return out


@dataclass
class LBVH:
    codes: np.ndarray       # (n,) uint32, input order
    sorted_ids: np.ndarray  # (n,) int32
    child: np.ndarray       # (n-1, 2) int32; < 0 = leaf ~k
    node_box: np.ndarray    # (n-1, 6) float32 lo xyz, hi xyz
    leaf_box: np.ndarray    # (n, 6) float32 (sorted order)
    range: np.ndarray       # (n-1, 2) int32 first/last sorted position


def lbvh(tris) -> LBVH:
    tr = _c(tris, np.float32)
    n = tr.shape[0]
    codes = np.zeros(n, np.uint32)
    ids = np.zeros(n, np.int32)
    ni = max(n - 1, 0)
    child = np.zeros((max(ni, 1), 2), np.int32)
    nb = np.zeros((max(ni, 1), 6), np.float32)
    lb = np.zeros((max(n, 1), 6), np.float32)
    rg = np.zeros((max(ni, 1), 2), np.int32)
    rc = lib().or_lbvh(_p(tr), n, _p(codes), _p(ids), _p(child), _p(nb), _p(lb), _p(rg))
    if rc != 0:
        raise RuntimeError("or_lbvh failed")
    return LBVH(codes, ids, child[:ni], nb[:ni], lb[:n], rg[:ni])


# ---------------------------------------------------------------------------
# whole-path conveniences


def render_lp(scene_tris, albedo, light_dir, layout, width, height, fov_v_deg, gaze, pose,
              texels=None, bvh: Optional[CpuBVH] = None, point_lights=None):
    """LP colours (n, 4) FP64, hit ids and ray directions for the given texels."""
    o, d, _ = lp_rays(layout, width, height, fov_v_deg, gaze, pose, texels)
    if bvh is not None:
        ids, t = bvh.cast(o, d)
    else:
        ids, t = cast_brute(scene_tris, o, d)
    rgba = shade(scene_tris, albedo, light_dir, d, ids, point_lights, o, t)
    return rgba, ids, t, o, d


def pt_uniform(seed: int, texel: int, k: int, dim: int) -> float:
    """The path tracer's counter-based uniform for (seed, texel, bounce k, dim)."""
    return float(lib().or_pt_uniform(int(seed), int(texel), int(k), int(dim)))


def path_trace_lp(scene_tris, albedo, light_dir, layout, width, height, fov_v_deg, gaze, pose,
                  seed: int, max_diffuse: int = 3, texels=None, bvh: Optional[CpuBVH] = None,
                  segments: bool = False):
    """Path-traced LP texels (Sec. 8).  Returns (rgba (n, 4), signature (n, D + 2)
    [, segment rays (n, D + 1, 6)]): signature = hit id per segment (-1 miss,
    -2 not traced) then a mask: bit k = segment k's shadow ray saw the light,
    bit 16 + k = a shadow ray was cast."""
    if texels is None:
        texels = np.arange(layout.total, dtype=np.int64)
    tex = _c(texels, np.int64)
    o, d, _ = lp_rays(layout, width, height, fov_v_deg, gaze, pose, tex)
    b = bvh or CpuBVH(scene_tris)
    n = tex.size
    rgba = np.empty((n, 4))
    sig = np.empty((n, max_diffuse + 2), np.int32)
    seg = np.empty((n, max_diffuse + 1, 6)) if segments else None
    lib().or_path_trace(b.h, _p(_c(albedo, np.float32)), _p(_c(light_dir, np.float64)), _p(o), _p(d),
                        _p(tex), n, int(seed) & (2**64 - 1), int(max_diffuse), _p(rgba), _p(sig),
                        _p(seg) if seg is not None else None)
    return (rgba, sig, seg) if segments else (rgba, sig)


def reproject_lp(layout: Layout, width, height, fov_v_deg, gaze_left, pose_left, gaze_right,
                 pose_right, left_t, left_rgba, acuity: Optional[Acuity] = None,
                 e_max: float = PAPER_E_MAX):
    """VaFR_Rep's forward grid warp of a left LP buffer (hit distances `left_t`,
    inf on a miss, and colours) to the right eye.  Returns (right rgba (n, 4),
    winning left triangle per right texel, -1 for a hole)."""
    a = acuity or Acuity()
    vl = _view(width, height, fov_v_deg, gaze_left, pose_left)
    vr = _view(width, height, fov_v_deg, gaze_right, pose_right)
    lt = _c(left_t, np.float64)
    lc = _c(left_rgba, np.float64)
    out = np.empty((layout.total, 4))
    tri = np.empty(layout.total, np.int32)
    lib().or_reproject_lp(a.ptr, float(e_max), _p(_c(layout.e_col, np.float64)), _p(layout.n_col),
                          _p(layout.off_col), layout.n_cols, layout.total, ctypes.byref(vl),
                          ctypes.byref(vr), _p(lt), _p(lc), _p(out), _p(tri))
    return out, tri


REP_PROBE_FIELDS = ("exists", "in_front", "front_margin", "n_inf", "depth_ratio", "u_span",
                    "f_span_raw", "f_span", "cover_margin", "depth")


def rep_probe(layout: Layout, width, height, fov_v_deg, gaze_left, pose_left, gaze_right, pose_right,
              left_t, tids, texels, acuity: Optional[Acuity] = None, e_max: float = PAPER_E_MAX):
    """For warped triangle tids[q] at right texel texels[q]: the quantities the
    warp's raster decides on (REP_PROBE_FIELDS), as a dict of arrays."""
    a = acuity or Acuity()
    vl = _view(width, height, fov_v_deg, gaze_left, pose_left)
    vr = _view(width, height, fov_v_deg, gaze_right, pose_right)
    t = _c(tids, np.int32)
    k = _c(texels, np.int64)
    out = np.empty((t.size, 10))
    lib().or_rep_probe(a.ptr, float(e_max), _p(_c(layout.e_col, np.float64)), _p(layout.n_col),
                       _p(layout.off_col), layout.n_cols, layout.total, ctypes.byref(vl), ctypes.byref(vr),
                       _p(_c(left_t, np.float64)), t.size, _p(t), _p(k), _p(out))
    return {name: out[:, i] for i, name in enumerate(REP_PROBE_FIELDS)}


def render_lp_rep(scene_tris, albedo, light_dir, layout, width, height, fov_v_deg, gazes, poses,
                  bvh: Optional[CpuBVH] = None):
    """VaFR_Rep (Sec. 5.1): the left eye cast, the right eye warped from it with
    its holes cast.  Returns (left rgba, right rgba, right triangle / -1)."""
    b = bvh or CpuBVH(scene_tris)
    rgba_l, ids_l, t_l, _, _ = render_lp(scene_tris, albedo, light_dir, layout, width, height,
                                         fov_v_deg, gazes[0], poses[0], bvh=b)
    t_l = np.where(ids_l >= 0, t_l, np.inf)
    right, tri = reproject_lp(layout, width, height, fov_v_deg, gazes[0], poses[0], gazes[1],
                              poses[1], t_l, rgba_l)
    holes = np.flatnonzero(tri < 0)
    if holes.size:
        rgba_h, _, _, _, _ = render_lp(scene_tris, albedo, light_dir, layout, width, height,
                                       fov_v_deg, gazes[1], poses[1], texels=holes, bvh=b)
        right[holes] = rgba_h
    return rgba_l, right, tri


def render_gt(scene_tris, albedo, light_dir, width, height, fov_v_deg, pose, pixels=None,
              bvh: Optional[CpuBVH] = None, point_lights=None):
    o, d = pixel_rays(width, height, fov_v_deg, pose, pixels)
    if bvh is not None:
        ids, t = bvh.cast(o, d)
    else:
        ids, t = cast_brute(scene_tris, o, d)
    return shade(scene_tris, albedo, light_dir, d, ids, point_lights, o, t), ids, t, o, d
