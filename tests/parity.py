"""Shared helpers of the GPU parity tests: device set-up through the C ABI and the
classification of hit-id mismatches as ray-edge / depth ties.

A mismatch between the GPU's hit triangle (FP32 ray, FP32 watertight test) and
the oracle's (FP64 ray, FP64 test) is a tie when the FP64 ray passes within
``rel`` x (distance along the ray) of an edge of the oracle's triangle, or when
the GPU's triangle is within that distance of being hit by the FP64 ray and
its plane lies no farther than the oracle's hit (relative ``rel``); ``rel``
defaults to TIE_REL, a bound on the FP32 rounding of the GPU's ray and test.  Anything
else is a genuine error.  A colour comparison skips rays that graze their
triangle (|n.d| < 1e-5), where the face-forward flip is ambiguous.

Every classified tie's width (|margin| / (t |d|), and the relative depth
excess of the GPU's triangle) is recorded in TIE_WIDTHS, and the session
summary prints the largest, so the window can be checked against the FP32
rounding bound it stands for.
"""

from __future__ import annotations

import numpy as np

import oracle

# (kind, width) of every classified tie of the session: kind "edge" = |margin| /
# (t |d|) of the oracle's triangle, "gpu-edge" = the GPU triangle's outside
# margin over (t |d|), "depth" = relative depth excess of the GPU's triangle
TIE_WIDTHS: list = []


def device_scene(V, scene, torch):
    tris = torch.from_numpy(np.ascontiguousarray(scene.tris.reshape(-1, 9))).cuda()
    alb = torch.from_numpy(np.ascontiguousarray(scene.albedo)).cuda()
    h = V.vafr_build_scene(tris if scene.n_tris else None, alb if scene.n_tris else None,
                           scene.light_dir)
    return h, (tris, alb)


def lp_slots(V, sess):
    """The library's LP layout: slot of every texel (c, j) in the oracle's
    column order, slots per eye, counts and column offsets.  Column c is framed
    by guard slots offs[c] - 1 (a copy of texel n_c - 1) and offs[c] + n_c (a
    copy of texel 0)."""
    counts, offs, _, n_tex = V.vafr_lp_layout(sess)
    counts = counts.astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    slot = np.repeat(offs - starts, counts) + np.arange(n_tex)
    return slot, int(offs[-1] + counts[-1] + 1), counts, offs


def check_guards(buf, counts, offs):
    """Guard slots equal the texels across the angular wrap."""
    assert np.array_equal(buf[offs - 1], buf[offs + counts - 1])
    assert np.array_equal(buf[offs + counts], buf[offs])


def to_device_lp(lp, V, sess):
    """Oracle-ordered LP texels -> the library's slot layout, guards filled."""
    slot, n_slots, counts, offs = lp_slots(V, sess)
    out = np.zeros((n_slots,) + lp.shape[1:], lp.dtype)
    out[slot] = lp
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    out[offs - 1] = lp[starts + counts - 1]
    out[offs + counts] = lp[starts]
    return out


def _plane_t(tri, o, d):
    v0, v1, v2 = tri.astype(np.float64)
    n = np.cross(v1 - v0, v2 - v0)
    den = float(n @ d)
    if den == 0.0:
        return np.inf
    return float(n @ (v0 - o)) / den


# Width of the tie window, relative to the distance along the ray t |d|.  The
# GPU ray differs from the oracle's FP64 ray by the FP32 roundings of its
# generation (tan e_c and the angle (2j+1)/n_c rounded to FP32, sincospi, two
# FMAs into the camera direction, the FP32 camera rotation: at most ~25 units
# of 2^-24 of |d| when every rounding adds up), and the FP32 watertight test
# moves an edge by up to ~12 units of 2^-24 of the vertex distance (the
# subtraction from the origin, the shear, the edge-function products).  The
# window takes 64 units of 2^-24 (3.8e-6), above that sum; the widest tie
# measured over the whole GPU suite is 8.5 units (5.0e-7).
TIE_REL = 64.0 * 2.0 ** -24


def classify(tris, o, d, gpu_ids, ora_ids, ora_t, rel=TIE_REL):
    """Returns (n_ties, n_errors, error_indices) over the mismatching rays."""
    mism = np.flatnonzero(gpu_ids != ora_ids)
    ties, errs = 0, []
    for k in mism:
        dist_scale = np.linalg.norm(d[k])
        tie = False
        if ora_ids[k] >= 0:
            m = oracle.edge_margin(tris[ora_ids[k]], o[k], d[k])
            delta = rel * ora_t[k] * dist_scale
            if abs(m) < delta:
                tie = True
                TIE_WIDTHS.append(("edge", abs(m) / (ora_t[k] * dist_scale)))
        if not tie and gpu_ids[k] >= 0:
            tg = _plane_t(tris[gpu_ids[k]], o[k], d[k])
            delta = rel * max(tg, 1e-30) * dist_scale
            m = oracle.edge_margin(tris[gpu_ids[k]], o[k], d[k])
            if m > -delta and tg > 0 and (ora_ids[k] < 0 or tg <= ora_t[k] * (1 + rel)):
                tie = True
                TIE_WIDTHS.append(("gpu-edge", max(-m, 0.0) / (max(tg, 1e-30) * dist_scale)))
                if ora_ids[k] >= 0:
                    TIE_WIDTHS.append(("depth", max(tg / ora_t[k] - 1.0, 0.0)))
        if tie:
            ties += 1
        else:
            errs.append(k)
    return ties, len(errs), np.array(errs, dtype=np.int64)


def compare_hits_and_colours(tris, o, d, gpu_ids, gpu_rgba, ora_ids, ora_t, ora_rgba,
                             colour_tol, tie_budget=1e-4):
    ties, n_err, err_idx = classify(tris, o, d, gpu_ids, ora_ids, ora_t)
    n = len(gpu_ids)
    same = gpu_ids == ora_ids
    graze = oracle.grazing(tris, d, ora_ids) < 1e-5
    ok = same & ~graze
    cerr = np.abs(gpu_rgba[ok].astype(np.float64) - ora_rgba[ok]).max(initial=0.0)
    summary = dict(n=n, mismatches=int((~same).sum()), ties=ties, errors=n_err,
                   tie_frac=(ties + int((same & graze).sum())) / max(n, 1), colour_err=float(cerr))
    assert n_err == 0, f"{n_err} non-tie hit mismatches, e.g. rays {err_idx[:8]}: {summary}"
    assert summary["tie_frac"] <= tie_budget, f"too many ties: {summary}"
    assert cerr <= colour_tol, f"colour error {cerr} > {colour_tol}: {summary}"
    return summary
