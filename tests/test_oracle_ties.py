"""Pins of the oracle's tie classifier: the edge margin, the grazing measure and
the single-triangle hit distance that the GPU parity tests use to tell a
ray-edge tie from a genuine hit error (closest hit with the lower-id tie rule,
Sec. 6.1 ray casting; the tie window of the hit-id comparison).

Each check compares with a closed form that does not reuse the oracle's
formula: for a triangle lying in a plane perpendicular to the ray's dominant
axis, the margin is the signed in-plane distance from the ray's crossing point
to the nearest edge line; the grazing measure of a plane with a known normal
is |cos| of a known angle; the hit distance is the plane's distance over the
direction's component.  The last tests compile copies of the oracle with one
plausible mistake each (a shear sign, a dropped orientation, an unnormalised
edge, a reversed edge, a wrong normal edge, a missing |d|, a wrong division)
and check that these same closed-form checks reject every copy.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle

ORACLE_C = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                        "vafr_oracle.c")

# right triangle in the plane z = 5: legs on the x and y axes, hypotenuse 3x + 4y = 12
TRI = np.array([[0.0, 0.0, 5.0], [4.0, 0.0, 5.0], [0.0, 3.0, 5.0]], np.float32)


def _dev(got, want):
    """|got - want|, infinite when got is NaN (NaN would vanish inside max())."""
    return abs(got - want) if got == got else math.inf


def _inplane_margin(x, y):
    """Signed distance of (x, y) from the nearest edge line of TRI (> 0 inside)."""
    return min(x, y, (12.0 - 3.0 * x - 4.0 * y) / 5.0)


# points inside (each edge the nearest once), on an edge, and outside each edge
POINTS = [(0.3, 1.0), (1.5, 0.2), (1.7, 1.5), (1.0, 1.0), (0.0, 1.0), (2.0, 0.0),
          (-0.4, 1.0), (1.0, -0.7), (3.0, 2.0), (5.0, -1.0), (1e-6, 1.2), (-1e-6, 1.2)]

# cyclic coordinate permutations: the plane z = 5 becomes x = 5 or y = 5, so the
# ray's dominant axis (and the shear frame built on it) changes with it
PERMS = [(0, 1, 2), (2, 0, 1), (1, 2, 0)]


def _permute(a, p):
    a = np.asarray(a)
    out = np.empty_like(a)
    out[..., list(p)] = a[..., [0, 1, 2]]
    return out


def _margin_cases():
    """(triangle, origin, direction, expected margin) over points, dominant
    axes, ray senses, windings, slants and direction lengths."""
    cases = []
    for (x, y) in POINTS:
        want = _inplane_margin(x, y)
        for p in PERMS:
            for sense in (1.0, -1.0):
                for slant in ((0.0, 0.0), (0.3, -0.2), (-0.45, 0.35)):
                    for scale in (1.0, 7.0):
                        d = np.array([slant[0] * sense, slant[1] * sense, sense]) * scale
                        # origin such that the ray crosses z = 5 at (x, y)
                        o = np.array([x, y, 5.0]) - 2.0 * d
                        for tri in (TRI, TRI[::-1]):
                            cases.append((_permute(tri, p).astype(np.float32), _permute(o, p),
                                          _permute(d, p), want))
    return cases


def check_edge_margin(fn):
    """Largest deviation of fn(tri, o, d) from the closed form over all cases."""
    worst = 0.0
    for tri, o, d, want in _margin_cases():
        got = fn(tri, o, d)
        worst = max(worst, _dev(got, want))
    return worst


def test_edge_margin_closed_form():
    assert check_edge_margin(oracle.edge_margin) < 1e-12


def test_edge_margin_sign_decides_inside():
    # strictly inside -> positive, strictly outside -> negative, on an edge -> 0
    for tri, o, d, want in _margin_cases():
        m = oracle.edge_margin(tri, o, d)
        if want > 1e-9:
            assert m > 0
        elif want < -1e-9:
            assert m < 0
        else:
            assert abs(m) < 1e-12


# grazing: a triangle in the plane x = y (normal (1, -1, 0)/sqrt 2) and one in z = 0
GRAZE_TRIS = np.array([[[0, 0, 0], [1, 1, 0], [0, 0, 1]],
                       [[0, 0, 0], [2, 0, 0], [0, 3, 0]]], np.float32)


def _grazing_cases():
    cases = []
    for theta in (0.0, 10.0, 30.0, 60.0, 85.0, 89.99, 90.0):
        for psi in (0.0, 40.0, 200.0):
            for length in (1.0, 0.01, 50.0):
                th, ps = math.radians(theta), math.radians(psi)
                # angle theta from the z axis (the normal of GRAZE_TRIS[1])
                d = length * np.array([math.sin(th) * math.cos(ps), math.sin(th) * math.sin(ps),
                                       math.cos(th)])
                cases.append((1, d, abs(math.cos(th))))
    for d, want in (((1, 0, 0), 1 / math.sqrt(2)), ((1, 1, 0), 0.0), ((0, 0, 1), 0.0),
                    ((1, -1, 0), 1.0), ((3, -3, 0), 1.0), ((0, 1, 0), 1 / math.sqrt(2)),
                    ((1, 0, 1), 0.5)):
        cases.append((0, np.array(d, float), want))
    return cases


def check_grazing(fn):
    worst = 0.0
    for which, d, want in _grazing_cases():
        for tri in (GRAZE_TRIS[which], GRAZE_TRIS[which][::-1]):
            got = fn(tri[None], d[None], np.array([0], np.int32))[0]
            worst = max(worst, _dev(got, want))
    # a miss is never grazing
    worst = max(worst, _dev(fn(GRAZE_TRIS[:1], np.array([[0.0, 0.0, 1.0]]), np.array([-1], np.int32))[0], 1.0))
    return worst


def test_grazing_closed_form():
    assert check_grazing(oracle.grazing) < 1e-12


def _tri_t_cases():
    """(triangles, id, origin, direction, expected t) with t from the plane."""
    plane = np.array([[3, 0, 0], [0, 3, 0], [0, 0, 3]], np.float32)   # x + y + z = 3
    cases = []
    for p in PERMS:
        for d, o in (((0.3, -0.2, 1.0), (0.0, 1.2, 0.0)), ((0.6, -0.4, 2.0), (0.0, 1.2, 0.0)),
                     ((0.0, 0.0, -1.0), (1.0, 1.0, 9.0))):
            d, o = np.array(d), np.array(o)
            t = (5.0 - o[2]) / d[2]
            cases.append((_permute(TRI, p).astype(np.float32)[None], 0, _permute(o, p), _permute(d, p), t))
    for d in ((1, 1, 1), (1, 2, 3), (3, 0.5, 0.25)):
        d = np.array(d, float)
        cases.append((plane[None], 0, np.zeros(3), d, 3.0 / d.sum()))
    cases.append((plane[None], 0, np.zeros(3), np.array([-1.0, -1.0, -1.0]), math.inf))   # behind
    cases.append((TRI[None], 0, np.array([5.0, 5.0, 0.0]), np.array([0.0, 0.0, 1.0]), math.inf))  # beside
    cases.append((TRI[None], -1, np.array([1.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), math.inf))  # no id
    return cases


def check_ray_tri_t(fn):
    worst = 0.0
    for tris, i, o, d, want in _tri_t_cases():
        got = fn(tris, np.array([i], np.int32), o[None], d[None])[0]
        if math.isinf(want) or math.isinf(got):
            worst = max(worst, 0.0 if got == want else math.inf)
        else:
            worst = max(worst, _dev(got, want) / want)
    return worst


def test_ray_tri_t_closed_form():
    assert check_ray_tri_t(oracle.ray_tri_t) < 1e-14


# ---- planted mistakes: each mutant copy of the oracle must fail a check above ----

MUTANTS = [
    ("edge_margin", "shear sign",
     "P[v][0] = a[r.kx] - r.Sx * a[r.kz];", "P[v][0] = a[r.kx] + r.Sx * a[r.kz];"),
    ("edge_margin", "shear of the second row",
     "P[v][1] = a[r.ky] - r.Sy * a[r.kz];", "P[v][1] = a[r.ky] - r.Sx * a[r.kz];"),
    ("edge_margin", "orientation dropped",
     "double sgn = area >= 0.0 ? 1.0 : -1.0;", "double sgn = 1.0;"),
    ("edge_margin", "edge not normalised",
     "double dist = len > 0.0 ? fn / len : -INFINITY;", "double dist = len > 0.0 ? fn : -INFINITY;"),
    ("edge_margin", "edge reversed",
     "const double* q = P[(e + 1) % 3];", "const double* q = P[(e + 2) % 3];"),
    ("edge_margin", "largest instead of smallest",
     "if (dist < best) best = dist;", "if (dist > best || best == INFINITY) best = dist;"),
    ("grazing", "wrong second edge",
     "e2[a] = (double)t[6 + a] - t[a];", "e2[a] = (double)t[3 + a] - t[a];"),
    ("grazing", "direction not normalised",
     "/ (nl * dl);", "/ (nl);"),
    ("grazing", "signed instead of absolute",
     "out[k] = fabs(nrm[0] * d[0]", "out[k] = (nrm[0] * d[0]"),
    ("ray_tri_t", "depth scale dropped",
     "double Az = r->Sz * A[r->kz], Bz = r->Sz * B[r->kz], Cz = r->Sz * C[r->kz];",
     "double Az = A[r->kz], Bz = B[r->kz], Cz = C[r->kz];"),
    ("ray_tri_t", "shear sign in the hit test",
     "double Ax = A[r->kx] - r->Sx * A[r->kz], Ay = A[r->ky] - r->Sy * A[r->kz];",
     "double Ax = A[r->kx] + r->Sx * A[r->kz], Ay = A[r->ky] - r->Sy * A[r->kz];"),
]


def _mutant_lib(tmp_path, src, tag):
    c = tmp_path / f"m_{tag}.c"
    so = tmp_path / f"m_{tag}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
                    str(c), "-o", str(so), "-lm"], check=True, capture_output=True)
    L = ctypes.CDLL(str(so))
    P, i64 = ctypes.c_void_p, ctypes.c_int64
    L.or_edge_margin.argtypes = [P, P, P]
    L.or_edge_margin.restype = ctypes.c_double
    L.or_grazing.argtypes = [P, P, P, i64, P]
    L.or_ray_tri_t.argtypes = [P, P, P, P, i64, P]
    return L


def _bind(L):
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731

    def margin(tri, o, d):
        t = np.ascontiguousarray(tri, np.float32).reshape(9)
        return float(L.or_edge_margin(p(np.ascontiguousarray(o, np.float64)),
                                      p(np.ascontiguousarray(d, np.float64)), p(t)))

    def grazing(tris, d, h):
        tr, dd, hh = (np.ascontiguousarray(tris, np.float32), np.ascontiguousarray(d, np.float64),
                      np.ascontiguousarray(h, np.int32))
        out = np.empty(hh.size)
        L.or_grazing(p(tr), p(dd), p(hh), hh.size, p(out))
        return out

    def tri_t(tris, ids, o, d):
        tr, ii = np.ascontiguousarray(tris, np.float32), np.ascontiguousarray(ids, np.int32)
        oo, dd = np.ascontiguousarray(o, np.float64), np.ascontiguousarray(d, np.float64)
        out = np.empty(ii.size)
        L.or_ray_tri_t(p(tr), p(ii), p(oo), p(dd), ii.size, p(out))
        return out
    return margin, grazing, tri_t


def test_unmutated_copy_passes(tmp_path):
    """The harness itself: an unchanged copy passes all three checks."""
    margin, grazing, tri_t = _bind(_mutant_lib(tmp_path, open(ORACLE_C).read(), "orig"))
    assert check_edge_margin(margin) < 1e-12
    assert check_grazing(grazing) < 1e-12
    assert check_ray_tri_t(tri_t) < 1e-14


# the C function each mutation edits (the hit distance comes from the shared hit test)
FUNC_SIG = {"edge_margin": "double or_edge_margin(", "grazing": "void or_grazing(",
            "ray_tri_t": "static int wray_hit("}


def _mutate(src, func, old, new):
    """src with `old` replaced by `new` inside the body of one C function."""
    beg = src.index(FUNC_SIG[func])
    end = src.index("\n}\n", beg)
    body = src[beg:end]
    assert body.count(old) == 1, f"mutation anchor not unique in {func}: {old}"
    return src[:beg] + body.replace(old, new) + src[end:]


@pytest.mark.parametrize("func,what,old,new", MUTANTS, ids=[f"{m[0]}: {m[1]}" for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, func, what, old, new):
    src = _mutate(open(ORACLE_C).read(), func, old, new)
    margin, grazing, tri_t = _bind(_mutant_lib(tmp_path, src, func))
    checks = {"edge_margin": lambda: check_edge_margin(margin) > 1e-6,
              "grazing": lambda: check_grazing(grazing) > 1e-6,
              "ray_tri_t": lambda: check_ray_tri_t(tri_t) > 1e-6}
    assert checks[func](), f"planted mistake '{what}' in {func} not detected"
