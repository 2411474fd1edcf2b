"""Pins of the oracle's FXAA inside the LP buffer (Sec. 3.4 internal
anti-aliasing, Sec. 7): invariants the method fixes and closed forms derived
by hand on a rectangular grid."""

import numpy as np
import pytest

import oracle


def _grey(v):
    v = np.asarray(v, np.float64)
    return np.stack([v, v, v, np.ones_like(v)], -1)


def test_neighbour_holds_the_angle(layout):
    # across the radius, the chosen texel's angular interval contains the angle
    rng = np.random.default_rng(0)
    for _ in range(300):
        c = int(rng.integers(0, layout.n_cols))
        j = int(rng.integers(0, layout.n_col[c]))
        phi = (j + 0.5) / layout.n_col[c]
        for c2 in (c - 1, c + 1):
            t = oracle.lp_neighbor(layout, c, j, c2, 0)
            cc = min(max(c2, 0), layout.n_cols - 1)
            j2 = t - layout.off_col[cc]
            assert 0 <= j2 < layout.n_col[cc]
            if cc != c:
                assert j2 / layout.n_col[cc] <= phi < (j2 + 1) / layout.n_col[cc]
    # along the angle, rows wrap modulo n_c
    c = 100
    n = layout.n_col[c]
    assert oracle.lp_neighbor(layout, c, n - 1, c, 1) == layout.off_col[c]
    assert oracle.lp_neighbor(layout, c, 0, c, -1) == layout.off_col[c] + n - 1


def test_constant_and_low_contrast_are_unchanged(layout):
    lp = np.tile([0.3, 0.6, 0.2, 1.0], (layout.total, 1))
    assert np.array_equal(oracle.fxaa_lp(lp, layout), lp)
    rng = np.random.default_rng(1)
    noise = 0.5 + rng.uniform(-0.03, 0.03, (layout.total, 4))   # luma range < 1/12
    assert np.array_equal(oracle.fxaa_lp(noise, layout), noise)


def test_output_is_a_blend_with_one_neighbour(layout):
    # each texel moves towards one of its four neighbours, by a weight in
    # [0, 3/4] (edge offsets stay <= 1/2, the subpixel term <= 3/4)
    rng = np.random.default_rng(2)
    lp = rng.uniform(0, 1, (layout.total, 4))
    lp[rng.random(layout.total) < 0.5] *= 0.1           # strong edges everywhere
    out = oracle.fxaa_lp(lp, layout)
    col = np.repeat(np.arange(layout.n_cols), layout.n_col)
    j = np.arange(layout.total) - layout.off_col[col]
    idx = np.flatnonzero(np.any(out != lp, 1))
    assert idx.size > layout.total // 20
    for t in rng.choice(idx, 400, replace=False):
        c, jj = int(col[t]), int(j[t])
        ok = False
        for c2, dj in ((c, 1), (c, -1), (c + 1, 0), (c - 1, 0)):
            q = lp[oracle.lp_neighbor(layout, c, jj, c2, dj)]
            d = q - lp[t]
            w = np.divide(out[t] - lp[t], d, out=np.full(4, np.nan), where=np.abs(d) > 1e-12)
            w = w[np.isfinite(w)]
            if w.size and np.allclose(w, w[0], atol=1e-9) and -1e-12 <= w[0] <= 0.75 + 1e-12 \
                    and np.allclose(lp[t] + w[0] * d, out[t], atol=1e-12):
                ok = True
        assert ok, t


def test_straight_edge_gets_only_subpixel_blend():
    # Columns < 8 dark, >= 8 bright, every row alike: the search never finds an
    # end, so only step 6 acts.  At the dark texel next to the edge the 3 x 3
    # mean is 1/3 (a = 1/3): weight ((3 - 2/3)/9)^2 * 3/4 = 0.75 (7/27)^2; the
    # bright side mirrors it.
    lay = oracle.uniform_layout(16, 64)
    v = np.repeat((np.arange(16) >= 8).astype(float), 64)
    lp = _grey(v)
    out = oracle.fxaa_lp(lp, lay)
    w = 0.75 * (7 / 27) ** 2
    luma1 = np.float32(np.float32(np.float32(0.299) + np.float32(0.587)) + np.float32(0.114))
    assert abs(float(luma1) - 1.0) < 1e-6
    for j in (0, 17, 63):
        np.testing.assert_allclose(out[7 * 64 + j, :3], w, atol=1e-6)
        np.testing.assert_allclose(out[8 * 64 + j, :3], 1 - w, atol=1e-6)
        assert np.array_equal(out[3 * 64 + j], lp[3 * 64 + j])     # far from the edge


def test_staircase_edge_offsets():
    # Bright where c >= 8 for rows j < 32 and c >= 9 for j >= 32: a one-column
    # step at j = 32.  Bright texel (8, 32 - d), d = 1..9: the walk towards
    # larger j ends after d steps (the row where column 8 turns dark), the
    # other way never (12); the texel is brighter than the mid-line and the
    # end darker, so step 5 gives 1/2 - d/(d + 12), which beats the subpixel
    # term; the neighbour is column 7 (dark): output 1/2 + d/(d + 12).
    lay = oracle.uniform_layout(16, 64)
    c = np.repeat(np.arange(16), 64)
    j = np.tile(np.arange(64), 16)
    v = np.where(j < 32, c >= 8, c >= 9).astype(float)
    out = oracle.fxaa_lp(_grey(v), lay)
    for d in range(1, 10):
        np.testing.assert_allclose(out[8 * 64 + 32 - d, :3], 0.5 + d / (d + 12), atol=2e-6)
