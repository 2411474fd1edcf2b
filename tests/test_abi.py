"""The C-ABI library builds, loads and exports every symbol include/vafr.h declares;
host-only entry points behave; compute entry points fail loudly without a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names += re.findall(r"^VAFR_API\s+[\w\s\*]*?\b(vafr_\w+)\s*\(", txt, re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2503_23410_gb300 import build
    build.build()
    from paper_2503_23410_gb300 import vafr
    return vafr.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    from paper_2503_23410_gb300 import vafr as V
    a = V.vafr_acuity_default()
    assert a.n_pivots == 5
    assert list(a.pivot_ecc_deg[:5]) == [0, 10, 20, 30, 60]
    assert list(a.pivot_cpd[:5]) == [40, 10, 6, 5, 4]
    assert a.e_max_deg == 60
    assert V.vafr_tuning_space() == (8, 9)
    assert V.vafr_error_string(0) == "ok"
    assert "invalid" in V.vafr_error_string(V.ERR_INVALID_ARG)
    assert V.vafr_version() >= 10000


def test_null_arguments_rejected(lib):
    from paper_2503_23410_gb300 import vafr as V
    out = ctypes.c_void_p()
    assert lib.vafr_session_create(None, ctypes.byref(out)) == V.ERR_INVALID_ARG
    assert lib.vafr_render_lp(None, None, 1, None, None, None) == V.ERR_INVALID_ARG
    assert lib.vafr_reconstruct(None, 0, None, None, None) == V.ERR_INVALID_ARG
    assert lib.vafr_set_gaze(None, 0, 1.0, 1.0) == V.ERR_INVALID_ARG
    assert lib.vafr_batch_replay(None, None) == V.ERR_INVALID_ARG


def test_compute_fails_loudly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_23410_gb300 import vafr as V
    desc = V.make_session_desc(64, 64, 90.0, [[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]])
    with pytest.raises(V.VafrError):
        V.vafr_session_create(desc)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2503_23410_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "vafr_oracle" not in txt and "liboracle" not in txt, fn


def test_noalloc_wrapper_checks_sizes_before_the_call():
    """The C entry point cannot see buffer sizes, so the binding refuses a flat
    tri_xyz whose length is not 9 n, outputs shorter than n and outputs that are
    not 32-bit integers -- before anything reaches the library."""
    import numpy as np
    from paper_2503_23410_gb300 import vafr as V
    tris = np.zeros((10, 9), np.float32)
    ok = np.zeros(10, np.int32)
    assert V._noalloc_n(tris, ok, ok) == 10
    assert V._noalloc_n(tris.reshape(-1), ok, np.zeros(12, np.uint32)) == 10
    for bad in ((tris.reshape(-1)[:89], ok, ok),          # flat, not a multiple of 9
                (tris.reshape(30, 3), ok, ok),            # wrong shape
                (tris, np.zeros(9, np.int32), ok),        # codes too short
                (tris, ok, np.zeros(9, np.int32)),        # ids too short
                (tris, np.zeros(10, np.float32), ok),     # not integers
                (tris, ok, np.zeros(10, np.int64))):      # not 32-bit
        with pytest.raises(ValueError):
            V.vafr_morton_sort_noalloc(*bad)
    with pytest.raises(TypeError):
        V.vafr_morton_sort_noalloc(tris.astype(np.float64), ok, ok)
