"""The reconstruction kernel's angle polynomial is the output of its fitting
script: re-running the fit (csrc/fit_atan.py, Lawson's reweighted least
squares) reproduces the FP32 coefficients compiled into the kernel
(VAFR_ATAN_COEFS in csrc/lp_map.cuh), and an FP32 Horner evaluation of those
coefficients stays within the stated 3e-8 of atan(t)/2pi on [0, 1]."""

import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_23410_gb300", "csrc")


def _kernel_coefs():
    txt = open(os.path.join(CSRC, "lp_map.cuh")).read()
    body = re.search(r"#define VAFR_ATAN_COEFS((?:[^\n]*\\\n)*[^\n]*)", txt).group(1)
    vals = [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    assert len(vals) == 8
    return np.array(vals[::-1], np.float32)      # the header lists t^15 ... t^1


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(CSRC, "fit_atan.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_coefficients_are_the_fit():
    fit = _fit_module()
    c = fit.fit().astype(np.float32)
    k = _kernel_coefs()
    # the same FP32 values, up to the last bit the least-squares solver may move
    assert np.all(np.abs(c - k) <= 2 * np.spacing(np.abs(k)))


def test_kernel_coefficients_meet_the_error_bound():
    fit = _fit_module()
    assert fit.fp32_error(_kernel_coefs()) < 3e-8
