"""Fits the odd polynomial used by the reconstruction kernel for the angle
fraction atan(t) / (2 pi), t in [0, 1]:

    atan(t) / (2 pi) ~= t * (c0 + c1 t^2 + ... + c7 t^14)

Method: near-minimax (Chebyshev) fit by Lawson's iteratively reweighted least
squares on 4,000 Chebyshev-distributed samples, FP64.  Prints the FP32
coefficients and the error of an FP32 Horner evaluation against FP64 atan.
Run: python paper_2503_23410_gb300/csrc/fit_atan.py
"""

import numpy as np


def fit(k: int = 8, n: int = 4000, iters: int = 200):
    t = (1 - np.cos(np.linspace(0, np.pi, n))) / 2
    y = np.arctan(t) / (2 * np.pi)
    A = np.stack([t ** (2 * j + 1) for j in range(k)], 1)
    w = np.ones(n)
    c = None
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(A * np.sqrt(w)[:, None], y * np.sqrt(w), rcond=None)
        err = np.abs(A @ c - y)
        w = w * (err / err.max() + 1e-12)
        w /= w.sum() / n
    return c


def fp32_error(c32: np.ndarray) -> float:
    t = np.linspace(0, 1, 400001).astype(np.float32)
    s = t * t
    acc = np.full_like(s, c32[-1])
    for j in range(len(c32) - 2, -1, -1):
        acc = (acc * s + c32[j]).astype(np.float32)
    p = (acc * t).astype(np.float32)
    return float(np.abs(p.astype(np.float64) - np.arctan(t.astype(np.float64)) / (2 * np.pi)).max())


if __name__ == "__main__":
    c = fit().astype(np.float32)
    for j, v in enumerate(c):
        print(f"c{j} = {float(v)!r}f")
    print("max |error| of the FP32 evaluation:", fp32_error(c))
