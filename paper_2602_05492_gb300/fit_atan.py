"""Minimax polynomial for atan on [0, 1], written into csrc/fastmath.cuh.

atan(a) ~= a * p(a^2), p of degree `deg` in s = a^2, fitted for minimal
maximum absolute error of atan by Lawson's algorithm (iteratively reweighted
least squares converging to the Chebyshev/minimax solution) on a dense grid.
Run: python paper_2602_05492_gb300/fit_atan.py [deg]
"""
import sys

import numpy as np


def fit(deg: int, iters: int = 400):
    a = np.cos(np.linspace(0, np.pi / 2, 20001)) ** 1  # dense, clustered near 1 and 0
    a = np.unique(np.concatenate([a, np.linspace(0, 1, 20001)]))
    s = a * a
    V = np.stack([a * s ** k for k in range(deg + 1)], 1)   # columns a, a^3, ...
    y = np.arctan(a)
    w = np.ones_like(a) / len(a)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
        e = np.abs(V @ c - y)
        w = w * e
        w /= w.sum()
    err = np.abs(V @ c - y).max()
    return c, err


if __name__ == "__main__":
    deg = int(sys.argv[1]) if len(sys.argv) > 1 else 7
    c, err = fit(deg)
    c32 = c.astype(np.float32)
    a = np.linspace(0, 1, 200001)
    s = (a * a).astype(np.float32)
    p = np.float32(0)
    for k in range(deg, -1, -1):
        p = p * s + c32[k]
    e32 = np.abs(a.astype(np.float32) * p - np.arctan(a)).max()
    print(f"deg {deg}: max |err| {err:.3e} (float64 coefficients), {e32:.3e} (float32 Horner)")
    print(", ".join(f"{v:.9e}f" for v in c32))
