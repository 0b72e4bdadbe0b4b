"""Numbers written out in the kernel sources (CPU only): the float
arctangent's polynomial (the project's own minimax fit, within the 2e-7 its
header states under float Horner evaluation), the mathematical constants,
and the 3-point Gauss-Legendre rule of the Galerkin integrals."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _kernel_coefficients():
    src = open(os.path.join(ROOT, "paper_2602_05492_gb300", "csrc", "fastmath.cuh")).read()
    body = src[src.index("fm_atan01"):]
    body = body[:body.index("return")]
    # p = c7; p = fmaf(p, s, c6); ... ; p = fmaf(p, s, c0)
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    assert len(vals) == 8
    return np.array(vals[::-1], np.float32)      # c0 .. c7


def _horner32(c, a):
    s = (a * a).astype(np.float32)
    p = np.float32(c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p * s + c[k]).astype(np.float32)
    return (a.astype(np.float32) * p).astype(np.float64)


def test_kernel_polynomial_error_bound():
    c = _kernel_coefficients()
    a = np.linspace(0.0, 1.0, 400001)
    err = np.abs(_horner32(c, a) - np.arctan(a)).max()
    assert err < 2e-7, err


def test_kernel_coefficients_are_the_fit():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "fit_atan", os.path.join(ROOT, "paper_2602_05492_gb300", "fit_atan.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    c, err = mod.fit(7, iters=200)
    assert err < 1.2e-7
    np.testing.assert_allclose(c.astype(np.float32), _kernel_coefficients(), rtol=2e-4, atol=2e-7)


def _const(path, name):
    src = open(os.path.join(ROOT, "paper_2602_05492_gb300", "csrc", path)).read()
    m = re.search(name + r"\s*=\s*([-+]?[0-9.]+(?:e[-+]?\d+)?)(f?)", src)
    assert m, name
    v = float(m.group(1))
    return np.float32(v) if m.group(2) else np.float64(v)


def test_kernel_constants_round_to_their_values():
    """Each written-out constant of the kernels is its value rounded to the
    constant's type."""
    d = {("common.cuh", "kPi"): np.pi, ("common.cuh", "kInv2Pi"): 1 / (2 * np.pi),
         ("common.cuh", "kInv4Pi"): 1 / (4 * np.pi), ("dmath.cuh", "kLn2d"): np.log(2.0),
         ("dmath.cuh", "kPiD"): np.pi, ("dmath.cuh", "kPi2D"): np.pi / 2,
         ("fastmath.cuh", "kLn2f"): np.log(2.0), ("fastmath.cuh", "kLn2Halff"): np.log(2.0) / 2,
         ("fastmath.cuh", "kFltMinNormal"): float(np.finfo(np.float32).tiny)}
    for (f, name), want in d.items():
        got = _const(f, name)
        assert got == type(got)(want), (f, name, got, want)


def test_gauss_rule_is_three_point_gauss_legendre():
    """Nodes 1/2 -+ sqrt(15)/10 and weights 5/18, 8/18, 5/18 on [0, 1]: exact
    for polynomials up to degree 5, not for degree 6."""
    src = open(os.path.join(ROOT, "paper_2602_05492_gb300", "csrc", "common.cuh")).read()
    body = src[src.index("gauss_node"):src.index("gauss_weight")]
    lo, mid, hi = sorted(float(v) for v in re.findall(r"(0\.\d{6,}|0\.5)", body))
    assert mid == 0.5
    import decimal
    decimal.getcontext().prec = 40
    r = decimal.Decimal(15).sqrt() / 10                 # the nodes to 40 digits, rounded once
    assert lo == float(decimal.Decimal("0.5") - r) and hi == float(decimal.Decimal("0.5") + r)
    x, w = np.array([lo, mid, hi]), np.array([5, 8, 5]) / 18
    for k in range(6):
        assert abs(w @ x ** k - 1 / (k + 1)) < 1e-15
    assert abs(w @ x ** 6 - 1 / 7) > 1e-6
