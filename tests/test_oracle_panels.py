"""Pins of the oracle's per-panel integrals (CPU only).

Each quantity is checked against something other than the oracle itself:
hand-derived closed forms (tests/golden), adaptive quadrature of the
paper's integrals in parametric form (Sec. 3.2.2), central finite
differences, and the translation invariance d/da + d/db = -d/dx.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "panel_closed_forms.txt")


def _golden():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append((np.array([float(v) for v in f[:4]]), float(f[4]), float(f[5]),
                     float(f[6]), f[7], float(f[8])))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[4]}@({r[1]},{r[2]})eps{r[3]}")
def test_golden_closed_forms(row):
    ab, x, y, eps, q, val = row
    S, Dl, dS, dD = oracle.pair_terms(np.array([[x, y]]), ab[None], eps, eps, grad=True)
    got = {"S": S[0, 0], "Dl": Dl[0, 0], "dS/dbx": dS[0, 0, 2], "dS/dby": dS[0, 0, 3],
           "dDl/dbx": dD[0, 0, 2], "dDl/dby": dD[0, 0, 3]}[q]
    assert got == pytest.approx(val, rel=1e-13, abs=1e-15)


# ---- brute-force quadrature of the parametric form --------------------------

def _G(x, z, eps):
    return -np.log(np.sum((z - x) ** 2) + eps * eps) / (4 * math.pi)


def _dGdn(x, z, n, eps):
    d = z - x
    return -np.dot(n, d) / (np.sum(d * d) + eps * eps) / (2 * math.pi)


def _quad(fun, breaks=()):
    pts = sorted(b for b in breaks if 0.0 < b < 1.0)
    v, err = integrate.quad(fun, 0.0, 1.0, points=pts or None, epsabs=1e-15, epsrel=1e-13,
                            limit=400)
    return v


def _brute(ab, x, eps):
    """S, Dl and all 8 endpoint derivatives by adaptive quadrature in s."""
    a, b = ab[:2], ab[2:]
    e = b - a
    L = np.linalg.norm(e)
    tau = e / L
    n = np.array([tau[1], -tau[0]])
    s0 = np.clip(np.dot(x - a, e) / (L * L), 0.0, 1.0)      # closest parameter
    z = lambda s: a + s * e
    S = _quad(lambda s: _G(x, z(s), eps) * L, [s0])
    Dl = _quad(lambda s: _dGdn(x, z(s), n, eps) * L, [s0])
    # d/da, d/db of int_0^1 F(z(s)) L ds under the integral sign:
    #   single layer: d/da [L G] = -tau G + L grad_z G (1-s);   d/db: +tau G + L grad_z G s
    #   double layer: L dG/dn = -(1/2pi) cross(z-x... ) written as e_perp.(z-x) / (r^2+eps^2)
    def gradG(zz):
        d = zz - x
        return -2.0 * d / (np.sum(d * d) + eps * eps) / (4 * math.pi)

    dS = np.zeros(4)
    for k in range(2):
        dS[k] = _quad(lambda s: -tau[k] * _G(x, z(s), eps) + L * gradG(z(s))[k] * (1 - s), [s0])
        dS[2 + k] = _quad(lambda s: tau[k] * _G(x, z(s), eps) + L * gradG(z(s))[k] * s, [s0])

    def lDl(aa, bb, s):
        ee = bb - aa
        zz = aa + s * ee
        d = zz - x
        perp = np.array([ee[1], -ee[0]])      # L * n
        return -np.dot(perp, d) / (np.sum(d * d) + eps * eps) / (2 * math.pi)

    dD = np.zeros(4)
    hstep = 1e-6
    # derivative of the integrand in the endpoint coordinates, taken by a
    # central difference inside the quadrature (integrand is smooth for eps>0)
    for k in range(4):
        def integrand(s, k=k):
            dp = np.zeros(4)
            dp[k] = hstep
            p1, p2 = ab + dp, ab - dp
            return (lDl(p1[:2], p1[2:], s) - lDl(p2[:2], p2[2:], s)) / (2 * hstep)
        dD[k] = _quad(integrand, [s0])
    return S, Dl, dS, dD


def _cases():
    rng = np.random.default_rng(7)
    out = []
    ab = np.array([0.2, 0.3, 0.35, 0.32])
    for eps in (1e-2, 1e-3):
        # far, near (h << eps), collinear beyond the end, at an endpoint, on the panel
        out += [(ab, np.array([0.7, 0.8]), eps), (ab, np.array([0.27, 0.3135]), eps),
                (ab, np.array([0.5, 0.33]), eps), (ab, ab[:2].copy(), eps),
                (ab, np.array([0.275, 0.315]), eps)]
    for _ in range(6):
        a = rng.uniform(0, 1, 2)
        b = a + rng.normal(0, 0.05, 2)
        x = a + rng.normal(0, 0.03, 2)
        out.append((np.concatenate([a, b]), x, 1e-2))
    return out


@pytest.mark.parametrize("case", _cases())
def test_bruteforce_quadrature(case):
    ab, x, eps = case
    S, Dl, dS, dD = oracle.pair_terms(x[None], ab[None], eps, eps, grad=True)
    bS, bD, bdS, bdD = _brute(ab, x, eps)
    assert S[0, 0] == pytest.approx(bS, rel=1e-11, abs=1e-13)
    assert Dl[0, 0] == pytest.approx(bD, rel=1e-11, abs=1e-13)
    np.testing.assert_allclose(dS[0, 0], bdS, rtol=1e-9, atol=1e-11 * (1 + abs(bdS).max()))
    np.testing.assert_allclose(dD[0, 0], bdD, rtol=1e-6, atol=1e-7 * (1 + abs(bdD).max()))


def test_finite_differences_endpoints():
    rng = np.random.default_rng(3)
    for eps in (1e-2, 3e-3):
        ab = rng.uniform(0.2, 0.8, size=(16, 4))
        ab[:, 2:] = ab[:, :2] + rng.normal(0, 0.04, size=(16, 2))
        xy = rng.uniform(0, 1, size=(32, 2))
        xy[:16] = ab[:, :2] + rng.normal(0, 0.02, size=(16, 2))   # near field
        S, Dl, dS, dD = oracle.pair_terms(xy, ab, eps, eps, grad=True)
        h = 1e-6
        for k in range(4):
            ap, am = ab.copy(), ab.copy()
            ap[:, k] += h
            am[:, k] -= h
            Sp, Dp = oracle.pair_terms(xy, ap, eps, eps)
            Sm, Dm = oracle.pair_terms(xy, am, eps, eps)
            fS = (Sp - Sm) / (2 * h)
            fD = (Dp - Dm) / (2 * h)
            np.testing.assert_allclose(dS[:, :, k], fS, rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(dD[:, :, k], fD, rtol=1e-6, atol=1e-7 * np.abs(fD).max())


def test_translation_invariance():
    """d/da + d/db = -d/dx for both layers (the integrals depend on a-x, b-x)."""
    rng = np.random.default_rng(11)
    ab = rng.uniform(0.3, 0.7, size=(8, 4))
    xy = rng.uniform(0.2, 0.8, size=(20, 2))
    eps = 1e-2
    S, Dl, dS, dD = oracle.pair_terms(xy, ab, eps, eps, grad=True)
    h = 1e-6
    for k in range(2):
        xp, xm = xy.copy(), xy.copy()
        xp[:, k] += h
        xm[:, k] -= h
        Sp, Dp = oracle.pair_terms(xp, ab, eps, eps)
        Sm, Dm = oracle.pair_terms(xm, ab, eps, eps)
        np.testing.assert_allclose(dS[:, :, k] + dS[:, :, 2 + k], -(Sp - Sm) / (2 * h),
                                   rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(dD[:, :, k] + dD[:, :, 2 + k], -(Dp - Dm) / (2 * h),
                                   rtol=1e-6, atol=1e-7)


def test_zero_length_panel():
    S, Dl, dS, dD = oracle.pair_terms(np.array([[0.5, 0.5]]), np.array([[0.3, 0.3, 0.3, 0.3]]),
                                      1e-2, 1e-2, grad=True)
    assert S[0, 0] == 0 and Dl[0, 0] == 0 and not dS.any() and not dD.any()


def test_separate_eps():
    """S follows eps_c only and Dl follows eps_d only."""
    ab = np.array([[0.1, 0.1, 0.4, 0.2]])
    xy = np.array([[0.25, 0.16]])
    S1, D1 = oracle.pair_terms(xy, ab, 1e-2, 1e-3)
    S2, D2 = oracle.pair_terms(xy, ab, 1e-2, 1e-2)
    S3, D3 = oracle.pair_terms(xy, ab, 1e-3, 1e-3)
    assert D1 == D2 and S1 == S3 and S1 != S2 and D1 != D3
