"""Pins of the oracle's boundary-element solve (CPU only).

Checked against identities and closed forms the paper's formulation fixes
(Sec. 3.1): the double-layer identity, reproduction of harmonic data on a
closed curve, the null space of the Neumann Galerkin matrix, the SVD
pseudo-inverse against an independent bordered LU solve, the exact
piecewise-constant solution for a handle that cuts the square in two, and
the symmetry of the square under quarter turns.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy import integrate

import oracle


def _ngon(N, c=(0.5, 0.5), R=0.2, ccw=True):
    th = 2 * math.pi * np.arange(N + 1) / N
    if not ccw:
        th = -th
    pts = np.stack([c[0] + R * np.cos(th), c[1] + R * np.sin(th)], 1)
    return np.concatenate([pts[:-1], pts[1:]], 1)          # [N, 4]


def test_double_layer_identity():
    """sum_p Dl_p = -1 inside, -1/2 on a panel, 0 outside (closed CCW polygon, eps=0)."""
    ab = _ngon(40)
    rng = np.random.default_rng(0)
    r = np.sqrt(rng.uniform(0, 1, 50)) * 0.19
    a = rng.uniform(0, 2 * math.pi, 50)
    inside = np.stack([0.5 + r * np.cos(a), 0.5 + r * np.sin(a)], 1)
    outside = rng.uniform(0, 1, (200, 2))
    outside = outside[np.hypot(outside[:, 0] - 0.5, outside[:, 1] - 0.5) > 0.21]
    on = 0.5 * (ab[:, :2] + ab[:, 2:])
    for pts, want in ((inside, -1.0), (outside, 0.0)):
        S, Dl = oracle.pair_terms(pts, ab, 0.0, 0.0)
        np.testing.assert_allclose(Dl.sum(1), want, atol=1e-13)
    # on the curve: principal value, the flat self panel contributes 0
    S, Dl = oracle.pair_terms(on, ab, 0.0, 0.0)
    Dl[np.arange(len(on)), np.arange(len(on))] = 0.0
    np.testing.assert_allclose(Dl.sum(1), -0.5, atol=1e-13)


def test_double_layer_regularised_far_field():
    """With eps>0 the identity still holds away from the curve up to O(eps^2)."""
    ab = _ngon(40)
    pts = np.array([[0.5, 0.5], [0.45, 0.55], [0.9, 0.9], [0.1, 0.2]])
    want = np.array([-1, -1, 0, 0.0])
    for eps in (1e-2, 1e-3):
        S, Dl = oracle.pair_terms(pts, ab, eps, eps)
        err = np.abs(Dl.sum(1) - want).max()
        assert err < 10 * eps * eps / 0.1 ** 2


@pytest.mark.parametrize("name", ["one", "x", "x2-y2"])
def test_harmonic_reproduction(name):
    """Green's representation: w_d = h, w_c = dh/dn on a closed curve gives f = h
    inside and 0 outside (Eq. handleterm); panel-constant data converges as O(L^2)."""
    hfun = {"one": lambda p: np.ones(len(p)),
            "x": lambda p: p[:, 0],
            "x2-y2": lambda p: p[:, 0] ** 2 - p[:, 1] ** 2}[name]
    grad = {"one": lambda p: np.zeros_like(p),
            "x": lambda p: np.stack([np.ones(len(p)), np.zeros(len(p))], 1),
            "x2-y2": lambda p: np.stack([2 * p[:, 0], -2 * p[:, 1]], 1)}[name]
    inside = np.array([[0.5, 0.5], [0.55, 0.47], [0.44, 0.52]])
    outside = np.array([[0.95, 0.5], [0.1, 0.1], [0.5, 0.05]])
    errs = []
    for N in (64, 128, 256):
        ab = _ngon(N)
        mid = 0.5 * (ab[:, :2] + ab[:, 2:])
        e = ab[:, 2:] - ab[:, :2]
        n = np.stack([e[:, 1], -e[:, 0]], 1) / np.linalg.norm(e, axis=1)[:, None]
        wd = np.repeat(hfun(mid)[:, None], 3, 1)
        wc = np.repeat(np.sum(grad(mid) * n, 1)[:, None], 3, 1)
        fi = oracle.handle_field(inside, ab, wd, wc, 1e-12, 1e-12)[:, 0]
        fo = oracle.handle_field(outside, ab, wd, wc, 1e-12, 1e-12)[:, 0]
        errs.append(max(np.abs(fi - hfun(inside)).max(), np.abs(fo).max()))
    if name == "one":
        assert max(errs) < 1e-12
    else:
        assert errs[-1] < 2e-5
        assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_square_boundary_angles():
    """Segments of the square subtend 2 pi at interior points (CCW, outward normal)."""
    seg = oracle.square_boundary(16)
    pts = np.random.default_rng(1).uniform(0.01, 0.99, (50, 2))
    phi = oracle.angles(pts, seg)
    np.testing.assert_allclose(phi.sum(1), 2 * math.pi, atol=1e-12)
    # outward right normal
    e = seg[:, 2:] - seg[:, :2]
    n = np.stack([e[:, 1], -e[:, 0]], 1)
    mid = 0.5 * (seg[:, :2] + seg[:, 2:])
    assert np.all(np.sum((mid - 0.5) * n, 1) > 0)


def test_galerkin_entries_quadrature():
    """A_ij against adaptive quadrature of the inner kernel n.(y-x)/r^2."""
    M = 8
    seg = oracle.square_boundary(M)
    A = oracle.assemble_A(seg)
    gp = oracle.gauss_points(seg)
    ell = 1.0 / M
    for (i, j) in [(0, 1), (0, 5), (3, 12), (9, 20), (31, 0), (7, 8), (15, 16)]:
        a, b = seg[j, :2], seg[j, 2:]
        e = b - a
        n = np.array([e[1], -e[0]]) / np.linalg.norm(e)
        val = 0.0
        for q in range(3):
            x = gp[i, q]
            inner, _ = integrate.quad(
                lambda s: -np.dot(n, a + s * e - x) / np.sum((a + s * e - x) ** 2) / (2 * math.pi)
                * np.linalg.norm(e), 0, 1, epsabs=1e-15, epsrel=1e-13, limit=200)
            val += oracle.GAUSS_WEIGHTS[q] * ell * inner
        assert A[i, j] == pytest.approx(val, rel=1e-11, abs=1e-15)
    assert A[5, 5] == 0.5 * ell


def test_null_space_and_pinv():
    """A 1 = 0; the SVD pseudo-inverse equals the bordered-LU solution."""
    M = 32
    seg = oracle.square_boundary(M)
    A = oracle.assemble_A(seg)
    Nb = A.shape[0]
    assert np.abs(A @ np.ones(Nb)).max() < 1e-15
    Ap = oracle.pinv_svd(A)
    # left null vector by an LU solve of (A^T + 1 1^T) w = 1
    one = np.ones(Nb)
    w = scipy.linalg.lu_solve(scipy.linalg.lu_factor(A.T + np.outer(one, one)), one)
    v = w / np.linalg.norm(w)
    assert np.abs(A.T @ v).max() < 1e-13
    B = np.zeros((Nb + 1, Nb + 1))
    B[:Nb, :Nb] = A
    B[:Nb, Nb] = v
    B[Nb, :Nb] = 1.0
    lu = scipy.linalg.lu_factor(B)
    rng = np.random.default_rng(2)
    for _ in range(3):
        f = rng.normal(size=Nb)
        x = scipy.linalg.lu_solve(lu, np.concatenate([f, [0.0]]))[:Nb]
        np.testing.assert_allclose(Ap @ f, x, rtol=0, atol=1e-10 * np.abs(x).max())
        assert abs(np.sum(Ap @ f)) < 1e-10


def _line_oracle(M, eps=1e-9, mean=(0.3, 0.4, 0.5)):
    o = oracle.Oracle(1, [64], [0], mean, segs_per_side=M, eps_d=eps, eps_c=eps)
    th = np.zeros(32)
    for j in range(4):
        th[j * 8:j * 8 + 2] = (j / 3.0, 0.5)
        th[j * 8 + 2:j * 8 + 5] = (1.0, -0.5, 0.25)     # w_d per channel
    return o, th


def test_handle_splitting_square():
    """A straight handle across the square with constant w_d: the Neumann
    solution is piecewise constant, mean +- w_d/2 (left side of a->b is '+')."""
    pts = np.array([[0.5, 0.8], [0.2, 0.7], [0.8, 0.9], [0.5, 0.2], [0.3, 0.1], [0.7, 0.3]])
    sgn = np.array([1, 1, 1, -1, -1, -1.0])
    wd = np.array([1.0, -0.5, 0.25])
    errs = []
    for M in (32, 64, 128):
        o, th = _line_oracle(M)
        u = o.eval(th, pts)
        want = np.array([0.3, 0.4, 0.5]) + 0.5 * sgn[:, None] * wd
        errs.append(np.abs(u - want).max())
    # the exact boundary solution (+-1/2, jumping where the handle meets the
    # square, at a segment end) lies in the piecewise-constant space and the
    # inner integrals are exact, so the discrete solution is exact too
    assert max(errs) < 1e-12


def test_quarter_turn_symmetry():
    """Rotating handles and points by 90 degrees about the centre maps the
    square's boundary discretisation onto itself: colours are unchanged."""
    import gen
    sc = gen.make_scene(1)
    o = oracle.Oracle.from_scene(sc, segs_per_side=32)
    th = sc.theta_true.reshape(-1, 8).copy()
    rot = lambda p: np.stack([1.0 - p[..., 1], p[..., 0]], -1)
    th2 = th.copy()
    th2[:, 0:2] = rot(th[:, 0:2])
    pts = gen.make_samples(16, 2, 5)
    u1 = o.eval(sc.theta_true, pts)
    u2 = o.eval(th2.reshape(-1), rot(pts))
    np.testing.assert_allclose(u1, u2, atol=1e-11)


# ---- paper-literal 3 x 3 Galerkin rule (galerkin_mode = 1) ----------------------

def test_galerkin_3x3_gauss_order():
    """The 3-point Gauss inner integral of a smooth kernel converges to the
    exact (mode 0) entry with the rule's order: the relative error of the
    pair (centre of the bottom side, centre of the top side) falls by 2^6 per
    halving of the segment length."""
    from oracle.bem import assemble_A, square_boundary
    errs = []
    for M in (16, 32, 64):
        seg = square_boundary(M)
        A0, A1 = assemble_A(seg, 0), assemble_A(seg, 1)
        i, j = M // 2, 2 * M + M // 2          # bottom centre, top centre (opposite)
        errs.append(abs(A1[i, j] - A0[i, j]) / abs(A0[i, j]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 40 < r1 < 90 and 40 < r2 < 90, (errs, r1, r2)


def test_galerkin_3x3_structure():
    """Quarter-turn invariance of the square (side s -> side s+1), zero
    entries for collinear segments of one side, and the diagonal."""
    from oracle.bem import assemble_A, square_boundary
    M = 12
    seg = square_boundary(M)
    A1 = assemble_A(seg, 1)
    Nb = 4 * M
    idx = (np.arange(Nb) + M) % Nb
    assert np.allclose(A1[np.ix_(idx, idx)], A1, rtol=0, atol=1e-15)
    for i in range(M):
        for j in range(M):
            if i != j:
                assert A1[i, j] == 0.0
    ell = 1.0 / M
    assert np.allclose(np.diag(A1), 0.5 * ell, rtol=0, atol=1e-16)
    # not exactly singular any more: the constants are no null vector, but
    # the smallest singular value stays well separated (the truncation of
    # Sec. 3.1.3 remains well defined)
    s = np.linalg.svd(A1, compute_uv=False)
    assert s[-1] < 1e-3 * s[-2]


# ---- polygon subdomains -----------------------------------------------------------

L_SHAPE = [(0.0, 0.0), (1.0, 0.0), (1.0, 0.5), (0.5, 0.5), (0.5, 1.0), (0.0, 1.0)]


def test_polygon_boundary_identities():
    """On a non-convex (L-shaped) polygon: the square's segmentation is the
    4-vertex case, the angles of all segments sum to 2 pi inside, 0 outside,
    and the exact-inner Galerkin rows sum to zero."""
    from oracle.bem import polygon_boundary, square_boundary
    sq = polygon_boundary([(0, 0), (1, 0), (1, 1), (0, 1)], 8)
    assert np.array_equal(sq, square_boundary(8))
    seg = polygon_boundary(L_SHAPE, 8)
    inside = np.array([[0.25, 0.25], [0.75, 0.25], [0.25, 0.75], [0.45, 0.45]])
    outside = np.array([[0.75, 0.75], [0.6, 0.9], [1.2, 0.2]])
    assert np.allclose(oracle.angles(inside, seg).sum(1), 2 * np.pi, atol=1e-13)
    assert np.allclose(oracle.angles(outside, seg).sum(1), 0.0, atol=1e-13)
    A = oracle.assemble_A(seg)
    assert np.abs(A.sum(1)).max() < 1e-15


def test_handle_splitting_l_shape():
    """A straight handle at y = 1/4 across the L-shaped subdomain with constant
    w_d and w_c = 0: the Neumann solution is piecewise constant, the top part
    w_d above the bottom part, and the zero-mean boundary solution fixes the
    constants by the segment counts on each side: c_bot = -w_d n_top/(n_top +
    n_bot), c_top = w_d n_bot/(n_top + n_bot)."""
    mean = np.array([0.3, 0.4, 0.5])
    wd = np.array([1.0, -0.5, 0.25])
    pts_bot = np.array([[0.2, 0.1], [0.8, 0.2], [0.5, 0.05]])
    pts_top = np.array([[0.2, 0.4], [0.8, 0.4], [0.25, 0.9], [0.4, 0.6]])
    for M in (8, 16, 32):
        o = oracle.Oracle(1, [64], [0], mean, segs_per_side=M, eps_d=1e-9, eps_c=1e-9,
                          polygon=L_SHAPE)
        th = np.zeros(32)
        for j in range(4):
            th[j * 8:j * 8 + 2] = (j / 3.0, 0.25)
            th[j * 8 + 2:j * 8 + 5] = wd
        # segments below the line: bottom edge M, lower half of the right edge
        # M/2, lowest quarter of the left edge M/4
        n_bot = M + M // 2 + M // 4
        n_top = 6 * M - n_bot
        c_bot = -wd * n_top / (n_top + n_bot)
        c_top = wd * n_bot / (n_top + n_bot)
        assert np.abs(o.eval(th, pts_bot) - (mean + c_bot)).max() < 1e-12
        assert np.abs(o.eval(th, pts_top) - (mean + c_top)).max() < 1e-12
