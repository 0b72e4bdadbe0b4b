"""Pins of the oracle's Sec. 4.4 regularisers, pruning and the Sec. 4.2
initialisation of segment handles (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from oracle import regularize as R


def _rand_handles(H, seed, long_frac=0.5):
    rng = np.random.default_rng(seed)
    th = np.zeros((H, 10))
    th[:, 0:2] = rng.uniform(0.2, 0.8, size=(H, 2))
    ang = rng.uniform(0, 2 * np.pi, H)
    ln = np.where(rng.random(H) < long_frac, rng.uniform(0.12, 0.3, H), rng.uniform(0.02, 0.08, H))
    th[:, 2:4] = th[:, 0:2] + ln[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    th[:, 4:10] = rng.uniform(-0.3, 0.3, size=(H, 6))
    return th.reshape(-1)


def _saturation_curvature(th, rp):
    """The dropped part of the exact sparsity Hessian,
    -lam s (2 tanh(rho/t) / (t rho^2)) w w^T per weight vector."""
    n = th.size
    D = np.zeros((n, n))
    t = rp.sparse_t
    for lam, off in ((rp.sparse_wd, 4), (rp.sparse_wc, 7)):
        if not lam > 0:
            continue
        for h in range(n // 10):
            w = th[10 * h + off:10 * h + off + 3]
            rho = math.sqrt(float(w @ w) + rp.sparse_eps ** 2)
            tn = math.tanh(rho / t)
            i = 10 * h + off
            D[i:i + 3, i:i + 3] -= lam * (1 - tn * tn) * (2 * tn / (t * rho * rho)) * np.outer(w, w)
    return D


def _fd_check(th, rp, pairs, h=1e-6):
    g, Hm = R.reg_grad_hess(th, rp, pairs)
    # the kept Hessian is PSD; with the dropped saturation curvature added
    # back it must be the exact Hessian of the loss
    assert np.linalg.eigvalsh(Hm).min() >= -1e-10 * max(1.0, np.abs(Hm).max())
    Hm = Hm + _saturation_curvature(th, rp)
    n = th.size
    gfd = np.zeros(n)
    Hfd = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        gfd[i] = (R.reg_loss(th + e, rp, pairs) - R.reg_loss(th - e, rp, pairs)) / (2 * h)
        gp, _ = R.reg_grad_hess(th + e, rp, pairs)
        gm, _ = R.reg_grad_hess(th - e, rp, pairs)
        Hfd[:, i] = (gp - gm) / (2 * h)
    np.testing.assert_allclose(g, gfd, rtol=1e-6, atol=1e-8 * max(1.0, np.abs(g).max()))
    np.testing.assert_allclose(Hm, Hfd, rtol=1e-5, atol=1e-6 * max(1.0, np.abs(Hm).max()))
    np.testing.assert_array_equal(Hm, Hm.T)


# ---- handle length --------------------------------------------------------------

def test_length_closed_form():
    th = np.zeros(10)
    th[2:4] = (0.3, 0.4)                      # |b - a| = 0.5
    rp = R.RegParams(len_weight=2.0, len_max=0.3)
    assert R.reg_loss(th, rp) == pytest.approx(2.0 * 0.2 ** 2, rel=1e-15)
    g, Hm = R.reg_grad_hess(th, rp)
    # gradient along the handle: 2 lam (L - l) u = 2*2*0.2*(0.6, 0.8)
    np.testing.assert_allclose(g[2:4], [0.48, 0.64], rtol=1e-14)
    np.testing.assert_allclose(g[0:2], [-0.48, -0.64], rtol=1e-14)
    short = th.copy()
    short[2:4] = (0.1, 0.1)
    assert R.reg_loss(short, rp) == 0.0
    gs, Hs = R.reg_grad_hess(short, rp)
    assert not gs.any() and not Hs.any()


def test_length_derivatives_fd():
    th = _rand_handles(6, 1)
    _fd_check(th, R.RegParams(len_weight=3.0, len_max=0.1), None)


# ---- snapping -----------------------------------------------------------------

def _snap_layout():
    th = np.zeros((3, 10))
    th[0, 0:4] = (0.2, 0.2, 0.4, 0.2)         # b_0 = endpoint 1
    th[1, 0:4] = (0.405, 0.2, 0.6, 0.2)       # a_1 = endpoint 2: collinear, gap 0.005
    th[2, 0:4] = (0.41, 0.205, 0.41, 0.4)     # a_2 = endpoint 4: perpendicular, near both
    return th.reshape(-1)


def test_snap_pairs_hand_built():
    th = _snap_layout()
    rp = R.RegParams(snap_weight=1.0, snap_radius=0.02, snap_alpha=0.5)
    # b_0 and a_1 choose each other; a_2 would choose a_1 but is not chosen back
    assert R.snap_pairs(th, rp) == [(1, 2)]
    assert R.reg_loss(th, rp) == pytest.approx(0.005 ** 2, rel=1e-12)
    # move a_2 nearer to a_1 than b_0 is, so that distance and direction disagree
    th2 = th.reshape(3, 10).copy()
    th2[2, 0:2] = (0.407, 0.2015)             # |a_1 - a_2| = 0.0025
    th2 = th2.reshape(-1)
    assert R.snap_pairs(th2, rp) == [(1, 2)]                  # direction wins
    rp_d = R.RegParams(snap_weight=1.0, snap_radius=0.02, snap_alpha=1.0)
    assert R.snap_pairs(th2, rp_d) == [(2, 4)]                # distance only


def test_snap_radius_and_same_handle():
    th = np.zeros((2, 10))
    th[0, 0:4] = (0.2, 0.2, 0.21, 0.2)        # a_0, b_0 closer than r: same handle
    th[1, 0:4] = (0.5, 0.5, 0.7, 0.5)
    rp = R.RegParams(snap_weight=1.0, snap_radius=0.02)
    assert R.snap_pairs(th.reshape(-1), rp) == []


def test_snap_derivatives_fd():
    th = _snap_layout()
    rp = R.RegParams(snap_weight=5.0, snap_radius=0.02)
    _fd_check(th, rp, R.snap_pairs(th, rp))


# ---- sparsity -----------------------------------------------------------------

def test_sparsity_closed_form():
    lam, eps, t = 0.3, 1e-3, 0.05
    rp = R.RegParams(sparse_wd=lam, sparse_wc=0.0, sparse_eps=eps, sparse_t=t)
    th = np.zeros(10)
    th[2] = 0.1
    assert R.reg_loss(th, rp) == pytest.approx(lam * t * math.tanh(eps / t), rel=1e-14)
    th[4:7] = (30.0, 0.0, 40.0)               # saturated: lam t tanh(50 / 0.05) = lam t
    assert R.reg_loss(th, rp) == pytest.approx(lam * t, rel=1e-14)
    th[4:7] = (0.03, 0.0, 0.04)               # rho = sqrt(0.05^2 + eps^2)
    rho = math.sqrt(0.0025 + eps * eps)
    assert R.reg_loss(th, rp) == pytest.approx(lam * t * math.tanh(rho / t), rel=1e-14)


def test_sparsity_derivatives_fd():
    th = _rand_handles(4, 2)
    th.reshape(4, 10)[0, 4:7] = (1e-4, -2e-4, 0.0)   # near the smoothed kink
    _fd_check(th, R.RegParams(sparse_wd=0.5, sparse_wc=0.1, sparse_eps=1e-3, sparse_t=0.05), None)


def test_all_terms_together_fd():
    th = _snap_layout()
    th.reshape(3, 10)[:, 4:10] = np.random.default_rng(3).uniform(-0.2, 0.2, (3, 6))
    rp = R.RegParams(len_weight=2.0, len_max=0.15, snap_weight=1.0, snap_radius=0.02,
                     sparse_wd=0.1, sparse_wc=0.05)
    _fd_check(th, rp, R.snap_pairs(th, rp))


# ---- pruning ------------------------------------------------------------------

def test_prune():
    th = _rand_handles(6, 4).reshape(6, 10)
    th[1, 4:10] = 1e-4                        # both norms tiny: pruned
    th[3, 4:7] = 1e-4                         # w_c still large: kept
    th[5, 4:10] = 0.0
    out, keep = R.prune(th.reshape(-1), 1e-2)
    assert list(keep) == [0, 2, 3, 4]
    o = out.reshape(4, 10)
    np.testing.assert_array_equal(o[:, 0:7], th[keep, 0:7])
    a = np.hypot(o[:, 2] - o[:, 0], o[:, 3] - o[:, 1])
    assert np.abs(a @ o[:, 7:10]).max() < 1e-15
    none, k0 = R.prune(th.reshape(-1), 10.0)
    assert none.size == 0 and k0.size == 0


# ---- initialisation -----------------------------------------------------------

def test_radical_inverse_values():
    np.testing.assert_allclose([R.radical_inverse(k, 3) for k in (1, 2, 3, 4, 5, 13)],
                               [1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9, 13 / 27], rtol=0, atol=2e-16)
    assert [R.radical_inverse(k, 2) for k in (1, 2, 3, 6)] == [0.5, 0.25, 0.75, 0.375]
    assert R.radical_inverse(0, 3) == 0.0


def test_point_in_polygon():
    L = [(0, 0), (1, 0), (1, 0.5), (0.5, 0.5), (0.5, 1), (0, 1)]
    assert R.point_in_polygon(0.25, 0.75, L)
    assert R.point_in_polygon(0.75, 0.25, L)
    assert not R.point_in_polygon(0.75, 0.75, L)
    assert not R.point_in_polygon(1.5, 0.25, L)


def test_init_first_points_and_lengths():
    th = R.init_segments(16, 0.05).reshape(-1, 10)
    assert th.shape[0] == 16                  # every Sobol point of (0,1)^2 is inside
    # the classic first points of the 2-D Sobol sequence (Gray-code order)
    np.testing.assert_array_equal(th[:4, 0:2], [[0.5, 0.5], [0.75, 0.25], [0.25, 0.75],
                                                [0.375, 0.375]])
    ln = np.hypot(th[:, 2] - th[:, 0], th[:, 3] - th[:, 1])
    ang = np.arctan2(th[:, 3] - th[:, 1], th[:, 2] - th[:, 0]) % (2 * np.pi)
    full = ln > 0.05 - 1e-12
    np.testing.assert_allclose(ln[full], 0.05, rtol=1e-12)
    want = np.array([2 * np.pi * R.radical_inverse(k, 3) for k in range(1, 17)])
    np.testing.assert_allclose(ang, want % (2 * np.pi), atol=1e-12)
    assert not th[:, 4:10].any()


def test_init_clips_to_subdomain():
    L = [(0, 0), (1, 0), (1, 0.5), (0.5, 0.5), (0.5, 1), (0, 1)]
    th = R.init_segments(64, 0.3, polygon=L).reshape(-1, 10)
    assert 0 < th.shape[0] < 64
    for h in th:
        assert R.point_in_polygon(h[0], h[1], L)
        mid = 0.5 * (h[0:2] + h[2:4])
        assert R.point_in_polygon(mid[0], mid[1], L)
    ln = np.hypot(th[:, 2] - th[:, 0], th[:, 3] - th[:, 1])
    assert (ln <= 0.3 + 1e-12).all() and (ln < 0.3 - 1e-6).any()
    # a clipped handle ends on an edge of the polygon
    h = th[np.argmin(ln)]
    bx, by = h[2], h[3]
    on_edge = any(abs((qx - px) * (by - py) - (qy - py) * (bx - px)) < 1e-12 and
                  min(px, qx) - 1e-12 <= bx <= max(px, qx) + 1e-12 and
                  min(py, qy) - 1e-12 <= by <= max(py, qy) + 1e-12
                  for (px, py), (qx, qy) in zip(L, L[1:] + L[:1]))
    assert on_edge


# ---- LM step with the regularisers --------------------------------------------

def test_lm_step_zero_weights_is_plain_step():
    H = 4
    th = _rand_handles(H, 5, long_frac=0.0)
    o = oracle.Oracle.segments(H, np.array([0.5, 0.5, 0.5]), segs_per_side=16)
    th = oracle.project_compat(o.geo, th)
    pts = np.random.default_rng(6).uniform(0.02, 0.98, size=(300, 2))
    tgt = o.eval(th + 0.01, pts)
    a = o.lm_step(th, pts, tgt, 1e-3)
    b = o.lm_step(th, pts, tgt, 1e-3, reg=R.RegParams())
    np.testing.assert_array_equal(a["theta_trial"], b["theta_trial"])
    assert a["loss_after"] == b["loss_after"]


def test_lm_step_length_penalty_shortens():
    """A heavy length penalty on one long handle: the damped step shortens it
    toward l_max, and the reported losses include the penalty."""
    H = 3
    th = _rand_handles(H, 7, long_frac=0.0).reshape(H, 10)
    th[0, 2:4] = th[0, 0:2] + (0.25, 0.0)
    th = th.reshape(-1)
    o = oracle.Oracle.segments(H, np.array([0.5, 0.5, 0.5]), segs_per_side=16)
    th = oracle.project_compat(o.geo, th)
    pts = np.random.default_rng(8).uniform(0.02, 0.98, size=(300, 2))
    tgt = o.eval(th, pts)                     # data already fit: only the penalty acts
    rp = R.RegParams(len_weight=10.0, len_max=0.1)
    res = o.lm_step(th, pts, tgt, 1e-4, reg=rp)
    assert res["loss_before"] == pytest.approx(10.0 * 0.15 ** 2, rel=1e-12)
    t1 = res["theta_trial"].reshape(H, 10)
    assert np.hypot(*(t1[0, 2:4] - t1[0, 0:2])) < 0.2
    assert res["accepted"]
