"""Pins of the oracle's Jacobian, gradient and LM step (CPU only).

Against finite differences of the evaluation (Sec. 3.2: J = du/dtheta),
the exact linearity of the colour in the jump parameters (Eq. handleterm),
the constrained linear least-squares solution a Gauss-Newton step must reach
when only colours move (Eq. optimstep with lambda -> 0, Sec. 4.3), the
compatibility condition after every step (Sec. 3.1.2, 4.3), and recovery of
a noiseless target.
"""
import numpy as np
import pytest
import scipy.linalg

import gen
import oracle


def _small(seed=5, C=2, K=8, M=16, n=60):
    sc = gen.make_scene(dict(C=C, K=K, W=8, spp=2, layout="random", cross=0.5,
                             noise="gauss", sigma=0.05, n_closed=1), seed=seed)
    o = oracle.Oracle.from_scene(sc, segs_per_side=M)
    xy = np.random.default_rng(seed).uniform(0.02, 0.98, (n, 2))
    return sc, o, xy


def test_jacobian_vs_finite_differences():
    sc, o, xy = _small()
    th = sc.theta_init
    J = o.jac(th, xy)
    h = 1e-6
    act = o.geo.active()
    for k in range(o.geo.n_theta):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (o.eval(tp, xy) - o.eval(tm, xy)) / (2 * h)
        if not act[k]:
            assert np.abs(J[:, :, k]).max() == 0.0
            assert np.abs(fd).max() < 1e-8
            continue
        np.testing.assert_allclose(J[:, :, k], fd, rtol=1e-5, atol=1e-6 * (1 + np.abs(fd).max()))


def test_colour_columns_are_exact_differences():
    """u is affine in the jump parameters: J's colour columns equal unit-step differences."""
    sc, o, xy = _small(seed=6)
    th = sc.theta_init
    J = o.jac(th, xy)
    u0 = o.eval(th, xy)
    for h in range(4 * sc.n_curves):
        for off in range(2, 8):
            k = h * 8 + off
            tp = th.copy()
            tp[k] += 1.0
            np.testing.assert_allclose(o.eval(tp, xy) - u0, J[:, :, k], atol=1e-12)


def test_gradient_vs_finite_differences():
    sc, o, xy = _small(seed=7)
    th = sc.theta_init
    target = np.random.default_rng(1).uniform(0, 1.2, (xy.shape[0], 3))
    L, g, H = o.gauss_newton(th, xy, target)
    assert L == pytest.approx(o.loss(th, xy, target), rel=1e-14)
    h = 1e-6
    fd = np.empty_like(g)
    for k in range(len(g)):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (o.loss(tp, xy, target) - o.loss(tm, xy, target)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())
    # H is the Gauss-Newton matrix: symmetric positive semi-definite
    np.testing.assert_allclose(H, H.T, atol=1e-14 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > -1e-10 * np.abs(H).max()
    # vjp form
    r = o.eval(th, xy) - np.minimum(target, 1.0)
    np.testing.assert_allclose(o.grad(th, xy, r) / xy.shape[0], g, rtol=1e-12, atol=1e-15)


def test_colour_step_is_constrained_least_squares():
    """With positions frozen and lambda -> 0 the LM step is the linear
    least-squares fit of the colours under the compatibility constraint."""
    sc, o, xy = _small(seed=8, n=200)
    th = oracle.project_compat(o.geo, sc.theta_init)
    target = np.random.default_rng(2).uniform(0, 1, (xy.shape[0], 3))
    L, g, H = o.gauss_newton(th, xy, target)
    nt = o.geo.n_theta
    free = np.zeros(nt, bool)
    for h in range(4 * sc.n_curves):
        free[h * 8 + 2:h * 8 + 8] = True
    delta = o.solve_step(th, H, g, 1e-14, free=free)
    # independent solution: design matrix probed by evaluation, constraint by null space
    cols = np.nonzero(free)[0]
    u0 = o.eval(th, xy)
    X = np.stack([(o.eval(th + np.eye(nt)[k], xy) - u0).reshape(-1) for k in cols], 1)
    r = (u0 - target).reshape(-1)
    Ac = o.constraint_matrix(th)[cols]
    N = scipy.linalg.null_space(Ac.T)
    z, *_ = np.linalg.lstsq(X @ N, -r, rcond=None)
    want = N @ z
    np.testing.assert_allclose(delta[cols], want, rtol=1e-6, atol=1e-8 * np.abs(want).max())
    assert np.abs(delta[~free]).max() == 0.0


def test_compatibility_after_steps():
    sc, o, xy = _small(seed=9, n=150)
    th = sc.theta_init.copy()
    target = np.random.default_rng(3).uniform(0, 1, (xy.shape[0], 3))
    lam = 1e-3
    for _ in range(3):
        res = o.lm_step(th, xy, target, lam)
        tn = res["theta_trial"]
        a = oracle.compat_vectors(o.geo, tn)
        wc = tn.reshape(-1, 8)[:, 5:8]
        assert np.abs(a @ wc).max() < 1e-14 * (1 + np.abs(wc).max() * np.abs(a).sum())
        th, lam = res["theta"], res["lambda_next"]


def test_noiseless_recovery():
    """Target = exact colours of a compatible truth: g vanishes there, and LM
    started from a perturbation drives the loss down by orders of magnitude."""
    sc, o, xy = _small(seed=10, n=400)
    truth = oracle.project_compat(o.geo, sc.theta_true)
    target = o.eval(truth, xy)
    L, g, H = o.gauss_newton(truth, xy, target)
    assert L < 1e-28 and np.abs(g).max() < 1e-14
    rng = np.random.default_rng(4)
    th = gen.perturb(truth, sc.closed, rng, 0.003, 0.02)
    th = oracle.project_compat(o.geo, th)
    lam = 1e-3
    L0 = o.loss(th, xy, target)
    for _ in range(8):
        res = o.lm_step(th, xy, target, lam)
        th, lam = res["theta"], res["lambda_next"]
    assert o.loss(th, xy, target) < 1e-6 * L0


def test_split_hessian_sets():
    """lm_step with a separate Hessian set: the same set gives the plain step,
    and H of the union of two sets is the sample-weighted mean of their Hs."""
    import gen
    import oracle
    sc = gen.make_scene(1)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)[::64]
    o = oracle.Oracle.from_scene(sc, segs_per_side=16)
    t = o.eval(sc.theta_true, xy)
    a = o.lm_step(sc.theta_init, xy, t, 1e-3)
    b = o.lm_step(sc.theta_init, xy, t, 1e-3, xy_h=xy)
    assert np.array_equal(a["theta"], b["theta"]) and a["loss_after"] == b["loss_after"]
    h1, h2 = xy[:200], xy[200:]
    H = o.hessian(sc.theta_init, xy)
    Hm = (200 * o.hessian(sc.theta_init, h1) + (len(xy) - 200) * o.hessian(sc.theta_init, h2)) / len(xy)
    assert np.abs(H - Hm).max() <= 1e-12 * np.abs(H).max()
