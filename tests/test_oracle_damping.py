"""Pins of the oracle's LM damping (CPU only).

The paper names the Levenberg-Marquardt update with D = diag(H) (Sec. 4.3,
Eq. (optimstep)) and damping "per Transtrum & Sethna" without constants.  The
readings taken: lambda / 3 after an accepted step, 2 lambda after a rejected
single trial, 10 times the largest lambda after several rejected trials, the
trial with the lowest loss taken when it lowers the loss, and lambda raised
tenfold (0 -> 1e-9) while H + lambda D does not factor, at most 12 times.

Each case here is built so that the outcome is known without the oracle:
  - at a stationary point (target = the colours of theta) g = 0, so every
    trial's step is 0 and its loss equals the current one: rejected;
  - a small perturbation of a noiseless truth with moderate damping lowers
    the loss (the step is a descent direction of a nearly quadratic model);
  - a hand-made H whose damped matrix is positive definite exactly when
    lambda > 1.5 (eigenvalues 1 + lambda +- 2.5 of the 2 x 2 block) fixes the
    lambda the retries must reach.
"""
import math

import numpy as np
import pytest

import gen
import oracle


def _scene(seed=21, C=2, K=8, M=16, n=120):
    sc = gen.make_scene(dict(C=C, K=K, W=8, spp=2, layout="random", cross=0.5,
                             noise="gauss", sigma=0.05, n_closed=0), seed=seed)
    o = oracle.Oracle.from_scene(sc, segs_per_side=M, mean_color=[0.3, 0.35, 0.4])
    xy = np.random.default_rng(seed).uniform(0.03, 0.97, (n, 2))
    return sc, o, xy


def _stationary(seed=22):
    """theta compatible, target = its own colours (all below the clamp at 1)."""
    sc, o, xy = _scene(seed)
    th = oracle.project_compat(o.geo, sc.theta_init)
    # keep the colours below 1 so that min(t, 1) leaves the target as it is
    th.reshape(-1, 8)[:, 2:8] *= 0.2
    th = oracle.project_compat(o.geo, th)
    target = o.eval(th, xy)
    assert target.max() < 1.0
    return sc, o, xy, th, target


def _descent(seed=23):
    sc, o, xy = _scene(seed)
    truth = oracle.project_compat(o.geo, sc.theta_true)
    truth.reshape(-1, 8)[:, 2:8] *= 0.3
    truth = oracle.project_compat(o.geo, truth)
    target = np.minimum(o.eval(truth, xy), 1.0)
    th = gen.perturb(truth, sc.closed, np.random.default_rng(seed), 0.002, 0.02)
    th = oracle.project_compat(o.geo, th)
    return sc, o, xy, th, target


def test_reject_at_stationary_point_doubles_lambda():
    sc, o, xy, th, target = _stationary()
    res = o.lm_step(th, xy, target, 1e-2)
    assert res["loss_before"] < 1e-28
    assert np.abs(res["g"]).max() < 1e-14
    assert not res["accepted"] and res["best_trial"] == -1
    assert res["lambda_next"] == 2e-2
    assert np.array_equal(res["theta"], th)


def test_reject_with_several_trials_takes_ten_times_the_largest():
    sc, o, xy, th, target = _stationary()
    res = o.lm_step(th, xy, target, [1e-3, 1e-2, 1e-1, 1.0])
    assert not res["accepted"] and res["best_trial"] == -1
    assert res["lambda_next"] == 10.0
    assert res["lambdas_used"] == [1e-3, 1e-2, 1e-1, 1.0]
    assert np.array_equal(res["theta"], th)


def test_accept_divides_lambda_by_three():
    sc, o, xy, th, target = _descent()
    res = o.lm_step(th, xy, target, 0.1)
    assert res["accepted"] and res["best_trial"] == 0
    assert res["loss_after"] < res["loss_before"]
    assert res["lambda_next"] == 0.1 / 3.0
    assert np.array_equal(res["theta"], res["theta_trial"])


def test_several_trials_take_the_lowest_loss():
    """The multi-trial step equals the single-trial step of the trial with the
    lowest loss; each single-trial loss is computed on its own."""
    sc, o, xy, th, target = _descent(seed=24)
    lams = [1.0, 1e-1, 1e-2, 1e-3]
    single = [o.lm_step(th, xy, target, lt) for lt in lams]
    losses = [s["loss_after"] for s in single]
    res = o.lm_step(th, xy, target, lams)
    k = int(np.argmin(losses))
    assert res["trial_losses"] == losses
    assert res["best_trial"] == k and res["accepted"]
    assert res["loss_after"] == losses[k]
    assert res["lambda_next"] == lams[k] / 3.0
    assert np.array_equal(res["theta"], single[k]["theta"])
    # the largest damping takes the shortest step; with a nearly quadratic
    # model it is not the best of these
    assert k != 0


def _one_handle_oracle():
    return oracle.Oracle.segments(1, [0.5, 0.5, 0.5], segs_per_side=4)


def _indefinite_H():
    """10 x 10, unit diagonal, one 2 x 2 block [[1, 2.5], [2.5, 1]] on x_a, y_a:
    H + lam diag(H) is positive definite exactly when lam > 1.5."""
    H = np.eye(10)
    H[0, 1] = H[1, 0] = 2.5
    return H


@pytest.mark.parametrize("lam0,want", [(1e-3, 1e-3 * 10 ** 4), (0.0, 1e-9 * 10 ** 10),
                                       (2.0, 2.0)])
def test_retry_raises_lambda_tenfold(lam0, want):
    o = _one_handle_oracle()
    th = np.array([0.3, 0.3, 0.6, 0.5, 0.1, 0.2, 0.3, 0.0, 0.0, 0.0])
    g = np.linspace(-1.0, 1.0, 10)
    delta = o.solve_step(th, _indefinite_H(), g, lam0)
    assert o.last_lambda == pytest.approx(want, rel=1e-12)
    assert np.all(np.isfinite(delta))
    # the step solves the damped system at the raised lambda on the
    # compatibility subspace: (H + lam D) delta + Ac mu = -g with Ac^T delta = 0
    lam = o.last_lambda
    K = _indefinite_H() + lam * np.eye(10)
    Ac = o.constraint_matrix(th)
    r = K @ delta + g
    mu, *_ = np.linalg.lstsq(Ac, -r, rcond=None)
    assert np.abs(r + Ac @ mu).max() < 1e-12 * (1 + np.abs(g).max())
    assert np.abs(Ac.T @ delta).max() < 1e-13


def test_retry_gives_up_after_twelve_raises():
    o = _one_handle_oracle()
    th = np.array([0.3, 0.3, 0.6, 0.5, 0.1, 0.2, 0.3, 0.0, 0.0, 0.0])
    H = np.eye(10)
    H[0, 1] = H[1, 0] = 1e16          # needs lam > 1e16: beyond 1e-3 * 10^12
    with pytest.raises(np.linalg.LinAlgError):
        o.solve_step(th, H, np.ones(10), 1e-3)
    assert o.last_lambda == pytest.approx(1e-3 * 10.0 ** 12, rel=1e-12)
    assert math.isfinite(o.last_lambda)
