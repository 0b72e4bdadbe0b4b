"""Sec. 4.4 regularisers and pruning of segment handles: CUDA path vs the
FP64 oracle (GPU only).  FP64 LM steps agree to <= 1e-9 relative, the mixed
step's loss and gradient norm to the mixed-path bounds."""
import numpy as np
import pytest

import gen
import oracle
from oracle import regularize as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 40
REG = dict(len_weight=5.0, len_max=0.06, snap_weight=2.0, snap_radius=0.03, snap_alpha=0.5,
           sparse_wd=2e-3, sparse_wc=1e-3, sparse_eps=1e-3, sparse_t=0.05)


def _bg():
    import paper_2602_05492_gb300 as bg
    return bg


@pytest.fixture(scope="module")
def scene():
    sc = gen.make_segment_scene("seg500", H=H, W=48, spp=4, seed=91)
    th = sc.theta_init.reshape(H, 10).copy()
    # a few endpoints put near others (some collinear, some not) so that
    # snapping pairs exist, and two long handles for the length penalty
    def move(h, s, to):                      # translate handle h so endpoint s lands at `to`
        d = np.asarray(to) - th[h, 2 * s:2 * s + 2]
        th[h, 0:2] += d
        th[h, 2:4] += d

    move(1, 0, th[0, 2:4] + (0.004, 0.002))
    move(3, 1, th[2, 2:4] + (-0.006, 0.003))
    move(5, 0, th[4, 0:2] + (0.01, -0.01))
    th[6, 2:4] = th[6, 0:2] + (0.09, 0.03)
    th[7, 2:4] = th[7, 0:2] + (-0.02, 0.08)
    th[:, 0:4] = np.clip(th[:, 0:4], 0.02, 0.98)
    o = oracle.Oracle.segments(H, sc.mean_true, segs_per_side=48)
    theta = oracle.project_compat(o.geo, th.reshape(-1))
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)
    truth = o.eval(oracle.project_compat(o.geo, sc.theta_true), xy)
    target = gen.add_noise(truth, sc.noise, sc.seed)
    mean = np.minimum(target, 1.0).mean(0)
    o.mean = mean
    return theta, xy, target, mean, o


def _ctx(theta, mean, prec, **kw):
    m = _bg().BEM(precision=prec, segs_per_side=48, **kw)
    m.setup_segments(H, theta, mean)
    m.factor()
    return m


def _t(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")


def test_layout_exercises_every_term(scene):
    theta, *_ = scene
    rp = R.RegParams(**REG)
    assert len(R.snap_pairs(theta, rp)) >= 2
    th = theta.reshape(H, 10)
    assert (np.hypot(th[:, 2] - th[:, 0], th[:, 3] - th[:, 1]) > rp.len_max).sum() >= 2


@pytest.mark.parametrize("lam,tol", [(1e-1, 1e-9), (1e-2, 1e-9), (1e-5, 1e-6)])
def test_reg_lm_step_fp64(scene, lam, tol):
    """At the smallest damping the damped matrix is ill-conditioned and two
    correct double solvers agree to about cond * eps only."""
    theta, xy, target, mean, o = scene
    sub, tsub = xy[::4], target[::4]
    m = _ctx(theta, mean, _bg().BEM_FP64)
    m.set_regularizers(**REG)
    res = m.lm_step(_t(sub, torch.float64), _t(tsub, torch.float64), [lam])
    want = o.lm_step(theta, sub, tsub, lam, reg=R.RegParams(**REG))
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-11)
    assert res["grad_norm"] == pytest.approx(np.linalg.norm(want["g"]), rel=1e-10)
    assert res["accepted"] == want["accepted"]
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=tol)
    th = m.get_params()
    ref = want["theta"]
    assert np.abs(th - ref).max() <= tol * np.abs(ref).max()


def test_reg_lm_step_mixed(scene):
    bg = _bg()
    theta, xy, target, mean, o = scene
    sub, tsub = xy[::4], target[::4]
    m = _ctx(theta, mean, bg.BEM_MIXED, jtj_mode=bg.BEM_JTJ_3XTF32)
    m.set_regularizers(**REG)
    res = m.lm_step(_t(sub, torch.float32), _t(tsub, torch.float32), [1e-2])
    want = o.lm_step(theta, sub, tsub, 1e-2, reg=R.RegParams(**REG))
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-5)
    assert res["grad_norm"] == pytest.approx(np.linalg.norm(want["g"]), rel=1e-4)
    assert res["accepted"] == want["accepted"]
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=1e-4)


def test_reg_off_is_plain_step(scene):
    """Clearing the regularisers gives back the unregularised step."""
    theta, xy, target, mean, o = scene
    sub, tsub = xy[::4], target[::4]
    m = _ctx(theta, mean, _bg().BEM_FP64)
    m.set_regularizers(**REG)
    m.set_regularizers()
    res = m.lm_step(_t(sub, torch.float64), _t(tsub, torch.float64), [1e-2])
    want = o.lm_step(theta, sub, tsub, 1e-2)
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-11)
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=1e-9)


def test_prune_matches_oracle(scene):
    theta, xy, target, mean, o = scene
    th = theta.reshape(H, 10).copy()
    th[8, 4:10] = 1e-4                       # both jumps small: pruned
    th[9, 4:7] = 1e-4                        # w_c still large: kept
    th[11, 4:10] = 0.0
    theta = th.reshape(-1)
    m = _ctx(theta, mean, _bg().BEM_FP64)
    thr = 0.05
    kept = m.prune(thr)
    want, keep = R.prune(theta, thr)
    np.testing.assert_array_equal(kept, keep)
    assert m.n_theta == want.size
    got = m.get_params()
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # the pruned scene evaluates like the oracle's scene of the kept handles
    ok = oracle.Oracle.segments(keep.size, mean, segs_per_side=48)
    u = m.eval(_t(xy[:2000], torch.float64)).cpu().numpy()
    v = ok.eval(want, xy[:2000])
    assert np.abs(u - v).max() <= 1e-10 * np.abs(v).max()
    # nothing left to remove: a no-op that reports every handle
    again = m.prune(thr)
    np.testing.assert_array_equal(again, np.arange(keep.size))
    # a threshold that would remove all: the scene stays
    assert m.prune(1e9).size == 0
    assert m.n_theta == want.size


def test_regularizer_errors(scene):
    bg = _bg()
    theta, xy, target, mean, o = scene
    m = _ctx(theta, mean, bg.BEM_FP64)
    for bad in (dict(len_weight=-1.0), dict(snap_weight=1.0, snap_radius=0.0),
                dict(snap_weight=1.0, snap_alpha=1.5), dict(sparse_wd=1.0, sparse_t=0.0),
                dict(len_weight=float("nan"))):
        with pytest.raises(bg.BemError):
            m.set_regularizers(**bad)
    sc = gen.make_scene(1)
    c = bg.BEM(precision=bg.BEM_FP64, segs_per_side=16)
    c.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
    with pytest.raises(bg.BemError):
        c.set_regularizers(len_weight=1.0)
    c.factor()
    with pytest.raises(bg.BemError):
        c.prune(0.1)
