"""The paper's handle parametrisation in the oracle: independent straight
segments of 10 parameters (a, b, w_d RGB, w_c RGB), Sec. 4.2.

Pinned to the (separately pinned) Bezier path: a segment is the one-panel
cubic curve with control points a, (2a+b)/3, (a+2b)/3, b and four equal
colour sets, so colours agree and the segment Jacobian is the chain-ruled
curve Jacobian; central differences check the Jacobian directly."""
import numpy as np

import oracle


def _segments(H, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.15, 0.85, size=(H, 2))
    ang = rng.uniform(0, 2 * np.pi, size=H)
    b = np.clip(a + 0.12 * np.stack([np.cos(ang), np.sin(ang)], 1), 0.05, 0.95)
    th = np.zeros((H, 10))
    th[:, 0:2], th[:, 2:4] = a, b
    th[:, 4:7] = rng.uniform(-0.8, 0.8, size=(H, 3))
    th[:, 7:10] = rng.uniform(-0.5, 0.5, size=(H, 3))
    return th


def _as_curves(th):
    H = th.shape[0]
    cb = np.zeros((H, 4, 8))
    a, b = th[:, 0:2], th[:, 2:4]
    for j, t in enumerate((0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0)):
        cb[:, j, 0:2] = (1 - t) * a + t * b
        cb[:, j, 2:8] = th[:, 4:10]
    return cb.reshape(-1)


def test_segments_match_straight_curves():
    H = 5
    th = _segments(H, 1)
    mean = np.array([0.4, 0.5, 0.6])
    os_ = oracle.Oracle.segments(H, mean, segs_per_side=16)
    oc = oracle.Oracle(H, [1] * H, [0] * H, mean, segs_per_side=16)
    pts = np.random.default_rng(2).uniform(0.02, 0.98, size=(300, 2))
    ts, tc = th.reshape(-1), _as_curves(th)
    np.testing.assert_allclose(os_.eval(ts, pts), oc.eval(tc, pts), rtol=0, atol=1e-13)
    Js, Jc = os_.jac(ts, pts[:40]), oc.jac(tc, pts[:40])
    Jc = Jc.reshape(40, 3, H, 4, 8)
    want = np.zeros((40, 3, H, 10))
    want[..., 0:2] = Jc[:, :, :, 0, 0:2]          # a = p0 (the panel's start)
    want[..., 2:4] = Jc[:, :, :, 3, 0:2]          # b = p3 (its end)
    want[..., 4:10] = Jc[:, :, :, :, 2:8].sum(3)  # one colour set = all four
    np.testing.assert_allclose(Js.reshape(40, 3, H, 10), want, rtol=0,
                               atol=1e-12 * np.abs(want).max())
    # the inner control points of a one-panel curve have no effect
    assert np.abs(Jc[:, :, :, 1:3, 0:2]).max() == 0.0


def test_segment_jacobian_fd():
    H = 3
    th = _segments(H, 3).reshape(-1)
    o = oracle.Oracle.segments(H, np.zeros(3), segs_per_side=16)
    pts = np.array([[0.3, 0.4], [0.7, 0.2], [0.5, 0.8]])
    J = o.jac(th, pts)
    h = 1e-6
    for t in range(th.size):
        e = np.zeros_like(th)
        e[t] = h
        fd = (o.eval(th + e, pts) - o.eval(th - e, pts)) / (2 * h)
        np.testing.assert_allclose(J[:, :, t], fd, rtol=1e-5, atol=1e-7)


def test_segment_lm_step_keeps_compatibility():
    H = 4
    th = _segments(H, 4).reshape(-1)
    o = oracle.Oracle.segments(H, np.array([0.5, 0.5, 0.5]), segs_per_side=16)
    th = oracle.project_compat(o.geo, th)
    pts = np.random.default_rng(5).uniform(0.02, 0.98, size=(400, 2))
    tgt = o.eval(th + 0.01, pts)
    res = o.lm_step(th, pts, tgt, 1e-3)
    a = oracle.compat_vectors(o.geo, res["theta_trial"])
    wc = res["theta_trial"].reshape(H, 10)[:, 7:10]
    assert np.abs(a @ wc).max() < 1e-13
