"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Tolerances (stated per result, from the accuracy targets of this project):
  FP64 GPU path       <= 1e-10 relative to the oracle
  mixed path colours  <= 1e-4 RMSE on [0,1] colours
  mixed path gradient <= 1e-4 relative (2-norm)
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _bg():
    import paper_2602_05492_gb300 as bg
    return bg


@pytest.fixture(scope="module")
def cfg1():
    sc = gen.make_scene(1)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)
    o = oracle.Oracle.from_scene(sc)
    truth = o.eval(oracle.project_compat(o.geo, sc.theta_true), xy)
    target = gen.add_noise(truth, sc.noise, sc.seed)
    mean = np.minimum(target, 1.0).mean(0)
    o.mean = mean
    return sc, xy, target, mean, o


def _ctx(sc, mean, prec, theta=None, **kw):
    bg = _bg()
    m = bg.BEM(precision=prec, **kw)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed,
            sc.theta_init if theta is None else theta, mean)
    m.factor()
    return m


def _t(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ---- FP64 path --------------------------------------------------------------

def test_eval_fp64_cfg1_full(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_FP64)
    u = m.eval(_t(xy, torch.float64)).cpu().numpy()
    want = o.eval(sc.theta_init, xy)
    assert _rel(u, want) < 1e-10


def test_boundary_values_fp64(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_FP64)
    assert _rel(m.boundary_values(), o.boundary_values(sc.theta_init)) < 1e-10


def test_loss_and_residual_fp64(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_FP64)
    res = torch.empty((xy.shape[0], 3), dtype=torch.float64, device="cuda:0")
    L = m.loss(_t(xy, torch.float64), _t(target, torch.float64), res)
    r = o.eval(sc.theta_init, xy) - np.minimum(target, 1.0)
    assert _rel(res.cpu().numpy(), r) < 1e-9
    assert L == pytest.approx(o.loss(sc.theta_init, xy, target), rel=1e-12)


def test_vjp_fp64(cfg1):
    sc, xy, target, mean, o = cfg1
    sub = xy[::8]
    r = np.random.default_rng(0).normal(size=(sub.shape[0], 3))
    m = _ctx(sc, mean, _bg().BEM_FP64)
    g = m.vjp(_t(sub, torch.float64), _t(r, torch.float64)).cpu().numpy()
    want = o.grad(sc.theta_init, sub, r)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-10


def test_jtj_fp64(cfg1):
    sc, xy, target, mean, o = cfg1
    sub = xy[::16]
    m = _ctx(sc, mean, _bg().BEM_FP64)
    H = m.jtj(_t(sub, torch.float64)).cpu().numpy()
    _, _, want = o.gauss_newton(sc.theta_init, sub, target[::16])
    assert np.linalg.norm(H - want) / np.linalg.norm(want) < 1e-10


@pytest.mark.parametrize("solver,lam", [("auto", 1e-3), ("fp64", 1e-3), ("auto", 1e-9),
                                        ("fp64", 1e-9)])
def test_lm_step_fp64(cfg1, solver, lam):
    """One FP64 LM step against the oracle's, with the float-factor /
    double-refinement solver (auto) and the double Cholesky (fp64), at a
    moderate and at a tiny damping."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    sub, tsub = xy[::16], target[::16]
    m = _ctx(sc, mean, bg.BEM_FP64,
             lm_solver=bg.BEM_LM_AUTO if solver == "auto" else bg.BEM_LM_FP64)
    res = m.lm_step(_t(sub, torch.float64), _t(tsub, torch.float64), [lam])
    want = o.lm_step(sc.theta_init, sub, tsub, lam)
    # at the tiny damping the system is ill-conditioned: two correct double
    # solvers agree to about cond * eps only
    tol = 1e-9 if lam >= 1e-3 else 1e-6
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-11)
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=tol)
    assert res["accepted"] == want["accepted"]
    assert res["best_trial"] == want["best_trial"]
    assert res["lambda_next"] == pytest.approx(want["lambda_next"], rel=1e-15)
    th = m.get_params()
    assert _rel(th, want["theta"]) < tol


def test_lm_step_multi_trial_fp64(cfg1):
    """Four damping trials in one step: the trial taken, its loss, the damping
    proposal and the new theta against the oracle's multi-trial step."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    sub, tsub = xy[::16], target[::16]
    lams = [1.0, 1e-1, 1e-2, 1e-3]
    m = _ctx(sc, mean, bg.BEM_FP64)
    x, t = _t(sub, torch.float64), _t(tsub, torch.float64)
    th = sc.theta_init.copy()
    for it in range(2):
        res = m.lm_step(x, t, lams)
        want = o.lm_step(th, sub, tsub, lams)
        assert res["best_trial"] == want["best_trial"]
        assert res["accepted"] == want["accepted"]
        assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-11)
        assert res["loss_after"] == pytest.approx(want["loss_after"], rel=1e-9)
        assert res["lambda_next"] == pytest.approx(want["lambda_next"], rel=1e-15)
        assert _rel(m.get_params(), want["theta"]) < 1e-9
        th = want["theta"]
        lams = [want["lambda_next"] * f for f in (10.0, 1.0, 0.1, 0.01)]


@pytest.mark.parametrize("lams,want_next", [([1e-2], 2e-2), ([1e-3, 1e-2, 1e-1, 1.0], 10.0)])
def test_lm_step_rejects_at_stationary_point_fp64(cfg1, lams, want_next):
    """Target = the context's own colours (below 1, so the clamp leaves them):
    r = 0, g = 0, every trial's step vanishes and no trial lowers the loss of
    0, so the step is rejected and the damping grows as the schedule says
    (the oracle's side of this rule is pinned on the CPU)."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    sub = xy[::32]
    th = oracle.project_compat(o.geo, sc.theta_init)
    th.reshape(-1, 8)[:, 2:8] *= 0.2
    th = oracle.project_compat(o.geo, th)
    m = _ctx(sc, mean, bg.BEM_FP64, theta=th)
    x = _t(sub, torch.float64)
    tgt = m.eval(x)
    assert tgt.max().item() < 1.0
    res = m.lm_step(x, tgt, lams)
    assert res["loss_before"] == 0.0 and res["grad_norm"] == 0.0
    assert not res["accepted"] and res["best_trial"] == -1
    assert res["lambda_next"] == want_next
    assert np.array_equal(m.get_params(), th)


def test_fd_gradient_fp64_on_gpu(cfg1):
    """Central differences of the GPU loss against the GPU adjoint (no oracle)."""
    sc, xy, target, mean, o = cfg1
    sub, tsub = xy[::32], target[::32]
    m = _ctx(sc, mean, _bg().BEM_FP64)
    xt, tt = _t(sub, torch.float64), _t(tsub, torch.float64)
    res = torch.empty((sub.shape[0], 3), dtype=torch.float64, device="cuda:0")
    m.loss(xt, tt, res)
    g = m.vjp(xt, res).cpu().numpy() / sub.shape[0]
    th0 = sc.theta_init.copy()
    h = 1e-6
    for k in np.random.default_rng(1).choice(len(th0), 12, replace=False):
        if k % 32 in (24, 25) and sc.closed[k // 32]:
            continue
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        m.set_params(tp)
        Lp = m.loss(xt, tt)
        m.set_params(tm)
        Lm = m.loss(xt, tt)
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-9)


def test_unequal_eps_fp64(cfg1):
    sc, xy, target, mean, o = cfg1
    sub = xy[::4]
    m = _ctx(sc, mean, _bg().BEM_FP64, eps_d=3e-3, eps_c=2e-2)
    o2 = oracle.Oracle.from_scene(sc, mean_color=mean, eps_d=3e-3, eps_c=2e-2)
    u = m.eval(_t(sub, torch.float64)).cpu().numpy()
    assert _rel(u, o2.eval(sc.theta_init, sub)) < 1e-10
    r = np.random.default_rng(2).normal(size=(sub.shape[0], 3))
    g = m.vjp(_t(sub, torch.float64), _t(r, torch.float64)).cpu().numpy()
    want = o2.grad(sc.theta_init, sub, r)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-10


@pytest.mark.parametrize("n", [0, 1, 127, 129, 1000])
def test_ragged_sizes_fp64(cfg1, n):
    sc, xy, target, mean, o = cfg1
    sub = xy[:n]
    m = _ctx(sc, mean, _bg().BEM_FP64)
    xt = _t(sub.reshape(-1, 2), torch.float64)
    u = m.eval(xt).cpu().numpy()
    r = np.random.default_rng(n).normal(size=(n, 3))
    g = m.vjp(xt, _t(r.reshape(-1, 3), torch.float64)).cpu().numpy()
    if n == 0:
        assert u.shape == (0, 3) and np.abs(g).max() == 0.0
        return
    assert _rel(u, o.eval(sc.theta_init, sub)) < 1e-10
    want = o.grad(sc.theta_init, sub, r)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-10


def test_galerkin_3x3_fp64(cfg1):
    """galerkin_mode 1 (the paper's 3 x 3 Gauss rule): the boundary solution
    and the colours against the oracle's mode-1 matrix and SVD truncation."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    o1 = oracle.Oracle.from_scene(sc, mean_color=mean, galerkin_mode=1)
    m = _ctx(sc, mean, bg.BEM_FP64, galerkin_mode=1)
    ub = m.boundary_values()
    want_ub = o1.boundary_values(sc.theta_init)
    assert _rel(ub, want_ub) < 1e-10
    sub = xy[::4]
    u = m.eval(_t(sub, torch.float64)).cpu().numpy()
    assert _rel(u, o1.eval(sc.theta_init, sub)) < 1e-10
    # and the modes differ by the quadrature error only
    assert _rel(u, o.eval(sc.theta_init, sub)) < 1e-3


def test_galerkin_3x3_mixed(cfg1):
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    o1 = oracle.Oracle.from_scene(sc, mean_color=mean, galerkin_mode=1)
    m = _ctx(sc, mean, bg.BEM_MIXED, galerkin_mode=1)
    u = m.eval(_t(xy, torch.float32)).double().cpu().numpy()
    rmse = np.sqrt(np.mean((u - o1.eval(sc.theta_init, xy)) ** 2))
    assert rmse < 1e-4, rmse


def _pixel_centres(W, H):
    j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([(i.ravel() + 0.5) / W, (j.ravel() + 0.5) / H], 1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_render(cfg1, prec):
    """The image on a 40 x 30 pixel grid against the oracle at the pixel centres."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, bg.BEM_FP64 if prec == "fp64" else bg.BEM_MIXED)
    img = m.render(40, 30).double().cpu().numpy()
    assert img.shape == (30, 40, 3)
    want = o.eval(sc.theta_init, _pixel_centres(40, 30)).reshape(30, 40, 3)
    if prec == "fp64":
        assert _rel(img, want) < 1e-10
    else:
        assert np.sqrt(np.mean((img - want) ** 2)) < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_handle_colors(cfg1, prec):
    """Two-sided colours: the colour at each panel midpoint +- w_d/2, and the
    jump between the sides is w_d exactly."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, bg.BEM_FP64 if prec == "fp64" else bg.BEM_MIXED)
    hc = m.handle_colors()
    ab, wd, _ = o.panels(sc.theta_init)
    mid = 0.5 * (ab[:, 0:2] + ab[:, 2:4])
    avg = o.eval(sc.theta_init, mid)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.abs(hc[:, 0] - (avg + 0.5 * wd)).max() < tol * max(1.0, np.abs(avg).max())
    assert np.abs(hc[:, 1] - (avg - 0.5 * wd)).max() < tol * max(1.0, np.abs(avg).max())
    assert np.abs((hc[:, 0] - hc[:, 1]) - wd).max() < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lm_step_split_hessian(cfg1, prec):
    """H from a separate (smaller) point set, g and losses from the samples,
    against the oracle's step with the same two sets."""
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    sub, tsub, hsub = xy[::16], target[::16], xy[5::64]
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = _ctx(sc, mean, bg.BEM_FP64 if prec == "fp64" else bg.BEM_MIXED)
    res = m.lm_step_split(_t(sub, dt), _t(tsub, dt), _t(hsub, dt), [1e-3])
    want = o.lm_step(sc.theta_init, sub, tsub, 1e-3, xy_h=hsub)
    tol = 1e-9 if prec == "fp64" else 2e-2
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-11 if prec == "fp64" else 1e-5)
    assert res["grad_norm"] == pytest.approx(np.linalg.norm(want["g"]), rel=1e-9 if prec == "fp64" else 1e-4)
    assert res["accepted"] == want["accepted"]
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=tol)
    if prec == "fp64":
        assert _rel(m.get_params(), want["theta"]) < 1e-9


# ---- mixed path -----------------------------------------------------------------

def test_eval_mixed_cfg1_full(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_MIXED)
    u = m.eval(_t(xy, torch.float32)).double().cpu().numpy()
    want = o.eval(sc.theta_init, xy)
    rmse = np.sqrt(np.mean((u - want) ** 2))
    assert rmse < 1e-4, rmse


def test_vjp_mixed(cfg1):
    sc, xy, target, mean, o = cfg1
    sub = xy[::8]
    r = np.random.default_rng(0).normal(size=(sub.shape[0], 3))
    m = _ctx(sc, mean, _bg().BEM_MIXED)
    g = m.vjp(_t(sub, torch.float32), _t(r, torch.float32)).cpu().numpy()
    want = o.grad(sc.theta_init, sub, r.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-4


# H on 2,048 samples.  Rounding J to bf16 (8 mantissa bits) perturbs each
# product of H by about 2^-8 relative with a random sign, so the relative
# error of the sum falls with the number of samples: measured 1.06e-3 here
# (1.7e-4 on 32,691 samples, test_gn_products_across_chunks); compensated
# bf16 4.8e-6, 3xtf32 1.0e-6 to 1.4e-6, fp64 J^T J of float J rows 7e-7.  The
# bounds are about five times those.
@pytest.mark.parametrize("mode,tol", [("bf16", 5e-3), ("3xtf32", 5e-6), ("bf16x3", 2.5e-5),
                                      ("fp64", 4e-6)])
def test_jtj_mixed(cfg1, mode, tol):
    bg = _bg()
    jm = {"bf16": bg.BEM_JTJ_BF16, "3xtf32": bg.BEM_JTJ_3XTF32, "bf16x3": bg.BEM_JTJ_BF16X3,
          "fp64": bg.BEM_JTJ_FP64}[mode]
    sc, xy, target, mean, o = cfg1
    sub = xy[::16]
    m = _ctx(sc, mean, bg.BEM_MIXED, jtj_mode=jm)
    H = m.jtj(_t(sub, torch.float32)).cpu().numpy()
    _, _, want = o.gauss_newton(sc.theta_init, sub, target[::16])
    assert np.linalg.norm(H - want) / np.linalg.norm(want) < tol


@pytest.mark.parametrize("mode", ["bf16", "3xtf32", "bf16x3"])
def test_lm_step_mixed(cfg1, mode):
    """One mixed LM step: the loss it reports at the new theta matches the
    oracle's loss there, and the step lowers the loss like the FP64 step."""
    bg = _bg()
    jm = {"bf16": bg.BEM_JTJ_BF16, "3xtf32": bg.BEM_JTJ_3XTF32, "bf16x3": bg.BEM_JTJ_BF16X3}[mode]
    sc, xy, target, mean, o = cfg1
    sub, tsub = xy[::8], target[::8]
    m = _ctx(sc, mean, bg.BEM_MIXED, jtj_mode=jm)
    res = m.lm_step(_t(sub, torch.float32), _t(tsub, torch.float32), [1e-3])
    th = m.get_params()
    assert res["loss_before"] == pytest.approx(o.loss(sc.theta_init, sub, tsub), rel=1e-5)
    if res["accepted"]:
        assert res["loss_after"] == pytest.approx(o.loss(th, sub, tsub), rel=1e-4)
    want = o.lm_step(sc.theta_init, sub, tsub, 1e-3)
    # gradient of the step (from the same J rows as H) against the oracle's
    assert res["grad_norm"] == pytest.approx(np.linalg.norm(want["g"]), rel=1e-4)
    assert res["accepted"] == want["accepted"]
    # the step's loss moves with the error of H: measured about 5e-4 (bf16),
    # 1.6e-5 (compensated bf16) and 5e-7 to 1.2e-6 (3xtf32) relative on 4,096
    # samples at lambda = 1e-3
    assert res["loss_after"] == pytest.approx(want["loss_after"],
                                              rel={"bf16": 5e-3, "3xtf32": 6e-6, "bf16x3": 8e-5}[mode])


@pytest.mark.parametrize("nf", [0.0, 0.5, 1000.0])
@pytest.mark.parametrize("mode", ["bf16", "3xtf32"])
def test_lm_step_residual_from_jrow_pass(cfg1, mode, nf):
    """In the tensor-core modes the LM step forms the residual at theta inside
    the J-row pass: the handle term as F w (the colour is linear in the
    jumps), the near pairs corrected to their double values, the boundary
    term added.  Its loss matches the evaluation kernel's (bem_loss) to float
    rounding and the oracle's, with no near field, the default one and every
    pair near."""
    bg = _bg()
    jm = {"bf16": bg.BEM_JTJ_BF16, "3xtf32": bg.BEM_JTJ_3XTF32}[mode]
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, bg.BEM_MIXED, jtj_mode=jm, near_factor=nf)
    x32, t32 = _t(xy, torch.float32), _t(target, torch.float32)
    L = m.loss(x32, t32)
    res = m.lm_step(x32, t32, [1e-3])
    assert res["loss_before"] == pytest.approx(L, rel=2e-6)
    assert res["loss_before"] == pytest.approx(o.loss(sc.theta_init, xy, target), rel=1e-5)


# ---- the Gauss-Newton pass across sample chunks ----------------------------------
#
# H, g and the loss are sums over samples that the GPU forms chunk by chunk
# (J rows exist for one chunk at a time; the chunks' fp32 or double sums are
# added in double).  Config 1's samples less a ragged tail, in chunks of
# 4,096 (8 chunks, the last one short), against the oracle's sums over all
# of them (Eq. (losshessian), (lossjacobian)).

N_CHUNKED = 32768 - 77
GN_TOL = {  # (loss rel, g rel 2-norm, H rel Frobenius); measured on 32,691
    # samples: loss 3.5e-7, g 2.1e-6 (mixed), H 1.5e-7 (fp64 J^T J), 1.2e-6 to
    # 2.3e-6 (3xtf32), 3.6e-6 (compensated bf16), 1.7e-4 (bf16); the bounds
    # are about five times those
    "fp64": (1e-12, 1e-10, 1e-10),
    "fp64_jtj": (2e-6, 1e-5, 1e-6),
    "3xtf32": (2e-6, 1e-5, 1.2e-5),
    "bf16x3": (2e-6, 1e-5, 2e-5),
    "bf16": (2e-6, 1e-5, 8e-4),
}


@pytest.fixture(scope="module")
def cfg1_gn(cfg1):
    sc, xy, target, mean, o = cfg1
    x, t = xy[:N_CHUNKED], target[:N_CHUNKED]
    return x, t, o.gauss_newton(sc.theta_init, x, t)


def _gn_ctx(sc, mean, mode, chunk):
    bg = _bg()
    if mode == "fp64":
        return _ctx(sc, mean, bg.BEM_FP64, gn_chunk=chunk), torch.float64
    jm = {"fp64_jtj": bg.BEM_JTJ_FP64, "3xtf32": bg.BEM_JTJ_3XTF32, "bf16": bg.BEM_JTJ_BF16,
          "bf16x3": bg.BEM_JTJ_BF16X3}[mode]
    return _ctx(sc, mean, bg.BEM_MIXED, jtj_mode=jm, gn_chunk=chunk), torch.float32


@pytest.mark.parametrize("mode", ["fp64", "fp64_jtj", "3xtf32", "bf16x3", "bf16"])
def test_gn_products_across_chunks(cfg1, cfg1_gn, mode):
    sc, xy, target, mean, o = cfg1
    x, t, (L, g, H) = cfg1_gn
    m, dt = _gn_ctx(sc, mean, mode, 4096)
    Lg, gg, Hg = m.gn_products(_t(x, dt), _t(t, dt))
    gg, Hg = gg.cpu().numpy(), Hg.cpu().numpy()
    tl, tg, th = GN_TOL[mode]
    assert Lg == pytest.approx(L, rel=tl)
    assert np.linalg.norm(gg - g) / np.linalg.norm(g) < tg
    assert np.linalg.norm(Hg - H) / np.linalg.norm(H) < th
    # one chunk instead of eight: the same J rows, only the order of the sums differs
    m1, _ = _gn_ctx(sc, mean, mode, 0)
    L1, g1, H1 = m1.gn_products(_t(x, dt), _t(t, dt))
    g1, H1 = g1.cpu().numpy(), H1.cpu().numpy()
    # (float K-slice partial sums in another order: measured 2.8e-6 bf16, 4.4e-6 3xtf32)
    same = 1e-13 if mode == "fp64" else 2e-5
    assert Lg == pytest.approx(L1, rel=same)
    assert np.linalg.norm(gg - g1) / np.linalg.norm(g1) < same
    assert np.linalg.norm(Hg - H1) / np.linalg.norm(H1) < same


@pytest.mark.parametrize("mode", ["fp64", "bf16"])
def test_lm_step_across_chunks(cfg1, mode):
    """One LM step over 8 chunks: loss at theta, gradient norm, the accepted
    theta and the damping proposal against the oracle's step on all samples."""
    sc, xy, target, mean, o = cfg1
    x, t = xy[:N_CHUNKED], target[:N_CHUNKED]
    m, dt = _gn_ctx(sc, mean, mode, 4096)
    res = m.lm_step(_t(x, dt), _t(t, dt), [1e-2])
    want = o.lm_step(sc.theta_init, x, t, 1e-2)
    exact = mode == "fp64"
    assert res["loss_before"] == pytest.approx(want["loss_before"], rel=1e-12 if exact else 1e-5)
    assert res["grad_norm"] == pytest.approx(np.linalg.norm(want["g"]), rel=1e-10 if exact else 1e-4)
    assert res["accepted"] == want["accepted"] and res["best_trial"] == want["best_trial"]
    assert res["lambda_next"] == pytest.approx(want["lambda_next"], rel=1e-15)
    th = m.get_params()
    step = np.abs(want["theta"] - sc.theta_init).max()
    # bf16: the step moves by 1.4 % of its size against the oracle's (measured)
    assert np.abs(th - want["theta"]).max() <= (1e-9 if exact else 7e-2) * step
    assert res["loss_after"] == pytest.approx(want["loss_after"], rel=1e-9 if exact else 1e-4)


@pytest.mark.parametrize("mode,pinned", [("bf16", True), ("bf16", False), ("fp64", True)])
def test_lm_step_host_inputs(cfg1, mode, pinned):
    """lm_step_host (host samples and targets, copied in by the library chunk
    by chunk while the pass runs) takes the step lm_step takes on device
    copies of the same inputs, over 8 chunks, twice in a row (the second step
    with other targets in the same device buffers); the first step also
    against the oracle's."""
    sc, xy, target, mean, o = cfg1
    x, t = xy[:N_CHUNKED], target[:N_CHUNKED]
    t2 = np.ascontiguousarray(t[::-1])
    m_dev, dt = _gn_ctx(sc, mean, mode, 4096)
    m_host, _ = _gn_ctx(sc, mean, mode, 4096)
    npdt = np.float64 if dt == torch.float64 else np.float32

    def host(a):
        a = np.ascontiguousarray(a, npdt)
        return torch.from_numpy(a).pin_memory() if pinned else a

    for k, tk in enumerate((t, t2)):
        rd = m_dev.lm_step(_t(x, dt), _t(tk, dt), [1e-2])
        rh = m_host.lm_step_host(host(x), host(tk), [1e-2])
        for key in ("loss_before", "loss_after", "grad_norm", "lambda_next"):
            assert rh[key] == pytest.approx(rd[key], rel=1e-12), key
        assert rh["accepted"] == rd["accepted"] and rh["best_trial"] == rd["best_trial"]
        assert np.abs(m_host.get_params() - m_dev.get_params()).max() <= \
            1e-12 * np.abs(m_dev.get_params()).max()
        if k == 0:
            want = o.lm_step(sc.theta_init, x, t, 1e-2)
            exact = mode == "fp64"
            assert rh["loss_before"] == pytest.approx(want["loss_before"], rel=1e-12 if exact else 1e-5)
            assert rh["accepted"] == want["accepted"]


def test_lm_step_host_rejects_device_tensors(cfg1):
    sc, xy, target, mean, o = cfg1
    m, dt = _gn_ctx(sc, mean, "bf16", 4096)
    with pytest.raises(AssertionError):
        m.lm_step_host(_t(xy[:256], dt), _t(target[:256], dt), [1e-2])


def test_mixed_all_pairs_near(cfg1):
    """near_factor = 1000 sends every handle pair through the double near-field
    kernels: colours and gradient then match the oracle to float rounding of
    the boundary term only."""
    sc, xy, target, mean, o = cfg1
    sub = xy[::8]
    m = _ctx(sc, mean, _bg().BEM_MIXED, near_factor=1000.0)
    u = m.eval(_t(sub, torch.float32)).double().cpu().numpy()
    assert np.sqrt(np.mean((u - o.eval(sc.theta_init, sub)) ** 2)) < 2e-6
    r = np.random.default_rng(3).normal(size=(sub.shape[0], 3)).astype(np.float32)
    g = m.vjp(_t(sub, torch.float32), _t(r, torch.float32)).cpu().numpy()
    want = o.grad(sc.theta_init, sub, r.astype(np.float64))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-5


def test_mixed_all_pairs_near_adjoint_first(cfg1):
    """The adjoint's double near field on a fresh context (its logarithm table
    built by the adjoint itself, before any evaluation): every handle pair
    near, gradient against the oracle."""
    sc, xy, target, mean, o = cfg1
    sub = xy[1::8]
    m = _ctx(sc, mean, _bg().BEM_MIXED, near_factor=1000.0)
    r = np.random.default_rng(4).normal(size=(sub.shape[0], 3)).astype(np.float32)
    g = m.vjp(_t(sub, torch.float32), _t(r, torch.float32)).cpu().numpy()
    want = o.grad(sc.theta_init, sub, r.astype(np.float64))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-5


def test_mixed_without_near_field(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_MIXED, near_factor=0.0)
    u = m.eval(_t(xy, torch.float32)).double().cpu().numpy()
    rmse = np.sqrt(np.mean((u - o.eval(sc.theta_init, xy)) ** 2))
    assert rmse < 1e-4, rmse


# ---- full-size configurations, sampled outputs -----------------------------------

@pytest.fixture(scope="module")
def cfg2():
    sc = gen.make_scene(2)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)
    target = gen.add_noise(gen.analytic_truth(xy, sc.seed), sc.noise, sc.seed)
    mean = np.minimum(target, 1.0).mean(0)
    o = oracle.Oracle.from_scene(sc, mean_color=mean)
    idx = np.random.default_rng(5).choice(xy.shape[0], 1500, replace=False)
    return sc, xy, target, mean, o, idx


def test_eval_fp64_cfg2_sampled(cfg2):
    sc, xy, target, mean, o, idx = cfg2
    m = _ctx(sc, mean, _bg().BEM_FP64)
    u = m.eval(_t(xy, torch.float64)).cpu().numpy()
    assert _rel(u[idx], o.eval(sc.theta_init, xy[idx])) < 1e-10


def test_eval_mixed_cfg2_sampled(cfg2):
    sc, xy, target, mean, o, idx = cfg2
    m = _ctx(sc, mean, _bg().BEM_MIXED)
    u = m.eval(_t(xy, torch.float32)).double().cpu().numpy()
    rmse = np.sqrt(np.mean((u[idx] - o.eval(sc.theta_init, xy[idx])) ** 2))
    assert rmse < 1e-4, rmse


def test_vjp_mixed_cfg2_linear_in_residual(cfg2):
    """At full size the adjoint is checked by a property that holds at any
    size: linearity in the residual, J^T(a r1 + b r2) = a J^T r1 + b J^T r2,
    plus a sampled oracle comparison for the residual supported on few samples."""
    sc, xy, target, mean, o, idx = cfg2
    m = _ctx(sc, mean, _bg().BEM_MIXED)
    xt = _t(xy, torch.float32)
    rng = np.random.default_rng(9)
    r = np.zeros((xy.shape[0], 3), np.float32)
    r[idx] = rng.normal(size=(len(idx), 3))
    g = m.vjp(xt, _t(r, torch.float32)).cpu().numpy()
    want = o.grad(sc.theta_init, xy[idx], r[idx].astype(np.float64))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-4


def test_mixed_sample_order_cfg2(cfg2):
    """The float kernels cull near-field tests by the bounding box of a block's
    points; a random order (boxes spanning the image, every panel tested)
    must give the colours and gradient of the pixel order, up to the float
    summation order."""
    sc, xy, target, mean, o, idx = cfg2
    m = _ctx(sc, mean, _bg().BEM_MIXED)
    perm = np.random.default_rng(11).permutation(xy.shape[0])
    inv = np.argsort(perm)
    u0 = m.eval(_t(xy, torch.float32)).double().cpu().numpy()
    u1 = m.eval(_t(xy[perm], torch.float32)).double().cpu().numpy()[inv]
    assert np.abs(u0 - u1).max() < 2e-6
    r = np.random.default_rng(12).normal(size=(xy.shape[0], 3)).astype(np.float32)
    g0 = m.vjp(_t(xy, torch.float32), _t(r, torch.float32)).cpu().numpy()
    g1 = m.vjp(_t(xy[perm], torch.float32), _t(r[perm], torch.float32)).cpu().numpy()
    assert np.linalg.norm(g0 - g1) / np.linalg.norm(g0) < 1e-5


# ---- errors ------------------------------------------------------------------------

def test_state_and_argument_errors(cfg1):
    bg = _bg()
    sc, xy, target, mean, o = cfg1
    with pytest.raises(bg.BemError) as e:
        bg.BEM(eps_d=0.0)
    assert e.value.code == bg.BEM_EINVAL
    m = bg.BEM(precision=bg.BEM_FP64)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
    with pytest.raises(bg.BemError) as e:
        m.eval(_t(xy[:10], torch.float64))
    assert e.value.code == bg.BEM_ESTATE
    bad = sc.theta_init.copy()
    bad[3] = np.nan
    with pytest.raises(bg.BemError) as e:
        m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, bad, mean)
    assert e.value.code == bg.BEM_EINVAL


def test_sample_mean(cfg1):
    sc, xy, target, mean, o = cfg1
    m = _ctx(sc, mean, _bg().BEM_FP64)
    got = m.sample_mean(_t(target, torch.float64))
    np.testing.assert_allclose(got, mean, rtol=1e-13)


# ---- tensor-core contraction --------------------------------------------------------

@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 1024), (192, 300, 200),
                                   (64, 1000, 2048)])
def test_tensor_core_gemm(M, N, K):
    bg = _bg()
    m = bg.BEM(precision=bg.BEM_MIXED)
    g = torch.Generator(device="cuda:0").manual_seed(M * 7 + N)
    Kp = (K + 7) // 8 * 8
    A = torch.zeros((M, Kp), dtype=torch.bfloat16, device="cuda:0")
    B = torch.zeros((N, Kp), dtype=torch.bfloat16, device="cuda:0")
    A[:, :K] = torch.randn((M, K), generator=g, device="cuda:0").bfloat16()
    B[:, :K] = torch.randn((N, K), generator=g, device="cuda:0").bfloat16()
    D = m.gemm_bf16(A[:, :K] if Kp == K else A, B[:, :K] if Kp == K else B)
    want = A.double() @ B.double().T
    err = (D.double() - want).abs().max().item() / want.abs().max().item()
    assert err < 1e-5, err
