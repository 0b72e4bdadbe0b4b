"""A whole fit: 50 LM iterations (Eq. (optimstep)) of the mixed path and of the
FP64 path from the same start, on the 4-curve scene (128 panels, 32,768
samples, Gaussian noise), each iteration's damping from the previous one's
proposal.  The two trajectories differ in rounding only: both lower the loss
monotonically, end below the loss of the true handles (the fit explains the
data as well as the handles that made it, up to fitting some noise) and at
the same loss within 0.5 % (the oracle's own 50 iterations from this start
end at 4.2372e-3 from 6.4583e-3, against 4.3209e-3 at the true handles;
measured: FP64 4.2372e-3, the oracle's end point, and mixed 4.2296e-3, each
with 12 accepted iterations) (GPU only)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STEPS = 50


def _fit(prec, sc, xy, target, mean):
    import paper_2602_05492_gb300 as bg
    m = bg.BEM(precision=prec)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
    m.factor()
    dt = torch.float64 if prec == bg.BEM_FP64 else torch.float32
    x = torch.tensor(xy, dtype=dt, device="cuda:0")
    t = torch.tensor(target, dtype=dt, device="cuda:0")
    lam, before, accepted = 1e-3, [], 0
    for _ in range(STEPS):
        r = m.lm_step(x, t, [lam])
        before.append(r["loss_before"])
        accepted += r["accepted"]
        lam = r["lambda_next"]
    end = m.loss(x, t)
    th = m.get_params()
    m.close()
    return np.array(before), end, accepted, th


def test_fit_mixed_vs_fp64():
    import paper_2602_05492_gb300 as bg
    sc = gen.make_scene(1)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)
    o = oracle.Oracle.from_scene(sc)
    truth = o.eval(oracle.project_compat(o.geo, sc.theta_true), xy)
    target = gen.add_noise(truth, sc.noise, sc.seed)
    mean = np.minimum(target, 1.0).mean(0)
    o.mean = mean
    l_true = o.loss(oracle.project_compat(o.geo, sc.theta_true), xy, target)
    b64, e64, a64, th64 = _fit(bg.BEM_FP64, sc, xy, target, mean)
    b32, e32, a32, th32 = _fit(bg.BEM_MIXED, sc, xy, target, mean)
    print(f"loss at theta_init {b64[0]:.6e}; after {STEPS} LM iterations: FP64 {e64:.6e} "
          f"({a64} accepted), mixed {e32:.6e} ({a32} accepted), "
          f"relative difference {abs(e32 - e64) / e64:.2e}")
    for b, e in ((b64, e64), (b32, e32)):
        # an LM iteration never raises the loss (a trial that would is
        # rejected); the mixed path forms the loss at theta and at a trial
        # in different kernels, which agree to float rounding
        assert np.all(np.diff(np.append(b, e)) <= 1e-6 * b[0])
        assert e < l_true
    assert b32[0] == pytest.approx(b64[0], rel=1e-5)
    assert e32 == pytest.approx(e64, rel=5e-3)
    # the oracle's loss at the mixed fit's end point agrees with the mixed path's
    assert o.loss(th32, xy, target) == pytest.approx(e32, rel=5e-5)
