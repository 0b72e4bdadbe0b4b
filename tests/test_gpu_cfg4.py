"""Config 4 at full size (128 curves x 64 panels = 8,192 panels, 1024^2 px x
64 spp = 67,108,864 samples), in the launch configuration the bench times:
sampled outputs against the FP64 oracle (GPU only).

The mixed path runs with the configuration's near field (sample-panel
distance below 2 panel lengths in double).  Colours: RMSE <= 1e-4 over a
seeded sample of points; gradient: <= 1e-4 relative for a residual supported
on those points, which the oracle can evaluate one by one.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cfg4():
    import paper_2602_05492_gb300 as bg
    sc = gen.make_scene(4)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed, dtype=np.float32)
    assert xy.shape[0] == 1024 * 1024 * 64
    mean = np.array([0.45, 0.5, 0.55])
    idx = np.sort(np.random.default_rng(41).choice(xy.shape[0], 1200, replace=False))
    o = oracle.Oracle.from_scene(sc, mean_color=mean)
    m = bg.BEM(precision=bg.BEM_MIXED, near_factor=2.0)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
    m.factor()
    xt = torch.from_numpy(xy).to("cuda:0")
    return sc, xy, xt, idx, o, m


def test_eval_mixed_cfg4_sampled(cfg4):
    sc, xy, xt, idx, o, m = cfg4
    u = m.eval(xt)
    us = u[torch.from_numpy(idx).to(u.device)].double().cpu().numpy()
    want = o.eval(sc.theta_init, xy[idx].astype(np.float64))
    rmse = np.sqrt(np.mean((us - want) ** 2))
    assert rmse < 1e-4, rmse
    assert np.isfinite(u.sum().item())


def test_vjp_mixed_cfg4_sampled(cfg4):
    sc, xy, xt, idx, o, m = cfg4
    r = torch.zeros((xy.shape[0], 3), dtype=torch.float32, device="cuda:0")
    rs = np.random.default_rng(42).normal(size=(len(idx), 3)).astype(np.float32)
    r[torch.from_numpy(idx).to(r.device)] = torch.from_numpy(rs).to(r.device)
    g = m.vjp(xt, r).cpu().numpy()
    want = o.grad(sc.theta_init, xy[idx].astype(np.float64), rs.astype(np.float64))
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-4
