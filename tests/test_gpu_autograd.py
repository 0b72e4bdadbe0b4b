"""Differentiation through torch.autograd (config 3 scale: 32 curves, 1,024
parameters): the adjoint behind backward() against the oracle gradient and
central finite differences, and device memory of the recomputing adjoint
against a stored samples x panels matrix."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cfg3():
    sc = gen.make_scene(3)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)
    o = oracle.Oracle.from_scene(sc, mean_color=[0.4, 0.5, 0.6])
    return sc, xy, o


def _model(sc, prec, **kw):
    import paper_2602_05492_gb300 as bg
    m = bg.BEM(precision=prec, **kw)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, [0.4, 0.5, 0.6])
    m.factor()
    return m


def test_autograd_matches_oracle_and_fd(cfg3):
    import paper_2602_05492_gb300 as bg
    from paper_2602_05492_gb300.autograd import bem_eval
    sc, xy, o = cfg3
    sub = xy[::256]                                   # 4,096 samples
    dev = "cuda:0"
    m = _model(sc, bg.BEM_FP64)
    xt = torch.tensor(sub, dtype=torch.float64, device=dev)
    tgt = torch.tensor(np.random.default_rng(0).uniform(0, 1, (sub.shape[0], 3)), device=dev)
    theta = torch.tensor(sc.theta_init, dtype=torch.float64, device=dev, requires_grad=True)
    u = bem_eval(theta, xt, m)
    loss = 0.5 * ((u - tgt) ** 2).sum()
    loss.backward()
    g = theta.grad.cpu().numpy()
    r = (u.detach() - tgt).cpu().numpy()
    want = o.grad(sc.theta_init, sub, r)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-10
    # central differences of the GPU forward, h = 1e-6, FP64
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in rng.choice(sc.n_theta, 10, replace=False):
        if k % 32 in (24, 25) and sc.closed[k // 32]:
            continue
        th = theta.detach().clone()
        th[k] += h
        lp = 0.5 * ((bem_eval(th, xt, m) - tgt) ** 2).sum().item()
        th[k] -= 2 * h
        lm = 0.5 * ((bem_eval(th, xt, m) - tgt) ** 2).sum().item()
        assert (lp - lm) / (2 * h) == pytest.approx(g[k], rel=1e-6, abs=1e-8)


def test_autograd_mixed_vs_fp64(cfg3):
    import paper_2602_05492_gb300 as bg
    from paper_2602_05492_gb300.autograd import bem_eval
    sc, xy, o = cfg3
    sub = xy[::64]
    dev = "cuda:0"
    grads = {}
    for prec, dt in ((bg.BEM_FP64, torch.float64), (bg.BEM_MIXED, torch.float32)):
        m = _model(sc, prec)
        xt = torch.tensor(sub, dtype=dt, device=dev)
        tgt = torch.tensor(np.random.default_rng(0).uniform(0, 1, (sub.shape[0], 3)), dtype=dt,
                           device=dev)
        theta = torch.tensor(sc.theta_init, dtype=torch.float64, device=dev, requires_grad=True)
        loss = 0.5 * ((bem_eval(theta, xt, m) - tgt) ** 2).sum()
        loss.backward()
        grads[prec] = theta.grad.cpu().numpy()
    a, b = grads[bg.BEM_MIXED], grads[bg.BEM_FP64]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4


def test_adjoint_memory_vs_stored_matrix(cfg3):
    """The adjoint recomputes kernel values: its device footprint for all
    1,048,576 samples stays far below one stored 1M x 2,048 float matrix."""
    import paper_2602_05492_gb300 as bg
    sc, xy, o = cfg3
    m = _model(sc, bg.BEM_MIXED)
    xt = torch.tensor(xy, dtype=torch.float32, device="cuda:0")
    r = torch.randn((xy.shape[0], 3), dtype=torch.float32, device="cuda:0")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    g = m.vjp(xt, r)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = max(free0 - free1, 0)
    stored = xy.shape[0] * sc.n_panels * 4
    assert used < 0.02 * stored, (used, stored)
    assert torch.isfinite(g).all()
