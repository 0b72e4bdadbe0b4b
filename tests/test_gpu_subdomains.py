"""Polygon subdomains (bem_set_boundary) against the oracle, and a
two-subdomain image stepped with bem_batch_lm (GPU only)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L_SHAPE = [(0.0, 0.0), (1.0, 0.0), (1.0, 0.5), (0.5, 0.5), (0.5, 1.0), (0.0, 1.0)]
TOP_RIGHT = [(0.5, 0.5), (1.0, 0.5), (1.0, 1.0), (0.5, 1.0)]


def _bg():
    import paper_2602_05492_gb300 as bg
    return bg


def _t(a, dt):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")


def _points_in(poly, n, seed):
    """Seeded points strictly inside a polygon (rejection from the unit square)."""
    rng = np.random.default_rng(seed)
    seg = oracle.polygon_boundary(poly, 1)
    out = []
    while len(out) < n:
        p = rng.uniform(0.01, 0.99, size=(4 * n, 2))
        w = oracle.angles(p, seg).sum(1) / (2 * np.pi)      # winding number
        out.extend(p[w > 0.5])
    return np.asarray(out[:n], np.float32).astype(np.float64)


def _split_scene(wd):
    th = np.zeros(32)
    for j in range(4):
        th[j * 8:j * 8 + 2] = (j / 3.0, 0.25)
        th[j * 8 + 2:j * 8 + 5] = wd
    return th


def test_split_l_shape_fp64():
    """The handle at y = 1/4 across the L-shaped subdomain: the GPU colours
    are the exact piecewise constants and the oracle's."""
    bg = _bg()
    M = 16
    mean = np.array([0.3, 0.4, 0.5])
    wd = np.array([1.0, -0.5, 0.25])
    th = _split_scene(wd)
    m = bg.BEM(precision=bg.BEM_FP64, eps_d=1e-9, eps_c=1e-9, segs_per_side=M)
    m.setup(1, [64], [0], th, mean)
    m.set_boundary(L_SHAPE, M)
    m.factor()
    pts = _points_in(L_SHAPE, 400, 1)
    pts = pts[np.abs(pts[:, 1] - 0.25) > 0.02]
    u = m.eval(_t(pts, torch.float64)).cpu().numpy()
    n_bot = M + M // 2 + M // 4
    n_top = 6 * M - n_bot
    c = np.where(pts[:, 1:2] < 0.25, -wd * n_top, wd * n_bot) / (n_top + n_bot)
    assert np.abs(u - (mean + c)).max() < 1e-9
    o = oracle.Oracle(1, [64], [0], mean, segs_per_side=M, eps_d=1e-9, eps_c=1e-9, polygon=L_SHAPE)
    assert np.abs(u - o.eval(th, pts)).max() < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_subdomain_scene_against_oracle(prec):
    """Random curves inside the L-shaped subdomain: colours and the gradient
    against the oracle on that polygon."""
    bg = _bg()
    spec = dict(C=3, K=16, W=32, spp=4, layout="random", cross=0.2, noise="gauss", sigma=0.05)
    sc = gen.make_scene(spec, seed=4100)
    th = sc.theta_init.reshape(-1, 8).copy()
    th[:, 0:2] = 0.05 + 0.4 * th[:, 0:2]              # curves in the lower-left quarter
    th = th.reshape(-1)
    mean = np.array([0.5, 0.45, 0.55])
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = bg.BEM(precision=bg.BEM_FP64 if prec == "fp64" else bg.BEM_MIXED, segs_per_side=32)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, th, mean)
    m.set_boundary(L_SHAPE, 32)
    m.factor()
    o = oracle.Oracle(sc.n_curves, sc.panels_per_curve, sc.closed, mean, segs_per_side=32,
                      polygon=L_SHAPE)
    pts = _points_in(L_SHAPE, 600, 2)
    u = m.eval(_t(pts, dt)).double().cpu().numpy()
    want = o.eval(th, pts)
    r = np.random.default_rng(3).normal(size=(len(pts), 3))
    g = m.vjp(_t(pts, dt), _t(r, dt)).cpu().numpy()
    rr = r.astype(np.float32).astype(np.float64) if prec == "mixed" else r
    gw = o.grad(th, pts, rr)
    if prec == "fp64":
        assert np.abs(u - want).max() < 1e-10 * max(1.0, np.abs(want).max())
        assert np.linalg.norm(g - gw) / np.linalg.norm(gw) < 1e-9
    else:
        assert np.sqrt(np.mean((u - want) ** 2)) < 1e-4
        assert np.linalg.norm(g - gw) / np.linalg.norm(gw) < 1e-4


def test_two_subdomains_batched():
    """An image split into the L-shaped subdomain and the top-right square,
    each with its own curves, samples and mean colour, stepped together: each
    subdomain's batched step is its own lm_step, and its loss is the oracle's."""
    bg = _bg()
    doms = []
    for k, (poly, lo, hi) in enumerate([(L_SHAPE, 0.05, 0.45), (TOP_RIGHT, 0.55, 0.95)]):
        spec = dict(C=2 + k, K=16, W=32, spp=4, layout="random", cross=0.2, noise="gauss",
                    sigma=0.05)
        sc = gen.make_scene(spec, seed=4200 + k)
        th = sc.theta_init.reshape(-1, 8).copy()
        th[:, 0:2] = lo + (hi - lo) * th[:, 0:2]
        th = th.reshape(-1)
        xy = _points_in(poly, 3000, 10 + k).astype(np.float32)
        tgt = np.clip(0.5 + 0.3 * np.sin(7 * xy[:, :1] + np.arange(3)), 0, 1).astype(np.float32)
        mean = np.minimum(tgt, 1.0).mean(0).astype(np.float64)
        doms.append((poly, sc, th, xy, tgt, mean))

    def ctxs():
        out = []
        for poly, sc, th, xy, tgt, mean in doms:
            m = bg.BEM(precision=bg.BEM_MIXED, segs_per_side=32)
            m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, th, mean)
            m.set_boundary(poly, 32)
            m.factor()
            out.append(m)
        return out

    lams = [1e-3, 1e-2, 1e-1, 1.0]
    single, batched = ctxs(), ctxs()
    b = bg.BEMBatch(batched)
    xs = [_t(d[3], torch.float32) for d in doms]
    ts = [_t(d[4], torch.float32) for d in doms]
    rb = b.lm_step(xs, ts, lams)
    for s, (poly, sc, th, xy, tgt, mean) in enumerate(doms):
        r = single[s].lm_step(xs[s], ts[s], lams)
        assert rb[s]["loss_before"] == pytest.approx(r["loss_before"], rel=1e-6)
        assert rb[s]["accepted"] == r["accepted"]
        o = oracle.Oracle(sc.n_curves, sc.panels_per_curve, sc.closed, mean, segs_per_side=32,
                          polygon=poly)
        want = o.loss(th, xy.astype(np.float64), tgt.astype(np.float64))
        assert rb[s]["loss_before"] == pytest.approx(want, rel=1e-5)
    b.close()


def test_set_boundary_errors():
    bg = _bg()
    m = bg.BEM(precision=bg.BEM_FP64, segs_per_side=8)
    with pytest.raises(bg.BemError):
        m.set_boundary(L_SHAPE[::-1], 8)          # clockwise
    with pytest.raises(bg.BemError):
        m.set_boundary([(0, 0), (1, 0)], 8)       # too few vertices
    with pytest.raises(bg.BemError):
        m.set_boundary([(0, 0), (2, 0), (0, 1)], 8)   # outside the unit square
