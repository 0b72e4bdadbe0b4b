"""The library's float transcendentals against CUDA's accurate float functions
(GPU only), over the ranges the pair formulas use."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def model():
    import paper_2602_05492_gb300 as bg
    return bg.BEM(precision=bg.BEM_MIXED)


def _t(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


def test_atan2(model):
    rng = np.random.default_rng(0)
    ang = rng.uniform(-math.pi, math.pi, 200000)
    r = 10.0 ** rng.uniform(-6, 1, ang.size)
    y, x = r * np.sin(ang), r * np.cos(ang)
    special = np.array([[1, 1], [1, -1], [-1, -1], [1e-7, -1], [-1e-7, -1], [1, 0], [0, 1],
                        [3e-8, 2.0], [1.0, 1e-8]], np.float32)
    y = np.concatenate([y, special[:, 0]])
    x = np.concatenate([x, special[:, 1]])
    fast, ref = model.fastmath(0, _t(y), _t(x))
    err = (fast - ref).abs().max().item()
    assert err < 3e-7, err


def test_log(model):
    x = 10.0 ** np.random.default_rng(1).uniform(-6, 1, 200000)
    fast, ref = model.fastmath(1, _t(x))
    err = ((fast - ref).abs() / torch.clamp(ref.abs(), min=1.0)).max().item()
    assert err < 1e-6, err


def test_log1p(model):
    rng = np.random.default_rng(2)
    z = np.concatenate([rng.uniform(-0.999, 10, 100000), rng.uniform(-0.3, 0.3, 100000),
                        10.0 ** rng.uniform(-9, -1, 50000), -(10.0 ** rng.uniform(-9, -1, 50000))])
    fast, ref = model.fastmath(2, _t(z))
    rel = ((fast - ref).abs() / torch.clamp(ref.abs(), min=1e-30)).max().item()
    assert rel < 2e-6, rel


def test_atan2_ypos(model):
    rng = np.random.default_rng(3)
    ang = rng.uniform(0, math.pi, 200000)
    r = 10.0 ** rng.uniform(-6, 1, ang.size)
    y, x = r * np.sin(ang), r * np.cos(ang)
    special = np.array([[1, 1], [1, -1], [0, -1], [0, 1], [1, 0], [0, 0], [3e-8, 2.0],
                        [3e-8, -2.0], [1.0, 1e-8]], np.float32)
    y = np.concatenate([y, special[:, 0]])
    x = np.concatenate([x, special[:, 1]])
    fast, ref = model.fastmath(3, _t(y), _t(x))
    err = (fast - ref).abs().max().item()
    assert err < 3e-7, err


def test_log1p_half(model):
    rng = np.random.default_rng(4)
    z = np.concatenate([rng.uniform(-0.999, 10, 100000), rng.uniform(-0.3, 0.3, 100000),
                        10.0 ** rng.uniform(-9, -1, 50000), -(10.0 ** rng.uniform(-9, -1, 50000))])
    fast, ref = model.fastmath(4, _t(z))
    rel = ((fast - ref).abs() / torch.clamp(ref.abs(), min=1e-30)).max().item()
    assert rel < 2e-6, rel


def test_dlog_double(model):
    """The near field's double logarithm (table-driven, Tang 1990) against
    CUDA's log: absolute error within a few units of 2^-53 times max(1, |log
    x|), over the whole normal range and densely where the near pairs put
    q = t^2 + h^2 + eps^2."""
    rng = np.random.default_rng(3)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000),
                        10.0 ** rng.uniform(-14, 2, 300000),
                        1.0 + rng.uniform(-1e-3, 1e-3, 20000),
                        np.array([1.0, 2.0, 0.5, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0),
                                  2.2250738585072014e-308, 1.7976931348623157e308])])
    xt = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    own, ref = model.dlog(xt)
    own, ref = own.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(own))
    err = np.abs(own - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 8 * 2.0 ** -53, err.max()



def test_datan2_double(model):
    """The near field's double arctangent (octant reduction, table of 64
    breakpoints, addition theorem) against CUDA's atan2 for y >= 0: relative
    error within a few units of 2^-53 (the two errors add), over wide
    magnitude ranges, densely
    where the near pairs put (h' L, h'^2 + t1 t2), across the octant and
    table breakpoints, and at the special values."""
    rng = np.random.default_rng(5)
    n = 400000
    # (magnitudes up to 1e150, so that every ratio y/x stays a normal double)
    y = np.concatenate([10.0 ** rng.uniform(-150, 150, n), 10.0 ** rng.uniform(-6, 0, n),
                        rng.uniform(0, 1, n)])
    x = np.concatenate([rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-150, 150, n),
                        rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-6, 0, n),
                        rng.uniform(-1, 1, n)])
    # y / |x| at and next to the table breakpoints j/64 and at 1 (the octant edge)
    j = rng.integers(0, 65, n)
    r = j / 64.0 * (1.0 + rng.choice([-1, 0, 1], n) * 2.0 ** -50)
    ax = 10.0 ** rng.uniform(-3, 3, n)
    y = np.concatenate([y, r * ax, ax, ax / np.maximum(r, 1e-300) * (r > 0) + ax * (r == 0),
                        np.array([0.0, 0.0, 1.0, 1.0, 1.0, 0.0])])
    x = np.concatenate([x, ax * rng.choice([-1.0, 1.0], n), ax * r, -ax,
                        np.array([1.0, -1.0, 0.0, 1.0, -1.0, 0.0])])
    yt = torch.tensor(y, dtype=torch.float64, device="cuda:0")
    xt = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    own, ref = model.datan2(yt, xt)
    own, ref = own.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(own))
    err = np.abs(own - ref) / np.maximum(np.abs(ref), 1e-300)
    # (a few units of 2^-53 each for the library's and CUDA's; measured ...)
    print(f"datan2_ypos: max relative difference to CUDA's atan2 {err.max() / 2.0 ** -53:.2f} x 2^-53")
    assert err.max() < 8 * 2.0 ** -53, err.max()
    assert own[-1] == 0.0 and own[-6] == 0.0 and own[-5] == ref[-5]
