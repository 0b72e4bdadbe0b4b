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

