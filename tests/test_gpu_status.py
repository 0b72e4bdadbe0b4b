"""Device-side failure reporting through the context's status word (GPU only).

The tensor-core kernels wait on shared-memory barriers for their copies and
MMAs.  Every such wait is bounded: a pipeline wait gives up after the
context's limit (bem_set_wait_limit), the kernel records the failure in the
device status word, lets the copies and MMAs it has issued finish, frees its
tensor memory and returns; the call reports BEM_ETIMEDOUT at its next sync
point.  With the limit at 0 every pipeline wait that is not already complete
gives up, which makes the failure happen on purpose without hanging or
faulting anything.  The same context must then work normally again.
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


def _ab(M, N, K, seed):
    g = torch.Generator(device="cuda:0").manual_seed(seed)
    A = torch.randn((M, K), generator=g, device="cuda:0").bfloat16()
    B = torch.randn((N, K), generator=g, device="cuda:0").bfloat16()
    return A, B


def test_gemm_wait_limit_zero_times_out_then_recovers():
    bg = _bg()
    m = bg.BEM(precision=bg.BEM_MIXED)
    A, B = _ab(256, 384, 1024, 7)
    m.set_wait_limit(0.0)
    with pytest.raises(bg.BemError) as e:
        m.gemm_bf16(A, B)
    assert e.value.code == bg.BEM_ETIMEDOUT
    m.set_wait_limit(1.0)
    for _ in range(2):
        D = m.gemm_bf16(A, B)
        want = A.double() @ B.double().T
        err = (D.double() - want).abs().max().item() / want.abs().max().item()
        assert err < 1e-5, err
    with pytest.raises(bg.BemError) as e:
        m.set_wait_limit(-1.0)
    assert e.value.code == bg.BEM_EINVAL
    m.close()


@pytest.mark.parametrize("mode", ["bf16", "3xtf32", "bf16x3"])
def test_gauss_newton_wait_limit_zero_times_out_then_recovers(mode):
    """bem_gn_products (J rows and Gram blocks on the tensor cores) with the
    limit at 0 reports BEM_ETIMEDOUT; with the default limit the same context
    then matches the oracle's Gauss-Newton matrix and gradient."""
    bg = _bg()
    jm = {"bf16": bg.BEM_JTJ_BF16, "3xtf32": bg.BEM_JTJ_3XTF32, "bf16x3": bg.BEM_JTJ_BF16X3}[mode]
    sc = gen.make_scene(1)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)[::16]
    o = oracle.Oracle.from_scene(sc)
    target = gen.add_noise(o.eval(sc.theta_true, xy), sc.noise, sc.seed)
    mean = np.minimum(target, 1.0).mean(0)
    o.mean = mean
    m = bg.BEM(precision=bg.BEM_MIXED, jtj_mode=jm)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, mean)
    m.factor()
    x = torch.tensor(xy, dtype=torch.float32, device="cuda:0")
    t = torch.tensor(target, dtype=torch.float32, device="cuda:0")
    m.set_wait_limit(0.0)
    with pytest.raises(bg.BemError) as e:
        m.gn_products(x, t)
    assert e.value.code == bg.BEM_ETIMEDOUT
    m.set_wait_limit(1.0)
    L, g, H = m.gn_products(x, t)
    Lw, gw, Hw = o.gauss_newton(sc.theta_init, xy, target)
    assert L == pytest.approx(Lw, rel=1e-5)
    g, H = g.cpu().numpy(), H.cpu().numpy()
    assert np.linalg.norm(g - gw) / np.linalg.norm(gw) < 1e-4
    # five times the measured error (2,048 samples)
    tol = {"bf16": 5e-3, "3xtf32": 7e-6, "bf16x3": 2.5e-5}[mode]
    assert np.linalg.norm(H - Hw) / np.linalg.norm(Hw) < tol
    m.close()
