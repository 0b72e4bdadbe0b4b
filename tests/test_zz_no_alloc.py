"""The allocation-free adjoint (bem_vjp_noalloc) against bem_vjp, through the C ABI.

This entry point serves callers that cannot allocate GPU memory while they
run: real-time loops that must stay out of the allocator (an allocation can
stall the whole device), and hosts whose own memory pool owns the GPU.  It
takes its scratch from one static device array instead.  The test calls it
twice in a row (the second call reuses the array the first one left behind)
and compares both results with bem_vjp at the tolerances of the other
gradient tests: 1e-10 relative in FP64 contexts, 1e-4 relative in mixed
ones.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(bg, sc, prec):
    m = bg.BEM(precision=prec)
    m.setup(sc.n_curves, sc.panels_per_curve, sc.closed, sc.theta_init, [0.4, 0.5, 0.6])
    m.factor()
    return m


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_vjp_noalloc_matches_vjp_twice(prec, tol):
    """On a fresh context (set up and factored, no adjoint run yet, so none
    of bem_vjp's buffers exists) two bem_vjp_noalloc calls in a row: the
    context's allocation count stays where it was, the device's free memory
    does not move across the calls, and both results match bem_vjp on a
    second context."""
    import paper_2602_05492_gb300 as bg
    p = {"fp64": bg.BEM_FP64, "mixed": bg.BEM_MIXED}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    sc = gen.make_scene(3)
    xy = gen.make_samples(sc.W, sc.spp, sc.seed)[::16]          # 65,536 samples
    m = _ctx(bg, sc, p)
    xt = torch.tensor(xy, dtype=dt, device="cuda:0")
    r = torch.tensor(np.random.default_rng(4).normal(size=(xy.shape[0], 3)), dtype=dt,
                     device="cuda:0")
    gs = [torch.full((m.n_theta,), float("nan"), dtype=torch.float64, device="cuda:0")
          for _ in range(2)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    allocs0 = m.alloc_count()
    for k, g in enumerate(gs):
        free0 = torch.cuda.mem_get_info()[0]
        rc = bg.bem_vjp_noalloc(m.h, xt.shape[0], ctypes.c_void_p(xt.data_ptr()),
                                ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                stream)
        assert rc == 0, bg.bem_last_error(m.h).decode()
        torch.cuda.synchronize()
        # the first call on a device may load the library's device code (and
        # with it the static array) there; from the second call on nothing
        # may change the device's free memory
        if k == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        assert m.alloc_count() == allocs0
    ref = _ctx(bg, sc, p)
    want = ref.vjp(xt, r).cpu().numpy()
    for g in gs:
        g = g.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.linalg.norm(g - want) / np.linalg.norm(want) < tol
    m.close()
    ref.close()


def test_vjp_noalloc_rejects_oversized_scene():
    import paper_2602_05492_gb300 as bg
    C = 3200                                         # 204,800 panels: beyond the static array
    rng = np.random.default_rng(0)
    th = np.zeros((C, 4, 8))
    th[:, :, 0:2] = rng.uniform(0.1, 0.9, (C, 4, 2))
    m = bg.BEM(precision=bg.BEM_MIXED, segs_per_side=16)
    m.setup(C, np.full(C, 64, np.int32), np.zeros(C, np.uint8), th.reshape(-1), [0.5, 0.5, 0.5])
    m.factor()
    xt = torch.full((4, 2), 0.5, dtype=torch.float32, device="cuda:0")
    r = torch.zeros((4, 3), dtype=torch.float32, device="cuda:0")
    g = torch.zeros(m.n_theta, dtype=torch.float64, device="cuda:0")
    with pytest.raises(bg.BemError) as e:
        m.vjp_noalloc(xt, r, g)
    assert e.value.code == bg.BEM_EINVAL and "static scratch" in str(e.value)
    m.close()
