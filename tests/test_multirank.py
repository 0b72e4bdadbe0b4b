"""World-size-2 gloo ranks on CPU: sharded Gauss-Newton sums reduced in rank
order equal the unsharded sums (the exchange step a sample-sharded LM step
would need), and the bench's max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import gen
    import oracle
    from paper_2602_05492_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = gen.make_scene(dict(C=2, K=8, W=8, spp=2, layout="random", cross=0.5, noise="gauss",
                             sigma=0.05), seed=21)
    o = oracle.Oracle.from_scene(sc, segs_per_side=16)
    xy = gen.make_samples(8, 4, 21)
    target = np.random.default_rng(0).uniform(0, 1, (xy.shape[0], 3))
    b, e = shard.shard_range(xy.shape[0], world, rank)
    L, g, H = o.gauss_newton(sc.theta_init, xy[b:e], target[b:e])
    m = e - b
    parts = [torch.tensor([L * m], dtype=torch.float64), torch.tensor(g * m), torch.tensor(H * m)]
    Ls, gs, Hs = shard.reduce_fixed_order(parts)
    n = xy.shape[0]
    t = shard.max_over_ranks(float(rank + 1))
    if rank == 0:
        np.savez(os.path.join(result_dir, "out.npz"), L=Ls.numpy()[0] / n, g=gs.numpy() / n,
                 H=Hs.numpy() / n, t=t)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_gauss_newton_two_ranks(tmp_path):
    import gen
    import oracle
    import __graft_entry__
    __graft_entry__._load_build_module().build()     # the package loads its library on import
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = np.load(tmp_path / "out.npz")
    sc = gen.make_scene(dict(C=2, K=8, W=8, spp=2, layout="random", cross=0.5, noise="gauss",
                             sigma=0.05), seed=21)
    o = oracle.Oracle.from_scene(sc, segs_per_side=16)
    xy = gen.make_samples(8, 4, 21)
    target = np.random.default_rng(0).uniform(0, 1, (xy.shape[0], 3))
    L, g, H = o.gauss_newton(sc.theta_init, xy, target)
    assert float(r["L"]) == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(r["g"], g, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(r["H"], H, rtol=1e-11, atol=1e-15 * np.abs(H).max())
    assert float(r["t"]) == 2.0


@pytest.mark.parametrize("n,world", [(10, 3), (7, 2), (1, 4), (0, 2)])
def test_shard_ranges_cover(n, world):
    from paper_2602_05492_gb300 import shard
    rs = [shard.shard_range(n, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    for (b0, e0), (b1, e1) in zip(rs, rs[1:]):
        assert e0 == b1 and b0 <= e0
