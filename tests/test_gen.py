"""The seeded input recipe (CPU only): scene sizes of the five workloads,
crossing fraction, sample layout, noise models and the independence of the
random streams."""
import numpy as np
import pytest

import gen
from gen import scenes


@pytest.mark.parametrize("cfg,C,K,W,spp", [(1, 4, 32, 64, 8), (2, 32, 64, 256, 16),
                                           (3, 32, 64, 256, 16), (4, 128, 64, 1024, 64)])
def test_scene_sizes(cfg, C, K, W, spp):
    sc = gen.make_scene(cfg)
    assert sc.n_curves == C and np.all(sc.panels_per_curve == K)
    assert sc.theta_true.shape == sc.theta_init.shape == (32 * C,)
    assert (sc.W, sc.spp) == (W, spp)
    assert sc.n_samples == W * W * spp
    # closed curves repeat their first control point, before and after the perturbation
    for th in (sc.theta_true, sc.theta_init):
        t = th.reshape(C, 4, 8)
        for i in np.nonzero(sc.closed)[0]:
            assert np.array_equal(t[i, 3, 0:2], t[i, 0, 0:2])


def test_config1_layout():
    sc = gen.make_scene(1)
    ctrl = sc.theta_true.reshape(4, 4, 8)[:, :, 0:2]
    assert list(sc.closed) == [0, 0, 1, 0]
    # curves 0 and 1 cross
    assert scenes.crossing_fraction(ctrl[:2], sc.closed[:2]) == 1.0


@pytest.mark.parametrize("cfg", [2, 3, 4])
def test_crossing_fraction_near_one_fifth(cfg):
    sc = gen.make_scene(cfg)
    ctrl = sc.theta_true.reshape(sc.n_curves, 4, 8)[:, :, 0:2]
    assert abs(scenes.crossing_fraction(ctrl, sc.closed) - 0.2) <= 0.02


def test_samples_are_jittered_inside_their_pixels():
    W, spp = 64, 8
    xy = gen.make_samples(W, spp, 7)
    assert xy.shape == (W * W * spp, 2)
    pix = np.arange(xy.shape[0]) // spp
    assert np.array_equal(np.floor(xy[:, 0] * W).astype(int), pix % W)
    assert np.array_equal(np.floor(xy[:, 1] * W).astype(int), pix // W)
    # float32-exact positions, and a prefix is the prefix of the full set
    assert np.array_equal(xy, xy.astype(np.float32).astype(np.float64))
    assert np.array_equal(gen.make_samples(W, spp, 7, n=1000), xy[:1000])
    assert not np.array_equal(gen.make_samples(W, spp, 8, n=1000), xy[:1000])


def test_gaussian_noise():
    truth = np.full((200000, 3), 0.5)
    t = gen.add_noise(truth, {"noise": "gauss", "sigma": 0.05}, 3)
    r = t - truth
    assert abs(r.mean()) < 1e-3 and abs(r.std() / 0.05 - 1) < 0.01


def test_lognormal_noise_with_fireflies():
    truth = np.full((400000, 3), 0.5)
    noise = {"noise": "lognormal", "sigma": 0.3, "firefly": 0.01, "firefly_gain": 20.0}
    t = gen.add_noise(truth, noise, 3)
    z = np.log(t / truth)
    # a firefly sample carries log 20 on all three channels on top of its noise
    ff = z.mean(1) > np.log(20.0) / 2
    assert abs(ff.mean() - 0.01) < 0.0015
    zc = z[~ff]
    assert abs(zc.mean()) < 3e-3 and abs(zc.std() / 0.3 - 1) < 0.01
    assert abs(z[ff].mean() - np.log(20.0)) < 0.02


def test_streams_are_independent_of_other_sizes():
    """The scene of a seed does not depend on how many samples are drawn,
    and the noise of a seed not on the scene: each purpose has its own
    stream."""
    a = gen.make_scene(2)
    b = gen.make_scene(2, W=128, spp=4)
    assert np.array_equal(a.theta_true, b.theta_true)
    assert np.array_equal(a.theta_init, b.theta_init)
    truth = np.full((1000, 3), 0.5)
    n1 = gen.add_noise(truth, {"noise": "gauss", "sigma": 0.05}, a.seed)
    n2 = gen.add_noise(truth, {"noise": "gauss", "sigma": 0.05}, a.seed)
    assert np.array_equal(n1, n2)
