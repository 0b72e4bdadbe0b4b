"""Seeded synthetic scenes, sample sets and noisy targets.

A scene is a set of cubic Bezier diffusion curves on the unit square.  Each
curve has four control handles; every control handle carries eight numbers:
position (x, y), colour jump w_d (RGB) and normal-derivative jump w_c (RGB).
The flat parameter vector is therefore theta[curve][handle][8], n_theta =
32 * n_curves.  A closed curve repeats its first control point as its last
(the last point's position entries are then not free parameters).

The paper fits line-segment handles to Monte Carlo colour samples (Sec. 4);
Bezier curves with interpolated jumps are its suggested extension (Sec. 6,
"Post-processing").  The workloads below follow five benchmark
configurations (sizes, noise models, perturbations); where those leave a
detail open, the choice is stated with the function that makes it.

Random streams are independent children of one SeedSequence per config, in a
fixed order (geometry, colours, mean colour, initial perturbation, sample
jitter, noise), so that changing one array's size never shifts another.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# stream indices of SeedSequence.spawn(); never reorder
_GEOM, _COLOR, _MEAN, _PERTURB, _JITTER, _NOISE, _TRUTH = range(7)


CONFIGS = {
    # plain method, FP64: 4 curves (0 and 1 cross, 2 closed), 32 panels each
    1: dict(C=4, K=32, W=64, spp=8, noise="gauss", sigma=0.05, layout="cfg1",
            lm_steps=10, seed=1001),
    # FP64 vs FP32: 32 random curves, ~20% crossing pairs, 64 panels each
    2: dict(C=32, K=64, W=256, spp=16, noise="lognormal", sigma=0.3,
            firefly=0.01, firefly_gain=20.0, layout="random", cross=0.2,
            lm_steps=50, seed=1002),
    # differentiation: config-1 generator with 32 curves (1,024 parameters)
    3: dict(C=32, K=64, W=256, spp=16, noise="gauss", sigma=0.05,
            layout="random", cross=0.2, lm_steps=1, seed=1003),
    # precision: 128 curves x 64 panels, 1024^2 px x 64 spp
    4: dict(C=128, K=64, W=1024, spp=64, noise="lognormal", sigma=0.3,
            firefly=0.01, firefly_gain=20.0, layout="random", cross=0.2,
            lm_steps=1, seed=1004),
}


@dataclasses.dataclass
class Scene:
    """Geometry and parameters of one synthetic diffusion-curve scene."""
    n_curves: int
    panels_per_curve: np.ndarray   # int32 [C]
    closed: np.ndarray             # uint8 [C]
    theta_true: np.ndarray         # float64 [C*32]
    theta_init: np.ndarray         # float64 [C*32]
    mean_true: np.ndarray          # float64 [3]
    W: int
    spp: int
    noise: dict
    seed: int

    @property
    def n_theta(self) -> int:
        return 32 * self.n_curves

    @property
    def n_panels(self) -> int:
        return int(self.panels_per_curve.sum())

    @property
    def n_samples(self) -> int:
        return self.W * self.W * self.spp


def _streams(seed: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(8)]


# ---------------------------------------------------------------------------
# geometry helpers (crossing statistic only; no panel integrals)

def _polyline(ctrl: np.ndarray, closed: bool, n: int) -> np.ndarray:
    """Dense polyline of a cubic Bezier for the crossing statistic [n+1, 2]."""
    p = ctrl.copy()
    if closed:
        p[3] = p[0]
    s = np.linspace(0.0, 1.0, n + 1)[:, None]
    # power basis of the cubic: c0 + c1 s + c2 s^2 + c3 s^3
    c0 = p[0]
    c1 = 3.0 * (p[1] - p[0])
    c2 = 3.0 * (p[0] - 2.0 * p[1] + p[2])
    c3 = p[3] - p[0] + 3.0 * (p[1] - p[2])
    return c0 + s * (c1 + s * (c2 + s * c3))


def _segments_cross(P: np.ndarray, Q: np.ndarray) -> bool:
    """True if any segment of polyline P properly crosses any segment of Q."""
    a, b = P[:-1], P[1:]
    c, d = Q[:-1], Q[1:]
    lo1, hi1 = np.minimum(a, b), np.maximum(a, b)
    lo2, hi2 = np.minimum(c, d), np.maximum(c, d)
    if (hi1.max(0) < lo2.min(0)).any() or (hi2.max(0) < lo1.min(0)).any():
        return False
    A = a[:, None, :]
    B = b[:, None, :]
    Cc = c[None, :, :]
    D = d[None, :, :]

    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - \
               (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])

    o1 = orient(A, B, Cc)
    o2 = orient(A, B, D)
    o3 = orient(Cc, D, A)
    o4 = orient(Cc, D, B)
    return bool(np.any((o1 * o2 < 0) & (o3 * o4 < 0)))


def crossing_fraction(ctrl: np.ndarray, closed: np.ndarray, n: int = 32) -> float:
    """Fraction of curve pairs whose polylines cross (ctrl: [C, 4, 2])."""
    C = ctrl.shape[0]
    if C < 2:
        return 0.0
    polys = [_polyline(ctrl[i], bool(closed[i]), n) for i in range(C)]
    hits = 0
    for i in range(C):
        for j in range(i + 1, C):
            hits += _segments_cross(polys[i], polys[j])
    return hits / (C * (C - 1) / 2)


def _random_layout(rng, C: int, target: float, closed: np.ndarray) -> np.ndarray:
    """Control points of C random curves with ~target crossing-pair fraction.

    Each curve is a centre plus four offsets drawn once; a common scale s is
    bisected so that the measured crossing fraction lands within +-0.02 of
    the target (deterministic for a given seed).
    """
    centre = rng.uniform(0.0, 1.0, size=(C, 1, 2))
    offs = rng.uniform(-0.5, 0.5, size=(C, 4, 2))

    def build(s):
        c = 0.5 + (centre - 0.5) * (1.0 - s)   # keeps points inside [0, 1]^2
        return np.clip(c + s * offs, 0.0, 1.0)

    lo, hi = 0.02, 1.0
    best = build(0.3)
    if C >= 2:
        for _ in range(30):
            s = 0.5 * (lo + hi)
            ctrl = build(s)
            f = crossing_fraction(ctrl, closed)
            best = ctrl
            if abs(f - target) <= 0.02:
                break
            if f < target:
                lo = s
            else:
                hi = s
    return best


def _cfg1_layout(rng) -> np.ndarray:
    """Four curves: 0 and 1 cross near the centre, 2 is a closed loop, 3 is free."""
    j = lambda: rng.uniform(-0.03, 0.03, size=2)
    c0 = np.array([[0.15, 0.40], [0.40, 0.55], [0.60, 0.35], [0.85, 0.55]])
    c1 = np.array([[0.45, 0.15], [0.60, 0.40], [0.40, 0.60], [0.55, 0.85]])
    c2 = np.array([[0.25, 0.80], [0.05, 0.98], [0.45, 0.98], [0.25, 0.80]])
    c3 = np.array([[0.70, 0.10], [0.85, 0.20], [0.80, 0.30], [0.92, 0.40]])
    ctrl = np.stack([c0, c1, c2, c3])
    for i in range(4):
        for k in range(4):
            ctrl[i, k] += j()
    ctrl[2, 3] = ctrl[2, 0]
    return np.clip(ctrl, 0.01, 0.99)


def _colors(rng, C: int) -> tuple[np.ndarray, np.ndarray]:
    """w_d = c_left - c_right with both colours U[0,1]^3; w_c ~ U[-0.5,0.5]^3."""
    c_plus = rng.uniform(0.0, 1.0, size=(C, 4, 3))
    c_minus = rng.uniform(0.0, 1.0, size=(C, 4, 3))
    wc = rng.uniform(-0.5, 0.5, size=(C, 4, 3))
    return c_plus - c_minus, wc


def _pack(ctrl, wd, wc) -> np.ndarray:
    C = ctrl.shape[0]
    th = np.zeros((C, 4, 8))
    th[:, :, 0:2] = ctrl
    th[:, :, 2:5] = wd
    th[:, :, 5:8] = wc
    return th.reshape(-1)


def perturb(theta: np.ndarray, closed: np.ndarray, rng, pos_sigma: float,
            color_sigma: float) -> np.ndarray:
    """Gaussian perturbation of positions and colour jumps (closed loops stay closed)."""
    th = theta.reshape(-1, 4, 8).copy()
    th[:, :, 0:2] += rng.normal(0.0, pos_sigma, size=th[:, :, 0:2].shape)
    th[:, :, 2:8] += rng.normal(0.0, color_sigma, size=th[:, :, 2:8].shape)
    for i in np.nonzero(closed)[0]:
        th[i, 3, 0:2] = th[i, 0, 0:2]
    return th.reshape(-1)


def make_scene(cfg, seed: int | None = None, **over) -> Scene:
    """Build the scene of a benchmark configuration (int) or of a dict."""
    spec = dict(CONFIGS[cfg]) if isinstance(cfg, int) else dict(cfg)
    spec.update(over)
    seed = spec.get("seed", 0) if seed is None else seed
    rs = _streams(seed)
    C, K = int(spec["C"]), int(spec["K"])
    layout = spec.get("layout", "random")
    if layout == "cfg1":
        assert C == 4
        closed = np.array([0, 0, 1, 0], np.uint8)
        ctrl = _cfg1_layout(rs[_GEOM])
    else:
        n_closed = int(spec.get("n_closed", max(0, C // 8)))
        closed = np.zeros(C, np.uint8)
        closed[:n_closed] = 1
        ctrl = _random_layout(rs[_GEOM], C, float(spec.get("cross", 0.2)), closed)
        for i in range(n_closed):
            ctrl[i, 3] = ctrl[i, 0]
    wd, wc = _colors(rs[_COLOR], C)
    theta_true = _pack(ctrl, wd, wc)
    mean_true = rs[_MEAN].uniform(0.25, 0.75, size=3)
    theta_init = perturb(theta_true, closed, rs[_PERTURB],
                         spec.get("pos_sigma", 0.02), spec.get("color_sigma", 0.1))
    noise = {k: spec[k] for k in ("noise", "sigma", "firefly", "firefly_gain") if k in spec}
    return Scene(n_curves=C,
                 panels_per_curve=np.full(C, K, np.int32),
                 closed=closed,
                 theta_true=theta_true,
                 theta_init=theta_init,
                 mean_true=mean_true,
                 W=int(spec["W"]), spp=int(spec["spp"]),
                 noise=noise, seed=seed)


# ---------------------------------------------------------------------------
# samples and targets

def make_samples(W: int, spp: int, seed: int, n: int | None = None,
                 dtype=np.float64) -> np.ndarray:
    """Jittered pixel samples [S, 2] in the open unit square.

    Pixel (i, j) (column i, row j, row-major) holds spp consecutive samples
    x = (i + u) / W, y = (j + v) / W with u, v uniform.  Positions are
    rounded to float32 so that single- and double-precision paths see the
    same points.  If n is given only the first n samples are returned.
    """
    rng = _streams(seed)[_JITTER]
    S = W * W * spp
    if n is not None:
        S = min(S, n)
    idx = np.arange(S)
    pix = idx // spp
    i = pix % W
    j = pix // W
    u = rng.random((S, 2))
    xy = np.empty((S, 2))
    xy[:, 0] = (i + u[:, 0]) / W
    xy[:, 1] = (j + u[:, 1]) / W
    xy = np.clip(xy, 1e-6, 1.0 - 1e-6).astype(np.float32)
    return xy.astype(dtype)


def analytic_truth(xy: np.ndarray, seed: int) -> np.ndarray:
    """A piecewise-smooth synthetic image [S, 3] in [0, 1].

    Stands in for a converged render: a few sharp edges along random lines
    (tanh profiles, width 1/512), a soft shadow-like ramp and smooth shading.
    It is an arbitrary target, not a diffusion-curve image.
    """
    rng = _streams(seed)[_TRUTH]
    x = np.asarray(xy, np.float64)
    base = rng.uniform(0.3, 0.6, size=3)
    out = np.tile(base, (x.shape[0], 1))
    for _ in range(4):
        ang = rng.uniform(0, 2 * math.pi)
        nrm = np.array([math.cos(ang), math.sin(ang)])
        d = rng.uniform(0.3, 0.7)
        amp = rng.uniform(-0.25, 0.25, size=3)
        s = np.tanh((x @ nrm - d) * 512.0)
        out += 0.5 * s[:, None] * amp
    ang = rng.uniform(0, 2 * math.pi)
    soft = np.tanh((x @ np.array([math.cos(ang), math.sin(ang)]) - 0.5) * 8.0)
    out += 0.1 * soft[:, None] * rng.uniform(-1, 1, size=3)
    f = rng.uniform(0.5, 2.0, size=2)
    out += 0.05 * np.sin(2 * math.pi * (f[0] * x[:, :1] + f[1] * x[:, 1:2]) +
                         rng.uniform(0, 2 * math.pi, size=3))
    return np.clip(out, 0.0, 1.0)


def add_noise(truth: np.ndarray, noise: dict, seed: int) -> np.ndarray:
    """Monte Carlo-like sample noise; the upper clamp is left to the method.

    gauss:     t = truth + N(0, sigma^2) per channel
    lognormal: t = truth * exp(N(0, sigma^2)); a fraction `firefly` of the
               samples is multiplied by `firefly_gain`
    """
    rng = _streams(seed)[_NOISE]
    kind = noise.get("noise", "gauss")
    if kind == "gauss":
        return truth + rng.normal(0.0, noise.get("sigma", 0.05), size=truth.shape)
    if kind == "lognormal":
        t = truth * np.exp(rng.normal(0.0, noise.get("sigma", 0.3), size=truth.shape))
        ff = rng.random(truth.shape[0]) < noise.get("firefly", 0.0)
        t[ff] *= noise.get("firefly_gain", 20.0)
        return t
    if kind == "none":
        return truth.copy()
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# batch of uneven scenes

def batch_scenes(n_scenes: int = 64, seed: int = 1005) -> list[Scene]:
    """Uneven scenes: panels log-uniform in [256, 4096] (64 per curve),
    images 128^2..512^2 at 4..32 spp, Gaussian or lognormal noise per scene."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(1)[0])
    out = []
    for s in range(n_scenes):
        P = math.exp(rng.uniform(math.log(256), math.log(4096)))
        C = int(np.clip(round(P / 64), 4, 64))
        W = int(rng.choice([128, 192, 256, 384, 512]))
        spp = int(rng.choice([4, 8, 16, 32]))
        if rng.random() < 0.5:
            nz = dict(noise="gauss", sigma=0.05)
        else:
            nz = dict(noise="lognormal", sigma=0.3, firefly=0.01, firefly_gain=20.0)
        spec = dict(C=C, K=64, W=W, spp=spp, layout="random", cross=0.2, **nz)
        out.append(make_scene(spec, seed=seed * 1000 + s))
    return out


# ---------------------------------------------------------------------------
# segment handles (the paper's own parametrisation, Sec. 4.2)

@dataclasses.dataclass
class SegmentScene:
    """Independent straight handles, theta[h][10] = (a, b, w_d RGB, w_c RGB)."""
    n_handles: int
    theta_true: np.ndarray         # float64 [H*10]
    theta_init: np.ndarray         # float64 [H*10]
    mean_true: np.ndarray          # float64 [3]
    W: int
    spp: int
    noise: dict
    seed: int

    @property
    def n_theta(self) -> int:
        return 10 * self.n_handles

    @property
    def n_samples(self) -> int:
        return self.W * self.W * self.spp


SEGMENT_CONFIGS = {
    # the paper's optimiser state: 500 handles on a 256^2 image at 16 spp
    "seg500": dict(H=500, W=256, spp=16, noise="lognormal", sigma=0.3, firefly=0.01,
                   firefly_gain=20.0, seed=1006),
}


def make_segment_scene(cfg="seg500", seed: int | None = None, **over) -> SegmentScene:
    """Random segment handles: endpoint a uniform in [0.05, 0.95]^2, direction
    uniform, length uniform in [0.025, 0.1] (around the paper's initial 1/20 of
    the image width), b clipped to [0.02, 0.98]^2; jumps as for curves
    (w_d = c+ - c- with colours U[0,1]^3, w_c ~ U[-0.5, 0.5]^3).  theta_init
    moves endpoints by N(0, 0.01^2) and jumps by N(0, 0.1^2)."""
    spec = dict(SEGMENT_CONFIGS[cfg]) if isinstance(cfg, str) else dict(cfg)
    spec.update(over)
    seed = spec.get("seed", 0) if seed is None else seed
    rs = _streams(seed)
    H = int(spec["H"])
    g = rs[_GEOM]
    a = g.uniform(0.05, 0.95, size=(H, 2))
    ang = g.uniform(0.0, 2.0 * math.pi, size=H)
    ln = g.uniform(0.025, 0.1, size=H)
    b = np.clip(a + ln[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1), 0.02, 0.98)
    c_plus = rs[_COLOR].uniform(0.0, 1.0, size=(H, 3))
    c_minus = rs[_COLOR].uniform(0.0, 1.0, size=(H, 3))
    wc = rs[_COLOR].uniform(-0.5, 0.5, size=(H, 3))
    th = np.concatenate([a, b, c_plus - c_minus, wc], 1)
    mean_true = rs[_MEAN].uniform(0.25, 0.75, size=3)
    p = rs[_PERTURB]
    init = th.copy()
    init[:, 0:4] += p.normal(0.0, spec.get("pos_sigma", 0.01), size=(H, 4))
    init[:, 4:10] += p.normal(0.0, spec.get("color_sigma", 0.1), size=(H, 6))
    noise = {k: spec[k] for k in ("noise", "sigma", "firefly", "firefly_gain") if k in spec}
    return SegmentScene(n_handles=H, theta_true=th.reshape(-1), theta_init=init.reshape(-1),
                        mean_true=mean_true, W=int(spec["W"]), spp=int(spec["spp"]),
                        noise=noise, seed=seed)
