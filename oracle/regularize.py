"""Oracle of the regularisers, pruning and initialisation for segment handles
(test infrastructure, plain FP64 NumPy).

The paper's handles are independent straight segments theta[h] = (a, b, w_d
RGB, w_c RGB) (Sec. 4.2).  Sec. 4.4 adds three optional losses to the
reconstruction loss; each contributes its analytic gradient and Hessian to
the Gauss-Newton gradient and matrix of the LM step (Eq. optimstep):

  handle length  lam_len * (|b - a| - l_max)^2 for handles longer than l_max,
                 nothing otherwise;
  snapping       lam_snap * |p - q|^2 for each pair of endpoints p, q of two
                 different handles that are closer than r_snap and pick each
                 other as the lowest snapping score
                   s(p, q) = alpha |p - q| / r_snap + (1 - alpha)(1 - |d_p . d_q|)
                 (d = the unit directions of the two handles, the dot product
                 taken in absolute value because a segment's orientation a->b
                 carries no meaning for its line);
  sparsity       lam_w t tanh(sqrt(w.w + eps^2) / t) for w = w_d (lam_d) and
                 w = w_c (lam_c) of every handle.

Reading of the sparsity Hessian: the exact Hessian of the saturated term is
lam s (I / rho - w w^T / rho^3) - lam s (2 tanh(rho/t) / (t rho^2)) w w^T
with s = sech^2(rho / t); the second part is the negative curvature of the
saturation and can turn diagonal entries of H negative, and then H + lam D
with D = diag(H) (floored) does not factor for any damping.  H receives the
first, positive semidefinite part only (the saturation factor s held fixed
at the current w); the gradient and the loss are exact.

Pruning (Sec. 4.4, Sparsity): a handle whose |w_d| and |w_c| are both below a
threshold is removed; w_c is then re-projected onto the compatibility
hyperplane of the remaining handles (Sec. 4.3).

Initialisation (Sec. 4.2): the first endpoint of handle k is the k-th point of
the two-dimensional Sobol sequence (scipy's unscrambled generator), its
direction angle 2 pi times the base-3 radical inverse of k (a stated stand-in
for the third Sobol coordinate), its length a given fraction of the image
width; the second endpoint is pulled back along the handle to the first
crossing with the subdomain's boundary polygon, so that each handle lies in
the subdomain of its first endpoint.  Only sequence points whose first
endpoint lies inside the polygon make handles.  The jumps start at zero.

Parity status: every function is pinned in tests/test_oracle_regularize.py
(closed-form values, central differences of the losses, brute-force pair
choice on hand-built layouts, the radical inverse's exact values, scipy's
Sobol points).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .bem import Geometry, project_compat

__all__ = ["RegParams", "reg_loss", "reg_grad_hess", "snap_pairs", "prune",
           "radical_inverse", "point_in_polygon", "init_segments"]


@dataclasses.dataclass
class RegParams:
    """Weights and shapes of the Sec. 4.4 losses (a zero weight turns one off)."""
    len_weight: float = 0.0
    len_max: float = 0.1
    snap_weight: float = 0.0
    snap_radius: float = 0.02
    snap_alpha: float = 0.5
    sparse_wd: float = 0.0
    sparse_wc: float = 0.0
    sparse_eps: float = 1e-3
    sparse_t: float = 0.05


def _handles(theta):
    th = np.asarray(theta, np.float64).reshape(-1, 10)
    return th[:, 0:2], th[:, 2:4], th[:, 4:7], th[:, 7:10]


def _endpoint(theta, e):
    """Endpoint e (= 2 h + 0 for a_h, 2 h + 1 for b_h) as a 2-vector."""
    th = np.asarray(theta).reshape(-1, 10)
    h, k = divmod(int(e), 2)
    return th[h, 2 * k:2 * k + 2]


def snap_pairs(theta, rp: RegParams) -> list[tuple[int, int]]:
    """Mutually best endpoint pairs (p < q) by the snapping score.

    Endpoint e = 2 h + s: s = 0 for a_h, 1 for b_h.  Candidates of p are the
    endpoints q of other handles with |p - q| < r_snap; p's choice is the
    candidate of lowest score, ties to the lower index.
    """
    a, b, _, _ = _handles(theta)
    H = a.shape[0]
    d = b - a
    ln = np.hypot(d[:, 0], d[:, 1])
    u = np.zeros_like(d)
    nz = ln > 0
    u[nz] = d[nz] / ln[nz, None]
    E = 2 * H
    pts = np.empty((E, 2))
    pts[0::2], pts[1::2] = a, b
    best = np.full(E, -1)
    for p in range(E):
        bs = math.inf
        for q in range(E):
            if q // 2 == p // 2:
                continue
            dist = math.hypot(pts[p, 0] - pts[q, 0], pts[p, 1] - pts[q, 1])
            if not dist < rp.snap_radius:
                continue
            cos = abs(u[p // 2, 0] * u[q // 2, 0] + u[p // 2, 1] * u[q // 2, 1])
            s = rp.snap_alpha * dist / rp.snap_radius + (1.0 - rp.snap_alpha) * (1.0 - cos)
            if s < bs:
                bs, best[p] = s, q
    return [(p, int(best[p])) for p in range(E) if best[p] > p and best[best[p]] == p]


def reg_loss(theta, rp: RegParams, pairs=None) -> float:
    """Sum of the three losses at theta (pairs: fixed snapping pairs, else chosen at theta)."""
    a, b, wd, wc = _handles(theta)
    L = 0.0
    if rp.len_weight > 0:
        ln = np.hypot(b[:, 0] - a[:, 0], b[:, 1] - a[:, 1])
        ex = np.maximum(ln - rp.len_max, 0.0)
        L += rp.len_weight * float(np.sum(ex * ex))
    if rp.snap_weight > 0:
        if pairs is None:
            pairs = snap_pairs(theta, rp)
        for p, q in pairs:
            dv = _endpoint(theta, p) - _endpoint(theta, q)
            L += rp.snap_weight * float(dv @ dv)
    for lam, w in ((rp.sparse_wd, wd), (rp.sparse_wc, wc)):
        if lam > 0:
            rho = np.sqrt(np.sum(w * w, 1) + rp.sparse_eps ** 2)
            L += lam * rp.sparse_t * float(np.sum(np.tanh(rho / rp.sparse_t)))
    return L


def reg_grad_hess(theta, rp: RegParams, pairs=None):
    """Analytic gradient [10H] and Hessian [10H, 10H] of reg_loss (Sec. 4.4);
    the sparsity part of the Hessian without its saturation curvature."""
    a, b, wd, wc = _handles(theta)
    H = a.shape[0]
    n = 10 * H
    g = np.zeros(n)
    Hm = np.zeros((n, n))
    I2 = np.eye(2)
    if rp.len_weight > 0:
        lam = rp.len_weight
        for h in range(H):
            e = b[h] - a[h]
            ln = math.hypot(e[0], e[1])
            k = ln - rp.len_max
            if not k > 0:
                continue
            u = e / ln
            gb = 2.0 * lam * k * u               # d/db of lam (|b - a| - l)^2
            M = 2.0 * lam * (np.outer(u, u) + (k / ln) * (I2 - np.outer(u, u)))
            ia, ib = 10 * h, 10 * h + 2
            g[ia:ia + 2] -= gb
            g[ib:ib + 2] += gb
            Hm[ia:ia + 2, ia:ia + 2] += M
            Hm[ib:ib + 2, ib:ib + 2] += M
            Hm[ia:ia + 2, ib:ib + 2] -= M
            Hm[ib:ib + 2, ia:ia + 2] -= M
    if rp.snap_weight > 0:
        if pairs is None:
            pairs = snap_pairs(theta, rp)
        lam = rp.snap_weight
        for p, q in pairs:
            ip = 10 * (p // 2) + 2 * (p % 2)
            iq = 10 * (q // 2) + 2 * (q % 2)
            dv = _endpoint(theta, p) - _endpoint(theta, q)
            g[ip:ip + 2] += 2.0 * lam * dv
            g[iq:iq + 2] -= 2.0 * lam * dv
            Hm[ip:ip + 2, ip:ip + 2] += 2.0 * lam * I2
            Hm[iq:iq + 2, iq:iq + 2] += 2.0 * lam * I2
            Hm[ip:ip + 2, iq:iq + 2] -= 2.0 * lam * I2
            Hm[iq:iq + 2, ip:ip + 2] -= 2.0 * lam * I2
    I3 = np.eye(3)
    for lam, w, off in ((rp.sparse_wd, wd, 4), (rp.sparse_wc, wc, 7)):
        if not lam > 0:
            continue
        t = rp.sparse_t
        for h in range(H):
            v = w[h]
            rho = math.sqrt(float(v @ v) + rp.sparse_eps ** 2)
            th_ = math.tanh(rho / t)
            s = 1.0 - th_ * th_                  # sech^2(rho / t)
            i = 10 * h + off
            g[i:i + 3] += lam * s * v / rho
            Hm[i:i + 3, i:i + 3] += lam * s * (I3 / rho - np.outer(v, v) / rho ** 3)
    return g, Hm


def prune(theta, threshold: float):
    """Remove handles with |w_d| < threshold and |w_c| < threshold, then
    re-project w_c of the rest; returns (theta, kept handle indices)."""
    _, _, wd, wc = _handles(theta)
    keep = np.nonzero(~((np.linalg.norm(wd, axis=1) < threshold) &
                        (np.linalg.norm(wc, axis=1) < threshold)))[0]
    th = np.asarray(theta).reshape(-1, 10)[keep].reshape(-1)
    if keep.size:
        th = project_compat(Geometry.build_segments(keep.size), th)
    return th, keep


def radical_inverse(k: int, base: int) -> float:
    """Digits of k in the given base mirrored about the radix point."""
    x, f = 0.0, 1.0 / base
    while k > 0:
        k, d = divmod(k, base)
        x += d * f
        f /= base
    return x


def point_in_polygon(x, y, poly) -> bool:
    """Even-odd rule: a horizontal ray to +x crosses the boundary an odd number of times."""
    V = len(poly)
    inside = False
    for i in range(V):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % V]
        if (y0 > y) != (y1 > y):
            xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
            if x < xc:
                inside = not inside
    return inside


def _first_crossing(a, b, poly) -> float:
    """Smallest t in (0, 1] where a + t (b - a) meets an edge of the polygon, else 1."""
    t_hit = 1.0
    dx, dy = b[0] - a[0], b[1] - a[1]
    V = len(poly)
    for i in range(V):
        px, py = poly[i]
        qx, qy = poly[(i + 1) % V]
        ex, ey = qx - px, qy - py
        den = dx * ey - dy * ex
        if den == 0.0:
            continue
        wx, wy = px - a[0], py - a[1]
        t = (wx * ey - wy * ex) / den           # along the handle
        s = (wx * dy - wy * dx) / den           # along the edge
        if 0.0 < t <= t_hit and 0.0 <= s <= 1.0:
            t_hit = t
    return t_hit


def init_segments(n_points: int, length: float, first_index: int = 1, polygon=None):
    """Handles from the sequence points first_index .. first_index + n_points - 1
    whose first endpoint lies inside the polygon (default: the unit square)."""
    import warnings
    from scipy.stats import qmc
    poly = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)] if polygon is None else \
        [tuple(map(float, v)) for v in np.asarray(polygon).reshape(-1, 2)]
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")       # counts that are not powers of two
        pts = qmc.Sobol(d=2, scramble=False).random(first_index + n_points)[first_index:]
    out = []
    for j in range(n_points):
        k = first_index + j
        a = pts[j]
        if not point_in_polygon(a[0], a[1], poly):
            continue
        phi = 2.0 * math.pi * radical_inverse(k, 3)
        b = np.array([a[0] + length * math.cos(phi), a[1] + length * math.sin(phi)])
        t = _first_crossing(a, b, poly)
        b = a + t * (b - a)
        th = np.zeros(10)
        th[0:2], th[2:4] = a, b
        out.append(th)
    return np.concatenate(out) if out else np.zeros(0)
