"""Oracle BEM + Levenberg-Marquardt in plain FP64 NumPy (test infrastructure).

Follows the paper's Sec. 3 and Sec. 4 step by step:

  Sec. 3.1.3   the image boundary (the unit square) is cut into equal straight
               segments with a piecewise-constant unknown; the Galerkin system
               of Eq. (bie_galerkin) is assembled with 3-point Gauss quadrature
               over the test segment and the exact inner integral; the
               coincident term is zero.
  Sec. 3.1.3   the system has a one-dimensional null space (constants); it is
               solved with the SVD, the smallest singular value dropped.
  Eq. (bie)    interior colour = mean colour + boundary double layer + handle term.
  Sec. 3.2     the Jacobian is formed column by column (forward mode): the
               handle-term derivatives plus the boundary part obtained by
               solving the same system with the stacked right-hand sides.
  Eq. (optimstep), (losshessian), (lossjacobian)
               LM step with D = diag(H), H and g as Monte Carlo sums (uniform
               density p = 1 on the unit square, the same samples for both).
  Sec. 4.3     compatibility: the step is constrained to keep
               sum_panels length * w_c = 0 (per channel) with endpoints held
               fixed, and w_c is re-projected with the new lengths afterwards.

Handles are cubic Bezier curves cut into K straight panels (uniform in the
curve parameter); the jumps of a panel are the Bernstein interpolation of its
curve's four control-handle values at the panel's mid-parameter.

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
(closed forms, brute-force quadrature, finite differences, library routines,
invariants); none is "parity unpinned".
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.sparse

from . import lib as _lib_loader

__all__ = [
    "GAUSS_NODES", "GAUSS_WEIGHTS", "square_boundary", "polygon_boundary", "gauss_points",
    "bernstein",
    "Geometry", "panelize", "compat_vectors", "project_compat", "pair_terms",
    "handle_field", "angles", "boundary_field", "assemble_A", "pinv_svd", "Oracle",
    "set_threads", "num_threads",
]

# 3-point Gauss-Legendre rule on [0, 1]
GAUSS_NODES = np.array([0.5 - math.sqrt(15.0) / 10.0, 0.5, 0.5 + math.sqrt(15.0) / 10.0])
GAUSS_WEIGHTS = np.array([5.0, 8.0, 5.0]) / 18.0


def _p(a):
    import ctypes
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(_lib_loader().orc_num_threads())


def set_threads(k: int) -> None:
    _lib_loader().orc_set_num_threads(int(k))


# ---------------------------------------------------------------------------
# image boundary

def square_boundary(M: int) -> np.ndarray:
    """Segments of the counter-clockwise boundary of [0,1]^2, M per side.

    Returns [4M, 4] = (ax, ay, bx, by); sides in the order bottom, right,
    top, left.  The right normal of each segment points out of the square.
    """
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    dirs = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, -1.0]])
    seg = np.empty((4 * M, 4))
    m = np.arange(M)
    for s in range(4):
        a = corners[s] + dirs[s] * (m / M)[:, None]
        b = corners[s] + dirs[s] * ((m + 1) / M)[:, None]
        seg[s * M:(s + 1) * M, 0:2] = a
        seg[s * M:(s + 1) * M, 2:4] = b
    return seg


def polygon_boundary(verts, M: int) -> np.ndarray:
    """Segments of a closed counter-clockwise polygon (a subdomain boundary,
    Sec. 4.2): each edge v_e -> v_{e+1} cut into M equal segments, [V M, 4]."""
    v = np.asarray(verts, np.float64).reshape(-1, 2)
    V = v.shape[0]
    seg = np.empty((V * M, 4))
    m = np.arange(M)
    for e in range(V):
        a, b = v[e], v[(e + 1) % V]
        seg[e * M:(e + 1) * M, 0:2] = a + (b - a) * (m / M)[:, None]
        seg[e * M:(e + 1) * M, 2:4] = a + (b - a) * ((m + 1) / M)[:, None]
    return seg


def gauss_points(seg: np.ndarray) -> np.ndarray:
    """Gauss points of every segment, [Nb, 3, 2]."""
    a = seg[:, None, 0:2]
    b = seg[:, None, 2:4]
    g = GAUSS_NODES[None, :, None]
    return a + g * (b - a)


# ---------------------------------------------------------------------------
# curves -> panels

def bernstein(t) -> np.ndarray:
    """Cubic Bernstein basis [..., 4] at t."""
    t = np.asarray(t, np.float64)[..., None]
    k = np.arange(4)
    binom = np.array([1.0, 3.0, 3.0, 1.0])
    return binom * t ** k * (1.0 - t) ** (3 - k)


@dataclasses.dataclass
class Geometry:
    """Discretisation of the handles into straight panels.

    Two parametrisations share one layout: colour owners of pp position
    parameters followed by w_d (RGB) and w_c (RGB), stride pp + 6.
      Bezier curves (pp = 2): 4 control handles per curve (x, y, w_d, w_c)
      segments (pp = 4):      the paper's handles, endpoints a, b and jumps
                              constant over the handle (Sec. 4.2), one panel each
    """
    n_curves: int
    K: np.ndarray          # panels per curve
    closed: np.ndarray     # bool per curve
    curve: np.ndarray      # curve index of each panel
    k: np.ndarray          # panel index within its curve
    Tgeo: scipy.sparse.csr_matrix   # [4P, n_theta] d(ax, ay, bx, by)/d theta
    Tmid: np.ndarray                # [P, n_owner] colour weights of the panels
    pp: int = 2                     # position parameters per colour owner

    @property
    def stride(self):
        return self.pp + 6

    @property
    def n_owner(self):
        return 4 * self.n_curves if self.pp == 2 else self.n_curves

    @property
    def n_theta(self):
        return self.stride * self.n_owner

    @staticmethod
    def build_segments(n_handles: int) -> "Geometry":
        """H independent straight handles: panel h = handle h."""
        H = int(n_handles)
        rows = np.arange(4 * H)
        cols = (rows // 4) * 10 + rows % 4
        Tgeo = scipy.sparse.csr_matrix((np.ones(4 * H), (rows, cols)), shape=(4 * H, 10 * H))
        return Geometry(H, np.ones(H, np.int64), np.zeros(H, bool), np.arange(H),
                        np.zeros(H, np.int64), Tgeo, np.eye(H), pp=4)

    @property
    def P(self):
        return int(self.K.sum())

    @staticmethod
    def build(n_curves: int, panels_per_curve, closed) -> "Geometry":
        C = int(n_curves)
        K = np.asarray(panels_per_curve, np.int64).reshape(C)
        closed = np.asarray(closed).astype(bool).reshape(C)
        curve = np.repeat(np.arange(C), K)
        kk = np.concatenate([np.arange(K[i]) for i in range(C)]) if C else np.zeros(0, int)
        P = int(K.sum())
        rows, cols, vals = [], [], []
        Tmid = np.zeros((P, 4 * C))
        for p in range(P):
            i, k, Ki = curve[p], kk[p], K[curve[p]]
            w0 = bernstein(k / Ki)
            w1 = bernstein((k + 1) / Ki)
            wm = bernstein((k + 0.5) / Ki)
            for j in range(4):
                jj = 0 if (closed[i] and j == 3) else j   # closed loop: p3 is p0
                base = (i * 4 + jj) * 8
                for e, (w, off) in enumerate(((w0[j], 0), (w0[j], 1), (w1[j], 0), (w1[j], 1))):
                    rows.append(4 * p + e)
                    cols.append(base + off)
                    vals.append(w)
                Tmid[p, i * 4 + j] = wm[j]
        Tgeo = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(4 * P, 32 * C))
        Tgeo.sum_duplicates()
        return Geometry(C, K, closed, curve, kk, Tgeo, Tmid)

    def active(self) -> np.ndarray:
        """Free parameters: all but the duplicated end point of closed loops."""
        m = np.ones(self.n_theta, bool)
        if self.pp != 2:
            return m
        for i in np.nonzero(self.closed)[0]:
            m[(i * 4 + 3) * 8 + 0] = False
            m[(i * 4 + 3) * 8 + 1] = False
        return m


def panelize(geo: Geometry, theta: np.ndarray):
    """Panel endpoints ab [P, 4] and jumps wd, wc [P, 3] of a parameter vector."""
    ab = (geo.Tgeo @ theta).reshape(-1, 4)
    th = theta.reshape(-1, geo.stride)   # per colour owner
    wd = geo.Tmid @ th[:, geo.pp:geo.pp + 3]
    wc = geo.Tmid @ th[:, geo.pp + 3:geo.pp + 6]
    return ab, wd, wc


def compat_vectors(geo: Geometry, theta: np.ndarray) -> np.ndarray:
    """a_h = sum over the panels of h's curve of length * Bernstein weight.

    The compatibility condition (Sec. 3.1.2) for piecewise-constant w_c reads
    sum_p length_p w_c,p = sum_h a_h w_c,h = 0 per channel.
    """
    ab, _, _ = panelize(geo, theta)
    ell = np.hypot(ab[:, 2] - ab[:, 0], ab[:, 3] - ab[:, 1])
    return geo.Tmid.T @ ell


def project_compat(geo: Geometry, theta: np.ndarray) -> np.ndarray:
    """Orthogonal projection of w_c onto the compatibility hyperplane (Sec. 4.3)."""
    a = compat_vectors(geo, theta)
    th = theta.reshape(-1, geo.stride).copy()
    aa = float(a @ a)
    if aa > 0.0:
        for c in range(3):
            w = th[:, geo.pp + 3 + c]
            th[:, geo.pp + 3 + c] = w - a * (a @ w) / aa
    return th.reshape(-1)


# ---------------------------------------------------------------------------
# per-pair terms (C)

def pair_terms(xy, ab, eps_d, eps_c, grad=False):
    xy = np.ascontiguousarray(xy, np.float64)
    ab = np.ascontiguousarray(ab, np.float64)
    n, P = xy.shape[0], ab.shape[0]
    S = np.empty((n, P))
    Dl = np.empty((n, P))
    dS = np.empty((n, P, 4)) if grad else None
    dD = np.empty((n, P, 4)) if grad else None
    import ctypes
    null = ctypes.POINTER(ctypes.c_double)()
    _lib_loader().orc_pair_terms(n, _p(xy), P, _p(ab), eps_d, eps_c, _p(S), _p(Dl),
                                 _p(dS) if grad else null, _p(dD) if grad else null)
    return (S, Dl, dS, dD) if grad else (S, Dl)


def handle_field(xy, ab, wd, wc, eps_d, eps_c):
    xy = np.ascontiguousarray(xy, np.float64)
    ab = np.ascontiguousarray(ab, np.float64)
    wd = np.ascontiguousarray(wd, np.float64)
    wc = np.ascontiguousarray(wc, np.float64)
    out = np.empty((xy.shape[0], 3))
    _lib_loader().orc_handle_field(xy.shape[0], _p(xy), ab.shape[0], _p(ab), _p(wd), _p(wc),
                                   eps_d, eps_c, _p(out))
    return out


def angles(xy, seg):
    xy = np.ascontiguousarray(xy, np.float64)
    seg = np.ascontiguousarray(seg, np.float64)
    out = np.empty((xy.shape[0], seg.shape[0]))
    _lib_loader().orc_angles(xy.shape[0], _p(xy), seg.shape[0], _p(seg), _p(out))
    return out


def boundary_field(xy, seg, ub):
    xy = np.ascontiguousarray(xy, np.float64)
    seg = np.ascontiguousarray(seg, np.float64)
    ub = np.ascontiguousarray(ub, np.float64)
    out = np.empty((xy.shape[0], 3))
    _lib_loader().orc_boundary_field(xy.shape[0], _p(xy), seg.shape[0], _p(seg), _p(ub), _p(out))
    return out


# ---------------------------------------------------------------------------
# Galerkin system and its pseudo-inverse

def assemble_A(seg: np.ndarray, mode: int = 0) -> np.ndarray:
    """Galerkin matrix of Eq. (bie_galerkin).

    A_ii = |G_i| / 2 (the coincident double-layer term is zero for a straight
    segment); A_ij = int_{G_i} int_{G_j} dG/dn_y dy dx with the outer
    integral by 3-point Gauss and the inner one
      mode 0: exact, -phi_j(x)/2pi (the signed angle segment j subtends);
      mode 1: 3-point Gauss as well (the paper's 3 x 3 rule), with
              dG/dn_y = -(1/2pi) n_y.(y - x)/|y - x|^2, n_y the right normal.
    """
    Nb = seg.shape[0]
    ell = np.hypot(seg[:, 2] - seg[:, 0], seg[:, 3] - seg[:, 1])
    gp = gauss_points(seg).reshape(-1, 2)                 # [3 Nb, 2]
    if mode == 0:
        inner = -angles(gp, seg) / (2.0 * math.pi)        # [3 Nb, Nb]
    elif mode == 1:
        a, b = seg[:, 0:2], seg[:, 2:4]
        tau = (b - a) / ell[:, None]
        nrm = np.stack([tau[:, 1], -tau[:, 0]], 1)        # right normal
        y = gauss_points(seg)                             # [Nb, 3, 2]
        inner = np.empty((gp.shape[0], Nb))
        for r0 in range(0, gp.shape[0], 256):
            x = gp[r0:r0 + 256]
            d = y[None, :, :, :] - x[:, None, None, :]    # [r, Nb, 3, 2]
            r2 = np.sum(d * d, axis=-1)
            num = np.sum(d * nrm[None, :, None, :], axis=-1)
            with np.errstate(invalid="ignore", divide="ignore"):
                k = np.where(r2 > 0, num / r2, 0.0)
            inner[r0:r0 + 256] = -(ell[None, :] / (2.0 * math.pi)) * (k @ GAUSS_WEIGHTS)
    else:
        raise ValueError(f"galerkin mode {mode}")
    A = ell[:, None] * np.einsum("q,iqj->ij", GAUSS_WEIGHTS, inner.reshape(Nb, 3, Nb))
    A[np.arange(Nb), np.arange(Nb)] = 0.5 * ell
    return A


def pinv_svd(A: np.ndarray) -> np.ndarray:
    """Pseudo-inverse with the smallest singular value discarded (Sec. 3.1.3)."""
    U, s, Vt = np.linalg.svd(A)
    r = len(s) - 1
    return (Vt[:r].T / s[:r]) @ U[:, :r].T


# ---------------------------------------------------------------------------

class Oracle:
    """FP64 reference of one scene: fixed boundary, varying handle parameters."""

    def __init__(self, n_curves, panels_per_curve, closed, mean_color,
                 segs_per_side: int = 256, eps_d: float = 1e-2, eps_c: float = 1e-2,
                 galerkin_mode: int = 0, polygon=None):
        self.geo = (Geometry.build_segments(n_curves) if panels_per_curve is None
                    else Geometry.build(n_curves, panels_per_curve, closed))
        self.mean = np.asarray(mean_color, np.float64).reshape(3)
        self.eps_d = float(eps_d)
        self.eps_c = float(eps_c)
        # the unit square, or a counter-clockwise polygon with segs_per_side
        # segments per edge (one subdomain)
        self.seg = (square_boundary(segs_per_side) if polygon is None
                    else polygon_boundary(polygon, segs_per_side))
        self.Nb = self.seg.shape[0]
        self.ell = np.hypot(self.seg[:, 2] - self.seg[:, 0], self.seg[:, 3] - self.seg[:, 1])
        self.gp = gauss_points(self.seg)                 # [Nb, 3, 2]
        self.A = assemble_A(self.seg, galerkin_mode)
        self.Apinv = pinv_svd(self.A)

    @staticmethod
    def segments(n_handles, mean_color, **kw) -> "Oracle":
        """The paper's parametrisation: n_handles straight handles of 10
        parameters (a, b, w_d RGB, w_c RGB)."""
        return Oracle(n_handles, None, None, mean_color, **kw)

    @staticmethod
    def from_scene(scene, mean_color=None, **kw) -> "Oracle":
        m = scene.mean_true if mean_color is None else mean_color
        return Oracle(scene.n_curves, scene.panels_per_curve, scene.closed, m, **kw)

    # ---- forward ---------------------------------------------------------
    def panels(self, theta):
        return panelize(self.geo, theta)

    def rhs(self, theta) -> np.ndarray:
        """f_b,i = int_{G_i} f dx by 3-point Gauss, [Nb, 3]."""
        ab, wd, wc = self.panels(theta)
        f = handle_field(self.gp.reshape(-1, 2), ab, wd, wc, self.eps_d, self.eps_c)
        f = f.reshape(self.Nb, 3, 3)
        return self.ell[:, None] * np.einsum("q,iqc->ic", GAUSS_WEIGHTS, f)

    def boundary_values(self, theta) -> np.ndarray:
        """Zero-mean boundary solution u_b = A^+ f_b, [Nb, 3]."""
        return self.Apinv @ self.rhs(theta)

    def eval(self, theta, xy, ub=None) -> np.ndarray:
        """Interior colour u(x) = mean + sum_j phi_j/2pi u_b,j + f(x), [n, 3]."""
        if ub is None:
            ub = self.boundary_values(theta)
        ab, wd, wc = self.panels(theta)
        return (self.mean + boundary_field(xy, self.seg, ub)
                + handle_field(xy, ab, wd, wc, self.eps_d, self.eps_c))

    def loss(self, theta, xy, target) -> float:
        r = self.eval(theta, xy) - np.minimum(target, 1.0)
        return 0.5 * float(np.sum(r * r)) / xy.shape[0]

    # ---- Jacobian (forward mode) -----------------------------------------
    def handle_jac(self, theta, xy) -> np.ndarray:
        """d f_c(x) / d theta for every point, [n, 3, n_theta]."""
        geo = self.geo
        ab, wd, wc = self.panels(theta)
        S, Dl, dS, dD = pair_terms(xy, ab, self.eps_d, self.eps_c, grad=True)
        n = xy.shape[0]
        F = np.zeros((n, 3, geo.n_theta))
        hidx = np.arange(geo.n_owner) * geo.stride
        colD = -Dl @ geo.Tmid            # [n, n_owner] d f_c / d w_d,c of each colour owner
        colS = S @ geo.Tmid              # [n, n_owner] d f_c / d w_c,c
        for c in range(3):
            G = -wd[None, :, c, None] * dD + wc[None, :, c, None] * dS   # [n, P, 4]
            F[:, c, :] = (geo.Tgeo.T @ G.reshape(n, -1).T).T
            F[:, c, hidx + geo.pp + c] += colD
            F[:, c, hidx + geo.pp + 3 + c] += colS
        return F

    def boundary_jac(self, theta) -> np.ndarray:
        """d u_b / d theta = A^+ d f_b / d theta (stacked right-hand sides), [Nb, 3, n_theta]."""
        Fg = self.handle_jac(theta, self.gp.reshape(-1, 2)).reshape(self.Nb, 3, 3, -1)
        dfb = self.ell[:, None, None] * np.einsum("q,iqct->ict", GAUSS_WEIGHTS, Fg)
        return np.einsum("ij,jct->ict", self.Apinv, dfb)

    def jac(self, theta, xy, Mb=None) -> np.ndarray:
        """Image-space Jacobian J(x) = du/dtheta, [n, 3, n_theta]."""
        if Mb is None:
            Mb = self.boundary_jac(theta)
        Phi = angles(xy, self.seg) / (2.0 * math.pi)      # [n, Nb]
        J = self.handle_jac(theta, xy)
        for c in range(3):
            J[:, c, :] += Phi @ Mb[:, c, :]
        return J

    def gauss_newton(self, theta, xy, target, chunk: int = 512):
        """Loss, g = (1/S) sum J^T r and H = (1/S) sum J^T J (Eq. losshessian/lossjacobian)."""
        n = xy.shape[0]
        t = np.minimum(target, 1.0)
        ub = self.boundary_values(theta)
        Mb = self.boundary_jac(theta)
        nt = self.geo.n_theta
        g = np.zeros(nt)
        H = np.zeros((nt, nt))
        L = 0.0
        for s0 in range(0, n, chunk):
            x = xy[s0:s0 + chunk]
            r = self.eval(theta, x, ub) - t[s0:s0 + chunk]
            J = self.jac(theta, x, Mb)
            L += 0.5 * float(np.sum(r * r))
            g += np.einsum("sct,sc->t", J, r)
            Jf = J.reshape(-1, nt)
            H += Jf.T @ Jf
        return L / n, g / n, H / n

    def grad(self, theta, xy, resid, chunk: int = 512) -> np.ndarray:
        """J^T resid (no 1/S), the vector-Jacobian product of the evaluation."""
        Mb = self.boundary_jac(theta)
        g = np.zeros(self.geo.n_theta)
        for s0 in range(0, xy.shape[0], chunk):
            J = self.jac(theta, xy[s0:s0 + chunk], Mb)
            g += np.einsum("sct,sc->t", J, resid[s0:s0 + chunk])
        return g

    # ---- LM ------------------------------------------------------------------
    def constraint_matrix(self, theta) -> np.ndarray:
        """Columns = compatibility constraint of each channel on theta, [n_theta, 3]."""
        a = compat_vectors(self.geo, theta)
        Ac = np.zeros((self.geo.n_theta, 3))
        idx = np.arange(self.geo.n_owner) * self.geo.stride
        for c in range(3):
            Ac[idx + self.geo.pp + 3 + c, c] = a
        return Ac

    def solve_step(self, theta, H, g, lam, free=None) -> np.ndarray:
        """delta minimising the damped model on the compatibility subspace.

        (H + lam D) delta + Ac mu = -g,  Ac^T delta = 0,  D = diag(H) floored
        at 1e-12 max diag(H); Cholesky of H + lam D and a 3x3 Schur complement.
        `free` (optional bool mask) freezes the parameters it leaves out.

        H is positive semi-definite only up to rounding.  When H + lam D does
        not factor, lam is raised tenfold (a zero lam becomes 1e-9) and the
        factorisation tried again, 13 attempts in all; the lam that factored
        (or the last one tried, when every attempt failed and LinAlgError is
        raised) is left in self.last_lambda.
        """
        act = self.geo.active()
        if free is not None:
            act = act & np.asarray(free, bool)
        Ha = H[np.ix_(act, act)]
        ga = g[act]
        dg = np.diag(Ha).copy()
        D = np.maximum(dg, 1e-12 * dg.max())
        for attempt in range(13):
            self.last_lambda = lam
            try:
                cf = scipy.linalg.cho_factor(Ha + lam * np.diag(D), lower=True)
                break
            except np.linalg.LinAlgError:
                if attempt == 12:
                    raise
                lam = 10.0 * lam if lam > 0 else 1e-9
        Ac = self.constraint_matrix(theta)[act]
        y = scipy.linalg.cho_solve(cf, -ga)
        Z = scipy.linalg.cho_solve(cf, Ac)
        mu = np.linalg.solve(Ac.T @ Z, Ac.T @ y)
        da = y - Z @ mu
        delta = np.zeros(self.geo.n_theta)
        delta[act] = da
        return delta

    def hessian(self, theta, xy, chunk: int = 512) -> np.ndarray:
        """H = (1/M_H) sum over the M_H points of J^T J (Eq. losshessian, p = 1)."""
        Mb = self.boundary_jac(theta)
        nt = self.geo.n_theta
        H = np.zeros((nt, nt))
        for s0 in range(0, xy.shape[0], chunk):
            Jf = self.jac(theta, xy[s0:s0 + chunk], Mb).reshape(-1, nt)
            H += Jf.T @ Jf
        return H / xy.shape[0]

    def lm_step(self, theta, xy, target, lam, xy_h=None, reg=None):
        """One LM iteration (Eq. optimstep) with the paper's two-stage projection.
        With xy_h, the Hessian integral uses those M_H points and the gradient
        and the losses the M_J points xy (Sec. 4.3, Monte Carlo integration).
        With reg (segment handles, a regularize.RegParams), the Sec. 4.4
        losses add their analytic gradient and Hessian to g and H and their
        values to both losses; the snapping pairs are chosen once, at theta.

        lam is one damping value or a sequence of trial values.  Every trial
        solves the damped system (raising its lam tenfold while H + lam D
        does not factor, see solve_step) and evaluates the loss at its
        re-projected theta on the same samples.  The trial with the lowest
        loss (the first of equal ones) is taken if its loss is below the
        current one.  The damping schedule after Transtrum & Sethna, whose
        constants the paper does not give: the taken trial's lam / 3 after
        an accepted step; after a rejected one 2 lam with a single trial and
        10 times the largest lam tried with several.  A trial whose matrix
        never factors is skipped (its last lam still counts in that maximum);
        LinAlgError if no trial factors."""
        lams = [float(v) for v in np.atleast_1d(np.asarray(lam, np.float64))]
        L0, g, H = self.gauss_newton(theta, xy, target)
        if xy_h is not None:
            H = self.hessian(theta, xy_h)
        pairs = None
        if reg is not None:
            from . import regularize
            pairs = regularize.snap_pairs(theta, reg)
            gr, Hr = regularize.reg_grad_hess(theta, reg, pairs)
            g, H = g + gr, H + Hr
            L0 += regularize.reg_loss(theta, reg, pairs)
        used, losses, trials, deltas = [], [], [], []
        for lt in lams:
            try:
                delta = self.solve_step(theta, H, g, lt)
            except np.linalg.LinAlgError:
                used.append(self.last_lambda)
                losses.append(math.inf)
                trials.append(None)
                deltas.append(None)
                continue
            used.append(self.last_lambda)
            th_new = project_compat(self.geo, theta + delta)
            L1 = self.loss(th_new, xy, target)
            if reg is not None:
                L1 += regularize.reg_loss(th_new, reg, pairs)
            losses.append(L1)
            trials.append(th_new)
            deltas.append(delta)
        if all(t is None for t in trials):
            raise np.linalg.LinAlgError("no trial's damped matrix factors")
        best = int(np.argmin(losses))          # first of equal minima
        accept = losses[best] < L0
        if accept:
            lam_next = used[best] / 3.0
        else:
            lam_next = 2.0 * used[0] if len(lams) == 1 else 10.0 * max(used)
        return dict(loss_before=L0, loss_after=losses[best], accepted=bool(accept),
                    best_trial=best if accept else -1, lambda_next=lam_next,
                    lambdas_used=used, trial_losses=losses,
                    theta=trials[best] if accept else theta.copy(), theta_trial=trials[best],
                    delta=deltas[best], g=g, H=H)
