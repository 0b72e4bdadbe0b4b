"""GB300 differential-BEM hot path: thin Python binding of libbemgb.

Every computation runs in the CUDA library behind the C ABI declared in
include/bemgb.h; this module only marshals arguments (torch tensors'
device pointers, the current CUDA stream, host numpy arrays).  There is no
CPU fallback: importing the binding without the built library raises.

The raw entry points are exposed under their C names (bem_create, bem_setup,
bem_factor, bem_eval, bem_loss, bem_vjp, bem_jtj, lm_step, ...); `BEM` wraps
one context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbemgb.so")

BEM_OK, BEM_EINVAL, BEM_ESTATE, BEM_ESINGULAR, BEM_ENOTSPD, BEM_ECUDA, BEM_ETIMEDOUT, BEM_ENOMEM = \
    0, -1, -2, -3, -4, -5, -6, -7
BEM_FP64, BEM_MIXED = 0, 1
BEM_JTJ_FP64, BEM_JTJ_BF16, BEM_JTJ_3XTF32, BEM_JTJ_BF16X3 = 0, 1, 2, 3
BEM_LM_AUTO, BEM_LM_FP64 = 0, 1

_STATUS = {0: "BEM_OK", -1: "BEM_EINVAL", -2: "BEM_ESTATE", -3: "BEM_ESINGULAR",
           -4: "BEM_ENOTSPD", -5: "BEM_ECUDA", -6: "BEM_ETIMEDOUT", -7: "BEM_ENOMEM"}


class bem_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps_d", ctypes.c_double),
                ("eps_c", ctypes.c_double), ("segs_per_side", ctypes.c_int),
                ("near_factor", ctypes.c_double), ("jtj_mode", ctypes.c_int),
                ("lm_solver", ctypes.c_int), ("galerkin_mode", ctypes.c_int),
                ("gn_chunk", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class lm_result(ctypes.Structure):
    _fields_ = [("loss_before", ctypes.c_double), ("loss_after", ctypes.c_double),
                ("accepted", ctypes.c_int), ("best_trial", ctypes.c_int),
                ("lambda_next", ctypes.c_double), ("grad_norm", ctypes.c_double)]


class bem_reg(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "len_weight", "len_max", "snap_weight", "snap_radius", "snap_alpha",
        "sparse_wd", "sparse_wc", "sparse_eps", "sparse_t")]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libbemgb.so is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
            f"(expected at {LIB_PATH})")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, ci, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    sig = {
        "bem_default_opts": (ci, [ctypes.POINTER(bem_opts)]),
        "bem_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(bem_opts), ci]),
        "bem_destroy": (None, [vp]),
        "bem_last_error": (ctypes.c_char_p, [vp]),
        "bem_setup": (ci, [vp, ci, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8),
                           dp, dp]),
        "bem_factor": (ci, [vp, vp]),
        "bem_setup_segments": (ci, [vp, ci, dp, dp]),
        "bem_set_boundary": (ci, [vp, ci, dp, ci]),
        "bem_set_params": (ci, [vp, vp, ci, vp]),
        "bem_get_params": (ci, [vp, dp, vp]),
        "bem_set_mean_color": (ci, [vp, dp]),
        "bem_sample_mean": (ci, [vp, i64, vp, dp, vp]),
        "bem_eval": (ci, [vp, i64, vp, vp, vp]),
        "bem_loss": (ci, [vp, i64, vp, vp, vp, dp, vp]),
        "bem_vjp": (ci, [vp, i64, vp, vp, vp, vp]),
        "bem_jtj": (ci, [vp, i64, vp, vp, vp]),
        "lm_step": (ci, [vp, i64, vp, vp, ci, dp, ctypes.POINTER(lm_result), vp]),
        "lm_step_split": (ci, [vp, i64, vp, vp, i64, vp, ci, dp, ctypes.POINTER(lm_result), vp]),
        "lm_step_host": (ci, [vp, i64, vp, vp, ci, dp, ctypes.POINTER(lm_result), vp]),
        "bem_sizes": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]),
        "bem_boundary_values": (ci, [vp, dp, vp]),
        "bem_launch_count": (i64, [vp]),
        "bem_alloc_count": (i64, [vp]),
        "bem_pipe_peak": (ci, [vp, ci, ci, dp, vp]),
        "bem_set_wait_limit": (ci, [vp, ctypes.c_double]),
        "bem_gn_products": (ci, [vp, i64, vp, vp, dp, vp, vp, vp]),
        "bem_profile_enable": (ci, [vp, ci]),
        "bem_gemm_bf16": (ci, [vp, ci, ci, ci, vp, ci, vp, ci, vp, ci, vp]),
        "bem_fastmath_eval": (ci, [vp, ci, i64, vp, vp, vp, vp, vp]),
        "bem_dlog_eval": (ci, [vp, i64, vp, vp, vp, vp]),
        "bem_datan2_eval": (ci, [vp, i64, vp, vp, vp, vp, vp]),
        "bem_vjp_noalloc": (ci, [vp, i64, vp, vp, vp, vp]),
        "bem_profile_read": (ci, [vp, ci, ctypes.c_char_p, dp, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ci)]),
        "bem_batch_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(vp), ci]),
        "bem_batch_destroy": (None, [vp]),
        "bem_batch_lm": (ci, [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp), ci,
                              dp, ctypes.POINTER(lm_result), vp]),
        "bem_batch_tile_shape": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]),
        "bem_render": (ci, [vp, ci, ci, vp, vp]),
        "bem_handle_colors": (ci, [vp, dp, vp]),
        "bem_set_regularizers": (ci, [vp, ctypes.POINTER(bem_reg)]),
        "bem_prune": (ci, [vp, ctypes.c_double, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_int32),
                           vp]),
        "bem_init_segments": (ci, [ci, ctypes.c_double, i64, ci, dp, dp, ctypes.POINTER(ci)]),
        "bem_gram_unit": (ci, [ci, ci, ci, ctypes.POINTER(ctypes.c_int32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()
EXPORTED = [
    "bem_default_opts", "bem_create", "bem_destroy", "bem_last_error", "bem_setup", "bem_factor",
    "bem_set_params", "bem_get_params", "bem_set_mean_color", "bem_sample_mean", "bem_eval",
    "bem_loss", "bem_vjp", "bem_jtj", "lm_step", "bem_sizes", "bem_boundary_values",
    "bem_launch_count", "bem_profile_enable", "bem_profile_read", "bem_gemm_bf16",
    "bem_fastmath_eval", "bem_dlog_eval", "bem_vjp_noalloc", "bem_batch_create", "bem_batch_destroy",
    "bem_batch_lm", "bem_batch_tile_shape", "bem_render", "bem_handle_colors", "lm_step_split",
    "bem_set_boundary", "bem_setup_segments", "bem_set_regularizers", "bem_prune",
    "bem_init_segments", "bem_gram_unit", "bem_alloc_count", "bem_set_wait_limit",
    "bem_gn_products", "bem_pipe_peak", "lm_step_host", "bem_datan2_eval",
]
globals().update({name: getattr(_lib, name) for name in EXPORTED})


def lib():
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _lib_sizes(m):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    m._check(_lib.bem_sizes(m.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


class BEM:
    """One library context (scene + factored boundary) on one CUDA device."""

    def __init__(self, precision=BEM_FP64, eps_d=1e-2, eps_c=1e-2, segs_per_side=256,
                 near_factor=0.5, jtj_mode=None, lm_solver=0, galerkin_mode=0, device=0,
                 gn_chunk=0):
        o = bem_opts()
        _lib.bem_default_opts(ctypes.byref(o))
        o.precision = precision
        o.eps_d, o.eps_c = eps_d, eps_c
        o.segs_per_side = segs_per_side
        o.near_factor = near_factor
        o.jtj_mode = (BEM_JTJ_FP64 if precision == BEM_FP64 else BEM_JTJ_BF16) \
            if jtj_mode is None else jtj_mode
        o.lm_solver = lm_solver
        o.galerkin_mode = galerkin_mode
        o.gn_chunk = gn_chunk
        self.opts = o
        self.device = device
        h = ctypes.c_void_p()
        rc = _lib.bem_create(ctypes.byref(h), ctypes.byref(o), device)
        if rc:
            raise BemError(rc, _lib.bem_last_error(None).decode())
        self.h = h
        self.n_theta = 0
        self.Nb = 4 * segs_per_side

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.opts.precision == BEM_FP64 else torch.float32

    def _check(self, rc):
        if rc:
            raise BemError(rc, _lib.bem_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            _lib.bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup --------------------------------------------------------------
    def setup(self, n_curves, panels_per_curve, closed, theta, mean_color):
        K = np.ascontiguousarray(panels_per_curve, np.int32)
        cl = np.ascontiguousarray(closed, np.uint8)
        th = np.ascontiguousarray(theta, np.float64)
        m = np.ascontiguousarray(mean_color, np.float64)
        self._check(_lib.bem_setup(self.h, int(n_curves),
                                   K.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   cl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   _dp(th), _dp(m)))
        self.n_theta = 32 * int(n_curves)

    def setup_segments(self, n_handles, theta, mean_color):
        """Independent straight handles, 10 parameters each (Sec. 4.2)."""
        th = np.ascontiguousarray(theta, np.float64)
        m = np.ascontiguousarray(mean_color, np.float64)
        assert th.size == 10 * int(n_handles)
        self._check(_lib.bem_setup_segments(self.h, int(n_handles), _dp(th), _dp(m)))
        self.n_theta = 10 * int(n_handles)

    def set_regularizers(self, **kw):
        """Sec. 4.4 regularisers of a segment-handle scene (bem_reg field
        names as keywords; none given clears them)."""
        if not kw:
            self._check(_lib.bem_set_regularizers(self.h, None))
            return
        r = bem_reg(len_max=0.1, snap_radius=0.02, snap_alpha=0.5, sparse_eps=1e-3,
                    sparse_t=0.05)
        for k, v in kw.items():
            if k not in dict(bem_reg._fields_):
                raise TypeError(f"unknown regulariser setting {k}")
            setattr(r, k, float(v))
        self._check(_lib.bem_set_regularizers(self.h, ctypes.byref(r)))

    def prune(self, threshold, stream=None) -> np.ndarray:
        """Remove handles whose |w_d| and |w_c| are below threshold; returns
        the former indices of the kept handles (empty: nothing removed
        because nothing would remain)."""
        H = self.n_theta // 10
        kept = np.zeros(H, np.int32)
        n = ctypes.c_int(0)
        self._check(_lib.bem_prune(self.h, float(threshold), ctypes.byref(n),
                                   kept.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   _stream(stream)))
        if n.value:
            self.n_theta = 10 * n.value
        return kept[:n.value].copy()

    def factor(self, stream=None):
        self._check(_lib.bem_factor(self.h, _stream(stream)))

    def set_params(self, theta, stream=None):
        import torch
        if isinstance(theta, torch.Tensor):
            assert theta.dtype == torch.float64 and theta.is_cuda and theta.is_contiguous()
            self._check(_lib.bem_set_params(self.h, _ptr(theta), 1, _stream(stream)))
        else:
            th = np.ascontiguousarray(theta, np.float64)
            self._check(_lib.bem_set_params(self.h, th.ctypes.data_as(ctypes.c_void_p), 0,
                                            _stream(stream)))

    def get_params(self, stream=None) -> np.ndarray:
        out = np.empty(self.n_theta)
        self._check(_lib.bem_get_params(self.h, _dp(out), _stream(stream)))
        return out

    def set_mean_color(self, mean):
        m = np.ascontiguousarray(mean, np.float64)
        self._check(_lib.bem_set_mean_color(self.h, _dp(m)))

    # ---- hot path -------------------------------------------------------------
    def _samples(self, *ts):
        for t in ts:
            assert t.is_cuda and t.dtype == self.dtype and t.is_contiguous(), \
                f"expected contiguous CUDA {self.dtype}, got {t.dtype} {t.device}"

    def sample_mean(self, target, stream=None) -> np.ndarray:
        self._samples(target)
        out = np.empty(3)
        self._check(_lib.bem_sample_mean(self.h, target.shape[0], _ptr(target), _dp(out),
                                         _stream(stream)))
        return out

    def eval(self, xy, out=None, stream=None):
        import torch
        self._samples(xy)
        if out is None:
            out = torch.empty((xy.shape[0], 3), dtype=self.dtype, device=xy.device)
        self._check(_lib.bem_eval(self.h, xy.shape[0], _ptr(xy), _ptr(out), _stream(stream)))
        return out

    def loss(self, xy, target, resid=None, stream=None) -> float:
        self._samples(xy, target)
        v = ctypes.c_double()
        self._check(_lib.bem_loss(self.h, xy.shape[0], _ptr(xy), _ptr(target),
                                  _ptr(resid) if resid is not None else None,
                                  ctypes.byref(v), _stream(stream)))
        return v.value

    def _grad_buffer(self, grad, xy):
        import torch
        assert (isinstance(grad, torch.Tensor) and grad.is_cuda and grad.dtype == torch.float64
                and grad.is_contiguous() and grad.numel() == self.n_theta
                and grad.device == xy.device), \
            f"grad must be a contiguous CUDA float64 tensor of {self.n_theta} entries on {xy.device}"

    def vjp(self, xy, resid, grad=None, stream=None):
        import torch
        self._samples(xy, resid)
        if grad is None:
            grad = torch.empty(self.n_theta, dtype=torch.float64, device=xy.device)
        self._grad_buffer(grad, xy)
        self._check(_lib.bem_vjp(self.h, xy.shape[0], _ptr(xy), _ptr(resid), _ptr(grad),
                                 _stream(stream)))
        return grad

    def vjp_noalloc(self, xy, resid, grad, stream=None):
        """bem_vjp into a caller-provided gradient buffer, with no device allocation."""
        self._samples(xy, resid)
        self._grad_buffer(grad, xy)
        self._check(_lib.bem_vjp_noalloc(self.h, xy.shape[0], _ptr(xy), _ptr(resid), _ptr(grad),
                                         _stream(stream)))
        return grad

    def jtj(self, xy, H=None, stream=None):
        import torch
        self._samples(xy)
        if H is None:
            H = torch.empty((self.n_theta, self.n_theta), dtype=torch.float64, device=xy.device)
        self._check(_lib.bem_jtj(self.h, xy.shape[0], _ptr(xy), _ptr(H), _stream(stream)))
        return H

    def lm_step(self, xy, target, lambdas, stream=None) -> dict:
        self._samples(xy, target)
        lam = np.ascontiguousarray(np.atleast_1d(lambdas), np.float64)
        r = lm_result()
        self._check(_lib.lm_step(self.h, xy.shape[0], _ptr(xy), _ptr(target), len(lam), _dp(lam),
                                 ctypes.byref(r), _stream(stream)))
        return dict(loss_before=r.loss_before, loss_after=r.loss_after, accepted=bool(r.accepted),
                    best_trial=r.best_trial, lambda_next=r.lambda_next, grad_norm=r.grad_norm)

    def _host_samples(self, t, cols):
        """Pointer and row count of a host array or CPU tensor [n, cols] of
        the sample type, C-contiguous."""
        import torch
        if isinstance(t, torch.Tensor):
            assert not t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and \
                t.dim() == 2 and t.shape[1] == cols, \
                f"expected a contiguous CPU {self.dtype} tensor [n, {cols}]"
            return ctypes.c_void_p(t.data_ptr()), t.shape[0]
        want = np.float64 if self.dtype == torch.float64 else np.float32
        assert isinstance(t, np.ndarray) and t.dtype == want and t.flags.c_contiguous and \
            t.ndim == 2 and t.shape[1] == cols, f"expected a C-contiguous {want.__name__} array [n, {cols}]"
        return ctypes.c_void_p(t.ctypes.data), t.shape[0]

    def lm_step_host(self, xy, target, lambdas, stream=None) -> dict:
        """lm_step on host samples and targets (numpy arrays or CPU tensors;
        page-locked memory lets the library's copies overlap the step)."""
        px, n = self._host_samples(xy, 2)
        pt, nt = self._host_samples(target, 3)
        assert n == nt, "xy and target must have the same number of rows"
        lam = np.ascontiguousarray(np.atleast_1d(lambdas), np.float64)
        r = lm_result()
        self._check(_lib.lm_step_host(self.h, n, px, pt, len(lam), _dp(lam), ctypes.byref(r),
                                      _stream(stream)))
        return dict(loss_before=r.loss_before, loss_after=r.loss_after, accepted=bool(r.accepted),
                    best_trial=r.best_trial, lambda_next=r.lambda_next, grad_norm=r.grad_norm)

    def render(self, width, height, out=None, stream=None):
        """Colours at the pixel centres of a width x height grid, [height, width, 3]."""
        import torch
        if out is None:
            out = torch.empty((height, width, 3), dtype=self.dtype, device=f"cuda:{self.device}")
        self._samples(out)
        self._check(_lib.bem_render(self.h, width, height, _ptr(out), _stream(stream)))
        return out

    def handle_colors(self, stream=None) -> np.ndarray:
        """[n_panels, 2, 3]: colour on the left / right of each panel (c_avg +- w_d/2)."""
        P = _lib_sizes(self)[1]
        out = np.empty((P, 2, 3))
        self._check(_lib.bem_handle_colors(self.h, _dp(out), _stream(stream)))
        return out

    def lm_step_split(self, xy, target, xy_h, lambdas, stream=None) -> dict:
        """LM iteration with H from the points xy_h and g, losses from (xy, target)."""
        self._samples(xy, target, xy_h)
        lam = np.ascontiguousarray(np.atleast_1d(lambdas), np.float64)
        r = lm_result()
        self._check(_lib.lm_step_split(self.h, xy.shape[0], _ptr(xy), _ptr(target), xy_h.shape[0],
                                       _ptr(xy_h), len(lam), _dp(lam), ctypes.byref(r),
                                       _stream(stream)))
        return dict(loss_before=r.loss_before, loss_after=r.loss_after, accepted=bool(r.accepted),
                    best_trial=r.best_trial, lambda_next=r.lambda_next, grad_norm=r.grad_norm)

    def set_boundary(self, vertices, segs_per_edge):
        """Use a counter-clockwise polygon (one subdomain) as the image boundary;
        call factor() afterwards."""
        v = np.ascontiguousarray(np.asarray(vertices, np.float64).reshape(-1, 2))
        self._check(_lib.bem_set_boundary(self.h, v.shape[0], _dp(v), int(segs_per_edge)))
        self.Nb = v.shape[0] * int(segs_per_edge)

    def boundary_values(self, stream=None) -> np.ndarray:
        out = np.empty((self.Nb, 3))
        self._check(_lib.bem_boundary_values(self.h, _dp(out), _stream(stream)))
        return out

    def launch_count(self) -> int:
        return int(_lib.bem_launch_count(self.h))

    def pipe_peak(self, which: int, launches: int = 5, stream=None) -> float:
        """Operations per second of one SM pipe (bem_pipe_peak): 0 FP32 FMA,
        1 MUFU lg2, 2 MUFU rcp, 3 MUFU rsqrt."""
        v = ctypes.c_double()
        self._check(_lib.bem_pipe_peak(self.h, int(which), int(launches), ctypes.byref(v),
                                       _stream(stream)))
        return v.value

    def alloc_count(self) -> int:
        """Device allocations the context has made so far (bem_alloc_count)."""
        return int(_lib.bem_alloc_count(self.h))

    def set_wait_limit(self, seconds: float):
        """Limit of the tensor-core kernels' pipeline waits (bem_set_wait_limit)."""
        self._check(_lib.bem_set_wait_limit(self.h, float(seconds)))

    def gn_products(self, xy, target, stream=None):
        """(loss, g, H) at the current theta as lm_step forms them (bem_gn_products)."""
        import torch
        self._samples(xy, target)
        g = torch.empty(self.n_theta, dtype=torch.float64, device=xy.device)
        H = torch.empty((self.n_theta, self.n_theta), dtype=torch.float64, device=xy.device)
        L = ctypes.c_double()
        self._check(_lib.bem_gn_products(self.h, xy.shape[0], _ptr(xy), _ptr(target),
                                         ctypes.byref(L), _ptr(g), _ptr(H), _stream(stream)))
        return L.value, g, H

    def gemm_bf16(self, A, B, stream=None):
        """D = A B^T on the tensor cores (A [M][K], B [N][K] bf16 CUDA tensors)."""
        import torch
        assert A.dtype == B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
        M, K = A.shape
        N = B.shape[0]
        D = torch.empty((M, N), dtype=torch.float32, device=A.device)
        self._check(_lib.bem_gemm_bf16(self.h, M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                       _ptr(D), N, _stream(stream)))
        return D

    def fastmath(self, which: int, a, b=None, stream=None):
        """(library approximation, CUDA accurate) of atan2 (0), log (1), log1p (2),
        atan2 for y >= 0 (3, a taken as |a|) and log1p/2 (4)."""
        import torch
        fast = torch.empty_like(a)
        ref = torch.empty_like(a)
        self._check(_lib.bem_fastmath_eval(self.h, which, a.numel(), _ptr(a),
                                           _ptr(b) if b is not None else None, _ptr(fast),
                                           _ptr(ref), _stream(stream)))
        return fast, ref

    def dlog(self, x, stream=None):
        """(library, CUDA) double logarithm of the positive double CUDA tensor x
        (bem_dlog_eval)."""
        import torch
        assert x.dtype == torch.float64 and x.is_cuda
        own = torch.empty_like(x)
        ref = torch.empty_like(x)
        self._check(_lib.bem_dlog_eval(self.h, x.numel(), _ptr(x), _ptr(own), _ptr(ref),
                                       _stream(stream)))
        return own, ref

    def datan2(self, y, x, stream=None):
        """(library, CUDA) double atan2(y, x) of double CUDA tensors, y >= 0
        (bem_datan2_eval)."""
        import torch
        assert y.dtype == torch.float64 and y.is_cuda and y.is_contiguous()
        assert x.dtype == torch.float64 and x.is_cuda and x.is_contiguous()
        assert x.shape == y.shape
        own = torch.empty_like(x)
        ref = torch.empty_like(x)
        self._check(_lib.bem_datan2_eval(self.h, x.numel(), _ptr(y), _ptr(x), _ptr(own), _ptr(ref),
                                         _stream(stream)))
        return own, ref

    def profile(self, on: bool = True):
        self._check(_lib.bem_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} recorded since profile(True)."""
        mx = 64
        names = ctypes.create_string_buffer(32 * mx)
        ms = np.zeros(mx)
        cnt = np.zeros(mx, np.int64)
        n = ctypes.c_int()
        self._check(_lib.bem_profile_read(self.h, mx, names, _dp(ms),
                                          cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                          ctypes.byref(n)))
        out = {}
        for k in range(n.value):
            nm = names.raw[32 * k:32 * k + 32].split(b"\0", 1)[0].decode()
            out[nm] = (float(ms[k]), int(cnt[k]))
        return out


class BEMBatch:
    """Scenes (BEM_MIXED contexts, set up and factored) stepped together by
    bem_batch_lm.  The contexts must outlive the batch."""

    def __init__(self, scenes):
        self.scenes = list(scenes)
        arr = (ctypes.c_void_p * len(self.scenes))(*[m.h.value for m in self.scenes])
        self.h = ctypes.c_void_p()
        rc = _lib.bem_batch_create(ctypes.byref(self.h), arr, len(self.scenes))
        if rc:
            raise BemError(rc, _lib.bem_last_error(self.scenes[0].h).decode())

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _lib.bem_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lm_step(self, xys, targets, lambdas, stream=None) -> list:
        """One LM iteration of every scene; xys[s] float [n_s, 2], targets[s]
        float [n_s, 3] CUDA tensors.  Returns one lm_step dict per scene."""
        S = len(self.scenes)
        assert len(xys) == S and len(targets) == S
        for m, x, t in zip(self.scenes, xys, targets):
            m._samples(x, t)
        n = (ctypes.c_int64 * S)(*[x.shape[0] for x in xys])
        px = (ctypes.c_void_p * S)(*[x.data_ptr() for x in xys])
        pt = (ctypes.c_void_p * S)(*[t.data_ptr() for t in targets])
        lam = np.ascontiguousarray(np.atleast_1d(lambdas), np.float64)
        res = (lm_result * S)()
        rc = _lib.bem_batch_lm(self.h, n, px, pt, len(lam), _dp(lam), res, _stream(stream))
        if rc:
            raise BemError(rc, _lib.bem_last_error(self.scenes[0].h).decode())
        return [dict(loss_before=r.loss_before, loss_after=r.loss_after, accepted=bool(r.accepted),
                     best_trial=r.best_trial, lambda_next=r.lambda_next, grad_norm=r.grad_norm)
                for r in res]

    def tile_shape(self) -> tuple:
        """(points per tile, CTAs per SM) chosen by the batch's autotuner."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _lib.bem_batch_tile_shape(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value


def init_segments(n_points, length, first_index=1, polygon=None) -> np.ndarray:
    """Initial segment handles of Sec. 4.2 (host computation in the library):
    theta [10 * n_handles] for the Sobol points first_index .. + n_points - 1
    that fall inside the polygon (default: the unit square)."""
    out = np.zeros(10 * max(int(n_points), 1))
    n = ctypes.c_int(0)
    if polygon is None:
        rc = _lib.bem_init_segments(int(n_points), float(length), int(first_index), 0, None,
                                    _dp(out), ctypes.byref(n))
    else:
        v = np.ascontiguousarray(polygon, np.float64).reshape(-1, 2)
        rc = _lib.bem_init_segments(int(n_points), float(length), int(first_index), v.shape[0],
                                    _dp(v), _dp(out), ctypes.byref(n))
    if rc != BEM_OK:
        raise BemError(rc, "bem_init_segments: bad arguments")
    return out[:10 * n.value].copy()


def gram_units(tiles: int, rows: int | None = None) -> list:
    """The bf16 Gram kernel's units over the block rows 0 .. rows-1 (default
    all) of a `tiles` x `tiles` block triangle, as (kind, a0, a1, b) tuples in
    launch order (bem_gram_unit; host only)."""
    units = []
    out = (ctypes.c_int32 * 4)()
    rows = tiles if rows is None else rows
    while True:
        rc = _lib.bem_gram_unit(int(tiles), int(rows), len(units), out)
        if rc == BEM_EINVAL:
            return units
        if rc != BEM_OK:
            raise BemError(rc, "bem_gram_unit failed")
        units.append(tuple(int(v) for v in out))
