"""Thin Python binding of the C ABI in ``include/bx.h`` (argument marshalling only).

Every step of the likelihood runs in the CUDA library ``libbx.so``; this module converts
numpy arrays / torch tensors to pointers and back.  There is no fallback: if the library
cannot be loaded (not built, or no sm_103a device) the calls raise.

Functions carry the C names (``bx_model_create``, ``bx_nll``, ``bx_nll_grad``,
``bx_expected``, ``bx_nll_batch``, ``bx_fit``); :class:`Model` wraps them for a list of
:class:`paper_1805_11125_gb300.inputs.ModelSpec`, and :class:`BxNLL` exposes the
evaluation with its hand-written adjoint as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

BX_OK, BX_EINVAL, BX_ENOMEM, BX_ECUDA, BX_EDOMAIN, BX_ETIMEOUT, BX_ENOTCONV = 0, -1, -2, -3, -4, -5, -6
BX_FP64, BX_FP32, BX_BF16X3, BX_TF32X3 = 0, 1, 2, 3

_P = C.c_void_p


class bx_model_desc(C.Structure):
    _fields_ = [
        ("n_grid", C.c_int), ("e_max", C.c_double),
        ("n_species", C.c_int), ("shapes", _P), ("stop_pow", _P), ("tag_frac", _P),
        ("n_pileup", C.c_int), ("pileup", _P),
        ("width", C.c_double), ("m_lo", C.c_int), ("m_hi", C.c_int),
        ("counts_sub", _P), ("counts_tag", _P),
        ("n_rad", C.c_int), ("rad_class", _P),
        ("r_fid", C.c_double), ("r_iv", C.c_double), ("att_len", C.c_double),
        ("counts_rad", _P),
        ("n_psd", C.c_int), ("psd_prob", _P), ("counts_psd", _P),
        ("n_rad2d", C.c_int), ("n_psd2d", C.c_int), ("psd2d_prob", _P), ("field2d", _P),
        ("field_amp", C.c_double), ("counts_rad2d", _P), ("counts_psd2d", _P),
        ("quench", _P),
        ("n_eslice", C.c_int), ("eslice_edges", _P),
        ("joint2d", C.c_int),
        ("resp_skew", C.c_double), ("resp_kurt", C.c_double),
        ("n_shell", C.c_int), ("shell_ly", _P), ("shell_frac", _P),
    ]


class bx_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_batch", C.c_int), ("band_sigmas", C.c_double),
                ("watchdog_s", C.c_double)]


class bx_fit_opts(C.Structure):
    _fields_ = [("tol_edm", C.c_double), ("max_iter", C.c_int), ("free_mask", _P), ("lo", _P), ("hi", _P),
                ("iters_per_launch", C.c_int), ("cov_out", _P), ("time_budget_s", C.c_double),
                ("fits_in_flight", C.c_int)]


class bx_fit_plan(C.Structure):
    _fields_ = [("fits", C.c_int), ("fits_in_flight", C.c_int), ("slots_per_fit", C.c_int),
                ("iters_per_launch", C.c_int), ("graph_launches", C.c_int), ("rounds", C.c_int),
                ("fwd_tile", C.c_int), ("tuned_evals_per_s", C.c_double)]


class bx_fit_result(C.Structure):
    _fields_ = [("nll", C.c_double), ("edm", C.c_double), ("iters", C.c_int), ("n_evals", C.c_int),
                ("status", C.c_int), ("n_at_bound", C.c_int), ("damping", C.c_double)]


class BxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bx status {status}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every entry point declared in include/bx.h
SIGNATURES = [
    ("bx_model_create", C.c_int, [_P, C.c_int, _P, _P, _P]),
    ("bx_model_create_estimators", C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P]),
    ("bx_model_destroy", None, [_P]),
    ("bx_model_set_stream", C.c_int, [_P, _P]),
    ("bx_model_n_params", C.c_int, [_P]),
    ("bx_model_n_bins", C.c_int, [_P, C.c_int]),
    ("bx_model_status", C.c_int, [_P]),
    ("bx_model_profile", C.c_int, [_P, C.c_int, _P, _P, _P]),
    ("bx_nll", C.c_int, [_P, _P, _P]),
    ("bx_nll_grad", C.c_int, [_P, _P, _P, _P]),
    ("bx_expected", C.c_int, [_P, C.c_int, _P, _P]),
    ("bx_nll_batch", C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.c_int]),
    ("bx_fit", C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    ("bx_fit_last_plan", C.c_int, [_P, _P]),
    ("bx_selftest_tensor_core", C.c_int, [_P]),
    ("bx_selftest_watchdog", C.c_int, [C.c_double]),
    ("bx_spectra_noalloc", C.c_int, [C.c_int, C.c_double, C.c_int, _P, _P, _P, C.c_double, C.c_int, _P, _P, _P]),
    ("bx_ceiling", C.c_int, [C.c_int, C.c_int, _P, _P, _P]),
    ("bx_last_error", C.c_char_p, []),
    ("bx_status_string", C.c_char_p, [C.c_int]),
]


def lib(build_if_missing: bool = True):
    """Load ``libbx.so`` (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise OSError(f"CUDA library not built: {path}")
            L = C.CDLL(path)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(st: int):
    if st != BX_OK:
        raise BxError(st, lib().bx_last_error().decode())


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Model:
    """A bx_model built from one or more :class:`ModelSpec` (toys)."""

    def __init__(self, specs, precision: int = BX_FP32, max_batch: int = 1, band_sigmas: float = 0.0,
                 watchdog_s: float = 0.0, stream=None, n_est: int = 1):
        """n_est > 1: ``specs`` are n_data x n_est energy estimators, dataset-major
        (bx_model_create_estimators); toys are then datasets and theta the joint vector."""
        specs = list(specs) if isinstance(specs, (list, tuple)) else [specs]
        self.specs = specs
        self._keep = []
        descs = (bx_model_desc * len(specs))()
        for d, s in zip(descs, specs):
            arr = lambda x, dt=np.float64: None if x is None else np.ascontiguousarray(x, dtype=dt)
            k = dict(shapes=arr(s.shapes), stop=arr(s.stop_pow), tag=arr(s.tag_frac), g=arr(s.pileup),
                     sub=arr(s.counts.get("sub")), tagc=arr(s.counts.get("tag")),
                     rcls=arr(s.rad_class, np.int32), rad=arr(s.counts.get("rad")), psd=arr(s.psd_prob),
                     psdc=arr(s.counts.get("psd")), psd2=arr(s.psd2d_prob), field=arr(s.field2d),
                     r2c=arr(s.counts.get("j2d" if getattr(s, "joint2d", False) else "r2d")),
                     p2c=arr(s.counts.get("p2d")),
                     quench=arr(getattr(s, "quench", None)), es=arr(getattr(s, "eslices", None), np.int32),
                     shly=arr(getattr(s, "shell_ly", None)), shfr=arr(getattr(s, "shell_frac", None)))
            self._keep.append(k)
            has_rad = s.rad_class is not None and s.n_rad > 0
            d.n_grid, d.e_max, d.n_species = s.n_grid, s.e_max, s.K
            d.shapes, d.stop_pow, d.tag_frac = _ptr(k["shapes"]), _ptr(k["stop"]), _ptr(k["tag"])
            d.n_pileup, d.pileup = s.L, _ptr(k["g"])
            d.width, d.m_lo, d.m_hi = s.width, s.m_lo, s.m_hi
            d.counts_sub, d.counts_tag = _ptr(k["sub"]), _ptr(k["tagc"])
            d.n_rad = s.n_rad if has_rad else 0
            d.rad_class, d.counts_rad = _ptr(k["rcls"]), _ptr(k["rad"])
            d.r_fid, d.r_iv, d.att_len = s.r_fid, s.r_iv, s.att_len
            d.n_psd, d.psd_prob, d.counts_psd = s.n_psd, _ptr(k["psd"]), _ptr(k["psdc"])
            d.n_rad2d, d.n_psd2d, d.psd2d_prob = s.n_rad2d, s.n_psd2d, _ptr(k["psd2"])
            d.field2d, d.field_amp = _ptr(k["field"]), s.field_amp
            d.counts_rad2d, d.counts_psd2d = _ptr(k["r2c"]), _ptr(k["p2c"])
            d.quench = _ptr(k["quench"])
            d.n_eslice = 0 if k["es"] is None else len(k["es"]) - 1
            d.eslice_edges = _ptr(k["es"])
            d.joint2d = 1 if getattr(s, "joint2d", False) else 0
            d.resp_skew, d.resp_kurt = getattr(s, "resp_skew", 0.0), getattr(s, "resp_kurt", 0.0)
            d.n_shell = 0 if k["shly"] is None else len(k["shly"])
            d.shell_ly, d.shell_frac = _ptr(k["shly"]), _ptr(k["shfr"])
        opts = bx_options(precision, max_batch, band_sigmas, watchdog_s)
        h = C.c_void_p()
        if n_est == 1:
            _check(lib().bx_model_create(C.cast(descs, _P), len(specs), C.byref(opts), _stream_handle(stream),
                                         C.byref(h)))
        else:
            _check(lib().bx_model_create_estimators(C.cast(descs, _P), len(specs) // n_est, n_est, C.byref(opts),
                                                    _stream_handle(stream), C.byref(h)))
        self.n_est = n_est
        self.h = h
        self.precision = precision
        self.max_batch = max_batch
        self.P = lib().bx_model_n_params(h)
        self._keep = None  # arrays were copied at creation

    def close(self):
        if getattr(self, "h", None):
            lib().bx_model_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        _check(lib().bx_model_set_stream(self.h, _stream_handle(stream)))

    def n_bins(self, toy: int = 0) -> int:
        return lib().bx_model_n_bins(self.h, toy)

    def status(self) -> int:
        return lib().bx_model_status(self.h)

    STAGES = ("prep", "forward", "assembly", "adjoint", "gather")

    def profile(self, enable: bool):
        """(per-stage device ms, evaluations, in-band response entries) recorded since the last call."""
        ms = np.zeros(5)
        n = C.c_int(0)
        ent = np.zeros(1)
        _check(lib().bx_model_profile(self.h, int(enable), _ptr(ms), C.byref(n), _ptr(ent)))
        return dict(zip(self.STAGES, ms)), n.value, float(ent[0])

    def _row(self, theta):
        th = _f64(theta).ravel()
        out = np.zeros(self.P)
        out[: th.shape[0]] = th
        return out

    def nll(self, theta) -> float:
        th = self._row(theta)
        f = np.zeros(1)
        _check(lib().bx_nll(self.h, _ptr(th), _ptr(f)))
        return float(f[0])

    def nll_grad(self, theta):
        th = self._row(theta)
        f, g = np.zeros(1), np.zeros(self.P)
        _check(lib().bx_nll_grad(self.h, _ptr(th), _ptr(f), _ptr(g)))
        return float(f[0]), g

    def expected(self, theta, toy: int = 0) -> np.ndarray:
        th = self._row(theta)
        mu = np.zeros(self.n_bins(toy))
        _check(lib().bx_expected(self.h, int(toy), _ptr(th), _ptr(mu)))
        return mu

    def nll_batch(self, theta, toy_idx: Optional[Sequence[int]] = None, grad: bool = False, check: bool = True):
        """theta [n, P] (numpy: host path; CUDA tensor: device path on the current stream)."""
        ti = None if toy_idx is None else np.ascontiguousarray(toy_idx, dtype=np.int32)
        if hasattr(theta, "is_cuda") and theta.is_cuda:
            import torch
            th = theta.contiguous().to(torch.float64)
            n = th.shape[0]
            f = torch.empty(n, dtype=torch.float64, device=th.device)
            g = torch.empty((n, self.P), dtype=torch.float64, device=th.device) if grad else None
            self.set_stream(torch.cuda.current_stream())
            st = lib().bx_nll_batch(self.h, n, _ptr(ti), _ptr(th), _ptr(f), _ptr(g), 1)
            if check:
                _check(st)
            return (f, g) if grad else f
        th = _f64(theta)
        if hasattr(theta, "pin_memory"):
            th = theta
        n = th.shape[0]
        f = np.zeros(n)
        g = np.zeros((n, self.P)) if grad else None
        st = lib().bx_nll_batch(self.h, n, _ptr(ti), _ptr(th), _ptr(f), _ptr(g), 0)
        if check:
            _check(st)
        return (f, g) if grad else f

    @property
    def fit_slots(self) -> int:
        """Evaluation slots one fit occupies (max_batch must be >= n_fits * fit_slots)."""
        return 8 + 2 * self.P

    def fit(self, theta0, toy_idx=None, tol_edm: float = 0.0, max_iter: int = 0, free=None, lo=None, hi=None,
            iters_per_launch: int = 0, want_cov: bool = False, time_budget_s: float = 0.0, fits_in_flight: int = 0):
        """n fits (one row of theta0 each) on the device; returns (theta[n, P], info, status).
        info[j]: nll, edm, iters, n_evals, status, n_at_bound, damping, and with want_cov the
        inverse Hessian of -lnL ("cov", P x P; zero rows for fixed and bound-held parameters)."""
        th0 = _f64(theta0)
        th0 = th0[None, :] if th0.ndim == 1 else th0
        n = th0.shape[0]
        if th0.shape[1] != self.P:
            t = np.zeros((n, self.P)); t[:, : th0.shape[1]] = th0; th0 = t
        ti = None if toy_idx is None else np.ascontiguousarray(toy_idx, dtype=np.int32)
        fr = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        l, h = _f64(lo), _f64(hi)
        cov = np.zeros((n, self.P, self.P)) if want_cov else None
        o = bx_fit_opts(tol_edm, max_iter, _ptr(fr), _ptr(l), _ptr(h), iters_per_launch, _ptr(cov), time_budget_s,
                        fits_in_flight)
        out = np.zeros((n, self.P))
        res = (bx_fit_result * n)()
        st = lib().bx_fit(self.h, n, _ptr(ti), _ptr(th0), C.byref(o), _ptr(out), C.cast(res, _P))
        if st not in (BX_OK, BX_ENOTCONV, BX_ETIMEOUT, BX_EDOMAIN):
            _check(st)
        info = [dict(nll=r.nll, edm=r.edm, iters=r.iters, n_evals=r.n_evals, status=r.status,
                     n_at_bound=r.n_at_bound, damping=r.damping) for r in res]
        if want_cov:
            for j in range(n):
                info[j]["cov"] = cov[j]
        return out, info, st


    def fit_plan(self) -> dict:
        """The launch plan of the last fit call (bx_fit_last_plan)."""
        p = bx_fit_plan()
        _check(lib().bx_fit_last_plan(self.h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in bx_fit_plan._fields_}

    def profile_scan(self, param: int, values, theta_start, toy: int = 0, free=None, tol_edm: float = 0.0,
                     max_iter: int = 0):
        """Profile likelihood of one parameter: for every value v in ``values`` the fit of all
        other free parameters with theta[param] held at v, all scan points as one batch of fits
        (one bx_fit call; max_batch >= len(values) * fit_slots).  ``free``: the free mask of
        the toy's layout (default: the spec's default_free()).  Returns (nll[len], theta[len, P],
        info) with nll the minimised -lnL at each value."""
        spec = self.specs[toy]
        vals = np.asarray(values, dtype=np.float64)
        fr = (spec.default_free() if free is None else np.asarray(free)).astype(np.uint8).copy()
        fr[param] = 0
        # the options' free mask is in the layout of a toy with the model's largest K
        Kmax = self.P - 7
        mask = np.zeros(self.P, dtype=np.uint8)
        mask[: spec.K] = fr[: spec.K]
        mask[Kmax:] = fr[spec.K:]
        th0 = np.zeros((len(vals), self.P))
        th0[:, : spec.P] = np.asarray(theta_start, dtype=np.float64)[: spec.P]
        th0[:, param] = vals
        out, info, _ = self.fit(th0, toy_idx=np.full(len(vals), toy), tol_edm=tol_edm, max_iter=max_iter,
                                free=mask)
        return np.array([r["nll"] for r in info]), out, info


# C-named conveniences -------------------------------------------------------------------

def toy_study(spec, n_toys: int, theta_true=None, precision: int = BX_FP32, seed: int = 0, start=None,
              free=None, tol_edm: float = 0.0, max_iter: int = 0, stream=None) -> dict:
    """Toy-based sensitivity with the batched fit engine: n_toys pseudo-experiments, the
    Poisson counts of the expected counts at theta_true (computed by the FP64 GPU model), all
    fitted in one bx_fit call from ``start`` (default theta_true).  Returns theta[n, P],
    sigma[n, P] (square roots of the inverse Hessian's diagonal at each fit), pull[n, P] =
    (theta - theta_true) / sigma (NaN where sigma = 0: fixed or bound-held parameters),
    status[n] and nll[n]."""
    from . import inputs as _inputs
    th_true = np.asarray(spec.theta_true if theta_true is None else theta_true, dtype=np.float64)
    gen = Model(spec.with_counts(np.zeros(spec.n_bins_total)), precision=BX_FP64, stream=stream)
    mu = gen.expected(th_true)
    gen.close()
    toys = [spec.with_counts(_inputs.poisson_counts(mu, seed + t)) for t in range(n_toys)]
    P = spec.P
    m = Model(toys, precision=precision, max_batch=n_toys * (8 + 2 * P), stream=stream)
    th0 = np.tile(th_true if start is None else np.asarray(start, dtype=np.float64), (n_toys, 1))
    out, info, _ = m.fit(th0, toy_idx=np.arange(n_toys), free=free, tol_edm=tol_edm, max_iter=max_iter,
                         want_cov=True)
    m.close()
    theta = out[:, :P]
    sig = np.sqrt(np.maximum(np.array([np.diag(r["cov"])[:P] for r in info]), 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        pull = np.where(sig > 0, (theta - th_true[None, :]) / sig, np.nan)
    return dict(theta=theta, sigma=sig, pull=pull, status=np.array([r["status"] for r in info]),
                nll=np.array([r["nll"] for r in info]))


def bx_model_create(specs, precision=BX_FP32, max_batch=1, **kw) -> Model:
    return Model(specs, precision=precision, max_batch=max_batch, **kw)


def bx_nll(model: Model, theta) -> float:
    return model.nll(theta)


def bx_nll_grad(model: Model, theta):
    return model.nll_grad(theta)


def bx_expected(model: Model, toy: int, theta):
    return model.expected(theta, toy)


def bx_nll_batch(model: Model, theta, toy_idx=None, grad=False):
    return model.nll_batch(theta, toy_idx, grad)


def bx_fit(model: Model, theta0, toy_idx=None, **kw):
    return model.fit(theta0, toy_idx, **kw)


def bx_selftest_tensor_core() -> float:
    e = np.zeros(1)
    _check(lib().bx_selftest_tensor_core(_ptr(e)))
    return float(e[0])


class BxNLL:
    """-lnL with the hand-written adjoint as a torch.autograd.Function.

    ``BxNLL.apply(theta, model)``: theta is a CUDA float64 tensor [n, P]; returns the [n]
    -lnL values; backward returns grad_output[:, None] * dNLL/dtheta.
    """

    _fn = None

    @classmethod
    def apply(cls, theta, model: Model):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, mdl):
                    f, g = mdl.nll_batch(th.detach(), grad=True)
                    ctx.save_for_backward(g)
                    return f

                @staticmethod
                def backward(ctx, gout):
                    (g,) = ctx.saved_tensors
                    return gout[:, None] * g, None

            cls._fn = _F
        return cls._fn.apply(theta, model)


BX_CEIL_RESP, BX_CEIL_RESP_ACC, BX_CEIL_FMA64, BX_CEIL_FMA32 = 0, 1, 2, 3


def bx_ceiling(which: int, reps: int, stream=None):
    """(ms, units) of one ceiling microkernel launch (see include/bx.h)."""
    ms, units = np.zeros(1), np.zeros(1)
    _check(lib().bx_ceiling(int(which), int(reps), _stream_handle(stream), _ptr(ms), _ptr(units)))
    return float(ms[0]), float(units[0])


def bx_selftest_watchdog(budget_s: float = 0.05) -> int:
    """Status of the watchdog diagnostic (BX_ETIMEOUT when the bounded wait ran out)."""
    return lib().bx_selftest_watchdog(float(budget_s))
