"""ctypes front end of the plain FP64 CPU oracle (``bx_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports, links or runs
anything here, and this module imports nothing from the CUDA side: a model is handed
over as a :class:`paper_1805_11125_gb300.inputs.ModelSpec` (plain numpy arrays produced
by the seeded input generator, which holds no likelihood arithmetic).

Functions follow the paper's steps (arXiv:1805.11125 Sec. 3):
``quench`` (Eq. 1 parameters), ``response`` (Eq. 1), ``pileup`` (Eq. 2),
``expected`` (Eq. 1-4 expected counts), ``nll`` (Eq. 3-4 with dual-number gradient),
``poisson_nll`` (the binned Poisson sum alone), ``radial`` (Eq. 4 radial term) and
``fit`` (the minimisation of Sec. 4).  Models with 2D energy x radius / energy x pulse-shape
histograms (the discrimination regime) are evaluated through the same entry points.
``est_theta``, ``nll_estimators``, ``expected_estimators`` and ``fit_estimators`` evaluate and
fit several energy estimators of one dataset jointly (Sec. 3: charge, detected photons, fired
channels; shared rates, kB, eps and s_r, per-estimator LY, a, b, c).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bx_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbx_oracle.so")

_lock = threading.Lock()
_lib = None

OM_EDOMAIN = -4
OM_ENOTCONV = -6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no fast-math, no contraction)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Model(C.Structure):
    _fields_ = [
        ("n_grid", C.c_int), ("e_max", C.c_double),
        ("K", C.c_int), ("shapes", C.c_void_p), ("stop_pow", C.c_void_p),
        ("tag_frac", C.c_void_p),
        ("L", C.c_int), ("pileup", C.c_void_p),
        ("width", C.c_double), ("m_lo", C.c_int), ("m_hi", C.c_int),
        ("n_sub", C.c_void_p), ("n_tag", C.c_void_p),
        ("n_rad", C.c_int), ("rad_class", C.c_void_p),
        ("r_fid", C.c_double), ("r_iv", C.c_double), ("att_len", C.c_double),
        ("n_rad_counts", C.c_void_p),
        ("n_psd", C.c_int), ("psd_prob", C.c_void_p), ("n_psd_counts", C.c_void_p),
        ("n_r2", C.c_int), ("n_p2", C.c_int), ("field", C.c_void_p), ("amp", C.c_double),
        ("psd2", C.c_void_p), ("n_r2_counts", C.c_void_p), ("n_p2_counts", C.c_void_p),
        ("quench", C.c_void_p),
        ("n_es", C.c_int), ("es_edges", C.c_void_p),
        ("gc_skew", C.c_double), ("gc_kurt", C.c_double),
        ("joint2", C.c_int),
        ("n_shell", C.c_int), ("shell_ly", C.c_void_p), ("shell_frac", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.c_void_p
            _lib.om_expected.argtypes = [P, P, P]
            _lib.om_nll.argtypes = [P, P, P, P]
            _lib.om_quench.argtypes = [P, P, P, P, P, P]
            _lib.om_response.argtypes = [P, P, P, P]
            _lib.om_pileup.argtypes = [P, C.c_double, P, P]
            _lib.om_radial.argtypes = [P, C.c_double, C.c_int, P, P]
            _lib.om_poisson_nll.argtypes = [C.c_int, P, P, P]
            _lib.om_fit.argtypes = [P, P, P, P, P, C.c_double, C.c_int, P, P, P]
            _lib.om_n_bins.argtypes = [P]
            _lib.om_est_theta.argtypes = [C.c_int, C.c_int, P, P]
            _lib.om_nll_est.argtypes = [P, C.c_int, P, P, P]
            _lib.om_fit_est.argtypes = [P, C.c_int, P, P, P, P, C.c_double, C.c_int, P, P, P]
        return _lib


def _arr(x, dtype=np.float64):
    return None if x is None else np.ascontiguousarray(x, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleModel:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, spec):
        self.spec = spec
        s = spec
        self._keep = {
            "shapes": _arr(s.shapes), "stop_pow": _arr(s.stop_pow), "pileup": _arr(s.pileup),
            "tag_frac": _arr(s.tag_frac), "rad_class": _arr(s.rad_class, np.int32),
            "psd_prob": _arr(s.psd_prob),
            "n_sub": _arr(s.counts.get("sub")), "n_tag": _arr(s.counts.get("tag")),
            "n_rad": _arr(s.counts.get("rad")), "n_psd": _arr(s.counts.get("psd")),
            "field": _arr(s.field2d), "psd2": _arr(s.psd2d_prob),
            "n_r2": _arr(s.counts.get("j2d" if getattr(s, "joint2d", False) else "r2d")),
            "n_p2": _arr(s.counts.get("p2d")),
            "quench": _arr(getattr(s, "quench", None)),
            "es_edges": _arr(getattr(s, "eslices", None), np.int32),
            "shell_ly": _arr(getattr(s, "shell_ly", None)),
            "shell_frac": _arr(getattr(s, "shell_frac", None)),
        }
        k = self._keep
        has_rad = s.rad_class is not None and s.n_rad > 0
        self.c = _Model(
            n_grid=s.n_grid, e_max=s.e_max, K=s.K, shapes=_ptr(k["shapes"]), stop_pow=_ptr(k["stop_pow"]),
            tag_frac=_ptr(k["tag_frac"]), L=s.L, pileup=_ptr(k["pileup"]), width=s.width,
            m_lo=s.m_lo, m_hi=s.m_hi, n_sub=_ptr(k["n_sub"]), n_tag=_ptr(k["n_tag"]),
            n_rad=s.n_rad if has_rad else 0, rad_class=_ptr(k["rad_class"]), r_fid=s.r_fid,
            r_iv=s.r_iv, att_len=s.att_len, n_rad_counts=_ptr(k["n_rad"]),
            n_psd=s.n_psd, psd_prob=_ptr(k["psd_prob"]), n_psd_counts=_ptr(k["n_psd"]),
            n_r2=s.n_rad2d, n_p2=s.n_psd2d, field=_ptr(k["field"]), amp=s.field_amp, psd2=_ptr(k["psd2"]),
            n_r2_counts=_ptr(k["n_r2"]), n_p2_counts=_ptr(k["n_p2"]), quench=_ptr(k["quench"]),
            n_es=0 if k["es_edges"] is None else len(k["es_edges"]) - 1, es_edges=_ptr(k["es_edges"]),
            gc_skew=getattr(s, "resp_skew", 0.0), gc_kurt=getattr(s, "resp_kurt", 0.0),
            joint2=1 if getattr(s, "joint2d", False) else 0,
            n_shell=0 if k["shell_ly"] is None else len(k["shell_ly"]), shell_ly=_ptr(k["shell_ly"]),
            shell_frac=_ptr(k["shell_frac"]))
        self.ref = C.byref(self.c)

    @property
    def n_bins(self) -> int:
        return lib().om_n_bins(self.ref)


def _model(spec_or_model):
    return spec_or_model if isinstance(spec_or_model, OracleModel) else OracleModel(spec_or_model)


def expected(spec, theta) -> np.ndarray:
    """Expected counts of every bin (histograms concatenated: vetoed, tagged, radial, PSD)."""
    m = _model(spec)
    th = _arr(theta)
    out = np.zeros(m.n_bins)
    st = lib().om_expected(m.ref, _ptr(th), _ptr(out))
    if st not in (0, OM_EDOMAIN):
        raise RuntimeError(f"om_expected status {st}")
    return out


def nll(spec, theta, grad: bool = False):
    """-lnL (Baker-Cousins form) and, if ``grad``, its dual-number gradient."""
    m = _model(spec)
    th = _arr(theta)
    f = np.zeros(1)
    g = np.zeros(th.shape[0]) if grad else None
    st = lib().om_nll(m.ref, _ptr(th), _ptr(f), _ptr(g))
    if st not in (0, OM_EDOMAIN):
        raise RuntimeError(f"om_nll status {st}")
    return (f[0], g) if grad else f[0]


def quench(spec, theta):
    """(Q, mu, sigma, Phi(mu/sigma)) on the true-energy grid."""
    m = _model(spec)
    th = _arr(theta)
    N = spec.n_grid
    out = [np.zeros(N) for _ in range(4)]
    st = lib().om_quench(m.ref, _ptr(th), *[_ptr(o) for o in out])
    if st:
        raise RuntimeError(f"om_quench status {st}")
    return tuple(out)


def response(spec, theta, want_R: bool = True):
    """(R [m_hi, n_grid] or None, v [m_hi, K]) -- Eq. 1 on the full axis."""
    m = _model(spec)
    th = _arr(theta)
    R = np.zeros((spec.m_hi, spec.n_grid)) if want_R else None
    v = np.zeros((spec.m_hi, spec.K))
    st = lib().om_response(m.ref, _ptr(th), _ptr(R), _ptr(v))
    if st:
        raise RuntimeError(f"om_response status {st}")
    return R, v


def pileup(spec, eps: float, x) -> np.ndarray:
    """Eq. 2 with scale eps on a spectrum x[0..m_hi), returned on the window."""
    m = _model(spec)
    xx = _arr(x)
    y = np.zeros(spec.n_window)
    lib().om_pileup(m.ref, float(eps), _ptr(xx), _ptr(y))
    return y


def radial(spec, s_r: float, cls: int):
    """Radial bin probabilities of one class and their derivative in s_r."""
    m = _model(spec)
    p, dp = np.zeros(spec.n_rad), np.zeros(spec.n_rad)
    lib().om_radial(m.ref, float(s_r), int(cls), _ptr(p), _ptr(dp))
    return p, dp


def poisson_nll(counts, mu) -> float:
    n, u = _arr(counts), _arr(mu)
    out = np.zeros(1)
    st = lib().om_poisson_nll(n.shape[0], _ptr(n), _ptr(u), _ptr(out))
    if st not in (0, OM_EDOMAIN):
        raise RuntimeError(f"om_poisson_nll status {st}")
    return out[0]


def fit(spec, theta0, free=None, lo=None, hi=None, tol_edm=1e-12, max_iter=60):
    """Damped Newton fit; returns dict(theta, nll, edm, iters, status, cov).

    Pinned by two invariants (an Asimov fit returns theta_true; the expected and observed
    totals agree at the optimum) and one closed form (a single free rate of a one-species model
    ends at sum(n) / sum(u)); parity unpinned beyond them: the paper prints no fitted values."""
    m = _model(spec)
    P = spec.P
    free = spec.default_free() if free is None else free
    dlo, dhi = spec.default_bounds()
    lo = dlo if lo is None else lo
    hi = dhi if hi is None else hi
    th0, fr, l, h = _arr(theta0), _arr(free, np.uint8), _arr(lo), _arr(hi)
    out = np.zeros(P)
    info = np.zeros(4)
    cov = np.zeros((P, P))
    lib().om_fit(m.ref, _ptr(th0), _ptr(fr), _ptr(l), _ptr(h), float(tol_edm), int(max_iter),
                 _ptr(out), _ptr(info), _ptr(cov))
    return dict(theta=out, nll=info[0], edm=info[1], iters=int(info[2]), status=int(info[3]), cov=cov)


# ---- several energy estimators of one dataset (Sec. 3), fitted jointly

class _Estimators:
    """The estimators' C models as one contiguous array (estimator 0 first)."""

    def __init__(self, specs):
        self.models = [OracleModel(s) for s in specs]
        self.arr = (_Model * len(specs))(*[m.c for m in self.models])
        self.E = len(specs)
        self.K = specs[0].K
        self.P = self.K + 7 + 4 * (self.E - 1)


def est_theta(K: int, e: int, theta) -> np.ndarray:
    """The parameter vector of estimator e ([r, LY_e, a_e, b_e, c_e, kB, eps, s_r]) taken from
    the joint vector [r, LY_0, a_0, b_0, c_0, kB, eps, s_r, LY_1, a_1, b_1, c_1, ...]."""
    th = _arr(theta)
    out = np.zeros(K + 7)
    lib().om_est_theta(int(K), int(e), _ptr(th), _ptr(out))
    return out


def nll_estimators(specs, theta, grad: bool = False):
    """Joint -lnL of the estimators (the sum of each estimator's -lnL at its own parameter
    vector) and, with ``grad``, its gradient in the joint layout."""
    m = specs if isinstance(specs, _Estimators) else _Estimators(specs)
    th = _arr(theta)
    f = np.zeros(1)
    g = np.zeros(m.P) if grad else None
    st = lib().om_nll_est(m.arr, m.E, _ptr(th), _ptr(f), _ptr(g))
    if st not in (0, OM_EDOMAIN):
        raise RuntimeError(f"om_nll_est status {st}")
    return (f[0], g) if grad else f[0]


def expected_estimators(specs, theta) -> np.ndarray:
    """Expected counts of every estimator's bins, estimator after estimator."""
    K = specs[0].K
    return np.concatenate([expected(s, est_theta(K, e, theta)) for e, s in enumerate(specs)])


def estimator_defaults(specs):
    """Free mask and bounds of the joint layout: those of estimator 0's single model, then
    LY, a, b, c of every further estimator with the bounds of LY, a, b, c."""
    free = specs[0].default_free()
    lo, hi = specs[0].default_bounds()
    K = specs[0].K
    for _ in specs[1:]:
        free = np.concatenate([free, np.ones(4, dtype=np.uint8)])
        lo = np.concatenate([lo, lo[K:K + 4]])
        hi = np.concatenate([hi, hi[K:K + 4]])
    return free, lo, hi


def fit_estimators(specs, theta0, free=None, lo=None, hi=None, tol_edm=1e-12, max_iter=60):
    """The joint fit of the estimators by the same damped Newton method as :func:`fit`.
    Parity unpinned beyond its invariants (an Asimov fit returns theta_true)."""
    m = _Estimators(specs)
    dfree, dlo, dhi = estimator_defaults(specs)
    free = dfree if free is None else free
    lo = dlo if lo is None else lo
    hi = dhi if hi is None else hi
    th0, fr, l, h = _arr(theta0), _arr(free, np.uint8), _arr(lo), _arr(hi)
    out = np.zeros(m.P)
    info = np.zeros(4)
    cov = np.zeros((m.P, m.P))
    lib().om_fit_est(m.arr, m.E, _ptr(th0), _ptr(fr), _ptr(l), _ptr(h), float(tol_edm), int(max_iter),
                     _ptr(out), _ptr(info), _ptr(cov))
    return dict(theta=out, nll=info[0], edm=info[1], iters=int(info[2]), status=int(info[3]), cov=cov)
