"""Shared helpers of the test-suite: data drawn from the oracle's expected counts."""
import functools

import numpy as np

from oracle import oracle as O
from paper_1805_11125_gb300 import inputs as I


@functools.lru_cache(maxsize=None)
def dataset(name: str, seed: int = 0):
    """Config `name` with Poisson data drawn from the oracle's expected counts at theta_true."""
    s = I.config(name)
    return s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), seed))


def points(spec, n, rel=0.02, seed=1):
    return I.parameter_points(spec.theta_true, n, rel=rel, seed=seed, free=spec.default_free())


def per_bin_ok(mu_gpu, mu_ref, rel=1e-5, abs_frac=1e-8, floor_frac=1e-3):
    """Per-bin criterion: relative error <= rel on bins with mu >= floor_frac * max(mu),
    absolute error <= abs_frac * max(mu) below."""
    top = np.max(np.abs(mu_ref))
    big = np.abs(mu_ref) >= floor_frac * top
    rel_err = np.abs(mu_gpu[big] - mu_ref[big]) / np.abs(mu_ref[big])
    abs_err = np.abs(mu_gpu[~big] - mu_ref[~big])
    worst_rel = float(rel_err.max()) if rel_err.size else 0.0
    worst_abs = float(abs_err.max()) / top if abs_err.size else 0.0
    return worst_rel <= rel and worst_abs <= abs_frac, worst_rel, worst_abs
