"""Full-size fit parity (Sec. 4: the minimiser finds the best-fit rates).

The multivariate model (K = 15, 22 parameters, 2e6 events) and the plain model (K = 8, 1e6
events) are fitted on the GPU and compared with the oracle's fit of the same data.  The oracle's
fit of the full multivariate model takes minutes on the host cores, so it is stored:
tests/golden/fit_<name>.json, written by tests/golden/make_fit_golden.py from the oracle alone,
with a fingerprint of the data it fitted (a stale file fails here instead of comparing against
other data).  Acceptance: every free parameter within max(1e-4 |theta|, 0.01 sigma) of the
oracle's optimum (sigma from its inverse Hessian) and -2 lnL within 1e-3.

The discrimination model (2D histograms, 100,800 bins; the GPU runs it in BX_FP32 only) is fitted
on Asimov data, whose optimum is theta_true with -lnL = 0 by construction.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, f"fit_{name}.json")) as f:
        g = json.load(f)
    s = dataset(name)
    sha = hashlib.sha256(np.ascontiguousarray(s.counts_vector(), dtype=np.float64).tobytes()).hexdigest()
    assert sha == g["counts_sha256"], "stored oracle fit is for other data: rerun tests/golden/make_fit_golden.py"
    assert g["status"] == 0
    return s, g


def check(s, g, out, info, n):
    free = s.default_free().astype(bool)
    ref = np.asarray(g["theta"])
    tol = np.maximum(1e-4 * np.abs(ref), 0.01 * np.asarray(g["sigma"]))
    for j in range(n):
        assert info[j]["status"] == bx.BX_OK, info[j]
        d = np.abs(out[j, : s.P] - ref)
        assert np.all(d[free] <= tol[free]), (int(np.argmax(d[free] / tol[free])), float((d[free] / tol[free]).max()))
        assert 2 * abs(info[j]["nll"] - g["nll"]) <= 1e-3, (info[j]["nll"], g["nll"])


@pytest.mark.parametrize("name", ["multivariate", "plain"])
def test_fp64_fit_matches_the_oracle_fit(name):
    s, g = golden(name)
    m = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.1, seed=900, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-9)
    check(s, g, out, info, 2)
    m.close()


@pytest.mark.parametrize("name", ["multivariate", "plain"])
def test_fp32_fit_polished_in_fp64_matches_the_oracle_fit(name):
    s, g = golden(name)
    m32 = bx.Model(s, precision=bx.BX_FP32, max_batch=2 * (8 + 2 * s.P))
    m64 = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.1, seed=901, free=s.default_free())
    out32, info32, st32 = m32.fit(th0)
    assert st32 == bx.BX_OK, info32
    out, info, st = m64.fit(out32, tol_edm=1e-9)
    check(s, g, out, info, 2)
    assert max(r["n_evals"] for r in info) < max(r["n_evals"] for r in info32)
    m32.close()
    m64.close()


def test_discrimination_fit_on_asimov_data_returns_truth():
    """The full 2D model on Asimov data (n = the oracle's expected counts at theta_true): the FP32
    fit from 2% starts returns theta_true within max(1e-4 |theta|, 0.05 sigma) (the FP32 noise
    floor; sigma from the fit's inverse Hessian) and -2 lnL within 1e-3 of the optimum's 0."""
    s = I.config("discrimination")
    s = s.with_counts(O.expected(s, s.theta_true))
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.02, seed=902, free=s.default_free())
    out, info, st = m.fit(th0, want_cov=True)
    free = s.default_free().astype(bool)
    for j in range(2):
        assert info[j]["status"] == bx.BX_OK, info[j]
        sig = np.sqrt(np.maximum(np.diag(info[j]["cov"])[: s.P], 0.0))
        tol = np.maximum(1e-4 * np.abs(s.theta_true), 0.05 * sig)
        d = np.abs(out[j, : s.P] - s.theta_true)
        assert np.all(d[free] <= tol[free]), (int(np.argmax(d[free] / tol[free])), float((d[free] / tol[free]).max()))
        assert 2 * abs(info[j]["nll"]) <= 1e-3
    m.close()
