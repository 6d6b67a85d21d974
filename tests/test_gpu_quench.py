"""Species-specific quenching (the alpha and gamma species quench with their own multiple of
kB, each group with its own Birks map and response columns) against the FP64 oracle, through
the C ABI, with the tolerances of the plain model (tests/test_gpu_parity.py)."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

PRECS = [bx.BX_FP64, bx.BX_FP32]
TOL = {bx.BX_FP64: dict(rel=1e-10, abs=1e-12, d2nll=1e-7, grad=1e-9, bias=1e-12),
       bx.BX_FP32: dict(rel=1e-5, abs=1e-8, d2nll=1e-3, grad=1e-3, bias=1e-8)}

_models = {}


def model(name, prec, max_batch=8):
    key = (name, prec, max_batch)
    if key not in _models:
        _models[key] = bx.Model(dataset(name), precision=prec, max_batch=max_batch)
    return _models[key]


def grad_ok(g, go, th, tol):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small_quenched", "quenched"])
def test_quenched_expected_counts_per_bin(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=71)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= TOL[prec]["bias"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small_quenched", "quenched"])
def test_quenched_nll_and_gradient(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=72)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= TOL[prec]["d2nll"], (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, TOL[prec]["grad"])
        assert ok, worst


@pytest.mark.parametrize("prec", PRECS)
def test_quench_of_one_is_the_plain_model(prec):
    """Multipliers of 1 for every species take the plain path: bit-identical results."""
    s = dataset("small_quenched")
    plain = dataclasses.replace(s, quench=None)
    ones = dataclasses.replace(s, quench=np.ones(s.K))
    th = points(s, 1, seed=73)[0]
    m1, m2 = bx.Model(plain, precision=prec), bx.Model(ones, precision=prec)
    f1, g1 = m1.nll_grad(th)
    f2, g2 = m2.nll_grad(th)
    assert f1 == f2
    np.testing.assert_array_equal(g1, g2)
    m1.close()
    m2.close()


@pytest.mark.parametrize("prec", PRECS)
def test_quenched_fit_agrees_with_oracle(prec):
    """Fits of the quenched model on the device against the oracle's Newton fit: every free
    parameter within max(1e-4 |theta|, nsig sigma), nsig = 0.01 (FP64), 0.05 (FP32); a rate the
    oracle holds at its bound 0 within 5e-4 / g (g its gradient there: at most 1e-3 in -2 lnL)."""
    s = dataset("small_quenched")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    nsig = 0.01 if prec == bx.BX_FP64 else 0.05
    free = s.default_free().astype(bool)
    m = bx.Model(s, precision=prec, max_batch=4 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 4, rel=0.03, seed=74, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-8, max_iter=5000)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), nsig * sig)
    at_bound = free & (sig == 0.0)
    if at_bound.any():
        _, g = O.nll(s, ref["theta"], grad=True)
        assert np.all(g[at_bound] > 0.0), g[at_bound]
        tol[at_bound] = 5e-4 / g[at_bound]
    for j in range(4):
        assert info[j]["status"] == bx.BX_OK, info[j]
        d = np.abs(out[j, : s.P] - ref["theta"])
        bad = np.nonzero(free & (d > tol))[0]
        assert bad.size == 0, (j, bad, d[bad], tol[bad], out[j, bad], ref["theta"][bad])
    m.close()
