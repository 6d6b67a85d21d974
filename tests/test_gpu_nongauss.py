"""The non-Gaussian (Gram-Charlier) response on the GPU against the oracle, through the C ABI.
BX_FP64: expected counts per bin (relative 1e-10), -lnL (|Delta(-2 lnL)| <= 1e-7) and gradient
(|Delta g_j| |theta_j| <= 1e-9 (1 + |g_j theta_j|)) of the reduced and the full-size model,
batch = single calls, the fit against the oracle's fit.  BX_FP32 (the generator's Gram-Charlier
nodes, the row-by-row adjoint) with the mixed modes' bounds: per bin 1e-5 relative (1e-8 max(mu)
absolute), mean signed per-bin error 1e-8, |Delta(-2 lnL)| <= 1e-3, gradient 1e-3 (1 + |g theta|),
and its fit polished in FP64 against the oracle's.  The rejections (BX_TF32X3, a density that
turns negative within the band)."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

_models = {}


def model(name, max_batch=8, prec=bx.BX_FP64):
    key = (name, max_batch, prec)
    if key not in _models:
        _models[key] = bx.Model(dataset(name), precision=prec, max_batch=max_batch)
    return _models[key]


def grad_ok(g, go, th, tol=1e-9):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


@pytest.mark.parametrize("name", ["small_nongauss", "nongauss"])
def test_nongauss_expected_counts(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2, seed=120)):
        ok, wr, wa = per_bin_ok(m.expected(th), O.expected(s, th), rel=1e-10, abs_frac=1e-12)
        assert ok, (wr, wa)


@pytest.mark.parametrize("name", ["small_nongauss", "nongauss"])
def test_nongauss_nll_and_gradient(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2, seed=121)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-7, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th)
        assert ok, worst


def test_nongauss_differs_from_the_gaussian():
    """The skewness and kurtosis move counts: the expected counts differ from the Gaussian model's
    by far more than the parity bound (the test above would not notice a dropped term otherwise)."""
    s = dataset("small_nongauss")
    g = dataclasses.replace(s, resp_skew=0.0, resp_kurt=0.0)
    mg = bx.Model(g, precision=bx.BX_FP64)
    a, b = model("small_nongauss").expected(s.theta_true), mg.expected(s.theta_true)
    big = b > 1e-3 * b.max()
    assert np.max(np.abs(a[big] / b[big] - 1)) > 1e-3
    mg.close()


def test_nongauss_batch_equals_single_calls():
    s = dataset("small_nongauss")
    m = model("small_nongauss")
    th = points(s, 6, seed=122)
    f, g = m.nll_batch(th, grad=True)
    for k in range(6):
        fk, gk = m.nll_grad(th[k])
        assert f[k] == fk
        np.testing.assert_array_equal(g[k], gk)


def test_nongauss_fit_agrees_with_oracle():
    s = dataset("small_nongauss")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    m = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.03, seed=123, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-9)
    free = s.default_free().astype(bool)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), 0.01 * sig)
    for k in range(2):
        assert info[k]["status"] == bx.BX_OK, info[k]
        d = np.abs(out[k, : s.P] - ref["theta"])
        assert np.all(d[free] <= tol[free]), (d[free] / tol[free]).max()
        assert 2 * abs(info[k]["nll"] - ref["nll"]) <= 1e-3
    m.close()


@pytest.mark.parametrize("name", ["small_nongauss", "nongauss"])
def test_nongauss_fp32_expected_counts(name):
    s = dataset(name)
    m = model(name, prec=bx.BX_FP32)
    for th in [s.theta_true] + list(points(s, 2, seed=124)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=1e-5, abs_frac=1e-8)
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= 1e-8


@pytest.mark.parametrize("name", ["small_nongauss", "nongauss"])
def test_nongauss_fp32_nll_and_gradient(name):
    s = dataset(name)
    m = model(name, prec=bx.BX_FP32)
    for th in [s.theta_true] + list(points(s, 2, seed=125)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, tol=1e-3)
        assert ok, worst


def test_nongauss_fp32_fit_polished_in_fp64_agrees_with_oracle():
    s = dataset("small_nongauss")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    m32 = bx.Model(s, precision=bx.BX_FP32, max_batch=2 * (8 + 2 * s.P))
    m64 = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.03, seed=126, free=s.default_free())
    out32, info32, st32 = m32.fit(th0)
    assert st32 == bx.BX_OK, info32
    out, info, st = m64.fit(out32, tol_edm=1e-9)
    free = s.default_free().astype(bool)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), 0.01 * sig)
    for k in range(2):
        assert info[k]["status"] == bx.BX_OK, info[k]
        d = np.abs(out[k, : s.P] - ref["theta"])
        assert np.all(d[free] <= tol[free]), (d[free] / tol[free]).max()
        assert 2 * abs(info[k]["nll"] - ref["nll"]) <= 1e-3
    m32.close()
    m64.close()


def test_nongauss_rejections():
    s = dataset("small_nongauss")
    with pytest.raises(bx.BxError) as e:
        bx.Model(s, precision=bx.BX_TF32X3)
    assert e.value.status == bx.BX_EINVAL
    bad = dataclasses.replace(s, resp_skew=0.6, resp_kurt=0.0)   # 1 + 0.1 (z^3 - 3z) < 0 below z ~ -2.5
    with pytest.raises(bx.BxError) as e:
        bx.Model(bad, precision=bx.BX_FP64)
    assert e.value.status == bx.BX_EINVAL
