"""The position-dependent response (radial shells, each with its own light-yield factor, every
species spread over them by fixed fractions) on the GPU against the oracle, through the C ABI
(also together with the Gram-Charlier response and with energy slices of the Eq. 4 terms).
BX_FP64: expected counts per bin (relative 1e-10), -lnL (|Delta(-2 lnL)| <= 1e-7) and gradient
(|Delta g_j| |theta_j| <= 1e-9 (1 + |g_j theta_j|)) of the reduced and the full-size model, one
shell and four, batch = single calls, the fit against the oracle's fit.  BX_FP32 with the mixed
modes' bounds: per bin 1e-5 relative (1e-8 max(mu) absolute), mean signed per-bin error 1e-8,
|Delta(-2 lnL)| <= 1e-3 (points 2 % and 6 % from the truth), gradient 1e-3 (1 + |g theta|), and
its fit polished in FP64 against the oracle's.  The rejections (BX_TF32X3, 2D histograms,
several Birks multipliers, several energy estimators)."""
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


def one_shell(s, f=1.07):
    return dataclasses.replace(s, shell_ly=np.array([f]), shell_frac=np.ones((s.K, 1)))


@pytest.mark.parametrize("name", ["small_shelled", "shelled"])
def test_shells_expected_counts(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2, seed=130)):
        ok, wr, wa = per_bin_ok(m.expected(th), O.expected(s, th), rel=1e-10, abs_frac=1e-12)
        assert ok, (wr, wa)


@pytest.mark.parametrize("name", ["small_shelled", "shelled"])
def test_shells_nll_and_gradient(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2, seed=131)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-7, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th)
        assert ok, worst


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
def test_one_shell_against_oracle(prec):
    """A single shell (one set of columns, its light-yield factor folded into Q) in both precisions."""
    s = one_shell(dataset("small_shelled"))
    m = bx.Model(s, precision=prec)
    rel, gtol, ftol = (1e-10, 1e-9, 1e-7) if prec == bx.BX_FP64 else (1e-5, 1e-3, 1e-3)
    for th in [s.theta_true] + list(points(s, 2, seed=132)):
        ok, wr, wa = per_bin_ok(m.expected(th), O.expected(s, th), rel=rel, abs_frac=1e-8)
        assert ok, (wr, wa)
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= ftol, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, tol=gtol)
        assert ok, worst
    m.close()


def test_shells_differ_from_the_single_response():
    """The shells move counts: the expected counts differ from those of one response for the
    whole volume by far more than the parity bound."""
    s = dataset("small_shelled")
    base = dataclasses.replace(s, shell_ly=None, shell_frac=None)
    mb = bx.Model(base, precision=bx.BX_FP64)
    a, b = model("small_shelled").expected(s.theta_true), mb.expected(s.theta_true)
    big = b > 1e-3 * b.max()
    assert np.max(np.abs(a[big] / b[big] - 1)) > 1e-3
    mb.close()


def test_shells_batch_equals_single_calls():
    s = dataset("small_shelled")
    m = model("small_shelled")
    th = points(s, 6, seed=133)
    f, g = m.nll_batch(th, grad=True)
    for k in range(6):
        fk, gk = m.nll_grad(th[k])
        assert f[k] == fk
        np.testing.assert_array_equal(g[k], gk)


def test_shells_fit_agrees_with_oracle():
    s = dataset("small_shelled")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    m = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.03, seed=134, free=s.default_free())
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


@pytest.mark.parametrize("name", ["small_shelled", "shelled"])
def test_shells_fp32_expected_counts(name):
    s = dataset(name)
    m = model(name, prec=bx.BX_FP32)
    for th in [s.theta_true] + list(points(s, 2, seed=135)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=1e-5, abs_frac=1e-8)
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= 1e-8


@pytest.mark.parametrize("name", ["small_shelled", "shelled"])
def test_shells_fp32_nll_and_gradient(name):
    s = dataset(name)
    m = model(name, prec=bx.BX_FP32)
    for th in [s.theta_true] + list(points(s, 2, seed=136)) + list(points(s, 1, rel=0.06, seed=137)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, tol=1e-3)
        assert ok, worst


def test_shells_fp32_fit_polished_in_fp64_agrees_with_oracle():
    s = dataset("small_shelled")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    m32 = bx.Model(s, precision=bx.BX_FP32, max_batch=2 * (8 + 2 * s.P))
    m64 = bx.Model(s, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 2, rel=0.03, seed=138, free=s.default_free())
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


def test_shells_rejections():
    s = dataset("small_shelled")
    with pytest.raises(bx.BxError) as e:
        bx.Model(s, precision=bx.BX_TF32X3)
    assert e.value.status == bx.BX_EINVAL
    for bad in [dataclasses.replace(s, quench=np.where(np.arange(s.K) == 0, 2.0, 1.0)),
                dataclasses.replace(s, shell_ly=np.array([1.0, -1.0, 1.0, 1.0])),
                dataclasses.replace(s, shell_ly=np.ones(5), shell_frac=np.full((s.K, 5), 0.2))]:
        with pytest.raises(bx.BxError) as e:
            bx.Model(bad, precision=bx.BX_FP64)
        assert e.value.status == bx.BX_EINVAL
    d = I.config("small_2d")
    d = dataclasses.replace(d, shell_ly=np.ones(2), shell_frac=np.full((d.K, 2), 0.5))
    d = d.with_counts(np.ones(d.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(d, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
def test_shells_with_the_gram_charlier_response(prec):
    """Radial shells together with the non-Gaussian response (each shell's columns with the
    Gram-Charlier bin masses) against the oracle, with each precision's bounds."""
    s = dataclasses.replace(I.config("small_shelled"), resp_skew=0.1, resp_kurt=0.1)
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 5))
    m = bx.Model(s, precision=prec)
    rel, gtol, ftol = (1e-10, 1e-9, 1e-7) if prec == bx.BX_FP64 else (1e-5, 1e-3, 1e-3)
    for th in [s.theta_true] + list(points(s, 2, seed=139)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=rel, abs_frac=1e-8)
        assert ok, (wr, wa)
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= ftol, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, tol=gtol)
        assert ok, worst
    m.close()


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
def test_shells_with_energy_slices(prec):
    """Radial shells together with Eq. 4's terms in three energy slices (each slice's window
    masses per shell column, the species sums weighted per shell) against the oracle."""
    sh = I.config("small_shelled")
    s = dataclasses.replace(I.config("small_sliced"), shell_ly=sh.shell_ly, shell_frac=sh.shell_frac)
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 6))
    m = bx.Model(s, precision=prec)
    rel, gtol, ftol = (1e-10, 1e-9, 1e-7) if prec == bx.BX_FP64 else (1e-5, 1e-3, 1e-3)
    for th in [s.theta_true] + list(points(s, 2, seed=141)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=rel, abs_frac=1e-8)
        assert ok, (wr, wa)
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= ftol, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, tol=gtol)
        assert ok, worst
    m.close()
