"""Several energy estimators of one dataset fitted jointly (bx_model_create_estimators) against the
FP64 oracle, through the C ABI.  Sec. 3: the charge, the number of detected photons and the number
of fired channels are each an observable with its own response (Eq. 1); they share the rates, kB,
eps and s_r.  Tolerances as for the single models (tests/test_gpu_parity.py): per-bin relative 1e-5
(absolute 1e-8 max(mu) below 1e-3 max(mu)), |Delta(-2 lnL)| <= 1e-3 (FP64: 1e-7), gradient
|Delta g_j| |theta_j| <= tol (1 + |g_j theta_j|) with tol 1e-3 (FP32) or 1e-9 (FP64)."""
import functools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import per_bin_ok

pytestmark = pytest.mark.gpu

NAMES = ("npe", "charge", "nhits")
TOL = {bx.BX_FP64: dict(rel=1e-10, abs=1e-12, d2nll=1e-7, grad=1e-9),
       bx.BX_FP32: dict(rel=1e-5, abs=1e-8, d2nll=1e-3, grad=1e-3)}


@functools.lru_cache(maxsize=None)
def estimators(base="small_mv", names=NAMES, seed=60):
    sp = I.estimators(base, names)
    return tuple(s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), seed + e)) for e, s in enumerate(sp))


def joint_points(specs, n, seed, rel=0.02):
    free, _, _ = O.estimator_defaults(list(specs))
    return I.parameter_points(I.estimator_theta(list(specs)), n, rel=rel, seed=seed, free=free)


_models = {}


def model(base, prec, max_batch=8):
    key = (base, prec, max_batch)
    if key not in _models:
        _models[key] = bx.Model(list(estimators(base)), precision=prec, max_batch=max_batch, n_est=len(NAMES))
    return _models[key]


def grad_ok(g, go, th, tol):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
@pytest.mark.parametrize("base", ["small_mv", "multivariate"])
def test_estimators_expected_counts(base, prec):
    sp = list(estimators(base))
    m = model(base, prec)
    assert m.P == sp[0].K + 7 + 4 * (len(sp) - 1)
    assert m.n_bins() == sum(s.n_bins_total for s in sp)
    for th in joint_points(sp, 2, seed=61):
        ok, wr, wa = per_bin_ok(m.expected(th), O.expected_estimators(sp, th), rel=TOL[prec]["rel"],
                                abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
@pytest.mark.parametrize("base", ["small_mv", "multivariate"])
def test_estimators_nll_and_gradient(base, prec):
    sp = list(estimators(base))
    m = model(base, prec)
    for th in [I.estimator_theta(sp)] + list(joint_points(sp, 2, seed=62)):
        f, g = m.nll_grad(th)
        fo, go = O.nll_estimators(sp, th, grad=True)
        assert 2 * abs(f - fo) <= TOL[prec]["d2nll"], (f, fo)
        ok, worst = grad_ok(g, go, th, TOL[prec]["grad"])
        assert ok, worst


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
def test_one_estimator_is_the_single_model(prec):
    """bx_model_create_estimators with n_est = 1 gives the regular model's -lnL and gradient bit
    for bit."""
    s = estimators("small_mv")[0]
    one = bx.Model([s], precision=prec, max_batch=4, n_est=1)
    reg = bx.Model(s, precision=prec, max_batch=4)
    th = joint_points([s], 4, seed=63)
    f1, g1 = one.nll_batch(th, grad=True)
    f2, g2 = reg.nll_batch(th, grad=True)
    np.testing.assert_array_equal(f1, f2)
    np.testing.assert_array_equal(g1, g2)
    one.close()
    reg.close()


def test_estimators_batch_equals_single_calls():
    sp = list(estimators("small_mv"))
    m = model("small_mv", bx.BX_FP32)
    th = joint_points(sp, 8, seed=64)
    f, g = m.nll_batch(th, grad=True)
    for k in range(8):
        fk, gk = m.nll_grad(th[k])
        assert f[k] == fk
        np.testing.assert_array_equal(g[k], gk)


def test_estimators_ragged_datasets_in_one_model():
    """Two datasets of different species counts and windows, three estimators each."""
    a = list(estimators("small_mv"))
    b = [s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 70 + e))
         for e, s in enumerate(I.estimators("small_plain", NAMES))]
    m = bx.Model(a + b, precision=bx.BX_FP64, max_batch=4, n_est=3)
    P = m.P
    th = np.zeros((4, P))
    toys = [0, 1, 1, 0]
    sets = [a, b]
    for j, t in enumerate(toys):
        pj = joint_points(sets[t], 1, seed=80 + j)[0]
        th[j, : pj.shape[0]] = pj
    f, g = m.nll_batch(th, toy_idx=toys, grad=True)
    for j, t in enumerate(toys):
        n = sets[t][0].K + 7 + 8
        fo, go = O.nll_estimators(sets[t], th[j, :n], grad=True)
        assert 2 * abs(f[j] - fo) <= 1e-7
        ok, worst = grad_ok(g[j, :n], go, th[j, :n], 1e-9)
        assert ok, worst
        assert np.all(g[j, n:] == 0)
    m.close()


def test_estimators_reject_unshared_inputs():
    a = list(estimators("small_mv"))
    bad = list(a)
    bad[1] = a[1].with_counts(a[1].counts_vector())
    bad[1].shapes = a[1].shapes * 1.001                    # another deposited-energy spectrum
    with pytest.raises(bx.BxError) as e:
        bx.Model(bad, precision=bx.BX_FP64, n_est=3)
    assert e.value.status == bx.BX_EINVAL
    with pytest.raises(bx.BxError) as e:                   # radial term on estimator 1
        bx.Model([a[0], a[0], a[2]], precision=bx.BX_FP64, n_est=3)
    assert e.value.status == bx.BX_EINVAL


@pytest.mark.parametrize("prec", [bx.BX_FP64, bx.BX_FP32])
def test_estimators_fit_agrees_with_oracle(prec):
    """The joint fit of the three estimators (Poisson data) from 2% starts against the oracle's
    joint fit: |d theta| <= max(1e-4 |theta|, 0.01 sigma) and |Delta(-2 lnL)| <= 1e-3 in FP64;
    FP32 fits polished by FP64 meet the same bounds."""
    sp = list(estimators("small_mv"))
    th_true = I.estimator_theta(sp)
    ref = O.fit_estimators(sp, th_true, tol_edm=1e-12)
    assert ref["status"] == 0
    free, _, _ = O.estimator_defaults(sp)
    P = th_true.shape[0]
    m = bx.Model(sp, precision=prec, max_batch=2 * (8 + 2 * P), n_est=3)
    th0 = joint_points(sp, 2, seed=65)
    out, info, st = m.fit(th0, tol_edm=1e-8)
    assert all(r["status"] == bx.BX_OK for r in info), info
    if prec == bx.BX_FP32:
        m64 = bx.Model(sp, precision=bx.BX_FP64, max_batch=2 * (8 + 2 * P), n_est=3)
        out, info, st = m64.fit(out, tol_edm=1e-8)
        assert all(r["status"] == bx.BX_OK for r in info), info
        m64.close()
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), 0.01 * sig)
    fr = free.astype(bool)
    for k in range(2):
        d = np.abs(out[k] - ref["theta"])
        assert np.all(d[fr] <= tol[fr]), (d[fr] / tol[fr]).max()
        assert 2 * abs(info[k]["nll"] - ref["nll"]) <= 1e-3
    m.close()
