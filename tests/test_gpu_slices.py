"""Eq. 4's radial and pulse-shape terms in several energy slices (one radial and one
pulse-shape histogram per slice of the window) against the FP64 oracle, through the C ABI,
with the tolerances of the plain model (tests/test_gpu_parity.py)."""
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


def split(spec, mu):
    out, o = {}, 0
    for h, n in spec.hist_sizes().items():
        out[h] = mu[o:o + n]
        o += n
    return out


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small_sliced", "sliced"])
def test_sliced_expected_counts_per_bin(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=81)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= TOL[prec]["bias"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small_sliced", "sliced"])
def test_sliced_nll_and_gradient(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=82)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= TOL[prec]["d2nll"], (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, TOL[prec]["grad"])
        assert ok, worst


@pytest.mark.parametrize("prec", PRECS)
def test_slices_sum_to_the_unsliced_model(prec):
    """Two GPU models: the slices' radial and pulse-shape histograms add up, bin by bin, to
    those of the model without slices (which runs the one-slice kernels), and the energy
    spectra are the same."""
    s = dataset("sliced")
    base = dataclasses.replace(s, eslices=None)
    base = base.with_counts(np.concatenate([s.counts["sub"], s.counts["tag"],
                                            s.counts["rad"].reshape(s.n_eslices, -1).sum(axis=0),
                                            s.counts["psd"].reshape(s.n_eslices, -1).sum(axis=0)]))
    mb = bx.Model(base, precision=prec)
    th = points(s, 1, seed=83)[0]
    a, b = split(s, model("sliced", prec).expected(th)), split(base, mb.expected(th))
    rtol = 1e-12 if prec == bx.BX_FP64 else 2e-6
    S = s.n_eslices
    np.testing.assert_allclose(a["sub"], b["sub"], rtol=rtol)
    np.testing.assert_allclose(a["tag"], b["tag"], rtol=rtol)
    np.testing.assert_allclose(a["rad"].reshape(S, -1).sum(axis=0), b["rad"], rtol=rtol)
    np.testing.assert_allclose(a["psd"].reshape(S, -1).sum(axis=0), b["psd"], rtol=rtol)
    mb.close()


@pytest.mark.parametrize("prec", PRECS)
def test_sliced_batch_equals_single_calls(prec):
    s = dataset("small_sliced")
    m = model("small_sliced", prec)
    th = points(s, 8, seed=84)
    f, g = m.nll_batch(th, grad=True)
    for j in range(8):
        fj, gj = m.nll_grad(th[j])
        assert f[j] == fj
        np.testing.assert_array_equal(g[j], gj)


@pytest.mark.parametrize("prec", PRECS)
def test_slices_with_quenching_groups(prec):
    """Energy slices and species-specific quenching together (three quenching groups, three
    slices) against the oracle."""
    q = I.config("small_quenched")
    sl = I.config("small_sliced")
    s = dataclasses.replace(q, eslices=sl.eslices.copy(), name="small_quenched_sliced")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 0))
    m = bx.Model(s, precision=prec)
    for th in [s.theta_true] + list(points(s, 1, seed=85)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= TOL[prec]["d2nll"], (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, TOL[prec]["grad"])
        assert ok, worst
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_sliced_fit_agrees_with_oracle(prec):
    """Fits of the sliced model on the device against the oracle's Newton fit: every free
    parameter within max(1e-4 |theta|, nsig sigma), nsig = 0.01 (FP64), 0.05 (FP32)."""
    s = dataset("small_sliced")
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    nsig = 0.01 if prec == bx.BX_FP64 else 0.05
    free = s.default_free().astype(bool)
    m = bx.Model(s, precision=prec, max_batch=4 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 4, rel=0.03, seed=86, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-8, max_iter=5000)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), nsig * sig)
    for j in range(4):
        assert info[j]["status"] == bx.BX_OK, info[j]
        d = np.abs(out[j, : s.P] - ref["theta"])
        assert np.all(d[free] <= tol[free]), (np.argmax(d[free] / tol[free]), (d[free] / tol[free]).max())
    m.close()
