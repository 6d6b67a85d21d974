"""The discrimination regime (2D energy x radius and energy x pulse-shape histograms next to
the TFC spectra, all as slices of tensor-core GEMMs) against the FP64 oracle, through the C ABI.

Tolerances as for the FP32 mode: per-bin relative 1e-5 (absolute 1e-8 max(mu) below
1e-3 max(mu)), |Delta(-2 lnL)| <= 1e-3, gradient |Delta g_j| |theta_j| <= 1e-3 (1 + |g_j theta_j|).
The forward GEMM carries no systematic error (its hi*hi products are exact in the tensor
core's accumulator); the test also bounds the mean signed per-bin error at 1e-8.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

_models = {}


def model(name, max_batch=8):
    key = (name, max_batch)
    if key not in _models:
        _models[key] = bx.Model(dataset(name), precision=bx.BX_FP32, max_batch=max_batch)
    return _models[key]


def grad_ok(g, go, th, tol=1e-3):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


@pytest.mark.parametrize("name", ["small_2d", "discrimination"])
def test_2d_expected_counts_per_bin(name):
    s = dataset(name)
    m = model(name)
    pts = [s.theta_true] + list(points(s, 2 if name == "small_2d" else 1, seed=31))
    for th in pts:
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=1e-5, abs_frac=1e-8)
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= 1e-8


@pytest.mark.parametrize("name", ["small_2d", "discrimination"])
def test_2d_nll_and_gradient(name):
    s = dataset(name)
    m = model(name)
    pts = [s.theta_true] + list(points(s, 3 if name == "small_2d" else 1, seed=32))
    for th in pts:
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th)
        assert ok, worst


def test_2d_batch_equals_single_calls():
    s = dataset("small_2d")
    m = model("small_2d")
    th = points(s, 8, seed=33)
    f, g = m.nll_batch(th, grad=True)
    for j in range(8):
        fj, gj = m.nll_grad(th[j])
        assert f[j] == fj
        np.testing.assert_array_equal(g[j], gj)


def test_2d_without_field_matches_the_1d_path():
    """Two independent GPU paths: with amp = 0, the 2D slices summed over radius equal the
    TFC-vetoed spectrum of the rate-first CUDA-core path of the 1D model."""
    s = dataset("small_2d")
    s0 = dataclasses.replace(s, field_amp=0.0)
    m2 = bx.Model(s0, precision=bx.BX_FP32)
    s1 = dataclasses.replace(s0, n_rad2d=0, psd2d_prob=None, field2d=None)
    s1 = s1.with_counts(s0.counts_vector()[: 2 * s0.n_window])
    m1 = bx.Model(s1, precision=bx.BX_FP32)
    th = points(s, 1, seed=34)[0]
    mu2, mu1 = m2.expected(th), m1.expected(th)
    nw = s.n_window
    r2 = mu2[2 * nw:2 * nw + s.n_rad2d * nw].reshape(s.n_rad2d, nw).sum(axis=0)
    np.testing.assert_allclose(mu2[:nw], mu1[:nw], rtol=1e-6)
    np.testing.assert_allclose(r2, mu1[:nw], rtol=1e-6)
    m1.close()
    m2.close()


def test_2d_fit_agrees_with_oracle():
    """FP32 fits of the 2D model on the device against the oracle's Newton fit:
    |d theta| <= max(1e-4 |theta|, 0.05 sigma) (the FP32 noise floor), -2 lnL within 1e-3.
    Asimov data (n = mu(theta_true)): with Poisson data this small model's resolution and
    radial parameters are so weakly constrained that the likelihood has several minima on the
    bounds, and two correct minimisers may end in different ones; with Asimov data the
    optimum is theta_true, interior and unique."""
    s = I.config("small_2d")
    s = s.with_counts(O.expected(s, s.theta_true))
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    free = s.default_free().astype(bool)
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=4 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 4, rel=0.05, seed=35, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-8, max_iter=5000)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), 0.05 * sig)
    for j in range(4):
        assert info[j]["status"] == bx.BX_OK, info[j]
        d = np.abs(out[j, : s.P] - ref["theta"])
        assert np.all(d[free] <= tol[free]), (d[free] / tol[free]).max()
        assert 2 * abs(info[j]["nll"] - ref["nll"]) <= 1e-3
    m.close()


def test_2d_adjoint_through_autograd_matches_oracle_and_central_differences():
    """The differentiated 2D fit's gradient: torch autograd through bx.BxNLL (the hand-written
    adjoint, response regenerated in the adjoint kernel) at a point 2% off theta_true
    - is bit for bit the gradient of Model.nll_grad (the same kernels);
    - agrees with the oracle's dual-number gradient to 1e-3 (1 + |g_j theta_j|) in |dg_j theta_j|;
    - agrees with central differences of the FP32 -lnL (relative step 1e-3) within that bound
      plus the difference quotient's rounding noise, allowed at 1e-8 of -lnL per value (4e-9 of
      it was seen), i.e. 2e-8 |f| / (2 h) in the quotient."""
    import torch
    s = dataset("small_2d")
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=2)
    th = points(s, 1, seed=140)[0]
    t = torch.tensor(th[None, :], dtype=torch.float64, device="cuda", requires_grad=True)
    f0 = bx.BxNLL.apply(t, m)
    f0.sum().backward()
    g = t.grad[0].cpu().numpy()
    fd0, gd = m.nll_grad(th)
    np.testing.assert_array_equal(g, gd)
    assert float(f0.detach()[0]) == fd0
    fo, go = O.nll(s, th, grad=True)
    ok = np.abs(g[: s.P] - go) * np.abs(th) <= 1e-3 * (1 + np.abs(go * th))
    assert np.all(ok), np.nonzero(~ok)[0]
    for j in np.nonzero(s.default_free())[0]:
        h = 1e-3 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        f = bx.BxNLL.apply(torch.tensor(np.stack([tp, tm]), dtype=torch.float64, device="cuda"), m)
        fd = float(f[0] - f[1]) / (2 * h)
        noise = 2e-8 * abs(fd0) / (2 * h) * abs(th[j])
        assert abs(fd - g[j]) * abs(th[j]) <= 1e-3 * (1 + abs(g[j] * th[j])) + noise, (j, fd, g[j], go[j], fd0)
    m.close()
