"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic of each precision mode):
  * expected counts per bin: relative 1e-5 on bins with mu >= 1e-3 max(mu), absolute
    1e-8 max(mu) below (FP64 path: 1e-10 relative);
  * mean signed relative error over the bins with mu >= 1e-3 max(mu): <= 1e-8 in the
    mixed-precision modes (no systematic error: the Baker-Cousins sum turns a bias b into
    Delta(-2 lnL) ~ 2 b |sum(mu - n)|);
  * -lnL: |Delta(-2 lnL)| <= 1e-3 (FP64 path: 1e-7);
  * gradient: |Delta g_j| |theta_j| <= tol (1 + |g_j theta_j|), the change of -lnL predicted
    for a relative step of one in theta_j: tol = 1e-9 (FP64), 1e-3 (FP32, TF32X3).
The tensor-core mode BX_TF32X3 is held to the same bounds as BX_FP32: its contraction makes
the dominant hi * hi products exact in the FP32 accumulator (split3).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

PRECS = [bx.BX_FP64, bx.BX_FP32, bx.BX_TF32X3]
TOL = {bx.BX_FP64: dict(rel=1e-10, abs=1e-12, d2nll=1e-7, grad=1e-9, bias=1e-12),
       bx.BX_FP32: dict(rel=1e-5, abs=1e-8, d2nll=1e-3, grad=1e-3, bias=1e-8),
       bx.BX_TF32X3: dict(rel=1e-5, abs=1e-8, d2nll=1e-3, grad=1e-3, bias=1e-8)}


def d2nll_tol(prec, spec, theta):
    return TOL[prec]["d2nll"]


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
@pytest.mark.parametrize("name", ["small_plain", "small_mv", "plain", "multivariate"])
def test_expected_counts_per_bin(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=3)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= TOL[prec]["bias"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["small_plain", "small_mv", "plain", "multivariate"])
def test_nll_and_gradient(name, prec):
    s = dataset(name)
    m = model(name, prec)
    for th in [s.theta_true] + list(points(s, 2, seed=4)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= d2nll_tol(prec, s, th), (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th, TOL[prec]["grad"])
        assert ok, worst


@pytest.mark.parametrize("prec", [bx.BX_FP32, bx.BX_TF32X3])
def test_nll_far_from_the_optimum(prec):
    """Points 6% (rms) away from theta_true, where hundreds of bins have |n - mu| between mu/4
    and mu, the Baker-Cousins terms reach a few hundred and -lnL is ~1e5: |Delta(-2 lnL)| <= 1e-3
    all the same (the bound of every other point)."""
    s = dataset("multivariate")
    m = model("multivariate", prec)
    n = s.counts_vector()
    th = I.parameter_points(s.theta_true, 3, rel=0.06, seed=41, free=s.default_free())
    for t in th:
        mo = O.expected(s, t)
        x = (n - mo) / mo
        assert np.count_nonzero((np.abs(x) > 0.25) & (x >= -0.5) & (x <= 1.0)) > 300
        f, g = m.nll_grad(t)
        fo, go = O.nll(s, t, grad=True)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, t, TOL[prec]["grad"])
        assert ok, worst


@pytest.mark.parametrize("prec", PRECS)
def test_batch_equals_single_calls(prec):
    s = dataset("small_mv")
    m = model("small_mv", prec)
    th = points(s, 8, seed=5)
    f, g = m.nll_batch(th, grad=True)
    for j in range(8):
        fj, gj = m.nll_grad(th[j])
        assert f[j] == fj
        np.testing.assert_array_equal(g[j], gj)


def test_fd_gradient_fp64():
    """The adjoint against central finite differences of the GPU -lnL (step 1e-4 relative)."""
    s = dataset("small_mv")
    m = model("small_mv", bx.BX_FP64)
    th = points(s, 1, seed=6)[0]
    _, g = m.nll_grad(th)
    for j in np.nonzero(s.default_free())[0]:
        h = 1e-4 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (m.nll(tp) - m.nll(tm)) / (2 * h)
        assert abs(fd - g[j]) * abs(th[j]) <= 1e-6 * (1 + abs(g[j] * th[j])), (j, fd, g[j])


def test_device_pointers_and_autograd():
    import torch
    s = dataset("small_mv")
    m = model("small_mv", bx.BX_FP32)
    th = torch.tensor(points(s, 4, seed=7), dtype=torch.float64, device="cuda", requires_grad=True)
    f = bx.BxNLL.apply(th, m)
    (f * torch.arange(1, 5, device="cuda", dtype=torch.float64)).sum().backward()
    fh, gh = m.nll_batch(th.detach().cpu().numpy(), grad=True)
    np.testing.assert_array_equal(f.detach().cpu().numpy(), fh)
    np.testing.assert_array_equal(th.grad.cpu().numpy(), gh * np.arange(1, 5)[:, None])


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_toys_in_one_model(prec):
    """Toys with different bin counts, species sets and a window shorter than one tile."""
    base = I.toy_batch(n_toys=3, n_grid=700, seed=2, bins=(40, 700), L=120)
    specs = []
    for t, s in enumerate(base):
        s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 10 + t))
        specs.append(s)
    m = bx.Model(specs, precision=prec, max_batch=6)
    P = m.P
    th = np.zeros((6, P))
    toys = [0, 1, 2, 2, 1, 0]
    for j, t in enumerate(toys):
        th[j, : specs[t].P] = points(specs[t], 1, seed=20 + j)[0]
    f, g = m.nll_batch(th, toy_idx=toys, grad=True)
    for j, t in enumerate(toys):
        fo, go = O.nll(specs[t], th[j, : specs[t].P], grad=True)
        assert 2 * abs(f[j] - fo) <= d2nll_tol(prec, specs[t], th[j, : specs[t].P])
        ok, worst = grad_ok(g[j, : specs[t].P], go, th[j, : specs[t].P], TOL[prec]["grad"])
        assert ok, worst
        assert np.all(g[j, specs[t].P:] == 0)
        ok, wr, wa = per_bin_ok(m.expected(th[j], toy=t), O.expected(specs[t], th[j, : specs[t].P]),
                                rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
        assert ok, (wr, wa)


def test_domain_and_invalid_parameters():
    s = dataset("small_plain")
    m = model("small_plain", bx.BX_FP32)
    th = s.theta_true.copy()
    th[: s.K] = -1.0                       # negative rates: mu < 0 where data are present
    with pytest.raises(bx.BxError) as e:
        m.nll(th)
    assert e.value.status == bx.BX_EDOMAIN
    th = s.theta_true.copy()
    th[s.K + 3] = -1e6                     # sigma^2 <= 0
    with pytest.raises(bx.BxError) as e:
        m.nll(th)
    assert e.value.status == bx.BX_EDOMAIN
    th = s.theta_true.copy()
    th[0] = np.nan
    with pytest.raises(bx.BxError) as e:
        m.nll(th)
    assert e.value.status == bx.BX_EINVAL
    # the model still evaluates afterwards, and a domain item in a batch does not spoil the others
    th2 = np.stack([s.theta_true, th * 0 - 1.0 + 0 * s.theta_true])
    th2[1] = s.theta_true; th2[1, :s.K] = -1
    f = m.nll_batch(th2, check=False)
    assert np.isfinite(f[0]) and np.isinf(f[1])
    assert abs(f[0] - O.nll(s, s.theta_true)) * 2 <= 1e-3


def test_zero_count_bins():
    s = dataset("small_plain")
    s = s.with_counts(np.where(np.arange(s.n_bins_total) % 3 == 0, 0.0, s.counts_vector()))
    m = bx.Model(s, precision=bx.BX_FP32)
    th = points(s, 1, seed=9)[0]
    f, g = m.nll_grad(th)
    fo, go = O.nll(s, th, grad=True)
    assert 2 * abs(f - fo) <= 1e-3
