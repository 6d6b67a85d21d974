"""The joint energy x radius x pulse-shape grid (one 2D slice per radius x pulse-shape cell, on
the tensor-core path of the 2D model) against the FP64 oracle, through the C ABI.  Tolerances as
for the 2D model (tests/test_gpu_2d.py): per-bin relative 1e-5 (absolute 1e-8 max(mu) below
1e-3 max(mu)), |Delta(-2 lnL)| <= 1e-3, gradient |Delta g_j| |theta_j| <= 1e-3 (1 + |g_j theta_j|),
mean signed per-bin error <= 1e-8."""
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


def split(spec, mu):
    out, o = {}, 0
    for h, n in spec.hist_sizes().items():
        out[h] = mu[o:o + n]
        o += n
    return out


@pytest.mark.parametrize("name", ["small_joint", "joint"])
def test_joint_expected_counts_per_bin(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2 if name == "small_joint" else 1, seed=101)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=1e-5, abs_frac=1e-8)
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= 1e-8


def test_joint_nll_and_gradient():
    s = dataset("small_joint")
    m = model("small_joint")
    for th in [s.theta_true] + list(points(s, 3, seed=102)):
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)
        ok, worst = grad_ok(g[: s.P], go, th)
        assert ok, worst


def test_joint_full_size_nll():
    """|Delta(-2 lnL)| <= 1e-3 at theta_true and at two points 2% away (there a per-bin relative
    bias delta would add 2 delta |sum mu - sum n|, ~4.5e4 events here: the forward's exact
    accumulation keeps the mean per-bin error at ~1e-10)."""
    s = dataset("joint")
    m = model("joint")
    assert 2 * abs(m.nll(s.theta_true) - O.nll(s, s.theta_true)) <= 1e-3
    for th in points(s, 2, seed=103):
        assert 2 * abs(m.nll(th) - O.nll(s, th)) <= 1e-3


def test_joint_marginals_against_the_separate_2d_model():
    """Two GPU models at field amplitude 0: the joint grid summed over pulse shape is the separate
    model's energy x radius histogram, summed over radius its energy x pulse-shape histogram."""
    j = dataclasses.replace(I.config("small_joint"), field_amp=0.0)
    sep = dataclasses.replace(j, joint2d=False,
                              field2d=np.ascontiguousarray(I.smooth_field(j.n_grid, j.n_rad2d + j.n_psd2d, 0)))
    j = j.with_counts(np.ones(j.n_bins_total))
    sep = sep.with_counts(np.ones(sep.n_bins_total))
    mj, ms = bx.Model(j, precision=bx.BX_FP32), bx.Model(sep, precision=bx.BX_FP32)
    th = points(j, 1, seed=104)[0]
    hj, hs = split(j, mj.expected(th)), split(sep, ms.expected(th))
    grid = hj["j2d"].reshape(j.n_rad2d, j.n_psd2d, j.n_window)
    np.testing.assert_allclose(hj["sub"], hs["sub"], rtol=1e-6)
    np.testing.assert_allclose(grid.sum(axis=1).ravel(), hs["r2d"], rtol=2e-6, atol=1e-9 * hs["r2d"].max())
    np.testing.assert_allclose(grid.sum(axis=0).ravel(), hs["p2d"], rtol=2e-6, atol=1e-9 * hs["p2d"].max())
    mj.close()
    ms.close()


def test_joint_batch_equals_single_calls():
    s = dataset("small_joint")
    m = model("small_joint")
    th = points(s, 8, seed=105)
    f, g = m.nll_batch(th, grad=True)
    for k in range(8):
        fk, gk = m.nll_grad(th[k])
        assert f[k] == fk
        np.testing.assert_array_equal(g[k], gk)


def test_joint_fit_agrees_with_oracle():
    """FP32 fits of the small joint model on Asimov data (the optimum is theta_true, interior and
    unique) against the oracle's Newton fit: |d theta| <= max(1e-4 |theta|, 0.05 sigma) (the FP32
    noise floor), -2 lnL within 1e-3."""
    s = I.config("small_joint")
    s = s.with_counts(O.expected(s, s.theta_true))
    ref = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert ref["status"] == 0
    free = s.default_free().astype(bool)
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=4 * (8 + 2 * s.P))
    th0 = I.parameter_points(s.theta_true, 4, rel=0.05, seed=106, free=s.default_free())
    out, info, st = m.fit(th0, tol_edm=1e-8, max_iter=5000)
    sig = np.sqrt(np.maximum(np.diag(ref["cov"]), 0.0))
    tol = np.maximum(1e-4 * np.abs(ref["theta"]), 0.05 * sig)
    for k in range(4):
        assert info[k]["status"] == bx.BX_OK, info[k]
        d = np.abs(out[k, : s.P] - ref["theta"])
        assert np.all(d[free] <= tol[free]), (d[free] / tol[free]).max()
        assert 2 * abs(info[k]["nll"] - ref["nll"]) <= 1e-3
    m.close()
