"""BX_BF16X3: the 2D models' response GEMM on BF16 three-part operands (tcgen05.mma kind::f16, FP32
accumulation), against the FP64 oracle and beside the TF32 three-part GEMM of BX_FP32, through the
C ABI.  Bounds as for the 2D model (tests/test_gpu_2d.py): per-bin relative 1e-5 (absolute 1e-8
max(mu) below 1e-3 max(mu)), mean signed per-bin error <= 1e-8, |Delta(-2 lnL)| <= 1e-3, gradient
|Delta g_j| |theta_j| <= 1e-3 (1 + |g_j theta_j|)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

_models = {}


def model(name, prec=bx.BX_BF16X3, max_batch=4):
    key = (name, prec, max_batch)
    if key not in _models:
        _models[key] = bx.Model(dataset(name), precision=prec, max_batch=max_batch)
    return _models[key]


def grad_ok(g, go, th, tol=1e-3):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


@pytest.mark.parametrize("name", ["small_2d", "discrimination", "small_joint"])
def test_bf16x3_expected_counts(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 1, seed=130)):
        mg, mo = m.expected(th), O.expected(s, th)
        ok, wr, wa = per_bin_ok(mg, mo, rel=1e-5, abs_frac=1e-8)
        assert ok, (wr, wa)
        big = mo >= 1e-3 * mo.max()
        assert abs(float(np.mean((mg[big] - mo[big]) / mo[big]))) <= 1e-8


@pytest.mark.parametrize("name", ["small_2d", "discrimination"])
def test_bf16x3_nll_and_gradient(name):
    s = dataset(name)
    m = model(name)
    for th in [s.theta_true] + list(points(s, 2, seed=131)):
        f, g = m.nll_grad(th)
        if name == "small_2d":   # the oracle's dual-number gradient of the full model takes minutes
            fo, go = O.nll(s, th, grad=True)
            ok, worst = grad_ok(g[: s.P], go, th)
            assert ok, worst
        else:
            fo = O.nll(s, th)
        assert 2 * abs(f - fo) <= 1e-3, (f, fo)


def test_bf16x3_is_1d_rejected():
    with pytest.raises(bx.BxError) as e:
        bx.Model(dataset("small_mv"), precision=bx.BX_BF16X3)
    assert e.value.status == bx.BX_EINVAL
