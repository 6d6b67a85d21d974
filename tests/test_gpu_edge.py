"""Edge cases of the path through the C ABI: an empty batch, degenerate parameters (no pile-up,
no quenching, a resolution of the constant term only), a single species with a one-bin
pile-up spectrum, a model at the largest sizes the kernels take (16 species, an 8192-point
grid, 256 radial and 256 pulse-shape bins), and a model too large for the assembly stage's
shared memory, which creation rejects.  Parity against the FP64 oracle with the tolerances of
tests/test_gpu_parity.py."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import dataset, per_bin_ok, points

pytestmark = pytest.mark.gpu

PRECS = [bx.BX_FP64, bx.BX_FP32]
TOL = {bx.BX_FP64: dict(rel=1e-10, abs=1e-12, d2nll=1e-7, grad=1e-9),
       bx.BX_FP32: dict(rel=1e-5, abs=1e-8, d2nll=1e-3, grad=1e-3)}


def tail(spec, name):
    return spec.K + I.PARAM_TAIL.index(name)


def grad_ok(g, go, th, tol):
    lhs = np.abs(g - go) * np.abs(th)
    return np.all(lhs <= tol * (1.0 + np.abs(go * th))), float(np.max(lhs / (1.0 + np.abs(go * th))))


def check_point(m, s, th, prec, grad=True):
    mg, mo = m.expected(th), O.expected(s, th)
    ok, wr, wa = per_bin_ok(mg, mo, rel=TOL[prec]["rel"], abs_frac=TOL[prec]["abs"])
    assert ok, (wr, wa)
    if grad:
        f, g = m.nll_grad(th)
        fo, go = O.nll(s, th, grad=True)
        ok, worst = grad_ok(g[: s.P], go, th, TOL[prec]["grad"])
        assert ok, worst
    else:
        f, fo = m.nll(th), O.nll(s, th)
    assert 2 * abs(f - fo) <= TOL[prec]["d2nll"], (f, fo)


@pytest.mark.parametrize("prec", PRECS)
def test_empty_batch_is_a_no_op(prec):
    import torch
    s = dataset("small_mv")
    m = bx.Model(s, precision=prec, max_batch=4)
    f = m.nll_batch(np.zeros((0, m.P)))
    assert f.shape == (0,)
    f, g = m.nll_batch(np.zeros((0, m.P)), grad=True)
    assert f.shape == (0,) and g.shape == (0, m.P)
    fd = m.nll_batch(torch.zeros((0, m.P), dtype=torch.float64, device="cuda"))
    assert fd.shape == (0,)
    # the model still evaluates afterwards
    th = s.theta_true
    assert np.isfinite(m.nll(th))
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_degenerate_parameters(prec):
    """eps = 0 (no pile-up), kB = 0 (no quenching: mu = LY E) and a = b = 0 (the resolution's
    constant term alone), each alone and all together.  The FP64 mode takes sigma = sqrt(c) =
    2 npe, narrower than the 3-npe bins; the FP32 mode's 3-point Gauss-Legendre bin mass has a
    relative error of about 5e-7 (z w / sigma)^6, so it is held to the per-bin criterion with
    sigma = 12 npe (c = 144), inside that envelope."""
    s = dataset("small_mv")
    m = bx.Model(s, precision=prec)
    base = points(s, 1, seed=91)[0]
    flat = {"a": 0.0, "b": 0.0} if prec == bx.BX_FP64 else {"a": 0.0, "b": 0.0, "c": 144.0}
    cases = [{"eps": 0.0}, {"kB": 0.0}, flat, {"eps": 0.0, "kB": 0.0, **flat}]
    for c in cases:
        th = base.copy()
        for k, v in c.items():
            th[tail(s, k)] = v
        check_point(m, s, th, prec)
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_single_species_one_bin_pileup(prec):
    """K = 1 (a beta spectrum, its bulk inside the window) and a one-bin pile-up spectrum
    g = [1] (Eq. 2 is then the identity for any eps)."""
    s = I.config("small_plain")
    k = s.species.index("beta0")
    s = dataclasses.replace(s, shapes=np.ascontiguousarray(s.shapes[k:k + 1]), pileup=np.array([1.0]),
                            species=[s.species[k]])
    th0 = np.concatenate([[2e5], s.theta_true[-I.N_TAIL:]])
    s.theta_true = th0
    s = s.with_counts(I.poisson_counts(O.expected(s, th0), 2))
    m = bx.Model(s, precision=prec)
    for th in [th0] + list(points(s, 1, seed=92)):
        check_point(m, s, th, prec)
    # eps has no effect with g = [1]
    t2 = th0.copy()
    t2[tail(s, "eps")] = 0.5
    np.testing.assert_allclose(m.expected(t2), m.expected(th0), rtol=1e-14 if prec == bx.BX_FP64 else 1e-6)
    m.close()


def _max_spec():
    """16 species (the 15 of the library and one more peak) on an 8192-point grid, a 2048-bin
    axis of 0.75 npe with an 1800-bin window, a 1024-bin pile-up spectrum, 256 radial and 256
    pulse-shape bins."""
    s = I.multivariate(n_grid=8192, width=0.75, lo_npe=186.0, hi_npe=1536.0, L=1024, n_rad=256, n_psd=256,
                       name="max_sizes")
    E = I.grid_energies(s.n_grid, s.e_max)
    extra = I.alpha_peak(E, mu=1.2, sig=0.05)
    extra = extra / extra.sum()
    s = dataclasses.replace(
        s, shapes=np.ascontiguousarray(np.vstack([s.shapes, extra])),
        tag_frac=np.append(s.tag_frac, 0.1), rad_class=np.append(s.rad_class, I.RAD_INTERNAL).astype(np.int32),
        psd_prob=np.ascontiguousarray(np.vstack([s.psd_prob, I.psd_template(s.n_psd, 0.35)])),
        species=list(s.species) + ["peak1.2"])
    s.theta_true = np.concatenate([s.theta_true[: s.K - 1], [5e4], s.theta_true[s.K - 1:]])
    assert s.K == 16 and s.P == 23 and s.m_hi == 2048 and s.n_window == 1800
    return s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 3))


@pytest.mark.parametrize("prec", PRECS)
def test_maximum_sizes(prec):
    s = _max_spec()
    m = bx.Model(s, precision=prec, max_batch=2)
    th = points(s, 1, seed=93)[0]
    check_point(m, s, th, prec)
    f, g = m.nll_batch(np.stack([s.theta_true, th]), grad=True)
    f1, g1 = m.nll_grad(th)
    assert f[1] == f1
    np.testing.assert_array_equal(g[1], g1)
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_model_beyond_the_assembly_shared_memory_is_rejected(prec):
    """An 8192-point grid with a 4096-bin axis: one item's assembly stage would need more than
    the 227 KB of shared memory a thread block may have; creation says so instead of failing
    at the first launch."""
    s = I.multivariate(n_grid=8192, width=0.375, lo_npe=186.0, hi_npe=1536.0, L=1024, name="too_large")
    assert s.m_hi == 4096
    s = s.with_counts(np.ones(s.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(s, precision=prec)
    assert e.value.status == bx.BX_EINVAL and "shared memory" in str(e.value)
