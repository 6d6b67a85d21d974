"""The allocation-free forward stage (bx_spectra_noalloc) against the regular C-ABI path and
the oracle.

bx_spectra_noalloc serves callers that may not allocate device memory; it must give the
same spectra as the regular evaluation.  With the pile-up scale eps = 0 and a window that
covers the whole axis, the expected counts are exactly these spectra, so they are compared
bin by bin with bx_expected and with the FP64 oracle, on consecutive calls: the static
scratch keeps the previous call's contents, and a call must not be affected by them (a
call at the largest sizes the scratch holds is followed by a small one).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_1805_11125_gb300 import bx, inputs as I
from tests._util import per_bin_ok

pytestmark = pytest.mark.gpu

MAX_GRID = MAX_ROWS = 4096   # the fixed scratch's limits


def _spec(name):
    s = I.config(name)
    s = dataclasses.replace(s, m_lo=0)
    return s.with_counts(np.ones(s.n_bins_total))


def _largest():
    """n_grid = m_hi = 4096 (the scratch's limits), 15 species on a 0.4-npe axis to 1638 npe."""
    s = I.single_spectrum(n_grid=MAX_GRID, width=0.4, lo_npe=0.0, hi_npe=MAX_ROWS * 0.4, n_species=15,
                          total=1e6, L=50, name="noalloc_largest")
    assert s.m_lo == 0 and s.m_hi == MAX_ROWS
    return s.with_counts(np.ones(s.n_bins_total))


def _noalloc(s, th, torch):
    dev = torch.device("cuda")
    shapes = torch.tensor(s.shapes, dtype=torch.float64, device=dev)
    stop = torch.tensor(s.stop_pow, dtype=torch.float64, device=dev)
    tag = None if s.tag_frac is None else torch.tensor(s.tag_frac, dtype=torch.float64, device=dev)
    H = 1 if s.tag_frac is None else 2
    theta = torch.tensor(th, dtype=torch.float64, device=dev)
    lam = torch.full((H * s.m_hi,), 7.0, dtype=torch.float64, device=dev)   # stale contents
    st = bx.lib().bx_spectra_noalloc(s.n_grid, s.e_max, s.K, shapes.data_ptr(), stop.data_ptr(),
                                      None if tag is None else tag.data_ptr(), s.width, s.m_hi,
                                      theta.data_ptr(), lam.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == bx.BX_OK, bx.lib().bx_last_error()
    torch.cuda.synchronize()
    return lam.cpu().numpy()


def _point(s, seed):
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=seed, free=s.default_free())[0]
    th[s.K + 5] = 0.0                       # eps = 0: expected counts are the spectra
    return th


def _check_small(name, seed, torch):
    """Every bin against the regular path (the same FP32 kernels); against the oracle the bins
    of the configuration's own window (below it, at a few npe, the bins are wider than the
    resolution, outside the envelope of the FP32 generator's quadrature)."""
    s = _spec(name)
    lo = I.config(name).m_lo
    model = bx.Model(s, precision=bx.BX_FP32)
    H = 1 if s.tag_frac is None else 2
    th = _point(s, seed)
    got = _noalloc(s, th, torch)
    want = model.expected(th)[: H * s.m_hi]
    model.close()
    ok, wr, wa = per_bin_ok(got, want, rel=1e-5, abs_frac=1e-8)
    assert ok, (wr, wa)
    ref = O.expected(s, th)[: H * s.m_hi].reshape(H, s.m_hi)[:, lo:].ravel()
    ok, wr, wa = per_bin_ok(got.reshape(H, s.m_hi)[:, lo:].ravel(), ref, rel=1e-5, abs_frac=1e-8)
    assert ok, (wr, wa)


@pytest.mark.parametrize("name", ["small_plain", "small_mv"])
def test_noalloc_spectra_match_regular_path(name):
    import torch
    for call in range(2):
        _check_small(name, 31 + call, torch)


def test_noalloc_largest_sizes_then_a_small_call():
    """At n_grid = m_hi = 4096 (the scratch filled to its end) against the oracle, then a small
    call, which must not read what the large one left in the scratch."""
    import torch
    s = _largest()
    th = _point(s, 40)
    got = _noalloc(s, th, torch)
    ok, wr, wa = per_bin_ok(got, O.expected(s, th), rel=1e-5, abs_frac=1e-8)
    assert ok, (wr, wa)
    _check_small("small_mv", 41, torch)


def test_noalloc_domain_error_gives_nan():
    """sigma^2 = a mu + b mu^2 + c <= 0 (c far below zero): lambda is NaN, not the buffer's
    stale contents; the next valid call gives spectra again."""
    import torch
    s = _spec("small_plain")
    th = _point(s, 42)
    bad = th.copy()
    bad[s.K + 3] = -1e6
    assert np.all(np.isnan(_noalloc(s, bad, torch)))
    _check_small("small_plain", 43, torch)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = bx.lib()
    assert L.bx_spectra_noalloc(MAX_GRID + 1, 3.0, 4, 1, 1, None, 1.0, 100, 1, 1, None) == bx.BX_EINVAL
    assert b"4096" in L.bx_last_error()
    assert L.bx_spectra_noalloc(100, 3.0, 4, 1, 1, None, 1.0, MAX_ROWS + 1, 1, 1, None) == bx.BX_EINVAL
    assert b"4096" in L.bx_last_error()
    assert L.bx_spectra_noalloc(100, 3.0, 17, 1, 1, None, 1.0, 100, 1, 1, None) == bx.BX_EINVAL
