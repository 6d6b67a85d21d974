"""The allocation-free forward stage (bx_spectra_noalloc) against the regular C-ABI path.

bx_spectra_noalloc serves callers that may not allocate device memory; it must give the
same spectra as the regular evaluation.  With the pile-up scale eps = 0 and a window that
covers the whole axis, the expected counts returned by bx_expected are exactly these
spectra, so the two are compared bin by bin, on two consecutive calls (the static scratch
keeps the previous call's contents; the second call must not be affected by them).
"""
import dataclasses

import numpy as np
import pytest

from paper_1805_11125_gb300 import bx, inputs as I

pytestmark = pytest.mark.gpu


def _spec(name):
    s = I.config(name)
    s = dataclasses.replace(s, m_lo=0)
    return s.with_counts(np.ones(s.n_bins_total))


@pytest.mark.parametrize("name", ["small_plain", "small_mv"])
def test_noalloc_spectra_match_regular_path(name):
    import torch
    s = _spec(name)
    model = bx.Model(s, precision=bx.BX_FP32)
    dev = torch.device("cuda")
    shapes = torch.tensor(s.shapes, dtype=torch.float64, device=dev)
    stop = torch.tensor(s.stop_pow, dtype=torch.float64, device=dev)
    tag = None if s.tag_frac is None else torch.tensor(s.tag_frac, dtype=torch.float64, device=dev)
    H = 1 if s.tag_frac is None else 2
    pts = I.parameter_points(s.theta_true, 2, rel=0.02, seed=31, free=s.default_free())
    for call in range(2):
        th = pts[call].copy()
        th[s.K + 5] = 0.0                       # eps = 0: expected counts are the spectra
        theta = torch.tensor(th, dtype=torch.float64, device=dev)
        lam = torch.full((H * s.m_hi,), float("nan"), dtype=torch.float64, device=dev)
        st = bx.lib().bx_spectra_noalloc(s.n_grid, s.e_max, s.K, shapes.data_ptr(), stop.data_ptr(),
                                          None if tag is None else tag.data_ptr(), s.width, s.m_hi,
                                          theta.data_ptr(), lam.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
        assert st == bx.BX_OK, bx.lib().bx_last_error()
        torch.cuda.synchronize()
        got = lam.cpu().numpy()
        want = model.expected(th)[: H * s.m_hi]
        big = want > 1e-3 * want.max()
        np.testing.assert_allclose(got[big], want[big], rtol=1e-5)
        assert np.all(np.abs(got[~big] - want[~big]) <= 1e-8 * want.max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    st = bx.lib().bx_spectra_noalloc(5000, 3.0, 4, 1, 1, None, 1.0, 100, 1, 1, None)
    assert st == bx.BX_EINVAL
    assert b"4096" in bx.lib().bx_last_error()
