"""The C-ABI library builds for sm_103a, loads, exports every entry point of include/bx.h,
and rejects invalid model descriptions on the host (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1805_11125_gb300 import bx, build, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "bx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bx_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_header_symbol():
    L = bx.lib()
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == {s[0] for s in bx.SIGNATURES}


def test_build_is_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_status_strings():
    L = bx.lib()
    assert L.bx_status_string(0) == b"ok"
    assert b"time" in L.bx_status_string(-5)


def _desc_for(spec):
    m = bx.Model.__new__(bx.Model)   # reuse the marshalling without creating
    return m


@pytest.mark.parametrize("mutate,msg", [
    (lambda s: setattr(s, "n_species_override", 0), "n_species"),
])
def test_invalid_description_rejected_on_host(mutate, msg):
    s = I.config("small_plain")
    s = s.with_counts(np.ones(s.n_bins_total))
    L = bx.lib()
    d = bx.bx_model_desc()
    shapes = np.ascontiguousarray(s.shapes)
    d.n_grid, d.e_max, d.n_species = s.n_grid, s.e_max, 0      # K = 0 is invalid
    d.shapes = shapes.ctypes.data
    h = C.c_void_p()
    st = L.bx_model_create(C.byref(d), 1, None, None, C.byref(h))
    assert st == bx.BX_EINVAL
    assert msg in L.bx_last_error().decode()


def test_negative_counts_and_bad_window_rejected():
    s = I.config("small_plain")
    L = bx.lib()
    keep = []

    def make(**over):
        d = bx.bx_model_desc()
        arrs = dict(shapes=np.ascontiguousarray(s.shapes), stop=np.ascontiguousarray(s.stop_pow),
                    g=np.ascontiguousarray(s.pileup), cnt=np.ones(s.n_window))
        arrs.update(over.pop("arrays", {}))
        keep.append(arrs)
        d.n_grid, d.e_max, d.n_species = s.n_grid, s.e_max, s.K
        d.shapes, d.stop_pow = arrs["shapes"].ctypes.data, arrs["stop"].ctypes.data
        d.n_pileup, d.pileup = s.L, arrs["g"].ctypes.data
        d.width, d.m_lo, d.m_hi = s.width, s.m_lo, s.m_hi
        d.counts_sub = arrs["cnt"].ctypes.data
        for k, v in over.items():
            setattr(d, k, v)
        return d

    h = C.c_void_p()
    bad = np.ones(s.n_window); bad[3] = -1.0
    for d, frag in [(make(arrays=dict(cnt=bad)), "counts_sub"), (make(m_lo=10, m_hi=5), "window"),
                    (make(width=0.0), "width"), (make(n_pileup=0), "n_pileup"),
                    (make(arrays=dict(stop=np.zeros(s.n_grid))), "stop_pow")]:
        st = L.bx_model_create(C.byref(d), 1, None, None, C.byref(h))
        assert st == bx.BX_EINVAL, frag
        assert frag in L.bx_last_error().decode()
    # NULL output pointer
    assert L.bx_model_create(C.byref(make()), 1, None, None, None) == bx.BX_EINVAL
    # bad options
    o = bx.bx_options(7, 1, 0.0, 0.0)
    assert L.bx_model_create(C.byref(make()), 1, C.byref(o), None, C.byref(h)) == bx.BX_EINVAL


def test_2d_model_rejections_on_host():
    """2D histograms: BX_FP32 only, at most 128 slices, not together with the 1D Eq. 4 terms
    (all checked before any device is touched)."""
    import dataclasses
    s = I.config("small_2d")
    s = s.with_counts(np.ones(s.n_bins_total))
    for prec in (bx.BX_FP64, bx.BX_TF32X3):
        with pytest.raises(bx.BxError) as e:
            bx.Model(s, precision=prec)
        assert e.value.status == bx.BX_EINVAL and "BX_FP32" in str(e.value)
    big = dataclasses.replace(s, n_rad2d=120, field2d=np.zeros((s.n_grid, 120 + s.n_psd2d)))   # 132 slices
    big = big.with_counts(np.ones(big.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(big, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL and "slices" in str(e.value)
    both = dataclasses.replace(s, n_rad=10)
    both = both.with_counts(np.ones(both.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(both, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL


def test_quenching_group_rejections_on_host():
    """Species-specific quenching: multipliers finite and >= 0, at most four groups, and more
    than one group only with BX_FP32 / BX_FP64 and without 2D histograms (all checked before
    any device is touched)."""
    import dataclasses
    s = I.config("small_quenched")
    s = s.with_counts(np.ones(s.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(s, precision=bx.BX_TF32X3)
    assert e.value.status == bx.BX_EINVAL and "quenching" in str(e.value)
    neg = dataclasses.replace(s, quench=np.where(np.arange(s.K) == 1, -1.0, 1.0))
    with pytest.raises(bx.BxError) as e:
        bx.Model(neg, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL and "quench" in str(e.value)
    five = dataclasses.replace(s, quench=1.0 + np.minimum(np.arange(s.K), 4).astype(float))
    with pytest.raises(bx.BxError) as e:
        bx.Model(five, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL and "groups" in str(e.value)
    s2 = I.config("small_2d")
    s2 = dataclasses.replace(s2, quench=np.where(np.arange(s2.K) == 0, 2.0, 1.0))
    s2 = s2.with_counts(np.ones(s2.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(s2, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL and "2D" in str(e.value)


def test_energy_slice_rejections_on_host():
    """Energy slices of the Eq. 4 terms: at most four, edges from 0 to the window's end and
    strictly rising, slices x bins within the marginal buffers, and more than one slice only
    with BX_FP32 / BX_FP64 and without 2D histograms (all checked before any device is
    touched)."""
    import dataclasses
    s = I.config("small_sliced")
    nw = s.n_window

    def make(edges, spec=s, prec=bx.BX_FP32):
        t = dataclasses.replace(spec, eslices=np.array(edges, dtype=np.int32))
        t = t.with_counts(np.ones(t.n_bins_total))
        return bx.Model(t, precision=prec)

    with pytest.raises(bx.BxError) as e:
        make(s.eslices, prec=bx.BX_TF32X3)
    assert e.value.status == bx.BX_EINVAL and "energy slices" in str(e.value)
    for edges in ([1, 60, nw], [0, 60, nw - 1], [0, 60, 60, nw], [0, 140, 60, nw]):
        with pytest.raises(bx.BxError) as e:
            make(edges)
        assert e.value.status == bx.BX_EINVAL and ("energy slices" in str(e.value) or "eslice_edges" in str(e.value))
    with pytest.raises(bx.BxError) as e:
        make([0, 40, 80, 120, 160, nw])
    assert e.value.status == bx.BX_EINVAL and "n_eslice" in str(e.value)
    wide = dataclasses.replace(s, n_rad=100, rad_class=s.rad_class)
    with pytest.raises(bx.BxError) as e:
        make([0, 60, 140, nw], spec=wide)
    assert e.value.status == bx.BX_EINVAL
    s2 = I.config("small_2d")
    with pytest.raises(bx.BxError) as e:
        make([0, 50, s2.n_window], spec=s2)
    assert e.value.status == bx.BX_EINVAL and "2D" in str(e.value)


def test_joint_grid_rejections_on_host():
    """The joint energy x radius x pulse-shape grid needs both axes and at most 128 slices with
    the TFC spectra (checked before any device is touched)."""
    import dataclasses
    s = I.config("small_joint")

    def make(spec):
        spec = spec.with_counts(np.ones(spec.n_bins_total))
        return bx.Model(spec, precision=bx.BX_FP32)

    nopsd = dataclasses.replace(s, psd2d_prob=None)
    with pytest.raises(bx.BxError) as e:
        make(nopsd)
    assert e.value.status == bx.BX_EINVAL and "joint grid" in str(e.value)
    wide = I.joint(n_rad=12, n_psd=11, n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9,
                   total=3e5, L=90, name="too_many_cells")
    with pytest.raises(bx.BxError) as e:
        make(wide)
    assert e.value.status == bx.BX_EINVAL and "exceed" in str(e.value)


def test_radial_shell_rejections_on_host():
    """The position-dependent response: at most four shells, light-yield factors > 0, fractions
    finite and >= 0, a single Birks multiplier, no 2D histograms, BX_FP32 / BX_FP64 only, one
    energy estimator (all checked before any device is touched)."""
    import dataclasses
    s = I.config("small_shelled")
    s = s.with_counts(np.ones(s.n_bins_total))
    bad = [
        (dataclasses.replace(s, shell_ly=np.ones(5), shell_frac=np.full((s.K, 5), 0.2)), bx.BX_FP32, "n_shell"),
        (dataclasses.replace(s, shell_ly=np.array([1.0, 0.0, 1.0, 1.0])), bx.BX_FP32, "shell_ly"),
        (dataclasses.replace(s, shell_frac=np.where(np.arange(4)[None, :] == 2, -0.1, 0.25) * np.ones((s.K, 1))),
         bx.BX_FP64, "shell_frac"),
        (dataclasses.replace(s, quench=np.where(np.arange(s.K) == 0, 2.0, 1.0)), bx.BX_FP32, "Birks"),
        (s, bx.BX_TF32X3, "shells"),
    ]
    for spec, prec, msg in bad:
        with pytest.raises(bx.BxError) as e:
            bx.Model(spec, precision=prec)
        assert e.value.status == bx.BX_EINVAL and msg in str(e.value), str(e.value)
    d = I.config("small_2d")
    d = dataclasses.replace(d, shell_ly=np.ones(2), shell_frac=np.full((d.K, 2), 0.5))
    d = d.with_counts(np.ones(d.n_bins_total))
    with pytest.raises(bx.BxError) as e:
        bx.Model(d, precision=bx.BX_FP32)
    assert e.value.status == bx.BX_EINVAL and "2D" in str(e.value)
    est = [dataclasses.replace(e_, shell_ly=np.ones(2), shell_frac=np.full((e_.K, 2), 0.5))
           for e_ in I.estimators("small_mv", names=("npe", "charge"))]
    est = [e_.with_counts(np.ones(e_.n_bins_total)) for e_ in est]
    with pytest.raises(bx.BxError) as e:
        bx.Model(est, precision=bx.BX_FP32, n_est=len(est))
    assert e.value.status == bx.BX_EINVAL and "shells" in str(e.value)
