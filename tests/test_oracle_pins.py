"""Pins of the FP64 CPU oracle to facts fixed by the paper's definitions and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an independent quadrature, an invariant, brute force on tiny inputs, or central
finite differences.  Passages: Eq. 1 (response convolution), Eq. 2 (pile-up), Eq. 3
(TFC joint likelihood), Eq. 4 (multivariate likelihood) of arXiv:1805.11125 Sec. 3.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate, signal, special

from oracle import oracle as O
from paper_1805_11125_gb300 import inputs as I

K_LY, K_A, K_B, K_C, K_KB, K_EPS, K_SR = range(7)


def tail(spec, name):
    return spec.K + I.PARAM_TAIL.index(name)


def with_theta(spec, **kw):
    th = spec.theta_true.copy()
    for k, v in kw.items():
        th[tail(spec, k)] = v
    return th


def gauss_bin_quad(lo, hi, mu, sig):
    f = lambda x: math.exp(-0.5 * ((x - mu) / sig) ** 2) / (sig * math.sqrt(2 * math.pi))
    pts = [p for p in (mu - sig, mu, mu + sig) if lo < p < hi]
    val, _ = integrate.quad(f, lo, hi, points=pts or None, epsabs=0, epsrel=1e-13, limit=200)
    return val


# ---------------------------------------------------------------------------------- a1

def test_a1_kb_zero_is_linear_light_yield():
    """kB = 0: the Birks integral is the deposited energy itself, Q_i = E_i = (i + 1/2) dE."""
    s = I.config("small_plain")
    th = with_theta(s, kB=0.0)
    Q, mu, sig, den = O.quench(s, th)
    E = (np.arange(s.n_grid) + 0.5) * s.e_max / s.n_grid
    np.testing.assert_allclose(Q, E, rtol=1e-13)
    np.testing.assert_allclose(mu, 500.0 * E, rtol=1e-13)
    a, b, c = 1.1, 2e-4, 4.0
    np.testing.assert_allclose(sig ** 2, a * mu + b * mu ** 2 + c, rtol=1e-13)
    np.testing.assert_allclose(den, special.ndtr(mu / sig), rtol=1e-13)


def test_a1_constant_stopping_power_closed_form():
    """Constant S: Q(E) = E / (1 + kB S) exactly."""
    s = dataclasses.replace(I.config("small_plain"), stop_pow=np.full(600, 2.7))
    kB = 0.011
    Q, mu, _, _ = O.quench(s, with_theta(s, kB=kB))
    E = (np.arange(s.n_grid) + 0.5) * s.e_max / s.n_grid
    np.testing.assert_allclose(Q, E / (1 + kB * 2.7), rtol=1e-13)


def test_a1_quenching_is_monotone_and_below_energy():
    s = I.config("plain")
    Q, _, _, _ = O.quench(s, s.theta_true)
    E = (np.arange(s.n_grid) + 0.5) * s.e_max / s.n_grid
    assert np.all(np.diff(Q) > 0) and np.all(Q < E)


# ------------------------------------------------------------------------------- a2/a3

def test_delta_spectrum_returns_response_column():
    """A delta-function spectrum s = e_i0 returns column i0 of the response, which is
    recomputed here by adaptive quadrature of the Gaussian density (no erfc)."""
    s0 = I.config("small_plain")
    for i0 in (37, 300, 555):
        shapes = np.zeros((1, s0.n_grid)); shapes[0, i0] = 1.0
        s = dataclasses.replace(s0, shapes=shapes, species=["delta"])
        s.theta_true = np.concatenate([[1.0], s0.theta_true[s0.K:]])
        th = with_theta(s, kB=0.0)
        _, v = O.response(s, th, want_R=False)
        E = (i0 + 0.5) * s.e_max / s.n_grid
        mu = 500.0 * E
        sig = math.sqrt(1.1 * mu + 2e-4 * mu * mu + 4.0)
        norm = gauss_bin_quad(0.0, mu + 60 * sig, mu, sig)
        col = np.array([gauss_bin_quad(m * s.width, (m + 1) * s.width, mu, sig) / norm
                        for m in range(s.m_hi)])
        big = col > 1e-12
        np.testing.assert_allclose(v[big, 0], col[big], rtol=1e-9)
        assert np.all(np.abs(v[~big, 0] - col[~big]) < 1e-14)


def test_gaussian_convolved_with_gaussian_closed_form():
    """kB = 0, a = b = 0, c = sr^2 and a Gaussian shape in E: the visible spectrum is the
    bin-integrated Gaussian of variance (LY sigma_E)^2 + sr^2 (Eq. 1 closed form)."""
    s0 = I.single_spectrum(n_grid=2000, width=4.0, lo_npe=200, hi_npe=800, n_species=1, L=10)
    E = (np.arange(2000) + 0.5) * 3.0 / 2000
    E0, sE, sr = 1.0, 0.05, 3.0
    shape = np.exp(-0.5 * ((E - E0) / sE) ** 2)
    s = dataclasses.replace(s0, shapes=(shape / shape.sum())[None, :])
    th = s0.theta_true.copy()
    th[tail(s, "kB")] = 0.0
    th[tail(s, "a")] = 0.0
    th[tail(s, "b")] = 0.0
    th[tail(s, "c")] = sr * sr
    _, v = O.response(s, th, want_R=False)
    sig = math.sqrt((500 * sE) ** 2 + sr ** 2)
    edges = np.arange(s.m_hi + 1) * s.width
    z = (edges - 500 * E0) / sig
    # upper-tail differences above the mean keep full relative precision
    want = np.where(z[:-1] >= 0, special.ndtr(-z[:-1]) - special.ndtr(-z[1:]),
                    special.ndtr(z[1:]) - special.ndtr(z[:-1]))
    big = want > 1e-10 * want.max()
    np.testing.assert_allclose(v[big, 0], want[big], rtol=1e-10)


def test_count_conservation_away_from_edges():
    """Each response column integrates to 1 over [0, inf); a spectrum far below the top of
    the axis keeps all its events."""
    s = I.config("small_plain")
    s = dataclasses.replace(s, m_hi=400, m_lo=40)  # axis up to 1600 npe
    _, v = O.response(s, s.theta_true, want_R=False)
    np.testing.assert_allclose(v.sum(axis=0), 1.0, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------------- a5

def _pile_spec(L=7, m_lo=0, m_hi=40, g=None):
    s = I.config("small_plain")
    g = np.full(L, 1.0 / L) if g is None else g
    return dataclasses.replace(s, pileup=np.asarray(g, float), m_lo=m_lo, m_hi=m_hi)


def test_pileup_eps_zero_is_identity():
    s = _pile_spec(m_lo=5, m_hi=40)
    x = np.random.default_rng(0).random(40)
    np.testing.assert_array_equal(O.pileup(s, 0.0, x), x[5:40])


@pytest.mark.parametrize("d", [0, 1, 6])
def test_pileup_delta_kernel_is_exact_shift(d):
    g = np.zeros(7); g[d] = 1.0
    s = _pile_spec(g=g, m_lo=3, m_hi=40)
    x = np.random.default_rng(1).random(40)
    eps = 0.25
    want = (1 - eps) * x + eps * np.concatenate([np.zeros(d), x[:40 - d]])
    np.testing.assert_allclose(O.pileup(s, eps, x), want[3:40], rtol=1e-15, atol=1e-16)


def test_pileup_conserves_total_and_matches_fft():
    g = np.random.default_rng(2).random(9); g /= g.sum()
    s = _pile_spec(g=g, L=9, m_lo=0, m_hi=60)
    x = np.zeros(60); x[:45] = np.random.default_rng(3).random(45)
    y = O.pileup(s, 1.0, x)
    assert abs(y.sum() - x.sum()) < 1e-13
    np.testing.assert_allclose(y, signal.fftconvolve(x, g)[:60], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------- a6

def test_poisson_nll_special_cases():
    assert O.poisson_nll([5.0, 7.0, 0.0], [5.0, 7.0, 0.0]) == 0.0
    assert O.poisson_nll([0.0, 0.0], [2.5, 0.5]) == pytest.approx(3.0, rel=1e-15)
    assert O.poisson_nll([1.0], [math.e]) == pytest.approx(math.e - 2.0, rel=1e-15)
    assert O.poisson_nll([3.0], [0.0]) == math.inf


def test_poisson_nll_brute_force_long_double():
    rng = np.random.default_rng(4)
    mu = 10 ** rng.uniform(-2, 6, size=2000)
    n = rng.poisson(mu).astype(float)
    nl, ml = n.astype(np.longdouble), mu.astype(np.longdouble)
    terms = np.where(nl > 0, ml - nl + nl * np.log(np.where(nl > 0, nl, 1) / ml), ml)
    want = float(np.sum(terms))
    assert O.poisson_nll(n, mu) == pytest.approx(want, rel=1e-13)


def test_baker_cousins_differs_by_data_constant():
    """-lnL differences between parameter points equal those of sum(mu - n ln mu)."""
    s = I.config("small_mv")
    mu0 = O.expected(s, s.theta_true)
    s = s.with_counts(I.poisson_counts(mu0, 11))
    n = s.counts_vector()
    th1 = s.theta_true * 1.01
    mu1 = O.expected(s, th1)
    plain = lambda mu: float(np.sum(mu.astype(np.longdouble) - n * np.log(mu.astype(np.longdouble))))
    d_or = O.nll(s, th1) - O.nll(s, s.theta_true)
    assert d_or == pytest.approx(plain(mu1) - plain(mu0), rel=1e-9, abs=1e-9)


# ------------------------------------------------------------------ radial term (Eq. 4)

def test_radial_probabilities_closed_form():
    s = I.config("small_mv")
    edges = np.linspace(0, s.r_fid, s.n_rad + 1)
    p_int, dp_int = O.radial(s, 1.0, I.RAD_INTERNAL)
    np.testing.assert_allclose(p_int, np.diff(edges ** 3) / s.r_fid ** 3, rtol=1e-13)
    assert np.all(dp_int == 0)
    for s_r in (0.6, 1.0, 1.7):
        lam = s.att_len * s_r
        F = lambda r: np.exp((r - s.r_iv) / lam) * (lam * r * r - 2 * lam ** 2 * r + 2 * lam ** 3)
        want = np.diff(F(edges)); want /= want.sum()
        p, dp = O.radial(s, s_r, I.RAD_EXTERNAL)
        np.testing.assert_allclose(p, want, rtol=1e-12)
        h = 1e-6 * s_r
        pp, _ = O.radial(s, s_r + h, 1)
        pm, _ = O.radial(s, s_r - h, 1)
        np.testing.assert_allclose(dp, (pp - pm) / (2 * h), rtol=1e-6, atol=1e-12)


# ------------------------------------------------------------- whole model, brute force

def _tiny_spec():
    rng = np.random.default_rng(5)
    shapes = rng.random((2, 5)); shapes /= shapes.sum(axis=1, keepdims=True)
    s = I.ModelSpec(name="tiny", n_grid=5, e_max=3.0, shapes=shapes, stop_pow=1.5 + rng.random(5),
                    pileup=np.array([0.7, 0.3]), width=300.0, m_lo=1, m_hi=4,
                    tag_frac=np.array([0.9, 0.1]), rad_class=np.array([0, 1], np.int32), n_rad=3,
                    psd_prob=np.array([[0.6, 0.4], [0.2, 0.8]]), species=["a", "b"])
    s.theta_true = np.array([3000.0, 1200.0, 480.0, 1.3, 3e-4, 6.0, 0.02, 0.1, 1.2])
    s.counts = {"sub": np.array([400.0, 900.0, 150.0]), "tag": np.array([90.0, 300.0, 0.0]),
                "rad": np.array([100.0, 500.0, 1900.0]), "psd": np.array([1500.0, 1000.0])}
    return s


def _tiny_brute_force(s, th):
    K, N, M = s.K, s.n_grid, s.m_hi
    r = th[:K]
    LY, a, b, c, kB, eps, s_r = th[K:]
    dE = s.e_max / N
    Q, run = [], 0.0
    for i in range(N):
        x = dE / (1 + kB * s.stop_pow[i])
        Q.append(run + 0.5 * x)
        run += x
    v = np.zeros((M, K))
    for i in range(N):
        mu = LY * Q[i]
        sig = math.sqrt(a * mu + b * mu * mu + c)
        norm = gauss_bin_quad(0.0, mu + 60 * sig, mu, sig)
        for m in range(M):
            R = gauss_bin_quad(m * s.width, (m + 1) * s.width, mu, sig) / norm
            for k in range(K):
                v[m, k] += R * s.shapes[k, i]
    def pile(x):
        out = []
        for m in range(s.m_lo, s.m_hi):
            conv = sum(s.pileup[d] * x[m - d] for d in range(min(m, s.L - 1) + 1))
            out.append((1 - eps) * x[m] + eps * conv)
        return np.array(out)
    sub = pile(v @ (r * (1 - s.tag_frac)))
    tag = pile(v @ (r * s.tag_frac))
    A = np.array([r[k] * (1 - s.tag_frac[k]) * pile(v[:, k]).sum() for k in range(K)])
    lam = s.att_len * s_r
    edges = np.linspace(0, s.r_fid, s.n_rad + 1)
    prad = []
    for k in range(K):
        f = (lambda x: x * x) if s.rad_class[k] == 0 else (lambda x: x * x * math.exp(-(s.r_iv - x) / lam))
        bins = np.array([integrate.quad(f, edges[j], edges[j + 1], epsrel=1e-14)[0] for j in range(s.n_rad)])
        prad.append(bins / bins.sum())
    rad = sum(A[k] * prad[k] for k in range(K))
    psd = A @ s.psd_prob
    mu = np.concatenate([sub, tag, rad, psd])
    n = s.counts_vector()
    tot = np.longdouble(0)
    for nj, mj in zip(n, mu):
        tot += np.longdouble(mj) if nj == 0 else np.longdouble(mj) - nj + nj * np.log(np.longdouble(nj) / np.longdouble(mj))
    return mu, float(tot)


def test_tiny_model_brute_force():
    """N = 5 grid points, 4 bins, 2 species with TFC, radial and pulse-shape terms, summed
    by hand-written loops with quadrature in place of erfc (Eq. 1-4)."""
    s = _tiny_spec()
    for th in (s.theta_true, s.theta_true * np.array([1.1, 0.9, 1.05, 0.8, 1.5, 0.9, 1.3, 0.5, 0.7])):
        mu_bf, nll_bf = _tiny_brute_force(s, th)
        np.testing.assert_allclose(O.expected(s, th), mu_bf, rtol=1e-10)
        assert O.nll(s, th) == pytest.approx(nll_bf, rel=1e-10)


# ------------------------------------------------------------------------ gradient (a7)

@pytest.mark.parametrize("name", ["small_plain", "small_mv"])
def test_dual_gradient_matches_central_differences(name):
    s = I.config(name)
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 3))
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=5)[0]
    f, g = O.nll(s, th, grad=True)
    gfd = np.zeros_like(g)
    for j in range(s.P):
        h = 1e-5 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h; tm[j] -= h
        gfd[j] = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
    scale = np.abs(g * th)
    np.testing.assert_allclose(g * th, gfd * th, rtol=2e-6, atol=2e-7 * scale.max())


def test_rate_gradient_is_linear_in_mu():
    """sum_k r_k dNLL/dr_k = sum_bins (mu - n): every expected count is homogeneous of
    degree one in the rates."""
    s = I.config("small_mv")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 4))
    th = s.theta_true * 1.03
    _, g = O.nll(s, th, grad=True)
    mu = O.expected(s, th)
    lhs = float(np.dot(th[:s.K], g[:s.K]))
    assert lhs == pytest.approx(float(np.sum(mu - s.counts_vector())), rel=1e-10)


# ----------------------------------------------------------------------------- fit (a8)

def test_fit_asimov_returns_truth():
    s = I.config("small_plain")
    s = s.with_counts(O.expected(s, s.theta_true))   # non-integer Asimov data
    th0 = I.parameter_points(s.theta_true, 1, rel=0.05, seed=6, free=s.default_free())[0]
    r = O.fit(s, th0, tol_edm=1e-16)
    assert r["status"] == 0
    assert r["nll"] < 1e-8
    np.testing.assert_allclose(r["theta"], s.theta_true, rtol=1e-5)


def test_fit_normalisation_invariant_at_optimum():
    """With free rates at an interior optimum, sum(mu) = sum(n) over all bins."""
    s = I.config("small_mv")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 8))
    r = O.fit(s, s.theta_true, tol_edm=1e-14)
    assert r["status"] == 0
    assert np.all(r["theta"][:s.K] > 0)
    mu = O.expected(s, r["theta"])
    assert mu.sum() == pytest.approx(s.counts_vector().sum(), rel=1e-9)


def test_fit_single_free_rate_has_the_closed_form_optimum():
    """One species (the other rates fixed at 0) with only its rate free: mu = r u in every bin
    (Eq. 2-4 are linear in the spectra), so d(-lnL)/dr = sum u - sum n / r and the maximum
    likelihood rate is sum(n) / sum(u), whatever the data.  The data here come from another
    response (LY 3 % higher) and another rate, with Poisson noise."""
    s = I.config("small_mv")
    j = 3
    th = s.theta_true.copy()
    th[: s.K] = 0.0
    th[j] = 1.0
    u = O.expected(s, th)
    gen = th.copy()
    gen[j] = 1.2e5
    gen[tail(s, "LY")] *= 1.03
    n = I.poisson_counts(O.expected(s, gen), 17)
    s = s.with_counts(n)
    free = np.zeros(s.P, dtype=np.uint8)
    free[j] = 1
    th0 = th.copy()
    th0[j] = 0.7e5
    r = O.fit(s, th0, free=free, tol_edm=1e-16)
    assert r["status"] == 0
    assert r["theta"][j] == pytest.approx(n.sum() / u.sum(), rel=1e-9)
    np.testing.assert_array_equal(np.delete(r["theta"], j), np.delete(th0, j))


# ------------------------------------------------------------- 2D histograms (discrimination)

def _split_2d(s, mu):
    nw = s.n_window
    o = {}
    off = 0
    for h, n in s.hist_sizes().items():
        o[h] = mu[off:off + n]
        off += n
    return o["sub"], o["r2d"].reshape(s.n_rad2d, nw), o["p2d"].reshape(s.n_psd2d, nw)


def test_2d_without_field_marginalises_to_the_vetoed_spectrum():
    """With amp = 0 the templates factorise, sum_b q_k[b] = 1 and N_k = 1: summed over its
    radial (or pulse-shape) slices the 2D histogram is the TFC-vetoed energy spectrum, bin by bin."""
    s = dataclasses.replace(I.config("small_2d"), field_amp=0.0)
    sub, r2, p2 = _split_2d(s, O.expected(s, s.theta_true))
    np.testing.assert_allclose(r2.sum(axis=0), sub, rtol=1e-12)
    np.testing.assert_allclose(p2.sum(axis=0), sub, rtol=1e-12)


def test_2d_without_field_marginalises_to_the_eq4_terms():
    """With amp = 0, summed over the energy window the 2D histograms are the Eq. 4 radial and
    pulse-shape terms of the same species (the already pinned 1D marginal model)."""
    s2 = dataclasses.replace(I.config("small_2d"), field_amp=0.0)
    _, r2, p2 = _split_2d(s2, O.expected(s2, s2.theta_true))
    s1 = dataclasses.replace(s2, n_rad2d=0, psd2d_prob=None, field2d=None, n_rad=s2.n_rad2d,
                             psd_prob=s2.psd2d_prob)
    mu1 = O.expected(s1, s2.theta_true)
    nw = s1.n_window
    rad, psd = mu1[2 * nw:2 * nw + s1.n_rad], mu1[2 * nw + s1.n_rad:]
    np.testing.assert_allclose(r2.sum(axis=1), rad, rtol=1e-9)
    np.testing.assert_allclose(p2.sum(axis=1), psd, rtol=1e-9)


def test_2d_field_is_non_separable_and_normalised():
    """The field makes the slices differ in energy shape (a true dense contraction), while
    each species keeps its total: the 2D spectra are linear in the rates."""
    s = I.config("small_2d")
    _, r2, _ = _split_2d(s, O.expected(s, s.theta_true))
    s0 = dataclasses.replace(s, field_amp=0.0)
    _, r20, _ = _split_2d(s0, O.expected(s0, s.theta_true))
    ratio = r2 / r20
    assert np.ptp(ratio[:, 100:200], axis=1).max() > 1e-3     # energy dependence differs per slice
    th2 = s.theta_true.copy()
    th2[:s.K] *= 1.7
    _, r2b, p2b = _split_2d(s, O.expected(s, th2))
    np.testing.assert_allclose(r2b, 1.7 * r2, rtol=1e-12)


def test_2d_dual_gradient_matches_central_differences():
    s = I.config("small_2d")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 13))
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=15)[0]
    f, g = O.nll(s, th, grad=True)
    gfd = np.zeros_like(g)
    for j in range(s.P):
        h = 1e-5 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h; tm[j] -= h
        gfd[j] = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
    scale = np.abs(g * th)
    np.testing.assert_allclose(g * th, gfd * th, rtol=2e-6, atol=2e-7 * scale.max())


# ------------------------------------------------- species-specific quenching (Eq. 1, next)

def _quench_spec(counts=True):
    s = I.config("small_quenched")
    if counts:
        s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 3))
    return s


def test_quench_of_one_is_the_base_model():
    """Multipliers of 1 for every species reproduce the model without species quenching bit
    for bit."""
    s = _quench_spec()
    base = dataclasses.replace(s, quench=None)
    ones = dataclasses.replace(s, quench=np.ones(s.K))
    np.testing.assert_array_equal(O.expected(ones, s.theta_true), O.expected(base, s.theta_true))


def test_common_quench_is_a_rescaled_birks_constant():
    """One multiplier q for every species is the base model with kB replaced by q kB."""
    s = _quench_spec()
    q = 3.5
    scaled = dataclasses.replace(s, quench=np.full(s.K, q))
    base = dataclasses.replace(s, quench=None)
    th = s.theta_true.copy()
    th2 = th.copy()
    th2[tail(s, "kB")] = th[tail(s, "kB")] * q
    np.testing.assert_allclose(O.expected(scaled, th), O.expected(base, th2), rtol=1e-13, atol=0)


def test_quench_sets_decompose_into_base_models():
    """Expected counts are linear in the rates, so a model with three quenching groups is the
    sum, over the groups, of the base model with kB scaled by the group's multiplier and only
    that group's rates kept (every bin: vetoed, tagged, radial, pulse shape)."""
    s = _quench_spec()
    base = dataclasses.replace(s, quench=None)
    th = s.theta_true.copy()
    total = np.zeros(s.n_bins_total)
    for q in np.unique(s.quench):
        t = th.copy()
        t[: s.K] = np.where(s.quench == q, th[: s.K], 0.0)
        t[tail(s, "kB")] = th[tail(s, "kB")] * q
        total += O.expected(base, t)
    np.testing.assert_allclose(O.expected(s, th), total, rtol=1e-12, atol=1e-12 * total.max())


def test_alpha_is_quenched_to_low_visible_energy():
    """The alpha peak at 2.3 MeV true energy, quenched with 150 kB, appears between 0.3 and
    0.7 MeV electron-equivalent (Birks' law with the electron stopping-power table): the
    vetoed spectrum of the alpha species alone peaks there."""
    s = _quench_spec(counts=False)
    th = s.theta_true.copy()
    ia = s.species.index("alpha")
    th[: s.K] = 0.0
    th[ia] = 1e5
    mu = O.expected(s, th)[: s.n_window]
    m_peak = s.m_lo + int(np.argmax(mu))
    e_vis = m_peak * s.width / th[tail(s, "LY")]
    assert 0.3 < e_vis < 0.7, e_vis


def test_quench_dual_gradient_matches_central_differences():
    s = _quench_spec()
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=9, free=s.default_free())[0]
    f, g = O.nll(s, th, grad=True)
    for j in [0, s.species.index("alpha"), s.species.index("ext0"), tail(s, "LY"), tail(s, "kB"), tail(s, "c")]:
        h = 1e-5 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
        assert abs(fd - g[j]) * abs(th[j]) <= 1e-6 * (1 + abs(g[j] * th[j])), (j, fd, g[j])


def test_quench_with_2d_slices_is_rejected():
    s = I.config("small_2d")
    s = dataclasses.replace(s, quench=np.where(np.arange(s.K) == 0, 2.0, 1.0))
    with pytest.raises(RuntimeError):
        O.expected(s, s.theta_true)


# ---- energy slices of Eq. 4's radial and pulse-shape terms

def _sliced_spec(counts=True):
    s = I.config("small_sliced")
    if counts:
        s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 5))
    return s


def _split(spec, mu):
    out, o = {}, 0
    for h, n in spec.hist_sizes().items():
        out[h] = mu[o:o + n]
        o += n
    return out


def test_one_energy_slice_is_the_base_model():
    """A single slice spanning the window reproduces the model without slices bit for bit."""
    s = _sliced_spec(counts=False)
    one = dataclasses.replace(s, eslices=np.array([0, s.n_window], dtype=np.int32))
    base = dataclasses.replace(s, eslices=None)
    np.testing.assert_array_equal(O.expected(one, s.theta_true), O.expected(base, s.theta_true))


def test_energy_slices_sum_to_the_window_marginals():
    """The slices partition the window, so the radial (pulse-shape) histograms of all slices
    add up to the single-slice histogram, bin by bin; the energy spectra are unchanged."""
    s = _sliced_spec(counts=False)
    base = dataclasses.replace(s, eslices=None)
    th = I.parameter_points(s.theta_true, 1, rel=0.03, seed=21, free=s.default_free())[0]
    sl, b = _split(s, O.expected(s, th)), _split(base, O.expected(base, th))
    S = s.n_eslices
    assert S == 3
    np.testing.assert_array_equal(sl["sub"], b["sub"])
    np.testing.assert_array_equal(sl["tag"], b["tag"])
    np.testing.assert_allclose(sl["rad"].reshape(S, s.n_rad).sum(axis=0), b["rad"], rtol=1e-12)
    np.testing.assert_allclose(sl["psd"].reshape(S, s.n_psd).sum(axis=0), b["psd"], rtol=1e-12)


def test_energy_slice_histograms_hold_the_vetoed_events_of_the_slice():
    """Radial and pulse-shape probabilities each sum to 1 per species, so each slice's radial
    and pulse-shape histograms both hold the TFC-vetoed events of that slice's window bins:
    the Eq. 4 marginals checked against the Eq. 3 spectrum after Eq. 2."""
    s = _sliced_spec(counts=False)
    th = I.parameter_points(s.theta_true, 1, rel=0.03, seed=22, free=s.default_free())[0]
    h = _split(s, O.expected(s, th))
    e = s.eslices
    for q in range(s.n_eslices):
        ev = h["sub"][e[q]:e[q + 1]].sum()
        np.testing.assert_allclose(h["rad"][q * s.n_rad:(q + 1) * s.n_rad].sum(), ev, rtol=1e-11)
        np.testing.assert_allclose(h["psd"][q * s.n_psd:(q + 1) * s.n_psd].sum(), ev, rtol=1e-11)


def test_energy_slice_dual_gradient_matches_central_differences():
    s = _sliced_spec()
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=23, free=s.default_free())[0]
    f, g = O.nll(s, th, grad=True)
    for j in [0, 3, s.K - 1, tail(s, "LY"), tail(s, "kB"), tail(s, "eps"), tail(s, "s_r")]:
        h = 1e-5 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
        assert abs(fd - g[j]) * abs(th[j]) <= 1e-6 * (1 + abs(g[j] * th[j])), (j, fd, g[j])


@pytest.mark.parametrize("edges", [[1, 60, 260], [0, 60, 259], [0, 60, 60, 260], [0, 140, 60, 260]])
def test_bad_energy_slice_edges_are_rejected(edges):
    s = _sliced_spec(counts=False)
    bad = dataclasses.replace(s, eslices=np.array(edges, dtype=np.int32))
    with pytest.raises(RuntimeError):
        O.expected(bad, s.theta_true)


def test_energy_slices_with_2d_slices_are_rejected():
    s = I.config("small_2d")
    s = dataclasses.replace(s, eslices=np.array([0, 50, s.n_window], dtype=np.int32))
    with pytest.raises(RuntimeError):
        O.expected(s, s.theta_true)


# ---- the joint energy x radius x pulse-shape grid

def _joint_pair(amp=0.0):
    """The small joint model and the separate 2D model with the same binning, both at amp."""
    j = dataclasses.replace(I.config("small_joint"), field_amp=amp)
    sep = dataclasses.replace(j, joint2d=False,
                              field2d=np.ascontiguousarray(I.smooth_field(j.n_grid, j.n_rad2d + j.n_psd2d, 0)))
    return j, sep


def test_joint_grid_marginals_are_the_separate_2d_slices():
    """With the field amplitude 0 the templates are separable, so the joint histogram summed over
    pulse shape is the energy x radius histogram of the separate 2D model, summed over radius its
    energy x pulse-shape histogram, and summed over both the TFC-vetoed spectrum (bin by bin)."""
    j, sep = _joint_pair()
    th = I.parameter_points(j.theta_true, 1, rel=0.03, seed=31, free=j.default_free())[0]
    hj, hs = _split(j, O.expected(j, th)), _split(sep, O.expected(sep, th))
    nR, nP, nw = j.n_rad2d, j.n_psd2d, j.n_window
    grid = hj["j2d"].reshape(nR, nP, nw)
    np.testing.assert_array_equal(hj["sub"], hs["sub"])
    np.testing.assert_array_equal(hj["tag"], hs["tag"])
    np.testing.assert_allclose(grid.sum(axis=1).ravel(), hs["r2d"], rtol=1e-11, atol=1e-12 * hs["r2d"].max())
    np.testing.assert_allclose(grid.sum(axis=0).ravel(), hs["p2d"], rtol=1e-11, atol=1e-12 * hs["p2d"].max())
    np.testing.assert_allclose(grid.sum(axis=(0, 1)), hj["sub"], rtol=1e-11, atol=1e-12 * hj["sub"].max())


def test_joint_grid_is_linear_in_the_rates():
    j, _ = _joint_pair(amp=0.05)
    th = j.theta_true.copy()
    a, b = th.copy(), th.copy()
    a[: j.K // 2] = 0.0
    b[j.K // 2: j.K] = 0.0
    np.testing.assert_allclose(O.expected(j, a) + O.expected(j, b), O.expected(j, th), rtol=1e-12,
                               atol=1e-12 * O.expected(j, th).max())


def test_joint_grid_dual_gradient_matches_central_differences():
    j, _ = _joint_pair(amp=0.05)
    j = j.with_counts(I.poisson_counts(O.expected(j, j.theta_true), 6))
    th = I.parameter_points(j.theta_true, 1, rel=0.02, seed=32, free=j.default_free())[0]
    f, g = O.nll(j, th, grad=True)
    for p in [0, j.K - 1, tail(j, "LY"), tail(j, "c"), tail(j, "kB"), tail(j, "eps"), tail(j, "s_r")]:
        h = 1e-5 * abs(th[p])
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.nll(j, tp) - O.nll(j, tm)) / (2 * h)
        assert abs(fd - g[p]) * abs(th[p]) <= 1e-6 * (1 + abs(g[p] * th[p])), (p, fd, g[p])


def test_joint_grid_needs_both_axes():
    j, _ = _joint_pair()
    bad = dataclasses.replace(j, psd2d_prob=None)   # no pulse-shape axis
    with pytest.raises(RuntimeError):
        O.expected(bad, j.theta_true)


# ---- template normalisation with the field on (Eq. 4 slice sets, count conservation)

def _conserving(spec, amp):
    """The spec on an axis wide enough for every species (window = whole axis from 0 npe, the
    top 600 npe above the highest visible energy) at field amplitude amp."""
    top = int(math.ceil((spec.e_max * 500.0 + 600.0) / spec.width))
    return dataclasses.replace(spec, field_amp=amp, m_lo=0, m_hi=top)


@pytest.mark.parametrize("amp", [0.05, 0.5])
def test_2d_slice_sets_conserve_each_species_with_the_field_on(amp):
    """With eps = 0 and an axis that holds every species' whole response (Eq. 1 columns of unit
    mass), the energy x radius histogram summed over energy and over its slices holds exactly the
    TFC-vetoed events r_k (1 - t_k) of species k, whatever the field does to the template's
    energy shape per slice; likewise the energy x pulse-shape histogram.  A normalisation N_k
    without the field factor (1 + amp u), or over the wrong slice set, breaks it by ~amp."""
    s = _conserving(I.config("small_2d"), amp)
    for k in range(s.K):
        th = s.theta_true.copy()
        th[: s.K] = 0.0
        th[k] = 1234.5
        th[tail(s, "eps")] = 0.0
        th[tail(s, "s_r")] = 1.3                      # the external radial shape off its default
        sub, r2, p2 = _split_2d(s, O.expected(s, th))
        want = th[k] * (1.0 - s.tag_frac[k])
        assert sub.sum() == pytest.approx(want, rel=1e-12)
        assert r2.sum() == pytest.approx(want, rel=1e-12)
        assert p2.sum() == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("amp", [0.05, 0.5])
def test_joint_grid_conserves_each_species_with_the_field_on(amp):
    """The joint grid holds the TFC-vetoed events r_k (1 - t_k) of each species once, summed over
    energy and every radius x pulse-shape cell (one normalisation over the whole grid)."""
    j, _ = _joint_pair(amp)
    j = _conserving(j, amp)
    nR, nP, nw = j.n_rad2d, j.n_psd2d, j.n_window
    for k in range(j.K):
        th = j.theta_true.copy()
        th[: j.K] = 0.0
        th[k] = 987.0
        th[tail(j, "eps")] = 0.0
        th[tail(j, "s_r")] = 0.8
        h = _split(j, O.expected(j, th))
        want = th[k] * (1.0 - j.tag_frac[k])
        grid = h["j2d"].reshape(nR, nP, nw)
        assert h["sub"].sum() == pytest.approx(want, rel=1e-12)
        assert grid.sum() == pytest.approx(want, rel=1e-12)


# ---- several energy estimators of one dataset (Sec. 3), fitted jointly

def _est_specs(base="small_mv", names=("npe", "charge", "nhits"), seed=40):
    sp = I.estimators(base, names)
    return [s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), seed + e)) for e, s in enumerate(sp)]


def test_one_estimator_is_the_single_model():
    """E = 1: the joint -lnL and gradient are the single model's, bit for bit."""
    s = _est_specs(names=("npe",))
    th = I.parameter_points(s[0].theta_true, 1, rel=0.02, seed=50, free=s[0].default_free())[0]
    f, g = O.nll_estimators(s, th, grad=True)
    f1, g1 = O.nll(s[0], th, grad=True)
    assert f == f1
    np.testing.assert_array_equal(g, g1)


def test_estimators_sum_their_own_models():
    """Each estimator enters at its own parameter vector [r, LY_e, a_e, b_e, c_e, kB, eps, s_r]:
    the joint -lnL is the sum of the single models evaluated there, and the joint gradient puts
    each estimator's LY, a, b, c derivatives in its own slots and sums the shared ones."""
    s = _est_specs()
    K = s[0].K
    th = I.estimator_theta(s) * (1.0 + 0.02 * np.random.default_rng(3).standard_normal(K + 7 + 8))
    th[K + 6] = 1.0
    f, g = O.nll_estimators(s, th, grad=True)
    parts = []
    for e, sp in enumerate(s):
        the = np.concatenate([th[:K], th[K:K + 4] if e == 0 else th[K + 7 + 4 * (e - 1):K + 7 + 4 * e], th[K + 4:K + 7]])
        np.testing.assert_array_equal(O.est_theta(K, e, th), the)
        parts.append(O.nll(sp, the, grad=True))
    assert f == pytest.approx(sum(p[0] for p in parts), rel=1e-15)
    np.testing.assert_allclose(g[:K], sum(p[1][:K] for p in parts), rtol=1e-13)
    np.testing.assert_allclose(g[K + 4:K + 7], sum(p[1][K + 4:K + 7] for p in parts), rtol=1e-13, atol=1e-12)
    for e in range(3):
        o = K if e == 0 else K + 7 + 4 * (e - 1)
        np.testing.assert_array_equal(g[o:o + 4], parts[e][1][K:K + 4])


def test_identical_estimators_double_the_likelihood():
    """Two copies of one estimator: twice its -lnL, twice its rate gradient, and each copy's own
    response-parameter gradient equal to the single model's."""
    one = _est_specs(base="small_plain", names=("npe",))   # no radial / pulse-shape term to count once
    two = [one[0], one[0]]
    K = one[0].K
    th1 = one[0].theta_true * 1.01
    th2 = np.concatenate([th1, th1[K:K + 4]])
    f1, g1 = O.nll(one[0], th1, grad=True)
    f2, g2 = O.nll_estimators(two, th2, grad=True)
    assert f2 == pytest.approx(2 * f1, rel=1e-15)
    np.testing.assert_allclose(g2[:K], 2 * g1[:K], rtol=1e-15)
    np.testing.assert_array_equal(g2[K:K + 4], g1[K:K + 4])
    np.testing.assert_array_equal(g2[K + 7:K + 11], g1[K:K + 4])


def test_estimators_dual_gradient_matches_central_differences():
    s = _est_specs()
    K = s[0].K
    th = I.estimator_theta(s)
    th = th * (1.0 + 0.02 * np.random.default_rng(4).standard_normal(th.shape[0]))
    th[K + 6] = 1.0
    f, g = O.nll_estimators(s, th, grad=True)
    for p in [0, K - 1, K, K + 3, K + 4, K + 5, K + 7, K + 10, K + 11, K + 14]:
        h = 1e-5 * abs(th[p])
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.nll_estimators(s, tp) - O.nll_estimators(s, tm)) / (2 * h)
        assert abs(fd - g[p]) * abs(th[p]) <= 1e-6 * (1 + abs(g[p] * th[p])), (p, fd, g[p])


def test_estimators_asimov_fit_returns_truth():
    """Asimov data in every estimator: the joint fit returns the joint true vector."""
    sp = I.estimators("small_mv", ("npe", "nhits"))
    sp = [s.with_counts(O.expected(s, s.theta_true)) for s in sp]
    th_true = I.estimator_theta(sp)
    free, _, _ = O.estimator_defaults(sp)
    th0 = I.parameter_points(th_true, 1, rel=0.01, seed=51, free=free)[0]
    r = O.fit_estimators(sp, th0, tol_edm=1e-14)
    assert r["status"] == 0
    m = free.astype(bool)
    np.testing.assert_allclose(r["theta"][m], th_true[m], rtol=2e-5)
    assert r["nll"] < 1e-8


# ---- a non-Gaussian response: the Gram-Charlier series (Eq. 1's response, the paper's outlook)

def _gc_density(x, mu, sig, g1, g2):
    z = (x - mu) / sig
    return math.exp(-0.5 * z * z) / (sig * math.sqrt(2 * math.pi)) * (
        1.0 + g1 / 6.0 * (z ** 3 - 3 * z) + g2 / 24.0 * (z ** 4 - 6 * z * z + 3))


def _gc_spec(g1=0.1, g2=0.1, width=0.5, n_grid=40):
    """A response-only model: a few grid points, fine bins on an axis that holds every column."""
    s = I.single_spectrum(n_grid=n_grid, width=width, lo_npe=0.0, hi_npe=1700.0, n_species=3, total=1e5, L=5)
    return dataclasses.replace(s, resp_skew=g1, resp_kurt=g2)


def test_gram_charlier_with_zero_moments_is_the_gaussian():
    s = I.config("small_nongauss")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 8))
    g = dataclasses.replace(s, resp_skew=0.0, resp_kurt=0.0)
    base = I.config("small_mv").with_counts(s.counts_vector())
    np.testing.assert_array_equal(O.expected(g, s.theta_true), O.expected(base, s.theta_true))


def test_gram_charlier_bin_mass_matches_quadrature_of_its_density():
    """R[m,i] against an independent adaptive quadrature of the density over the bin, over the
    mass above 0 npe (the closed-form CDF is what the oracle uses)."""
    s = _gc_spec(width=7.0)
    th = s.theta_true
    R, _ = O.response(s, th)
    _, mu, sig, _ = O.quench(s, th)
    for i in (3, 17, 31):
        N = integrate.quad(lambda x: _gc_density(x, mu[i], sig[i], 0.1, 0.1), 0.0, mu[i] + 40 * sig[i],
                           points=[mu[i]], epsabs=0, epsrel=1e-13, limit=400)[0]
        m0 = int(mu[i] // s.width)
        for m in range(max(0, m0 - 12), min(s.m_hi, m0 + 12)):
            q = integrate.quad(lambda x: _gc_density(x, mu[i], sig[i], 0.1, 0.1), m * s.width, (m + 1) * s.width,
                               epsabs=0, epsrel=1e-13)[0]
            assert R[m, i] == pytest.approx(q / N, rel=1e-10, abs=1e-16)


def test_gram_charlier_response_has_the_stated_moments():
    """On 0.5-npe bins (sigma ~ 10-35 npe) each response column's binned moments are those of the
    density: mean mu (the light-yield map's), variance sigma^2 (+ w^2/12 of the binning), skewness
    g1, excess kurtosis g2 (binning corrections of order (w / sigma)^2)."""
    g1, g2 = 0.1, 0.1
    s = _gc_spec(g1, g2)
    th = s.theta_true
    R, _ = O.response(s, th)
    _, mu, sig, _ = O.quench(s, th)
    c = (np.arange(s.m_hi) + 0.5) * s.width
    for i in (5, 20, 35):
        r = R[:, i]
        assert r.sum() == pytest.approx(1.0, abs=1e-12)
        m1 = (r * c).sum()
        d = c - m1
        v = (r * d * d).sum()
        assert m1 == pytest.approx(mu[i], rel=1e-9)
        assert v == pytest.approx(sig[i] ** 2 + s.width ** 2 / 12.0, rel=1e-7)
        assert (r * d ** 3).sum() / v ** 1.5 == pytest.approx(g1, abs=2e-4)
        assert (r * d ** 4).sum() / v ** 2 - 3.0 == pytest.approx(g2, abs=2e-3)


def test_gram_charlier_dual_gradient_matches_central_differences():
    s = I.config("small_nongauss")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 9))
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=52, free=s.default_free())[0]
    f, g = O.nll(s, th, grad=True)
    for p in [0, s.K - 1, tail(s, "LY"), tail(s, "a"), tail(s, "b"), tail(s, "c"), tail(s, "kB"), tail(s, "eps")]:
        h = 1e-5 * abs(th[p])
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
        assert abs(fd - g[p]) * abs(th[p]) <= 1e-6 * (1 + abs(g[p] * th[p])), (p, fd, g[p])


# ------------------------------------------------------- position-dependent response (shells)

def _shell_spec(counts=True):
    s = I.config("small_shelled")
    if counts:
        s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 21))
    return s


def test_shells_of_unit_light_yield_are_the_base_model():
    """Shells whose light-yield factors are all 1 and whose fractions sum to 1 for every species
    give every bin, -lnL and gradient of the model without shells (the shells' responses are
    then identical, so only the summation order differs)."""
    s = _shell_spec()
    base = dataclasses.replace(s, shell_ly=None, shell_frac=None)
    fr = np.tile([0.3, 0.7], (s.K, 1))
    flat = dataclasses.replace(s, shell_ly=np.ones(2), shell_frac=fr)
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=61, free=s.default_free())[0]
    mb = O.expected(base, th)
    np.testing.assert_allclose(O.expected(flat, th), mb, rtol=1e-13, atol=1e-15 * mb.max())
    fb, gb = O.nll(base, th, grad=True)
    ff, gf = O.nll(flat, th, grad=True)
    assert ff == pytest.approx(fb, rel=1e-13)
    np.testing.assert_allclose(gf, gb, rtol=1e-9, atol=1e-9 * np.abs(gb).max())


@pytest.mark.parametrize("base_name", ["small_nongauss", "small_sliced"])
def test_unit_shells_leave_the_other_variants_unchanged(base_name):
    """Unit-factor shells on the Gram-Charlier model and on the energy-sliced model reproduce
    those models (bins and -lnL): the shells compose with the other variants."""
    b = I.config(base_name)
    b = b.with_counts(I.poisson_counts(O.expected(b, b.theta_true), 22))
    flat = dataclasses.replace(b, shell_ly=np.ones(3), shell_frac=np.tile([0.2, 0.5, 0.3], (b.K, 1)))
    th = I.parameter_points(b.theta_true, 1, rel=0.02, seed=65, free=b.default_free())[0]
    mb = O.expected(b, th)
    np.testing.assert_allclose(O.expected(flat, th), mb, rtol=1e-13, atol=1e-15 * mb.max())
    assert O.nll(flat, th) == pytest.approx(O.nll(b, th), rel=1e-13)


def test_one_shell_is_a_rescaled_light_yield():
    """One shell of light-yield factor f holding every event is the base model with LY replaced by
    f LY: the same bins and -lnL, the same gradient in every parameter but LY, and f times the
    base model's LY derivative (mu = f LY Q)."""
    s = _shell_spec()
    f = 1.07
    one = dataclasses.replace(s, shell_ly=np.array([f]), shell_frac=np.ones((s.K, 1)))
    base = dataclasses.replace(s, shell_ly=None, shell_frac=None)
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=62, free=s.default_free())[0]
    th2 = th.copy()
    th2[tail(s, "LY")] *= f
    np.testing.assert_allclose(O.expected(one, th), O.expected(base, th2), rtol=1e-13, atol=0)
    f1, g1 = O.nll(one, th, grad=True)
    f2, g2 = O.nll(base, th2, grad=True)
    assert f1 == pytest.approx(f2, rel=1e-14)
    scale = np.ones(s.P)
    scale[tail(s, "LY")] = f
    np.testing.assert_allclose(g1, scale * g2, rtol=1e-12, atol=1e-12 * np.abs(g2).max())


def test_shells_decompose_into_base_models():
    """Expected counts are linear in the rates and in each species' spectrum, so a model with
    three shells and species-dependent fractions is the sum, over species k and shell rho, of
    q_k[rho] times the base model with LY scaled by the shell's factor and only r_k kept (every
    bin: vetoed, tagged, radial, pulse shape)."""
    s = _shell_spec(counts=False)
    rng = np.random.default_rng(63)
    ly = np.array([1.05, 1.0, 0.93])
    fr = rng.uniform(0.0, 1.0, (s.K, 3))
    fr[0] = [1.0, 0.0, 0.0]
    fr[1] = [0.0, 0.0, 2.0]
    shells = dataclasses.replace(s, shell_ly=ly, shell_frac=fr)
    base = dataclasses.replace(s, shell_ly=None, shell_frac=None)
    th = s.theta_true.copy()
    total = np.zeros(s.n_bins_total)
    for k in range(s.K):
        for r in range(3):
            if fr[k, r] == 0.0:
                continue
            t = th.copy()
            t[: s.K] = np.where(np.arange(s.K) == k, th[: s.K], 0.0)
            t[tail(s, "LY")] = th[tail(s, "LY")] * ly[r]
            total += fr[k, r] * O.expected(base, t)
    np.testing.assert_allclose(O.expected(shells, th), total, rtol=1e-12, atol=1e-12 * total.max())


def test_shells_dual_gradient_matches_central_differences():
    s = _shell_spec()
    th = I.parameter_points(s.theta_true, 1, rel=0.02, seed=64, free=s.default_free())[0]
    f, g = O.nll(s, th, grad=True)
    ext = int(np.nonzero(s.rad_class == I.RAD_EXTERNAL)[0][0])
    for p in [0, ext, tail(s, "LY"), tail(s, "a"), tail(s, "c"), tail(s, "kB"), tail(s, "eps")]:
        h = 1e-5 * abs(th[p])
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (O.nll(s, tp) - O.nll(s, tm)) / (2 * h)
        assert abs(fd - g[p]) * abs(th[p]) <= 1e-6 * (1 + abs(g[p] * th[p])), (p, fd, g[p])


@pytest.mark.parametrize("bad", ["ly0", "frac_neg", "quench", "2d"])
def test_bad_shells_are_rejected(bad):
    s = _shell_spec(counts=False)
    if bad == "ly0":
        s = dataclasses.replace(s, shell_ly=np.array([1.0, 0.0, 1.0, 1.0]))
    elif bad == "frac_neg":
        fr = s.shell_frac.copy()
        fr[2, 1] = -0.1
        s = dataclasses.replace(s, shell_frac=fr)
    elif bad == "quench":
        s = dataclasses.replace(s, quench=np.where(np.arange(s.K) == 0, 2.0, 1.0))
    else:
        d = I.config("small_2d")
        s = dataclasses.replace(d, shell_ly=np.ones(2), shell_frac=np.full((d.K, 2), 0.5))
    with pytest.raises(RuntimeError):
        O.expected(s, s.theta_true)
