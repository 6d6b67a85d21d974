"""Seeded synthetic inputs for the Borexino-style binned likelihood (arXiv:1805.11125).

This module builds only the *inputs* of the likelihood: the true-energy species shapes
on the energy grid, the stopping-power table used by the Birks map, the random-trigger
(pile-up) spectrum, the pulse-shape templates, the histogram axes, the true parameter
vector and seeded parameter points.  It holds none of the likelihood's arithmetic: no
quenching, no detector response, no pile-up convolution, no likelihood.  Poisson data
are drawn by :func:`poisson_counts` from expected counts that the *caller* computes
with its own model evaluator (the CPU oracle in tests, the CUDA path in the benchmark).

The paper fixes no shapes, bin counts or species lists (Sec. 3 gives only Eq. 1-4);
the recipe below is the synthetic stand-in for the Borexino Phase-II spectra:

* grid: ``n_grid`` true-energy points ``E_i = (i + 1/2) * e_max / n_grid`` (0-3 MeV);
* species shapes (sampled at ``E_i`` and normalised to unit sum):
  - nu-e elastic-scattering recoil spectra of mono-energetic lines (Compton-edge-like),
  - allowed beta- spectra ``p W (Q - T)^2`` with seeded endpoints ``Q ~ U(0.5, 3)`` MeV,
  - one 11C-like beta+ spectrum (``Q = 0.96`` MeV shifted by the 1.022 MeV
    annihilation energy),
  - one alpha peak, a Gaussian at 0.4 MeV (sigma 0.02 MeV), already electron-equivalent,
  - external-gamma tails ``exp(-E / slope)``;
* stopping power ``S(E) = 1.9 (1 + (0.1 MeV / E)^0.95)`` MeV/cm on the grid;
* pile-up spectrum of ``L = 400`` bins, ``g[d] ~ exp(-d w / 30) + 0.1 exp(-(d w - 100)^2 / 800)``
  (``d w`` in photoelectrons), normalised to unit sum;
* pulse-shape templates: bin-integrated Gaussians N(0.35, 0.08) for beta-like and
  N(0.55, 0.08) for the beta+ species, renormalised to [0, 1);
* rates: log-uniform fractions ``10^U(-2, 0)`` scaled to the stated total number of events.

Parameter vector layout (``P = K + 7``):
``[r_0 .. r_{K-1}, LY, a, b, c, kB, eps, s_r]``.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np
from scipy.special import ndtr

MASTER_SEED = 1805
M_E = 0.51099895  # electron mass, MeV

PARAM_TAIL = ("LY", "a", "b", "c", "kB", "eps", "s_r")
N_TAIL = len(PARAM_TAIL)

# true values of the response / pile-up / radial parameters
TRUE_TAIL = dict(LY=500.0, a=1.1, b=2e-4, c=4.0, kB=0.011, eps=0.05, s_r=1.0)

RAD_INTERNAL = 0
RAD_EXTERNAL = 1


@dataclasses.dataclass
class ModelSpec:
    """One dataset and its model inputs (host arrays, float64)."""

    name: str
    n_grid: int
    e_max: float
    shapes: np.ndarray              # [K, n_grid], each row sums to 1
    stop_pow: np.ndarray            # [n_grid] MeV/cm
    pileup: np.ndarray              # [L], sums to 1
    width: float                    # npe per bin
    m_lo: int                       # energy window [m_lo, m_hi) on the full axis [0, m_hi)
    m_hi: int
    tag_frac: Optional[np.ndarray] = None   # [K]; None -> single (untagged) spectrum
    rad_class: Optional[np.ndarray] = None  # [K] int32 (0 internal, 1 external); None -> no radial term
    n_rad: int = 0
    r_fid: float = 3.0
    r_iv: float = 4.25
    att_len: float = 0.3
    psd_prob: Optional[np.ndarray] = None   # [K, n_psd]; None -> no PSD term
    # 2D histograms (energy x radius, energy x pulse shape): n_rad2d / n_psd2d slices of the
    # energy window each, templates s_k[i] q_k[b] (1 + field_amp u[i, b]) per slice set
    n_rad2d: int = 0                        # radial slices (uses rad_class, r_fid, r_iv, att_len)
    psd2d_prob: Optional[np.ndarray] = None  # [K, n_psd2d] pulse-shape bin probabilities
    field2d: Optional[np.ndarray] = None     # [n_grid, slices] smooth field u in [-1, 1]
    field_amp: float = 0.0
    # species-specific quenching: species k quenches with kB * quench[k] (None -> 1 for all)
    quench: Optional[np.ndarray] = None
    # energy slices of Eq. 4's radial and pulse-shape terms: slice s is the window bins
    # [eslices[s], eslices[s+1]), edges from 0 to n_window (None -> one slice, the window);
    # the radial and pulse-shape histograms are then one per slice, slice-major
    eslices: Optional[np.ndarray] = None
    # the 2D slices as the joint grid of radius and pulse shape: slice (rho, j) = rho n_psd2d + j
    # holds the energy window of the events in radial bin rho and pulse-shape bin j (the energy x
    # radius x pulse-shape histogram, one histogram "j2d" instead of "r2d" and "p2d")
    joint2d: bool = False
    # Gram-Charlier response: skewness and excess kurtosis of the photoelectron response
    # (0, 0: the Gaussian of Eq. 1)
    resp_skew: float = 0.0
    resp_kurt: float = 0.0
    # position-dependent response: the fiducial volume in radial shells, shell rho with the light
    # yield LY shell_ly[rho]; species k puts the fraction shell_frac[k, rho] of its events there
    # (None: one response for the whole volume)
    shell_ly: Optional[np.ndarray] = None
    shell_frac: Optional[np.ndarray] = None
    theta_true: Optional[np.ndarray] = None
    species: List[str] = dataclasses.field(default_factory=list)
    counts: Dict[str, np.ndarray] = dataclasses.field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.shapes.shape[0])

    @property
    def P(self) -> int:
        return self.K + N_TAIL

    @property
    def L(self) -> int:
        return int(self.pileup.shape[0])

    @property
    def n_window(self) -> int:
        return self.m_hi - self.m_lo

    @property
    def n_psd(self) -> int:
        return 0 if self.psd_prob is None else int(self.psd_prob.shape[1])

    @property
    def n_psd2d(self) -> int:
        return 0 if self.psd2d_prob is None else int(self.psd2d_prob.shape[1])

    @property
    def n_eslices(self) -> int:
        return 1 if self.eslices is None else len(self.eslices) - 1

    @property
    def n_slices2d(self) -> int:
        return self.n_rad2d * self.n_psd2d if self.joint2d else self.n_rad2d + self.n_psd2d

    def hist_sizes(self) -> Dict[str, int]:
        """Histogram names and bin counts, in the order every evaluator concatenates them."""
        out = {"sub": self.n_window}
        if self.tag_frac is not None:
            out["tag"] = self.n_window
        if self.rad_class is not None and self.n_rad > 0:
            out["rad"] = self.n_eslices * self.n_rad      # slice-major: [energy slice][radial bin]
        if self.psd_prob is not None:
            out["psd"] = self.n_eslices * self.n_psd      # slice-major: [energy slice][pulse-shape bin]
        if self.joint2d:
            out["j2d"] = self.n_slices2d * self.n_window  # slice-major: [rho][j][window bin]
            return out
        if self.n_rad2d > 0:
            out["r2d"] = self.n_rad2d * self.n_window    # slice-major: [rho][window bin]
        if self.n_psd2d > 0:
            out["p2d"] = self.n_psd2d * self.n_window    # slice-major: [j][window bin]
        return out

    @property
    def n_bins_total(self) -> int:
        return sum(self.hist_sizes().values())

    def param_names(self) -> List[str]:
        return [f"r_{s}" for s in self.species] + list(PARAM_TAIL)

    def default_free(self) -> np.ndarray:
        free = np.ones(self.P, dtype=np.uint8)
        if self.rad_class is None or (self.n_rad == 0 and self.n_rad2d == 0):
            free[self.K + PARAM_TAIL.index("s_r")] = 0
        return free

    def default_bounds(self):
        lo = np.full(self.P, -np.inf)
        hi = np.full(self.P, np.inf)
        lo[: self.K] = 0.0                         # rates
        t = {n: self.K + i for i, n in enumerate(PARAM_TAIL)}
        lo[t["LY"]] = 50.0
        lo[t["a"]] = 0.0
        lo[t["b"]] = 0.0
        lo[t["c"]] = 1e-3
        lo[t["kB"]] = 0.0
        lo[t["eps"]], hi[t["eps"]] = 0.0, 1.0
        lo[t["s_r"]] = 0.05
        return lo, hi

    def counts_vector(self) -> np.ndarray:
        return np.concatenate([self.counts[h] for h in self.hist_sizes()])

    def with_counts(self, flat: np.ndarray) -> "ModelSpec":
        """Copy of this spec with the flat data vector split back into histograms."""
        new = dataclasses.replace(self, counts={})
        o = 0
        for h, n in self.hist_sizes().items():
            new.counts[h] = np.ascontiguousarray(flat[o:o + n], dtype=np.float64)
            o += n
        assert o == flat.shape[0]
        return new


# ----------------------------------------------------------------------------------------
# shapes (input construction only)
# ----------------------------------------------------------------------------------------

def grid_energies(n_grid: int, e_max: float) -> np.ndarray:
    return (np.arange(n_grid) + 0.5) * (e_max / n_grid)


def nu_recoil(E: np.ndarray, e_nu: float) -> np.ndarray:
    """nu-e elastic-scattering recoil spectrum of a mono-energetic line (Compton-edge-like)."""
    gL, gR = 0.73, 0.23
    t_max = 2 * e_nu ** 2 / (M_E + 2 * e_nu)
    f = gL ** 2 + gR ** 2 * (1 - E / e_nu) ** 2 - gL * gR * M_E * E / e_nu ** 2
    return np.where(E <= t_max, np.maximum(f, 0.0), 0.0)


def beta_allowed(E: np.ndarray, q: float) -> np.ndarray:
    W = E + M_E
    p = np.sqrt(np.maximum(W * W - M_E * M_E, 0.0))
    return np.where(E < q, p * W * (q - E) ** 2, 0.0)


def beta_plus_11c(E: np.ndarray) -> np.ndarray:
    return beta_allowed(E - 2 * M_E, 0.96) * (E > 2 * M_E)


def alpha_peak(E: np.ndarray, mu=0.4, sig=0.02) -> np.ndarray:
    return np.exp(-0.5 * ((E - mu) / sig) ** 2)


def external_tail(E: np.ndarray, slope: float) -> np.ndarray:
    return np.exp(-E / slope)


def stopping_power(E: np.ndarray) -> np.ndarray:
    return 1.9 * (1.0 + (0.1 / E) ** 0.95)


def pileup_spectrum(L: int, width: float, scale: float = 1.0) -> np.ndarray:
    """Random-trigger spectrum in bins of ``width`` of an observable whose unit is ``scale``
    photoelectrons (1 for npe; the ratio of light yields for another energy estimator)."""
    x = np.arange(L) * width * scale
    g = np.exp(-x / 30.0) + 0.1 * np.exp(-((x - 100.0) ** 2) / (2 * 20.0 ** 2))
    return g / g.sum()


def smooth_field(n_grid: int, n_cols: int, seed: int = 0, n_modes: int = 4) -> np.ndarray:
    """Seeded smooth field u[i, b] in [-1, 1] on (true-energy point, slice): a sum of a few
    low-frequency products of cosines with random phases, scaled to max |u| = 1.  It makes
    the 2D templates non-separable in (energy, slice)."""
    rng = np.random.default_rng([MASTER_SEED, 21, seed])
    x = (np.arange(n_grid) + 0.5) / n_grid
    y = (np.arange(n_cols) + 0.5) / max(n_cols, 1)
    u = np.zeros((n_grid, n_cols))
    for _ in range(n_modes):
        fx, fy = rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0)
        px, py, a = rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi), rng.uniform(0.5, 1.0)
        u += a * np.cos(2 * np.pi * fx * x + px)[:, None] * np.cos(2 * np.pi * fy * y + py)[None, :]
    return u / np.abs(u).max()


def psd_template(n_psd: int, mean: float, sig: float = 0.08) -> np.ndarray:
    edges = np.linspace(0.0, 1.0, n_psd + 1)
    c = ndtr((edges - mean) / sig)
    p = np.diff(c)
    return p / p.sum()


def _normalise(rows: np.ndarray) -> np.ndarray:
    return rows / rows.sum(axis=1, keepdims=True)


def species_library(n_grid: int = 2000, e_max: float = 3.0, seed: int = 0):
    """The 15-shape library; its first 8 shapes are the 8-species single-spectrum set.

    Returns (names, shapes[15, n_grid], is_external[15], is_beta_plus[15]).
    """
    rng = np.random.default_rng([MASTER_SEED, 101, seed])
    E = grid_energies(n_grid, e_max)
    q = rng.uniform(0.5, 3.0, size=6)
    e_extra_line = rng.uniform(0.3, 1.5)
    rows, names = [], []
    for e_nu in (0.384, 0.862, 1.44):
        rows.append(nu_recoil(E, e_nu)); names.append(f"nu{e_nu:g}")
    for j in range(3):
        rows.append(beta_allowed(E, q[j])); names.append(f"beta{j}")
    rows.append(alpha_peak(E)); names.append("alpha")
    rows.append(external_tail(E, 0.5)); names.append("ext0")
    # the second half of the library
    rows.append(beta_plus_11c(E)); names.append("c11")
    for j in range(3, 6):
        rows.append(beta_allowed(E, q[j])); names.append(f"beta{j}")
    rows.append(nu_recoil(E, e_extra_line)); names.append("nu_x")
    rows.append(external_tail(E, 0.35)); names.append("ext1")
    rows.append(external_tail(E, 0.8)); names.append("ext2")
    shapes = _normalise(np.array(rows))
    is_ext = np.array([n.startswith("ext") for n in names])
    is_bp = np.array([n == "c11" for n in names])
    return names, shapes, is_ext, is_bp


def _rates(rng, K: int, total: float) -> np.ndarray:
    f = 10.0 ** rng.uniform(-2.0, 0.0, size=K)
    return total * f / f.sum()


def _theta(rates: np.ndarray) -> np.ndarray:
    return np.concatenate([rates, [TRUE_TAIL[n] for n in PARAM_TAIL]])


# ----------------------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------------------

def single_spectrum(n_grid=2000, e_max=3.0, width=2.0, lo_npe=150.0, hi_npe=950.0,
                    n_species=8, total=1e6, L=400, seed=0, name="single") -> ModelSpec:
    """K species, one energy spectrum (no TFC split, no radial or pulse-shape term)."""
    names, shapes, _, _ = species_library(n_grid, e_max, seed)
    rng = np.random.default_rng([MASTER_SEED, 1, seed])
    E = grid_energies(n_grid, e_max)
    m_lo, m_hi = int(round(lo_npe / width)), int(round(hi_npe / width))
    spec = ModelSpec(name=name, n_grid=n_grid, e_max=e_max,
                     shapes=np.ascontiguousarray(shapes[:n_species]),
                     stop_pow=stopping_power(E), pileup=pileup_spectrum(L, width),
                     width=width, m_lo=m_lo, m_hi=m_hi, species=names[:n_species])
    spec.theta_true = _theta(_rates(rng, n_species, total))
    return spec


def multivariate(n_grid=2000, e_max=3.0, width=1.0, lo_npe=100.0, hi_npe=1000.0,
                 n_species=15, total=2e6, L=400, n_rad=60, n_psd=50, tag_eff=0.9,
                 seed=0, name="multivariate") -> ModelSpec:
    """TFC-subtracted + TFC-tagged spectra, a radial and a pulse-shape histogram (Eq. 3, Eq. 4)."""
    names, shapes, is_ext, is_bp = species_library(n_grid, e_max, seed)
    rng = np.random.default_rng([MASTER_SEED, 2, seed])
    E = grid_energies(n_grid, e_max)
    K = n_species
    m_lo, m_hi = int(round(lo_npe / width)), int(round(hi_npe / width))
    tag = np.where(is_bp[:K], tag_eff, 0.1)
    psd = np.stack([psd_template(n_psd, 0.55 if bp else 0.35) for bp in is_bp[:K]])
    spec = ModelSpec(name=name, n_grid=n_grid, e_max=e_max,
                     shapes=np.ascontiguousarray(shapes[:K]), stop_pow=stopping_power(E),
                     pileup=pileup_spectrum(L, width), width=width, m_lo=m_lo, m_hi=m_hi,
                     tag_frac=tag.astype(np.float64),
                     rad_class=np.where(is_ext[:K], RAD_EXTERNAL, RAD_INTERNAL).astype(np.int32),
                     n_rad=n_rad, psd_prob=np.ascontiguousarray(psd), species=names[:K])
    spec.theta_true = _theta(_rates(rng, K, total))
    return spec


def quenched(alpha_true: float = 2.3, alpha_quench: float = 150.0, gamma_quench: Optional[float] = None,
             name: str = "quenched", **kw) -> ModelSpec:
    """The multivariate model with species-specific quenching: the alpha species is a peak at
    its true energy (alpha_true MeV, 30 keV wide) quenched with kB * alpha_quench, which puts it
    near 0.5 MeV electron-equivalent; with gamma_quench the external (gamma) species quench with
    kB * gamma_quench.  Every other species quenches with kB."""
    spec = multivariate(name=name, **kw)
    E = grid_energies(spec.n_grid, spec.e_max)
    names = list(spec.species)
    q = np.ones(spec.K)
    if "alpha" in names:
        ia = names.index("alpha")
        a = alpha_peak(E, mu=alpha_true, sig=0.03)
        a[a < 1e-12 * a.max()] = 0.0   # the peak's support: +-7.4 sigma
        spec.shapes[ia] = a / a.sum()
        q[ia] = alpha_quench
    if gamma_quench is not None:
        q[spec.rad_class == RAD_EXTERNAL] = gamma_quench
    spec.quench = q
    return spec


def shelled(ly=(1.03, 1.01, 0.99, 0.97), name: str = "shelled", **kw) -> ModelSpec:
    """The multivariate model with a position-dependent response: the fiducial sphere in
    len(ly) shells of equal volume, the light yield LY ly[rho] in shell rho (falling towards the
    vessel).  Internal species fill the shells in proportion to their volume (a fraction
    1/len(ly) each); external species follow the density exp(-(r_iv - r) / att_len) of the
    radial term at s_r = 1, integrated over each shell by the midpoint rule on 4000 points."""
    spec = multivariate(name=name, **kw)
    n = len(ly)
    edges = spec.r_fid * (np.arange(n + 1) / n) ** (1.0 / 3.0)
    r = (np.arange(4000) + 0.5) * (spec.r_fid / 4000)
    dens = r * r * np.exp(-(spec.r_iv - r) / spec.att_len)
    ext = np.array([dens[(r >= edges[j]) & (r < edges[j + 1])].sum() for j in range(n)])
    ext /= ext.sum()
    frac = np.where((spec.rad_class == RAD_EXTERNAL)[:, None], ext[None, :], 1.0 / n)
    spec.shell_ly = np.asarray(ly, dtype=np.float64)
    spec.shell_frac = np.ascontiguousarray(frac, dtype=np.float64)
    return spec


def sliced(edges_npe=(100.0, 250.0, 500.0, 1000.0), name: str = "sliced", **kw) -> ModelSpec:
    """The multivariate model with Eq. 4's radial and pulse-shape terms in several energy
    slices: one radial and one pulse-shape histogram of the TFC-vetoed events per slice of
    the window, the slices given by their npe edges (the first and last on the window's)."""
    spec = multivariate(name=name, **kw)
    e = np.array([int(round(x / spec.width)) - spec.m_lo for x in edges_npe], dtype=np.int32)
    if e[0] != 0 or e[-1] != spec.n_window or np.any(np.diff(e) <= 0):
        raise ValueError("energy slice edges must rise from the window's low to its high edge")
    spec.eslices = e
    return spec


def joint(n_rad=12, n_psd=10, name: str = "joint", **kw) -> ModelSpec:
    """The energy x radius x pulse-shape fit: the TFC-vetoed events binned jointly in energy (the
    window), radius (n_rad bins) and pulse shape (n_psd bins), next to the two TFC energy spectra;
    species templates s_k[i] p_k[rho] q_k[j] (1 + amp u[i, (rho, j)]), one slice per (rho, j)."""
    spec = discrimination(n_rad2d=n_rad, n_psd2d=n_psd, name=name, **kw)
    spec.joint2d = True
    spec.field2d = np.ascontiguousarray(smooth_field(spec.n_grid, n_rad * n_psd, kw.get("seed", 0)))
    return spec


def discrimination(n_grid=2000, e_max=3.0, width=1.0, lo_npe=100.0, hi_npe=1000.0,
                   n_species=15, total=2e6, L=400, n_rad2d=60, n_psd2d=50, tag_eff=0.9, amp=0.05,
                   seed=0, name="discrimination") -> ModelSpec:
    """TFC-subtracted + TFC-tagged energy spectra and the 2D energy x radius and energy x
    pulse-shape histograms of the TFC-subtracted events (the discrimination regime)."""
    names, shapes, is_ext, is_bp = species_library(n_grid, e_max, seed)
    rng = np.random.default_rng([MASTER_SEED, 3, seed])
    E = grid_energies(n_grid, e_max)
    K = n_species
    m_lo, m_hi = int(round(lo_npe / width)), int(round(hi_npe / width))
    tag = np.where(is_bp[:K], tag_eff, 0.1)
    psd = np.stack([psd_template(n_psd2d, 0.55 if bp else 0.35) for bp in is_bp[:K]])
    spec = ModelSpec(name=name, n_grid=n_grid, e_max=e_max,
                     shapes=np.ascontiguousarray(shapes[:K]), stop_pow=stopping_power(E),
                     pileup=pileup_spectrum(L, width), width=width, m_lo=m_lo, m_hi=m_hi,
                     tag_frac=tag.astype(np.float64),
                     rad_class=np.where(is_ext[:K], RAD_EXTERNAL, RAD_INTERNAL).astype(np.int32),
                     n_rad2d=n_rad2d, psd2d_prob=np.ascontiguousarray(psd),
                     field2d=np.ascontiguousarray(smooth_field(n_grid, n_rad2d + n_psd2d, seed)),
                     field_amp=amp, species=names[:K])
    spec.theta_true = _theta(_rates(rng, K, total))
    return spec


# Energy estimators (Sec. 3: the charge, the number of detected photons and the number of fired
# channels, each an observable with its own response of Eq. 1).  Synthetic stand-ins: each
# estimator's light yield in its own units per MeV, its resolution parameters, and its window
# (the npe window scaled by the ratio of light yields); 1-unit bins of the base configuration's
# width.  Estimator 0 is the base configuration itself.
ESTIMATORS = {
    "npe": dict(LY=500.0, a=1.1, b=2e-4, c=4.0),
    "charge": dict(LY=490.0, a=1.45, b=2e-4, c=6.0),
    "nhits": dict(LY=430.0, a=0.95, b=1.5e-4, c=3.0),
}
EST_TAIL = ("LY", "a", "b", "c")


def estimators(base: str = "multivariate", names=("npe", "charge", "nhits")) -> List[ModelSpec]:
    """One dataset seen by several energy estimators: the base configuration's species, stopping
    power, tag fractions and rates for every estimator; per estimator its own response parameters
    (``ESTIMATORS``), window (the base window scaled by LY_e / LY_0) and random-trigger spectrum (in
    its units).  The radial and pulse-shape terms stay with estimator 0.  Each spec's theta_true is
    the estimator's own vector [r, LY_e, a_e, b_e, c_e, kB, eps, s_r]; the joint vector is
    :func:`estimator_theta`."""
    b = config(base)
    out = []
    ly0 = ESTIMATORS[names[0]]["LY"]
    for e, n in enumerate(names):
        par = ESTIMATORS[n]
        f = par["LY"] / ly0
        m_lo, m_hi = int(round(b.m_lo * f)), int(round(b.m_hi * f))
        kw = dict(name=f"{base}:{n}", m_lo=m_lo, m_hi=m_hi, pileup=pileup_spectrum(b.L, b.width, 1.0 / f),
                  counts={})
        if e > 0:
            kw.update(rad_class=None, n_rad=0, psd_prob=None)
        spec = dataclasses.replace(b, **kw)
        th = b.theta_true.copy()
        for j, t in enumerate(EST_TAIL):
            th[b.K + j] = par[t]
        spec.theta_true = th
        out.append(spec)
    return out


def estimator_theta(specs: List[ModelSpec]) -> np.ndarray:
    """The joint parameter vector of the estimators' true values:
    [r_0 .. r_{K-1}, LY_0, a_0, b_0, c_0, kB, eps, s_r, LY_1, a_1, b_1, c_1, ...]."""
    K = specs[0].K
    parts = [specs[0].theta_true] + [s.theta_true[K:K + 4] for s in specs[1:]]
    return np.concatenate(parts)


def config(name: str) -> ModelSpec:
    """The named workloads.

    * ``plain``        K=8 single spectrum, 400 bins of 2 npe over 150-950 npe, 1e6 events.
    * ``multivariate`` K=15, TFC-subtracted/tagged 900 bins of 1 npe over 100-1000 npe,
                       60 radial bins, 50 pulse-shape bins, 22 parameters, 2e6 events.
    * ``discrimination`` K=15, TFC-subtracted/tagged 900 bins of 1 npe over 100-1000 npe and
                       the 2D energy x radius (900 x 60) and energy x pulse-shape (900 x 50)
                       histograms, 22 parameters, 2e6 events.
    * ``quenched`` the multivariate model with species-specific quenching (the alpha species
                  at its true energy, quenched with 150 kB); ``small_quenched`` its reduced
                  grid, with the external (gamma) species quenched with 1.3 kB as well.
    * ``sliced``   the multivariate model with the radial and pulse-shape terms in three
                  energy slices (100-250, 250-500, 500-1000 npe: Eq. 4's sums over radial
                  and pulse-shape terms); ``small_sliced`` its reduced grid.
    * ``joint``    the energy x radius x pulse-shape fit: the TFC-vetoed events in 12 radial x 10
                  pulse-shape bins of the 900-bin window (120 slices) next to the TFC spectra;
                  ``small_joint`` its reduced grid with 6 x 5 slices.
    * ``nongauss`` the multivariate model with a non-Gaussian (Gram-Charlier) response of
                  skewness 0.1 and excess kurtosis 0.1; ``small_nongauss`` its reduced grid.
    * ``shelled``  the multivariate model with a position-dependent response: four radial shells
                  of equal volume with light yields 1.03, 1.01, 0.99, 0.97 LY; ``small_shelled``
                  its reduced grid.
    * ``small_plain`` / ``small_mv`` / ``small_2d`` reduced grids that the oracle evaluates in
      well under a second (a few seconds for ``small_2d``) but that still span several
      128-row tiles and ragged tails.
    """
    if name == "plain":
        return single_spectrum(name=name)
    if name == "multivariate":
        return multivariate(name=name)
    if name == "small_plain":
        return single_spectrum(n_grid=600, width=4.0, lo_npe=160.0, hi_npe=1100.0,
                               n_species=5, total=2e5, L=100, name=name)
    if name == "discrimination":
        return discrimination(name=name)
    if name == "small_2d":
        return discrimination(n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9,
                              total=3e5, L=90, n_rad2d=12, n_psd2d=10, name=name)
    if name == "small_mv":
        return multivariate(n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9,
                            total=3e5, L=90, n_rad=20, n_psd=16, name=name)
    if name == "quenched":
        return quenched(name=name)
    if name == "sliced":
        return sliced(name=name)
    if name == "joint":
        return joint(name=name)
    if name == "small_joint":
        return joint(n_rad=6, n_psd=5, n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9,
                     total=3e5, L=90, name=name)
    if name == "small_sliced":
        return sliced(edges_npe=(120.0, 300.0, 540.0, 900.0), n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0,
                      n_species=9, total=3e5, L=90, n_rad=20, n_psd=16, name=name)
    if name == "nongauss":
        return dataclasses.replace(multivariate(name=name), resp_skew=0.1, resp_kurt=0.1)
    if name == "small_nongauss":
        return dataclasses.replace(multivariate(n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9,
                                                total=3e5, L=90, n_rad=20, n_psd=16, name=name),
                                   resp_skew=0.1, resp_kurt=0.1)
    if name == "shelled":
        return shelled(name=name)
    if name == "small_shelled":
        return shelled(n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=9, total=3e5, L=90,
                       n_rad=20, n_psd=16, name=name)
    if name == "small_quenched":
        return quenched(n_grid=520, width=3.0, lo_npe=120.0, hi_npe=900.0, n_species=12, total=3e5, L=90,
                        n_rad=20, n_psd=16, gamma_quench=1.3, name=name)
    raise KeyError(name)


def toy_batch(n_toys=4096, n_grid=2000, e_max=3.0, width=2.0, lo_npe=150.0, L=400,
              bins=(400, 1200), species=(6, 15), events=(1e4, 1e7), seed=0) -> List[ModelSpec]:
    """Pseudo-experiments of uneven size: bin count U{400..1200}, a random subset of 6-15
    shapes of the 15-shape library, and log-uniform event counts 1e4-1e7 (single spectrum,
    2 npe bins starting at 150 npe)."""
    names, shapes, _, _ = species_library(n_grid, e_max, seed)
    rng = np.random.default_rng([MASTER_SEED, 4, seed])
    E = grid_energies(n_grid, e_max)
    S = stopping_power(E)
    g = pileup_spectrum(L, width)
    m_lo = int(round(lo_npe / width))
    out = []
    for t in range(n_toys):
        nb = int(rng.integers(bins[0], bins[1] + 1))
        K = int(rng.integers(species[0], species[1] + 1))
        sub = np.sort(rng.choice(len(names), size=K, replace=False))
        total = 10.0 ** rng.uniform(np.log10(events[0]), np.log10(events[1]))
        spec = ModelSpec(name=f"toy{t}", n_grid=n_grid, e_max=e_max,
                         shapes=np.ascontiguousarray(shapes[sub]), stop_pow=S, pileup=g,
                         width=width, m_lo=m_lo, m_hi=m_lo + nb,
                         species=[names[j] for j in sub])
        spec.theta_true = _theta(_rates(rng, K, total))
        out.append(spec)
    return out


def parameter_points(theta: np.ndarray, n: int, rel: float = 0.02, seed: int = 0,
                     free: Optional[np.ndarray] = None) -> np.ndarray:
    """``n`` seeded points ``theta * (1 + rel * z)``, z ~ N(0, 1) per component (fixed
    components untouched)."""
    rng = np.random.default_rng([MASTER_SEED, 7, seed])
    z = rng.standard_normal((n, theta.shape[0]))
    if free is not None:
        z[:, free == 0] = 0.0
    return theta[None, :] * (1.0 + rel * z)


def poisson_counts(mu: np.ndarray, seed: int = 0) -> np.ndarray:
    """Poisson draws of expected counts ``mu`` (computed by the caller's model)."""
    rng = np.random.default_rng([MASTER_SEED, 9, seed])
    return rng.poisson(np.maximum(mu, 0.0)).astype(np.float64)
