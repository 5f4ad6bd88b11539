"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only builds the
problem description (grid, gas density, sources, spectrum tables, run length,
option values) that both the CUDA path and the CPU oracle take as input.  It
imports neither of them.

Configurations (sizes, distributions and recipes):

* ``stromgren``      -- isothermal Stromgren sphere in the style of the
  paper's Test 1 (Sec. 5.1): uniform n_H = 1e-3 cm^-3, T = 1e4 K, one
  13.6 eV source of 3e48 photons/s, 32^3 cells in a 12 kpc box, 30 x 1 Myr.
* ``cosmo16``        -- 16 sources in a 128^3 lognormal field, 0.5 Mpc/h box
  at z = 9, 4-bin 1e5 K blackbody, temperature evolution (the shape of the
  paper's Test 4, Sec. 5.4, with a synthetic density field), 100 x 0.1 Myr.
* ``cosmo20k``       -- 2e4 sources in a 200^3 lognormal field, 200 Mpc/h at
  z = 7, 3 bins, sub-grid mean free path law (the shape of Sec. 7.2's run,
  synthetic), 200 x 1 Myr.
* ``batch64``        -- 64 independent uneven simulations (grids 32..96^3).
* ``serve``          -- a Poisson request stream of such simulations.

The paper's own inputs (the CRTCP density and halo files, the hydro and
N-body fields behind Sec. 7.2) are not available; these seeded fields stand
in for them.
"""
from __future__ import annotations

import dataclasses as dc
import math

import numpy as np

# physical constants and units (cgs)
EV = 1.602176634e-12
KPC = 3.0856775814913673e21
MPC = 1000.0 * KPC
MYR = 3.15576e13
# cosmology of the paper (Sec. 1): Omega_m = 0.305, Omega_b = 0.048, h = 0.68
H_LITTLE = 0.68
OMEGA_B = 0.048
X_H = 0.76
M_P = 1.67262192e-24
RHO_CRIT_H2 = 1.87847e-29  # g cm^-3 h^-2


def mean_nH_comoving() -> float:
    """Mean hydrogen number density today (comoving), cm^-3."""
    return X_H * OMEGA_B * RHO_CRIT_H2 * H_LITTLE ** 2 / M_P


@dc.dataclass
class Spectrum:
    nbins: int
    frac: np.ndarray        # photon fraction per bin (sums to 1)
    sigma_cm2: np.ndarray   # photon-weighted HI cross-section per bin
    eheat_erg: np.ndarray   # mean excess energy per photo-ionisation per bin


@dc.dataclass
class Mfp:
    mode: int = 0                       # 0 none, 1 constant lambda, 2 power law in ionised cells,
                                        # 3 photo-ionisation equilibrium (Generalized mode only)
    lambda0_cm_comoving: float = 0.0
    delta_exp: float = 1.0
    gamma_ref: float = 1e-12
    gamma_exp: float = 2.0 / 3.0
    gamma_floor: float = 1e-15
    xion_threshold: float = 0.5
    nH_mean: float = 0.0                # density defining Delta; 0 = mean of the grid


@dc.dataclass
class Options:
    l_src: int = 0
    l_max: int = 12
    n_ray_min: float = 3.0
    eps_term: float = 1e-10
    seed: int = 1
    rotate: bool = True
    isothermal: bool = True
    rates: int = 0                      # 0: constant alpha_B, no collisional ionisation; 1: Hui & Gnedin fits
    chem_iters: int = 5
    alpha_B_const: float = 2.59e-13
    x_init: float = 1.2e-3
    T_init: float = 1.0e4
    merge: bool = False                 # ray merging at the end of each step
    l_merge: int = 0                    # HEALPix level of the merge sphere
    n_ex: float = 16.0                  # rays exempt from merging per RT cell
    gamma_iters: int = 1                # passes of the Gamma - <n_HI> (and lambda - Gamma) iteration
    gen_mode: bool = False              # Generalized Opacity mode (moving-screen I-fronts)
    chi: float = 0.0                    # He/H number ratio (singly ionised helium, Eq. 18)
    t_reion: float = 2.0e4              # Generalized mode, not isothermal: T of newly ionised gas (K)
    alpha_pl: float = 1.5               # Generalized mode: spectral index of the Eq. 22 photo-heating


@dc.dataclass
class Problem:
    name: str
    grid: tuple
    box_cm_comoving: float
    redshift: float
    nH: np.ndarray                      # physical cm^-3, flat, x fastest
    spectrum: Spectrum
    mfp: Mfp
    options: Options
    source_cells: np.ndarray            # int32 [n,3] (i, j, k)
    source_ndot: np.ndarray             # photons / s
    dt: float
    nsteps: int

    @property
    def dx_phys_cm(self) -> float:
        return self.box_cm_comoving / self.grid[0] / (1.0 + self.redshift)

    @property
    def ncell(self) -> int:
        return int(self.grid[0] * self.grid[1] * self.grid[2])


# --------------------------------------------------------------------------
# spectra
# --------------------------------------------------------------------------
def sigma_HI(E_eV, sigma0=6.3e-18, beta=2.75):
    """Power-law HI cross-section sigma0 (E/13.6 eV)^-beta; beta = 2.75 is the
    paper's own scaling (Sec. 4.2)."""
    return sigma0 * (np.asarray(E_eV) / 13.6) ** (-beta)


def _simpson(f, a, b, n=4096):
    x = np.linspace(a, b, n + 1)
    y = f(x)
    h = (b - a) / n
    return h / 3.0 * (y[0] + y[-1] + 4.0 * y[1:-1:2].sum() + 2.0 * y[2:-1:2].sum())


def blackbody_bins(T_bb: float, edges_eV, sigma0=6.3e-18, beta=2.75) -> Spectrum:
    """Bin a blackbody photon spectrum n(E) ~ E^2/(exp(E/kT)-1) (composite
    Simpson, 4096 panels per bin): photon fraction, photon-weighted sigma and
    the (sigma x photon)-weighted mean excess energy E - 13.6 eV per bin."""
    kT = 8.617333262e-5 * T_bb
    n = lambda E: E * E / np.expm1(E / kT)
    edges = np.asarray(edges_eV, float)
    tot = _simpson(n, edges[0], edges[-1], 4096 * (len(edges) - 1))
    frac, sig, eh = [], [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        nb = _simpson(n, lo, hi)
        sn = _simpson(lambda E: sigma_HI(E, sigma0, beta) * n(E), lo, hi)
        sne = _simpson(lambda E: sigma_HI(E, sigma0, beta) * n(E) * (E - 13.6), lo, hi)
        frac.append(nb / tot)
        sig.append(sn / nb)
        eh.append(sne / sn * EV)
    frac = np.array(frac)
    frac /= frac.sum()
    return Spectrum(len(frac), frac, np.array(sig), np.array(eh))


def monochromatic(E_eV=13.6, sigma=6.3e-18) -> Spectrum:
    return Spectrum(1, np.array([1.0]), np.array([sigma]), np.array([(E_eV - 13.6) * EV]))


# --------------------------------------------------------------------------
# density fields and sources
# --------------------------------------------------------------------------
def lognormal_delta(n: int, sigma_ln: float, seed: int, slope: float = -2.0) -> np.ndarray:
    """Delta = exp(g - sigma^2/2) with g a Gaussian random field of power
    spectrum P(k) ~ k^slope (P(0) = 0), normalised to mean 0 and std sigma_ln.
    Returned flat with x fastest (index = (k*n + j)*n + i)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    kx = np.fft.fftfreq(n)
    kz = np.fft.rfftfreq(n)
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P) = k^(slope/2)
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std() * sigma_ln
    return np.exp(g - 0.5 * sigma_ln ** 2).reshape(-1)


def cell_ijk(lin, n):
    lin = np.asarray(lin, np.int64)
    return np.stack([lin % n, (lin // n) % n, lin // (n * n)], axis=1).astype(np.int32)


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------
def stromgren(n: int = 32, nsteps: int = 30, seed: int = 1) -> Problem:
    """Isothermal Stromgren sphere (Sec. 5.1 style)."""
    box = 12.0 * KPC * (n / 32.0)
    nH = np.full(n ** 3, 1e-3)
    c = n // 2
    opts = Options(l_src=0, n_ray_min=3.0, seed=seed, isothermal=True, rates=0,
                   alpha_B_const=2.59e-13, x_init=1.2e-3, T_init=1e4)
    return Problem("stromgren", (n, n, n), box, 0.0, nH, monochromatic(), Mfp(), opts,
                   np.array([[c, c, c]], np.int32), np.array([3e48]), 1.0 * MYR, nsteps)


def cosmo16(n: int = 128, nsteps: int = 100, nsrc: int = 16, seed: int = 2) -> Problem:
    """16 brightest-density sources in a lognormal field, T evolution on."""
    z = 9.0
    delta = lognormal_delta(n, 1.0, seed)
    nH = mean_nH_comoving() * (1 + z) ** 3 * delta
    order = np.argsort(-delta, kind="stable")[:nsrc]
    rng = np.random.default_rng(seed + 1000)
    ndot = 10.0 ** rng.uniform(51.0, 52.0, nsrc)
    edges = 13.6 * 2.0 ** (np.arange(5) / 2.0)       # 13.6 .. 54.4 eV, 4 bins
    opts = Options(l_src=0, n_ray_min=3.0, seed=seed, isothermal=False, rates=1,
                   x_init=1.2e-3, T_init=100.0)
    box = 0.5 * MPC / H_LITTLE * (n / 128.0)
    return Problem("cosmo16", (n, n, n), box, z, nH, blackbody_bins(1e5, edges), Mfp(), opts,
                   cell_ijk(order, n), ndot, 0.1 * MYR, nsteps)


def cosmo20k(n: int = 200, nsteps: int = 200, nsrc: int = 20000, seed: int = 3) -> Problem:
    """Many sources drawn in proportion to density, sub-grid mfp law."""
    z = 7.0
    delta = lognormal_delta(n, 0.6, seed)
    nbar = mean_nH_comoving() * (1 + z) ** 3
    nH = nbar * delta
    rng = np.random.default_rng(seed + 1000)
    p = delta / delta.sum()
    cells = rng.choice(delta.size, size=nsrc, replace=True, p=p)
    ndot = np.exp(rng.normal(math.log(1e53), 1.0, nsrc))
    edges = 13.6 * 4.0 ** (np.arange(4) / 3.0)        # 3 bins over 13.6 .. 54.4 eV
    mfp = Mfp(mode=2, lambda0_cm_comoving=5.0 * MPC, delta_exp=1.0, gamma_ref=1e-12,
              gamma_exp=2.0 / 3.0, gamma_floor=1e-15, xion_threshold=0.5, nH_mean=nbar)
    opts = Options(l_src=0, n_ray_min=3.0, seed=seed, isothermal=True, rates=1,
                   x_init=1.2e-3, T_init=1e4)
    box = 200.0 * MPC / H_LITTLE * (n / 200.0)
    return Problem("cosmo20k", (n, n, n), box, z, nH, blackbody_bins(1e5, edges), mfp, opts,
                   cell_ijk(cells, n), ndot, 1.0 * MYR, nsteps)


_UNIT_FIELDS = {}


def _unit_field(n: int, k: int) -> np.ndarray:
    """A seeded Gaussian field of P(k) ~ k^-2 with mean 0 and std 1 (cached;
    a few per grid size serve every request of a stream)."""
    key = (n, k)
    if key not in _UNIT_FIELDS:
        _UNIT_FIELDS[key] = np.log(lognormal_delta(n, 1.0, 30_000 + 97 * n + k)) + 0.5
    return _UNIT_FIELDS[key]


def batch_member(seed: int, sizes=(32, 48, 64, 96), nsteps: int = 50, shared_fields: bool = False) -> Problem:
    """One member of the uneven batch: grid from `sizes`, sigma_ln in
    [0.3,1.2], 1..32 sources drawn in proportion to density, mfp scale in
    [1,20] cell widths, 1 cMpc/h cells at z = 7, 3 bins, isothermal.
    With shared_fields the Gaussian field is one of four cached per grid
    size, periodically shifted by a seeded offset (cheap for long streams)."""
    rng = np.random.default_rng(10_000 + seed)
    n = int(rng.choice(sizes))
    sig = float(rng.uniform(0.3, 1.2))
    nsrc = int(rng.integers(1, 33))
    scale = float(rng.uniform(1.0, 20.0))
    z = 7.0
    if shared_fields:
        g = _unit_field(n, seed % 4).reshape(n, n, n)
        g = np.roll(g, tuple(int(v) for v in rng.integers(0, n, 3)), axis=(0, 1, 2)).reshape(-1)
        delta = np.exp(sig * g - 0.5 * sig * sig)
    else:
        delta = lognormal_delta(n, sig, 20_000 + seed)
    nbar = mean_nH_comoving() * (1 + z) ** 3
    p = delta / delta.sum()
    cells = rng.choice(delta.size, size=nsrc, replace=True, p=p)
    ndot = np.exp(rng.normal(math.log(1e53), 1.0, nsrc))
    dx_c = MPC / H_LITTLE
    edges = 13.6 * 4.0 ** (np.arange(4) / 3.0)
    mfp = Mfp(mode=2, lambda0_cm_comoving=scale * dx_c, nH_mean=nbar)
    opts = Options(l_src=0, n_ray_min=3.0, seed=seed, isothermal=True, rates=1,
                   x_init=1.2e-3, T_init=1e4)
    return Problem(f"batch{seed}", (n, n, n), n * dx_c, z, nbar * delta, blackbody_bins(1e5, edges),
                   mfp, opts, cell_ijk(cells, n), ndot, 1.0 * MYR, nsteps)


def batch64(count: int = 64, sizes=(32, 48, 64, 96), nsteps: int = 50):
    return [batch_member(s, sizes, nsteps) for s in range(count)]


def request_stream(count: int = 1000, mean_gap_s: float = 0.05, sizes=(32, 64, 96, 128, 160),
                   steps=(50, 200), seed: int = 5):
    """Poisson arrivals (exponential gaps) of batch-style simulations with
    uniform grid sizes and step counts."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(mean_gap_s, count))
    out = []
    for i in range(count):
        nst = int(rng.integers(steps[0], steps[1] + 1))
        prob = batch_member(100_000 + i, sizes, nst, shared_fields=True)
        out.append((float(t[i]), prob))
    return out
