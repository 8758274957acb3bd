"""Seeded synthetic inputs for the FLD step: grids, parameters, fields.

This module holds no arithmetic of the FLD method itself (no limiter, no
assembly, no solver).  It only builds the inputs that both the CUDA path and
the CPU oracle are fed: physical constants, grid and parameter records, and
the fields E^n, n_HI and eta of the benchmark workloads.

Workloads (the paper's test problems and cosmological boxes are replaced by
these generators; no dataset is read):

* ``config_uniform``: a uniform neutral medium with point sources, built after
  the isothermal Stromgren test of Sec. 4.1.1 (n_H = 1e-3 cm^-3, box 6.6 kpc,
  sources of 5e48 photons/s at h nu = 13.6 eV, sigma = 1.6e-18 cm^2,
  initial E = 1e-30 erg/cm^3, dt = 1e5 yr).
* ``config_lognormal``: a log-normal density from a Gaussian random field with
  P(k) ~ k^-2, sources at the densest 26-neighbour local maxima.
* ``request_stream``: a Poisson stream of independent grids of mixed sizes.

Arrays are shaped (nz, ny, nx) (x fastest) and float64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------- constants
C_LIGHT = 2.99792458e10          # cm/s
KPC = 3.0856776e21               # cm
YEAR = 3.15576e7                 # s (Julian)
EV = 1.602176634e-12             # erg
HNU_HI = 13.6 * EV               # erg, HI threshold (Sec. 2, Sec. 4.1.1)
SIGMA_HI = 1.6e-18               # cm^2, grey HI cross-section of the workloads
ALPHA_B = 2.59e-13               # cm^3/s, case-B recombination at 1e4 K
BOX = 6.6 * KPC                  # cm (Sec. 4.1.1)
DT = 1e5 * YEAR                  # s
E0 = 1e-30                       # erg/cm^3
NDOT = 5e48                      # photons/s per source (Sec. 4.1.1)

LIMITER_PAPER, LIMITER_LP = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
SMOOTH_RBGS, SMOOTH_JACOBI = 0, 1
BC_ZERO_GRADIENT, BC_PERIODIC = 0, 1


@dataclasses.dataclass
class Grid:
    """Uniform Cartesian grid: cells per axis, cell widths (cm), periodicity,
    and the faces held at a fixed E (Dirichlet; value 0 = outflow), per side
    in the order x lo, x hi, y lo, y hi, z lo, z hi.  Other non-periodic faces
    reflect (zero gradient)."""
    n: Tuple[int, int, int]
    h: Tuple[float, float, float]
    periodic: Tuple[bool, bool, bool] = (False, False, False)
    dirichlet: Tuple[bool, bool, bool, bool, bool, bool] = (False,) * 6
    ebc: Tuple[float, float, float, float, float, float] = (0.0,) * 6

    def outflow_upper(self) -> "Grid":
        """The boundary set of the Sec. 4.1 tests: reflecting faces at x = 0,
        y = 0, z = 0 and outflow at the three upper faces."""
        return dataclasses.replace(self, dirichlet=(False, True) * 3, ebc=(0.0,) * 6)

    @property
    def shape(self):
        """Array shape (nz, ny, nx): x is the fastest index."""
        return (self.n[2], self.n[1], self.n[0])

    @property
    def cells(self) -> int:
        """Number of cells."""
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def volume(self) -> float:
        """Cell volume, cm^3."""
        return self.h[0] * self.h[1] * self.h[2]

    @staticmethod
    def cube(n: int, box: float = BOX, periodic: bool = False) -> "Grid":
        """n^3 cubic cells filling a box of side box (cm)."""
        return Grid((n, n, n), (box / n,) * 3, (periodic,) * 3)


@dataclasses.dataclass
class Params:
    """Physical and solver parameters of one FLD step (CGS)."""
    dt: float = DT
    c: float = C_LIGHT
    L_unit: float = BOX
    dmax_coef: float = 0.006
    rmin_coef: float = 1e-20
    sigma: float = SIGMA_HI
    adot_over_a: float = 0.0
    hnu: float = HNU_HI
    limiter: int = LIMITER_PAPER
    precision: int = PREC_FP64
    smoother: int = SMOOTH_RBGS
    jacobi_omega: float = 0.8
    rtol: float = 1e-8
    max_iter: int = 50
    pre: int = 1
    post: int = 1
    inner_rtol: float = 1e-4
    coarse_cap: int = 1024
    graphs: int = -1
    fused_post: int = 0
    theta: float = 1.0
    scale_factor: float = 1.0
    tail_cells: int = 32768
    paper_order: int = 0
    persistent_cells: int = 0
    precond_bf16: int = 1


@dataclasses.dataclass
class Case:
    """One workload instance: grid, parameters and the three input fields."""
    name: str
    grid: Grid
    params: Params
    E: np.ndarray
    nHI: np.ndarray
    eta: np.ndarray
    nH: Optional[np.ndarray] = None
    sources: Optional[np.ndarray] = None   # (S, 3) cell indices (i, j, k)


# ------------------------------------------------------------------ helpers

def point_source_eta(grid: Grid, cells: np.ndarray, rates: np.ndarray,
                     hnu: float = HNU_HI) -> np.ndarray:
    """Emissivity field of point sources: each source deposits N_dot h nu / V
    (erg s^-1 cm^-3) in its cell; sources sharing a cell add up."""
    eta = np.zeros(grid.shape)
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, 3)
    rates = np.broadcast_to(np.asarray(rates, dtype=np.float64), (cells.shape[0],))
    np.add.at(eta, (cells[:, 2], cells[:, 1], cells[:, 0]), rates * hnu / grid.volume)
    return eta


def gaussian_field(n: int, seed: int, slope: float = -2.0, device: str = "cpu") -> np.ndarray:
    """Unit-variance periodic Gaussian random field with P(k) ~ k^slope:
    seeded white noise, FFT, amplitude times k^(slope/2), k = 0 removed."""
    import torch
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    t = torch.from_numpy(white).to(device)
    f = torch.fft.rfftn(t)
    kz = torch.fft.fftfreq(n, device=device, dtype=torch.float64).view(-1, 1, 1)
    ky = torch.fft.fftfreq(n, device=device, dtype=torch.float64).view(1, -1, 1)
    kx = torch.fft.rfftfreq(n, device=device, dtype=torch.float64).view(1, 1, -1)
    k2 = kx * kx + ky * ky + kz * kz
    amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (slope / 4.0), torch.zeros_like(k2))
    f = f * amp
    delta = torch.fft.irfftn(f, s=(n, n, n))
    delta = delta - delta.mean()
    delta = delta / delta.std()
    return delta.cpu().numpy()


def lognormal_density(n: int, seed: int, sigma_ln: float, mean: float,
                      clamp: Optional[Tuple[float, float]] = None,
                      device: str = "cpu") -> np.ndarray:
    """rho = exp(sigma delta - sigma^2/2) scaled to the requested mean."""
    delta = gaussian_field(n, seed, device=device)
    rho = np.exp(sigma_ln * delta - 0.5 * sigma_ln * sigma_ln)
    rho *= mean / rho.mean()
    if clamp is not None:
        rho = np.clip(rho, clamp[0] * mean, clamp[1] * mean)
    return rho


def density_peaks(rho: np.ndarray, count: int, periodic: bool,
                  device: str = "cpu") -> np.ndarray:
    """Cell indices (i, j, k) of the ``count`` densest 26-neighbour local
    maxima (topped up with the densest remaining cells if there are fewer)."""
    import torch
    import torch.nn.functional as F
    count = min(count, rho.size)
    t = torch.from_numpy(np.ascontiguousarray(rho)).to(device)[None, None]
    if periodic:
        pad = F.pad(t, (1, 1, 1, 1, 1, 1), mode="circular")
    else:
        pad = F.pad(t, (1, 1, 1, 1, 1, 1), mode="constant", value=-math.inf)
    mx = F.max_pool3d(pad, 3, stride=1)
    flat = t.flatten()
    is_peak = (t >= mx).flatten()
    score = torch.where(is_peak, flat, torch.full_like(flat, -math.inf))
    k = min(count, int(is_peak.sum().item()))
    idx = torch.topk(score, k).indices
    if k < count:
        rest = torch.where(is_peak, torch.full_like(flat, -math.inf), flat)
        idx = torch.cat([idx, torch.topk(rest, count - k).indices])
    idx = idx.cpu().numpy()
    nz, ny, nx = rho.shape
    return np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], axis=1)


def nearest_source_distance(grid: Grid, cells: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    """Distance (cm) from each cell centre to the nearest source cell centre,
    minimum image on periodic axes."""
    nz, ny, nx = grid.shape
    src = np.asarray(cells, dtype=np.float64).reshape(-1, 3)
    out = np.empty(grid.cells)
    flat = np.arange(grid.cells)
    n = np.array(grid.n, dtype=np.float64)
    h = np.array(grid.h)
    for s in range(0, grid.cells, chunk):
        f = flat[s:s + chunk]
        pos = np.stack([f % nx, (f // nx) % ny, f // (nx * ny)], axis=1).astype(np.float64)
        best = np.full(len(f), np.inf)
        for c in src:
            d = np.abs(pos - c)
            for ax in range(3):
                if grid.periodic[ax]:
                    d[:, ax] = np.minimum(d[:, ax], n[ax] - d[:, ax])
            dist = np.sqrt(((d * h) ** 2).sum(axis=1))
            np.minimum(best, dist, out=best)
        out[s:s + chunk] = best
    return out.reshape(grid.shape)


# ---------------------------------------------------------------- workloads

def config_uniform(n: int = 32, sources: int = 1, seed: int = 0, periodic: bool = False,
                   limiter: int = LIMITER_LP, precision: int = PREC_FP64,
                   n_H: float = 1e-3, centre: bool = True) -> Case:
    """Uniform neutral hydrogen with point sources of 5e48 photons/s.

    ``sources == 1`` and ``centre`` puts the source in cell (n/2, n/2, n/2);
    otherwise sources go to seeded uniform-random distinct cells."""
    g = Grid.cube(n, periodic=periodic)
    p = Params(limiter=limiter, precision=precision)
    if sources == 1 and centre:
        cells = np.array([[n // 2, n // 2, n // 2]])
    else:
        rng = np.random.default_rng(seed)
        pick = rng.choice(g.cells, size=min(sources, g.cells), replace=False)
        cells = np.stack([pick % n, (pick // n) % n, pick // (n * n)], axis=1)
    nH = np.full(g.shape, n_H)
    return Case(name=f"uniform{n}_s{len(cells)}", grid=g, params=p,
                E=np.full(g.shape, E0), nHI=nH.copy(),
                eta=point_source_eta(g, cells, NDOT), nH=nH, sources=cells)


def config_two_sources(nx: int = 128, theta: float = 1.0, precision: int = PREC_FP64) -> Case:
    """Two sources of 5e48 photons/s 8 kpc apart in a uniform static medium
    (n_H = 1e-3 cm^-3, neutral) filling a 20 x 10 x 10 kpc box resolved by
    nx x nx/2 x nx/2 cubic cells (128 x 64 x 64 in the paper's test of two
    merging HII regions, Sec. 4.1).  The sources sit on the long axis, 4 kpc
    either side of the centre.  Radiation leaves through all six faces
    (outflow), L_unit = 20 kpc."""
    ny = nx // 2
    h = 20.0 * KPC / nx
    g = Grid((nx, ny, ny), (h, h, h), dirichlet=(True,) * 6, ebc=(0.0,) * 6)
    p = Params(L_unit=20.0 * KPC, theta=theta, precision=precision)
    centre = np.array([10.0, 5.0, 5.0]) * KPC
    pos = [centre + np.array([dx, 0.0, 0.0]) * KPC for dx in (-4.0, 4.0)]
    cells = np.array([[int(v // h) for v in q] for q in pos])
    nH = np.full(g.shape, 1e-3)
    return Case(name=f"two_sources{nx}", grid=g, params=p, E=np.full(g.shape, E0), nHI=nH.copy(),
                eta=point_source_eta(g, cells, NDOT), nH=nH, sources=cells)


def config_lognormal(n: int = 128, seed: int = 2, sigma_ln: float = 1.0,
                     mean_nH: float = 2e-4, sources: int = 256, periodic: bool = True,
                     tanh_ionised: bool = True, log_uniform_rates: Tuple[float, float] = (1e50, 1e53),
                     clamp: Optional[Tuple[float, float]] = None, limiter: int = LIMITER_PAPER,
                     precision: int = PREC_FP64, device: str = "cpu") -> Case:
    """Log-normal density (sigma_ln, mean) with sources at the densest peaks.

    With ``tanh_ionised`` the neutral fraction is max(tanh(d / 4h), 1e-6) with
    d the distance to the nearest source; otherwise the gas is fully neutral.
    ``log_uniform_rates`` draws each source's photon rate log-uniformly in the
    interval; None gives every source 5e48 photons/s."""
    g = Grid.cube(n, periodic=periodic)
    p = Params(limiter=limiter, precision=precision)
    rho = lognormal_density(n, seed, sigma_ln, mean_nH, clamp=clamp, device=device)
    cells = density_peaks(rho, sources, periodic, device=device)
    rng = np.random.default_rng(seed + 1000)
    if log_uniform_rates is None:
        rates = np.full(len(cells), NDOT)
    else:
        lo, hi = np.log(log_uniform_rates[0]), np.log(log_uniform_rates[1])
        rates = np.exp(rng.uniform(lo, hi, size=len(cells)))
    if tanh_ionised:
        d = nearest_source_distance(g, cells)
        x = np.maximum(np.tanh(d / (4.0 * g.h[0])), 1e-6)
    else:
        x = np.ones(g.shape)
    return Case(name=f"lognormal{n}_s{len(cells)}", grid=g, params=p,
                E=np.full(g.shape, E0), nHI=rho * x, eta=point_source_eta(g, cells, rates),
                nH=rho, sources=cells)


def config1(n: int = 32) -> Case:
    """FP64 step, 32^3, zero-gradient, one central 5e48 source, LP limiter."""
    return config_uniform(n=n, sources=1, limiter=LIMITER_LP, precision=PREC_FP64)


def config2(n: int = 128, device: str = "cpu") -> Case:
    """FP64 step, 128^3 periodic, log-normal sigma 1, mean 2e-4, 256 sources,
    rates log-uniform in [1e50, 1e53], tanh neutral fraction."""
    c = config_lognormal(n=n, seed=2, sigma_ln=1.0, mean_nH=2e-4, sources=max(1, 256 * n ** 3 // 128 ** 3),
                         periodic=True, device=device)
    c.name = f"config2_{n}"
    return c


def config3(n: int = 256, sources: int = 4096) -> Case:
    """Mixed precision, 256^3 zero-gradient uniform medium, 4096 random sources."""
    c = config_uniform(n=n, sources=sources, seed=3, limiter=LIMITER_PAPER, precision=PREC_MIXED)
    c.name = f"config3_{n}"
    return c


def config4(n: int = 512, sources: int = 65536, device: str = "cpu") -> Case:
    """Mixed precision, 512^3 zero-gradient, log-normal sigma 1.5 with mean
    n_H = 1e-3 clamped to [1e-3, 1e3] x mean, fully neutral, 65536 sources
    of 5e48 photons/s at the densest peaks."""
    c = config_lognormal(n=n, seed=4, sigma_ln=1.5, mean_nH=1e-3, sources=sources, periodic=False,
                         tanh_ionised=False, log_uniform_rates=None, clamp=(1e-3, 1e3),
                         precision=PREC_MIXED, device=device)
    c.name = f"config4_{n}"
    return c


@dataclasses.dataclass
class Request:
    """One serving request: id, arrival time, grid size n (n^3 cells), the
    seed of its source positions and its number of sources."""

    rid: int
    arrival: float   # s after the stream starts
    n: int
    seed: int
    sources: int


def request_stream(count: int = 2000, rate: float = 500.0, seed: int = 5,
                   sizes: Sequence[int] = (16, 32, 48, 64, 96, 128)) -> List[Request]:
    """Poisson arrivals (exponential gaps of mean 1/rate), uniform sizes,
    1-64 sources each, one seed per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = rng.choice(np.asarray(sizes), size=count)
    srcs = rng.integers(1, 65, size=count)
    seeds = rng.integers(0, 2 ** 31 - 1, size=count)
    return [Request(i, float(t[i]), int(ns[i]), int(seeds[i]), int(srcs[i])) for i in range(count)]


def request_case(r: Request) -> Case:
    """Host arrays of one request: a uniform neutral medium (n_H = 1e-3) with
    the request's seeded sources of 5e48 photons/s, mixed precision."""
    c = config_uniform(n=r.n, sources=r.sources, seed=r.seed, centre=False,
                       limiter=LIMITER_PAPER, precision=PREC_MIXED)
    c.name = f"req{r.rid}_{r.n}"
    return c


def request_sources(r: Request) -> Tuple[np.ndarray, np.ndarray]:
    """The payload of one request: source cells (i, j, k) and photon rates,
    the same ones request_case places."""
    g = Grid.cube(r.n)
    rng = np.random.default_rng(r.seed)
    pick = rng.choice(g.cells, size=min(r.sources, g.cells), replace=False)
    cells = np.stack([pick % r.n, (pick // r.n) % r.n, pick // (r.n * r.n)], axis=1)
    return cells, np.full(len(cells), NDOT)


def random_case(n: Sequence[int], seed: int, periodic=(False, False, False),
                limiter: int = LIMITER_PAPER, E_decades: Tuple[float, float] = (-30, -12),
                nHI_decades: Tuple[float, float] = (-6, 0), zero_frac: float = 0.0,
                box: float = BOX) -> Case:
    """Small random instance for parity tests: log-uniform E and n_HI over the
    given decades, a few sources, optional exact zeros in E and n_HI."""
    nx, ny, nz = (int(v) for v in n)
    g = Grid((nx, ny, nz), (box / nx, box / ny, box / nz), tuple(bool(v) for v in periodic))
    rng = np.random.default_rng(seed)
    E = 10.0 ** rng.uniform(*E_decades, size=g.shape)
    nHI = 10.0 ** rng.uniform(*nHI_decades, size=g.shape) * 1e-3
    if zero_frac > 0:
        E[rng.random(g.shape) < zero_frac] = 0.0
        nHI[rng.random(g.shape) < zero_frac] = 0.0
    ns = max(1, g.cells // 64)
    pick = rng.choice(g.cells, size=ns, replace=False)
    cells = np.stack([pick % nx, (pick // nx) % ny, pick // (nx * ny)], axis=1)
    rates = 10.0 ** rng.uniform(48, 52, size=ns)
    p = Params(limiter=limiter)
    return Case(name=f"random{nx}x{ny}x{nz}_{seed}", grid=g, params=p, E=E, nHI=nHI,
                eta=point_source_eta(g, cells, rates), sources=cells)
