"""Grey spectral integrals of the FLD model and the fields built from them
(oracle side; TEST INFRASTRUCTURE ONLY, like the rest of this package).

What it computes (Sec. 2, "Model coupling"): with the assumed spectral
energy distribution chi(nu) of the radiation,
  - the grey opacity (Eq. "opacity"):
        kappa = sum_i n_i K_i,  K_i = int_{nu_i} sigma_i chi dnu / int_{nu_1} chi dnu;
  - the photoionisation rates (Eq. "photoionization"):
        Gamma_i = (c E / h) P_i,  P_i = int_{nu_i} sigma_i chi / nu dnu / int_{nu_1} chi dnu;
  - the photoheating rate (Eq. "photoheating"):
        G = (c E / rho_b) sum_i n_i H_i,
        H_i = int_{nu_i} sigma_i chi (1 - nu_i / nu) dnu / int_{nu_1} chi dnu;
for the species HI, HeI, HeII (thresholds 13.6, 24.6, 54.4 eV).  For a
multigroup radiation field the same integrals are taken over each group
[nu_g, nu_{g+1}] (lower limits max(nu_g, nu_i)), and the group's share of
the emissivity is F_g = int_g chi / int_{nu_1}^{nu_max} chi.

Readings where the paper is silent or at odds with itself:
  - the denominator of K_i runs from nu_1 (the grey energy's own lower
    limit, Eq. "grey_definition"), not from nu_i as printed in Eq.
    "opacity": photons below nu_i are part of E but cannot be absorbed by
    species i;
  - "infinity" is an upper frequency nu_max of the SED (default 1000 nu_HI);
  - sigma_i(nu) = sigma_0 [beta (nu/nu_i)^-s + (1 - beta)(nu/nu_i)^(-s-1)]
    for nu >= nu_i (Osterbrock 1989, Table 2.1 fits; the paper cites
    Osterbrock for these rates), with (sigma_0, beta, s) = (6.30e-18, 1.34,
    2.99) for HI, (7.83e-18, 1.66, 2.05) for HeI, (1.58e-18, 1.34, 2.99) for
    HeII; exposed as parameters;
  - SEDs: monochromatic (a line at nu_mono), blackbody (chi ~ nu^3 /
    (exp(h nu / k T) - 1)) and power law (chi ~ nu^-alpha).  The Pop II SED
    of the production runs is a table the paper does not give.

The integrals are taken with scipy's adaptive quadrature (a library
primitive), in the variable u = ln(nu / nu_i) on each species' range.
"""
from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np

H_PLANCK = 6.62607015e-27       # erg s
K_BOLTZ = 1.380649e-16          # erg / K
EV = 1.602176634e-12            # erg
C_LIGHT = 2.99792458e10         # cm / s

NU_HI = 13.6 * EV / H_PLANCK
NU_HEI = 24.6 * EV / H_PLANCK
NU_HEII = 54.4 * EV / H_PLANCK

SPECIES = ("HI", "HeI", "HeII")
CROSS_SECTIONS = {      # nu_threshold (Hz), sigma_0 (cm^2), beta, s
    "HI": (NU_HI, 6.30e-18, 1.34, 2.99),
    "HeI": (NU_HEI, 7.83e-18, 1.66, 2.05),
    "HeII": (NU_HEII, 1.58e-18, 1.34, 2.99),
}

MONO, BLACKBODY, POWERLAW = 0, 1, 2


def sigma(species: str, nu, xs=None):
    """Photoionisation cross section of a species at frequency nu (0 below
    its threshold)."""
    nu_t, s0, beta, s = (xs or CROSS_SECTIONS)[species]
    nu = np.asarray(nu, dtype=np.float64)
    r = nu / nu_t
    out = s0 * (beta * r ** (-s) + (1.0 - beta) * r ** (-s - 1.0))
    return np.where(nu >= nu_t, out, 0.0)


def chi(sed: Dict, nu):
    """Unnormalised spectral shape chi(nu)."""
    nu = np.asarray(nu, dtype=np.float64)
    if sed["kind"] == BLACKBODY:
        x = H_PLANCK * nu / (K_BOLTZ * sed["T"])
        with np.errstate(over="ignore"):       # exp(x) beyond FP64: chi = 0
            return nu ** 3 / np.expm1(x)
    if sed["kind"] == POWERLAW:
        return nu ** (-sed["alpha"])
    raise ValueError("chi of a monochromatic SED is a delta function")


def _quad_log(f, lo, hi):
    """int_lo^hi f(nu) dnu in u = ln nu (adaptive Gauss-Kronrod)."""
    from scipy.integrate import quad
    if not hi > lo:
        return 0.0
    g = lambda u: f(math.exp(u)) * math.exp(u)
    ul, uh = math.log(lo), math.log(hi)
    # split the range so the adaptive rule sees every decade
    edges = np.linspace(ul, uh, max(2, int((uh - ul) / 0.5) + 2))
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        v, _ = quad(g, a, b, epsabs=0.0, epsrel=1e-13, limit=200)
        total += v
    return total


def group_integrals(sed: Dict, edges: Sequence[float], xs=None) -> np.ndarray:
    """For groups [edges[g], edges[g+1]]: rows g of (K_HI, K_HeI, K_HeII,
    P_HI, P_HeI, P_HeII, H_HI, H_HeI, H_HeII, F) as defined in the module
    docstring, normalised by int_g chi (K, P, H) and by int over all groups
    of chi (F).  A grey field is the single group [nu_1, nu_max]."""
    xs = xs or CROSS_SECTIONS
    edges = [float(e) for e in edges]
    G = len(edges) - 1
    out = np.zeros((G, 10))
    if sed["kind"] == MONO:
        nu0 = sed["nu"]
        for g in range(G):
            if not (edges[g] <= nu0 < edges[g + 1]):
                continue
            for i, sp in enumerate(SPECIES):
                nu_t = xs[sp][0]
                sg = float(sigma(sp, nu0, xs))
                out[g, i] = sg
                out[g, 3 + i] = sg / nu0
                out[g, 6 + i] = sg * (1.0 - nu_t / nu0) if nu0 >= nu_t else 0.0
            out[g, 9] = 1.0
        return out
    norm_all = _quad_log(lambda v: float(chi(sed, v)), edges[0], edges[-1])
    for g in range(G):
        lo, hi = edges[g], edges[g + 1]
        norm = _quad_log(lambda v: float(chi(sed, v)), lo, hi)
        for i, sp in enumerate(SPECIES):
            nu_t = xs[sp][0]
            a = max(lo, nu_t)
            k = _quad_log(lambda v: float(sigma(sp, v, xs) * chi(sed, v)), a, hi)
            p = _quad_log(lambda v: float(sigma(sp, v, xs) * chi(sed, v)) / v, a, hi)
            h = _quad_log(lambda v: float(sigma(sp, v, xs) * chi(sed, v)) * (1.0 - nu_t / v), a, hi)
            out[g, i] = k / norm
            out[g, 3 + i] = p / norm
            out[g, 6 + i] = h / norm
        out[g, 9] = norm / norm_all
    return out


def group_fields(coef: np.ndarray, n_HI, n_HeI=None, n_HeII=None, eta=None):
    """Per group: kappa_g = sum_i n_i K_gi and eta_g = F_g eta."""
    dens = [np.asarray(n_HI, dtype=np.float64)]
    for d in (n_HeI, n_HeII):
        dens.append(np.zeros_like(dens[0]) if d is None else np.asarray(d, dtype=np.float64))
    kap = [sum(coef[g, i] * dens[i] for i in range(3)) for g in range(coef.shape[0])]
    etas = None if eta is None else [coef[g, 9] * np.asarray(eta, dtype=np.float64) for g in range(coef.shape[0])]
    return kap, etas


def photo_rates(coef: np.ndarray, E_groups, n_HI, n_HeI=None, n_HeII=None, rho_b=None, c=C_LIGHT):
    """Gamma_i = sum_g (c E_g / h) P_gi and G = sum_g (c E_g / rho_b) sum_i n_i H_gi."""
    dens = [np.asarray(n_HI, dtype=np.float64)]
    for d in (n_HeI, n_HeII):
        dens.append(np.zeros_like(dens[0]) if d is None else np.asarray(d, dtype=np.float64))
    gam = [sum(c * np.asarray(E_groups[g]) / H_PLANCK * coef[g, 3 + i] for g in range(coef.shape[0]))
           for i in range(3)]
    heat = None
    if rho_b is not None:
        heat = sum(c * np.asarray(E_groups[g]) / np.asarray(rho_b) * sum(dens[i] * coef[g, 6 + i] for i in range(3))
                   for g in range(coef.shape[0]))
    return gam, heat
