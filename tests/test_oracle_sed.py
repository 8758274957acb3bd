"""Pins of the oracle's grey spectral integrals (Sec. 2, Eqs. "opacity",
"photoionization", "photoheating") against closed forms: hydrogenic cross
sections with power-law and blackbody spectra, monochromatic lines, and the
additivity of group integrals.  CPU only."""
import math

import numpy as np
import pytest

from oracle import sed

# hydrogenic cross sections sigma_0 (nu / nu_i)^-3 for closed forms
HYDRO = {sp: (v[0], v[1], 1.0, 3.0) for sp, v in sed.CROSS_SECTIONS.items()}


def test_cross_section_fits_at_threshold():
    for sp, (nu_t, s0, beta, s) in sed.CROSS_SECTIONS.items():
        assert float(sed.sigma(sp, nu_t)) == pytest.approx(s0, rel=1e-15)
        assert float(sed.sigma(sp, 0.999 * nu_t)) == 0.0
        # decreasing above threshold
        v = sed.sigma(sp, nu_t * np.array([1.0, 2.0, 4.0]))
        assert v[0] > v[1] > v[2] > 0


@pytest.mark.parametrize("alpha", [1.5, 3.0, 4.5])
def test_powerlaw_hydrogenic_closed_forms(alpha):
    # chi ~ nu^-alpha, sigma = s0 (nu/nu_1)^-3 from nu_1 to (effectively)
    # infinity: K = s0 (alpha-1)/(alpha+2), P = s0 (alpha-1)/((alpha+3) nu_1),
    # H = s0 (alpha-1) (1/(alpha+2) - 1/(alpha+3))
    nu1 = sed.NU_HI
    numax = nu1 * 1e9
    c = sed.group_integrals({"kind": sed.POWERLAW, "alpha": alpha}, [nu1, numax], HYDRO)[0]
    s0 = sed.CROSS_SECTIONS["HI"][1]
    tail = (numax / nu1) ** (1 - alpha)       # the spectrum's share beyond nu_max
    assert c[0] == pytest.approx(s0 * (alpha - 1) / (alpha + 2), rel=1e-9 + 3 * tail)
    assert c[3] == pytest.approx(s0 * (alpha - 1) / ((alpha + 3) * nu1), rel=1e-9 + 3 * tail)
    assert c[6] == pytest.approx(s0 * (alpha - 1) * (1 / (alpha + 2) - 1 / (alpha + 3)), rel=1e-9 + 3 * tail)
    # HeI and HeII: the same forms scaled by (nu_1 / nu_i)^(alpha - 1) and their own sigma_0
    for i, sp in ((1, "HeI"), (2, "HeII")):
        nu_i, s0i = sed.CROSS_SECTIONS[sp][:2]
        f = (nu1 / nu_i) ** (alpha - 1)
        assert c[i] == pytest.approx(f * s0i * (alpha - 1) / (alpha + 2), rel=1e-9 + 3 * tail)
    assert c[9] == pytest.approx(1.0, rel=1e-14)


def planck_tail(x1, n, kmax=200):
    """int_{x1}^inf x^n / (e^x - 1) dx by its exponential series."""
    tot = 0.0
    for k in range(1, kmax + 1):
        s = sum(math.factorial(n) / math.factorial(j) * x1 ** j / k ** (n - j + 1) for j in range(n + 1))
        tot += math.exp(-k * x1) * s
    return tot


@pytest.mark.parametrize("T", [3e4, 1e5])
def test_blackbody_hydrogenic_opacity_closed_form(T):
    # sigma chi dnu ~ dx / (e^x - 1) and chi dnu ~ x^3 dx / (e^x - 1), x = h nu / k T:
    # K = s0 x1^3 (-ln(1 - e^-x1)) / int_{x1} x^3/(e^x - 1) dx
    nu1 = sed.NU_HI
    x1 = sed.H_PLANCK * nu1 / (sed.K_BOLTZ * T)
    c = sed.group_integrals({"kind": sed.BLACKBODY, "T": T}, [nu1, 1e3 * nu1], HYDRO)[0]
    s0 = sed.CROSS_SECTIONS["HI"][1]
    K = s0 * x1 ** 3 * (-math.log(-math.expm1(-x1))) / planck_tail(x1, 3)
    assert c[0] == pytest.approx(K, rel=1e-10)
    # P: sigma chi / nu ~ x^-1 / (e^x - 1); by series int_{x1} x^-1 e^{-kx} = E1(k x1)
    from scipy.special import exp1
    P = s0 * x1 ** 3 * sum(exp1(k * x1) for k in range(1, 400)) / planck_tail(x1, 3) / nu1
    assert c[3] == pytest.approx(P, rel=1e-9)


def test_monochromatic_line():
    nu0 = 1.5 * sed.NU_HEI
    c = sed.group_integrals({"kind": sed.MONO, "nu": nu0}, [sed.NU_HI, 1e3 * sed.NU_HI])[0]
    for i, sp in enumerate(sed.SPECIES):
        s = float(sed.sigma(sp, nu0))
        assert c[i] == s and c[3 + i] == s / nu0
    assert c[2] == 0.0                      # below the HeII threshold
    assert c[6] == pytest.approx(float(sed.sigma("HI", nu0)) * (1 - sed.NU_HI / nu0), rel=1e-15)


@pytest.mark.parametrize("sedd", [{"kind": sed.BLACKBODY, "T": 5e4}, {"kind": sed.POWERLAW, "alpha": 1.8}])
def test_groups_add_up_to_the_grey_integrals(sedd):
    # group integrals are additive: K_grey = sum_g F_g K_g (and so P, H);
    # edges straddling the He thresholds
    nu1 = sed.NU_HI
    edges = [nu1, 1.5 * nu1, sed.NU_HEI, 3.0 * nu1, sed.NU_HEII, 10 * nu1, 1e3 * nu1]
    grey = sed.group_integrals(sedd, [edges[0], edges[-1]])[0]
    grp = sed.group_integrals(sedd, edges)
    assert grp[:, 9].sum() == pytest.approx(1.0, rel=1e-12)
    for k in range(9):
        assert (grp[:, 9] * grp[:, k]).sum() == pytest.approx(grey[k], rel=1e-10)
    # groups below a threshold see no absorption by that species
    assert grp[0, 1] == 0.0 and grp[1, 1] == 0.0 and grp[3, 2] == 0.0


def test_fields_and_rates():
    coef = sed.group_integrals({"kind": sed.BLACKBODY, "T": 1e5}, [sed.NU_HI, 2 * sed.NU_HI, 1e3 * sed.NU_HI])
    rng = np.random.default_rng(1)
    nHI, nHeI, nHeII, eta = (rng.random(50) for _ in range(4))
    kap, etas = sed.group_fields(coef, nHI, nHeI, nHeII, eta)
    for g in range(2):
        np.testing.assert_allclose(kap[g], coef[g, 0] * nHI + coef[g, 1] * nHeI + coef[g, 2] * nHeII, rtol=1e-15)
    np.testing.assert_allclose(etas[0] + etas[1], eta, rtol=1e-12)
    E = [rng.random(50), rng.random(50)]
    rho = rng.random(50) + 1
    gam, heat = sed.photo_rates(coef, E, nHI, nHeI, nHeII, rho)
    np.testing.assert_allclose(gam[0], sed.C_LIGHT / sed.H_PLANCK * (E[0] * coef[0, 3] + E[1] * coef[1, 3]),
                               rtol=1e-14)
    assert np.all(heat > 0)
