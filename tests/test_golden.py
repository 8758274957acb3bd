"""Values the paper prints, kept as text fixtures under tests/golden/ (each
file names its section or table), against the library's defaults, the
oracle's limiter and the synthetic inputs of the tests.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1306_0645_gb300 import fld, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("=", 1))
                out[k] = v
    return out


def test_table1_solver_defaults():
    # Table 1: PCG, at most 50 iterations, tolerance 1e-8, red/black GS with
    # one pre- and one post-sweep (the "12 MG iterations" are unused: one
    # V-cycle per CG iteration)
    t = load("table1_solver.txt")
    p = fld.make_params(synth.Params())
    assert t["outer_solver"] == "PCG"
    assert p.max_iter == int(t["cg_iterations"])
    assert p.rtol == float(t["cg_tolerance"])
    assert p.smoother == synth.SMOOTH_RBGS and "red/black" in t["mg_relaxation"]
    assert p.pre == int(t["mg_pre_sweeps"]) and p.post == int(t["mg_post_sweeps"])


def test_limiter_constants_in_library_and_oracle():
    t = load("limiter_constants.txt")
    dmax, rmin = float(t["dmax_coef"]), float(t["rmin_coef"])
    p = synth.Params()
    assert p.dmax_coef == dmax and p.rmin_coef == rmin
    lp = fld.make_params(p)
    assert lp.dmax_coef == dmax and lp.rmin_coef == rmin
    # the oracle caps at D_max = 0.006 c L_unit: a thin face with a flat E
    D = oracle.face_D(1.0, 1.0, 1e-40, 1e-40, 1e20, p)
    assert D == pytest.approx(dmax * p.c * p.L_unit, rel=1e-15)


def test_test1_parameters_and_closed_forms():
    t = load("test1_isothermal.txt")
    assert synth.NDOT == float(t["ndot"])
    assert synth.BOX == pytest.approx(float(t["box_kpc"]) * synth.KPC, rel=1e-15)
    assert synth.HNU_HI == pytest.approx(float(t["hnu_eV"]) * synth.EV, rel=1e-15)
    # the printed 2.59e-12 "cm^2/s" has a garbled unit; case-B at 1e4 K is 2.59e-13 cm^3/s
    assert synth.ALPHA_B == pytest.approx(float(t["alpha_B_printed"]) / 10, rel=1e-15)
    n_H = float(t["n_H"])
    r_s = (3 * synth.NDOT / (4 * math.pi * synth.ALPHA_B * n_H ** 2)) ** (1 / 3)
    t_rec = 1.0 / (synth.ALPHA_B * n_H)
    # the values the Stromgren tests compare against: r_s = 5.39 kpc, inside
    # the 6.6 kpc box, and t_rec = 122 Myr
    assert r_s / synth.KPC == pytest.approx(5.39, abs=0.01)
    assert t_rec / (1e6 * synth.YEAR) == pytest.approx(122.4, abs=0.1)
    assert r_s < synth.BOX


def test_two_sources_setup():
    # Sec. 4.1's consolidated HII region: the synthetic recipe places two
    # sources of the printed rate the printed distance apart in the printed
    # box and mesh
    t = load("two_sources.txt")
    case = synth.config_two_sources(int(t["mesh_x"]))
    g = case.grid
    assert tuple(g.n) == (int(t["mesh_x"]), int(t["mesh_y"]), int(t["mesh_z"]))
    extent = [g.n[a] * g.h[a] / synth.KPC for a in range(3)]
    assert extent == pytest.approx([float(t["width_kpc"]), float(t["height_kpc"]), float(t["depth_kpc"])], rel=1e-12)
    assert case.nH.min() == case.nH.max() == float(t["n_H"])
    cells = case.sources
    assert len(cells) == 2
    centres = [(c + 0.5) * g.h[0] / synth.KPC for c in cells[:, 0]]
    assert abs(centres[1] - centres[0]) == pytest.approx(float(t["separation_kpc"]), abs=g.h[0] / synth.KPC)
    rate = case.eta.max() * g.volume / synth.HNU_HI
    assert rate == pytest.approx(float(t["ndot_each"]), rel=1e-12)
    assert np.count_nonzero(case.eta) == 2
