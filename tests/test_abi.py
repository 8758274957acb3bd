"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fld.h declares; the binding's names match.  No GPU needed (no
compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fld.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(fld_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libfld():
    from paper_1306_0645_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fld_create", "fld_assemble", "fld_solve", "fld_step", "fld_step_batched",
                     "fld_footprint_bytes", "fld_last_error", "fld_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libfld):
    missing = [n for n in declared_functions() if not hasattr(libfld, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1306_0645_gb300 import fld
    assert set(declared_functions()) == set(fld.EXPORTS)
    for n in declared_functions():
        assert callable(getattr(fld, n))


def test_host_only_calls(libfld):
    # calls that touch no device: defaults, footprint, level shapes, errors
    from paper_1306_0645_gb300 import fld, synth
    p = fld.make_params(synth.Params())
    assert p.max_iter == 50 and p.rtol == 1e-8 and p.pre == 1 and p.post == 1
    g = synth.Grid.cube(32)
    assert fld.fld_levels(g) == [(32, 32, 32), (16, 16, 16), (8, 8, 8), (4, 4, 4)]
    fp = fld.fld_footprint_bytes(g, synth.Params())
    assert 32 ** 3 * 8 * 10 < fp < 32 ** 3 * 8 * 40
    mixed = synth.Params(precision=synth.PREC_MIXED)
    big = fld.fld_footprint_bytes(synth.Grid.cube(512), mixed)
    assert 10e9 < big < 30e9
    # invalid: odd large grid whose coarsest level exceeds the cap
    assert fld.fld_footprint_bytes(synth.Grid.cube(101), synth.Params()) == 0
    bad = synth.Params(dt=-1.0)
    assert fld.fld_footprint_bytes(g, bad) == 0
    # persistent inner solves: off by default; a mixed grid within the limit
    # holds one more buffer (its device descriptor); negative is invalid
    assert fld.fld_params_default().persistent_cells == 0
    base = fld.fld_footprint_bytes(g, mixed)
    ps = fld.fld_footprint_bytes(g, synth.Params(precision=synth.PREC_MIXED, persistent_cells=1 << 20))
    assert 0 < ps - base <= 4096
    assert fld.fld_footprint_bytes(g, synth.Params(precision=synth.PREC_MIXED, persistent_cells=1000)) == base
    assert fld.fld_footprint_bytes(g, synth.Params(persistent_cells=1 << 20)) == fp
    assert fld.fld_footprint_bytes(g, synth.Params(persistent_cells=-1)) == 0


def test_noalloc_rejects_inconsistent_faces():
    # the same boundary rule as fld_create: a periodic axis cannot have an
    # outflow upper face; refused before any device pointer is read
    from paper_1306_0645_gb300 import fld, synth
    g = fld.make_grid(synth.Grid((4, 4, 4), (1.0, 1.0, 1.0), (True, False, False)))
    g.bc_hi[0] = fld.FLD_BC_OUTFLOW
    p = ctypes.c_void_p(16)
    st = fld.lib().fld_residual_noalloc(ctypes.byref(g), p, p, p, p, p, p, None, p, None)
    assert st == fld.FLD_EINVAL
    assert "periodic" in fld.fld_last_error()


def test_bf16_coefficient_footprint(libfld):
    # fld_params.precond_bf16 (on by default): the levels whose V-cycle sweeps
    # run four cells per thread outside the persistent coarse tail (and
    # above the coarsest level) hold bfloat16 copies of wx, wy, wz and invd,
    # two bytes per cell each, in mixed contexts with red/black Gauss-Seidel,
    # one pre-sweep and separate colour sweeps; nothing otherwise
    from paper_1306_0645_gb300 import fld, synth
    g = synth.Grid((128, 64, 96), (1.0,) * 3, (False,) * 3)
    levels = fld.fld_levels(g)
    tail = synth.Params().tail_cells

    def fp(**kw):
        return fld.fld_footprint_bytes(g, synth.Params(precision=synth.PREC_MIXED, **kw))

    assert fld.fld_params_default().precond_bf16 == 1
    want = sum(4 * ((2 * nx * ny * nz + 511) // 512 * 512) for (nx, ny, nz) in levels[:-1]
               if nx % 4 == 0 and nx >= 16 and nx * ny * nz > tail)
    assert want > 0 and fp() - fp(precond_bf16=0) == want
    # no copies where the sweeps keep FP32 coefficients
    for kw in ({"pre": 2}, {"smoother": synth.SMOOTH_JACOBI}, {"fused_post": 1}, {"persistent_cells": 1 << 24},
               {"tail_cells": 1 << 24}):
        assert fp(precond_bf16=1, **kw) == fp(precond_bf16=0, **kw), kw
    assert fld.fld_footprint_bytes(g, synth.Params(precond_bf16=1)) == \
        fld.fld_footprint_bytes(g, synth.Params(precond_bf16=0))
    # an x extent that is not a multiple of 4 keeps the one-cell sweeps
    g2 = synth.Grid((130, 64, 96), (1.0,) * 3, (False,) * 3)
    assert fld.fld_footprint_bytes(g2, synth.Params(precision=synth.PREC_MIXED)) == \
        fld.fld_footprint_bytes(g2, synth.Params(precision=synth.PREC_MIXED, precond_bf16=0))
    # only 0 and 1
    assert fp(precond_bf16=2) == 0 and fp(precond_bf16=-1) == 0
