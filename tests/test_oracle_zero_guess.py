"""The residual after one red/black Gauss-Seidel sweep from a zero guess
(red cells, (i + j + k) even, first; black cells last) vanishes at every
black cell and equals the weighted sum of the black neighbours,
sum_f w_f z_nbr, at every red cell.  The FP32 cycle's residual kernel
computes that form instead of r - A z.  Checked in FP64 on the dense
matrices the oracle assembles (7-point operators with zero-gradient,
periodic and Dirichlet faces, random coefficients over many decades),
with the sweep written out on the matrix rows.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1306_0645_gb300 import synth


CASES = [
    ((8, 6, 4), (False, False, False), False),
    ((6, 8, 6), (True, False, True), False),
    ((8, 4, 6), (False, True, False), False),
    ((6, 6, 8), (False, False, False), True),     # Dirichlet (outflow) upper faces
]


@pytest.mark.parametrize("n,per,outflow", CASES)
def test_zero_guess_sweep_residual(n, per, outflow):
    case = synth.random_case(n, seed=31 + sum(n), periodic=per, E_decades=(-24, -12))
    grid = case.grid.outflow_upper() if outflow else case.grid
    op = oracle.assemble(grid, case.params, case.E, case.nHI, case.eta)
    A = oracle.dense_matrix(grid, op)
    nx, ny, nz = n
    cell = np.arange(nx * ny * nz)
    red = ((cell % nx) + (cell // nx) % ny + cell // (nx * ny)) % 2 == 0
    d = np.diag(A).copy()
    off = A - np.diag(d)
    # the 7-point stencil couples only cells of opposite colours
    assert not np.any(off[np.ix_(red, red)]) and not np.any(off[np.ix_(~red, ~red)])
    r = np.random.default_rng(5).standard_normal(cell.size)
    z = np.zeros_like(r)
    z[red] = r[red] / d[red]
    z[~red] = (r[~red] - off[~red] @ z) / d[~red]
    res = r - A @ z
    scale = np.abs(r).max()
    assert np.abs(res[~red]).max() <= 1e-13 * scale
    nbr_sum = -(off[red] @ z)          # sum_f w_f z_nbr (off-diagonal entries are -w_f)
    np.testing.assert_allclose(res[red], nbr_sum, rtol=1e-12, atol=1e-13 * scale)
    # and the red cells' residual is not trivially zero
    assert np.abs(res[red]).max() > 1e-3 * scale
