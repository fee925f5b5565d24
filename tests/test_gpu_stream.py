"""GPU parity of the finest-level streaming upwind sweep (TMA-fed warp bands,
all nu levels at once) through whole cycles of the upwind fine scheme: FP32
on grids whose rows are 16-byte multiples (the layouts the streaming kernel
takes), vacuum and reflective incoming sides in every combination, partial
bands and column groups, and nu = 1..4, against the FP64 oracle's cycles
(relative L2 <= 1e-6, the FP32 cycle tolerance of the parity tests).
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b)


def _cycles(prob, nu, cycles=3):
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, nu=nu)
    op = O.OracleProblem(prob, pg=0, nu=nu)
    psi = gp.zeros()
    ref = op.zeros()
    errs = []
    for _ in range(cycles):
        gp.mg_cycle(psi)
        ref, _, _ = op.mg_cycle(ref)
        errs.append(rel(psi.double().cpu().numpy(), ref))
    return errs


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 0, 1, 0), (0, 1, 0, 1), (1, 1, 1, 1)])
def test_stream_sweep_cycles_match_oracle_reflective_sides(bc):
    # 68 x 37: two 60-column groups (the second partial) and a partial last band
    prob = I.checkerboard(n=68, ny=37, n_polar=4, n_azim=8, blocks=4, seed=41, bc=bc)
    errs = _cycles(prob, nu=3)
    assert max(errs) < 1e-6, errs


@pytest.mark.parametrize("nu", [1, 2, 4])
def test_stream_sweep_cycles_match_oracle_sweep_counts(nu):
    prob = I.checkerboard(n=64, ny=24, n_polar=8, n_azim=8, blocks=4, seed=42, bc=(1, 0, 0, 1))
    errs = _cycles(prob, nu=nu)
    assert max(errs) < 1e-6, (nu, errs)
