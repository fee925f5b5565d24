"""The kernels of a cycle are launched with programmatic dependent launch
(each waits on its predecessor inside the kernel); BTMG_PDL=0 launches them
plainly.  Both must give the same psi bit for bit: three eager cycles and
three graph cycles of an FP32 PG problem and of the upwind scheme, the
plain launches in a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2301_09991_gb300 import btmg, inputs as I
prob = I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=81)
out = []
for pg in (1, 0):
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=pg)
    psi = torch.tensor(I.random_field(gp.shape, seed=82), dtype=torch.float32, device="cuda")
    for _ in range(3):
        gp.mg_cycle(psi, want_residual=False)
    gp.solve(psi, rtol=0.0, max_cycles=3, check_every=3, history=False)
    out.append(psi.cpu().numpy())
np.save(sys.argv[2], np.stack(out))
"""


def test_plain_and_programmatic_launches_agree(tmp_path):
    path = str(tmp_path / "plain.npy")
    env = dict(os.environ, BTMG_PDL="0")
    subprocess.run([sys.executable, "-c", CHILD, ROOT, path], env=env, check=True, timeout=600)
    plain = np.load(path)
    prob = I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=81)
    for k, pg in enumerate((1, 0)):
        gp = btmg.Problem(prob, dtype=btmg.F32, pg=pg)
        psi = torch.tensor(I.random_field(gp.shape, seed=82), dtype=torch.float32, device="cuda")
        for _ in range(3):
            gp.mg_cycle(psi, want_residual=False)
        gp.solve(psi, rtol=0.0, max_cycles=3, check_every=3, history=False)
        assert np.array_equal(psi.cpu().numpy(), plain[k]), pg
