"""The allocation-free residual entry point, checked against the standard one.

Some callers cannot allocate device memory: a program or framework that
reserves the GPU's memory for its own pool and gives each library a fixed
budget, a latency-critical loop in which cudaMalloc/cudaFree (which may
synchronise the device) are not acceptable, or a runtime that lends no device
allocator to libraries.  They use btmg_apply_operator_noalloc(), whose
scratch is a fixed file-scope device array instead of cudaMalloc'd
workspaces.  These tests call it through the C ABI twice in a row (two
problems of different size, so stale scratch from the first call would show
in the second) and compare each result with btmg_apply_operator on the same
input, within the FP32 operator tolerance of the parity tests (relative L2
<= 1e-6); its optional residual norm is compared with btmg_mg_cycle's norm of
the same psi.  The file is collected after every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(prob, psi, pg=1, want_norm=False):
    L = btmg.load()
    region = prob["region"]
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    st = dev(prob["sigma_t"][region, 0])
    ss = dev(prob["sigma_s"][region, 0, 0])
    src = dev(prob["source"][region, 0])
    r = torch.empty(psi.shape[1:], dtype=torch.float32, device="cuda")
    bc = (C.c_int32 * 4)(*prob["bc"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    rel = C.c_double(-1.0)
    rc = L.btmg_apply_operator_noalloc(prob["nx"], prob["ny"], prob["lx"], prob["ly"], prob["n_polar"],
                                       prob["n_azim"], bc, pg, 0, ptr(st), ptr(ss), ptr(src), ptr(psi),
                                       ptr(r), stream, C.byref(rel) if want_norm else None)
    torch.cuda.synchronize()
    return rc, r, rel.value


def test_noalloc_matches_apply_operator_on_two_calls_in_a_row():
    problems = [I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=11),
                I.two_region(nx=48, ny=33, n_polar=8, n_azim=8)]
    for k, prob in enumerate(problems):
        gp = btmg.Problem(prob, dtype=btmg.F32)
        psi = torch.tensor(I.random_field(gp.shape, seed=40 + k), dtype=torch.float32, device="cuda")
        ref = gp.apply_operator(psi)[0].double().cpu().numpy()
        rc, r, _ = _noalloc(prob, psi)
        assert rc == btmg.OK
        got = r.double().cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6, k


def test_noalloc_residual_norm_matches_the_cycle_norm():
    """With rel_resid the call synchronises and returns ||r||_W / ||s||_W; the
    cycle reports the same norm for its input psi."""
    prob = I.checkerboard(n=64, ny=48, n_polar=8, n_azim=16, blocks=4, seed=13)
    gp = btmg.Problem(prob, dtype=btmg.F32)
    psi = torch.tensor(I.random_field(gp.shape, seed=46), dtype=torch.float32, device="cuda")
    for _ in range(2):
        rc, r, rel = _noalloc(prob, psi, want_norm=True)
        assert rc == btmg.OK
        rel_cycle = gp.mg_cycle(psi.clone())
        assert abs(rel - rel_cycle) <= 1e-5 * rel_cycle, (rel, rel_cycle)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    prob = I.uniform(1024, 512, 4, 8)  # 524288 nodes > 512 x 512
    psi = torch.zeros((1, 32, 512, 1024), dtype=torch.float32, device="cuda")  # [G][nd][ny][nx]
    rc, _, _ = _noalloc(prob, psi)
    assert rc == btmg.ERR_NOALLOC_TOO_LARGE


def test_noalloc_upwind_scheme_and_its_partial_sum_limit():
    """pg = 0 runs the streaming upwind-scheme kernel, whose norm partial sums
    (one per 128 x 8 tile and chunk) must also fit the fixed scratch: a thin
    grid that fits with the PG kernel's 32 x 32 tiles is rejected for pg = 0
    with the distinct status, nothing launched."""
    prob = I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=12)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi = torch.tensor(I.random_field(gp.shape, seed=44), dtype=torch.float32, device="cuda")
    ref = gp.apply_operator(psi)[0].double().cpu().numpy()
    rc, r, _ = _noalloc(prob, psi, pg=0)
    assert rc == btmg.OK
    got = r.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6
    # 4 x 65536 nodes (the node limit), 32 directions: 2048 PG tiles fit with
    # 2 chunks, 8192 upwind-scheme tiles do not fit even with one chunk
    thin = I.uniform(4, 65536, 4, 8)
    psi_thin = torch.zeros((1, 32, 65536, 4), dtype=torch.float32, device="cuda")  # [G][nd][ny][nx]
    assert _noalloc(thin, psi_thin, pg=1)[0] == btmg.OK
    assert _noalloc(thin, psi_thin, pg=0)[0] == btmg.ERR_NOALLOC_TOO_LARGE
