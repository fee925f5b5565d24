"""Variant of the hot path: the linear ConvFEM order (3x3 filters derived
from linear elements, Sec. 2.7; alpha_kabs = 2^p/16 and alpha_ksq = 2^p/2
with p = 1) with the anisotropic PG dissipation, against the oracle's order-1
operator and cycle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("checker_72x40", lambda: I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=11)),
    ("reflective_33x17", lambda: I.checkerboard(n=33, ny=17, n_polar=4, n_azim=8, blocks=3, seed=13,
                                                bc=(1, 0, 1, 1))),
    ("tiny_5x3", lambda: I.checkerboard(n=5, ny=3, n_polar=4, n_azim=8, blocks=2, seed=12)),
]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _linear(prob):
    return dict(prob, order=1)


@pytest.mark.parametrize("name,mk", CASES)
def test_linear_order_operator_fp64(name, mk):
    prob = _linear(mk())
    gp = btmg.Problem(prob, dtype=btmg.F64, pg=1)
    op = O.OracleProblem(prob, pg=1)
    psi = I.random_field(gp.shape, seed=31)
    r = gp.apply_operator(torch.tensor(psi, device="cuda")).cpu().numpy()
    assert rel(r, op.apply(psi)) < 1e-12


def test_linear_order_operator_fp32_and_cycle_fp64():
    prob = _linear(I.checkerboard(n=48, ny=40, n_polar=8, n_azim=8, blocks=4, seed=14))
    op = O.OracleProblem(prob, pg=1)
    g32 = btmg.Problem(prob, dtype=btmg.F32, pg=1)
    psi = I.random_field(g32.shape, seed=32).astype(np.float32)
    r32 = g32.apply_operator(torch.tensor(psi, device="cuda")).double().cpu().numpy()
    assert rel(r32, op.apply(psi.astype(np.float64))) < 1e-6
    g64 = btmg.Problem(prob, dtype=btmg.F64, pg=1)
    x = g64.zeros()
    ref = op.zeros()
    for _ in range(2):
        g64.mg_cycle(x, want_residual=False)
        ref, _, _ = op.mg_cycle(ref)
    assert rel(x.cpu().numpy(), ref) < 1e-10


def test_linear_order_lowp_rejected_and_bad_order():
    prob = I.checkerboard(n=24, n_polar=4, n_azim=8, blocks=2, seed=15)
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(dict(prob, order=1), dtype=btmg.BF16, pg=1)
    assert e.value.code == btmg.ERR_UNSUPPORTED
    with pytest.raises(btmg.BtmgError) as e:
        btmg.Problem(dict(prob, order=4), dtype=btmg.F32, pg=1)
    assert e.value.code == btmg.ERR_INVALID_ARG


CUBIC = [
    ("checker_40x29", lambda: I.checkerboard(n=40, ny=29, n_polar=8, n_azim=8, blocks=4, seed=16)),
    ("reflective_37x35", lambda: I.checkerboard(n=37, ny=35, n_polar=4, n_azim=8, blocks=3, seed=17,
                                                bc=(1, 0, 0, 1))),
    ("tiny_5x4", lambda: I.checkerboard(n=5, ny=4, n_polar=4, n_azim=8, blocks=2, seed=18)),
]


@pytest.mark.parametrize("name,mk", CUBIC)
def test_cubic_order_operator_and_cycle(name, mk):
    """Cubic ConvFEM (7 x 7 filters, halo 9) in the direct-pass PG kernels:
    the operator in FP64 (1e-12) and FP32, two FP64 cycles (1e-10).  FP32
    bound: the quadratic operator's 1e-6 scaled by the tap count of its
    correlations, (7 / 5)^2 ~ 2 (random fields: every term of a 49-point
    sum is of the size of psi)."""
    prob = dict(mk(), order=3)
    op = O.OracleProblem(prob, pg=1)
    g64 = btmg.Problem(prob, dtype=btmg.F64, pg=1)
    psi = I.random_field(g64.shape, seed=33)
    r64 = g64.apply_operator(torch.tensor(psi, device="cuda")).cpu().numpy()
    ref = op.apply(psi)
    assert rel(r64, ref) < 1e-12
    g32 = btmg.Problem(prob, dtype=btmg.F32, pg=1)
    r32 = g32.apply_operator(torch.tensor(psi.astype(np.float32), device="cuda")).double().cpu().numpy()
    assert rel(r32, op.apply(psi.astype(np.float32).astype(np.float64))) < 2e-6
    x = g64.zeros()
    refc = op.zeros()
    for _ in range(2):
        g64.mg_cycle(x, want_residual=False)
        refc, _, _ = op.mg_cycle(refc)
    assert rel(x.cpu().numpy(), refc) < 1e-10


def test_cubic_order_bf16_storage_operator():
    prob = dict(I.checkerboard(n=48, ny=40, n_polar=8, n_azim=8, blocks=4, seed=19), order=3)
    op = O.OracleProblem(prob, pg=1)
    gb = btmg.Problem(prob, dtype=btmg.BF16, pg=1)
    psi = torch.tensor(I.random_field(gb.shape, seed=34), dtype=torch.bfloat16, device="cuda")
    r = gb.apply_operator(psi).double().cpu().numpy()
    assert rel(r, op.apply(psi.double().cpu().numpy())) < 2e-6  # FP32 arithmetic, as above


def test_duct_streaming_qualitative():
    """The straight-duct problem of Sec. 3.1 (28 x 36 cm, a 6 x 6 cm source,
    absorbers beside it, void ducts above and below; no scattering), solved
    with the upwind fine scheme: the flux is mirror symmetric about the
    source's centre lines, and along the void duct it stays far above the
    flux at the same distance into the absorber (streaming against
    attenuation e^{-sigma d}).  Parity with the paper's plots is unpinned:
    the paper prints no numbers for this problem."""
    for dx in (0.8, 0.4):
        prob = I.duct(dx=dx, n_polar=8, n_azim=16)
        gp = btmg.Problem(prob, dtype=btmg.F64, pg=0)
        psi = gp.zeros()
        out = gp.solve(psi, rtol=1e-9, max_cycles=3000)
        assert out["status"] == btmg.OK, out
        phi = gp.scalar_flux(psi).cpu().numpy()[0]  # [ny][nx]
        assert np.all(phi >= -1e-12)
        assert rel(phi, phi[::-1, :]) < 1e-9 and rel(phi, phi[:, ::-1]) < 1e-9
        x = (np.arange(prob["nx"]) + 0.5) * dx
        y = (np.arange(prob["ny"]) + 0.5) * dx
        ic, jc = np.argmin(abs(x - 14.0)), np.argmin(abs(y - 18.0))
        for d in (4.0, 8.0):
            duct = phi[np.argmin(abs(y - (21.0 + d))), ic]
            absorber = phi[jc, np.argmin(abs(x - (17.0 + d)))]
            assert duct > 3.0 * absorber, (dx, d, duct, absorber)
