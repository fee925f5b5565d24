"""The cycle on host buffers (btmg_mg_cycle_host) against the cycle on device
buffers (btmg_mg_cycle): from the same input the same psi bit for bit and
the same residual norm (to 1e-6: with one group on the paired kernel the
copy in overlaps the residual, whose norm is then summed from the FP32
residual in another order),
on two calls in a row.  Cases: FP32 with PG and 8 direction chunks (the
paired kernel's final launch split into four direction ranges, each copied
back as it completes; with one group also the copy in split, each range's
residual launched as it arrives), one group and three groups, and the
256^2 x 512 workload; FP64 with PG and FP32 with the upwind fine scheme (one final launch,
the copy after it); page-locked and pageable host memory; in place and into
a second buffer; a cycle with the learned correction.
"""
import pytest
import torch

from paper_2301_09991_gb300 import btmg, inputs as I

pytestmark = pytest.mark.gpu

CASES = [
    ("f32_pg_72x40", lambda: I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=61), btmg.F32, 1, 8),
    ("f32_pg_3_groups", lambda: I.multigroup(n=40, n_polar=8, n_azim=16, G=3, blocks=4, seed=62), btmg.F32, 1, 8),
    ("f64_pg_40x24", lambda: I.checkerboard(n=40, ny=24, n_polar=4, n_azim=8, blocks=4, seed=63), btmg.F64, 1, 0),
    ("f32_upwind_64x32", lambda: I.checkerboard(n=64, ny=32, n_polar=4, n_azim=8, blocks=4, seed=64), btmg.F32, 0, 0),
]


@pytest.mark.parametrize("name,mk,dtype,pg,chunks", CASES)
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("inplace", [True, False])
def test_host_cycle_equals_device_cycle(name, mk, dtype, pg, chunks, pinned, inplace):
    prob = mk()
    gp = btmg.Problem(prob, dtype=dtype, pg=pg, chunks=chunks)
    psi0 = I.random_field(gp.shape, seed=65)
    d = torch.tensor(psi0, dtype=gp.torch_dtype, device="cuda")
    h = torch.tensor(psi0, dtype=gp.torch_dtype)
    if pinned:
        h = h.pin_memory()
    out = h if inplace else (torch.empty_like(h).pin_memory() if pinned else torch.empty_like(h))
    for call in range(2):
        r_dev = gp.mg_cycle(d)
        r_host = gp.mg_cycle_host(h, out)
        assert abs(r_host - r_dev) <= 1e-6 * r_dev, (call, r_host, r_dev)
        assert torch.equal(out, d.cpu()), call
        if not inplace:
            h.copy_(out)  # the next call starts from this result


def test_host_cycle_full_size():
    """256^2 nodes x 512 directions, PG on, FP32 (the benchmark's workload
    and launch configuration): two host-buffer cycles against two
    device-buffer cycles."""
    prob = I.checkerboard(n=256, n_polar=16, n_azim=32, blocks=8, seed=2)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=1)
    psi0 = I.random_field(gp.shape, seed=71).astype("float32")
    d = torch.from_numpy(psi0).cuda()
    h = torch.from_numpy(psi0).pin_memory()
    for call in range(2):
        r_dev = gp.mg_cycle(d)
        r_host = gp.mg_cycle_host(h)
        assert abs(r_host - r_dev) <= 1e-6 * r_dev, (call, r_host, r_dev)
        assert torch.equal(h, d.cpu()), call


def test_host_cycle_without_residual_completes_with_the_stream():
    """Without the residual the call returns after queueing; psi_out is
    complete once the stream is."""
    prob = I.checkerboard(n=72, ny=40, n_polar=8, n_azim=16, blocks=4, seed=66)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=1, chunks=8)
    psi0 = I.random_field(gp.shape, seed=67)
    d = torch.tensor(psi0, dtype=torch.float32, device="cuda")
    h = torch.tensor(psi0, dtype=torch.float32).pin_memory()
    gp.mg_cycle(d, want_residual=False)
    assert gp.mg_cycle_host(h, want_residual=False) is None
    torch.cuda.current_stream().synchronize()
    assert torch.equal(h, d.cpu())


def test_host_cycle_rejects_device_tensors():
    prob = I.checkerboard(n=32, ny=32, n_polar=4, n_azim=8, blocks=2, seed=68)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=1)
    with pytest.raises(ValueError):
        gp.mg_cycle_host(gp.zeros())


def test_host_cycle_with_the_learned_step():
    """A cycle with the learned correction changes psi after its final PG
    Jacobi launch, so its copy back follows the whole cycle: two problems
    with the same network, one cycled on device buffers and one on host
    buffers, agree bit for bit over three cycles (learned steps in the first
    and third)."""
    prob = I.checkerboard(n=48, ny=40, n_polar=8, n_azim=16, blocks=4, seed=69, c=0.95, length=5.0)
    net = btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=3)
    dev = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    hst = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    dev.set_learned(net, every=2)
    hst.set_learned(net, every=2)
    psi0 = I.random_field(dev.shape, seed=70)
    d = torch.tensor(psi0, dtype=torch.float32, device="cuda")
    h = torch.tensor(psi0, dtype=torch.float32).pin_memory()
    for call in range(3):
        r_dev = dev.mg_cycle(d)
        r_host = hst.mg_cycle_host(h)
        assert abs(r_host - r_dev) <= 1e-6 * r_dev, (call, r_host, r_dev)
        assert torch.equal(h, d.cpu()), call
