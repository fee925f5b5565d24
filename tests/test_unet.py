"""Learned-correction U-net: the float64 numpy reference is pinned by finite
differences (CPU); the GPU BF16 kernels are checked against it (GPU)."""
import numpy as np
import pytest

import unet_oracle as UO


def _theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    th = np.zeros(UO.NPARAM)
    for woff, boff, cin, cout, ks, relu in UO.LAYOUT:
        th[woff:boff] = rng.standard_normal(boff - woff) * np.sqrt(2.0 / (ks * ks * cin)) * scale
        th[boff:boff + cout] = 0.05 * rng.standard_normal(cout)
    th[UO.padding_mask(3)] = 0.0
    return th


def test_unet_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = _theta(1)
    x = rng.standard_normal((1, 16, 16, 3))
    t = rng.standard_normal((1, 16, 16))
    loss, g = UO.loss_and_grad(th, x, t, 3)
    free = np.flatnonzero(~UO.padding_mask(3))
    # one weight from every layer plus random picks
    picks = [UO.LAYOUT[l][0] + 3 for l in range(12)] + list(rng.choice(free, 12, replace=False))
    h = 1e-6
    for i in picks:
        e = np.zeros_like(th)
        e[i] = h
        fd = (UO.loss_and_grad(th + e, x, t, 3)[0] - UO.loss_and_grad(th - e, x, t, 3)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_unet_reference_shapes_and_param_count():
    assert UO.NPARAM == sum(co * ks * ks * ci + co for ci, co, ks, r in UO.SPEC)
    y, _ = UO.forward(_theta(2), np.zeros((2, 8, 8, 3)), 3)
    assert y.shape == (2, 8, 8)


@pytest.mark.gpu
def test_unet_gpu_forward_and_gradients_match_reference():
    import torch
    from paper_2301_09991_gb300 import btmg
    net = btmg.UNet(in_channels=3, seed=5)
    th = _theta(3).astype(np.float32)
    net.set_params(th)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 32, 32, 3)).astype(np.float32)
    t = rng.standard_normal((2, 32, 32)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    y = net.forward(xd).cpu().numpy()
    y_ref, _ = UO.forward(th.astype(np.float64), x.astype(np.float64), 3)
    ferr = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    loss = net.train_step(xd, torch.tensor(t, device="cuda"), lr=0.0)
    g = net.get_grads().astype(np.float64)
    loss_ref, g_ref = UO.loss_and_grad(th.astype(np.float64), x.astype(np.float64), t.astype(np.float64), 3)
    gerr = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print("BF16 U-net vs float64 reference: forward %.2e, loss %.4f vs %.4f, gradient %.2e"
          % (ferr, loss, loss_ref, gerr))
    assert ferr < 3e-2 and abs(loss - loss_ref) < 3e-2 * loss_ref and gerr < 5e-2
    # per layer, weight gradients point the same way
    for woff, boff, cin, cout, ks, relu in UO.LAYOUT:
        a, b = g[woff:boff], g_ref[woff:boff]
        assert np.dot(a, b) > 0.95 * np.linalg.norm(a) * np.linalg.norm(b)


@pytest.mark.gpu
def test_unet_gpu_training_reduces_loss():
    import torch
    from paper_2301_09991_gb300 import btmg
    net = btmg.UNet(in_channels=3, seed=7)
    rng = np.random.default_rng(8)
    x = torch.tensor(rng.standard_normal((8, 32, 32, 3)).astype(np.float32), device="cuda")
    # target: a smooth linear functional of the input (a blurred first channel)
    k = torch.ones(1, 1, 5, 5, device="cuda") / 25.0
    t = torch.nn.functional.conv2d(x[..., 0].unsqueeze(1), k, padding=2).squeeze(1).contiguous()
    l0 = net.train_step(x, t, lr=0.0)
    for _ in range(150):
        net.train_step(x, t, lr=2e-3, want_loss=False)
    l1 = net.train_step(x, t, lr=0.0)
    print("training loss %.4e -> %.4e" % (l0, l1))
    assert l1 < 0.2 * l0
