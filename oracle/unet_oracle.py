"""Plain float64 numpy reference of the learned-correction U-net.

TEST INFRASTRUCTURE ONLY (gradient and forward checks of the GPU kernels).
Same architecture and flat parameter layout as the CUDA implementation:
for every layer, weights [cout][ks][ks][cin] then biases [cout]; layer 0
has 16 input channels of which the first `in_ch` are real, layer 11 has 16
output channels of which channel 0 is the output.  Activations are NHWC.

  e1 = relu(c1(relu(c0(x))))                 H x W,    16 ch
  e2 = relu(c3(relu(c2(pool(e1)))))          H/2,      32 ch
  e3 = relu(c5(relu(c4(pool(e2)))))          H/4,      48 ch
  b  = relu(c7(relu(c6(pool(e3)))))          H/8,      64 ch
  d3 = relu(c8(cat(e3, up(b))))              H/4,      48 ch
  d2 = relu(c9(cat(e2, up(d3))))             H/2,      32 ch
  d1 = relu(c10(cat(e1, up(d2))))            H,        16 ch
  y  = c11(d1)[..., 0]                       (1x1 convolution)
Loss: mean over pixels of (y - t)^2.
"""
import numpy as np

SPEC = [  # cin, cout, ks, relu
    (16, 16, 3, 1), (16, 16, 3, 1), (16, 32, 3, 1), (32, 32, 3, 1), (32, 48, 3, 1), (48, 48, 3, 1),
    (48, 64, 3, 1), (64, 64, 3, 1), (112, 48, 3, 1), (80, 32, 3, 1), (48, 16, 3, 1), (16, 16, 1, 0),
]


def layout():
    out, off = [], 0
    for cin, cout, ks, relu in SPEC:
        nw = cout * ks * ks * cin
        out.append((off, off + nw, cin, cout, ks, relu))
        off += nw + cout
    return out, off


LAYOUT, NPARAM = layout()


def unpack(theta):
    ws = []
    for woff, boff, cin, cout, ks, relu in LAYOUT:
        w = theta[woff:boff].reshape(cout, ks, ks, cin)
        b = theta[boff:boff + cout]
        ws.append((w, b, ks, relu))
    return ws


def conv(x, w, b):
    """y[n,y,x,o] = b[o] + sum_{dy,dx,c} w[o,dy,dx,c] x[n, y+dy-p, x+dx-p, c], zero padding."""
    ks = w.shape[1]
    p = ks // 2
    n, h, wd, c = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    y = np.zeros((n, h, wd, w.shape[0])) + b
    for dy in range(ks):
        for dx in range(ks):
            y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + h, dx:dx + wd, :], w[:, dy, dx, :])
    return y


def conv_bwd(x, w, dy):
    ks = w.shape[1]
    p = ks // 2
    n, h, wd, c = x.shape
    xp = np.pad(x, ((0, 0), (p, p), (p, p), (0, 0)))
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for a in range(ks):
        for bb in range(ks):
            dw[:, a, bb, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, a:a + h, bb:bb + wd, :])
            dxp[:, a:a + h, bb:bb + wd, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, a, bb, :])
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, p:p + h, p:p + wd, :], dw, db


def pool(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool_bwd(d):
    return np.repeat(np.repeat(d, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(d):
    n, h, w, c = d.shape
    return d.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def forward(theta, x, in_ch):
    """x: [N,H,W,in_ch]; returns y [N,H,W] and the tape for backward."""
    ws = unpack(theta)
    n, h, w, _ = x.shape
    x16 = np.zeros((n, h, w, 16))
    x16[..., :in_ch] = x
    relu = lambda v: np.maximum(v, 0.0)
    t = {}
    t["x"] = x16
    t["a0"] = relu(conv(x16, *ws[0][:2]))
    t["e1"] = relu(conv(t["a0"], *ws[1][:2]))
    t["p1"] = pool(t["e1"])
    t["a2"] = relu(conv(t["p1"], *ws[2][:2]))
    t["e2"] = relu(conv(t["a2"], *ws[3][:2]))
    t["p2"] = pool(t["e2"])
    t["a4"] = relu(conv(t["p2"], *ws[4][:2]))
    t["e3"] = relu(conv(t["a4"], *ws[5][:2]))
    t["p3"] = pool(t["e3"])
    t["a6"] = relu(conv(t["p3"], *ws[6][:2]))
    t["b"] = relu(conv(t["a6"], *ws[7][:2]))
    t["c3"] = np.concatenate([t["e3"], up(t["b"])], axis=3)
    t["d3"] = relu(conv(t["c3"], *ws[8][:2]))
    t["c2"] = np.concatenate([t["e2"], up(t["d3"])], axis=3)
    t["d2"] = relu(conv(t["c2"], *ws[9][:2]))
    t["c1"] = np.concatenate([t["e1"], up(t["d2"])], axis=3)
    t["d1"] = relu(conv(t["c1"], *ws[10][:2]))
    t["out"] = conv(t["d1"], *ws[11][:2])
    return t["out"][..., 0], t


def loss_and_grad(theta, x, target, in_ch):
    """Mean squared error and its gradient with respect to theta."""
    ws = unpack(theta)
    y, t = forward(theta, x, in_ch)
    P = y.size
    loss = float(np.mean((y - target) ** 2))
    g = np.zeros_like(theta)

    def put(li, dw, db):
        woff, boff, cin, cout, ks, relu = LAYOUT[li]
        g[woff:boff] = dw.reshape(-1)
        g[boff:boff + cout] = db

    dout = np.zeros_like(t["out"])
    dout[..., 0] = 2.0 * (y - target) / P
    dd1, dw, db = conv_bwd(t["d1"], ws[11][0], dout)
    put(11, dw, db)
    dd1 = dd1 * (t["d1"] > 0)
    dc1, dw, db = conv_bwd(t["c1"], ws[10][0], dd1)
    put(10, dw, db)
    de1 = dc1[..., :16].copy()
    dd2 = up_bwd(dc1[..., 16:]) * (t["d2"] > 0)
    dc2, dw, db = conv_bwd(t["c2"], ws[9][0], dd2)
    put(9, dw, db)
    de2 = dc2[..., :32].copy()
    dd3 = up_bwd(dc2[..., 32:]) * (t["d3"] > 0)
    dc3, dw, db = conv_bwd(t["c3"], ws[8][0], dd3)
    put(8, dw, db)
    de3 = dc3[..., :48].copy()
    db_ = up_bwd(dc3[..., 48:]) * (t["b"] > 0)
    da6, dw, db = conv_bwd(t["a6"], ws[7][0], db_)
    put(7, dw, db)
    da6 = da6 * (t["a6"] > 0)
    dp3, dw, db = conv_bwd(t["p3"], ws[6][0], da6)
    put(6, dw, db)
    de3 = (de3 + pool_bwd(dp3)) * (t["e3"] > 0)
    da4, dw, db = conv_bwd(t["a4"], ws[5][0], de3)
    put(5, dw, db)
    da4 = da4 * (t["a4"] > 0)
    dp2, dw, db = conv_bwd(t["p2"], ws[4][0], da4)
    put(4, dw, db)
    de2 = (de2 + pool_bwd(dp2)) * (t["e2"] > 0)
    da2, dw, db = conv_bwd(t["a2"], ws[3][0], de2)
    put(3, dw, db)
    da2 = da2 * (t["a2"] > 0)
    dp1, dw, db = conv_bwd(t["p1"], ws[2][0], da2)
    put(2, dw, db)
    de1 = (de1 + pool_bwd(dp1)) * (t["e1"] > 0)
    da0, dw, db = conv_bwd(t["a0"], ws[1][0], de1)
    put(1, dw, db)
    da0 = da0 * (t["a0"] > 0)
    _, dw, db = conv_bwd(t["x"], ws[0][0], da0)
    put(0, dw, db)
    # padding parameters are held at zero by the GPU optimiser
    g[padding_mask(in_ch)] = 0.0
    return loss, g


def padding_mask(in_ch):
    m = np.zeros(NPARAM, dtype=bool)
    woff, boff, cin, cout, ks, relu = LAYOUT[0]
    w = m[woff:boff].reshape(cout, ks, ks, cin)
    w[..., in_ch:] = True
    woff, boff, cin, cout, ks, relu = LAYOUT[11]
    m[woff + cin:boff] = True  # output channels >= 1 (weights)
    m[boff + 1:boff + cout] = True  # and biases
    return m
