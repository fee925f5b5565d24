"""Learned correction of the space-angle multigrid: training pairs generated
by the solver, training of the U-net with the library's own GPU kernels, and
evaluation against plain multigrid.

A training pair is taken at cycle k of plain multigrid on a seeded
checkerboard problem (upwind fine scheme, FP32):
  input  = the features of the learned step for psi_k after psi_{k-1}
           (btmg_learn_features: rho / rms(rho), log optical thickness,
           scattering ratio, (phi_k - phi_{k-1}) / rms);
  target = e / rms(e), e = phi* - phi_k the scalar-flux error of psi_k
           (phi* from an FP64-refined solve of the same problem): the shape
           of the error, since the step length of the learned step sets its
           size.
The pairs are augmented by the eight symmetries of the square (the features
and the target are isotropic quantities and the cycle is D4-symmetric).

Command line (on a GPU):
  python -m paper_2301_09991_gb300.learned train --out weights.npy
  python -m paper_2301_09991_gb300.learned eval --weights weights.npy
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import btmg
from . import inputs as I

CYCLES = (1, 3, 6, 10, 20, 40, 70, 100, 140, 180)


def training_problem(seed, n=64, n_polar=8, n_azim=16, c=None, length=None):
    """Config-2-class problem reaching into the scattering-dominated regime:
    checkerboard of sigma_t ~ logU[0.1, 10] with a seeded block count (4 or 8
    per side), scattering ratio c ~ U[0.9, 0.995] and domain side
    ~ logU[1, 30] (or the given c and side)."""
    rng = np.random.default_rng(10_000 + seed)
    blocks = int(rng.choice([4, 8]))
    cc = float(rng.uniform(0.9, 0.995))
    ll = float(np.exp(rng.uniform(np.log(1.0), np.log(30.0))))
    c = cc if c is None else c
    length = ll if length is None else length
    return I.checkerboard(n=n, n_polar=n_polar, n_azim=n_azim, blocks=blocks, seed=seed, c=c, length=length)


def reference_flux(prob, rtol=1e-9):
    """Scalar flux of an FP64-refined solve (upwind fine scheme)."""
    import torch
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    out = gp.solve_refined(psi64, rtol=rtol, max_outer=400, inner_cycles=8)
    # phi = sum_n p_n psi_n of the FP64 solution by the library's kernel
    # (an FP64 problem, whose storage type is the solution's)
    phi = btmg.Problem(prob, dtype=btmg.F64, pg=0).scalar_flux(psi64)
    return phi, out["rel_resid"]


def pairs_for_problem(prob, cycles=CYCLES, min_rel=1e-4):
    """Features and targets [m][H8][W8][4], [m][H8][W8] (torch, CUDA); an
    iterate whose relative residual is below min_rel gives no pair (its
    error is mostly FP32 rounding)."""
    import torch
    phi_star, _ = reference_flux(prob)
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi = gp.zeros()
    X, Y = [], []
    _, _, f = gp.learn_canvas()
    prev = None
    for k in range(max(cycles) + 1):
        if k in cycles:
            feat, _ = gp.learn_features(psi, prev)
            err = coarse_mean((phi_star - gp.scalar_flux(psi).double())[0], f)
            err = err / max(float(torch.sqrt(torch.mean(err * err))), 1e-300)
            tgt = torch.zeros(feat.shape[1:3], dtype=torch.float32, device="cuda")
            tgt[:err.shape[0], :err.shape[1]] = err.float()
            X.append(feat[0].clone())
            Y.append(tgt)
        if k + 1 in cycles:
            prev = psi.clone()
        rel = gp.mg_cycle(psi)
        if k in cycles and rel < min_rel:
            X.pop()
            Y.pop()
            break
    return torch.stack(X) if X else None, torch.stack(Y) if Y else None


def coarse_mean(img, f):
    """Means of img [ny][nx] over f x f blocks (cut at the edge), the
    averaging of the learned correction's coarse canvas."""
    import torch
    if f == 1:
        return img
    ny, nx = img.shape
    cy, cx = -(-ny // f), -(-nx // f)
    pad = torch.zeros((cy * f, cx * f), dtype=img.dtype, device=img.device)
    cnt = torch.zeros_like(pad)
    pad[:ny, :nx] = img
    cnt[:ny, :nx] = 1.0
    s = pad.reshape(cy, f, cx, f).sum(dim=(1, 3))
    return s / cnt.reshape(cy, f, cx, f).sum(dim=(1, 3))


def d4(X, Y):
    """The eight symmetries of the square applied to images [m][H][W](...)."""
    import torch
    xs, ys = [], []
    for flip in (False, True):
        x0 = torch.flip(X, dims=[2]) if flip else X
        y0 = torch.flip(Y, dims=[2]) if flip else Y
        for r in range(4):
            xs.append(torch.rot90(x0, r, dims=[1, 2]))
            ys.append(torch.rot90(y0, r, dims=[1, 2]))
    return torch.cat(xs), torch.cat(ys)


def make_dataset(plan, n_polar=8, n_azim=16, augment=True, log=None):
    """plan: [(seed, n)]; all canvases are 64 x 64 for n in {64, 128, 256}."""
    import torch
    Xs, Ys = [], []
    t0 = time.time()
    for i, (s, n) in enumerate(plan):
        X, Y = pairs_for_problem(training_problem(s, n, n_polar, n_azim))
        if X is None:
            continue
        Xs.append(X)
        Ys.append(Y)
        if log and (i + 1) % 50 == 0:
            log("pairs from %d problems (%.0f s)" % (i + 1, time.time() - t0))
    X, Y = torch.cat(Xs), torch.cat(Ys)
    if augment:
        X, Y = d4(X, Y)
    return X.contiguous(), Y.contiguous()


def train(net, X, Y, steps=2000, batch=32, lr=1e-3, lr_min=1e-4, seed=0, log=None):
    """Adam on the mean squared error, cosine learning-rate decay."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    m = X.shape[0]
    hist = []
    for it in range(steps):
        idx = torch.randint(0, m, (batch,), generator=g).cuda()
        a = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * it / steps))
        want = (it % 100 == 0) or it == steps - 1
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), a, want_loss=want)
        if want:
            hist.append((it, loss))
            if log:
                log("step %d loss %.4e" % (it, loss))
    return hist


def solve_cycles(prob, net=None, rtol=1e-5, max_cycles=2000, dtype=btmg.F32, every=1):
    """Cycles and seconds of btmg_solve (upwind fine scheme) to rtol."""
    import torch
    gp = btmg.Problem(prob, dtype=dtype, pg=0)
    if net is not None:
        gp.set_learned(net, every=every)
    psi = gp.zeros()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = gp.solve(psi, rtol=rtol, max_cycles=max_cycles)
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    out["learn_stats"] = gp.learn_stats() if net is not None else (0, 0.0, 0.0, 0)
    return out, psi


def refined_cycles(prob, net=None, rtol=1e-6, inner=4, dtype=btmg.F32, max_outer=400, every=1):
    """FP64-refined solve to rtol: inner cycles and seconds."""
    import torch
    gp = btmg.Problem(prob, dtype=dtype, pg=0)
    if net is not None:
        gp.set_learned(net, every=every)
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = gp.solve_refined(psi64, rtol=rtol, max_outer=max_outer, inner_cycles=inner)
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    out["learn_stats"] = gp.learn_stats() if net is not None else (0, 0.0, 0.0, 0)
    return out, psi64


def load_net(path):
    net = btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=1)
    net.set_params(np.load(path))
    return net


# multiply-adds per canvas pixel of one U-net forward: the 3x3 convolutions
# cin x cout at full (1), 1/4, 1/16 and 1/64 of the pixels (encoder 16-16,
# 16-32 | 32-32, 32-48 | 48-48, 48-64 | 64-64; decoder 112-48 at 1/16, 80-32
# at 1/4, 48-16 at 1) and the 1x1 output layer 16-16
UNET_MACS_PER_PIXEL = (9 * (16 * 16 + 16 * 16) + 9 * (16 * 32 + 32 * 32) // 4 + 9 * (32 * 48 + 48 * 48) // 16
                       + 9 * (48 * 64 + 64 * 64) // 64 + 9 * 112 * 48 // 16 + 9 * 80 * 32 // 4 + 9 * 48 * 16
                       + 16 * 16)


def forward_timing(net, reps=20):
    """CUDA-event time of U-net forwards (BF16 tensor-core convolutions) for
    the learned step's canvas (one 64 x 64 image) and for batches of 32
    images of 64 x 64 and 256 x 256, with the achieved tensor rate."""
    import torch
    out = []
    for n, hw in ((1, 64), (32, 64), (32, 256)):
        x = torch.randn((n, hw, hw, btmg.LEARN_FEATURES), dtype=torch.float32, device="cuda")
        net.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.forward(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        flops = 2.0 * UNET_MACS_PER_PIXEL * n * hw * hw
        out.append(dict(images=n, canvas=hw, ms=round(ms, 4), gflop=round(flops / 1e9, 3),
                        tflops=round(flops / ms / 1e9, 2)))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval", "timing"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default="learned_unet.npy")
    ap.add_argument("--weights", default=None)
    ap.add_argument("--mix", default="64:200,128:60,256:30",
                    help="grid size:problem count, comma separated (seeds from 1000 on)")
    ap.add_argument("--steps", type=int, default=4000)
    args = ap.parse_args()
    log = lambda m: print(m, flush=True)
    if args.cmd == "timing":
        net = load_net(args.weights) if args.weights else btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=1)
        for row in forward_timing(net, args.reps):
            print(json.dumps(row), flush=True)
    elif args.cmd == "train":
        t0 = time.time()
        plan, seed = [], 1000
        for item in args.mix.split(","):
            n, count = (int(v) for v in item.split(":"))
            plan += [(seed + i, n) for i in range(count)]
            seed += count
        X, Y = make_dataset(plan, log=log)
        log("dataset: %d pairs of %s (%.0f s)" % (X.shape[0], tuple(X.shape[1:]), time.time() - t0))
        net = btmg.UNet(in_channels=btmg.LEARN_FEATURES, seed=1)
        t1 = time.time()
        hist = train(net, X, Y, steps=args.steps, log=log)
        log("training: %d steps in %.0f s" % (args.steps, time.time() - t1))
        np.save(args.out, net.get_params())
        print(json.dumps({"pairs": int(X.shape[0]), "loss_first": hist[0][1], "loss_last": hist[-1][1]}))
    else:
        import torch
        net = load_net(args.weights)
        cases = (("solve", 5001, 64, 8, 16, 0.99, 30.0), ("solve", 5003, 128, 8, 16, 0.99, 30.0),
                 ("solve", 5002, 128, 8, 16, 0.98, 20.0), ("refined", 5010, 256, 16, 32, 0.99, 30.0),
                 ("refined", 5011, 256, 16, 32, 0.95, 3.0), ("refined", 5012, 512, 32, 32, 0.99, 30.0),
                 ("refined", 5000, 512, 32, 32, 0.9, 1.0))
        for mode, s, n, npol, naz, c, L in cases:
            prob = training_problem(s, n=n, n_polar=npol, n_azim=naz, c=c, length=L)
            if mode == "solve":
                f = lambda nt, ev: solve_cycles(prob, nt, rtol=1e-5, max_cycles=3000, every=ev)
            else:
                f = lambda nt, ev: refined_cycles(prob, nt, rtol=1e-6, inner=8, every=ev, max_outer=400)
            f(None, 1)  # warm-up
            plain, p0 = f(None, 1)
            row = dict(case="%s n%d %dx%d c%.3f L%g" % (mode, n, npol, naz, c, L),
                       plain=dict(cycles=plain["cycles"], s=round(plain["seconds"], 4), rel=plain["rel_resid"]))
            for every in (2, 4):
                f(net, every)
                lr, p1 = f(net, every)
                st = lr["learn_stats"]
                row["every%d" % every] = dict(cycles=lr["cycles"], s=round(lr["seconds"], 4), rel=lr["rel_resid"],
                                              steps=st[0], factor=round(st[1], 4), fallbacks=st[3],
                                              diff=float(torch.linalg.norm(p1 - p0) / torch.linalg.norm(p0)))
            print(json.dumps(row), flush=True)

if __name__ == "__main__":
    main()
