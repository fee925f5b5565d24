"""Run a few sawtooth cycles of a seeded checkerboard problem through the C
ABI (btmg_mg_cycle), e.g. under a profiler:

    python -m paper_2301_09991_gb300.cycles --pg 0 --cycles 3
    python -m paper_2301_09991_gb300.cycles --pg 0 --scat 2 --cycles 2

Defaults: 256 x 256 nodes, 16 x 32 directions, 8 x 8 checkerboard of
sigma_t ~ logU[0.1, 10] (seed 2), c = 0.9, unit square, FP32 storage."""
import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--n-polar", type=int, default=16)
    ap.add_argument("--n-azim", type=int, default=32)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--c", type=float, default=0.9)
    ap.add_argument("--length", type=float, default=1.0)
    ap.add_argument("--pg", type=int, default=1)
    ap.add_argument("--scat", type=int, default=0, help="scat_levels: 0, 1 or 2")
    ap.add_argument("--dtype", default="f32", choices=["f64", "f32", "bf16", "f16"])
    ap.add_argument("--cycles", type=int, default=3)
    args = ap.parse_args(argv)
    import torch
    from . import btmg, inputs
    prob = inputs.checkerboard(n=args.n, n_polar=args.n_polar, n_azim=args.n_azim, blocks=8, seed=args.seed,
                               c=args.c, length=args.length)
    dt = {"f64": btmg.F64, "f32": btmg.F32, "bf16": btmg.BF16, "f16": btmg.F16}[args.dtype]
    gp = btmg.Problem(prob, dtype=dt, pg=args.pg, scat_levels=args.scat)
    psi = gp.zeros()
    rel = None
    for _ in range(args.cycles):
        rel = gp.mg_cycle(psi)
    torch.cuda.synchronize()
    print("%d cycles, relative residual of the last input %.3e" % (args.cycles, rel))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
