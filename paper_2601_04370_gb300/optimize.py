"""Thickness optimization of a synthetic design (Results, "Evaluation"):

  python -m paper_2601_04370_gb300.optimize --design representative --rays 1000000 --iters 300 [--omega-iters 60]

--design expander optimizes the two-dimensional pupil expander (30 fold + 16
output mirrors with 23-layer stacks: 1058 thicknesses, the scale of the
paper's design) instead of the six-mirror array (--layers does not apply).

With --omega-iters, the reflection probabilities are pre-optimized first
(Methods, "Learned reflection probabilities": scalar-reflectance geometric
model, throughput to the pupils). Starts from thicknesses drawn from a
Gaussian at the midpoint of the 20-200 nm bounds, then iterates forward
trace, loss (Eq. 1), adjoint and the projected
Adam step (layers can be eliminated through the soft gap 0-20 nm). Prints the
loss terms every `--every` iterations and, at the end, the eyebox throughput,
the CVs and how many layers were driven to zero thickness. The Philox keys
are fixed, so the objective is a deterministic function of the thicknesses.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--design", choices=("tiny", "representative", "expander"), default="representative")
    ap.add_argument("--rays", type=int, default=1_000_000)
    ap.add_argument("--layers", type=int, default=40)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--lr", type=float, default=2.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--omega-iters", type=int, default=0)
    ap.add_argument("--omega-lr", type=float, default=0.03)
    args = ap.parse_args(argv)
    import numpy as np

    from . import wg
    from . import workloads as W

    if args.design == "tiny":
        D, C = W.tiny(n_rays=args.rays)
    elif args.design == "expander":
        D, C = W.pupil_expander(n_rays=args.rays)
    else:
        D, C = W.representative(n_rays=args.rays, n_layers=args.layers)
    D = W.with_thickness(D, W.gaussian_thickness(D, seed=args.seed))
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    omega = None
    if args.omega_iters > 0:
        oh, om = wg.optimize_omega(ctx, dh, C, args.omega_iters, lr=args.omega_lr)
        omega = {"I_mean_start": float(oh[0]), "I_mean_end": float(oh[-1]), "omega": [float(x) for x in om]}
        print(json.dumps({"omega_preopt": omega}), flush=True)
    adam = wg.Adam(dh, lr_nm=args.lr)

    def report(it, h, a):
        if it % args.every == 0 or it == args.iters - 1:
            print(json.dumps({"iter": it, "loss": h[0], "I_mean": h[1], "cv_fov": h[2], "cv_eyebox": h[3]}), flush=True)

    t0 = time.perf_counter()
    hist, adam = wg.optimize(ctx, dh, C, args.iters, adam=adam, callback=report)
    wall = time.perf_counter() - t0
    th = adam.params()
    live = np.asarray(D.pruned) == 0
    out = {"design": args.design, "rays": args.rays, "iters": args.iters, "wall_s": wall, "omega_preopt": omega,
           "start": dict(zip(("loss", "I_mean", "cv_fov", "cv_eyebox"), map(float, hist[0]))),
           "end": dict(zip(("loss", "I_mean", "cv_fov", "cv_eyebox"), map(float, hist[-1]))),
           "layers": int(live.sum()), "driven_to_zero": int(((th == 0.0) & live).sum()),
           "at_bounds": {"20nm": int(((th == 20.0) & live).sum()), "200nm": int(((th == 200.0) & live).sum())}}
    print(json.dumps(out), flush=True)
    adam.close()
    dh.destroy()
    ctx.close()


if __name__ == "__main__":
    main()
