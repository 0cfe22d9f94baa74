"""Fixed workloads for profiling the trace kernels (e.g. under ncu):

  python -m paper_2601_04370_gb300.profile_case --rays 4000000 --layers 40 [--backward [--tilt]] [--repeat 3]
  python -m paper_2601_04370_gb300.profile_case --design expander --rays 1000000 [--backward [--tilt]]

Runs `repeat` forward traces of the representative design (3D slab, 6
mirrors, `layers` SiO2/TiO2/Ta2O5 layers each, 460/532/630 nm, 32x18 fields,
random linear polarization) with `rays` rays, then optionally the loss (Eq. 1)
and one adjoint pass (with --tilt also the mirror-tilt gradient, as the bench
step), and prints the work counters of each call. Kernel order per forward:
k_prep_fields, k_trace_fwd; backward: k_prep_fields, then per batch
k_bwd_replay, k_bwd_scan, k_bwd_scatter, k_bwd_adjoint (and k_tilt_grad with
--tilt); k_scatter_grad. --design expander traces the two-dimensional pupil
expander (46 general mirrors, 23 layers; --layers does not apply).
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--rays", type=int, default=4_000_000)
    ap.add_argument("--layers", type=int, default=40)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--backward", action="store_true")
    ap.add_argument("--tilt", action="store_true")
    ap.add_argument("--design", choices=("representative", "expander"), default="representative")
    args = ap.parse_args(argv)
    import torch

    from . import wg
    from . import workloads as W

    ctx = wg.Context(0)
    if args.design == "expander":
        D, C = W.pupil_expander(n_rays=args.rays)
    else:
        D, C = W.representative(n_rays=args.rays, n_layers=args.layers)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    keys = ("n_rays", "n_hits", "n_events", "n_layer_steps", "kernel_ms")
    for _ in range(args.repeat):
        st = ctx.trace_forward(dh, C, tally)
    print("forward", {k: st[k] for k in keys})
    if args.backward:
        G = torch.zeros_like(tally)
        ctx.loss(dh, C, tally, G)
        g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
        gt = torch.zeros(len(D.mirror_x_mm), dtype=torch.float64, device="cuda") if args.tilt else None
        sb = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
        print("backward", {k: sb[k] for k in ("n_rays", "n_hits", "n_tallied", "n_adjoint_steps", "kernel_ms")})
    torch.cuda.synchronize()
    dh.destroy()
    ctx.close()


if __name__ == "__main__":
    main()
