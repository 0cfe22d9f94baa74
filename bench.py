#!/usr/bin/env python3
"""Benchmark of the hot path: one step = forward Monte Carlo polarization trace
of the representative waveguide (3D slab n=1.71, 1.5 mm, 6 PRMA mirrors x 40
SiO2/TiO2/Ta2O5 layers, 460/532/630 nm, 32x18 fields over 30x17 deg, random
linear polarization, 1e7 rays, 64x48 eyebox bins) + loss (Eq. 1) + adjoint
with respect to the 240 layer thicknesses. Metric: ray-mirror interactions/s
(forward interactions per step / step time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank traces its own 1e7 rays (seed offset by rank, no
data-path collective: weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-mirror interactions/s fwd & fwd+bwd at <=1e-4 rel err; p50/p99 eval latency"
UNIT = "interactions/s"
# Algorithmic FP32 work per ray-mirror interaction (an FMA counts 2 flops):
# 33 flops per non-pruned layer of the hit's stack (phase, range reduction and
# the s and p 2x2 chain) plus 250 per hit for the coefficients, bases, Jones
# update and geometry. The thin-film adjoint costs about three forward layer
# chains per layer of each record (forward sweep, recomputation, reverse
# sweep with the layer gradients); with the mirror-tilt gradient the reverse
# sweep also forms d/d(cos theta_0) of each record: per layer the row's two
# products with the next substrate-side vector for each polarization and the
# rho-weighted sums, 29 flops.
FLOPS_PER_LAYER = 33
FLOPS_PER_HIT = 250
FLOPS_ADJ_LAYER = 3 * FLOPS_PER_LAYER
FLOPS_ADJ_LAYER_TILT = 3 * FLOPS_PER_LAYER + 29
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count, sm_mhz):
    """FP32 FMA-pipe peak: SMs x 128 lanes x 2 flops x SM clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def src_hash():
    """Hash of the sources that define the profiled kernels (device code and
    their argument layout)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2601_04370_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel):
    """DRAM bytes per launch from profiles/traffic.json if it was taken on the
    current kernel sources, else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            t = json.load(f)
        e = t.get(kernel)
        if e and e.get("src_hash") == src_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


class Clocks:
    """nvidia-smi sampling (every 50 ms, timestamped) around the timed region;
    start() returns once samples are being written, and the summary counts
    the samples that fall inside the window given to stop()."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.mkdtemp(prefix="wg_clocks_"), f"clocks_rank{device}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self, window=None):
        """window: (t0, t1) host times (time.time()) of the timed region."""
        if not self.proc:
            return None
        time.sleep(0.1)  # a sample after the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        import datetime
        rows = []
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(v[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append(dict(ts=ts, sm=float(v[2]), smax=float(v[3]), power=float(v[4]), hw=v[6], hwt=v[7],
                                 swt=v[8], swp=v[9]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = rows
        if window is not None:
            w = [r for r in rows if r["ts"] is not None and window[0] - 0.06 <= r["ts"] <= window[1] + 0.06]
            inside = w or rows
        smax = max(r["smax"] for r in rows)
        load = [r for r in inside if r["power"] > 200.0] or inside
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("swp", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in inside):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "samples_in_timed_region": len(inside), "samples_under_load": len(load),
                "interval_ms": 50}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg, device=None):
    if pg is not None:
        if device is not None:
            pg.barrier(device_ids=[device])
        else:
            pg.barrier()


def allmax(pg, x, device=None):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=("cuda" if device is not None else "cpu"))
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allsum(pg, x, device=None):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=("cuda" if device is not None else "cpu"))
    pg.all_reduce(t)
    return float(t.item())


def workload(rank, n_rays=None):
    from paper_2601_04370_gb300 import workloads as W
    D, C = W.representative() if n_rays is None else W.representative(n_rays=n_rays)
    return D, C.replace(seed=C.seed + 1000003 * rank)


WORKLOAD_NAME = ("representative fwd+loss+adjoint: 3D slab n=1.71 t=1.5mm, 6 PRMA mirrors x 40 layers "
                 "(SiO2/TiO2/Ta2O5, d~U[10,200] nm), 460/532/630 nm, 32x18 fields over 30x17 deg, "
                 "random linear pol, 1e7 rays per GPU, 64x48 eyebox bins, max 100 events")


def cpu_oracle_rate(D, C, G, budget_s=12.0, max_rays=None, sample=None):
    """Oracle (FP64 CPU) forward + adjoint on a bounded sample of the same
    workload: the first k rays of each of m cells spread evenly over the
    grid, k grown to a whole cell and then m, until the sample takes about
    the budget (small samples are dominated by per-call thread start-up).
    sample=(k, m) reuses a calibrated sample size. Returns (record, hits,
    seconds, (k, m))."""
    from oracle import oracle as O
    nthreads = O.hardware_threads()

    def cells_of(m):
        return list(range(0, C.n_cells, max(1, C.n_cells // m)))[:m]

    def run(k, cells):
        hits = 0
        t0 = time.perf_counter()
        for cell in cells:
            r0 = cell * C.n_cell
            o = O.trace(D, C, rays=(r0, r0 + k), nthreads=nthreads)
            hits += o["stats"]["n_hits"]
            O.trace_grad(D, C, G, rays=(r0, r0 + k), nthreads=nthreads)
        return hits, time.perf_counter() - t0

    if sample is not None:
        k, m = sample
        h, t = run(k, cells_of(m))
        return dict(value=h / t, unit=UNIT, cores=nthreads, kind="oracle",
                    sample=f"{k * m} rays ({k} per cell from {m} of {C.n_cells} cells), "
                           f"FP64 forward + adjoint, {t:.1f} s wall on {nthreads} host threads"), h, t, (k, m)
    m = min(64, C.n_cells)
    run(2, cells_of(m))  # one-time costs (library load, host threads) stay out of the calibration
    k = 8
    h, t = run(k, cells_of(m))
    limit = max_rays if max_rays else 1 << 62
    while t < 0.5 * budget_s and k * m < limit:
        grow = max(2.0, budget_s / max(t, 1e-3))
        if k < C.n_cell:
            k = int(min(C.n_cell, k * grow, max(1, limit // m)))
        elif m < C.n_cells:
            m = int(min(C.n_cells, m * grow, max(1, limit // k)))
        else:
            break
        h, t = run(k, cells_of(m))
    return dict(value=h / t, unit=UNIT, cores=nthreads, kind="oracle",
                sample=f"{k * m} rays ({k} per cell from {m} of {C.n_cells} cells), "
                       f"FP64 forward + adjoint, {t:.1f} s wall on {nthreads} host threads"), h, t, (k, m)


def run_child(argv, timeout):
    """One measurement in its own process (its own contexts; a failure there
    is reported in the line, not fatal to the bench)."""
    cmd = [sys.executable, "-X", "faulthandler", os.path.abspath(__file__), *argv]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout} s"}
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    if r.returncode == 0 and lines:
        return json.loads(lines[-1])
    return {"error": f"exit {r.returncode}", "stderr_tail": r.stderr[-1500:]}


def run_batching(dev, rounds):
    """The batching configuration: the 64 designs of the batching pool (K
    3..8, L 10..200 with 30% of layers pruned, 1e5..1e7 rays) traced by
    wg_trace_forward_batch, once as one batch (one fused launch per kernel
    variant and launch-shape group, graph-replayed from the third round) and
    once one design per call (each its own launch, also graph-replayed); three
    untimed rounds first (autotuning, capture), then `rounds` timed ones."""
    import numpy as np
    import torch
    from paper_2601_04370_gb300 import wg
    from paper_2601_04370_gb300 import workloads as W
    pool = W.batching(n_designs=64, seed=4)
    ctx = wg.Context(dev)
    dhs = [ctx.create_design(D) for D, _ in pool]
    cfgs = [C for _, C in pool]
    ts = [torch.zeros(C.tally_shape, dtype=torch.float64, device=f"cuda:{dev}") for C in cfgs]

    def longest_stack(D):
        kept = np.split(1 - D.pruned.astype(np.int64), np.cumsum(D.n_layers)[:-1])
        return max(int(k.sum()) for k in kept)
    n_acc = sum(1 for D, _ in pool if longest_stack(D) > 48)

    def batched():
        st, rep = ctx.trace_forward_batch(dhs, cfgs, ts)
        return sum(s["n_hits"] for s in st), rep

    def single():
        hits, rep = 0, True
        for dh, C, t in zip(dhs, cfgs, ts):
            st, r = ctx.trace_forward_batch([dh], [C], [t])
            hits += st[0]["n_hits"]
            rep = rep and r
        return hits, rep

    out = {"designs": len(pool), "rays": int(sum(C.total_rays for C in cfgs)),
           "designs_accurate_mode": n_acc}
    for name, fn in (("batched", batched), ("one_design_per_launch", single)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        n0 = wg.kernel_launches()
        t0 = time.perf_counter()
        hits, reps = 0, []
        for _ in range(rounds):
            h, rep = fn()
            hits += h
            reps.append(rep)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[name] = {"interactions_per_s": hits / wall, "ms_per_round": 1e3 * wall / rounds,
                     "interactions_per_round": hits // rounds, "graph_replayed": all(reps),
                     "kernel_launches_per_round": (wg.kernel_launches() - n0) / rounds}
    out["speedup"] = out["batched"]["interactions_per_s"] / out["one_design_per_launch"]["interactions_per_s"]
    for dh in dhs:
        dh.destroy()
    ctx.close()
    return out


def bench_differentiation(ctx, dev, args, pg, ws, rank, flush, stream, pk, pk_kind):
    """fwd + loss + bwd (thickness and tilt gradients) of the differentiation
    configuration at 1e8 rays, timed with CUDA events; rooflines of the forward
    and of the thin-film adjoint (accurate mode) in the same units as the
    headline; the oracle's forward + adjoint on a sample of at most 1e5 rays."""
    import torch
    from paper_2601_04370_gb300 import wg
    from paper_2601_04370_gb300 import workloads as W
    D, C = W.differentiation()
    C = C.replace(seed=C.seed + 1000003 * rank)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device=f"cuda:{dev}")
    G = torch.zeros_like(tally)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device=f"cuda:{dev}")
    gt = torch.zeros(D.n_mirrors, dtype=torch.float64, device=f"cuda:{dev}")
    st_f = ctx.trace_forward(dh, C, tally)
    ctx.loss(dh, C, tally, G)
    st_b = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    hits = st_f["n_hits"]
    ms, fm, bm, adj = [], [], [], []
    for i in range(1 + args.d_steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        flush.zero_()
        ev[0].record(stream)
        ctx.trace_forward(dh, C, tally, stats=False)
        ev[1].record(stream)
        ctx.loss(dh, C, tally, G)
        ev[2].record(stream)
        sb = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
        ev[3].record(stream)
        ev[3].synchronize()
        if i >= 1:
            ms.append(ev[0].elapsed_time(ev[3]))
            fm.append(ev[0].elapsed_time(ev[1]))
            bm.append(ev[2].elapsed_time(ev[3]))
            adj.append(sb)
    t = allmax(pg, sum(ms) / 1e3, dev)
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp32_peak_tflops(sm, float(pk.get("sm_max_mhz", 2070.0)))
    f_fwd = FLOPS_PER_LAYER * st_f["n_layer_steps"] + FLOPS_PER_HIT * hits
    ach_f = f_fwd / (statistics.mean(fm) / 1e3) / 1e12
    n_adj = sum(s["n_adjoint_launches"] for s in adj)
    adj_ms = sum(s["adjoint_ms"] for s in adj)
    adj_steps = sum(s["n_adjoint_steps"] for s in adj)
    f_adj = FLOPS_ADJ_LAYER_TILT * adj_steps / max(1, n_adj)
    ach_a = f_adj / (adj_ms / max(1, n_adj) / 1e3) / 1e12 if adj_ms > 0 else 0.0
    peak_source = f"derived: {sm} SMs x 128 FP32 lanes x 2 flop x {float(pk.get('sm_max_mhz', 2070.0)):.0f} MHz ({pk_kind})"
    step_ms = 1e3 * t / len(ms)
    adj_step_ms = adj_ms / max(1, len(adj))
    out = {"workload": "differentiation fwd+loss+adjoint: as representative with 6 mirrors x 200 layers (1200 "
                       "thicknesses) + 6 tilts, 1e8 rays per GPU, accurate layer evaluation",
           "value": allsum(pg, hits * len(ms), dev) / t, "unit": UNIT, "steps": len(ms), "warmup": 1,
           "ms_per_step": 1e3 * t / len(ms), "fwd_ms": statistics.mean(fm), "bwd_ms": statistics.mean(bm),
           "fwd_interactions_per_s": hits / (statistics.mean(fm) / 1e3), "interactions_per_step": hits,
           "rays": C.total_rays, "layer_steps_per_hit": st_f["n_layer_steps"] / max(1, hits),
           "overflow": st_b["overflow"], "nonfinite": st_b["n_nonfinite"],
           "roofline": {"bound": "alu", "kernel": "k_bwd_adjoint (tilt variant, accurate mode)", "achieved": ach_a,
                        "peak": peak, "unit": "TFLOP/s", "frac": ach_a / peak, "traffic": None,
                        "flops_per_launch": f_adj, "launch_ms": adj_ms / max(1, n_adj), "launches": n_adj,
                        "units": f"{adj_steps / max(1, n_adj):.4g} record layer steps per launch x "
                                 f"{FLOPS_ADJ_LAYER_TILT} flops", "peak_source": peak_source,
                        "ms_per_step": adj_step_ms, "share_of_step": adj_step_ms / step_ms},
           "roofline_fwd": {"bound": "alu", "kernel": "k_trace_fwd (accurate mode)", "achieved": ach_f, "peak": peak,
                            "unit": "TFLOP/s", "frac": ach_f / peak, "flops_per_launch": f_fwd,
                            "ms_per_step": statistics.mean(fm), "share_of_step": statistics.mean(fm) / step_ms,
                            "units": f"{hits} interactions x ({FLOPS_PER_LAYER} x "
                                     f"{st_f['n_layer_steps'] / max(1, hits):.1f} layers + {FLOPS_PER_HIT}) flops",
                            "peak_source": peak_source}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], _, _, _ = cpu_oracle_rate(D, C, G.cpu().numpy(), budget_s=max(2.0, args.cpu_budget / 2),
                                                       max_rays=100_000)
    dh.destroy()
    return out


def run_serving(dev, n_requests, max_slots, cache_path, rate_hz=200.0):
    """The serving trace (Poisson arrivals at rate_hz, designs drawn from the
    64-design batching pool and kept resident, 5% loss+gradient requests at
    1e6..1e8 rays) submitted at its arrival times through wg_submit; latency
    of a request = submit -> completion as the runtime measures it."""
    import numpy as np
    from paper_2601_04370_gb300 import wg
    from paper_2601_04370_gb300 import workloads as W
    reqs = W.serving_trace(n_requests=n_requests, rate_hz=rate_hz)
    ctx = wg.Context(dev, max_slots=max_slots, autotune_cache=cache_path)
    handles = {}
    for r in reqs:
        if id(r["design"]) not in handles:
            handles[id(r["design"])] = ctx.create_design(r["design"])

    def run(subset):
        keep, tickets = [], []
        t0 = time.perf_counter()
        for r in subset:
            dt = r["arrival_s"] - subset[0]["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            dh = handles[id(r["design"])]
            if r["kind"] == "fwd_bwd":
                g, lo = np.zeros(r["design"].total_layers), np.zeros(4)
                keep.append((g, lo))
                tickets.append(ctx.submit(dh, r["cfg"], kind=wg.REQ_LOSS_GRAD, grad=g, loss=lo))
            else:
                tickets.append(ctx.submit(dh, r["cfg"]))
        res = [ctx.poll(t) for t in tickets]
        wall = time.perf_counter() - t0
        return res, wall

    # warm-up, untimed and the same in both modes: the first 400 requests
    # once, so the classes they meet are autotuned before the timed pass
    run(reqs[:400])
    res, wall = run(reqs)
    ok = [r for r in res if r["status"] == wg.WG_OK]
    failed = [r for r in res if r["status"] != wg.WG_OK]
    if not ok:
        return {"requests": len(reqs), "completed": 0, "error": "no request completed",
                "failures": [(r["status"], r.get("error", "")) for r in failed[:5]]}
    lat = np.array([r["queue_ms"] + r["run_ms"] for r in ok])
    hits = sum(r["stats"]["n_hits"] for r in ok)
    out = {"requests": len(reqs), "completed": len(ok), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "interactions_per_s": hits / wall, "wall_s": wall,
           "mean_batch": float(np.mean([r["batch_size"] for r in ok])),
           "graph_replays": int(sum(r["graph_replayed"] for r in ok)), "failed": len(failed),
           "failures": [(r["status"], r.get("error", "")) for r in failed[:3]]}
    for dh in handles.values():
        dh.destroy()
    ctx.close()
    return out


def run_reference(args):
    ws, rank, local, pg = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    D, C = workload(0)
    rng = np.random.default_rng(0)
    G = rng.normal(size=C.tally_shape) / C.n_cell
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    base, h, t, smp = cpu_oracle_rate(D, C, G, budget_s=per_step)
    rates = []
    for i in range(args.warmup + args.steps):
        b, h, t, _ = cpu_oracle_rate(D, C, G, sample=smp)
        if i >= args.warmup:
            rates.append((h, t))
    H = sum(h for h, _ in rates)
    T = sum(t for _, t in rates)
    value = H / T
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(rates),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "reference": "FP64 CPU oracle (oracle/wg_oracle.cpp), "
                                                             "bounded sample per step"},
           "cpu_baseline": dict(base, value=value),
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    dev = local
    torch.cuda.set_device(dev)
    from paper_2601_04370_gb300 import wg
    pk, pk_kind = peaks()
    D, C = workload(rank)
    ctx = wg.Context(dev)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    G = torch.zeros_like(tally)
    grad = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    grad_t = torch.zeros(len(D.mirror_x_mm), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # work counts of one step (the same keys every step)
    st_f = ctx.trace_forward(dh, C, tally)
    loss = ctx.loss(dh, C, tally, G)
    st_b = ctx.trace_backward(dh, C, G, grad, grad_tilt=grad_t)
    hits = st_f["n_hits"]
    flops_fwd = FLOPS_PER_LAYER * st_f["n_layer_steps"] + FLOPS_PER_HIT * hits
    flops_bwd = (FLOPS_PER_LAYER * st_b["n_layer_steps"] + FLOPS_PER_HIT * st_b["n_hits"] +
                 FLOPS_ADJ_LAYER * st_b["n_adjoint_steps"])

    adj = []  # per timed step: the library's event times of its adjoint launches

    def step(evs, keep=False):
        flush.zero_()
        evs[0].record(stream)
        ctx.trace_forward(dh, C, tally, stats=False)
        evs[1].record(stream)
        ctx.loss(dh, C, tally, G)
        evs[2].record(stream)
        sb = ctx.trace_backward(dh, C, G, grad, stats=True, grad_tilt=grad_t)
        evs[3].record(stream)
        if keep:
            adj.append(sb)

    for _ in range(args.warmup):
        step([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    torch.cuda.synchronize()

    def bwd_ms_of(**kw):
        # outside the timed region: the backward with and without the tilt pass
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = []
        for _ in range(3):
            flush.zero_()
            e0.record(stream)
            ctx.trace_backward(dh, C, G, grad, stats=False, **kw)
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.median(t)
    tilt_ms = bwd_ms_of(grad_tilt=grad_t) - bwd_ms_of()
    barrier(pg, dev)
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.start()
    n0 = wg.kernel_launches()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_win0 = time.time()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        step(evs[i], keep=True)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    t_win1 = time.time()
    barrier(pg, dev)
    torch.cuda.synchronize()
    launches = wg.kernel_launches() - n0
    ck = clocks.stop(window=(t_win0, t_win1))
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    bwd_ms = [e[2].elapsed_time(e[3]) for e in evs]
    t_dev = sum(step_ms) / 1e3
    t_max = allmax(pg, t_dev, dev)
    hits_all = allsum(pg, hits * args.steps, dev)
    value = hits_all / t_max
    fwd_rate = allsum(pg, hits * args.steps, dev) / allmax(pg, sum(fwd_ms) / 1e3, dev)

    # end to end through the C ABI with host buffers: thickness from pinned
    # host memory in, loss and gradient out, every step
    th_host = torch.tensor(D.layer_d_nm, dtype=torch.float32).pin_memory().numpy()
    tl_host = torch.tensor(D.mirror_tilt_deg, dtype=torch.float32).pin_memory().numpy()
    g_host = np.zeros(D.total_layers)
    gt_host = np.zeros(len(D.mirror_x_mm))
    cfg_bytes = 4 * (len(C.lam_nm) + len(C.fx_deg) + len(C.fy_deg))
    h2d = th_host.nbytes + tl_host.nbytes + 2 * cfg_bytes
    d2h = 4 * 8 + g_host.nbytes + gt_host.nbytes
    e2e_t = []
    barrier(pg, dev)
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dh.set_params(thickness_nm=th_host, tilt_deg=tl_host)
        ctx.trace_forward(dh, C, tally, stats=False)
        ctx.loss(dh, C, tally, G)
        ctx.trace_backward(dh, C, G, g_host, stats=False, grad_tilt=gt_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_max = allmax(pg, sum(e2e_t), dev)
    e2e_value = hits_all / e2e_max

    # the coating look-up table (the paper's memory-saving variant): the same
    # step, after the timed region, with 16384 bins of cos(theta_0) (tallies
    # within ~1e-4 of the exact per-hit chain on this workload)
    lut_bins = 16384
    CL = C.replace(lut_bins=lut_bins)
    lut_ms, lut_f, lut_b = [], [], []
    for i in range(args.warmup + args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        flush.zero_()
        ev[0].record(stream)
        ctx.trace_forward(dh, CL, tally, stats=False)
        ev[1].record(stream)
        ctx.loss(dh, CL, tally, G)
        ev[2].record(stream)
        ctx.trace_backward(dh, CL, G, grad, stats=False, grad_tilt=grad_t)
        ev[3].record(stream)
        ev[3].synchronize()
        if i >= args.warmup:
            lut_ms.append(ev[0].elapsed_time(ev[3]))
            lut_f.append(ev[0].elapsed_time(ev[1]))
            lut_b.append(ev[2].elapsed_time(ev[3]))
    lut_t = allmax(pg, sum(lut_ms) / 1e3, dev)
    coating_table = {"lut_bins": lut_bins, "value": allsum(pg, hits * len(lut_ms), dev) / lut_t, "unit": UNIT,
                     "ms_per_step": 1e3 * lut_t / len(lut_ms), "fwd_ms": statistics.mean(lut_f),
                     "bwd_ms": statistics.mean(lut_b),
                     "note": "coefficients per (mirror, side, wavelength, cos bin) computed once per call and "
                             "interpolated per hit; the adjoint scatters dL/dc into the bins and runs the thin-film "
                             "adjoint once per bin (two-stage); measured after the timed region, not the headline"}

    # the two-dimensional pupil expander (general mirrors: 30 fold + 16 output,
    # 23 layers, 9 wavelengths, 16x16 fields, 1e7 rays): the same step
    # (forward, loss, backward with thickness and tilt gradients), after the
    # timed region, not the headline; the oracle timed beside it on a sample
    expander = None
    if not args.no_expander:
        from paper_2601_04370_gb300 import workloads as W
        DE, CE = W.pupil_expander(n_rays=C.total_rays)
        dhe = ctx.create_design(DE)
        te = torch.zeros(CE.tally_shape, dtype=torch.float64, device=f"cuda:{dev}")
        Ge = torch.zeros_like(te)
        ge = torch.zeros(DE.total_layers, dtype=torch.float64, device=f"cuda:{dev}")
        gte = torch.zeros(DE.n_mirrors, dtype=torch.float64, device=f"cuda:{dev}")
        e_ms, e_f, e_b, e_tilt, e_hits = [], [], [], [], 0
        for i in range(args.warmup + args.steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            flush.zero_()
            ev[0].record(stream)
            sfe = ctx.trace_forward(dhe, CE, te)
            ev[1].record(stream)
            ctx.loss(dhe, CE, te, Ge)
            ev[2].record(stream)
            sbe = ctx.trace_backward(dhe, CE, Ge, ge, grad_tilt=gte)
            ev[3].record(stream)
            ev[3].synchronize()
            if i >= args.warmup:
                e_ms.append(ev[0].elapsed_time(ev[3]))
                e_f.append(ev[0].elapsed_time(ev[1]))
                e_b.append(ev[2].elapsed_time(ev[3]))
                e_tilt.append(sbe["tilt_ms"])
                e_hits = sfe["n_hits"]
        e_t = allmax(pg, sum(e_ms) / 1e3, dev)
        expander = {"workload": "2D pupil expander: 30 fold + 16 output general mirrors, 23-layer Ta2O5/SiO2, "
                                "9 wavelengths, 16x16 fields over 38x38 deg, 64x64 bins over 16x16 mm, "
                                f"{CE.total_rays} rays",
                    "value": allsum(pg, e_hits * len(e_ms), dev) / e_t, "unit": UNIT,
                    "ms_per_step": 1e3 * e_t / len(e_ms), "fwd_ms": statistics.mean(e_f),
                    "bwd_ms": statistics.mean(e_b), "tilt_pass_ms": statistics.mean(e_tilt),
                    "fwd_interactions_per_s": e_hits / (statistics.mean(e_f) / 1e3),
                    "roofline_fwd": None,
                    "interactions_per_step": e_hits, "hits_per_ray": e_hits / CE.total_rays,
                    "overflow": sbe["overflow"], "nonfinite": sbe["n_nonfinite"]}
        # the forward's FP32 roofline on this design (33 flops per layer of the
        # hit's stack + 250 per hit, as for the representative workload)
        lay = sfe["n_layer_steps"] / max(1, e_hits)
        sm_e = torch.cuda.get_device_properties(dev).multi_processor_count
        pk_e = fp32_peak_tflops(sm_e, float(pk.get("sm_max_mhz", 2070.0)))
        ach_e = e_hits * (FLOPS_PER_LAYER * lay + FLOPS_PER_HIT) / (statistics.mean(e_f) / 1e3) / 1e12
        expander["roofline_fwd"] = {"bound": "alu", "kernel": "k_trace_fwd", "achieved": ach_e, "peak": pk_e,
                                    "unit": "TFLOP/s", "frac": ach_e / pk_e,
                                    "units": f"{FLOPS_PER_LAYER} x {lay:.1f} layers + {FLOPS_PER_HIT} flops per interaction"}
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:
            expander["cpu_baseline"], _, _, _ = cpu_oracle_rate(DE, CE, Ge.cpu().numpy(),
                                                             budget_s=max(2.0, args.cpu_budget / 3))
        dhe.destroy()

    # the differentiation configuration (6 mirrors x 200 layers = 1200
    # thicknesses + 6 tilts, 1e8 rays, the accurate layer evaluation): the
    # same step (forward, loss, backward with thickness and tilt gradients),
    # after the timed region, with its own rooflines and CPU baseline
    differentiation = None
    if not args.no_differentiation:
        differentiation = bench_differentiation(ctx, dev, args, pg, ws, rank, flush, stream, pk, pk_kind)

    # the batching configuration: 64 designs (K 3..8, L 10..200, 30% pruned,
    # 1e5..1e7 rays) in one fused launch per kernel variant with autotuned
    # shapes and graph replay, against one design per launch
    batching = None
    if args.batch_rounds > 0:
        batching = run_child(["--batch-child", f"{dev},{args.batch_rounds}"], timeout=900)

    # serving: the same request trace batched by the runtime and one design per launch
    serving = None
    if args.serve_requests > 0:
        import tempfile
        cache = os.path.join(tempfile.mkdtemp(prefix="wg_tune_"), "autotune.txt")
        barrier(pg, dev)

        def serve_child(slots, n_req, rate):
            return run_child(["--serve-child", f"{dev},{n_req},{slots},{cache},{rate}"], timeout=900)

        serving = {}
        for rate, n_req in ((200.0, args.serve_requests), (args.serve_low_rate, args.serve_low_requests)):
            if n_req <= 0:
                continue
            bt = serve_child(64, n_req, rate)
            ot = serve_child(1, n_req, rate)
            serving[f"{rate:g}_req_per_s"] = {
                "trace": f"{n_req} requests, Poisson {rate:g} req/s (seed 5), designs from the 64-design batching pool "
                         f"(K 3..8, L 10..200, 30% pruned), fwd at 1e5..1e7 rays, 5% loss+grad at 1e6..1e8 rays; "
                         f"the first {min(400, n_req)} requests served once untimed before",
                "batched": bt, "one_design_per_launch": ot}

    out = None
    if rank == 0:
        sm = torch.cuda.get_device_properties(dev).multi_processor_count
        smax = float(pk.get("sm_max_mhz", 2070.0))
        peak = fp32_peak_tflops(sm, smax)
        bwd_s = statistics.mean(bwd_ms) / 1e3 - max(tilt_ms, 0.0) / 1e3  # thickness adjoint only
        fwd_s = statistics.mean(fwd_ms) / 1e3
        ach_b = flops_bwd / bwd_s / 1e12
        ach_f = flops_fwd / fwd_s / 1e12
        peak_source = (f"derived: {sm} SMs x 128 FP32 lanes x 2 flop x {smax:.0f} MHz "
                       f"(sm_max_mhz of {pk_kind} peaks)")
        # the thin-film adjoint (tilt variant): its launches are timed by the
        # library with CUDA events on the launching stream during the timed
        # steps (wg_stats adjoint_ms / n_adjoint_launches)
        n_adj = sum(s["n_adjoint_launches"] for s in adj)
        adj_ms = sum(s["adjoint_ms"] for s in adj)
        adj_steps = sum(s["n_adjoint_steps"] for s in adj)
        flops_adj = FLOPS_ADJ_LAYER_TILT * adj_steps / max(1, n_adj)
        ach_a = flops_adj / (adj_ms / max(1, n_adj) / 1e3) / 1e12 if adj_ms > 0 else 0.0
        roof = {"bound": "alu", "kernel": "k_bwd_adjoint (tilt variant)", "achieved": ach_a, "peak": peak,
                "unit": "TFLOP/s", "frac": ach_a / peak, "traffic": profile_traffic("k_bwd_adjoint"),
                "flops_per_launch": flops_adj, "launch_ms": adj_ms / max(1, n_adj), "launches": n_adj,
                "units": f"{adj_steps / max(1, n_adj):.4g} record layer steps per launch x "
                         f"{FLOPS_ADJ_LAYER_TILT} flops",
                "peak_source": peak_source}
        # the forward trace: the event pair around the forward call on the
        # launching stream (the kernel plus two tiny preparation launches)
        roof_f = {"bound": "alu", "kernel": "k_trace_fwd", "achieved": ach_f, "peak": peak, "unit": "TFLOP/s",
                  "frac": ach_f / peak, "traffic": profile_traffic("k_trace_fwd"),
                  "flops_per_launch": flops_fwd,
                  "units": f"{hits} interactions x ({FLOPS_PER_LAYER} x {st_f['n_layer_steps'] / hits:.1f} layers "
                           f"+ {FLOPS_PER_HIT}) flops",
                  "peak_source": peak_source}
        roof_b = {"bound": "alu", "kernels": "k_bwd_replay + sort + k_bwd_adjoint (tilt pass excluded)", "achieved": ach_b,
                  "peak": peak, "unit": "TFLOP/s", "frac": ach_b / peak, "flops_per_call": flops_bwd}
        # "roofline" is the dominant kernel of the step: the one with the
        # larger device time per step (the launch list's largest share)
        step_ms_mean = 1e3 * t_max / args.steps
        fwd_step_ms = fwd_s * 1e3
        adj_step_ms = adj_ms / max(1, len(adj))
        roof_f["ms_per_step"] = fwd_step_ms
        roof_f["share_of_step"] = fwd_step_ms / step_ms_mean
        roof["ms_per_step"] = adj_step_ms
        roof["share_of_step"] = adj_step_ms / step_ms_mean
        roof_dom = roof_f if fwd_step_ms >= adj_step_ms else roof
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu, _, _, _ = cpu_oracle_rate(D, C, G.cpu().numpy(), budget_s=args.cpu_budget)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD_NAME, "rays_per_gpu": C.total_rays,
                          "interactions_per_step_per_gpu": hits, "l2": "flushed between steps (256 MiB write)",
                          "parallelism": f"replicas x{ws} (rays sharded by seed, no collective)"},
               "fwd_interactions_per_s": fwd_rate, "fwd_ms": statistics.mean(fwd_ms),
               "bwd_ms": statistics.mean(bwd_ms), "tilt_pass_ms": tilt_ms, "loss": loss[0], "wall_s": t_wall,
               "roofline": roof_dom, "roofline_fwd": roof_f, "roofline_adjoint": roof, "roofline_bwd": roof_b,
               "cpu_baseline": cpu,
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": launches, "clocks": ck, "coating_table": coating_table,
               "pupil_expander": expander, "differentiation": differentiation, "batching": batching,
               "serving": serving}
        print(json.dumps(out))
    dh.destroy()
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-expander", action="store_true", help="skip the two-dimensional pupil-expander entry")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving trace at 200 req/s (0: skip)")
    ap.add_argument("--serve-low-rate", type=float, default=50.0,
                    help="arrival rate of the second serving run, below the GPU's capacity")
    ap.add_argument("--serve-low-requests", type=int, default=400,
                    help="requests of the second serving run (0: skip)")
    ap.add_argument("--no-differentiation", action="store_true", help="skip the differentiation-configuration entry")
    ap.add_argument("--d-steps", type=int, default=3, help="timed steps of the differentiation entry")
    ap.add_argument("--batch-rounds", type=int, default=3,
                    help="timed rounds of the batching entry after its warm-up rounds (0: skip)")
    ap.add_argument("--serve-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--batch-child", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.serve_child:
        dev, n, slots, cache, rate = args.serve_child.split(",", 4)
        import torch
        torch.cuda.set_device(int(dev))
        print(json.dumps(run_serving(int(dev), int(n), int(slots), cache, float(rate))))
        return 0
    if args.batch_child:
        dev, rounds = args.batch_child.split(",", 1)
        import torch
        torch.cuda.set_device(int(dev))
        print(json.dumps(run_batching(int(dev), int(rounds))))
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
