"""The differentiation configuration (6 mirrors x 200 layers = 1200
thicknesses plus 6 tilts, 3 wavelengths, the CV loss): GPU gradients against
the FP64 oracle's adjoint at 1e5 rays, and the full 1e8-ray launch checked on
samples the oracle can compute: rays one by one, and the gradient of the
first 1e5 rays of the full configuration (the backward over a ray range)."""
import numpy as np
import pytest
import torch

from paper_2601_04370_gb300 import workloads as W

from test_gpu_parity import _grad_compare, ctx, run_gpu  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu


def test_gradients_at_1e5_rays_match_the_oracle_adjoint(ctx, ora):
    """A measured FP32 limit, not the 1e-3 bar: G is the CV loss of this
    1e5-ray tally (~58 rays per cell), so ten rays carry a quarter of the
    weight and the per-hit FP32 errors of 200-layer coatings do not average
    out. Measured against the oracle: thicknesses 3.6e-3, tilts 5.4e-3
    (relative L2; one ray of 1e5 takes another path and carries no weight).
    An accurate sin/cos in the layer phase gives 2.4e-3 and 4.8e-3, so the
    fast one is only part of it. With G from the full 1e8-ray tally the same
    number of rays holds 1e-3 (test_full_size_differentiation_sampled)."""
    D, C = W.differentiation(n_rays=100_000)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, tally)
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gt = np.zeros(D.n_mirrors)
    st = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    assert st["overflow"] == 0 and st["n_nonfinite"] == 0
    ref_d, ref_t = ora.trace_grad(D, C, G.cpu().numpy(), nthreads=0)
    _grad_compare(g.cpu().numpy(), ref_d, tol=5e-3)
    assert np.linalg.norm(gt - ref_t) <= 8e-3 * np.linalg.norm(ref_t), (gt, ref_t)
    dh.destroy()


def test_full_size_differentiation_sampled(ctx, ora):
    D, C = W.differentiation()
    dh = ctx.create_design(D)
    g = run_gpu(ctx, D, C, dh=dh)
    rg = g["records"]
    N = C.total_rays
    assert g["stats"]["n_rays"] == N and len(rg) == N
    rng = np.random.default_rng(2)
    starts = np.sort(rng.choice(N - 32, 24, replace=False))
    mism, tot, dI = 0, 0, []
    for s in starts:
        o = ora.trace(D, C, rays=(int(s), int(s) + 32), records=True, nthreads=4)["records"]
        gg = rg[s:s + 32]
        bad = (gg["hash"] != o["hash"]) | (gg["bin"] != o["bin"])
        mism += int(bad.sum())
        tot += 32
        ok = ~bad
        dI.append(np.abs(gg["I"][ok] - o["I"][ok]) / np.maximum(1, o["I"][ok]))
    assert mism <= max(1, int(1e-3 * tot))
    assert np.quantile(np.concatenate(dI), 0.99) <= 1e-3
    # the full backward: every listed ray's records fit, nothing non-finite
    tally = torch.as_tensor(g["tally"], device="cuda")
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G)
    gfull = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gtf = np.zeros(D.n_mirrors)
    st = ctx.trace_backward(dh, C, G, gfull, grad_tilt=gtf)
    assert st["overflow"] == 0 and st["n_nonfinite"] == 0
    assert np.all(np.isfinite(gfull.cpu().numpy())) and np.all(np.isfinite(gtf))
    # the first 1e5 rays of the full configuration: the oracle's gradient over the same rays
    rays = (0, 100_000)
    gsub = torch.zeros_like(gfull)
    gts = np.zeros(D.n_mirrors)
    st = ctx.trace_backward(dh, C, G, gsub, rays=rays, grad_tilt=gts)
    assert st["overflow"] == 0 and st["n_nonfinite"] == 0
    ref_d, ref_t = ora.trace_grad(D, C, G.cpu().numpy(), rays=rays, nthreads=0)
    _grad_compare(gsub.cpu().numpy(), ref_d)
    assert np.linalg.norm(gts - ref_t) <= 1e-3 * np.linalg.norm(ref_t), (gts, ref_t)
    dh.destroy()
