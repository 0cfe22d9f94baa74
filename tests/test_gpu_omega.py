"""The reflection-probability pre-optimization on the GPU (wg_omega_trace,
wg_set_omega; Methods, "Learned reflection probabilities") against the
oracle's model on the same rays, and its optimization loop."""
import numpy as np
import pytest
import torch

from paper_2601_04370_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_04370_gb300 import wg as _wg
    return _wg


@pytest.mark.parametrize("name", ["tiny", "rep"])
def test_omega_trace_matches_the_oracle(wg, ora, name):
    if name == "tiny":
        D, C = W.tiny(n_rays=50_000)
    else:
        D, C = W.representative(n_rays=1728 * 16)
    om = np.linspace(0.3, 0.7, len(D.mirror_x_mm)).astype(np.float32)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    dh.set_omega(om)
    Do = D.replace(mirror_omega=om)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G, w_f=0.0, w_e=0.0)
    g = np.zeros(len(om))
    ctx.omega_trace(dh, C, tally, G, g)
    ref_t, ref_g = ora.geo_trace(Do, C, G=G.cpu().numpy())
    t = tally.cpu().numpy()
    assert np.abs(t - ref_t).max() <= 1e-4 * np.abs(ref_t).max()
    assert np.linalg.norm(g - ref_g) <= 1e-3 * np.linalg.norm(ref_g), (g, ref_g)
    dh.destroy()
    ctx.close()


def test_omega_optimization_raises_throughput(wg):
    D, C = W.tiny(n_rays=50_000)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    dh.set_omega(np.full(len(D.mirror_x_mm), 0.5, dtype=np.float32))
    D = D.replace(mirror_omega=np.full(len(D.mirror_x_mm), 0.5, dtype=np.float32))
    dh.design = D
    hist, om = wg.optimize_omega(ctx, dh, C, 40, lr=0.03)
    assert np.all((om >= 0.02) & (om <= 0.98))
    assert hist[-1] > hist[0] * 1.02, hist
    dh.destroy()
    ctx.close()
