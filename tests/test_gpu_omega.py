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


def test_omega_adam_steps_match_the_oracle(wg, ora):
    """Five steps of wg_omega_adam_step on gradients spanning many decades,
    with values driven into both clip bounds, a non-finite entry, host and
    device gradients: the omega the design takes equals the oracle's step
    (FP64 state on both sides, FP32 in the design)."""
    D, _ = W.representative(n_rays=1000)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    K = D.n_mirrors
    w0 = np.array([0.5, 0.03, 0.97, 0.2, 0.6, 0.45], dtype=np.float32)[:K]
    dh.set_omega(w0)
    opt = wg.OmegaAdam(dh, lr=0.02)
    rng = np.random.default_rng(3)
    w, m, v = w0.astype(np.float64), np.zeros(K), np.zeros(K)
    for t in range(1, 6):
        g = rng.normal(size=K) * 10.0 ** rng.uniform(-5, 4, size=K)
        g[1] = 3.0    # pushes omega_1 below lo
        g[2] = -3.0   # pushes omega_2 above hi
        if t == 3:
            g[4] = np.nan
        gd = torch.as_tensor(g, device="cuda") if t % 2 else g
        got = opt.step(gd)
        w, m, v = ora.adam_clipped_step(w, m, v, g, t, lr=0.02)
        assert np.allclose(got, w.astype(np.float32), rtol=0, atol=1e-7), (t, got, w)
    assert got[1] == np.float32(0.02) and got[2] == np.float32(0.98)
    opt.close()
    dh.destroy()
    ctx.close()
