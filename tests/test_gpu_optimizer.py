"""The thickness optimizer (wg_adam_*, Results "Evaluation": 20-200 nm with a
soft gap that prunes layers) against the oracle's step, and the optimization
loop on the tiny design."""
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


@pytest.fixture(scope="module")
def ora():
    from oracle import oracle as O
    return O


def test_adam_steps_match_the_oracle(wg, ora):
    """Five steps on random gradients spanning many decades, with layers near
    the bounds and in the gap, host and device gradients, a design-pruned
    layer and a non-finite entry: thicknesses and the final projection equal
    the oracle's (FP32 storage, FP64 moments on both sides)."""
    D = W.batching(n_designs=1, seed=4)[0][0]
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    n = D.total_layers
    rng = np.random.default_rng(5)
    th0 = W.gaussian_thickness(D, seed=1)
    th0[:6] = np.where(D.pruned[:6] == 1, 0.0, [199.5, 21.0, 11.0, 0.0, 24.0, 150.0]).astype(np.float32)
    adam = wg.Adam(dh, lr_nm=2.0, thickness_nm=th0)
    th, m, v = th0.copy(), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.normal(size=n) * 10.0 ** rng.uniform(-5, 3, size=n)
        g[:6] = [-1.0, 1.0, 1.0, -1.0, 1.0, 1.0]
        if t == 3:
            g[7] = np.nan
        if t % 2:
            adam.step(torch.tensor(g, device="cuda"))
        else:
            adam.step(g)
        th, m, v = ora.adam_projected_step(th, m, v, g, t, lr=2.0, fixed=D.pruned)
    got = adam.params()
    assert np.allclose(got, th, rtol=0, atol=2e-5), np.abs(got - th).max()
    assert np.all(got[D.pruned == 1] == 0.0)
    assert np.all((got == 0.0) | ((got >= 20.0) & (got <= 200.0)))
    adam.close()
    dh.destroy()
    ctx.close()


def test_optimization_loop_lowers_the_loss(wg):
    """Random start within the bounds, the loss of Eq. 1, its adjoint and the
    projected Adam step: with the Philox keys fixed the objective is a
    deterministic function of the thicknesses, and 12 steps lower it."""
    D, C = W.tiny(n_rays=20_000)
    D = W.with_thickness(D, W.gaussian_thickness(D, seed=3))
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    hist, adam = wg.optimize(ctx, dh, C, 12, adam=wg.Adam(dh, lr_nm=3.0))
    L = hist[:, 0]
    assert np.all(np.isfinite(L))
    assert L[-1] < L[0] - 1e-3 * abs(L[0]), L
    th = adam.params()
    assert np.all((th == 0.0) | ((th >= 20.0) & (th <= 200.0)))
    adam.close()
    dh.destroy()
    ctx.close()
