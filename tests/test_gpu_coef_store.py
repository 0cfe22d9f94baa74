"""The listing forward keeps the applied coefficients of each ray's first
hits and the replay reads them back instead of re-running those hits' layer
chains: the gradients are the same as with the chains re-run, and a kept
coefficient is never used for other thicknesses or another coating method
than the ones it was computed for."""
import numpy as np
import pytest
import torch

from paper_2601_04370_gb300 import workloads as W

from test_gpu_parity import tilt_compare, _grad_compare, ctx  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu


def _fwd_loss(ctx, dh, C):
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, t)
    G = torch.zeros_like(t)
    ctx.loss(dh, C, t, G)
    return G


def _bwd(ctx, dh, D, C, G, tilts=True):
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gt = np.zeros(D.n_mirrors) if tilts else None
    st = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    return g.cpu().numpy(), gt, st


@pytest.mark.parametrize("name", ["rep", "expander"])
def test_kept_coefficients_give_the_recomputed_gradients(ctx, name):
    D, C = (W.representative(n_rays=1728 * 8, n_layers=40) if name == "rep" else W.pupil_expander_small())
    dh = ctx.create_design(D)
    G = _fwd_loss(ctx, dh, C)
    g1, t1, s1 = _bwd(ctx, dh, D, C, G)
    # the same thicknesses set again: the kept coefficients are stale by
    # version, so the replay re-runs every chain
    dh.set_params(thickness_nm=D.layer_d_nm)
    g2, t2, s2 = _bwd(ctx, dh, D, C, G)
    assert s2["n_layer_steps"] > s1["n_layer_steps"]   # the kept ones skipped work
    # the same records either way; the per-layer FP32 partial sums in shared
    # memory add in a different order from run to run (~1 ulp of FP32)
    assert np.abs(g1 - g2).max() <= 1e-6 * np.abs(g2).max()
    assert np.abs(t1 - t2).max() <= 1e-6 * np.abs(t2).max()
    dh.destroy()


def test_thickness_update_between_forward_and_backward(ctx, ora):
    """Paths do not depend on the thicknesses, so the eyebox list stays, but
    the coefficients do: the backward at new thicknesses is the oracle's
    gradient at those thicknesses."""
    D, C = W.representative(n_rays=1728 * 8, n_layers=40)
    dh = ctx.create_design(D)
    G = _fwd_loss(ctx, dh, C)
    rng = np.random.default_rng(9)
    d2 = np.clip(D.layer_d_nm + rng.normal(0.0, 5.0, D.total_layers), 10.0, 200.0).astype(np.float32)
    dh.set_params(thickness_nm=d2)
    g, gt, st = _bwd(ctx, dh, D, C, G)
    assert st["overflow"] == 0 and st["n_nonfinite"] == 0
    D2 = D.replace(layer_d_nm=d2)
    ref_d, ref_t = ora.trace_grad(D2, C, G.cpu().numpy())
    _grad_compare(g, ref_d)
    tilt_compare(gt, ref_t)
    dh.destroy()


def test_coating_method_change_between_forward_and_backward(ctx, ora):
    """A table forward keeps no coefficients (and a kept exact set from an
    earlier forward is not the table's): an exact backward after it re-runs
    the chains."""
    D, C = W.representative(n_rays=1728 * 8, n_layers=40)
    dh = ctx.create_design(D)
    G = _fwd_loss(ctx, dh, C.replace(lut_bins=4096))
    g, gt, st = _bwd(ctx, dh, D, C, G)
    ref_d, ref_t = ora.trace_grad(D, C, G.cpu().numpy())
    _grad_compare(g, ref_d)
    dh.destroy()
