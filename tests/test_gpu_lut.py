"""The coating look-up table (cfg.lut_bins > 0; the paper's memory-saving
variant, Fig. 3c): tallies and gradients (thicknesses and tilts) equal the
oracle's for the same tabulated method, the table differs from the exact
per-hit chain by its interpolation error only, and the calls that do not
support it refuse it."""
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


def _cfg(name):
    if name == "tiny":
        D, C = W.tiny()
        return D, C.replace(lut_bins=256)
    D, C = W.representative(n_rays=1728 * 8)
    return D, C.replace(lut_bins=16384)


def _grad_close(g, ref, tol=1e-3):
    assert np.all(np.isfinite(g))
    assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref), np.linalg.norm(g - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["tiny", "rep"])
def test_table_forward_and_gradients_match_the_oracle(wg, ora, name):
    D, C = _cfg(name)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    st = ctx.trace_forward(dh, C, tally)
    assert st["n_layer_steps"] == 0  # no per-hit layer chain
    ref = ora.trace(D, C)["tally"]
    t = tally.cpu().numpy()
    # FP32 table entries and interpolation against FP64: same tolerance as the exact path's tallies
    assert np.abs(t - ref).max() <= 1e-4 * np.abs(ref).max()
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gt = np.zeros(len(D.mirror_x_mm))
    sb = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    assert sb["n_adjoint_launches"] == 1 and sb["n_nonfinite"] == 0
    ref_d, ref_t = ora.trace_grad(D, C, G.cpu().numpy())
    _grad_close(g.cpu().numpy(), ref_d)
    _grad_close(gt, ref_t)
    dh.destroy()
    ctx.close()


def test_table_tallies_within_interpolation_error_of_exact(wg):
    """16384 bins on the representative design: the tabulated tally is the
    exact per-hit tally to ~1e-4 (the oracle measures 9e-5 max relative at
    this size)."""
    D, C = W.representative(n_rays=1728 * 8)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    ex = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    lt = torch.zeros_like(ex)
    ctx.trace_forward(dh, C, ex)
    ctx.trace_forward(dh, C.replace(lut_bins=16384), lt)
    e, l = ex.cpu().numpy(), lt.cpu().numpy()
    assert np.abs(l - e).max() <= 3e-4 * np.abs(e).max()
    assert np.abs(l - e).sum() <= 1e-4 * np.abs(e).sum()
    dh.destroy()
    ctx.close()


def test_table_is_refused_where_unsupported(wg):
    D, C = W.tiny()
    C = C.replace(lut_bins=256)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    with pytest.raises(wg.WGError) as e:
        ctx.submit(dh, C)
    assert e.value.status == wg.WG_EINVAL
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(wg.WGError) as e:
        ctx.trace_forward_noalloc(dh, C, t)
    assert e.value.status == wg.WG_EINVAL
    with pytest.raises(wg.WGError) as e:
        ctx.trace_forward(dh, C.replace(lut_bins=8), t)
    assert e.value.status == wg.WG_EINVAL
    dh.destroy()
    ctx.close()
