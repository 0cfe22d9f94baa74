"""Boundary checks of the C ABI on the GPU: a host pointer where the kernels
write device memory is rejected with WG_EINVAL (never handed to a kernel),
and WGTrace refuses a backward whose design changed after its forward."""
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


def test_host_ray_records_are_rejected(wg):
    D, C = W.tiny(n_rays=2000)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    host_rec = np.zeros(C.total_rays * 8, dtype=np.int32)
    with pytest.raises(wg.WGError) as e:
        ctx.trace_forward(dh, C, tally, records=host_rec)
    assert e.value.status == wg.WG_EINVAL and "ray_records" in str(e.value)
    # the allocation-free entry point takes the same configuration check
    import ctypes as C_
    h = wg._CfgHolder(C, wg._current_stream(), None, host_rec)
    st = wg.lib().wg_trace_forward_noalloc(ctx.h, dh.h, C_.byref(h.c), tally.data_ptr(), None)
    assert st == wg.WG_EINVAL and "ray_records" in wg.lib().wg_last_error().decode()
    # device records still work, and the context is usable after the rejections
    rec = torch.zeros(C.total_rays * 8, dtype=torch.int32, device="cuda")
    s = ctx.trace_forward(dh, C, tally, records=rec)
    assert s["n_rays"] == C.total_rays
    assert (rec.cpu().numpy().view(wg.RAY_RECORD_DTYPE)["n_events"] > 0).all()
    dh.destroy()
    ctx.close()


def test_wgtrace_refuses_a_backward_after_the_design_changed(wg):
    D, C = W.tiny(n_rays=4000)
    ctx = wg.Context(0)
    dh = ctx.create_design(D)
    WGTrace = wg.WGTrace
    th0 = torch.tensor(D.layer_d_nm, dtype=torch.float32, device="cuda", requires_grad=True)
    v0 = dh.version()
    t1 = WGTrace.apply(th0, ctx, dh, C)
    assert dh.version() > v0
    # a second forward on the same handle with other thicknesses
    th1 = (th0.detach() + 1.0).requires_grad_(True)
    t2 = WGTrace.apply(th1, ctx, dh, C)
    with pytest.raises(RuntimeError, match="changed after this forward"):
        t1.sum().backward()
    # the latest forward's backward is fine
    t2.sum().backward()
    assert th1.grad is not None and torch.isfinite(th1.grad).all()
    # an omega change counts as a parameter change too
    t3 = WGTrace.apply(th1.detach().requires_grad_(True), ctx, dh, C)
    dh.set_omega(np.full(D.n_mirrors, 0.4, dtype=np.float32))
    with pytest.raises(RuntimeError):
        t3.sum().backward()
    dh.destroy()
    ctx.close()
