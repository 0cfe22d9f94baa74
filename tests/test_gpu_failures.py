"""Failure paths and serving guarantees, exercised without any GPU fault:
a bounded device wait that runs out (the kernels return, the call reports
WG_ETIMEOUT, the GPU stays usable), a poll that times out on a running
request (WG_ENOTREADY), a full queue (WG_EBUSY), a loss+gradient request
that gives the same result alone and while the forward lane runs other
designs beside it, and the autotuner's choice and its cache file."""
import os
import tempfile

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


def test_a_wait_on_a_flag_nothing_sets_returns_etimeout(wg):
    """The bounded device wait of the trace kernels, on a flag that nothing
    sets: it gives up after its limit (1 ms here), sets the error word and
    returns; the call reports WG_ETIMEOUT and the context stays usable."""
    ctx = wg.Context(0)
    with pytest.raises(wg.WGError) as e:
        ctx.test_bounded_wait(1_000_000)
    assert e.value.status == wg.WG_ETIMEOUT and "wait ran out" in str(e.value)
    D, C = W.tiny(n_rays=10_000)
    dh = ctx.create_design(D)
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    st = ctx.trace_forward(dh, C, t)
    assert st["n_rays"] == C.total_rays and t.sum().item() > 0
    dh.destroy()
    ctx.close()


def test_wait_limit_of_a_context_reaches_the_trace_kernels(wg):
    """A context whose device waits give up after 1 ns: a wait that does not
    complete at once (the design staging, the idle wait of a warp without
    rays) runs out, the kernel sets the error word and returns, and the call
    reports WG_ETIMEOUT; whether any wait of a given call has to wait at all
    depends on timing, so each call either reports WG_ETIMEOUT or succeeds,
    and returns either way. A default context then traces normally."""
    D, C = W.tiny(n_rays=10_000)
    short = wg.Context(0, wait_limit_ns=1)
    dh = short.create_design(D)
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    try:
        short.trace_forward(dh, C, t)
    except wg.WGError as e:
        assert e.status == wg.WG_ETIMEOUT and "wait ran out" in str(e)
    G = torch.ones_like(t)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    try:
        short.trace_backward(dh, C, G, g)
    except wg.WGError as e2:
        assert e2.status == wg.WG_ETIMEOUT
    dh.destroy()
    short.close()
    torch.cuda.synchronize()
    ok = wg.Context(0)
    dh = ok.create_design(D)
    st = ok.trace_forward(dh, C, t)
    assert st["n_rays"] == C.total_rays and t.sum().item() > 0
    dh.destroy()
    ok.close()


def test_poll_with_a_short_timeout_returns_enotready(wg):
    ctx = wg.Context(0, max_slots=4)
    D, C = W.differentiation(n_rays=4_000_000)
    dh = ctx.create_design(D)
    tk = ctx.submit(dh, C)
    assert ctx.poll(tk, timeout_us=1) is None          # WG_ENOTREADY: still running
    r = ctx.poll(tk)                                    # then completes
    assert r["status"] == wg.WG_OK and r["stats"]["n_rays"] == C.total_rays
    dh.destroy()
    ctx.close()


def test_a_full_queue_returns_ebusy(wg):
    """max_queue = 1 with one lane: the scheduler runs the first long request
    while at most one more waits; a further submit is refused with WG_EBUSY
    and the accepted requests complete."""
    ctx = wg.Context(0, max_slots=1, max_queue=1)
    D, C = W.differentiation(n_rays=4_000_000)
    dh = ctx.create_design(D)
    accepted, busy = [], 0
    for _ in range(4):
        try:
            accepted.append(ctx.submit(dh, C))
        except wg.WGError as e:
            assert e.status == wg.WG_EBUSY
            busy += 1
    assert busy >= 1 and 1 <= len(accepted) <= 3
    assert all(ctx.poll(t)["status"] == wg.WG_OK for t in accepted)
    dh.destroy()
    ctx.close()


def test_loss_and_gradient_request_alone_equals_in_a_mix(wg):
    """The same loss+gradient request served alone, and again while the
    forward lane runs a batch of other designs beside it: loss and gradient
    agree to the FP32 summation order of the partial sums."""
    ctx = wg.Context(0)
    D, C = W.representative(n_rays=1728 * 16)
    dh = ctx.create_design(D)
    others = [(ctx.create_design(Dj), Cj.replace(n_rays=1728 * 64)) for Dj, Cj in W.batching(n_designs=6, seed=4)]
    g_alone, l_alone = np.zeros(D.total_layers), np.zeros(4)
    r = ctx.poll(ctx.submit(dh, C, kind=wg.REQ_LOSS_GRAD, grad=g_alone, loss=l_alone))
    assert r["status"] == wg.WG_OK
    g_mix, l_mix = np.zeros(D.total_layers), np.zeros(4)
    outs = [np.zeros(Cj.tally_size) for _, Cj in others]
    tks = [ctx.submit(dhj, Cj, tally=o) for (dhj, Cj), o in zip(others[:3], outs[:3])]
    tk = ctx.submit(dh, C, kind=wg.REQ_LOSS_GRAD, grad=g_mix, loss=l_mix)
    tks += [ctx.submit(dhj, Cj, tally=o) for (dhj, Cj), o in zip(others[3:], outs[3:])]
    res = [ctx.poll(t) for t in tks]
    r = ctx.poll(tk)
    assert r["status"] == wg.WG_OK and all(x["status"] == wg.WG_OK for x in res)
    assert max(x["batch_size"] for x in res) >= 2          # the forward lane batched the others
    assert abs(l_mix[0] - l_alone[0]) <= 1e-6 * abs(l_alone[0])
    assert np.abs(g_mix - g_alone).max() <= 1e-5 * np.abs(g_alone).max()
    for dhj, _ in others:
        dhj.destroy()
    dh.destroy()
    ctx.close()


def test_autotuner_keeps_the_fastest_shape_and_the_cache_round_trips(wg):
    tmp = tempfile.mkdtemp(prefix="wg_tune_test_")
    path = os.path.join(tmp, "tune.txt")
    D, C = W.representative(n_rays=1728 * 64)
    ctx = wg.Context(0, autotune_cache=path)
    dh = ctx.create_design(D)
    assert ctx.autotune_info(dh, C) is None
    ctx.autotune(dh, C)
    info = ctx.autotune_info(dh, C)
    assert info["n_tried"] >= 2
    best = min(info["tried"], key=lambda x: x[2])
    assert (info["chunk_rays"], info["ctas_per_sm"]) == (best[0], best[1])
    assert info["best_ms"] == pytest.approx(best[2]) and info["best_ms"] > 0
    dh.destroy()
    ctx.close()
    text = open(path).read()
    assert f"{info['chunk_rays']} {info['ctas_per_sm']}" in text
    # a new context reads the entry back and does not tune that class again
    ctx2 = wg.Context(0, autotune_cache=path)
    dh2 = ctx2.create_design(D)
    info2 = ctx2.autotune_info(dh2, C)
    assert info2 is not None and info2["n_tried"] == 0
    assert (info2["chunk_rays"], info2["ctas_per_sm"]) == (info["chunk_rays"], info["ctas_per_sm"])
    out = np.zeros(C.tally_size)
    assert ctx2.poll(ctx2.submit(dh2, C, tally=out))["status"] == wg.WG_OK
    assert open(path).read() == text
    assert ctx2.autotune_info(dh2, C)["n_tried"] == 0
    dh2.destroy()
    ctx2.close()
