"""Serving runtime (wg_submit / wg_poll / wg_cancel): design evaluations
batched into fused launches give the results of direct calls; a request's
result does not depend on what it was batched with; cancellation, admission
by device memory and graph replay."""
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


def _direct_forward(ctx, dh, C):
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, t)
    return t.cpu().numpy()


def _close(a, b, tol=1e-5):
    """Tallies of the same rays: the FP32 shared-memory partial sums depend on
    the chunking and the order of the additions (2^-24 per term)."""
    return np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300)


def _designs(n, rays):
    out = []
    for D, C in W.batching(n_designs=n, seed=4):
        out.append((D, C.replace(n_rays=rays)))
    return out


def test_served_forward_matches_direct_calls(wg):
    ctx = wg.Context(0)
    jobs = _designs(6, 1728 * 6)
    dhs = [ctx.create_design(D) for D, _ in jobs]
    outs = [np.zeros(C.tally_size) for _, C in jobs]
    tickets = [ctx.submit(dh, C, tally=o) for dh, (_, C), o in zip(dhs, jobs, outs)]
    res = [ctx.poll(t) for t in tickets]
    assert all(r["status"] == wg.WG_OK for r in res)
    assert max(r["batch_size"] for r in res) >= 1
    for dh, (D, C), o, r in zip(dhs, jobs, outs, res):
        ref = _direct_forward(ctx, dh, C)
        assert r["stats"]["n_rays"] == C.total_rays
        assert _close(o, ref.reshape(-1))
    for dh in dhs:
        dh.destroy()
    ctx.close()


def test_result_independent_of_batch_mix(wg):
    """The same request served alone and inside a batch of other designs."""
    jobs = _designs(5, 1728 * 4)
    ctx = wg.Context(0)
    dhs = [ctx.create_design(D) for D, _ in jobs]
    alone = np.zeros(jobs[0][1].tally_size)
    ctx.poll(ctx.submit(dhs[0], jobs[0][1], tally=alone))
    outs = [np.zeros(C.tally_size) for _, C in jobs]
    tickets = [ctx.submit(dh, C, tally=o) for dh, (_, C), o in zip(dhs, jobs, outs)]
    res = [ctx.poll(t) for t in tickets]
    assert all(r["status"] == wg.WG_OK for r in res)
    assert _close(outs[0], alone)
    for dh in dhs:
        dh.destroy()
    ctx.close()


def test_served_loss_and_gradient_match_direct_calls(wg):
    ctx = wg.Context(0)
    D, C = W.representative(n_rays=1728 * 8)
    dh = ctx.create_design(D)
    loss = np.zeros(4)
    grad = np.zeros(D.total_layers)
    r = ctx.poll(ctx.submit(dh, C, kind=wg.REQ_LOSS_GRAD, grad=grad, loss=loss))
    assert r["status"] == wg.WG_OK
    t = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, t)
    G = torch.zeros_like(t)
    L = ctx.loss(dh, C, t, G)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    ctx.trace_backward(dh, C, G, g)
    assert abs(loss[0] - L[0]) <= 1e-5 * abs(L[0])
    gg = g.cpu().numpy()
    assert np.abs(grad - gg).max() <= 1e-4 * np.abs(gg).max()
    dh.destroy()
    ctx.close()


def test_cancel_and_poll_states(wg):
    ctx = wg.Context(0, max_slots=1)
    jobs = _designs(3, 1728 * 64)
    dhs = [ctx.create_design(D) for D, _ in jobs]
    tickets = [ctx.submit(dhs[i % 3], jobs[i % 3][1]) for i in range(8)]
    ctx.cancel(tickets[-1])
    ctx.cancel(tickets[-2])
    res = [ctx.poll(t) for t in tickets]
    assert res[-1]["status"] == wg.WG_ECANCELED and res[-2]["status"] == wg.WG_ECANCELED
    assert all(r["status"] == wg.WG_OK for r in res[:-2])
    with pytest.raises(wg.WGError) as e:
        ctx.poll(tickets[0])
    assert e.value.status == wg.WG_ENOTFOUND
    for dh in dhs:
        dh.destroy()
    ctx.close()


def test_admission_by_device_memory(wg):
    ctx = wg.Context(0, hbm_budget_bytes=1 << 20)
    D, C = W.representative(n_rays=1728 * 4)
    dh = ctx.create_design(D)
    with pytest.raises(wg.WGError) as e:
        ctx.submit(dh, C)
    assert e.value.status == wg.WG_ENOMEM
    dh.destroy()
    ctx.close()


def test_identical_batch_replays_graph(wg):
    """A batch composition runs directly the first time, is captured the
    second time and replays the captured graph from the third on; all three
    give the same tally."""
    ctx = wg.Context(0, max_slots=1)
    D, C = W.representative(n_rays=1728 * 4)
    dh = ctx.create_design(D)
    a, b, c = np.zeros(C.tally_size), np.zeros(C.tally_size), np.zeros(C.tally_size)
    r1 = ctx.poll(ctx.submit(dh, C, tally=a))
    r2 = ctx.poll(ctx.submit(dh, C, tally=b))
    r3 = ctx.poll(ctx.submit(dh, C, tally=c))
    assert all(r["status"] == wg.WG_OK for r in (r1, r2, r3))
    assert not r1["graph_replayed"] and not r2["graph_replayed"] and r3["graph_replayed"]
    assert _close(a, b) and _close(a, c)
    dh.destroy()
    ctx.close()


def test_forward_batch_matches_direct_calls_and_replays_its_graph(wg):
    """wg_trace_forward_batch: designs of uneven mirror and layer counts
    (fast and accurate evaluations, pruned layers) in fused launches equal
    their direct traces; the same composition runs directly the first time,
    is captured the second time and replays the graph from the third."""
    jobs = _designs(8, 1728 * 4)
    ctx = wg.Context(0)
    dhs = [ctx.create_design(D) for D, _ in jobs]
    ts = [torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda") for _, C in jobs]
    reps = []
    for _ in range(3):
        st, rep = ctx.trace_forward_batch(dhs, [C for _, C in jobs], ts)
        reps.append(rep)
        assert all(s["n_rays"] == C.total_rays for s, (_, C) in zip(st, jobs))
    assert reps == [False, False, True]
    for dh, (D, C), t in zip(dhs, jobs, ts):
        assert _close(t.cpu().numpy(), _direct_forward(ctx, dh, C))
    for dh in dhs:
        dh.destroy()
    ctx.close()
