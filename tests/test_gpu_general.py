"""GPU parity on general mirrors, the geometry of the paper's
two-dimensional pupil expansion (Results, "System Architecture": folding
mirrors for one direction of expansion, output mirrors for the other):
per-ray paths, tallies, thickness and tilt gradients against the FP64
oracle on the same keys, the general form of a PRMA design, rays sampled
from the full-size expander in the benchmark's launch shape, the coating
table, and served requests that batch general and PRMA designs."""
import numpy as np
import pytest

from paper_2601_04370_gb300 import workloads as W

from test_gpu_parity import tilt_compare, _dev, _grad_compare, compare, ctx, run_gpu  # noqa: F401 (fixture)
from test_oracle_general import _as_general

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_expander_small_trace_matches_oracle(ctx, ora):
    D, C = W.pupil_expander_small()
    g = run_gpu(ctx, D, C)
    o = ora.trace(D, C, records=True)
    compare(C, g, o)
    assert g["stats"]["n_hits"] == o["stats"]["n_hits"] or abs(g["stats"]["n_hits"] - o["stats"]["n_hits"]) <= 64
    led = g["stats"]["ledger"]
    assert np.abs(led - o["ledger"]).max() <= 1e-4 * C.total_rays


def test_general_form_of_a_prma_design_on_the_gpu(ctx, ora):
    """The PRMA planes written as general mirrors (every plane tested, the
    rectangle test on): the oracle's paths and tallies, and the PRMA run's."""
    D, C = W.representative(n_rays=1728 * 4, n_layers=8)
    Dg = _as_general(D)
    g = run_gpu(ctx, Dg, C)
    compare(C, g, ora.trace(Dg, C, records=True))
    p = run_gpu(ctx, D, C, records=False)
    assert np.abs(g["tally"] - p["tally"]).sum() <= 2e-3 * np.abs(p["tally"]).sum()


@pytest.mark.parametrize("tilts", [False, True])
def test_expander_gradients_match_oracle(ctx, ora, tilts):
    D, C = W.pupil_expander_small()
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, tally)
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gt = np.zeros(D.n_mirrors) if tilts else None
    st = ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    assert st["overflow"] == 0 and st["n_nonfinite"] == 0
    ref_d, ref_t = ora.trace_grad(D, C, G.cpu().numpy())
    _grad_compare(g.cpu().numpy(), ref_d)
    if tilts:
        assert np.all(np.isfinite(gt))
        tilt_compare(gt, ref_t)
    dh.destroy()


def test_expander_tilt_update_matches_oracle(ctx, ora):
    """wg_set_params turns general mirrors about their own axes."""
    D, C = W.pupil_expander_small()
    dh = ctx.create_design(D)
    t2 = D.mirror_tilt_deg.copy()
    t2[1] += 0.4      # a fold mirror about z
    t2[-1] -= 0.3     # an output mirror about x
    dh.set_params(tilt_deg=t2)
    D2 = D.replace(mirror_tilt_deg=t2)
    g = run_gpu(ctx, D2, C, dh=dh)
    compare(C, g, ora.trace(D2, C, records=True))
    dh.destroy()


def test_expander_coating_table_matches_oracle(ctx, ora):
    D, C = W.pupil_expander_small()
    C = C.replace(lut_bins=1024)
    g = run_gpu(ctx, D, C)
    compare(C, g, ora.trace(D, C, records=True))


def test_full_size_expander_sampled(ctx, ora):
    """46 mirrors, 23 layers, 9 wavelengths, 16x16 fields, 1e7 rays in the
    launch shape the benchmark times: rays sampled across the whole range
    match the oracle one by one; the tally is the records' eyebox
    contributions; no tape or record overflow."""
    D, C = W.pupil_expander()
    g = run_gpu(ctx, D, C)
    rg = g["records"]
    N = C.total_rays
    assert g["stats"]["n_rays"] == N and len(rg) == N
    assert rg["n_hits"].max() <= 128
    rng = np.random.default_rng(1)
    starts = np.sort(rng.choice(N - 32, 40, replace=False))
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
    assert np.quantile(np.concatenate(dI), 0.99) <= 1e-4
    t = g["tally"].reshape(-1)
    ok = rg["bin"] >= 0
    from_recs = np.bincount(rg["bin"][ok], weights=rg["I"][ok].astype(np.float64), minlength=t.size)
    assert np.abs(from_recs - t).max() <= 1e-5 * max(1.0, t.max())
    w = rg["w"].astype(np.float64)
    assert abs(g["stats"]["ledger"].sum() - N) <= 6 * np.sqrt((w ** 2).sum())


def test_general_geometry_is_validated(ctx):
    """The descriptor's general rows are checked before anything is uploaded:
    unit normal and axis, axis perpendicular to the normal, a non-empty
    rectangle, finite values."""
    from paper_2601_04370_gb300 import wg
    D, _ = W.pupil_expander_small()
    bad = []
    g = D.mirror_geo.copy(); g[0, 0:3] *= 1.1; bad.append(g)            # normal not unit
    g = D.mirror_geo.copy(); g[1, 6:9] = [1.0, 0.0, 0.0]; bad.append(g)  # axis not perpendicular (fold normal has x)
    g = D.mirror_geo.copy(); g[2, 9:11] = [3.0, 2.0]; bad.append(g)      # x0 > x1
    g = D.mirror_geo.copy(); g[3, 4] = np.nan; bad.append(g)             # pivot not finite
    for gb in bad:
        with pytest.raises(wg.WGError) as e:
            ctx.create_design(D.replace(mirror_geo=gb))
        assert e.value.status == wg.WG_EINVAL


def test_served_general_and_prma_designs_match_direct_calls(ctx):
    Dg, Cg = W.pupil_expander_small()
    Dp, Cp = W.representative(n_rays=1728 * 4, n_layers=8)
    jobs = [(Dg, Cg), (Dp, Cp), (Dg, Cg.replace(seed=99))]
    dhs = [ctx.create_design(D) for D, _ in jobs]
    outs = [np.zeros(C.tally_size) for _, C in jobs]
    tickets = [ctx.submit(dh, C, tally=o) for dh, (_, C), o in zip(dhs, jobs, outs)]
    res = [ctx.poll(t) for t in tickets]
    for dh, (D, C), o, r in zip(dhs, jobs, outs, res):
        assert r["status"] == 0
        ref = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
        ctx.trace_forward(dh, C, ref)
        ref = ref.cpu().numpy().reshape(-1)
        assert np.abs(o - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-300)
    for dh in dhs:
        dh.destroy()


def test_tilt_gradient_with_rays_leaving_along_the_normal(ctx, ora):
    """The 0 deg field leaves the slab along the face normal, where the face
    s/p basis turns at a rate ~1/h (h = |(d_x, d_y)| -> 0); the tangent pass
    carries projections of the field tangent, so the exit term stays exact."""
    D, C = W.representative(n_rays=1728 * 4, n_layers=8)
    C = C.replace(fx_deg=[-6.0, 0.0, 6.0], fy_deg=[-4.0, 0.0, 4.0], eb_nx=24, eb_ny=16)
    dh = ctx.create_design(D)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    ctx.trace_forward(dh, C, tally)
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G)
    g = torch.zeros(D.total_layers, dtype=torch.float64, device="cuda")
    gt = np.zeros(D.n_mirrors)
    ctx.trace_backward(dh, C, G, g, grad_tilt=gt)
    _, ref_t = ora.trace_grad(D, C, G.cpu().numpy())
    tilt_compare(gt, ref_t)
    dh.destroy()


def test_expander_omega_trace_matches_oracle(ctx, ora):
    """The geometric trace of the omega pre-optimization with general mirrors
    (fold and output reflections in 3D) against the oracle's."""
    D, C = W.pupil_expander_small(n_rays=40_000)
    om = np.linspace(0.2, 0.8, D.n_mirrors).astype(np.float32)
    dh = ctx.create_design(D)
    dh.set_omega(om)
    Do = D.replace(mirror_omega=om)
    tally = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    G = torch.zeros_like(tally)
    ctx.loss(dh, C, tally, G, w_f=0.0, w_e=0.0)
    g = np.zeros(D.n_mirrors)
    ctx.omega_trace(dh, C, tally, G, g)
    ref_t, ref_g = ora.geo_trace(Do, C, G=G.cpu().numpy())
    t = tally.cpu().numpy()
    assert np.abs(t - ref_t).max() <= 1e-4 * np.abs(ref_t).max()
    assert np.linalg.norm(g - ref_g) <= 1e-3 * np.linalg.norm(ref_g), (g, ref_g)
    dh.destroy()


def test_expander_noalloc_forward_matches_trace_forward(ctx):
    D, C = W.pupil_expander_small()
    dh = ctx.create_design(D)
    a = torch.zeros(C.tally_shape, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    ctx.trace_forward(dh, C, a)
    ctx.trace_forward_noalloc(dh, C, b)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    dh.destroy()
