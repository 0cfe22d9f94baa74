"""Pins of the oracle's general mirrors (any normal, a tilt axis, an (x, y)
rectangle where the plane acts), which carry the paper's two-dimensional
pupil expansion (Results, "System Architecture": folding mirrors for one
direction of expansion, output mirrors for the other): the general form of a
PRMA design reproduces it, a mirror no ray meets inside its rectangle is
absent, fold and output reflections obey the mirror law in 3D, splitting
conserves energy and the MC estimate is its expectation, and the thickness
and tilt gradients match fixed-key differences."""
import numpy as np
import pytest

from paper_2601_04370_gb300 import workloads as W

from test_oracle_trace import _group_z


def _as_general(D):
    """The same PRMA planes written as general mirrors."""
    t = np.deg2rad(D.mirror_tilt_deg.astype(np.float64))
    inf = np.inf
    rows = [[-np.sin(a), 0.0, np.cos(a), x, 0.0, 0.5 * D.thickness_mm, 0.0, -1.0, 0.0, -inf, inf, -inf, inf, td]
            for a, x, td in zip(t, D.mirror_x_mm, D.mirror_tilt_deg)]
    return D.replace(mirror_geo=np.array(rows))


def _objective(ora, D, C, G):
    return float((ora.trace(D, C)["tally"] * G).sum())


@pytest.mark.parametrize("cfg", ["tiny", "rep"])
def test_general_form_of_a_prma_design_reproduces_it(ora, cfg):
    """Same planes up to the float32 rounding of the stored normal: the same
    paths for all but a handful of rays, the same tallies and gradients."""
    if cfg == "tiny":
        D, C = W.tiny(n_rays=4000)
    else:
        D, C = W.representative(n_rays=3000, n_layers=8)
        C = C.replace(fx_deg=[-12.0, 0.0, 9.0], fy_deg=[-6.0, 4.0], eb_nx=16, eb_ny=12)
    Dg = _as_general(D)
    a = ora.trace(D, C, records=True)
    b = ora.trace(Dg, C, records=True)
    same = (a["records"]["hash"] == b["records"]["hash"]) & (a["records"]["bin"] == b["records"]["bin"])
    assert same.mean() >= 0.999
    ta, tb = a["tally"], b["tally"]
    assert np.abs(ta - tb).sum() <= 2e-3 * np.abs(ta).sum()
    rng = np.random.default_rng(5)
    G = rng.normal(size=C.tally_shape)
    mask = same.astype(np.uint8)
    ga, gta = ora.trace_grad(D, C, G, mask=mask)
    gb, gtb = ora.trace_grad(Dg, C, G, mask=mask)
    assert np.linalg.norm(ga - gb) <= 1e-5 * np.linalg.norm(ga)
    assert np.linalg.norm(gta - gtb) <= 1e-5 * np.linalg.norm(gta)


def test_mirror_outside_its_rectangle_is_absent(ora):
    D, C = W.pupil_expander_small(n_rays=6000)
    ref = ora.trace(D, C)
    g = np.vstack([D.mirror_geo, D.mirror_geo[0]])
    g[-1, 9:13] = [200.0, 201.0, 200.0, 201.0]   # far outside the slab's reach
    L = int(D.n_layers[0])
    D2 = D.replace(mirror_x_mm=np.append(D.mirror_x_mm, 0.0), mirror_tilt_deg=np.append(D.mirror_tilt_deg, 45.0),
                   mirror_omega=np.append(D.mirror_omega, 0.5), n_layers=np.append(D.n_layers, L),
                   layer_mat=np.append(D.layer_mat, D.layer_mat[:L]), layer_d_nm=np.append(D.layer_d_nm, D.layer_d_nm[:L]),
                   pruned=np.append(D.pruned, D.pruned[:L]), mirror_geo=g)
    out = ora.trace(D2, C)
    assert np.array_equal(out["tally"], ref["tally"])
    assert out["stats"]["n_hits"] == ref["stats"]["n_hits"]
    # the same mirror with its rectangle over the fold band does act
    g2 = g.copy()
    g2[-1, 9:13] = D.mirror_geo[0, 9:13]
    g2[-1, 3] += 0.75
    out2 = ora.trace(D2.replace(mirror_geo=g2), C)
    assert out2["stats"]["n_hits"] > ref["stats"]["n_hits"]


def test_fold_and_output_reflections_follow_the_mirror_law(ora):
    """Every mirror event lies on its plane inside its rectangle; a reflection
    is d - 2 (d.N) N, which for the vertical 45 deg fold planes swaps d_x and
    d_y (the guided ray keeps its TIR angle)."""
    D, C = W.pupil_expander_small(n_rays=2000)
    g = D.mirror_geo.astype(np.float64)
    n_fold = int((g[:, 2] == 0.0).sum())
    seen = {"fold_r": 0, "out_r": 0, "t": 0}
    for ray in range(0, C.total_rays, 7):
        ev, _, _ = ora.trace_path(D, C, ray)
        for e in ev:
            if e["surf"] < 8:
                continue
            k = e["surf"] - 8
            N = g[k, 0:3] / np.linalg.norm(g[k, 0:3])   # normalized as both implementations do
            assert abs(np.dot(e["p"] - g[k, 3:6], N)) < 1e-9
            assert g[k, 9] <= e["p"][0] <= g[k, 10] and g[k, 11] <= e["p"][1] <= g[k, 12]
            d = e["d_in"]
            if e["refl"]:
                assert np.allclose(e["d_out"], d - 2 * np.dot(d, N) * N, atol=1e-12)
                if k < n_fold:
                    # up to the float32 rounding of the stored normal
                    assert np.allclose(e["d_out"], [d[1], d[0], d[2]], atol=1e-6)
                    seen["fold_r"] += 1
                else:
                    seen["out_r"] += 1
            else:
                assert np.allclose(e["d_out"], d, atol=0)
                seen["t"] += 1
    assert min(seen.values()) > 20, seen


def test_splitting_conserves_energy_in_the_expander(ora):
    D, C = W.pupil_expander_small(n_rays=300)
    s = ora.split(D, C, prune=0.0)
    assert abs(s["ledger"].sum() - C.total_rays) < 1e-10 * C.total_rays
    assert abs(s["tally"].sum() - s["ledger"][0]) < 1e-9 * max(1.0, s["ledger"][0])


def test_mc_expectation_equals_splitting_in_the_expander(ora):
    """omega = 0.5 on every mirror keeps the path weights O(1), so block
    z-scores of MC minus the splitting sum are meaningful."""
    D, C = W.pupil_expander_small(n_rays=20000)
    D = D.replace(mirror_omega=np.full(D.n_mirrors, 0.5, np.float32))
    s = ora.split(D, C, prune=1e-9)
    m = ora.trace(D, C, records=True)
    z, dead = _group_z(C, m["tally"], s["tally"], m["records"], block=4)
    assert len(z) >= 20
    assert z.max() < 5.0, z.max()
    assert (z ** 2).mean() < 1.8
    assert dead < 0.1


def test_expander_thickness_gradient_matches_fixed_key_differences(ora):
    D, C = W.pupil_expander_small(n_rays=1500)
    rng = np.random.default_rng(7)
    G = rng.normal(size=C.tally_shape)
    gd, _ = ora.trace_grad(D, C, G)
    base = D.layer_d_nm.astype(np.float64)

    def central(i, h):
        dp, dm = base.copy(), base.copy()
        dp[i] += h
        dm[i] -= h
        Dp, Dm = D.replace(), D.replace()
        Dp.layer_d_nm, Dm.layer_d_nm = dp, dm
        return (_objective(ora, Dp, C, G) - _objective(ora, Dm, C, G)) / (2 * h)

    h = 0.01
    for i in range(0, D.total_layers, 5):
        fd = (4 * central(i, h / 2) - central(i, h)) / 3
        assert abs(gd[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gd).max()), (i, gd[i], fd)


def test_expander_tilt_gradient_matches_differences_on_stable_rays(ora):
    """A tilt turns a general mirror about its own axis (z for the folds, x
    for the outputs); interior derivative on rays whose path is unchanged."""
    D, C = W.pupil_expander_small(n_rays=3000)
    rng = np.random.default_rng(8)
    G = rng.normal(size=C.tally_shape)
    Gf = G.reshape(-1)
    h = 1e-4
    base = ora.trace(D, C, records=True)["records"]
    for k in range(D.n_mirrors):
        tp = D.mirror_tilt_deg.astype(np.float64).copy()
        tm = tp.copy()
        tp[k] += h
        tm[k] -= h
        Dp, Dm = D.replace(), D.replace()
        Dp.mirror_tilt_deg, Dm.mirror_tilt_deg = tp, tm
        rp = ora.trace(Dp, C, records=True)["records"]
        rm = ora.trace(Dm, C, records=True)["records"]
        stable = ((rp["hash"] == base["hash"]) & (rm["hash"] == base["hash"]) &
                  (rp["bin"] == base["bin"]) & (rm["bin"] == base["bin"]))
        assert stable.mean() > 0.97
        tallied = stable & (base["bin"] >= 0)
        fd = (float((Gf[rp["bin"][tallied]] * rp["I"][tallied]).sum()) -
              float((Gf[rm["bin"][tallied]] * rm["I"][tallied]).sum())) / (2 * h)
        _, gt = ora.trace_grad(D, C, G, mask=stable.astype(np.uint8))
        assert abs(gt[k] - fd) <= 2e-5 * max(abs(fd), 1.0), (k, gt[k], fd)
