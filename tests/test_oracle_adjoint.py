"""Pins for the oracle's adjoint (reverse-mode through the traced paths and
the transfer matrices) against central finite differences, and for the FP64
loss head (Results, Eq. 1) against hand-computed values and finite
differences."""
import numpy as np
import pytest

from paper_2601_04370_gb300 import workloads as W

N_GLASS, N_SIO2, N_TIO2, N_TA2O5 = 1.71, 1.46, 2.35, 2.1


def _stack(seed, L):
    rng = np.random.default_rng(seed)
    n = np.array([(N_SIO2, N_TIO2, N_TA2O5)[i % 3] for i in range(L)])
    return n, rng.uniform(10, 200, L)


def _f(ora, n, d, lam, c0, As, Ap, which):
    rs, rp, ts, tp = ora.tmm(N_GLASS, N_GLASS, n, d, lam, c0)
    cs, cp = (rs, rp) if which == "r" else (ts, tp)
    return 2 * (As * cs + Ap * cp).real


@pytest.mark.parametrize("deg", [0.0, 25.0, 75.0])
@pytest.mark.parametrize("which", ["r", "t"])
def test_tmm_gradient_matches_central_differences(ora, deg, which):
    n, d = _stack(4, 12)
    c0, lam = np.cos(np.radians(deg)), 532.0
    As, Ap = 0.3 - 0.7j, -0.45 + 0.2j
    g, gc, f = ora.tmm_grad(N_GLASS, n, d, lam, c0, As, Ap, which)
    assert abs(f - _f(ora, n, d, lam, c0, As, Ap, which)) < 1e-14
    h = 0.01
    for l in range(len(n)):
        dp, dm = d.copy(), d.copy()
        dp[l] += h
        dm[l] -= h
        fd = (_f(ora, n, dp, lam, c0, As, Ap, which) - _f(ora, n, dm, lam, c0, As, Ap, which)) / (2 * h)
        assert abs(g[l] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (l, g[l], fd)
    hc = 1e-6
    fdc = (_f(ora, n, d, lam, c0 + hc, As, Ap, which) - _f(ora, n, d, lam, c0 - hc, As, Ap, which)) / (2 * hc)
    assert abs(gc - fdc) <= 1e-5 * max(1.0, abs(fdc))


def _objective(ora, D, C, G):
    return float((ora.trace(D, C)["tally"] * G).sum())


def test_trace_thickness_gradient_matches_fixed_key_differences(ora):
    """With the reparameterized sampling the path does not depend on the
    thicknesses, so the fixed-key objective sum(G * tally) is smooth in d and
    central differences (h = 0.01 nm) agree with the adjoint."""
    D, C = W.tiny(n_rays=4000)
    rng = np.random.default_rng(1)
    G = rng.normal(size=C.tally_shape)
    gd, gt = ora.trace_grad(D, C, G)
    assert gd.shape == (D.total_layers,) and gt.shape == (D.n_mirrors,)
    base = D.layer_d_nm.astype(np.float64)

    def central(i, h):
        dp, dm = base.copy(), base.copy()
        dp[i] += h
        dm[i] -= h
        Dp, Dm = D.replace(), D.replace()
        Dp.layer_d_nm, Dm.layer_d_nm = dp, dm   # FP64 thicknesses straight to the oracle
        return (_objective(ora, Dp, C, G) - _objective(ora, Dm, C, G)) / (2 * h)

    h = 0.01
    for i in range(D.total_layers):
        # Richardson extrapolation of central differences at h and h/2 (error O(h^4))
        fd = (4 * central(i, h / 2) - central(i, h)) / 3
        assert abs(gd[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gd).max()), (i, gd[i], fd)


def test_pruned_layers_get_zero_gradient(ora):
    D, C = W.tiny(n_rays=2000)
    pr = D.pruned.copy()
    pr[[1, 10]] = 1
    d = D.layer_d_nm.copy()
    d[[1, 10]] = 0.0
    D2 = D.replace(pruned=pr, layer_d_nm=d)
    G = np.ones(C.tally_shape)
    gd, _ = ora.trace_grad(D2, C, G)
    assert gd[1] == 0.0 and gd[10] == 0.0
    assert np.count_nonzero(gd) >= D.total_layers - 2 - 2
    # a pruned layer is the same as an absent one
    a = ora.trace(D2, C)["tally"]
    keep = pr == 0
    D3 = D2.replace(n_layers=np.array([7, 7]), layer_mat=D2.layer_mat[keep], layer_d_nm=d[keep],
                    pruned=np.zeros(14, np.uint8))
    b = ora.trace(D3, C)["tally"]
    assert np.abs(a - b).max() < 1e-12


def test_trace_tilt_gradient_matches_differences_on_stable_rays(ora):
    """Tilt moves the geometry, so the path of a few rays changes under +-h;
    the comparison is restricted to rays whose surface/decision sequence and
    eyebox bin are the same at -h, 0 and +h (interior derivative)."""
    D, C = W.tiny(n_rays=4000)
    rng = np.random.default_rng(2)
    G = rng.normal(size=C.tally_shape)
    Gf = G.reshape(-1)
    h = 1e-4  # degrees
    base = ora.trace(D, C, records=True)["records"]
    for k in range(D.n_mirrors):
        tp, tm = D.mirror_tilt_deg.astype(np.float64).copy(), D.mirror_tilt_deg.astype(np.float64).copy()
        tp[k] += h
        tm[k] -= h
        Dp, Dm = D.replace(), D.replace()
        Dp.mirror_tilt_deg, Dm.mirror_tilt_deg = tp, tm
        rp = ora.trace(Dp, C, records=True)["records"]
        rm = ora.trace(Dm, C, records=True)["records"]
        stable = ((rp["hash"] == base["hash"]) & (rm["hash"] == base["hash"]) &
                  (rp["bin"] == base["bin"]) & (rm["bin"] == base["bin"]))
        assert stable.mean() > 0.98
        tallied = stable & (base["bin"] >= 0)
        fp = float((Gf[rp["bin"][tallied]] * rp["I"][tallied]).sum())
        fm = float((Gf[rm["bin"][tallied]] * rm["I"][tallied]).sum())
        fd = (fp - fm) / (2 * h)
        gd, gt = ora.trace_grad(D, C, G, mask=stable.astype(np.uint8))
        assert abs(gt[k] - fd) <= 2e-5 * max(abs(fd), 1.0), (k, gt[k], fd)


# ---------------- loss head ----------------

def test_loss_of_uniform_image(ora):
    D, C = W.tiny()
    t = np.full(C.tally_shape, 2.0)
    L, parts, G = ora.loss_and_grad(t, D.dims, C)
    masks = ora.pupil_masks(D.dims, C)
    per_pupil = masks.reshape(len(masks), -1).sum(1) * 2.0 / C.n_cell
    assert parts["u_fov"] == 0.0                  # every field sees the same pupil value
    assert abs(parts["I_mean"] - per_pupil.mean()) < 1e-15
    cv_e = per_pupil.std() / per_pupil.mean()       # pupils differ only by their bin counts
    assert abs(parts["u_eyebox"] - cv_e) < 1e-13
    assert abs(L - (-per_pupil.mean() + 10.0 * 0.0 + 3.0 * cv_e)) < 1e-13


def test_pupils_are_3x3_discs_of_4mm(ora):
    D, C = W.representative(n_rays=1000)
    m = ora.pupil_masks(D.dims, C)
    assert m.shape == (9, 48, 64)
    # bin pitch 10/64 x 8/48 mm; a 4 mm disc covers about pi*4 mm^2
    area = m.reshape(9, -1).sum(1) * (10 / 64) * (8 / 48)
    assert np.all(np.abs(area - np.pi * 4.0) < 0.35)
    D2, C2 = W.tiny()
    m2 = ora.pupil_masks(D2.dims, C2)
    assert m2.shape == (3, 1, 64) and np.all(m2.reshape(3, -1).sum(1) == 32)


def test_loss_hand_example(ora):
    """Two fields, one wavelength, 1D eyebox; the three 4 mm pupils overlap
    (intervals [-4,0], [-2,2], [0,4] mm around the centre), so one value is
    placed in each quarter A, B, C, D and the pupils see A+B, B+C, C+D."""
    D, C = W.tiny()
    C = C.replace(fx_deg=[0.0, 5.0], n_rays=2)            # one ray per cell
    masks = ora.pupil_masks(D.dims, C)[:, 0, :]
    quarter = {"A": 8, "B": 24, "C": 40, "D": 56}
    assert masks[:, quarter["A"]].tolist() == [True, False, False]
    assert masks[:, quarter["B"]].tolist() == [True, True, False]
    assert masks[:, quarter["C"]].tolist() == [False, True, True]
    assert masks[:, quarter["D"]].tolist() == [False, False, True]
    t = np.zeros(C.tally_shape)
    for f, (a, b, c, d) in enumerate([(1.0, 0.0, 2.0, 1.0), (2.0, 1.0, 1.0, 0.0)]):
        for q, v in zip("ABCD", (a, b, c, d)):
            t[0, 0, f, 0, quarter[q]] = v
    # pupil values: field 0 -> (1, 2, 3), field 1 -> (3, 2, 1)
    L, parts, G = ora.loss_and_grad(t, D.dims, C)
    assert abs(parts["I_mean"] - 2.0) < 1e-15
    # CV over fields per pupil: pupils 0 and 2 see {1,3}: std 1, mean 2 -> 0.5; pupil 1: 0
    assert abs(parts["u_fov"] - (0.5 + 0.0 + 0.5) / 3) < 1e-15
    # CV over pupils per field: {1,2,3}: std sqrt(2/3), mean 2
    assert abs(parts["u_eyebox"] - np.sqrt(2.0 / 3.0) / 2.0) < 1e-15
    assert abs(L - (-2.0 + 10.0 / 3.0 + 3.0 * np.sqrt(2.0 / 3.0) / 2.0)) < 1e-14


@pytest.mark.parametrize("kind", ["cv", "variance"])
def test_loss_gradient_matches_differences(ora, kind):
    D, C = W.tiny(n_rays=2000)
    t = ora.trace(D, C)["tally"]
    L, _, G = ora.loss_and_grad(t, D.dims, C, kind=kind)
    rng = np.random.default_rng(0)
    flat = t.reshape(-1)
    def central(i, h):
        tp, tm = flat.copy(), flat.copy()
        tp[i] += h
        tm[i] -= h
        return (ora.loss_and_grad(tp.reshape(t.shape), D.dims, C, kind=kind)[0] -
                ora.loss_and_grad(tm.reshape(t.shape), D.dims, C, kind=kind)[0]) / (2 * h)

    for i in rng.choice(flat.size, 40, replace=False):
        h = 1e-3 * max(1.0, abs(flat[i]))
        fd = (4 * central(i, h / 2) - central(i, h)) / 3
        assert abs(G.reshape(-1)[i] - fd) <= 1e-6 * max(abs(fd), 1e-6), (i, G.reshape(-1)[i], fd)
