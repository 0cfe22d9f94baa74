"""Pins for the oracle's Monte Carlo trace: brute-force ray splitting, energy
conservation, omega independence, polarization linearity and geometric
invariants of every ray path (Methods, "Polarization ray tracing" and
"Differentiable Monte Carlo non-sequential ray tracing")."""
import numpy as np
import pytest

from paper_2601_04370_gb300 import workloads as W

TAG_GEN = 0x47454E30


def small_3d(n_layers=8, n_rays=6000, seed=21):
    D, C = W.representative(n_rays=n_rays, seed=seed, n_layers=n_layers)
    C = C.replace(lam_nm=[532.0], fx_deg=[-12.0, 0.0, 9.0], fy_deg=[-6.0, 4.0], eb_nx=16, eb_ny=12)
    return D, C


def small_3d_balanced(n_rays=24000, seed=101, K=3, omega=0.5):
    """3D, K mirrors with omega = 0.5: path weights stay O(1), so the MC
    error is close to Gaussian and a z-test is meaningful."""
    D, C = small_3d(n_rays=n_rays, seed=seed)
    L = int(D.n_layers[0])
    D = D.replace(mirror_x_mm=D.mirror_x_mm[:K], mirror_tilt_deg=D.mirror_tilt_deg[:K],
                  mirror_omega=np.full(K, omega, np.float32), n_layers=D.n_layers[:K],
                  layer_mat=D.layer_mat[:L * K], layer_d_nm=D.layer_d_nm[:L * K],
                  pruned=D.pruned[:L * K], x_end_mm=float(D.mirror_x_mm[K - 1] + 10.0))
    C = C.replace(eb_cx_mm=float(D.mirror_x_mm.mean()))
    return D, C


def _group_z(C, mc, ref, recs, block=8, min_count=30):
    """z-scores of |MC - splitting| over blocks of block x block eyebox bins
    per cell. sigma^2 = sum of squared per-ray contributions in the block (an
    upper bound of the MC variance); blocks with fewer than min_count
    contributions are reported separately (their expected energy)."""
    nl, nfy, nfx, ny, nx = C.tally_shape
    gx, gy = -(-nx // block), -(-ny // block)
    cell = np.arange(nl * nfy * nfx)[:, None, None]
    ey = np.arange(ny)[None, :, None] // block
    ex = np.arange(nx)[None, None, :] // block
    g = (cell * gy * gx + ey * gx + ex).reshape(-1)
    ng = int(g.max()) + 1
    sm = np.bincount(g, weights=ref.reshape(-1), minlength=ng)
    mm = np.bincount(g, weights=mc.reshape(-1), minlength=ng)
    ok = recs["bin"] >= 0
    var = np.bincount(g[recs["bin"][ok]], weights=recs["I"][ok] ** 2, minlength=ng)
    cnt = np.bincount(g[recs["bin"][ok]], minlength=ng)
    live = cnt >= min_count
    z = np.abs(mm - sm)[live] / np.sqrt(var[live])
    return z, sm[~live].sum() / max(sm.sum(), 1e-300)


@pytest.mark.parametrize("cfg", ["tiny", "small3d"])
def test_splitting_conserves_energy(ora, cfg):
    D, C = W.tiny() if cfg == "tiny" else small_3d(n_rays=1500)
    s = ora.split(D, C)
    assert abs(s["ledger"].sum() - C.total_rays) < 1e-11 * C.total_rays
    assert abs(s["tally"].sum() - s["ledger"][0]) < 1e-9 * max(1.0, s["ledger"][0])


@pytest.mark.parametrize("omega", [None, (0.3, 0.3), (0.7, 0.7), (0.45, 0.6)])
def test_mc_expectation_equals_splitting(ora, omega):
    """E[MC tally] is the splitting sum over the same launch points; the MC
    estimate is unbiased for any omega (Eq. 5 rescaling)."""
    D, C = W.tiny(n_rays=40000)
    if omega is not None:
        D = D.replace(mirror_omega=np.array(omega, dtype=np.float32))
    s = ora.split(D, C)
    m = ora.trace(D, C, records=True)
    z, dead = _group_z(C, m["tally"], s["tally"], m["records"])
    assert len(z) >= 15
    assert z.max() < 4.5, z.max()
    assert (z ** 2).mean() < 1.5
    assert dead < 0.01
    tot = m["records"]["I"]
    assert abs(tot.sum() - s["tally"].sum()) < 4 * np.sqrt((tot ** 2).sum())


@pytest.mark.parametrize("seed", [101, 102])
def test_mc_expectation_equals_splitting_3d(ora, seed):
    D, C = small_3d_balanced(seed=seed)
    s = ora.split(D, C)
    m = ora.trace(D, C, records=True)
    z, dead = _group_z(C, m["tally"], s["tally"], m["records"], block=4)
    assert len(z) >= 30
    assert z.max() < 5.0, z.max()
    assert (z ** 2).mean() < 1.6
    assert dead < 0.08
    assert abs(m["ledger"].sum() - C.total_rays) < 5 * np.sqrt((m["records"]["w"] ** 2).sum())


def test_unpolarized_pair_is_mean_of_s_and_p(ora):
    """Incoherent sum: the s+p pair gives (I_s + I_p)/2 exactly (same keys)."""
    for D, C in (W.tiny(n_rays=3000), small_3d(n_rays=3000)):
        tp = ora.trace(D, C.replace(pol=W.POL_PAIR))["tally"]
        ts = ora.trace(D, C.replace(pol=W.POL_S))["tally"]
        tq = ora.trace(D, C.replace(pol=W.POL_P))["tally"]
        assert np.abs(tp - 0.5 * (ts + tq)).max() < 1e-12 * max(1.0, tp.max())


def _phi(ora, C, rays):
    return np.array([np.pi * (ora.philox([r & 0xFFFFFFFF, r >> 32, 0, TAG_GEN],
                                         [C.seed & 0xFFFFFFFF, C.seed >> 32])[2] >> 8) * 2.0 ** -24
                     for r in rays])


def test_2d_s_and_p_never_mix(ora):
    """In 2D the s direction is y at every surface, so a linear state at angle
    phi gives exactly cos^2 phi I_s + sin^2 phi I_p per ray (no cross term)."""
    D, C = W.tiny(n_rays=2000)
    rl = ora.trace(D, C.replace(pol=W.POL_RANDOM_LINEAR), records=True)["records"]
    rs = ora.trace(D, C.replace(pol=W.POL_S), records=True)["records"]
    rp = ora.trace(D, C.replace(pol=W.POL_P), records=True)["records"]
    phi = _phi(ora, C, range(C.total_rays))
    want = np.cos(phi) ** 2 * rs["I"] + np.sin(phi) ** 2 * rp["I"]
    assert np.abs(rl["I"] - want).max() < 1e-12


def test_3d_linear_states_do_mix(ora):
    """In 3D the s/p bases rotate between surfaces, so the cross term is not
    zero for some rays (guards against a tracer that drops the rotation)."""
    D, C = small_3d(n_rays=1200)
    rl = ora.trace(D, C.replace(pol=W.POL_RANDOM_LINEAR), records=True)["records"]
    rs = ora.trace(D, C.replace(pol=W.POL_S), records=True)["records"]
    rp = ora.trace(D, C.replace(pol=W.POL_P), records=True)["records"]
    phi = _phi(ora, C, range(C.total_rays))
    want = np.cos(phi) ** 2 * rs["I"] + np.sin(phi) ** 2 * rp["I"]
    assert np.abs(rl["I"] - want).max() > 1e-6


def test_thread_count_does_not_change_result(ora):
    D, C = W.tiny(n_rays=4000)
    a = ora.trace(D, C, nthreads=1)
    b = ora.trace(D, C, nthreads=5)
    assert np.abs(a["tally"] - b["tally"]).max() < 1e-12
    assert a["stats"] == b["stats"]


def test_event_cap_books_truncated_energy(ora):
    D, C = W.tiny(n_rays=2000)
    C = C.replace(max_events=4)
    s = ora.split(D, C)
    assert s["ledger"][5] > 0
    assert abs(s["ledger"].sum() - C.total_rays) < 1e-10 * C.total_rays
    m = ora.trace(D, C, records=True)
    assert np.all(m["records"]["n_events"] <= 4)
    assert m["ledger"][5] > 0


# ---------------- geometry of single paths ----------------

def _surface_residual(D, ev):
    """Signed distance of the event position from its surface plane."""
    p = ev["p"]
    s = int(ev["surf"])
    a = np.radians(D.ic_tilt_deg)
    if s == 0:
        return p[2]
    if s == 1:
        return p[2] - D.thickness_mm
    if s == 2:
        return -np.sin(a) * p[0] + np.cos(a) * p[2]
    if s == 3:
        return p[0] - D.x_end_mm
    if s == 4:
        return p[1] + 0.5 * D.width_mm
    if s == 5:
        return p[1] - 0.5 * D.width_mm
    k = s - 8
    t = np.radians(float(D.mirror_tilt_deg[k]))
    N = np.array([-np.sin(t), 0.0, np.cos(t)])
    return float(np.dot(p - np.array([D.mirror_x_mm[k], 0.0, 0.5 * D.thickness_mm]), N))


def _planes(D):
    a = np.radians(D.ic_tilt_deg)
    out = [(0, np.array([0, 0, 1.0]), 0.0), (1, np.array([0, 0, 1.0]), D.thickness_mm),
           (2, np.array([-np.sin(a), 0, np.cos(a)]), 0.0), (3, np.array([1.0, 0, 0]), D.x_end_mm)]
    if D.dims == 3:
        out += [(4, np.array([0, 1.0, 0]), -0.5 * D.width_mm), (5, np.array([0, 1.0, 0]), 0.5 * D.width_mm)]
    for k in range(D.n_mirrors):
        t = np.radians(float(D.mirror_tilt_deg[k]))
        N = np.array([-np.sin(t), 0, np.cos(t)])
        out.append((8 + k, N, float(np.dot(N, [D.mirror_x_mm[k], 0, 0.5 * D.thickness_mm]))))
    return out


@pytest.mark.parametrize("cfg", ["tiny", "small3d"])
def test_path_invariants(ora, cfg):
    D, C = W.tiny() if cfg == "tiny" else small_3d(n_rays=600)
    n = D.n_slab
    planes = _planes(D)
    rng = np.random.default_rng(0)
    for ray in rng.choice(C.total_rays, 150, replace=False):
        ev, cat, I = ora.trace_path(D, C, int(ray))
        a = np.radians(D.ic_tilt_deg)
        Nic = np.array([-np.sin(a), 0, np.cos(a)])
        prev = None
        for i, e in enumerate(ev):
            assert abs(_surface_residual(D, e)) < 1e-9
            din, dout = e["d_in"], e["d_out"]
            assert abs(np.linalg.norm(din) - 1) < 1e-12
            s = int(e["surf"])
            if i == 0:
                # the first segment leaves the input mirror into the slab
                assert np.dot(din, Nic) < 0
            else:
                seg = e["p"] - prev
                L = np.linalg.norm(seg)
                assert np.allclose(seg / L, din, atol=1e-9)
                # nearest hit: no other surface plane is crossed inside the segment
                for sid, N, c in planes:
                    if sid == s or sid == int(ev[i - 1]["surf"]):
                        continue
                    den = np.dot(din, N)
                    if abs(den) < 1e-14:
                        continue
                    tt = (c - np.dot(prev, N)) / den
                    assert not (1e-9 < tt < L - 1e-9), (ray, i, sid)
            if s >= 8 and e["refl"]:
                t = np.radians(float(D.mirror_tilt_deg[s - 8]))
                N = np.array([-np.sin(t), 0, np.cos(t)])
                assert np.allclose(dout, din - 2 * np.dot(din, N) * N, atol=1e-12)
            elif s >= 8:
                assert np.allclose(dout, din, atol=0)
            if s in (0, 1):
                sin2 = 1 - din[2] ** 2
                if e["refl"]:
                    assert n * n * sin2 > 1
                    assert np.allclose(dout, din * [1, 1, -1], atol=0)
                else:
                    assert n * n * sin2 <= 1
                    if s == 1:  # refraction into air: tangential component times n
                        assert np.allclose(dout[:2], n * din[:2], atol=1e-12)
                        assert abs(np.linalg.norm(dout) - 1) < 1e-12
            prev = e["p"]


def test_parallel_mirrors_preserve_the_field_angle(ora):
    """Input mirror, an even number of TIR bounces and one reflection on a
    parallel PRMA mirror map the ray back onto its field direction: the exit
    direction in air equals the field direction (image preservation)."""
    for D, C, stride in ((*W.tiny(), 7), (*small_3d(n_rays=1200), 1)):
        nf = len(C.fx_deg) * len(C.fy_deg)
        checked = 0
        for ray in range(0, C.total_rays, stride):
            ev, cat, I = ora.trace_path(D, C, ray)
            surf = ev["surf"]
            if len(ev) < 2 or surf[-1] != 1 or ev[-1]["refl"]:
                continue
            mir = np.nonzero(surf >= 8)[0]
            if len(mir) != 1 or not ev[mir[0]]["refl"]:
                continue
            if mir[0] % 2 == 1 or mir[0] != len(ev) - 2:
                continue
            f = (ray // C.n_cell) % nf
            fx, fy = C.fx_deg[f % len(C.fx_deg)], C.fy_deg[f // len(C.fx_deg)]
            v = np.array([np.tan(np.radians(float(fx))), np.tan(np.radians(float(fy))) if D.dims == 3 else 0.0, 1.0])
            v /= np.linalg.norm(v)
            assert np.allclose(ev[-1]["d_out"], v, atol=1e-12)
            checked += 1
        assert checked > 20


def test_records_reproducible(ora):
    D, C = W.tiny(n_rays=3000)
    a = ora.trace(D, C, records=True)["records"]
    b = ora.trace(D, C, records=True)["records"]
    assert np.array_equal(a, b)
    c = ora.trace(D, C.replace(seed=C.seed + 1), records=True)["records"]
    assert not np.array_equal(a["hash"], c["hash"])
