"""Pins for the oracle's thin-film solver against closed forms and textbook
identities (Methods, "Multilayer thin-film solver": Fresnel equations, Airy
formulas, transfer-matrix method)."""
import numpy as np
import pytest

N_GLASS, N_SIO2, N_TIO2, N_TA2O5 = 1.71, 1.46, 2.35, 2.1


def _close(a, b, tol):
    return abs(complex(a) - complex(b)) <= tol


# ---------------- single interface ----------------

@pytest.mark.parametrize("ni,nj", [(1.71, 1.46), (1.46, 2.35), (1.0, 1.5), (1.71, 1.0)])
def test_fresnel_normal_incidence(ora, ni, nj):
    rs, ts, rp, tp = ora.fresnel(ni, nj, 1.0)
    assert _close(rs, (ni - nj) / (ni + nj), 1e-15)
    assert _close(rp, -(ni - nj) / (ni + nj), 1e-15)   # paper's sign convention
    assert _close(ts, 2 * ni / (ni + nj), 1e-15)
    assert _close(tp, 2 * ni / (ni + nj), 1e-15)
    assert abs(abs(rs) ** 2 - ((ni - nj) / (ni + nj)) ** 2) < 1e-15


@pytest.mark.parametrize("ni,nj", [(1.71, 1.46), (1.46, 2.35), (1.0, 1.5)])
@pytest.mark.parametrize("deg", [0.0, 10.0, 30.0, 50.0])
def test_fresnel_power_balance(ora, ni, nj, deg):
    ci = np.cos(np.radians(deg))
    st = ni / nj * np.sin(np.radians(deg))
    if st >= 1:
        pytest.skip("beyond the critical angle")
    ct = np.sqrt(1 - st * st)
    rs, ts, rp, tp = ora.fresnel(ni, nj, ci)
    f = nj * ct / (ni * ci)
    assert abs(abs(rs) ** 2 + f * abs(ts) ** 2 - 1) < 1e-14
    assert abs(abs(rp) ** 2 + f * abs(tp) ** 2 - 1) < 1e-14


def test_brewster_angle_zero_p_reflection(ora):
    # tan(theta_B) = n_j / n_i; glass 1.71 -> SiO2 1.46 gives 40.49 deg
    tb = np.arctan(N_SIO2 / N_GLASS)
    assert abs(np.degrees(tb) - 40.49) < 0.01
    rs, ts, rp, tp = ora.fresnel(N_GLASS, N_SIO2, np.cos(tb))
    assert abs(rp) < 1e-14
    assert abs(rs) > 0.1


def test_total_internal_reflection_unit_modulus(ora):
    crit = np.degrees(np.arcsin(1.0 / N_GLASS))
    assert abs(crit - 35.79) < 0.01
    for deg in (36.0, 45.0, 60.0, 89.0):
        rs, ts, rp, tp = ora.fresnel(N_GLASS, 1.0, np.cos(np.radians(deg)))
        assert abs(abs(rs) - 1) < 1e-14 and abs(abs(rp) - 1) < 1e-14


# ---------------- stacks ----------------

def _numpy_fresnel(ni, nj, ci, cj):
    """Eq. fresnel_coefficients written out, complex cosines allowed."""
    rs = (ni * ci - nj * cj) / (ni * ci + nj * cj)
    ts = 2 * ni * ci / (ni * ci + nj * cj)
    rp = (nj * ci - ni * cj) / (nj * ci + ni * cj)
    tp = 2 * ni * ci / (nj * ci + ni * cj)
    return rs, ts, rp, tp


def _cos_in(n0, cos0, n):
    rad = 1 - (n0 / n) ** 2 * (1 - cos0 ** 2)
    return np.sqrt(rad) if rad >= 0 else -1j * np.sqrt(-rad)


@pytest.mark.parametrize("deg", [0.0, 25.0, 55.0, 62.0, 75.0])
@pytest.mark.parametrize("nsub", [1.71, 1.0, 2.35, 1.46])
def test_zero_layer_stack_is_one_interface(ora, deg, nsub):
    c0 = np.cos(np.radians(deg))
    rs, rp, ts, tp = ora.tmm(N_GLASS, nsub, [], [], 532.0, c0)
    frs, fts, frp, ftp = ora.fresnel(N_GLASS, nsub, c0)
    for a, b in ((rs, frs), (rp, frp), (ts, fts), (tp, ftp)):
        assert _close(a, b, 1e-13), (a, b)


@pytest.mark.parametrize("deg", [0.0, 25.0, 50.0, 75.0])
@pytest.mark.parametrize("n1", [N_SIO2, N_TIO2])
def test_one_layer_matches_airy_formula(ora, deg, n1):
    """Eq. airy_formulas with the paper's Fresnel coefficients at both faces."""
    lam, d = 532.0, 137.0
    c0 = np.cos(np.radians(deg))
    c1 = _cos_in(N_GLASS, c0, n1)
    c2 = c0
    delta = 2 * np.pi * n1 * d * c1 / lam
    e1, e2 = np.exp(-1j * delta), np.exp(-2j * delta)
    rs12, ts12, rp12, tp12 = _numpy_fresnel(N_GLASS, n1, c0, c1)
    rs23, ts23, rp23, tp23 = _numpy_fresnel(n1, N_GLASS, c1, c2)
    r_s = (rs12 + rs23 * e2) / (1 + rs12 * rs23 * e2)
    t_s = ts12 * ts23 * e1 / (1 + rs12 * rs23 * e2)
    r_p = (rp12 + rp23 * e2) / (1 + rp12 * rp23 * e2)
    t_p = tp12 * tp23 * e1 / (1 + rp12 * rp23 * e2)
    rs, rp, ts, tp = ora.tmm(N_GLASS, N_GLASS, [n1], [d], lam, c0)
    for a, b in ((rs, r_s), (rp, r_p), (ts, t_s), (tp, t_p)):
        assert _close(a, b, 1e-12), (a, b)


def _random_stack(rng, L, mats=(N_SIO2, N_TIO2, N_TA2O5)):
    n = np.array([mats[i % len(mats)] for i in range(L)])
    d = rng.uniform(10, 200, L)
    return n, d


@pytest.mark.parametrize("deg", [0.0, 25.0, 60.0, 75.0, 87.0])
@pytest.mark.parametrize("L", [2, 8, 40])
def test_matrix_route_equals_repeated_airy(ora, deg, L):
    rng = np.random.default_rng(L * 100 + int(deg))
    n, d = _random_stack(rng, L)
    c0 = np.cos(np.radians(deg))
    a = ora.tmm(N_GLASS, N_GLASS, n, d, 530.0, c0)
    b = ora.airy_stack(N_GLASS, N_GLASS, n, d, 530.0, c0)
    for x, y in zip(a, b):
        assert abs(x - y) <= 1e-11 * max(1.0, abs(y)), (x, y)


@pytest.mark.parametrize("deg", [0.0, 30.0, 75.0])
def test_characteristic_matrix_unimodular(ora, deg):
    rng = np.random.default_rng(3)
    n, d = _random_stack(rng, 12)
    Ms, Mp = ora.stack_matrix(N_GLASS, n, d, 600.0, np.cos(np.radians(deg)))
    for M in (Ms, Mp):
        det = M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0]
        assert abs(det - 1) < 1e-10 * max(1, abs(M).max() ** 2)


@pytest.mark.parametrize("deg", [0.0, 25.0, 60.0, 75.0, 87.0])
def test_lossless_energy_balance(ora, deg):
    rng = np.random.default_rng(17)
    for L in (1, 5, 23, 40):
        n, d = _random_stack(rng, L)
        rs, rp, ts, tp = ora.tmm(N_GLASS, N_GLASS, n, d, 460.0, np.cos(np.radians(deg)))
        assert abs(abs(rs) ** 2 + abs(ts) ** 2 - 1) < 1e-12
        assert abs(abs(rp) ** 2 + abs(tp) ** 2 - 1) < 1e-12


@pytest.mark.parametrize("deg", [0.0, 25.0, 40.0])
@pytest.mark.parametrize("pairs", [1, 3, 6])
def test_quarter_wave_stack_closed_form(ora, deg, pairs):
    """(HL)^N of quarter-wave layers at the design angle: admittance
    Y = (eta_H/eta_L)^(2N) eta_sub, R = |(eta0 - Y)/(eta0 + Y)|^2 (Macleod,
    tilted admittances eta_s = n cos, eta_p = n / cos)."""
    lam = 550.0
    c0 = np.cos(np.radians(deg))
    cH, cL = _cos_in(N_GLASS, c0, N_TIO2), _cos_in(N_GLASS, c0, N_SIO2)
    dH, dL = lam / (4 * N_TIO2 * cH), lam / (4 * N_SIO2 * cL)
    n = [N_TIO2, N_SIO2] * pairs
    d = [dH, dL] * pairs
    rs, rp, ts, tp = ora.tmm(N_GLASS, N_GLASS, n, d, lam, c0)
    for pol, r in (("s", rs), ("p", rp)):
        if pol == "s":
            eH, eL, e0 = N_TIO2 * cH, N_SIO2 * cL, N_GLASS * c0
        else:
            eH, eL, e0 = N_TIO2 / cH, N_SIO2 / cL, N_GLASS / c0
        Y = (eH / eL) ** (2 * pairs) * e0
        R = ((e0 - Y) / (e0 + Y)) ** 2
        assert abs(abs(r) ** 2 - R) < 1e-12


def test_half_wave_layer_is_absent(ora):
    rng = np.random.default_rng(5)
    n, d = _random_stack(rng, 9)
    c0 = np.cos(np.radians(30.0))
    lam = 500.0
    base = ora.tmm(N_GLASS, N_GLASS, n, d, lam, c0)
    cH = _cos_in(N_GLASS, c0, N_TIO2)
    n2 = np.insert(n, 4, N_TIO2)
    d2 = np.insert(d, 4, lam / (2 * N_TIO2 * cH))
    plus = ora.tmm(N_GLASS, N_GLASS, n2, d2, lam, c0)
    # the half-wave characteristic matrix is -I: r unchanged, t changes sign
    assert abs(base[0] - plus[0]) < 1e-12 and abs(base[1] - plus[1]) < 1e-12
    assert abs(base[2] + plus[2]) < 1e-12 and abs(base[3] + plus[3]) < 1e-12


@pytest.mark.parametrize("deg", [10.0, 25.0, 75.0])
def test_reversed_stack_same_power_and_transmission(ora, deg):
    rng = np.random.default_rng(8)
    n, d = _random_stack(rng, 15)
    c0 = np.cos(np.radians(deg))
    a = ora.tmm(N_GLASS, N_GLASS, n, d, 630.0, c0)
    b = ora.tmm(N_GLASS, N_GLASS, n[::-1], d[::-1], 630.0, c0)
    assert abs(abs(a[0]) - abs(b[0])) < 1e-12 and abs(abs(a[1]) - abs(b[1])) < 1e-12
    assert abs(a[2] - b[2]) < 1e-12 and abs(a[3] - b[3]) < 1e-12


def test_normal_incidence_polarization_independent(ora):
    rng = np.random.default_rng(9)
    n, d = _random_stack(rng, 20)
    rs, rp, ts, tp = ora.tmm(N_GLASS, N_GLASS, n, d, 500.0, 1.0)
    assert abs(rs + rp) < 1e-12          # r_p = -r_s in the paper's convention
    assert abs(ts - tp) < 1e-12
