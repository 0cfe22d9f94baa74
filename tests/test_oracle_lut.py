"""Pins of the oracle's coating look-up table (the paper's memory-saving
variant, Fig. 3c: coefficients tabulated over cos(theta_0), linear
interpolation per hit): it converges to the exact per-hit coefficients as
the table grows, at the rate linear interpolation has (error ~ 1/N^2), and
its adjoint is the derivative of the tabulated objective."""
import numpy as np

from paper_2601_04370_gb300 import workloads as W


def _rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_table_tallies_converge_quadratically_to_exact(ora):
    D, C = W.tiny(n_rays=4000)
    ex = ora.trace(D, C)["tally"]
    e = [_rel(ora.trace(D, C.replace(lut_bins=n))["tally"], ex) for n in (256, 1024, 4096)]
    # linear interpolation: 4x the bins -> ~16x smaller error
    assert e[0] / e[1] > 8 and e[1] / e[2] > 8, e
    assert e[2] < 1e-5, e


def test_table_adjoint_matches_fixed_key_differences(ora):
    """The tabulated objective is smooth in the thicknesses (each table entry
    is), so central differences of sum(G * tally) agree with the adjoint
    through the interpolation weights and the two bracketing entries."""
    D, C = W.tiny(n_rays=2000)
    C = C.replace(lut_bins=256)
    rng = np.random.default_rng(3)
    G = rng.normal(size=C.tally_shape)
    gd, _ = ora.trace_grad(D, C, G)
    base = D.layer_d_nm.astype(np.float64)

    def obj(d):
        Dx = D.replace()
        Dx.layer_d_nm = d
        return float((ora.trace(Dx, C)["tally"] * G).sum())

    h = 0.01
    for i in range(0, D.total_layers, 3):
        dp, dm = base.copy(), base.copy()
        dp[i] += h
        dm[i] -= h
        fd = (obj(dp) - obj(dm)) / (2 * h)
        assert abs(gd[i] - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gd).max()), (i, gd[i], fd)


def test_table_gradient_differs_from_exact_by_the_interpolation_error(ora):
    """The table's gradient approaches the exact per-hit gradient as the table
    grows (it is the derivative of an approximation, not of the exact
    objective)."""
    D, C = W.tiny(n_rays=2000)
    rng = np.random.default_rng(4)
    G = rng.normal(size=C.tally_shape)
    ex, _ = ora.trace_grad(D, C, G)
    errs = []
    for n in (256, 4096):
        g, _ = ora.trace_grad(D, C.replace(lut_bins=n), G)
        errs.append(np.linalg.norm(g - ex) / np.linalg.norm(ex))
    assert errs[1] < errs[0] / 8 and errs[1] < 1e-3, errs
