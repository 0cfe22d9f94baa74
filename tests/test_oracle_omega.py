"""Pins of the oracle's reflection-probability model (Methods, "Learned
reflection probabilities": scalar reflectance equal to omega, geometric
tracing without polarization): the Monte Carlo tally estimates the exact
expectation that deterministic splitting gives, and the score-function
gradient estimates the derivative of that expectation with respect to
omega (both within four standard errors of batch means)."""
import numpy as np

from paper_2601_04370_gb300 import workloads as W


def _setup():
    D, C = W.tiny(n_rays=200_000)
    return D.replace(mirror_omega=np.array([0.35, 0.6], dtype=np.float32)), C


def _batches(ora, D, C, G=None, nb=10):
    n = C.total_rays // nb
    out = [ora.geo_trace(D, C, G=G, rays=(b * n, (b + 1) * n)) for b in range(nb)]
    return out, nb


def test_geometric_trace_estimates_the_splitting_expectation(ora):
    D, C = _setup()
    exact = ora.geo_split(D, C).sum()
    outs, nb = _batches(ora, D, C)
    tot = np.array([t.sum() for t, _ in outs])
    se = tot.std(ddof=1) * np.sqrt(nb)
    assert abs(tot.sum() - exact) <= 4.0 * se + 1e-9 * exact, (tot.sum(), exact, se)


def test_score_gradient_estimates_the_derivative_of_the_expectation(ora):
    D, C = _setup()
    # L = -I_mean (the brightness term of Eq. 1): dL/dtally does not depend on the tally
    _, _, G = ora.loss_and_grad(ora.geo_split(D, C), D.dims, C, w_f=0.0, w_e=0.0)
    outs, nb = _batches(ora, D, C, G=G)
    gs = np.array([g for _, g in outs])
    g, se = gs.sum(0), gs.std(0, ddof=1) * np.sqrt(nb)

    def L(om):
        t = ora.geo_split(D.replace(mirror_omega=np.asarray(om, dtype=np.float32)), C)
        return ora.loss_and_grad(t, D.dims, C, w_f=0.0, w_e=0.0)[0]

    om = D.mirror_omega.astype(np.float64)
    for k in range(len(om)):
        op, omn = om.copy(), om.copy()
        op[k] += 1e-3
        omn[k] -= 1e-3
        fd = (L(op) - L(omn)) / 2e-3
        assert abs(g[k] - fd) <= 4.0 * se[k], (k, g[k], fd, se[k])
