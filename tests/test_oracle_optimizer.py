"""Pins of the oracle's optimizer step (Adam on the thicknesses, then the
projection onto [0, d_max] with the soft gap (0, d_min); Results,
"Evaluation"), against what Adam's definition and the projection fix."""
import numpy as np

from oracle import oracle as O


def test_first_step_moves_each_layer_by_lr_against_its_gradient():
    # bias-corrected first step: m_hat = g, v_hat = g^2, so the step is
    # lr g / (|g| + eps) (= lr sign(g) for |g| >> eps), up to the FP32 storage
    rng = np.random.default_rng(1)
    th = rng.uniform(40.0, 160.0, size=64).astype(np.float32)
    g = rng.normal(size=64) * 10.0 ** rng.uniform(-6, 3, size=64)
    t1, m, v = O.adam_projected_step(th, np.zeros(64), np.zeros(64), g, 1, lr=3.0, eps=1e-8)
    step = -3.0 * g / (np.abs(g) + 1e-8)
    assert np.allclose(t1.astype(np.float64) - th.astype(np.float64), step, atol=3e-5)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_projection_bounds_and_soft_gap():
    th = np.array([199.0, 21.0, 11.0, 0.0, 100.0, 30.0], dtype=np.float32)
    # gradients push: up past 200, down into the gap (19 -> d_min), down below
    # d_min/2 (9 -> 0), up from zero by less than d_min/2 (stays 0), plain step,
    # down from 30 to 28 (no projection)
    g = np.array([-1.0, 1.0, 1.0, -1.0, 1.0, 1.0])
    t1, _, _ = O.adam_projected_step(th, np.zeros(6), np.zeros(6), g, 1, lr=2.0)
    assert np.allclose(t1, [200.0, 20.0, 0.0, 0.0, 98.0, 28.0], atol=1e-4)


def test_fixed_and_non_finite_entries_are_left_alone():
    th = np.array([50.0, 60.0, 70.0], dtype=np.float32)
    m0, v0 = np.array([0.1, 0.2, 0.3]), np.array([1.0, 2.0, 3.0])
    g = np.array([1.0, np.nan, 1.0])
    t1, m, v = O.adam_projected_step(th, m0, v0, g, 4, fixed=np.array([1, 0, 0], dtype=np.uint8))
    assert t1[0] == th[0] and t1[1] == th[1] and t1[2] < th[2]
    assert m[0] == m0[0] and m[1] == m0[1] and v[1] == v0[1] and m[2] != m0[2]


def test_adam_converges_to_the_minimum_of_a_quadratic():
    # f = sum (theta - a)^2 with a inside the bounds: a wrong sign or a
    # dropped bias correction would not settle near a
    rng = np.random.default_rng(2)
    a = rng.uniform(30.0, 190.0, size=32)
    th = np.full(32, 110.0, dtype=np.float32)
    m = np.zeros(32)
    v = np.zeros(32)
    for t in range(1, 4001):
        g = 2.0 * (th.astype(np.float64) - a)
        th, m, v = O.adam_projected_step(th, m, v, g, t, lr=0.5)
    assert np.max(np.abs(th - a)) < 0.3


# ---------------------------------------------------------------------------
# the reflection probabilities' step (Adam on omega, clipped to [lo, hi])
# ---------------------------------------------------------------------------

def test_omega_first_step_is_lr_against_the_gradient_and_clipped():
    w = np.array([0.5, 0.5, 0.03, 0.97, 0.4])
    g = np.array([2.0, -1e-3, 5.0, -7.0, np.nan])
    w1, m, v = O.adam_clipped_step(w, np.zeros(5), np.zeros(5), g, 1, lr=0.02, lo=0.02, hi=0.98)
    # bias-corrected first step: lr g / (|g| + eps); then the clip
    assert np.allclose(w1[:2], [0.48, 0.52], atol=1e-9)
    assert w1[2] == 0.02 and w1[3] == 0.98   # 0.03 - 0.02 and 0.97 + 0.02 leave [lo, hi]
    assert w1[4] == 0.4 and m[4] == 0.0 and v[4] == 0.0   # non-finite gradient: untouched
    assert np.allclose(m[:4], 0.1 * g[:4]) and np.allclose(v[:4], 0.001 * g[:4] ** 2)


def test_omega_adam_converges_to_an_interior_minimum():
    # f = sum (w - a)^2 with a inside (lo, hi): a sign error or a dropped bias
    # correction would not settle near a
    a = np.array([0.1, 0.35, 0.6, 0.9])
    w = np.full(4, 0.5)
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 3001):
        w, m, v = O.adam_clipped_step(w, m, v, 2.0 * (w - a), t, lr=0.005)
    assert np.max(np.abs(w - a)) < 2e-3
