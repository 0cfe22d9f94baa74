"""Pins for the oracle's Philox4x32-10 generator and the uniform mapping."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answer_vectors(ora):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert ora.philox(ctr, key) == out


def test_philox_is_a_bijection_of_the_counter_on_a_sample(ora):
    # distinct counters under one key give distinct outputs (a permutation)
    outs = {tuple(ora.philox([i, 0, 7, 3], [11, 0])) for i in range(2000)}
    assert len(outs) == 2000


def test_uniform_has_24_bits_and_mean_half(ora):
    u = np.array([(ora.philox([i, 0, 0, 0x47454E30], [7, 0])[0] >> 8) * 2.0 ** -24 for i in range(4000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))          # exactly 24-bit values
    assert np.float32(u).astype(np.float64).tolist() == u.tolist()  # exact in FP32
    assert abs(u.mean() - 0.5) < 4 * (1 / np.sqrt(12 * len(u)))
