"""The accurate layer evaluation's sin/cos polynomials (wg_device.cuh,
sincos_turns_acc): read the committed FP32 coefficients and check them
against numpy's sin/cos on the reduced range |r| <= 1/8 turn, in exact
arithmetic and as the kernel evaluates them (FP32 Horner, FMA emulated in
FP64), and the quadrant rotation over whole turns."""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2601_04370_gb300", "csrc", "wg_device.cuh")


def _coefs():
    src = open(HDR).read()
    c = {m.group(1): np.float32(float(m.group(2))) for m in re.finditer(r"SC_([SC]\d) = ([-+0-9.e]+)f", src)}
    assert set(c) == {"S1", "S3", "S5", "S7", "C2", "C4", "C6", "C8"}, c
    return c


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _fma(a, b, c):
    return _f32(np.float64(a) * np.float64(b) + np.float64(c))


def _poly(r, c):
    r = _f32(r)
    r2 = _f32(np.float64(r) * np.float64(r))
    sp = _f32(np.float64(r) * np.float64(_fma(_fma(_fma(c["S7"], r2, c["S5"]), r2, c["S3"]), r2, c["S1"])))
    cp = _fma(_fma(_fma(_fma(c["C8"], r2, c["C6"]), r2, c["C4"]), r2, c["C2"]), r2, np.float32(1.0))
    return sp.astype(np.float64), cp.astype(np.float64)


def test_polynomials_on_the_reduced_range():
    c = _coefs()
    r = np.linspace(-0.125, 0.125, 200001)
    s_ex = sum(np.float64(c[k]) * r ** int(k[1:]) for k in ("S1", "S3", "S5", "S7"))
    c_ex = 1.0 + sum(np.float64(c[k]) * r ** int(k[1:]) for k in ("C2", "C4", "C6", "C8"))
    assert np.abs(s_ex - np.sin(2 * np.pi * r)).max() < 1e-8
    assert np.abs(c_ex - np.cos(2 * np.pi * r)).max() < 1e-9
    sp, cp = _poly(r, c)
    rr = _f32(r).astype(np.float64)
    assert np.abs(sp - np.sin(2 * np.pi * rr)).max() < 1e-7      # ~1 ulp near 0.7
    assert np.abs(cp - np.cos(2 * np.pi * rr)).max() < 1e-7


def test_quadrant_rotation_over_whole_turns():
    # p turns -> q = round(4 p), r = p - q / 4, then (s, c) rotated by q pi/2
    c = _coefs()
    p = np.linspace(-3.0, 3.0, 60001)
    q = np.rint(4 * p)
    r = p - q / 4
    sp, cp = _poly(r, c)
    qb = q.astype(np.int64) & 3
    sw = (qb & 1) == 1
    so, co = np.where(sw, cp, sp), np.where(sw, sp, cp)
    s = np.where(qb & 2, -so, so)
    cc = np.where((qb + 1) & 2, -co, co)
    assert np.abs(s - np.sin(2 * np.pi * p)).max() < 2e-7
    assert np.abs(cc - np.cos(2 * np.pi * p)).max() < 2e-7
