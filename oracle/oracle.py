"""ctypes front end of the FP64 oracle, plus the FP64 loss head.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in
__graft_entry__ and by bench.py's CPU-baseline / reference legs. The product
path never imports it. It imports nothing from the CUDA path; its inputs come
from paper_2601_04370_gb300.workloads (seeded generators, no method arithmetic).

The C++ side (wg_oracle.cpp) follows the paper's Methods sections (Fresnel,
Airy, transfer matrices, polarization ray tracing, Monte Carlo sampling with
amplitude rescaling). The loss head below follows Results, Eq. 1:
L = -I_mean + w_f CV_FoV + w_e CV_eyebox with w_f = 10, w_e = 3.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEDGER_NAMES = ("eyebox", "missed", "exit_reflected", "leaked", "absorbed", "truncated")
CAT_EYEBOX, CAT_MISSED, CAT_EXIT_REFL, CAT_LEAKED, CAT_ABSORBED, CAT_TRUNCATED = range(6)


def build(force: bool = False) -> str:
    """Compile wg_oracle.cpp into liboracle.so next to it (g++, C++17)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OraDesign(C.Structure):
    _fields_ = [("dims", C.c_int32), ("n_mat", C.c_int32), ("n_mir", C.c_int32), ("pad0", C.c_int32),
                ("n_slab", C.c_double), ("thickness_mm", C.c_double), ("width_mm", C.c_double),
                ("x_end_mm", C.c_double), ("eye_relief_mm", C.c_double), ("ic_tilt_deg", C.c_double),
                ("mat_n", C.POINTER(C.c_double)), ("mir_x_mm", C.POINTER(C.c_double)),
                ("mir_tilt_deg", C.POINTER(C.c_double)), ("mir_omega", C.POINTER(C.c_float)),
                ("n_layers", C.POINTER(C.c_int32)), ("layer_mat", C.POINTER(C.c_int32)),
                ("layer_d_nm", C.POINTER(C.c_double)), ("pruned", C.POINTER(C.c_uint8)),
                ("mir_geo", C.POINTER(C.c_double))]


class OraCfg(C.Structure):
    _fields_ = [("n_lam", C.c_int32), ("n_fx", C.c_int32), ("n_fy", C.c_int32), ("pol", C.c_int32),
                ("n_rays", C.c_int64), ("seed", C.c_uint64), ("max_events", C.c_int32),
                ("eb_nx", C.c_int32), ("eb_ny", C.c_int32), ("lut_bins", C.c_int32),
                ("pupil_y_mm", C.c_double), ("eb_cx_mm", C.c_double), ("eb_cy_mm", C.c_double),
                ("eb_w_mm", C.c_double), ("eb_h_mm", C.c_double),
                ("lam_nm", C.POINTER(C.c_double)), ("fx_deg", C.POINTER(C.c_double)),
                ("fy_deg", C.POINTER(C.c_double))]


class OraStats(C.Structure):
    _fields_ = [("n_hits", C.c_int64), ("n_events", C.c_int64), ("n_tir", C.c_int64),
                ("n_rays", C.c_int64)]


PATHEV_DTYPE = np.dtype([("surf", np.int32), ("refl", np.int32), ("p", np.float64, 3),
                         ("d_in", np.float64, 3), ("d_out", np.float64, 3)])

RAYREC_DTYPE = np.dtype([("hash", np.uint32), ("n_events", np.int32), ("n_hits", np.int32),
                         ("cat", np.int32), ("bin", np.int32), ("pad", np.int32),
                         ("I", np.float64), ("w", np.float64)])

_P = np.ctypeslib.ndpointer


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.ora_philox.argtypes = [C.POINTER(C.c_uint32)] * 3
            L.ora_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, dp]
            L.ora_tmm.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp, C.c_double, C.c_double, dp]
            L.ora_airy_stack.argtypes = L.ora_tmm.argtypes
            L.ora_stack_matrix.argtypes = [C.c_double, C.c_int, dp, dp, C.c_double, C.c_double, dp]
            L.ora_tmm_grad.argtypes = [C.c_double, C.c_int, dp, dp, C.c_double, C.c_double, dp,
                                       C.c_int, dp, dp, dp]
            L.ora_trace.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64, C.c_int64,
                                    C.c_int, dp, dp, C.POINTER(OraStats), C.c_void_p]
            L.ora_split.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64, C.c_int64,
                                    C.c_int, C.c_double, dp, dp, C.POINTER(C.c_int64)]
            L.ora_geo_trace.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64, C.c_int64, C.c_int,
                                        C.c_void_p, dp, C.c_void_p]
            L.ora_geo_split.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64, C.c_int64, C.c_int,
                                        C.c_double, dp]
            L.ora_trace_grad.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64,
                                         C.c_int64, C.c_int, dp, C.c_void_p, dp, dp, C.c_void_p]
            L.ora_trace_path.argtypes = [C.POINTER(OraDesign), C.POINTER(OraCfg), C.c_int64,
                                         C.c_void_p, C.c_int, C.POINTER(C.c_int), dp]
            L.ora_trace_path.restype = C.c_int
            L.ora_hardware_threads.restype = C.c_int
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def hardware_threads() -> int:
    return int(lib().ora_hardware_threads())


# --------------------------------------------------------------------------
# Thin-film and RNG primitives
# --------------------------------------------------------------------------

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox(c, k, o)
    return [int(x) for x in o]


def _cx4(out):
    return out[0::2] + 1j * out[1::2]


def fresnel(n_i, n_j, cos_i):
    """(r_s, t_s, r_p, t_p) at one interface (paper's Fresnel equations)."""
    out = np.zeros(8)
    lib().ora_fresnel(float(n_i), float(n_j), float(cos_i), _dptr(out))
    return tuple(_cx4(out))


def tmm(n0, nsub, n, d, lam, cos0):
    """(r_s, r_p, t_s, t_p) of a stack by characteristic matrices."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(8)
    lib().ora_tmm(float(n0), float(nsub), len(n), _dptr(n), _dptr(d), float(lam), float(cos0), _dptr(out))
    return tuple(_cx4(out))


def airy_stack(n0, nsub, n, d, lam, cos0):
    """(r_s, r_p, t_s, t_p) of a stack by repeated Airy summation."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(8)
    lib().ora_airy_stack(float(n0), float(nsub), len(n), _dptr(n), _dptr(d), float(lam), float(cos0),
                         _dptr(out))
    return tuple(_cx4(out))


def stack_matrix(n0, n, d, lam, cos0):
    """Characteristic matrices (2x2 complex) for s and p."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(16)
    lib().ora_stack_matrix(float(n0), len(n), _dptr(n), _dptr(d), float(lam), float(cos0), _dptr(out))
    v = _cx4(out)
    return v[:4].reshape(2, 2), v[4:].reshape(2, 2)


def tmm_grad(n0, n, d, lam, cos0, A_s, A_p, which="r"):
    """d/d(thickness) and d/d(cos theta0) of f = 2 Re(A_s c_s + A_p c_p),
    c = r or t, by reverse-mode AD through the oracle's transfer matrices."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    A = np.array([A_s.real, A_s.imag, A_p.real, A_p.imag], dtype=np.float64)
    g = np.zeros(len(n))
    gc = np.zeros(1)
    f = np.zeros(1)
    lib().ora_tmm_grad(float(n0), len(n), _dptr(n), _dptr(d), float(lam), float(cos0), _dptr(A),
                       0 if which == "r" else 1, _dptr(g), _dptr(gc), _dptr(f))
    return g, float(gc[0]), float(f[0])


# --------------------------------------------------------------------------
# Trace
# --------------------------------------------------------------------------

class _Marshalled:
    """Keeps the float64 copies alive while the structs point at them."""

    def __init__(self, D, Cfg):
        self.keep = []

        def d64(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            self.keep.append(a)
            return _dptr(a)

        def typed(a, dt, ct):
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self.keep.append(a)
            return a.ctypes.data_as(C.POINTER(ct))

        self.d = OraDesign(dims=D.dims, n_mat=len(D.mat_n), n_mir=D.n_mirrors, pad0=0,
                           n_slab=D.n_slab, thickness_mm=D.thickness_mm, width_mm=D.width_mm,
                           x_end_mm=D.x_end_mm, eye_relief_mm=D.eye_relief_mm,
                           ic_tilt_deg=D.ic_tilt_deg, mat_n=d64(D.mat_n), mir_x_mm=d64(D.mirror_x_mm),
                           mir_tilt_deg=d64(D.mirror_tilt_deg),
                           mir_omega=typed(D.mirror_omega, np.float32, C.c_float),
                           n_layers=typed(D.n_layers, np.int32, C.c_int32),
                           layer_mat=typed(D.layer_mat, np.int32, C.c_int32),
                           layer_d_nm=d64(D.layer_d_nm), pruned=typed(D.pruned, np.uint8, C.c_uint8),
                           mir_geo=(d64(D.mirror_geo) if getattr(D, "mirror_geo", None) is not None
                                    else C.POINTER(C.c_double)()))
        self.c = OraCfg(n_lam=len(Cfg.lam_nm), n_fx=len(Cfg.fx_deg), n_fy=len(Cfg.fy_deg), pol=Cfg.pol,
                        n_rays=Cfg.n_rays, seed=Cfg.seed, max_events=Cfg.max_events, eb_nx=Cfg.eb_nx,
                        eb_ny=Cfg.eb_ny, lut_bins=int(getattr(Cfg, "lut_bins", 0)), pupil_y_mm=Cfg.pupil_y_mm,
                        eb_cx_mm=Cfg.eb_cx_mm,
                        eb_cy_mm=Cfg.eb_cy_mm, eb_w_mm=Cfg.eb_w_mm, eb_h_mm=Cfg.eb_h_mm,
                        lam_nm=d64(Cfg.lam_nm), fx_deg=d64(Cfg.fx_deg), fy_deg=d64(Cfg.fy_deg))


def _range(Cfg, rays):
    if rays is None:
        return 0, Cfg.total_rays
    return int(rays[0]), int(rays[1])


def trace(D, Cfg, rays=None, nthreads=0, records=False):
    """Monte Carlo forward trace. Returns dict(tally (shaped), ledger[6],
    stats, records (structured array or None))."""
    m = _Marshalled(D, Cfg)
    r0, r1 = _range(Cfg, rays)
    tally = np.zeros(Cfg.tally_size)
    ledger = np.zeros(6)
    st = OraStats()
    rec = np.zeros(r1 - r0, dtype=RAYREC_DTYPE) if records else None
    lib().ora_trace(C.byref(m.d), C.byref(m.c), r0, r1, int(nthreads), _dptr(tally), _dptr(ledger),
                    C.byref(st), rec.ctypes.data if records else None)
    return dict(tally=tally.reshape(Cfg.tally_shape), ledger=ledger,
                stats=dict(n_hits=st.n_hits, n_events=st.n_events, n_tir=st.n_tir, n_rays=st.n_rays),
                records=rec)


def trace_path(D, Cfg, ray, cap=256):
    """Event list of one ray: (events structured array, category, intensity)."""
    m = _Marshalled(D, Cfg)
    ev = np.zeros(cap, dtype=PATHEV_DTYPE)
    cat = C.c_int(0)
    I = np.zeros(1)
    n = lib().ora_trace_path(C.byref(m.d), C.byref(m.c), int(ray), ev.ctypes.data, cap, C.byref(cat),
                             _dptr(I))
    return ev[:n], int(cat.value), float(I[0])


def split(D, Cfg, rays=None, nthreads=0, prune=0.0):
    """Deterministic ray-splitting expectation for the same launch points."""
    m = _Marshalled(D, Cfg)
    r0, r1 = _range(Cfg, rays)
    tally = np.zeros(Cfg.tally_size)
    ledger = np.zeros(6)
    nb = C.c_int64(0)
    lib().ora_split(C.byref(m.d), C.byref(m.c), r0, r1, int(nthreads), float(prune), _dptr(tally),
                    _dptr(ledger), C.byref(nb))
    return dict(tally=tally.reshape(Cfg.tally_shape), ledger=ledger, n_branches=int(nb.value))


def geo_trace(D, Cfg, G=None, rays=None, nthreads=0):
    """Reflection-probability pre-optimization model (Methods, "Learned
    reflection probabilities"): geometric Monte Carlo trace with each coating
    a scalar reflectance equal to its mirror's omega, no polarization, the
    unpolarized Fresnel transmittance at the eye-side face. Returns (tally,
    dL/d omega [K] for G = dL/dtally, or None): the score-function estimator
    sum over tallied rays of G[bin] I (n_r/omega - n_t/(1 - omega))."""
    m = _Marshalled(D, Cfg)
    r0, r1 = _range(Cfg, rays)
    tally = np.zeros(Cfg.tally_size)
    grad = np.zeros(D.n_mirrors) if G is not None else None
    g = None if G is None else np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(-1))
    lib().ora_geo_trace(C.byref(m.d), C.byref(m.c), r0, r1, int(nthreads),
                        None if g is None else g.ctypes.data, _dptr(tally), None if grad is None else grad.ctypes.data)
    return tally.reshape(Cfg.tally_shape), grad


def geo_split(D, Cfg, rays=None, nthreads=0, prune=1e-12):
    """Expected tally of the geometric model for the same launch points, by
    deterministic splitting (reflect with probability omega, transmit 1 - omega)."""
    m = _Marshalled(D, Cfg)
    r0, r1 = _range(Cfg, rays)
    tally = np.zeros(Cfg.tally_size)
    lib().ora_geo_split(C.byref(m.d), C.byref(m.c), r0, r1, int(nthreads), float(prune), _dptr(tally))
    return tally.reshape(Cfg.tally_shape)


def trace_grad(D, Cfg, G, rays=None, nthreads=0, mask=None, ray_intensity=False):
    """Adjoint: (grad_thickness [sum L] per nm, grad_tilt [K] per degree)
    of sum_rays G[bin] I_ray along each ray's sampled path."""
    m = _Marshalled(D, Cfg)
    r0, r1 = _range(Cfg, rays)
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64).reshape(-1))
    assert G.size == Cfg.tally_size
    gd = np.zeros(D.total_layers)
    gt = np.zeros(D.n_mirrors)
    mk = None
    if mask is not None:
        mk = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        assert mk.size == r1 - r0
    rI = np.zeros(r1 - r0) if ray_intensity else None
    lib().ora_trace_grad(C.byref(m.d), C.byref(m.c), r0, r1, int(nthreads), _dptr(G),
                         mk.ctypes.data if mk is not None else None, _dptr(gd), _dptr(gt),
                         rI.ctypes.data if rI is not None else None)
    if ray_intensity:
        return gd, gt, rI
    return gd, gt


# --------------------------------------------------------------------------
# Loss head (Results, Eq. 1), FP64
# --------------------------------------------------------------------------

PUPIL_DIAMETER_MM = 4.0


def pupil_masks(dims, Cfg):
    """Boolean masks [P, eb_ny, eb_nx]: 3x3 pupils of 4 mm diameter whose
    centres span the eyebox (offsets -(W-4)/2, 0, +(W-4)/2 per axis); in 2D
    the eyebox is 1D and there are 3 pupils (4 mm intervals)."""
    xs = Cfg.eb_cx_mm - 0.5 * Cfg.eb_w_mm + (np.arange(Cfg.eb_nx) + 0.5) * (Cfg.eb_w_mm / Cfg.eb_nx)
    ox = 0.5 * (Cfg.eb_w_mm - PUPIL_DIAMETER_MM)
    r = 0.5 * PUPIL_DIAMETER_MM
    if dims == 2:
        cx = Cfg.eb_cx_mm + np.array([-ox, 0.0, ox])
        m = np.abs(xs[None, :] - cx[:, None]) <= r
        return m[:, None, :]
    ys = Cfg.eb_cy_mm - 0.5 * Cfg.eb_h_mm + (np.arange(Cfg.eb_ny) + 0.5) * (Cfg.eb_h_mm / Cfg.eb_ny)
    oy = 0.5 * (Cfg.eb_h_mm - PUPIL_DIAMETER_MM)
    masks = []
    for dy in (-oy, 0.0, oy):
        for dx in (-ox, 0.0, ox):
            d2 = (xs[None, :] - (Cfg.eb_cx_mm + dx)) ** 2 + (ys[:, None] - (Cfg.eb_cy_mm + dy)) ** 2
            masks.append(d2 <= r * r)
    return np.stack(masks)


def pupil_images(tally, dims, Cfg):
    """I[lam, field, pupil] = (sum of tally over the pupil's bins) / rays per cell."""
    t = np.asarray(tally, dtype=np.float64).reshape(Cfg.tally_shape)
    nl, nfy, nfx, ny, nx = Cfg.tally_shape
    t = t.reshape(nl, nfy * nfx, ny * nx)
    M = pupil_masks(dims, Cfg).reshape(-1, ny * nx).astype(np.float64)
    return t @ M.T / Cfg.n_cell


def _cv_and_grad(x, axis):
    """Coefficient of variation (population std / mean) along `axis`, averaged
    over the other axes, and its gradient with respect to x."""
    n = x.shape[axis]
    mu = x.mean(axis=axis, keepdims=True)
    dev = x - mu
    sd = np.sqrt((dev ** 2).mean(axis=axis, keepdims=True))
    safe = (mu != 0) & (sd > 0)
    cv = np.where(mu != 0, sd / np.where(mu != 0, mu, 1.0), 0.0)
    # d sd / dx_i = dev_i / (n sd); d mu / dx_i = 1/n
    dsd = np.where(safe, dev / (n * np.where(sd > 0, sd, 1.0)), 0.0)
    dcv = np.where(safe, dsd / np.where(mu != 0, mu, 1.0) - (cv / np.where(mu != 0, mu, 1.0)) / n, 0.0)
    m = cv.size
    return float(cv.mean()), dcv / m


def _var_and_grad(x, axis):
    n = x.shape[axis]
    mu = x.mean(axis=axis, keepdims=True)
    dev = x - mu
    var = (dev ** 2).mean(axis=axis, keepdims=True)
    m = var.size
    return float(var.mean()), (2.0 * dev / n) / m


def loss_and_grad(tally, dims, Cfg, kind="cv", w_f=10.0, w_e=3.0):
    """L = -I_mean + w_f U_FoV + w_e U_eyebox, U = CV (paper) or variance.
    Returns (L, parts dict, dL/dtally shaped like the tally)."""
    I = pupil_images(tally, dims, Cfg)            # [lam, f, p]
    mean = float(I.mean())
    dmean = np.full(I.shape, 1.0 / I.size)
    fn = _cv_and_grad if kind == "cv" else _var_and_grad
    u_f, du_f = fn(I, axis=1)
    u_e, du_e = fn(I, axis=2)
    L = -mean + w_f * u_f + w_e * u_e
    dI = -dmean + w_f * du_f + w_e * du_e
    nl, nfy, nfx, ny, nx = Cfg.tally_shape
    M = pupil_masks(dims, Cfg).reshape(-1, ny * nx).astype(np.float64)
    G = (dI @ M) / Cfg.n_cell                      # [lam, f, bins]
    return L, dict(I_mean=mean, u_fov=u_f, u_eyebox=u_e), G.reshape(Cfg.tally_shape)


def adam_projected_step(theta, m, v, g, t, lr=2.0, beta1=0.9, beta2=0.999, eps=1e-8, d_min=20.0, d_max=200.0,
                        fixed=None):
    """One optimizer step on the layer thicknesses (Results, "Evaluation":
    thicknesses within 20-200 nm, a soft gap between 0 and 20 nm through
    which layers can be eliminated). The paper does not name the optimizer;
    this is Adam (Kingma and Ba, 2015, Algorithm 1) written out in FP64 on
    the thicknesses in nm:
        m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
        theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
    then the projection: clamp to [0, d_max]; a value in the gap (0, d_min)
    goes to 0 below d_min / 2, else to d_min. Thicknesses are kept in FP32
    (as the design stores them). Layers with fixed[i] set, and layers whose
    gradient is not finite, are left as they are. Returns new (theta, m, v)."""
    theta = np.asarray(theta, dtype=np.float32).astype(np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    upd = np.isfinite(g)
    if fixed is not None:
        upd &= ~np.asarray(fixed, dtype=bool)
    gg = np.where(upd, g, 0.0)
    m_new = beta1 * m + (1.0 - beta1) * gg
    v_new = beta2 * v + (1.0 - beta2) * gg * gg
    mhat = m_new / (1.0 - beta1 ** t)
    vhat = v_new / (1.0 - beta2 ** t)
    x = theta - lr * mhat / (np.sqrt(vhat) + eps)
    x = np.clip(x, 0.0, d_max)
    gap = (x > 0.0) & (x < d_min)
    x = np.where(gap, np.where(x < 0.5 * d_min, 0.0, d_min), x)
    theta_new = np.where(upd, x, theta).astype(np.float32)
    return theta_new, np.where(upd, m_new, m), np.where(upd, v_new, v)


def adam_clipped_step(w, m, v, g, t, lr=0.02, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.02, hi=0.98):
    """One step of the reflection-probability pre-optimization's update
    (Methods, "Learned reflection probabilities"; the paper names no
    optimizer): Adam (Kingma and Ba, 2015, Algorithm 1) in FP64 on the
    mirrors' omega with dL/d omega of a loss to minimize,
        m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
        w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
    then each value clipped to [lo, hi]. Entries whose gradient is not
    finite are left as they are. Returns new (w, m, v)."""
    w = np.array(w, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    upd = np.isfinite(g)
    gg = np.where(upd, g, 0.0)
    m_new = beta1 * m + (1.0 - beta1) * gg
    v_new = beta2 * v + (1.0 - beta2) * gg * gg
    x = w - lr * (m_new / (1.0 - beta1 ** t)) / (np.sqrt(v_new / (1.0 - beta2 ** t)) + eps)
    x = np.clip(x, lo, hi)
    return np.where(upd, x, w), np.where(upd, m_new, m), np.where(upd, v_new, v)
