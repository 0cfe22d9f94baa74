"""Seeded synthetic workloads: waveguide designs and trace configurations.

This module only draws inputs. It holds none of the method's arithmetic, so
both the CUDA path and the FP64 oracle take their inputs from here. Every real
value is rounded to float32 before it is handed out, so both sides see
bit-identical inputs (the GPU computes in FP32, the oracle in FP64 from the
same float32 values).

The shapes follow the paper's workload (Results, "System Architecture": a
glass slab guiding light by TIR, an input mirror, a partially reflective
mirror array whose mirrors carry multilayer SiO2/Ta2O5-type stacks, an eyebox
at 15 mm eye relief, a grid of field angles, several wavelengths per run),
scaled to the named configurations below. Design RNG: numpy PCG64(seed).
"""
from __future__ import annotations

import dataclasses
import numpy as np

# refractive indices (lossless, non-dispersive)
N_SIO2 = 1.46
N_TIO2 = 2.35
N_TA2O5 = 2.1
N_TA2O5_PAPER = 2.13

POL_PAIR, POL_RANDOM_LINEAR, POL_S, POL_P = 0, 1, 2, 3

# energy ledger slots
LEDGER_NAMES = ("eyebox", "missed", "exit_reflected", "leaked", "absorbed", "truncated")


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


@dataclasses.dataclass
class Design:
    """Slab waveguide + PRMA. Lengths in mm, thicknesses in nm, angles in deg."""

    dims: int
    n_slab: float
    thickness_mm: float
    width_mm: float
    x_end_mm: float
    eye_relief_mm: float
    ic_tilt_deg: float
    mat_n: np.ndarray          # float32 [n_mat]
    mirror_x_mm: np.ndarray    # float32 [K] mirror centre x at mid-thickness
    mirror_tilt_deg: np.ndarray  # float32 [K]
    mirror_omega: np.ndarray   # float32 [K] reflection probability
    n_layers: np.ndarray       # int32 [K]
    layer_mat: np.ndarray      # int32 [sum L] material id, layer 1 first
    layer_d_nm: np.ndarray     # float32 [sum L]
    pruned: np.ndarray         # uint8 [sum L]
    # None: every mirror is a PRMA plane through (x_k, 0, t/2) tilted about y.
    # Else float32 [K, 14], mirror k a general plane: unit normal N0 (3) at
    # the tilt t0, pivot (3), tilt axis (3; unit, perpendicular to N0; the
    # tilt mirror_tilt_deg[k] rotates N0 about it by tilt - t0), the (x, y)
    # rectangle x0, x1, y0, y1 where the mirror acts (+-inf: unbounded), t0.
    mirror_geo: np.ndarray | None = None

    def __post_init__(self):
        for name in ("n_slab", "thickness_mm", "width_mm", "x_end_mm", "eye_relief_mm", "ic_tilt_deg"):
            setattr(self, name, float(np.float32(getattr(self, name))))
        self.mat_n = _f32(self.mat_n)
        self.mirror_x_mm = _f32(self.mirror_x_mm)
        self.mirror_tilt_deg = _f32(self.mirror_tilt_deg)
        self.mirror_omega = _f32(self.mirror_omega)
        self.n_layers = np.asarray(self.n_layers, dtype=np.int32)
        self.layer_mat = np.asarray(self.layer_mat, dtype=np.int32)
        self.layer_d_nm = _f32(self.layer_d_nm)
        self.pruned = np.asarray(self.pruned, dtype=np.uint8)
        if self.mirror_geo is not None:
            self.mirror_geo = _f32(self.mirror_geo).reshape(-1, 14)

    @property
    def n_mirrors(self) -> int:
        return int(self.n_layers.shape[0])

    @property
    def total_layers(self) -> int:
        return int(self.n_layers.sum())

    def layer_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_layers)]).astype(np.int64)

    def replace(self, **kw) -> "Design":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class TraceConfig:
    """Wavelengths, field grid, polarization, ray budget and eyebox grid."""

    lam_nm: np.ndarray        # float32 [n_lam]
    fx_deg: np.ndarray        # float32 [n_fx] field angle along x (in air)
    fy_deg: np.ndarray        # float32 [n_fy] field angle along y (in air)
    pol: int
    n_rays: int               # requested; rays per cell = ceil(n_rays / cells)
    seed: int                 # 64-bit Philox key
    max_events: int = 100
    pupil_y_mm: float = 8.0
    eb_cx_mm: float = 0.0
    eb_cy_mm: float = 0.0
    eb_w_mm: float = 8.0
    eb_h_mm: float = 8.0
    eb_nx: int = 64
    eb_ny: int = 1
    lut_bins: int = 0         # 0: each hit's exact layer chain; N: the coating table with N bins of cos(theta_0)

    def __post_init__(self):
        self.lam_nm = _f32(self.lam_nm)
        self.fx_deg = _f32(self.fx_deg)
        self.fy_deg = _f32(self.fy_deg)
        for name in ("pupil_y_mm", "eb_cx_mm", "eb_cy_mm", "eb_w_mm", "eb_h_mm"):
            setattr(self, name, float(np.float32(getattr(self, name))))
        self.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF

    @property
    def n_fields(self) -> int:
        return int(self.fx_deg.shape[0] * self.fy_deg.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.lam_nm.shape[0]) * self.n_fields

    @property
    def n_cell(self) -> int:
        return -(-int(self.n_rays) // self.n_cells)

    @property
    def total_rays(self) -> int:
        return self.n_cell * self.n_cells

    @property
    def tally_shape(self):
        return (int(self.lam_nm.shape[0]), int(self.fy_deg.shape[0]), int(self.fx_deg.shape[0]),
                int(self.eb_ny), int(self.eb_nx))

    @property
    def tally_size(self) -> int:
        return int(np.prod(self.tally_shape))

    def replace(self, **kw) -> "TraceConfig":
        return dataclasses.replace(self, **kw)


def default_omega(k_mirrors: int) -> np.ndarray:
    """Equal-extraction reflection probabilities clamp(1/(K-k), 0.02, 0.98)."""
    k = np.arange(k_mirrors)
    return np.clip(1.0 / (k_mirrors - k), 0.02, 0.98)


def cycling_stack(rng, n_mirrors, n_layers, n_materials, d_lo=10.0, d_hi=200.0, prune_p=0.0):
    """Stacks whose material cycles 0,1,..,n_materials-1 from layer 1."""
    nl = np.full(n_mirrors, n_layers, dtype=np.int32) if np.isscalar(n_layers) else np.asarray(n_layers)
    mats, ds, pr = [], [], []
    for k in range(n_mirrors):
        L = int(nl[k])
        mats.append(np.arange(L) % n_materials)
        d = rng.uniform(d_lo, d_hi, size=L)
        p = (rng.uniform(size=L) < prune_p) if prune_p > 0 else np.zeros(L, bool)
        d = np.where(p, 0.0, d)
        ds.append(d)
        pr.append(p)
    return nl, np.concatenate(mats), np.concatenate(ds), np.concatenate(pr).astype(np.uint8)


def _prma_design(dims, n_slab, t_mm, n_mirrors, n_layers, mat_n, seed, spacing=1.5, tilt=25.0,
                 prune_p=0.0, x0=8.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    nl, mats, ds, pr = cycling_stack(rng, n_mirrors, n_layers, len(mat_n), prune_p=prune_p)
    xs = x0 + spacing * np.arange(n_mirrors)
    return Design(dims=dims, n_slab=n_slab, thickness_mm=t_mm, width_mm=20.0,
                  x_end_mm=float(xs[-1] + 10.0), eye_relief_mm=15.0, ic_tilt_deg=tilt,
                  mat_n=mat_n, mirror_x_mm=xs, mirror_tilt_deg=np.full(n_mirrors, tilt),
                  mirror_omega=default_omega(n_mirrors), n_layers=nl, layer_mat=mats,
                  layer_d_nm=ds, pruned=pr)


def cell_centres(fov_deg, n):
    return -0.5 * fov_deg + (np.arange(n) + 0.5) * (fov_deg / n)


# --------------------------------------------------------------------------
# Named configurations
# --------------------------------------------------------------------------

def tiny(n_rays=10_000, seed=7):
    """2D slab n=1.71, 1.0 mm, 2 mirrors at 25 deg spaced 1.5 mm, 8-layer
    SiO2/TiO2 stacks (d ~ U[10,200] nm, seed 1), 532 nm, 5 fields in +-10 deg,
    s+p pair, 1e4 rays, 64-bin 1D eyebox over 8 mm."""
    D = _prma_design(2, 1.71, 1.0, 2, 8, [N_SIO2, N_TIO2], seed=1)
    C = TraceConfig(lam_nm=[532.0], fx_deg=[-10.0, -5.0, 0.0, 5.0, 10.0], fy_deg=[0.0],
                    pol=POL_PAIR, n_rays=n_rays, seed=seed, eb_cx_mm=float(D.mirror_x_mm.mean()),
                    eb_w_mm=8.0, eb_h_mm=1.0, eb_nx=64, eb_ny=1)
    return D, C


def representative(n_rays=10_000_000, seed=11, n_layers=40, design_seed=2):
    """3D slab n=1.71, 1.5 mm, 6 mirrors at 25 deg, 40 layers cycling
    SiO2/TiO2/Ta2O5 (d ~ U[10,200] nm, seed 2), 460/532/630 nm, 32x18 field
    grid over 30x17 deg (cell centres), random linear polarization, 1e7 rays,
    10x8 mm eyebox on 64x48 bins."""
    D = _prma_design(3, 1.71, 1.5, 6, n_layers, [N_SIO2, N_TIO2, N_TA2O5], seed=design_seed)
    C = TraceConfig(lam_nm=[460.0, 532.0, 630.0], fx_deg=cell_centres(30.0, 32),
                    fy_deg=cell_centres(17.0, 18), pol=POL_RANDOM_LINEAR, n_rays=n_rays, seed=seed,
                    pupil_y_mm=8.0, eb_cx_mm=float(D.mirror_x_mm.mean()), eb_cy_mm=0.0,
                    eb_w_mm=10.0, eb_h_mm=8.0, eb_nx=64, eb_ny=48)
    return D, C


def differentiation(n_rays=100_000_000, seed=11):
    """As representative but 200 layers per mirror (1200 thickness parameters)
    plus 6 tilts, 1e8 rays."""
    return representative(n_rays=n_rays, seed=seed, n_layers=200, design_seed=2)


def _general_row(n0, pivot, axis, rect, t0):
    return list(n0) + list(pivot) + list(axis) + list(rect) + [t0]


def pupil_expander_design(n_fold=30, n_out=16, n_layers=23, seed=3, n_slab=1.9, t_mm=1.7, tilt=26.0,
                          fold_x0=5.0, fold_dx=0.5, band_mm=6.0, out_y0=8.0, out_dy=1.0,
                          mat_n=(N_TA2O5_PAPER, N_SIO2)):
    """Two-dimensional pupil expansion (Results, "System Architecture": a
    1.7 mm slab of index 1.9, an input mirror, 30 folding and 16 output
    mirrors, 23-layer Ta2O5/SiO2 stacks, thicknesses 20-200 nm). The paper
    gives no placement, so it is synthesized: guided light leaves the input
    mirror along +x; fold mirror k is the vertical plane x - y = fold_x0 +
    k fold_dx at 45 deg (a reflection swaps d_x and d_y, so TIR is kept),
    acting in the band |y| <= band_mm; the folded light travels along +y to
    output mirror j, the plane through (0, out_y0 + j out_dy, t/2) tilted
    about x by the input mirror's tilt, acting over the fold region's x
    range. Reflection probabilities follow the equal-extraction rule within
    each array. Tilt axes: z for the fold mirrors, x for the output mirrors."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = n_fold + n_out
    nl, mats, ds, pr = cycling_stack(rng, K, n_layers, len(mat_n), d_lo=20.0, d_hi=200.0)
    inf = np.inf
    s2 = np.sqrt(0.5)
    rows, xs, tilts = [], [], []
    for k in range(n_fold):
        xk = fold_x0 + fold_dx * k
        rows.append(_general_row((-s2, s2, 0.0), (xk, 0.0, 0.5 * t_mm), (0.0, 0.0, 1.0), (-inf, inf, -band_mm, band_mm),
                                 45.0))
        xs.append(xk)
        tilts.append(45.0)
    a = np.deg2rad(tilt)
    x_lo, x_hi = fold_x0 - band_mm - 2.0, fold_x0 + fold_dx * (n_fold - 1) + band_mm + 2.0
    for j in range(n_out):
        yj = out_y0 + out_dy * j
        rows.append(_general_row((0.0, -np.sin(a), np.cos(a)), (0.0, yj, 0.5 * t_mm), (1.0, 0.0, 0.0),
                                 (x_lo, x_hi, -inf, inf), tilt))
        xs.append(0.5 * (x_lo + x_hi))
        tilts.append(tilt)
    omega = np.concatenate([default_omega(n_fold), default_omega(n_out)])
    y_hi = out_y0 + out_dy * (n_out - 1) + t_mm / np.tan(a) + 1.0
    return Design(dims=3, n_slab=n_slab, thickness_mm=t_mm, width_mm=2.0 * y_hi, x_end_mm=x_hi + 1.0,
                  eye_relief_mm=15.0, ic_tilt_deg=tilt, mat_n=list(mat_n), mirror_x_mm=xs,
                  mirror_tilt_deg=tilts, mirror_omega=omega, n_layers=nl, layer_mat=mats, layer_d_nm=ds,
                  pruned=pr, mirror_geo=np.array(rows))


def pupil_expander(n_rays=10_000_000, seed=13, n_fields=16, eb_bins=64):
    """The two-dimensional pupil-expansion design (pupil_expander_design):
    9 wavelengths (450/470/490, 500/530/560, 620/660/700 nm), a 16x16 field
    grid over 38x38 deg (cell centres), random linear polarization, a
    1.6 mm panel, 16x16 mm eyebox at 15 mm eye relief centred over the output
    region, 64x64 bins."""
    D = pupil_expander_design()
    g = D.mirror_geo
    fold = g[:, 2] == 0.0
    xc = float(0.5 * (D.mirror_x_mm[fold].min() + D.mirror_x_mm[fold].max()))
    yc = float(0.5 * (g[~fold, 4].min() + g[~fold, 4].max()))
    C = TraceConfig(lam_nm=[450.0, 470.0, 490.0, 500.0, 530.0, 560.0, 620.0, 660.0, 700.0],
                    fx_deg=cell_centres(38.0, n_fields), fy_deg=cell_centres(38.0, n_fields),
                    pol=POL_RANDOM_LINEAR, n_rays=n_rays, seed=seed, pupil_y_mm=1.6, eb_cx_mm=xc, eb_cy_mm=yc,
                    eb_w_mm=16.0, eb_h_mm=16.0, eb_nx=eb_bins, eb_ny=eb_bins)
    return D, C


def pupil_expander_small(n_rays=20_000, seed=13):
    """A small two-dimensional expander for parity tests: 4 fold and 3 output
    mirrors with 6-layer stacks, 1 wavelength, 3x3 fields, 16x16 bins."""
    D = pupil_expander_design(n_fold=4, n_out=3, n_layers=6, fold_dx=1.5, band_mm=3.0, out_y0=5.0,
                              out_dy=1.5)
    g = D.mirror_geo
    fold = g[:, 2] == 0.0
    xc = float(0.5 * (D.mirror_x_mm[fold].min() + D.mirror_x_mm[fold].max()))
    yc = float(0.5 * (g[~fold, 4].min() + g[~fold, 4].max()))
    C = TraceConfig(lam_nm=[530.0], fx_deg=cell_centres(20.0, 3), fy_deg=cell_centres(20.0, 3),
                    pol=POL_RANDOM_LINEAR, n_rays=n_rays, seed=seed, pupil_y_mm=1.6, eb_cx_mm=xc, eb_cy_mm=yc,
                    eb_w_mm=12.0, eb_h_mm=12.0, eb_nx=16, eb_ny=16)
    return D, C


def batching(n_designs=64, seed=4):
    """64 designs: K ~ U{3..8}, L ~ U{10..200}, 30% of layers pruned (zero
    thickness), ray budgets log-uniform in [1e5, 1e7]; other parameters as in
    the representative configuration."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_designs):
        K = int(rng.integers(3, 9))
        L = rng.integers(10, 201, size=K)
        dseed = int(rng.integers(0, 2**31))
        D = _prma_design(3, 1.71, 1.5, K, L, [N_SIO2, N_TIO2, N_TA2O5], seed=dseed, prune_p=0.3)
        n = int(round(10 ** rng.uniform(5.0, 7.0)))
        C = TraceConfig(lam_nm=[460.0, 532.0, 630.0], fx_deg=cell_centres(30.0, 32),
                        fy_deg=cell_centres(17.0, 18), pol=POL_RANDOM_LINEAR, n_rays=n,
                        seed=int(rng.integers(0, 2**63)), pupil_y_mm=8.0,
                        eb_cx_mm=float(D.mirror_x_mm.mean()), eb_w_mm=10.0, eb_h_mm=8.0,
                        eb_nx=64, eb_ny=48)
        out.append((D, C))
    return out


def serving_trace(n_requests=2000, rate_hz=200.0, seed=5, fwd_bwd_frac=0.05):
    """Poisson arrivals (mean rate_hz); each request is a design evaluation
    drawn as in `batching`; a fraction are forward+backward requests at
    log-uniform 1e6..1e8 rays. Returns a list of dicts with arrival time (s),
    kind ('fwd' or 'fwd_bwd'), design and config."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    pool = batching(n_designs=64, seed=int(rng.integers(0, 2**31)))
    reqs = []
    for i in range(n_requests):
        D, C = pool[int(rng.integers(0, len(pool)))]
        kind = "fwd_bwd" if rng.uniform() < fwd_bwd_frac else "fwd"
        if kind == "fwd_bwd":
            C = C.replace(n_rays=int(round(10 ** rng.uniform(6.0, 8.0))))
        C = C.replace(seed=int(rng.integers(0, 2**63)))
        reqs.append(dict(arrival_s=float(t[i]), kind=kind, design=D, cfg=C))
    return reqs


def with_thickness(D: Design, d_nm) -> Design:
    return D.replace(layer_d_nm=_f32(d_nm))


def with_tilts(D: Design, tilt_deg) -> Design:
    return D.replace(mirror_tilt_deg=_f32(tilt_deg))


def gaussian_thickness(D: Design, seed=0, sigma_nm=30.0, lo_nm=20.0, hi_nm=200.0):
    """Starting thicknesses of an optimization (Results: a Gaussian centred at
    the midpoint of the thickness bounds; the spread is not given, 30 nm here),
    clipped to the bounds; layers the design prunes stay at 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.clip(rng.normal(0.5 * (lo_nm + hi_nm), sigma_nm, size=D.total_layers), lo_nm, hi_nm)
    return _f32(np.where(np.asarray(D.pruned, dtype=bool), 0.0, d))


def seeded_params(n_total, n_pick, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n_total, size=n_pick, replace=False))

