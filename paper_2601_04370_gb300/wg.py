"""Python binding of libwg.so (include/wg.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. Device buffers are torch
tensors (device memory and streams come from PyTorch); host buffers are numpy
arrays. If libwg.so is missing the import fails loudly: there is no CPU
fallback.

Names follow the C ABI: Context (wg_init / wg_shutdown), Context.create_design
(wg_create_design), DesignHandle.set_params (wg_set_params), trace_forward,
trace_backward, loss, eval_coating, eval_coating_grad. WGTrace is a
torch.autograd.Function over wg_trace_forward / wg_trace_backward.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwg.so")

WG_OK, WG_EINVAL, WG_ENOMEM, WG_EBUSY, WG_ENOTREADY, WG_ETIMEOUT, WG_ECANCELED, WG_EDEVICE, WG_ENOTFOUND = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "WG_OK", -1: "WG_EINVAL", -2: "WG_ENOMEM", -3: "WG_EBUSY", -4: "WG_ENOTREADY",
                -5: "WG_ETIMEOUT", -6: "WG_ECANCELED", -7: "WG_EDEVICE", -8: "WG_ENOTFOUND"}


class WGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class InitOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_slots", C.c_int32), ("hbm_budget_bytes", C.c_size_t),
                ("autotune_cache", C.c_char_p), ("wait_limit_ns", C.c_uint64), ("max_queue", C.c_int32),
                ("reserved", C.c_int32), ("max_batch_rays", C.c_int64)]


class TuneInfo(C.Structure):
    _fields_ = [("chunk_rays", C.c_int32), ("ctas_per_sm", C.c_int32), ("best_ms", C.c_float),
                ("n_tried", C.c_int32), ("tried_chunk_rays", C.c_int32 * 8), ("tried_ctas_per_sm", C.c_int32 * 8),
                ("tried_ms", C.c_float * 8)]


class DesignDesc(C.Structure):
    _fields_ = [("dims", C.c_int32), ("n_materials", C.c_int32), ("n_mirrors", C.c_int32), ("reserved", C.c_int32),
                ("n_slab", C.c_float), ("thickness_mm", C.c_float), ("width_mm", C.c_float),
                ("x_end_mm", C.c_float), ("eye_relief_mm", C.c_float), ("ic_tilt_deg", C.c_float),
                ("material_n", C.POINTER(C.c_float)), ("mirror_x_mm", C.POINTER(C.c_float)),
                ("mirror_tilt_deg", C.POINTER(C.c_float)), ("mirror_omega", C.POINTER(C.c_float)),
                ("n_layers", C.POINTER(C.c_int32)), ("layer_material", C.POINTER(C.c_int32)),
                ("layer_thickness_nm", C.POINTER(C.c_float)), ("layer_pruned", C.POINTER(C.c_uint8)),
                ("mirror_geometry", C.POINTER(C.c_float))]


class TraceCfg(C.Structure):
    _fields_ = [("n_lambda", C.c_int32), ("n_fx", C.c_int32), ("n_fy", C.c_int32), ("pol", C.c_int32),
                ("lambda_nm", C.POINTER(C.c_float)), ("field_x_deg", C.POINTER(C.c_float)),
                ("field_y_deg", C.POINTER(C.c_float)), ("n_rays", C.c_int64), ("seed", C.c_uint64),
                ("max_events", C.c_int32), ("eb_nx", C.c_int32), ("eb_ny", C.c_int32), ("flags", C.c_int32),
                ("pupil_y_mm", C.c_float), ("eb_cx_mm", C.c_float), ("eb_cy_mm", C.c_float),
                ("eb_w_mm", C.c_float), ("eb_h_mm", C.c_float), ("lut_bins", C.c_int32), ("stream", C.c_void_p),
                ("ray_begin", C.c_int64), ("ray_end", C.c_int64), ("ray_records", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("n_hits", C.c_int64), ("n_events", C.c_int64), ("n_tir", C.c_int64),
                ("n_layer_steps", C.c_int64), ("ledger", C.c_double * 6), ("kernel_ms", C.c_float),
                ("overflow", C.c_int32), ("n_tallied", C.c_int64), ("n_adjoint_steps", C.c_int64),
                ("n_nonfinite", C.c_int64), ("replay_ms", C.c_float), ("adjoint_ms", C.c_float),
                ("tilt_ms", C.c_float), ("n_adjoint_launches", C.c_int32)]

    def to_dict(self):
        return dict(n_rays=self.n_rays, n_hits=self.n_hits, n_events=self.n_events, n_tir=self.n_tir,
                    n_layer_steps=self.n_layer_steps, ledger=np.array(self.ledger[:]), kernel_ms=self.kernel_ms,
                    overflow=self.overflow, n_tallied=self.n_tallied, n_adjoint_steps=self.n_adjoint_steps,
                    n_nonfinite=self.n_nonfinite, replay_ms=self.replay_ms, adjoint_ms=self.adjoint_ms,
                    tilt_ms=self.tilt_ms, n_adjoint_launches=self.n_adjoint_launches)


# serving (include/wg.h)
REQ_FORWARD, REQ_LOSS_GRAD = 0, 1


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("loss_kind", C.c_int32), ("w_f", C.c_double), ("w_e", C.c_double),
                ("design", C.c_void_p), ("cfg", TraceCfg), ("tally", C.c_void_p), ("grad_thickness", C.c_void_p),
                ("loss", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("graph_replayed", C.c_int32),
                ("pad", C.c_int32), ("queue_ms", C.c_double), ("run_ms", C.c_double), ("stats", Stats)]

    def to_dict(self):
        return dict(status=self.status, batch_size=self.batch_size, graph_replayed=bool(self.graph_replayed),
                    queue_ms=self.queue_ms, run_ms=self.run_ms, stats=self.stats.to_dict())


# wg_trace_cfg.flags bits (include/wg.h)
TRACE_NO_EXIT_LIST = 1  # forward: do not list the eyebox rays for the adjoint

RAY_RECORD_DTYPE = np.dtype([("hash", np.uint32), ("n_events", np.int32), ("n_hits", np.int32),
                             ("cat", np.int32), ("bin", np.int32), ("I", np.float32), ("w", np.float32),
                             ("pad", np.int32)])

_lib = None


def lib():
    """The loaded libwg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwg.so not built ({LIB_PATH}); run python -m paper_2601_04370_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dp, fp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_void_p
        L.wg_init.argtypes = [C.POINTER(vp), C.POINTER(InitOpts)]
        L.wg_shutdown.argtypes = [vp]
        L.wg_shutdown.restype = None
        L.wg_last_error.restype = C.c_char_p
        L.wg_version.restype = C.c_char_p
        L.wg_kernel_launches.restype = C.c_uint64
        L.wg_create_design.argtypes = [vp, C.POINTER(DesignDesc), C.POINTER(vp)]
        L.wg_set_params.argtypes = [vp, fp, i64, fp, i32, vp]
        L.wg_destroy_design.argtypes = [vp]
        L.wg_destroy_design.restype = None
        L.wg_eval_coating.argtypes = [vp, vp, i32, i32, i64, fp, fp, fp, vp]
        L.wg_eval_coating_grad.argtypes = [vp, vp, i32, i32, i64, fp, fp, fp, i32, fp, vp]
        L.wg_eval_coating_dcos.argtypes = [vp, vp, i32, i32, i64, fp, fp, fp, i32, fp, vp]
        L.wg_trace_forward.argtypes = [vp, vp, C.POINTER(TraceCfg), vp, C.POINTER(Stats)]
        L.wg_trace_backward.argtypes = [vp, vp, C.POINTER(TraceCfg), vp, vp, vp, C.POINTER(Stats)]
        L.wg_loss.argtypes = [vp, vp, C.POINTER(TraceCfg), i32, C.c_double, C.c_double, vp, dp, vp]
        L.wg_trace_forward_noalloc.argtypes = [vp, vp, C.POINTER(TraceCfg), vp, C.POINTER(Stats)]
        L.wg_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.wg_poll.argtypes = [vp, C.c_uint64, i64, C.POINTER(Result)]
        L.wg_cancel.argtypes = [vp, C.c_uint64]
        L.wg_autotune.argtypes = [vp, vp, C.POINTER(TraceCfg)]
        L.wg_autotune_info.argtypes = [vp, vp, C.POINTER(TraceCfg), C.POINTER(TuneInfo)]
        L.wg_trace_forward_batch.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.wg_omega_trace.argtypes = [vp, vp, C.POINTER(TraceCfg), vp, vp, vp]
        L.wg_set_omega.argtypes = [vp, vp, i32, vp]
        L.wg_adam_create.argtypes = [vp, C.POINTER(AdamOpts), vp, C.POINTER(vp)]
        L.wg_adam_step.argtypes = [vp, vp, vp]
        L.wg_adam_params.argtypes = [vp, vp, vp]
        L.wg_adam_destroy.argtypes = [vp]
        L.wg_adam_destroy.restype = None
        L.wg_omega_adam_create.argtypes = [vp, C.POINTER(OmegaAdamOpts), C.POINTER(vp)]
        L.wg_omega_adam_step.argtypes = [vp, vp, vp, vp]
        L.wg_omega_adam_destroy.argtypes = [vp]
        L.wg_omega_adam_destroy.restype = None
        L.wg_design_version.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.wg_test_bounded_wait.argtypes = [vp, C.c_uint64]
        for name in ("wg_init", "wg_create_design", "wg_set_params", "wg_eval_coating", "wg_eval_coating_grad",
                     "wg_trace_forward", "wg_trace_backward", "wg_loss", "wg_trace_forward_noalloc",
                     "wg_submit", "wg_poll", "wg_cancel", "wg_autotune", "wg_omega_trace", "wg_set_omega",
                     "wg_adam_create", "wg_adam_step", "wg_adam_params", "wg_omega_adam_create",
                     "wg_omega_adam_step", "wg_design_version", "wg_autotune_info",
                     "wg_trace_forward_batch", "wg_eval_coating_dcos", "wg_test_bounded_wait"):
            getattr(L, name).restype = C.c_int32
        _lib = L
    return _lib


def _check(st):
    if st != WG_OK:
        raise WGError(st, lib().wg_last_error().decode())


def _ptr(x) -> Optional[int]:
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None


class _CfgHolder:
    """A TraceCfg whose host arrays stay alive as long as the holder."""

    def __init__(self, cfg, stream=None, rays=None, records=None, flags=0):
        self.lam = np.ascontiguousarray(cfg.lam_nm, dtype=np.float32)
        self.fx = np.ascontiguousarray(cfg.fx_deg, dtype=np.float32)
        self.fy = np.ascontiguousarray(cfg.fy_deg, dtype=np.float32)
        rb, re = (0, 0) if rays is None else (int(rays[0]), int(rays[1]))
        self.c = TraceCfg(n_lambda=len(self.lam), n_fx=len(self.fx), n_fy=len(self.fy), pol=int(cfg.pol),
                          lambda_nm=_fptr(self.lam), field_x_deg=_fptr(self.fx), field_y_deg=_fptr(self.fy),
                          n_rays=int(cfg.n_rays), seed=int(cfg.seed), max_events=int(cfg.max_events),
                          eb_nx=int(cfg.eb_nx), eb_ny=int(cfg.eb_ny), flags=int(flags), pupil_y_mm=cfg.pupil_y_mm,
                          eb_cx_mm=cfg.eb_cx_mm, eb_cy_mm=cfg.eb_cy_mm, eb_w_mm=cfg.eb_w_mm, eb_h_mm=cfg.eb_h_mm,
                          lut_bins=int(getattr(cfg, "lut_bins", 0)),
                          stream=stream, ray_begin=rb, ray_end=re, ray_records=_ptr(records))


class AdamOpts(C.Structure):
    _fields_ = [("lr_nm", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("d_min_nm", C.c_float), ("d_max_nm", C.c_float)]


class OmegaAdamOpts(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("lo", C.c_float), ("hi", C.c_float)]


class OmegaAdam:
    """Optimizer of a design's reflection probabilities (wg_omega_adam_*):
    Adam on omega with the gradient of a loss to minimize, clipped to
    [lo, hi]; each step writes omega to the design."""

    def __init__(self, dh, lr=0.02, beta1=0.9, beta2=0.999, eps=1e-8, lo=0.02, hi=0.98):
        self.n = dh.design.n_mirrors
        o = OmegaAdamOpts(lr, beta1, beta2, eps, lo, hi)
        h = C.c_void_p()
        _check(lib().wg_omega_adam_create(dh.h, C.byref(o), C.byref(h)))
        self.h = h

    def step(self, grad_omega, stream=None):
        """grad_omega: FP64 [K] (torch CUDA tensor or numpy array). Returns the new omega (FP32)."""
        out = np.zeros(self.n, dtype=np.float32)
        _check(lib().wg_omega_adam_step(self.h, _ptr(grad_omega), out.ctypes.data,
                                        stream if stream is not None else _current_stream()))
        return out

    def close(self):
        if self.h:
            lib().wg_omega_adam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adam:
    """Thickness optimizer of a design (wg_adam_*): Adam in nm, then the
    projection onto [0, d_max] with the soft gap (0, d_min) (0 below
    d_min / 2, else d_min). Each step writes the thicknesses to the design."""

    def __init__(self, dh, lr_nm=2.0, beta1=0.9, beta2=0.999, eps=1e-8, d_min_nm=20.0, d_max_nm=200.0,
                 thickness_nm=None):
        self.dh = dh
        self.n = dh.n_params
        o = AdamOpts(lr_nm, beta1, beta2, eps, d_min_nm, d_max_nm)
        h = C.c_void_p()
        keep = None
        ptr = None
        if thickness_nm is not None:
            if hasattr(thickness_nm, "data_ptr") and thickness_nm.is_cuda:
                ptr = thickness_nm.data_ptr()
            else:
                keep = np.ascontiguousarray(np.asarray(thickness_nm, dtype=np.float32))
                ptr = keep.ctypes.data
        _check(lib().wg_adam_create(dh.h, C.byref(o), ptr, C.byref(h)))
        self.h = h

    def step(self, grad_thickness, stream=None):
        """grad_thickness: FP64 [n] (torch CUDA tensor or numpy array)."""
        _check(lib().wg_adam_step(self.h, _ptr(grad_thickness), stream if stream is not None else _current_stream()))

    def params(self):
        out = np.zeros(self.n, dtype=np.float32)
        _check(lib().wg_adam_params(self.h, out.ctypes.data, None))
        return out

    def close(self):
        if self.h:
            lib().wg_adam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def optimize(ctx, dh, cfg, n_iter, adam=None, loss_kind=0, w_f=10.0, w_e=3.0, callback=None):
    """Thickness optimization of a design (the paper's loop, Results: the
    loss of Eq. 1 on the traced tally, its adjoint, one optimizer step per
    iteration). The Philox keys stay the same every iteration, so the
    objective is a deterministic function of the thicknesses. Returns the
    per-iteration (L, I_mean, U_fov, U_eyebox) and the optimizer."""
    import torch
    adam = adam if adam is not None else Adam(dh)
    tally = torch.zeros(cfg.tally_shape, dtype=torch.float64, device="cuda")
    G = torch.zeros_like(tally)
    g = torch.zeros(dh.n_params, dtype=torch.float64, device="cuda")
    hist = []
    for it in range(n_iter):
        ctx.trace_forward(dh, cfg, tally, stats=False)
        hist.append(ctx.loss(dh, cfg, tally, G, kind=loss_kind, w_f=w_f, w_e=w_e))
        ctx.trace_backward(dh, cfg, G, g, stats=False)
        adam.step(g)
        if callback is not None:
            callback(it, hist[-1], adam)
    return np.array(hist), adam


def optimize_omega(ctx, dh, cfg, n_iter, lr=0.02, lo=0.02, hi=0.98, beta1=0.9, beta2=0.999, eps=1e-8):
    """Reflection-probability pre-optimization (Methods, "Learned reflection
    probabilities"): maximizes the mean pupil throughput I_mean (the
    brightness term of Eq. 1) of the scalar-reflectance geometric model over
    the mirrors' omega. Each iteration traces cfg's rays (wg_omega_trace,
    fixed Philox keys), takes the score-function gradient and one Adam step
    on the K values (wg_omega_adam_step, on the GPU), clipped to [lo, hi],
    which sets omega. Returns the per-iteration I_mean and the final omega."""
    import torch
    tally = torch.zeros(cfg.tally_shape, dtype=torch.float64, device="cuda")
    G = torch.zeros_like(tally)
    ctx.loss(dh, cfg, tally, G, w_f=0.0, w_e=0.0)  # dL/dtally of L = -I_mean: the pupil masks, any tally
    g = torch.zeros(dh.design.n_mirrors, dtype=torch.float64, device="cuda")
    opt = OmegaAdam(dh, lr=lr, beta1=beta1, beta2=beta2, eps=eps, lo=lo, hi=hi)
    om = np.asarray(dh.design.mirror_omega, dtype=np.float32).copy()
    hist = []
    for _ in range(n_iter):
        ctx.omega_trace(dh, cfg, tally, G, g)
        hist.append(ctx.loss(dh, cfg, tally, w_f=0.0, w_e=0.0)[1])
        om = opt.step(g)
    opt.close()
    ctx.omega_trace(dh, cfg, tally)
    hist.append(ctx.loss(dh, cfg, tally, w_f=0.0, w_e=0.0)[1])
    return np.array(hist), om


class DesignHandle:
    def __init__(self, ctx, handle, design):
        self.ctx = ctx
        self.h = handle
        self.design = design

    def set_omega(self, omega, stream=None):
        """wg_set_omega: the mirrors' reflection probabilities ([K], each in (0, 1))."""
        a = np.ascontiguousarray(np.asarray(omega, dtype=np.float32))
        _check(lib().wg_set_omega(self.h, a.ctypes.data, int(a.size), stream if stream is not None else _current_stream()))

    @property
    def n_params(self):
        """Layer thicknesses of the design (its gradient's length)."""
        return int(self.design.total_layers)

    def set_params(self, thickness_nm=None, tilt_deg=None, stream=None):
        th = tl = None
        nth = ntl = 0
        keep = []
        if thickness_nm is not None:
            if hasattr(thickness_nm, "data_ptr") and thickness_nm.is_cuda:
                th = thickness_nm.data_ptr()
                nth = thickness_nm.numel()
            else:
                a = np.ascontiguousarray(np.asarray(thickness_nm, dtype=np.float32))
                keep.append(a)
                th, nth = a.ctypes.data, a.size
        if tilt_deg is not None:
            a = np.ascontiguousarray(np.asarray(tilt_deg, dtype=np.float32))
            keep.append(a)
            tl, ntl = a.ctypes.data, a.size
        _check(lib().wg_set_params(self.h, th, nth, tl, ntl, stream if stream is not None else _current_stream()))

    def version(self):
        """wg_design_version: increases with every change of the parameters."""
        v = C.c_uint64()
        _check(lib().wg_design_version(self.h, C.byref(v)))
        return int(v.value)

    def destroy(self):
        if self.h:
            lib().wg_destroy_design(self.h)
            self.h = None


class Context:
    def __init__(self, device: int = 0, max_slots: int = 0, hbm_budget_bytes: int = 0,
                 autotune_cache: Optional[str] = None, wait_limit_ns: int = 0, max_queue: int = 0,
                 max_batch_rays: int = 0):
        h = C.c_void_p()
        self._cache = autotune_cache.encode() if autotune_cache else None
        opts = InitOpts(device=device, max_slots=max_slots, hbm_budget_bytes=hbm_budget_bytes,
                        autotune_cache=self._cache, wait_limit_ns=wait_limit_ns, max_queue=max_queue,
                        max_batch_rays=max_batch_rays)
        _check(lib().wg_init(C.byref(h), C.byref(opts)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            lib().wg_shutdown(self.h)
            self.h = None

    # ---- serving ----
    def submit(self, dh, cfg, kind=REQ_FORWARD, tally=None, grad=None, loss=None, loss_kind=0, w_f=10.0, w_e=3.0):
        """wg_submit: returns a ticket. tally / grad: host (numpy float64) or
        device (torch float64) buffers, loss: numpy float64[4]; they must stay
        alive until the ticket is polled done."""
        h = _CfgHolder(cfg, None)
        r = Request(kind=kind, loss_kind=loss_kind, w_f=w_f, w_e=w_e, design=dh.h, cfg=h.c, tally=_ptr(tally),
                    grad_thickness=_ptr(grad), loss=_ptr(loss))
        t = C.c_uint64()
        _check(lib().wg_submit(self.h, C.byref(r), C.byref(t)))
        return int(t.value)

    def poll(self, ticket, timeout_us=-1):
        """wg_poll: the result dict when done, None while pending (timeout)."""
        res = Result()
        st = lib().wg_poll(self.h, ticket, int(timeout_us), C.byref(res))
        if st == WG_ENOTREADY:
            return None
        _check(st)
        out = res.to_dict()
        if out["status"] != WG_OK:
            out["error"] = lib().wg_last_error().decode()
        return out

    def cancel(self, ticket):
        _check(lib().wg_cancel(self.h, ticket))

    def test_bounded_wait(self, limit_ns: int):
        """wg_test_bounded_wait: a device wait on a flag that nothing sets
        gives up after limit_ns; raises WGError (WG_ETIMEOUT)."""
        _check(lib().wg_test_bounded_wait(self.h, int(limit_ns)))

    def autotune(self, dh, cfg):
        h = _CfgHolder(cfg, None)
        _check(lib().wg_autotune(self.h, dh.h, C.byref(h.c)))

    def trace_forward_batch(self, dhs, cfgs, tallies, stats=True):
        """wg_trace_forward_batch: the forwards of several designs in one fused
        launch per kernel variant (autotuned shapes, graph replay of a
        composition met before). tallies: torch CUDA float64 tensors.
        Returns (list of stats dicts or None, graph_replayed)."""
        n = len(dhs)
        holders = [_CfgHolder(c, None) for c in cfgs]
        carr = (TraceCfg * n)(*[h.c for h in holders])
        darr = (C.c_void_p * n)(*[dh.h.value if hasattr(dh.h, "value") else dh.h for dh in dhs])
        tarr = (C.c_void_p * n)(*[_ptr(t) for t in tallies])
        st = (Stats * n)() if stats else None
        rep = C.c_int32(0)
        _check(lib().wg_trace_forward_batch(self.h, n, darr, carr, tarr, st, C.byref(rep)))
        return ([s.to_dict() for s in st] if stats else None), bool(rep.value)

    def autotune_info(self, dh, cfg):
        """wg_autotune_info: the launch shape stored for the class of (dh, cfg)
        and the candidates timed for it, as a dict (None if there is none)."""
        h = _CfgHolder(cfg, None)
        t = TuneInfo()
        st = lib().wg_autotune_info(self.h, dh.h, C.byref(h.c), C.byref(t))
        if st == WG_ENOTFOUND:
            return None
        _check(st)
        n = t.n_tried
        return {"chunk_rays": t.chunk_rays, "ctas_per_sm": t.ctas_per_sm, "best_ms": t.best_ms, "n_tried": n,
                "tried": [(t.tried_chunk_rays[i], t.tried_ctas_per_sm[i], t.tried_ms[i]) for i in range(n)]}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def create_design(self, D) -> DesignHandle:
        keep = [np.ascontiguousarray(D.mat_n, dtype=np.float32), np.ascontiguousarray(D.mirror_x_mm, dtype=np.float32),
                np.ascontiguousarray(D.mirror_tilt_deg, dtype=np.float32),
                np.ascontiguousarray(D.mirror_omega, dtype=np.float32),
                np.ascontiguousarray(D.n_layers, dtype=np.int32), np.ascontiguousarray(D.layer_mat, dtype=np.int32),
                np.ascontiguousarray(D.layer_d_nm, dtype=np.float32), np.ascontiguousarray(D.pruned, dtype=np.uint8)]
        desc = DesignDesc(dims=D.dims, n_materials=len(keep[0]), n_mirrors=len(keep[1]), reserved=0,
                          n_slab=D.n_slab, thickness_mm=D.thickness_mm, width_mm=D.width_mm, x_end_mm=D.x_end_mm,
                          eye_relief_mm=D.eye_relief_mm, ic_tilt_deg=D.ic_tilt_deg, material_n=_fptr(keep[0]),
                          mirror_x_mm=_fptr(keep[1]), mirror_tilt_deg=_fptr(keep[2]), mirror_omega=_fptr(keep[3]),
                          n_layers=keep[4].ctypes.data_as(C.POINTER(C.c_int32)),
                          layer_material=keep[5].ctypes.data_as(C.POINTER(C.c_int32)),
                          layer_thickness_nm=_fptr(keep[6]), layer_pruned=keep[7].ctypes.data_as(C.POINTER(C.c_uint8)))
        geo = getattr(D, "mirror_geo", None)
        if geo is not None:
            keep.append(np.ascontiguousarray(geo, dtype=np.float32).reshape(-1))
            desc.mirror_geometry = _fptr(keep[-1])
        h = C.c_void_p()
        _check(lib().wg_create_design(self.h, C.byref(desc), C.byref(h)))
        return DesignHandle(self, h, D)

    # ---- coating hooks ----
    def eval_coating(self, dh, mirror, side, cos_theta, lambda_nm, out, stream=None):
        _check(lib().wg_eval_coating(self.h, dh.h, mirror, side, cos_theta.numel(), _ptr(cos_theta), _ptr(lambda_nm),
                                     _ptr(out), stream if stream is not None else _current_stream()))

    def eval_coating_grad(self, dh, mirror, side, cos_theta, lambda_nm, weights, which, grad, stream=None):
        _check(lib().wg_eval_coating_grad(self.h, dh.h, mirror, side, cos_theta.numel(), _ptr(cos_theta),
                                          _ptr(lambda_nm), _ptr(weights), which, _ptr(grad),
                                          stream if stream is not None else _current_stream()))

    # ---- trace ----
    def eval_coating_dcos(self, dh, mirror, side, cos_theta, lambda_nm, weights, which, grad_cos, stream=None):
        """wg_eval_coating_dcos: d f / d(cos theta_0) through the coating (device FP32 [n])."""
        _check(lib().wg_eval_coating_dcos(self.h, dh.h, mirror, side, cos_theta.numel(), _ptr(cos_theta),
                                          _ptr(lambda_nm), _ptr(weights), which, _ptr(grad_cos),
                                          stream if stream is not None else _current_stream()))

    def trace_forward(self, dh, cfg, tally, stats=True, stream=None, rays=None, records=None, flags=0):
        """tally: torch CUDA float64 tensor (device path) or numpy float64 array
        (host path, copies inside the call). flags: TRACE_* bits. Returns the
        stats dict or None."""
        h = _CfgHolder(cfg, stream if stream is not None else _current_stream(), rays, records, flags)
        st = Stats() if stats else None
        _check(lib().wg_trace_forward(self.h, dh.h, C.byref(h.c), _ptr(tally), C.byref(st) if stats else None))
        return st.to_dict() if stats else None

    def trace_forward_noalloc(self, dh, cfg, tally, stats=True, stream=None, rays=None):
        """wg_trace_forward_noalloc: the forward trace for callers that cannot
        allocate device memory; tally must be a CUDA tensor (float64)."""
        h = _CfgHolder(cfg, stream if stream is not None else _current_stream(), rays)
        st = Stats() if stats else None
        _check(lib().wg_trace_forward_noalloc(self.h, dh.h, C.byref(h.c), _ptr(tally),
                                              C.byref(st) if stats else None))
        return st.to_dict() if stats else None

    def trace_backward(self, dh, cfg, dL_dtally, grad_thickness, stats=True, stream=None, rays=None,
                       grad_tilt=None):
        """grad_thickness (and grad_tilt, [n_mirrors] per degree, optional):
        torch CUDA float64 tensors or numpy float64 arrays, overwritten."""
        h = _CfgHolder(cfg, stream if stream is not None else _current_stream(), rays)
        st = Stats() if stats else None
        _check(lib().wg_trace_backward(self.h, dh.h, C.byref(h.c), _ptr(dL_dtally), _ptr(grad_thickness),
                                       _ptr(grad_tilt), C.byref(st) if stats else None))
        return st.to_dict() if stats else None

    def omega_trace(self, dh, cfg, tally, dL_dtally=None, grad_omega=None, stream=None):
        """wg_omega_trace: the reflection-probability model's geometric trace
        (scalar reflectance = omega, no polarization): tally, and with
        dL_dtally the score-function dL/d omega into grad_omega ([K] FP64)."""
        h = _CfgHolder(cfg, stream if stream is not None else _current_stream())
        _check(lib().wg_omega_trace(self.h, dh.h, C.byref(h.c), _ptr(dL_dtally), _ptr(tally), _ptr(grad_omega)))

    def loss(self, dh, cfg, tally, dL_dtally=None, kind=0, w_f=10.0, w_e=3.0, stream=None):
        """Returns (L, I_mean, U_fov, U_eyebox); fills dL_dtally if given."""
        h = _CfgHolder(cfg, stream if stream is not None else _current_stream())
        out = np.zeros(4)
        _check(lib().wg_loss(self.h, dh.h, C.byref(h.c), kind, w_f, w_e, _ptr(tally),
                             out.ctypes.data_as(C.POINTER(C.c_double)), _ptr(dL_dtally)))
        return tuple(float(x) for x in out)


def version() -> str:
    return lib().wg_version().decode()


def kernel_launches() -> int:
    """Kernels launched by libwg.so in this process so far."""
    return int(lib().wg_kernel_launches())


def _torch_autograd():
    import torch

    class WGTrace(torch.autograd.Function):
        """tally = WGTrace.apply(thickness_nm, ctx, design_handle, cfg[, tilt_deg]).

        forward: wg_set_params (thicknesses, and the mirror tilts in degrees
        when given) + wg_trace_forward; backward: wg_trace_backward with
        grad_output as dL/dtally, returning dL/dthickness and, for a tilt
        tensor, dL/dtilt per degree (FP64 -> the inputs' dtypes). The
        backward differentiates the design as it is when it runs, so it
        refuses (RuntimeError) when the design's parameters changed after its
        forward (another forward or an optimizer step on the same handle)."""

        @staticmethod
        def forward(actx, thickness, ctx, dh, cfg, tilt_deg=None):
            tl = None if tilt_deg is None else tilt_deg.detach().float().cpu().numpy()
            dh.set_params(thickness_nm=thickness.detach().float().contiguous(), tilt_deg=tl)
            tally = torch.empty(cfg.tally_shape, dtype=torch.float64, device=thickness.device)
            ctx.trace_forward(dh, cfg, tally, stats=False)
            actx.wg = (ctx, dh, cfg)
            actx.version = dh.version()
            actx.n = thickness.numel()
            actx.dtype = thickness.dtype
            actx.tilt = None if tilt_deg is None else (tilt_deg.numel(), tilt_deg.dtype, tilt_deg.device)
            return tally

        @staticmethod
        def backward(actx, grad_tally):
            ctx, dh, cfg = actx.wg
            if dh.version() != actx.version:
                raise RuntimeError("WGTrace.backward: the design's parameters changed after this forward "
                                   "(another forward or an optimizer step on the same design handle); "
                                   "its gradient would be taken at other parameters")
            g = torch.empty(actx.n, dtype=torch.float64, device=grad_tally.device)
            gt = None
            if actx.tilt is not None and actx.needs_input_grad[4]:
                gt = torch.empty(actx.tilt[0], dtype=torch.float64, device=grad_tally.device)
            ctx.trace_backward(dh, cfg, grad_tally.contiguous().to(torch.float64), g, stats=False, grad_tilt=gt)
            g_tilt = None if gt is None else gt.to(device=actx.tilt[2], dtype=actx.tilt[1])
            return g.to(actx.dtype), None, None, None, g_tilt

    return WGTrace


def __getattr__(name):
    if name == "WGTrace":
        return _torch_autograd()
    raise AttributeError(name)
