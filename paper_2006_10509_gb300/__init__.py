"""Python binding of libhologen (GB300 phase-retrieval library) -- ctypes over the C ABI.

The functions below carry the C names (``hg_plan_create``, ``hg_propagate``, ``hg_gs_run`` ...) and
only marshal arguments: torch tensors become device pointers, the current torch stream becomes the
``cudaStream_t``, and a non-OK status becomes :class:`HologenError`.  Every step of the computation
runs in the library's CUDA kernels; there is no fallback path.  The library is built in-tree by
``paper_2006_10509_gb300.build.build()``; importing this package does not load it, the first call
does, and fails loudly if it has not been built.

Layout conventions follow ``include/hologen.h``: complex64 [H][W] fields (torch.complex64), float32
[H][W] images, FFT order (DC at [0][0]).
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

__all__ = [
    "HG_OK", "HG_ERR_INVALID_ARG", "HG_ERR_UNSUPPORTED_SIZE", "HG_ERR_OUT_OF_MEMORY", "HG_ERR_CUDA",
    "HG_ERR_TIMEOUT", "HG_ERR_INTERNAL", "HG_FOURIER", "HG_FRESNEL",
    "HologenError", "lib_path", "load", "hg_plan_create", "hg_plan_destroy", "hg_plan_sync",
    "hg_propagate", "hg_gs_run", "hg_status_string", "hg_last_error", "hg_supported_length", "Plan",
    "hg_plan_set_timing", "hg_plan_reset_timing", "hg_plan_kernel_time", "hg_kernel_kind_name",
    "hg_plan_launch_count", "hg_gs_run_noalloc", "hg_ospr_run", "hg_gd_step", "hg_gd_forward",
    "hg_gd_backward", "hologram_loss", "hg_plan_set_graph", "hg_plan_item_latency", "hg_plan_autotune",
    "hg_plan_strip_width", "hg_plan_set_strip_width", "HG_PLAN_AUTOTUNE", "hg_mraf_run",
    "hg_plan_set_illumination", "hg_hio_run", "HG_TARGET_CENTRED", "HG_STRIP_CLUSTER", "hg_dbs_run", "hg_sa_run", "hg_plan_set_slm_levels",
]

HG_OK, HG_ERR_INVALID_ARG, HG_ERR_UNSUPPORTED_SIZE, HG_ERR_OUT_OF_MEMORY = 0, 1, 2, 3
HG_ERR_CUDA, HG_ERR_TIMEOUT, HG_ERR_INTERNAL = 4, 5, 6
HG_FOURIER, HG_FRESNEL = 0, 1
HG_PLAN_AUTOTUNE = 1  # plan flag: autotune the strip widths at creation
HG_TARGET_CENTRED = 2  # plan flag: targets and signal masks in display order (DC at H/2, W/2)
HG_STRIP_CLUSTER = -1  # strip width: the whole GS run in one thread-block cluster per item

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "libhologen.so")


class hg_plan_desc(ctypes.Structure):
    _fields_ = [
        ("n_items", ctypes.c_int32),
        ("heights", ctypes.POINTER(ctypes.c_int32)),
        ("widths", ctypes.POINTER(ctypes.c_int32)),
        ("propagation", ctypes.c_int32),
        ("wavelength_m", ctypes.c_double),
        ("pitch_m", ctypes.c_double),
        ("n_planes", ctypes.c_int32),
        ("z_m", ctypes.POINTER(ctypes.c_double)),
        ("quant_levels", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]


class HologenError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        self.status = status
        super().__init__(f"{func}: {_status_name(status)}: {detail}")


_VP = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)

_SIGNATURES = {
    "hg_plan_create": (ctypes.c_int, [ctypes.POINTER(hg_plan_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "hg_plan_destroy": (ctypes.c_int, [_VP]),
    "hg_plan_sync": (ctypes.c_int, [_VP]),
    "hg_propagate": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _PP, _PP, _VP]),
    "hg_gs_run": (ctypes.c_int, [_VP, _PP, _PP, ctypes.c_uint64, ctypes.c_int32, _PP, _PP, _VP, _VP]),
    "hg_ospr_run": (ctypes.c_int, [_VP, _PP, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _PP, _VP, _VP]),
    "hg_gd_step": (ctypes.c_int, [_VP, _PP, _PP, _PP, _PP, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, _VP, _PP, _VP]),
    "hg_gd_forward": (ctypes.c_int, [_VP, _PP, _PP, _VP, _VP]),
    "hg_gd_backward": (ctypes.c_int, [_VP, _PP, _PP, _VP, _PP, _VP]),
    "hg_gs_run_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP, ctypes.c_uint64,
                                         ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "hg_plan_set_timing": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "hg_plan_reset_timing": (ctypes.c_int, [_VP]),
    "hg_plan_kernel_time": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "hg_kernel_kind_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "hg_plan_launch_count": (ctypes.c_int64, [_VP]),
    "hg_plan_set_graph": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "hg_plan_set_illumination": (ctypes.c_int, [_VP, _PP]),
    "hg_plan_set_slm_levels": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "hg_mraf_run": (ctypes.c_int, [_VP, _PP, _PP, ctypes.c_float, _PP, ctypes.c_uint64, ctypes.c_int32, _PP, _PP,
                                   _VP, _VP]),
    "hg_hio_run": (ctypes.c_int, [_VP, _PP, _PP, ctypes.c_float, _PP, ctypes.c_uint64, ctypes.c_int32, _PP, _PP,
                                  _VP, _VP]),
    "hg_dbs_run": (ctypes.c_int, [_VP, _PP, _PP, ctypes.c_uint64, ctypes.c_int32, _PP, _PP, _VP, _VP]),
    "hg_sa_run": (ctypes.c_int, [_VP, _PP, _PP, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                 _PP, _PP, _VP, _VP]),
    "hg_plan_item_latency": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "hg_plan_autotune": (ctypes.c_int, [_VP, _VP]),
    "hg_plan_strip_width": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "hg_plan_set_strip_width": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "hg_plan_radix_plan": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "hg_plan_set_radix_plan": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "hg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hg_last_error": (ctypes.c_char_p, []),
    "hg_supported_length": (ctypes.c_int32, [ctypes.c_int32]),
}


def load():
    """Loads libhologen.so (once).  Raises RuntimeError if it has not been built."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_2006_10509_gb300.build` "
                "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _status_name(s: int) -> str:
    try:
        return load().hg_status_string(s).decode()
    except Exception:  # noqa: BLE001 - naming a status must never raise
        return f"status {s}"


def _check(status: int, func: str):
    if status != HG_OK:
        raise HologenError(status, func, load().hg_last_error().decode())


def _ptr_array(items) -> ctypes.Array | None:
    """Host array of device pointers from a sequence of tensors / None (None stays NULL)."""
    if items is None:
        return None
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = None if t is None else _data_ptr(t)
    return arr


def _data_ptr(t) -> int:
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hg_status_string(status: int) -> str:
    return load().hg_status_string(status).decode()


def hg_last_error() -> str:
    return load().hg_last_error().decode()


def hg_supported_length(n: int) -> bool:
    return bool(load().hg_supported_length(n))


def hg_plan_create(heights: Sequence[int], widths: Sequence[int], propagation: int = HG_FOURIER,
                   wavelength_m: float = 0.0, pitch_m: float = 0.0, z_m: Sequence[float] | None = None,
                   quant_levels: int = 0, flags: int = 0) -> int:
    """Creates a plan on the current device; returns the opaque handle (int)."""
    n = len(heights)
    hs = (ctypes.c_int32 * n)(*heights)
    ws = (ctypes.c_int32 * len(widths))(*widths)
    zs = (ctypes.c_double * len(z_m))(*z_m) if z_m else None
    d = hg_plan_desc(n, hs, ws, propagation, wavelength_m, pitch_m, len(z_m) if z_m else 1, zs,
                     quant_levels, flags)
    out = ctypes.c_void_p()
    _check(load().hg_plan_create(ctypes.byref(d), ctypes.byref(out)), "hg_plan_create")
    return out.value


def hg_plan_destroy(plan: int | None):
    _check(load().hg_plan_destroy(plan), "hg_plan_destroy")


def hg_plan_sync(plan: int):
    _check(load().hg_plan_sync(plan), "hg_plan_sync")


def hg_propagate(plan: int, plane: int, direction: int, inputs, outputs, stream=None):
    """out_k = F(in_k c) (direction +1) or conj(c) F^-1(in_k) (direction -1) for every item."""
    _check(load().hg_propagate(plan, plane, direction, _ptr_array(inputs), _ptr_array(outputs), _stream(stream)),
           "hg_propagate")


def hg_gs_run(plan: int, target_amp, init_phase=None, seed: int = 0, n_iter: int = 1, phase_out=None,
              level_out=None, nmse_out=None, stream=None):
    """Gerchberg-Saxton for every item of the plan (see hologen.h for the argument layout)."""
    _check(load().hg_gs_run(plan, _ptr_array(target_amp), _ptr_array(init_phase), seed, n_iter,
                            _ptr_array(phase_out), _ptr_array(level_out),
                            None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_gs_run")


def hg_plan_set_illumination(plan: int, illum_amp=None):
    """Per-item SLM illumination amplitude tensors (None entries: uniform); None clears."""
    _check(load().hg_plan_set_illumination(plan, _ptr_array(illum_amp)), "hg_plan_set_illumination")


def hg_plan_set_slm_levels(plan: int, levels=None):
    """Complex SLM values (a sequence of complex numbers) for a multi-amplitude SLM; None restores the
    plan's phase-only levels."""
    if levels is None:
        _check(load().hg_plan_set_slm_levels(plan, None, 0), "hg_plan_set_slm_levels")
        return
    vals = [complex(v) for v in levels]
    arr = (ctypes.c_float * (2 * len(vals)))(*[x for v in vals for x in (v.real, v.imag)])
    _check(load().hg_plan_set_slm_levels(plan, arr, len(vals)), "hg_plan_set_slm_levels")


def hg_mraf_run(plan: int, target_amp, mix: float, signal_mask=None, init_phase=None, seed: int = 0,
                n_iter: int = 1, phase_out=None, level_out=None, nmse_out=None, stream=None):
    """Mixed-region amplitude freedom for every item of a single-plane plan (see hologen.h)."""
    _check(load().hg_mraf_run(plan, _ptr_array(target_amp), _ptr_array(signal_mask), mix, _ptr_array(init_phase),
                              seed, n_iter, _ptr_array(phase_out), _ptr_array(level_out),
                              None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_mraf_run")


def hg_dbs_run(plan: int, target_amp, init_phase=None, seed: int = 0, n_sweeps: int = 1, phase_out=None,
               level_out=None, nmse_out=None, stream=None):
    """Direct binary search for every item of a binary single-plane plan (see hologen.h)."""
    _check(load().hg_dbs_run(plan, _ptr_array(target_amp), _ptr_array(init_phase), seed, n_sweeps,
                             _ptr_array(phase_out), _ptr_array(level_out),
                             None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_dbs_run")


def hg_sa_run(plan: int, target_amp, t0: float, alpha: float, init_phase=None, seed: int = 0, n_sweeps: int = 1,
              phase_out=None, level_out=None, nmse_out=None, stream=None):
    """Simulated annealing for every item of a binary single-plane plan (see hologen.h)."""
    _check(load().hg_sa_run(plan, _ptr_array(target_amp), _ptr_array(init_phase), seed, n_sweeps, t0, alpha,
                            _ptr_array(phase_out), _ptr_array(level_out),
                            None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_sa_run")


def hg_hio_run(plan: int, target_amp, beta: float, signal_mask=None, init_phase=None, seed: int = 0,
               n_iter: int = 1, phase_out=None, level_out=None, nmse_out=None, stream=None):
    """Hybrid input-output for every item of a single-plane plan (see hologen.h)."""
    _check(load().hg_hio_run(plan, _ptr_array(target_amp), _ptr_array(signal_mask), beta, _ptr_array(init_phase),
                             seed, n_iter, _ptr_array(phase_out), _ptr_array(level_out),
                             None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_hio_run")


def hg_ospr_run(plan: int, target_amp, n_subframes: int, n_iter: int = 0, seed: int = 0, bits_out=None,
                nmse_out=None, stream=None):
    """One-Step Phase-Retrieval for every item of the plan (see hologen.h)."""
    _check(load().hg_ospr_run(plan, _ptr_array(target_amp), n_subframes, n_iter, seed, _ptr_array(bits_out),
                              None if nmse_out is None else _data_ptr(nmse_out), _stream(stream)), "hg_ospr_run")


def hg_gd_step(plan: int, phase, target_int, adam_m, adam_v, step: int, lr: float = 0.05, beta1: float = 0.9,
               beta2: float = 0.999, eps: float = 1e-8, loss_out=None, grad_out=None, stream=None):
    """One Adam step of gradient-descent hologram optimisation for every item (see hologen.h)."""
    _check(load().hg_gd_step(plan, _ptr_array(phase), _ptr_array(target_int), _ptr_array(adam_m), _ptr_array(adam_v),
                             step, lr, beta1, beta2, eps, None if loss_out is None else _data_ptr(loss_out),
                             _ptr_array(grad_out), _stream(stream)), "hg_gd_step")


def hg_gd_forward(plan: int, phase, target_int, loss_out=None, stream=None):
    _check(load().hg_gd_forward(plan, _ptr_array(phase), _ptr_array(target_int),
                                None if loss_out is None else _data_ptr(loss_out), _stream(stream)), "hg_gd_forward")


def hg_gd_backward(plan: int, phase, target_int, grad_out, grad_scale=None, stream=None):
    _check(load().hg_gd_backward(plan, _ptr_array(phase), _ptr_array(target_int),
                                 None if grad_scale is None else _data_ptr(grad_scale), _ptr_array(grad_out),
                                 _stream(stream)), "hg_gd_backward")


def hologram_loss(plan: "Plan", phase, target_int):
    """Differentiable multi-plane hologram loss L(phase) (mean over planes of the optimal-scale
    intensity NMSE) for a one-item plan; the backward pass is the library's hand-written adjoint.

    ``phase``: float32 [H][W] CUDA tensor (requires_grad as usual); ``target_int``: P float32 [H][W]
    CUDA tensors.  One backward per forward (the forward's per-plane fields are the checkpoint).
    """
    import torch

    class _HologramLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, ph):
            ph = ph.detach().contiguous()
            loss = torch.empty((plan.n_planes + 1,), dtype=torch.float32, device=ph.device)
            hg_gd_forward(plan.handle, [ph], list(target_int), loss)
            ctx.save_for_backward(ph)
            return loss[plan.n_planes].clone()

        @staticmethod
        def backward(ctx, grad_loss):
            (ph,) = ctx.saved_tensors
            grad = torch.empty_like(ph)
            gs = grad_loss.detach().reshape(1).to(torch.float32).contiguous()
            hg_gd_backward(plan.handle, [ph], list(target_int), [grad], gs)
            return grad

    return _HologramLoss.apply(phase)


def hg_gs_run_noalloc(height: int, width: int, quant_levels: int, target_amp, init_phase=None, seed: int = 0,
                      n_iter: int = 1, phase_out=None, level_out=None, nmse_out=None, stream=None):
    """GS for one Fourier hologram with no device allocation (static scratch; see hologen.h).

    For callers that cannot allocate device memory and so cannot hold a plan.  Tensors are single
    device tensors (not lists); calls that overlap on the GPU share the scratch and race.
    """

    def p(t):
        return None if t is None else _data_ptr(t)

    _check(load().hg_gs_run_noalloc(height, width, quant_levels, p(target_amp), p(init_phase), seed, n_iter,
                                    p(phase_out), p(level_out), p(nmse_out), _stream(stream)), "hg_gs_run_noalloc")


def hg_plan_set_timing(plan: int, enabled: bool):
    _check(load().hg_plan_set_timing(plan, int(bool(enabled))), "hg_plan_set_timing")


def hg_plan_reset_timing(plan: int):
    _check(load().hg_plan_reset_timing(plan), "hg_plan_reset_timing")


def hg_plan_kernel_time(plan: int, kind: int) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().hg_plan_kernel_time(plan, kind, ctypes.byref(ms), ctypes.byref(n)), "hg_plan_kernel_time")
    return ms.value, n.value


def hg_kernel_kind_name(kind: int) -> str | None:
    r = load().hg_kernel_kind_name(kind)
    return None if r is None else r.decode()


def hg_plan_launch_count(plan: int) -> int:
    return int(load().hg_plan_launch_count(plan))


def hg_plan_set_graph(plan: int, enabled: bool):
    _check(load().hg_plan_set_graph(plan, int(bool(enabled))), "hg_plan_set_graph")


def hg_plan_item_latency(plan: int, n_items: int) -> list[float]:
    out = (ctypes.c_double * n_items)()
    _check(load().hg_plan_item_latency(plan, out), "hg_plan_item_latency")
    return list(out)


def hg_plan_autotune(plan: int, stream=None):
    _check(load().hg_plan_autotune(plan, _stream(stream)), "hg_plan_autotune")


def hg_plan_strip_width(plan: int, item: int) -> int:
    out = ctypes.c_int32()
    _check(load().hg_plan_strip_width(plan, item, ctypes.byref(out)), "hg_plan_strip_width")
    return out.value


def hg_plan_radix_plan(plan: int, item: int) -> tuple[int, int]:
    r = ctypes.c_int32(0)
    c = ctypes.c_int32(0)
    _check(load().hg_plan_radix_plan(plan, item, ctypes.byref(r), ctypes.byref(c)), "hg_plan_radix_plan")
    return r.value, c.value


def hg_plan_set_radix_plan(plan: int, item: int, row_plan: int, col_plan: int):
    _check(load().hg_plan_set_radix_plan(plan, item, row_plan, col_plan), "hg_plan_set_radix_plan")


def hg_plan_set_strip_width(plan: int, item: int, width: int):
    _check(load().hg_plan_set_strip_width(plan, item, width), "hg_plan_set_strip_width")


class Plan:
    """Owning wrapper around a plan handle (destroyed on close / exit / garbage collection)."""

    def __init__(self, heights, widths, propagation=HG_FOURIER, wavelength_m=0.0, pitch_m=0.0, z_m=None,
                 quant_levels=0, flags=0):
        self.heights = list(heights)
        self.widths = list(widths)
        self.n_planes = len(z_m) if z_m else 1
        self.quant_levels = quant_levels
        self.handle = hg_plan_create(self.heights, self.widths, propagation, wavelength_m, pitch_m, z_m,
                                     quant_levels, flags)

    def close(self):
        if self.handle is not None:
            hg_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - never raise from a finaliser
            pass

    def propagate(self, inputs, outputs, direction=1, plane=0, stream=None):
        hg_propagate(self.handle, plane, direction, inputs, outputs, stream)

    def gs(self, target_amp, n_iter, init_phase=None, seed=0, phase_out=None, level_out=None, nmse_out=None,
           stream=None):
        hg_gs_run(self.handle, target_amp, init_phase, seed, n_iter, phase_out, level_out, nmse_out, stream)

    def mraf(self, target_amp, mix, n_iter, signal_mask=None, init_phase=None, seed=0, phase_out=None, level_out=None,
             nmse_out=None, stream=None):
        hg_mraf_run(self.handle, target_amp, mix, signal_mask, init_phase, seed, n_iter, phase_out, level_out,
                    nmse_out, stream)

    def dbs(self, target_amp, n_sweeps, init_phase=None, seed=0, phase_out=None, level_out=None, nmse_out=None,
            stream=None):
        hg_dbs_run(self.handle, target_amp, init_phase, seed, n_sweeps, phase_out, level_out, nmse_out, stream)

    def sa(self, target_amp, n_sweeps, t0, alpha, init_phase=None, seed=0, phase_out=None, level_out=None,
           nmse_out=None, stream=None):
        hg_sa_run(self.handle, target_amp, t0, alpha, init_phase, seed, n_sweeps, phase_out, level_out, nmse_out,
                  stream)

    def hio(self, target_amp, beta, n_iter, signal_mask=None, init_phase=None, seed=0, phase_out=None, level_out=None,
            nmse_out=None, stream=None):
        hg_hio_run(self.handle, target_amp, beta, signal_mask, init_phase, seed, n_iter, phase_out, level_out,
                   nmse_out, stream)

    def ospr(self, target_amp, n_subframes, n_iter=0, seed=0, bits_out=None, nmse_out=None, stream=None):
        hg_ospr_run(self.handle, target_amp, n_subframes, n_iter, seed, bits_out, nmse_out, stream)

    def gd_step(self, phase, target_int, adam_m, adam_v, step, lr=0.05, beta1=0.9, beta2=0.999, eps=1e-8,
                loss_out=None, grad_out=None, stream=None):
        hg_gd_step(self.handle, phase, target_int, adam_m, adam_v, step, lr, beta1, beta2, eps, loss_out, grad_out,
                   stream)

    def sync(self):
        hg_plan_sync(self.handle)

    def set_timing(self, enabled=True):
        hg_plan_set_timing(self.handle, enabled)

    def reset_timing(self):
        hg_plan_reset_timing(self.handle)

    def kernel_times(self) -> dict[str, tuple[float, int]]:
        """{kind name: (total ms, launches)} for every kind launched while timing was on."""
        out = {}
        k = 0
        while (name := hg_kernel_kind_name(k)) is not None:
            ms, n = hg_plan_kernel_time(self.handle, k)
            if n:
                out[name] = (ms, n)
            k += 1
        return out

    def launch_count(self) -> int:
        return hg_plan_launch_count(self.handle)

    def set_graph(self, enabled=True):
        hg_plan_set_graph(self.handle, enabled)

    def item_latency_ms(self) -> list[float]:
        return hg_plan_item_latency(self.handle, len(self.heights))

    def set_slm_levels(self, levels=None):
        hg_plan_set_slm_levels(self.handle, levels)

    def set_illumination(self, illum_amp=None):
        self._illum = illum_amp  # the plan reads these buffers on every run: keep them alive
        hg_plan_set_illumination(self.handle, illum_amp)

    def autotune(self, stream=None):
        hg_plan_autotune(self.handle, stream)

    def strip_width(self, item: int) -> int:
        return hg_plan_strip_width(self.handle, item)

    def radix_plan(self, item: int) -> tuple[int, int]:
        """(row plan, column plan) of the item's size class: 0 default, 1 alternative."""
        return hg_plan_radix_plan(self.handle, item)

    def set_radix_plan(self, item: int, row_plan: int, col_plan: int):
        hg_plan_set_radix_plan(self.handle, item, row_plan, col_plan)

    def set_strip_width(self, item: int, width: int):
        hg_plan_set_strip_width(self.handle, item, width)
