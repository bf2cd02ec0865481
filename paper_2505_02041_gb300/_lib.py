"""ctypes binding of the C ABI in include/hrc.h (argument marshalling only).

The functions keep the C names (``hrc_create``, ``hrc_fluence`` ...).  Every
step of the computation runs in the CUDA kernels of ``libhrc.so``; there is
no Python or CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhrc.so")

HRC_OK, HRC_EINVAL, HRC_ENOMEM, HRC_ECUDA, HRC_ESTATE, HRC_ETIMEOUT, HRC_EBOUNDS = range(7)
HRC_FP32, HRC_FP16_LOGT, HRC_BF16_LOGT, HRC_FP64_TEST = range(4)
STATUS_NAMES = ["HRC_OK", "HRC_EINVAL", "HRC_ENOMEM", "HRC_ECUDA", "HRC_ESTATE", "HRC_ETIMEOUT", "HRC_EBOUNDS"]

_vp = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong

# (name, restype, argtypes) for every function declared in include/hrc.h
SIGNATURES = [
    ("hrc_create", _i, [_i, _i, _i, _i, ctypes.POINTER(_vp)]),
    ("hrc_destroy", _i, [_vp]),
    ("hrc_set_stream", _i, [_vp, _vp]),
    ("hrc_set_precision", _i, [_vp, _i]),
    ("hrc_set_schedule", _i, [_vp, _i]),
    ("hrc_autotune", _i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    ("hrc_set_backward_recompute", _i, [_vp, _i]),
    ("hrc_sync", _i, [_vp]),
    ("hrc_set_cross_blur", _i, [_vp, _i, ctypes.c_float]),
    ("hrc_get_cross_blur", _i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_float)]),
    ("hrc_set_environment", _i, [_vp, _vp, _i]),
    ("hrc_set_top_radiance", _i, [_vp, _vp, _i]),
    ("hrc_set_channel_extinction", _i, [_vp, _i]),
    ("hrc_reserve_bounces", _i, [_vp, _i]),
    ("hrc_fluence_bounces", _i, [_vp, _vp, _vp, _vp, _i, _vp]),
    ("hrc_fluence_bounces_backward", _i, [_vp, _vp, _vp, _vp, _vp]),
    ("hrc_fluence_bounces_f64", _i, [_vp, _vp, _vp, _vp, _i, _vp]),
    ("hrc_fluence_bounces_backward_f64", _i, [_vp, _vp, _vp, _vp, _vp]),
    ("hrc_bounce_source", _i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("hrc_debug_bulk_wait", _i, [_vp, _i, ctypes.c_longlong]),
    ("hrc_get_launch_config", _i, [_vp, _vp]),
    ("hrc_set_launch_config", _i, [_vp, _vp]),
    ("hrc_fluence", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_fluence_host", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_fluence_backward", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_fluence_f64", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_fluence_backward_f64", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_create_batched", _i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _i, ctypes.POINTER(_vp)]),
    ("hrc_create_batched_prec", _i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _i, _i, ctypes.POINTER(_vp)]),
    ("hrc_scene_offsets", _i, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    ("hrc_fluence_batched", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_fluence_backward_batched", _i, [_vp, _vp, _vp, _vp]),
    ("hrc_batched_sync", _i, [_vp]),
    ("hrc_batched_tune", _i, [_vp, _i, _i]),
    ("hrc_batched_schedule", _i, [_vp, _i]),
    ("hrc_batched_debug", _i, [_vp, _i, _ll]),
    ("hrc_fluence_noalloc", _i, [_i, _i, _i, _vp, _vp, _vp, _vp]),
    ("hrc_noalloc_sync", _i, [_vp]),
    ("hrc_noalloc_debug_wait", _i, [_i, _ll]),
    ("hrc_set_graphs", _i, [_vp, _i]),
    ("hrc_graph_captures", _ll, [_vp]),
    ("hrc_copy_level", _i, [_vp, _i, _i, _i, _vp, ctypes.POINTER(_ll)]),
    ("hrc_last_launch_count", _i, [_vp]),
    ("hrc_set_timing", _i, [_vp, _i]),
    ("hrc_get_timing", _i, [_vp, _vp, _i]),
    ("hrc_last_error", ctypes.c_char_p, [_vp]),
    ("hrc_version", ctypes.c_char_p, []),
]

_lib = None


class HRCError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libhrc.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libhrc.so not built at {path}: run __graft_entry__.build() "
                               "(the CUDA path has no fallback)")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, ctx=None) -> None:
    if status != HRC_OK:
        msg = load().hrc_last_error(ctx).decode(errors="replace")
        raise HRCError(status, msg)


def ptr(t) -> int:
    """Device or host address of a tensor / ndarray (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


# Thin wrappers with the C names -------------------------------------------------

def hrc_create(W: int, H: int, channels: int, cascades: int = 0):
    out = _vp()
    check(load().hrc_create(W, H, channels, cascades, ctypes.byref(out)))
    return out


def hrc_destroy(ctx):
    check(load().hrc_destroy(ctx), ctx)


def hrc_set_stream(ctx, stream_handle: int):
    check(load().hrc_set_stream(ctx, stream_handle), ctx)


def hrc_set_precision(ctx, prec: int):
    check(load().hrc_set_precision(ctx, prec), ctx)


def hrc_set_schedule(ctx, schedule: int):
    check(load().hrc_set_schedule(ctx, schedule), ctx)


def hrc_set_backward_recompute(ctx, on: bool):
    check(load().hrc_set_backward_recompute(ctx, int(bool(on))), ctx)


def hrc_set_cross_blur(ctx, enable: bool, threshold: float = 0.5):
    check(load().hrc_set_cross_blur(ctx, int(bool(enable)), float(threshold)), ctx)


def hrc_get_cross_blur(ctx):
    """(enabled, threshold) of the context's cross blur."""
    en = _i()
    th = ctypes.c_float()
    check(load().hrc_get_cross_blur(ctx, ctypes.byref(en), ctypes.byref(th)), ctx)
    return bool(en.value), th.value


def hrc_set_environment(ctx, env, M: int):
    check(load().hrc_set_environment(ctx, ptr(env), M), ctx)


def hrc_set_top_radiance(ctx, top, K: int):
    check(load().hrc_set_top_radiance(ctx, ptr(top) if top is not None else None, K), ctx)


def hrc_set_channel_extinction(ctx, per_channel: bool):
    check(load().hrc_set_channel_extinction(ctx, int(bool(per_channel))), ctx)


def hrc_reserve_bounces(ctx, max_bounces: int):
    check(load().hrc_reserve_bounces(ctx, max_bounces), ctx)


def hrc_fluence_bounces(ctx, emission, sigma_t, albedo, bounces: int, out):
    check(load().hrc_fluence_bounces(ctx, ptr(emission), ptr(sigma_t), ptr(albedo), bounces, ptr(out)), ctx)


def hrc_fluence_bounces_backward(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo):
    check(load().hrc_fluence_bounces_backward(ctx, ptr(grad_F), ptr(grad_emission), ptr(grad_sigma_t),
                                              ptr(grad_albedo)), ctx)


def hrc_fluence_bounces_f64(ctx, emission, sigma_t, albedo, bounces: int, out):
    check(load().hrc_fluence_bounces_f64(ctx, ptr(emission), ptr(sigma_t), ptr(albedo), bounces, ptr(out)), ctx)


def hrc_fluence_bounces_backward_f64(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo):
    check(load().hrc_fluence_bounces_backward_f64(ctx, ptr(grad_F), ptr(grad_emission), ptr(grad_sigma_t),
                                                  ptr(grad_albedo)), ctx)


def hrc_bounce_source(ctx, emission, sigma_t, albedo, fluence, out):
    check(load().hrc_bounce_source(ctx, ptr(emission), ptr(sigma_t), ptr(albedo), ptr(fluence), ptr(out)), ctx)


class hrc_launch_config(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("groups", ctypes.c_int), ("threads", ctypes.c_int),
                ("vmajor", ctypes.c_int), ("mdown", ctypes.c_int)]


def hrc_get_launch_config(ctx) -> dict:
    c = hrc_launch_config()
    check(load().hrc_get_launch_config(ctx, ctypes.byref(c)), ctx)
    return {f: getattr(c, f) for f, _ in hrc_launch_config._fields_}


def hrc_sync(ctx):
    check(load().hrc_sync(ctx), ctx)


def hrc_debug_bulk_wait(ctx, extra_bytes: int, limit_ns: int):
    check(load().hrc_debug_bulk_wait(ctx, extra_bytes, limit_ns), ctx)


def hrc_set_launch_config(ctx, schedule: int, groups: int, threads: int, vmajor: int, mdown: int = 0):
    c = hrc_launch_config(schedule, groups, threads, vmajor, mdown)
    check(load().hrc_set_launch_config(ctx, ctypes.byref(c)), ctx)


def hrc_autotune(ctx) -> float:
    ms = ctypes.c_float()
    check(load().hrc_autotune(ctx, ctypes.byref(ms)), ctx)
    return ms.value


def hrc_fluence(ctx, emission, sigma_t, out):
    check(load().hrc_fluence(ctx, ptr(emission), ptr(sigma_t), ptr(out)), ctx)


def hrc_fluence_host(ctx, emission, sigma_t, out):
    check(load().hrc_fluence_host(ctx, ptr(emission), ptr(sigma_t), ptr(out)), ctx)


def hrc_fluence_backward(ctx, grad_F, grad_emission, grad_sigma_t):
    check(load().hrc_fluence_backward(ctx, ptr(grad_F), ptr(grad_emission), ptr(grad_sigma_t)), ctx)


def hrc_fluence_f64(ctx, emission, sigma_t, out):
    check(load().hrc_fluence_f64(ctx, ptr(emission), ptr(sigma_t), ptr(out)), ctx)


def hrc_fluence_backward_f64(ctx, grad_F, grad_emission, grad_sigma_t):
    check(load().hrc_fluence_backward_f64(ctx, ptr(grad_F), ptr(grad_emission), ptr(grad_sigma_t)), ctx)


def hrc_create_batched(Ws, Hs, channels: int, cascades: int = 0):
    n = len(Ws)
    out = _vp()
    Wa = (_i * n)(*Ws)
    Ha = (_i * n)(*Hs)
    check(load().hrc_create_batched(n, Wa, Ha, channels, cascades, ctypes.byref(out)))
    return out


def hrc_create_batched_prec(Ws, Hs, channels: int, cascades: int, prec: int):
    n = len(Ws)
    out = _vp()
    Wa = (_i * n)(*Ws)
    Ha = (_i * n)(*Hs)
    check(load().hrc_create_batched_prec(n, Wa, Ha, channels, cascades, prec, ctypes.byref(out)))
    return out


def hrc_scene_offsets(ctx, n: int):
    eo = (_ll * (n + 1))()
    so = (_ll * (n + 1))()
    check(load().hrc_scene_offsets(ctx, eo, so), ctx)
    return list(eo), list(so)


def hrc_fluence_batched(ctx, emission, sigma_t, out):
    check(load().hrc_fluence_batched(ctx, ptr(emission), ptr(sigma_t), ptr(out)), ctx)


def hrc_fluence_backward_batched(ctx, grad_F, grad_emission, grad_sigma_t):
    check(load().hrc_fluence_backward_batched(ctx, ptr(grad_F), ptr(grad_emission), ptr(grad_sigma_t)), ctx)


def hrc_batched_sync(ctx):
    check(load().hrc_batched_sync(ctx), ctx)


def hrc_batched_schedule(ctx, schedule: int):
    check(load().hrc_batched_schedule(ctx, schedule), ctx)


def hrc_batched_tune(ctx, blocks_per_sm: int, order: int):
    check(load().hrc_batched_tune(ctx, blocks_per_sm, order), ctx)


def hrc_batched_debug(ctx, withhold_counter: int, spin_limit: int):
    check(load().hrc_batched_debug(ctx, withhold_counter, spin_limit), ctx)


def hrc_fluence_noalloc(W: int, H: int, channels: int, emission, sigma_t, out, stream_handle=None):
    """Allocation-free forward (no context); see include/hrc.h."""
    check(load().hrc_fluence_noalloc(W, H, channels, ptr(emission), ptr(sigma_t), ptr(out), stream_handle))


def hrc_noalloc_sync(stream_handle=None):
    check(load().hrc_noalloc_sync(stream_handle))


def hrc_noalloc_debug_wait(extra_bytes: int, limit_ns: int):
    check(load().hrc_noalloc_debug_wait(extra_bytes, limit_ns))


def hrc_set_graphs(ctx, enable: bool):
    check(load().hrc_set_graphs(ctx, 1 if enable else 0), ctx)


def hrc_graph_captures(ctx) -> int:
    return int(load().hrc_graph_captures(ctx))


def hrc_copy_level(ctx, q: int, which: int, n: int, dst=None) -> int:
    cnt = _ll()
    check(load().hrc_copy_level(ctx, q, which, n, ptr(dst), ctypes.byref(cnt)), ctx)
    return cnt.value


def hrc_last_launch_count(ctx) -> int:
    return load().hrc_last_launch_count(ctx)


class hrc_kernel_time(ctypes.Structure):
    _fields_ = [("kind", _i), ("level", _i), ("ms", ctypes.c_float), ("bytes", ctypes.c_double), ("launches", _i)]


KERNEL_KINDS = ["trace012", "merge_up", "merge_down", "fluence_sum", "adj_sum", "adj_merge_down",
                "adj_merge_up", "adj_trace", "batched", "other", "cross_blur", "adj_cross_blur",
                "bounce_source", "adj_bounce"]


def hrc_set_timing(ctx, enable):
    """0 / False: off; 1 / True: direct launches bracketed by events;
    2: event-record nodes inside the replayed graphs."""
    check(load().hrc_set_timing(ctx, int(enable)), ctx)


def hrc_get_timing(ctx, cap: int = 512):
    """List of (kind name, level, ms, algorithmic bytes, launches) of the last
    call (launches > 1 only for the phase records of timing mode 3)."""
    arr = (hrc_kernel_time * cap)()
    n = load().hrc_get_timing(ctx, ctypes.cast(arr, _vp), cap)
    if n < 0:
        raise HRCError(HRC_ECUDA, "hrc_get_timing failed")
    return [(KERNEL_KINDS[arr[i].kind], arr[i].level, arr[i].ms, arr[i].bytes, arr[i].launches) for i in range(n)]


def hrc_last_error(ctx=None) -> str:
    return load().hrc_last_error(ctx).decode(errors="replace")


def hrc_version() -> str:
    return load().hrc_version().decode()
