"""PyTorch-facing API: device memory, streams and autograd around libhrc.so.

PyTorch is plumbing here: it allocates device tensors and provides the
current CUDA stream.  Every step of the method runs in the library's CUDA
kernels through the C ABI (``_lib``).
"""
from __future__ import annotations

import torch

from . import _lib

_PREC = {
    "fp32": _lib.HRC_FP32,
    "fp16": _lib.HRC_FP16_LOGT,
    "bf16": _lib.HRC_BF16_LOGT,
    "fp64": _lib.HRC_FP64_TEST,
}


def _dev_tensor(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        t = t.contiguous()
    if t.data_ptr() % 16:
        t = t.clone()
    return t


class HRC:
    """One HRC context: a W x H grid with C channels on the current device.

    ``precision`` is one of 'fp32', 'fp16', 'bf16' (reduced-precision
    interval storage with log-domain transmittance) or 'fp64' (test only).
    """

    def __init__(self, W: int, H: int, channels: int = 1, cascades: int = 0, precision: str = "fp32"):
        self.W, self.H, self.C, self.cascades = W, H, channels, cascades
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.ctx = _lib.hrc_create(W, H, channels, cascades)
        self.precision = "fp32"
        self._borrowed = (None, None, 0, 0)
        self._host_levels = False
        self._bounced = None
        self.per_channel = False
        self.set_precision(precision)

    # -- configuration -----------------------------------------------------
    def set_precision(self, precision: str) -> None:
        _lib.hrc_set_precision(self.ctx, _PREC[precision])
        self.precision = precision
        self._borrowed = (None, None, 0, 0)
        self._host_levels = False

    @property
    def dtype(self):
        return torch.float64 if self.precision == "fp64" else torch.float32

    def _stream(self):
        _lib.hrc_set_stream(self.ctx, torch.cuda.current_stream(self.device).cuda_stream)

    # -- compute -----------------------------------------------------------
    def forward(self, emission, sigma_t, out=None):
        C, H, W = self.C, self.H, self.W
        emission = _dev_tensor(emission, self.dtype, (C, H, W), "emission")
        sigma_t = _dev_tensor(sigma_t, self.dtype, self.sigma_shape, "sigma_t")
        if out is None:
            out = torch.empty((C, H, W), dtype=self.dtype, device=emission.device)
        self._stream()
        if self.precision == "fp64":
            _lib.hrc_fluence_f64(self.ctx, emission, sigma_t, out)
        else:
            _lib.hrc_fluence(self.ctx, emission, sigma_t, out)
        self._borrowed = (emission, sigma_t, emission._version, sigma_t._version)
        self._host_levels = False
        self._bounced = None
        return out

    __call__ = forward

    def _levels_current(self, emission, sigma_t) -> bool:
        """True when the context's levels are those of these inputs (same
        storage, not modified in place since the forward)."""
        b = self._borrowed
        if b[0] is None:
            return False
        if emission is None:
            emission, sigma_t = b[0], b[1]
        return (b[0].data_ptr() == emission.data_ptr() and b[1].data_ptr() == sigma_t.data_ptr() and
                b[0]._version == b[2] and b[1]._version == b[3])

    def forward_host(self, emission, sigma_t, out=None):
        """Host (CPU) float32 tensors in and out, copies included."""
        C, H, W = self.C, self.H, self.W
        emission = emission.contiguous()
        sigma_t = sigma_t.contiguous()
        assert emission.dtype == torch.float32 and tuple(emission.shape) == (C, H, W)
        assert sigma_t.dtype == torch.float32 and tuple(sigma_t.shape) == self.sigma_shape
        if out is None:
            out = torch.empty((C, H, W), dtype=torch.float32, pin_memory=emission.is_pinned())
        self._stream()
        _lib.hrc_fluence_host(self.ctx, emission, sigma_t, out)
        self._borrowed = (None, None, 0, 0)
        self._host_levels = True     # levels of the context's own device copies
        return out

    def backward(self, grad_F, emission=None, sigma_t=None):
        """dLoss/d(emission, sigma_t) at the inputs of the last forward (or at
        the given inputs).  The backward reads the levels that forward left in
        the context, so the forward runs again first when the inputs differ
        or were modified in place since."""
        C, H, W = self.C, self.H, self.W
        if emission is None and not self._host_levels and self._borrowed[0] is not None:
            emission, sigma_t = self._borrowed[0], self._borrowed[1]
        if emission is not None and not self._levels_current(emission, sigma_t):
            self.forward(emission, sigma_t)
        # (no forward at all: the library answers HRC_ESTATE)
        grad_F = _dev_tensor(grad_F, self.dtype, (C, H, W), "grad_F")
        ge = torch.empty((C, H, W), dtype=self.dtype, device=grad_F.device)
        gs = torch.empty(self.sigma_shape, dtype=self.dtype, device=grad_F.device)
        self._stream()
        if self.precision == "fp64":
            _lib.hrc_fluence_backward_f64(self.ctx, grad_F, ge, gs)
        else:
            _lib.hrc_fluence_backward(self.ctx, grad_F, ge, gs)
        return ge, gs

    def set_channel_extinction(self, per_channel: bool = True) -> None:
        """sigma_t per channel ([C][H][W]) instead of one shared [H][W] plane
        (hrc_set_channel_extinction); dL/dsigma_t then has the same shape."""
        _lib.hrc_set_channel_extinction(self.ctx, per_channel)
        self.per_channel = bool(per_channel)
        self._borrowed = (None, None, 0, 0)
        self._bounced = None

    @property
    def sigma_shape(self):
        return (self.C, self.H, self.W) if self.per_channel else (self.H, self.W)

    def set_environment(self, env=None) -> None:
        """Environment map (footnote 1 of Sec. 4.2): a CUDA float32 tensor
        [C][M] (or [M], the same for every channel) of radiance along the look
        angles 2 pi (m + 1/2) / M from +x towards +y; None removes it."""
        if env is None:
            _lib.hrc_set_environment(self.ctx, None, 0)
            self._env = None
        else:
            if env.dim() == 1:
                env = env.expand(self.C, env.shape[0])
            env = _dev_tensor(env, torch.float32, (self.C, env.shape[-1]), "env")
            self._stream()
            _lib.hrc_set_environment(self.ctx, env, env.shape[-1])
            self._env = env
        self._borrowed = (None, None, 0, 0)
        self._bounced = None

    def set_top_radiance(self, top=None) -> None:
        """Top-level radiance R_N supplied by the caller (footnote 1 of Sec.
        4.2): a CUDA float32 tensor [4][K][C], cone j of frame q at
        [q][j][c] (see hrc_set_top_radiance); None removes it."""
        if top is None:
            _lib.hrc_set_environment(self.ctx, None, 0)
            self._env = None
        else:
            top = _dev_tensor(top, torch.float32, (4, top.shape[1], self.C), "top")
            self._stream()
            _lib.hrc_set_top_radiance(self.ctx, top, top.shape[1])
            self._env = top
        self._borrowed = (None, None, 0, 0)
        self._bounced = None

    # -- multiple bounces (hrc_fluence_bounces) ----------------------------
    def reserve_bounces(self, max_bounces: int) -> None:
        """Context buffers for up to `max_bounces` bounces (hrc_reserve_bounces)."""
        _lib.hrc_reserve_bounces(self.ctx, max_bounces)

    def forward_bounces(self, emission, sigma_t, albedo, bounces: int, out=None):
        """F after `bounces` extra bounces: each feeds albedo * sigma * F / (2 pi)
        back into the emission (see hrc_fluence_bounces)."""
        C, H, W = self.C, self.H, self.W
        emission = _dev_tensor(emission, self.dtype, (C, H, W), "emission")
        sigma_t = _dev_tensor(sigma_t, self.dtype, self.sigma_shape, "sigma_t")
        albedo = _dev_tensor(albedo, self.dtype, (C, H, W), "albedo")
        if out is None:
            out = torch.empty((C, H, W), dtype=self.dtype, device=emission.device)
        self._stream()
        if self.precision == "fp64":
            _lib.hrc_fluence_bounces_f64(self.ctx, emission, sigma_t, albedo, bounces, out)
        else:
            _lib.hrc_fluence_bounces(self.ctx, emission, sigma_t, albedo, bounces, out)
        self._borrowed = (None, None, 0, 0)
        self._host_levels = False
        self._bounced = (emission, sigma_t, albedo, bounces, emission._version, sigma_t._version, albedo._version)
        return out

    def backward_bounces(self, grad_F, emission=None, sigma_t=None, albedo=None, bounces=None):
        """dLoss/d(emission, sigma_t, albedo) of the last forward_bounces (or of
        the given inputs: the bounce forward runs again first when they differ
        from the last one's or were modified in place since)."""
        C, H, W = self.C, self.H, self.W
        b = self._bounced
        if emission is not None:
            current = (b is not None and b[3] == bounces and
                       all(x.data_ptr() == y.data_ptr() and x._version == v
                           for x, y, v in zip(b[:3], (emission, sigma_t, albedo), b[4:])))
            if not current:
                self.forward_bounces(emission, sigma_t, albedo, bounces)
        grad_F = _dev_tensor(grad_F, self.dtype, (C, H, W), "grad_F")
        ge = torch.empty((C, H, W), dtype=self.dtype, device=grad_F.device)
        gs = torch.empty(self.sigma_shape, dtype=self.dtype, device=grad_F.device)
        ga = torch.empty((C, H, W), dtype=self.dtype, device=grad_F.device)
        self._stream()
        if self.precision == "fp64":
            _lib.hrc_fluence_bounces_backward_f64(self.ctx, grad_F, ge, gs, ga)
        else:
            _lib.hrc_fluence_bounces_backward(self.ctx, grad_F, ge, gs, ga)
        return ge, gs, ga

    def bounce_source(self, emission, sigma_t, albedo, fluence, out=None):
        """emission + albedo * sigma_t * fluence / (2 pi) (hrc_bounce_source), for
        one bounce per frame."""
        C, H, W = self.C, self.H, self.W
        emission = _dev_tensor(emission, torch.float32, (C, H, W), "emission")
        sigma_t = _dev_tensor(sigma_t, torch.float32, self.sigma_shape, "sigma_t")
        albedo = _dev_tensor(albedo, torch.float32, (C, H, W), "albedo")
        fluence = _dev_tensor(fluence, torch.float32, (C, H, W), "fluence")
        if out is None:
            out = torch.empty_like(emission)
        self._stream()
        _lib.hrc_bounce_source(self.ctx, emission, sigma_t, albedo, fluence, out)
        return out

    def level(self, q: int, which: str, n: int) -> torch.Tensor:
        """T_n (which='T': [U_n][2^n+1][V][C+1]) or R_n (which='R':
        [U_n][2^n][V][C]) of quadrant frame q from the last forward."""
        w = 0 if which == "T" else 1
        cnt = _lib.hrc_copy_level(self.ctx, q, w, n, None)
        U, V = (self.W, self.H) if q < 2 else (self.H, self.W)
        Un = -(-U // (1 << n))
        dst = torch.empty(cnt, dtype=torch.float32, device=self.device)
        self._stream()
        _lib.hrc_copy_level(self.ctx, q, w, n, dst)
        if w == 0:
            return dst.view(Un, (1 << n) + 1, V, self.C + 1)
        return dst.view(Un, 1 << n, V, self.C)

    def autotune(self) -> float:
        """Pick the fastest launch configuration for this grid (see
        hrc_autotune); returns its forward ms per frame."""
        self._stream()
        ms = _lib.hrc_autotune(self.ctx)
        self._borrowed = (None, None, 0, 0)
        self._host_levels = False
        return ms

    def set_backward_recompute(self, on: bool) -> None:
        """Recompute every level at the start of each backward (True) instead
        of reading the ones the forward left in the context (False, default);
        see hrc_set_backward_recompute."""
        _lib.hrc_set_backward_recompute(self.ctx, on)

    def set_cross_blur(self, enable: bool = True, threshold: float = 0.5) -> None:
        """Cross blur of Eq. 21 after the fluence sum, leaving out neighbours
        whose opacity 1 - exp(-sigma) differs by more than `threshold`
        (see hrc_set_cross_blur); the backward differentiates it."""
        _lib.hrc_set_cross_blur(self.ctx, enable, threshold)

    @property
    def cross_blur(self):
        """(enabled, threshold)."""
        return _lib.hrc_get_cross_blur(self.ctx)

    @property
    def launch_config(self) -> dict:
        """{schedule, groups, threads, vmajor, mdown} (see hrc_launch_config)."""
        return _lib.hrc_get_launch_config(self.ctx)

    def set_launch_config(self, schedule=0, groups=1, threads=128, vmajor=0, mdown=0) -> None:
        _lib.hrc_set_launch_config(self.ctx, schedule, groups, threads, vmajor, mdown)
        self._borrowed = (None, None, 0, 0)
        self._host_levels = False

    def sync(self) -> None:
        """Wait for the context's stream; raise HRCError(HRC_ETIMEOUT) if a
        bounded bulk-copy wait gave up."""
        _lib.hrc_sync(self.ctx)

    def launch_count(self) -> int:
        return _lib.hrc_last_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            _lib.hrc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedHRC:
    """Many scenes of uneven size, each pass in one persistent launch.

    Scenes are packed back to back: emission / fluence as the concatenation
    of the flattened [C][H_i][W_i] blocks, extinction as that of the [H_i][W_i]
    blocks (``offsets()`` gives the element offsets).
    """

    def __init__(self, sizes, channels: int = 1, cascades: int = 0, precision: str = "fp32"):
        self.sizes = [(int(w), int(h)) for (w, h) in sizes]
        self.C = channels
        Ws = [w for w, _ in self.sizes]
        Hs = [h for _, h in self.sizes]
        self.ctx = _lib.hrc_create_batched_prec(Ws, Hs, channels, cascades, _PREC[precision])
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.eoff, self.soff = _lib.hrc_scene_offsets(self.ctx, len(self.sizes))
        self._borrowed = None

    def offsets(self):
        return self.eoff, self.soff

    def pack(self, emissions, sigmas):
        """Lists of per-scene tensors -> packed device tensors."""
        e = torch.cat([t.reshape(-1) for t in emissions]).to(self.device, torch.float32).contiguous()
        s = torch.cat([t.reshape(-1) for t in sigmas]).to(self.device, torch.float32).contiguous()
        return e, s

    def unpack(self, packed, which="e"):
        off = self.eoff if which == "e" else self.soff
        out = []
        for i, (w, h) in enumerate(self.sizes):
            t = packed[off[i]:off[i + 1]]
            out.append(t.view(self.C, h, w) if which == "e" else t.view(h, w))
        return out

    def _stream(self):
        _lib.hrc_set_stream(self.ctx, torch.cuda.current_stream(self.device).cuda_stream)

    def forward(self, e_packed, s_packed, out=None):
        assert e_packed.numel() == self.eoff[-1] and s_packed.numel() == self.soff[-1]
        if out is None:
            out = torch.empty_like(e_packed)
        self._stream()
        _lib.hrc_fluence_batched(self.ctx, e_packed, s_packed, out)
        self._borrowed = (e_packed, s_packed)
        return out

    def backward(self, gF_packed, ge=None, gs=None):
        if ge is None:
            ge = torch.empty(self.eoff[-1], dtype=torch.float32, device=self.device)
        if gs is None:
            gs = torch.empty(self.soff[-1], dtype=torch.float32, device=self.device)
        self._stream()
        _lib.hrc_fluence_backward_batched(self.ctx, gF_packed.contiguous(), ge, gs)
        return ge, gs

    def sync(self):
        """Wait and raise HRCError(HRC_ETIMEOUT) if a dependency wait gave up."""
        _lib.hrc_batched_sync(self.ctx)

    def set_backward_recompute(self, on: bool) -> None:
        _lib.hrc_set_backward_recompute(self.ctx, on)

    def tune(self, blocks_per_sm: int = 0, order: int = 0, schedule: int = 0):
        """schedule 0: persistent launch (blocks per SM, ticket order apply);
        schedule 1: per-scene launch chains on parallel graph branches;
        schedule 2: level-major multi-scene launches."""
        _lib.hrc_batched_tune(self.ctx, blocks_per_sm, order)
        _lib.hrc_batched_schedule(self.ctx, schedule)

    def autotune(self, e_packed, s_packed, reps: int = 3):
        """Time each (schedule, blocks per SM, ticket order) candidate on these
        inputs and keep the fastest; returns {candidate: ms}."""
        res = {}
        out = torch.empty_like(e_packed)
        for cand in [(0, bpsm, order) for bpsm in (0, 1, 2) for order in (0, 1)] + [(1, 0, 0), (2, 0, 0)]:
            sched, bpsm, order = cand
            self.tune(bpsm, order, sched)
            self.forward(e_packed, s_packed, out)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                self.forward(e_packed, s_packed, out)
            b.record()
            b.synchronize()
            res[cand] = a.elapsed_time(b) / reps
        sched, bpsm, order = min(res, key=res.get)
        self.tune(bpsm, order, sched)
        return res

    def close(self):
        if getattr(self, "ctx", None) is not None:
            _lib.hrc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _FluenceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hrc: HRC, emission, sigma_t):
        out = hrc.forward(emission.detach(), sigma_t.detach())
        ctx.hrc = hrc
        ctx.save_for_backward(emission, sigma_t)
        return out

    @staticmethod
    def backward(ctx, grad_F):
        emission, sigma_t = ctx.saved_tensors
        ge, gs = ctx.hrc.backward(grad_F.contiguous(), emission.detach(), sigma_t.detach())
        return None, ge, gs


class _BouncesFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hrc: HRC, emission, sigma_t, albedo, bounces):
        out = hrc.forward_bounces(emission.detach(), sigma_t.detach(), albedo.detach(), bounces)
        ctx.hrc = hrc
        ctx.bounces = bounces
        ctx.save_for_backward(emission, sigma_t, albedo)
        return out

    @staticmethod
    def backward(ctx, grad_F):
        emission, sigma_t, albedo = ctx.saved_tensors
        ge, gs, ga = ctx.hrc.backward_bounces(grad_F.contiguous(), emission.detach(), sigma_t.detach(),
                                              albedo.detach(), ctx.bounces)
        return None, ge, gs, ga, None


def fluence_bounces(hrc: HRC, emission, sigma_t, albedo, bounces: int):
    """Differentiable multi-bounce fluence (forward -> hrc_fluence_bounces,
    backward -> hrc_fluence_bounces_backward); reserve the bounces first."""
    return _BouncesFn.apply(hrc, emission, sigma_t, albedo, bounces)


def fluence(hrc: HRC, emission, sigma_t):
    """Differentiable fluence F(emission, sigma_t) (torch.autograd.Function):
    forward -> hrc_fluence, backward -> hrc_fluence_backward."""
    return _FluenceFn.apply(hrc, emission, sigma_t)
