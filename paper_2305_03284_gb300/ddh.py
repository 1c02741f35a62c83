"""Python binding of libddh: torch tensors in, C ABI calls out (no compute here).

PyTorch supplies device memory and the CUDA stream; every step of the method runs in the
library's kernels.  Frames are complex64 ``(N, N)`` CUDA tensors, phase and reflectance float32.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_float, c_int64, c_void_p

import torch

from ._lib import DdhError, DdhParams, check, lib  # noqa: F401


def default_params(n: int, aperture_diam: float, snr: float, /, **overrides) -> DdhParams:
    """``ddh_default_params`` plus keyword overrides (field names of :class:`DdhParams`)."""
    p = DdhParams()
    check(lib().ddh_default_params(byref(p), int(n), float(aperture_diam), float(snr)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def static_params(n: int, aperture_diam: float, snr: float, reset_every: int = 200, /, **overrides) -> DdhParams:
    """Parameters of static DH-MBIR (Sec. 3) on top of the frame step: lambda = alpha = 1,
    n_k = ``reset_every``, no tip/tilt removal.  Each ``Stream.step`` on the same frame is then
    one bootstrap period: r reset to ``|A_phi^H y~|^2`` with the current phase, followed by
    ``reset_every`` EM iterations (the paper resets every 200)."""
    p = DdhParams()
    check(lib().ddh_static_params(byref(p), int(n), float(aperture_diam), float(snr), int(reset_every)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def tracking_params(n: int, aperture_diam: float, snr: float, /, **overrides) -> DdhParams:
    """``ddh_tracking_params`` (2 x 2 phase tiles under the tile prior, sigma_r 0.03, alpha
    0.0125: the set under which the loop tracks frozen-flow turbulence on a bar-chart object at
    the paper's parameters) plus keyword overrides."""
    p = DdhParams()
    check(lib().ddh_tracking_params(byref(p), int(n), float(aperture_diam), float(snr)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _stream_handle(stream) -> c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_void_p(stream.cuda_stream)


def _check_frame(y: torch.Tensor, n: int) -> None:
    if y.dtype != torch.complex64 or tuple(y.shape) != (n, n) or not y.is_cuda or not y.is_contiguous():
        raise ValueError(f"frame must be a contiguous complex64 CUDA tensor of shape ({n}, {n})")


def _check_image(t: torch.Tensor, n: int) -> None:
    if t.dtype != torch.float32 or tuple(t.shape) != (n, n) or not t.is_contiguous():
        raise ValueError(f"image must be a contiguous float32 tensor of shape ({n}, {n})")


class Stream:
    """One sensor stream: the device state ``(n, r, phi)`` of Fig. 1, owned by libddh."""

    def __init__(self, params: DdhParams, stream: torch.cuda.Stream | None = None):
        self.params = params
        self.n = int(params.n)
        self.torch_stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = c_void_p()
        check(lib().ddh_init(byref(self._h), byref(params), _stream_handle(self.torch_stream)))

    # -- stepping ---------------------------------------------------------------------
    def step(self, y: torch.Tensor) -> None:
        _check_frame(y, self.n)
        check(lib().ddh_step(self._h, c_void_p(y.data_ptr())))

    def step_trace(self, y: torch.Tensor) -> dict:
        _check_frame(y, self.n)
        n = self.n
        m = n * n
        buf = torch.zeros(lib().ddh_trace_floats(n), dtype=torch.float32, device=y.device)
        check(lib().ddh_step_trace(self._h, c_void_p(y.data_ptr()), c_void_p(buf.data_ptr())))
        cx = buf[: 6 * m].view(torch.complex64)
        return {
            "b": cx[:m].view(n, n), "mu": cx[m: 2 * m].view(n, n), "z": cx[2 * m: 3 * m].view(n, n),
            "r_init": buf[6 * m: 7 * m].view(n, n), "s": buf[7 * m: 8 * m].view(n, n),
            "stats": buf[8 * m: 8 * m + 8],
        }

    def step_host(self, y_host: torch.Tensor, phi_out: torch.Tensor) -> None:
        """Host frame in, host phase out (copies inside the call; synchronous)."""
        if y_host.is_cuda or phi_out.is_cuda:
            raise ValueError("step_host takes host tensors")
        if y_host.dtype != torch.complex64 or tuple(y_host.shape) != (self.n, self.n) or not y_host.is_contiguous():
            raise ValueError("bad host frame")
        _check_image(phi_out, self.n)
        check(lib().ddh_step_host(self._h, c_void_p(y_host.data_ptr()), c_void_p(phi_out.data_ptr())))

    def step_host_async(self, y_host: torch.Tensor, phi_out: torch.Tensor) -> int:
        """Pipelined host step: enqueues copy in, step and copy out and returns a ticket at
        once; both (pinned) tensors stay untouched until ``host_wait(ticket)`` or ``sync()``."""
        if y_host.is_cuda or phi_out.is_cuda:
            raise ValueError("step_host_async takes host tensors")
        if y_host.dtype != torch.complex64 or tuple(y_host.shape) != (self.n, self.n) or not y_host.is_contiguous():
            raise ValueError("bad host frame")
        _check_image(phi_out, self.n)
        t = c_int64()
        check(lib().ddh_step_host_async(self._h, c_void_p(y_host.data_ptr()), c_void_p(phi_out.data_ptr()),
                                        ctypes.byref(t)))
        return t.value

    def host_wait(self, ticket: int) -> None:
        """Block until frame ``ticket`` of ``step_host_async`` has its phase in host memory."""
        check(lib().ddh_host_wait(self._h, int(ticket)))

    # -- WriteData --------------------------------------------------------------------
    def phase(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float32, device="cuda")
        _check_image(out, self.n)
        check(lib().ddh_phase(self._h, c_void_p(out.data_ptr())))
        self._join_current()
        return out

    def _join_current(self) -> None:
        """Order the caller's current stream after this state's stream (device copies)."""
        cur = torch.cuda.current_stream()
        if cur != self.torch_stream:
            cur.wait_stream(self.torch_stream)

    def reflectance(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float32, device="cuda")
        _check_image(out, self.n)
        check(lib().ddh_reflectance(self._h, c_void_p(out.data_ptr())))
        self._join_current()
        return out

    def set_state(self, r: torch.Tensor, phi: torch.Tensor, frame_index: int) -> None:
        _check_image(r, self.n)
        _check_image(phi, self.n)
        check(lib().ddh_set_state(self._h, c_void_p(r.data_ptr()), c_void_p(phi.data_ptr()), int(frame_index)))

    def set_params(self, params: DdhParams) -> None:
        """Replace the parameters (same grid size), keeping r, phi and the frame count; steps
        enqueued afterwards use them."""
        check(lib().ddh_set_params(self._h, byref(params)))
        self.params = params

    def noise_estimate(self) -> float:
        """sigma^2 the next frame will use: the running estimate with ``noise_update``
        (synchronises the stream), else ``noise_var``."""
        v = c_float()
        check(lib().ddh_noise_estimate(self._h, byref(v)))
        return float(v.value)

    @property
    def frame_index(self) -> int:
        return int(lib().ddh_frame_index(self._h))

    def strehl(self, phi_true: torch.Tensor) -> float:
        _check_image(phi_true, self.n)
        if not phi_true.is_cuda:
            raise ValueError("phi_true must be a CUDA tensor")
        out = c_float()
        check(lib().ddh_strehl(self._h, c_void_p(phi_true.data_ptr()), byref(out)))
        return float(out.value)

    def sync(self) -> None:
        check(lib().ddh_sync(self._h))

    # -- checkpoint -------------------------------------------------------------------
    def save(self) -> bytes:
        nbytes = lib().ddh_checkpoint_bytes(self.n)
        buf = ctypes.create_string_buffer(nbytes)
        check(lib().ddh_save(self._h, buf, nbytes))
        return buf.raw

    def load(self, blob: bytes) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(lib().ddh_load(self._h, buf, len(blob)))

    def close(self) -> None:
        if self._h:
            lib().ddh_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_batch(streams: list[Stream], frames: list[torch.Tensor]) -> None:
    """Advance every stream by one frame (one cluster-per-stream launch per grid size)."""
    if len(streams) != len(frames):
        raise ValueError("one frame per stream")
    for s, y in zip(streams, frames):
        _check_frame(y, s.n)
    hs = (c_void_p * len(streams))(*[s._h for s in streams])
    ys = (c_void_p * len(frames))(*[c_void_p(y.data_ptr()) for y in frames])
    check(lib().ddh_step_batch(hs, ys, len(streams)))


class BatchGraph:
    """One captured CUDA graph advancing every stream of a fixed set by one frame."""

    def __init__(self, streams: list[Stream]):
        self.streams = list(streams)
        self._h = c_void_p()
        hs = (c_void_p * len(streams))(*[s._h for s in streams])
        check(lib().ddh_batch_create(byref(self._h), hs, len(streams)))

    def run(self, frames: list[torch.Tensor]) -> None:
        if len(frames) != len(self.streams):
            raise ValueError("one frame per stream")
        for s, y in zip(self.streams, frames):
            _check_frame(y, s.n)
        ys = (c_void_p * len(frames))(*[c_void_p(y.data_ptr()) for y in frames])
        check(lib().ddh_batch_run(self._h, ys))

    def run_ptrs(self, ptr_array) -> None:
        """Run with a prepared ``(c_void_p * count)`` array of frame device pointers."""
        check(lib().ddh_batch_run(self._h, ptr_array))

    def close(self) -> None:
        if self._h:
            lib().ddh_batch_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft_schedule_count(n: int) -> int:
    return int(lib().ddh_fft_schedule_count(int(n)))


def set_fft_schedule(n: int, schedule: int) -> None:
    check(lib().ddh_set_fft_schedule(int(n), int(schedule)))


def get_fft_schedule(n: int) -> int:
    return int(lib().ddh_get_fft_schedule(int(n)))


def fft2(x: torch.Tensor, inverse: bool = False, out: torch.Tensor | None = None) -> torch.Tensor:
    """Unitary 2-D DFT (``F`` of Sec. 2) or its inverse, computed by libddh."""
    n = x.shape[0]
    _check_frame(x, n)
    if out is None:
        out = torch.empty_like(x)
    check(lib().ddh_fft2(c_void_p(x.data_ptr()), c_void_p(out.data_ptr()), n, 1 if inverse else 0,
                         _stream_handle(None)))
    return out
