"""K unrolled DDH-MBIR frame steps as a ``torch.autograd.Function`` (forward and adjoint
kernels of libddh).

``unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params)`` runs ``len(frames)``
frame steps from the state ``(r0, phi0)`` and returns the final ``(r_K, phi_K)``.  The
forward pass keeps one checkpoint of the state per frame and, with ``store_traces`` (the
default), each frame's intermediates (``ddh_unrolled_forward``, about 40 bytes per pixel and
frame in all); the backward pass (``ddh_unrolled_backward``) runs the hand-written adjoint
frame by frame in reverse inside the library, from the stored intermediates or, without them,
recomputing each frame from its checkpoint (the same gradients bit for bit), giving gradients
with respect to ``r0``, ``phi0`` and the scalar tensors ``prior_sigma``, ``prior_p`` and
``noise_var``.
"""
from __future__ import annotations

import copy
import threading
from ctypes import c_void_p

import torch

from . import ddh

# One library state per (device, stream, grid size), reused by every call: creating a state
# allocates device memory and freeing it waits for the whole device (cudaFree), which would
# stall the GPU once per window.  The state is scratch here (each call sets r, phi and the
# parameters before it enqueues); the lock orders calls from different threads.
_states: dict = {}
_lock = threading.Lock()


def clear_cache() -> None:
    """Free the library states kept for reuse (device memory of r, phi and staging buffers per
    device, stream and grid size); the next call creates them again."""
    with _lock:
        _states.clear()


def _state(p, stream):
    key = (stream.device.index, stream.cuda_stream, int(p.n))
    s = _states.get(key)
    if s is None:
        s = _states[key] = ddh.Stream(p, stream=stream)
    else:
        s.set_params(p)
    return s


def _with(params, prior_sigma, prior_p, noise_var):
    p = copy.copy(params)
    p.prior_sigma = float(prior_sigma)
    p.prior_p = float(prior_p)
    p.noise_var = float(noise_var)
    return p


def _ptr_array(base, stride, count):
    """C array of `count` device pointers base, base + stride, ... (bytes)."""
    return (c_void_p * count)(*[base + k * stride for k in range(count)])


class UnrolledDDH(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, phi0, prior_sigma, prior_p, noise_var, frames, params, store_traces=True):
        p = _with(params, prior_sigma, prior_p, noise_var)
        n = int(p.n)
        if (frames.dtype != torch.complex64 or frames.dim() != 3 or tuple(frames.shape[1:]) != (n, n)
                or not frames.is_cuda or not frames.is_contiguous() or frames.shape[0] < 1):
            raise ValueError(f"frames must be a contiguous complex64 CUDA tensor of shape (K, {n}, {n})")
        K, img = frames.shape[0], n * n * 4
        # checkpoints: the state entering each frame, and the final state (ck[k, 0] = r, ck[k, 1] = phi)
        ck = torch.empty((K + 1, 2, n, n), dtype=torch.float32, device="cuda")
        ys = _ptr_array(frames.data_ptr(), 2 * img, K)
        rc = _ptr_array(ck.data_ptr(), 2 * img, K + 1)
        pc = _ptr_array(ck.data_ptr() + img, 2 * img, K + 1)
        tr, tc = None, None
        if store_traces:
            tf = int(ddh.lib().ddh_trace_floats(n))
            tr = torch.empty((K, tf), dtype=torch.float32, device="cuda")
            tc = _ptr_array(tr.data_ptr(), 4 * tf, K)
        with _lock:
            s = _state(p, torch.cuda.current_stream())
            s.set_state(r0.detach().contiguous(), phi0.detach().contiguous(), 0)
            ddh.check(ddh.lib().ddh_unrolled_forward(s._h, K, ys, rc, pc, tc))
        r_k, phi_k = ck[K, 0].clone(), ck[K, 1].clone()
        ctx.params, ctx.stream, ctx.ck, ctx.traces, ctx.arrays = p, s, ck, tr, (ys, rc, pc, tc)
        ctx.save_for_backward(frames)
        return r_k, phi_k

    @staticmethod
    def backward(ctx, r_bar, phi_bar):
        (frames,) = ctx.saved_tensors
        p, s, ck = ctx.params, ctx.stream, ctx.ck
        ys, rc, pc, tc = ctx.arrays
        n, K = p.n, frames.shape[0]
        L = ddh.lib()
        wsb = L.ddh_unrolled_workspace_bytes(n)
        ws = torch.empty(wsb // 4, dtype=torch.float32, device="cuda")
        grads = torch.zeros(3, dtype=torch.float32, device="cuda")
        rb = (r_bar if r_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        pb = (phi_bar if phi_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        r0b, p0b = torch.empty_like(rb), torch.empty_like(pb)
        cur = torch.cuda.current_stream()
        if cur != s.torch_stream:  # order the state's stream after the gradient inputs
            s.torch_stream.wait_stream(cur)
            for t in (ws, grads, rb, pb, r0b, p0b):
                t.record_stream(s.torch_stream)
        with _lock:
            s.set_params(p)
            ddh.check(L.ddh_unrolled_backward(s._h, K, ys, rc, pc, tc, c_void_p(rb.data_ptr()), c_void_p(pb.data_ptr()),
                                              c_void_p(r0b.data_ptr()), c_void_p(p0b.data_ptr()),
                                              c_void_p(grads.data_ptr()), c_void_p(ws.data_ptr()), wsb))
        s.sync()  # waits for the adjoint and raises a latched device error (a non-finite frame)
        g = grads.to(torch.float64)
        return r0b, p0b, g[0], g[1], g[2], None, None, None


def unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params, store_traces=True):
    return UnrolledDDH.apply(r0, phi0, prior_sigma, prior_p, noise_var, frames, params, store_traces)
