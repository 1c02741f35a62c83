"""K unrolled DDH-MBIR frame steps as a ``torch.autograd.Function`` (forward and adjoint
kernels of libddh).

``unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params)`` runs ``len(frames)``
frame steps from the state ``(r0, phi0)`` and returns the final ``(r_K, phi_K)``.  The
forward pass keeps one checkpoint of the state per frame (``ddh_unrolled_forward``); the
backward pass (``ddh_unrolled_backward``) recomputes each frame's intermediates from its
checkpoint and runs the hand-written adjoint, frame by frame in reverse inside the library,
giving gradients with respect to ``r0``, ``phi0`` and the scalar tensors ``prior_sigma``,
``prior_p`` and ``noise_var``.
"""
from __future__ import annotations

import copy
from ctypes import c_void_p

import torch

from . import ddh


def _with(params, prior_sigma, prior_p, noise_var):
    p = copy.copy(params)
    p.prior_sigma = float(prior_sigma)
    p.prior_p = float(prior_p)
    p.noise_var = float(noise_var)
    return p


def _ptrs(tensors):
    return (c_void_p * len(tensors))(*[c_void_p(t.data_ptr()) for t in tensors])


class UnrolledDDH(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, phi0, prior_sigma, prior_p, noise_var, frames, params):
        p = _with(params, prior_sigma, prior_p, noise_var)
        n, K = p.n, frames.shape[0]
        s = ddh.Stream(p)
        s.set_state(r0.detach().contiguous(), phi0.detach().contiguous(), 0)
        # checkpoints: the state entering each frame, and the final state (ck[k, 0] = r, ck[k, 1] = phi)
        ck = torch.empty((K + 1, 2, n, n), dtype=torch.float32, device="cuda")
        ys = [frames[k] for k in range(K)]
        for y in ys:
            ddh._check_frame(y, n)
        ddh.check(ddh.lib().ddh_unrolled_forward(s._h, K, _ptrs(ys), _ptrs([ck[k, 0] for k in range(K + 1)]),
                                                 _ptrs([ck[k, 1] for k in range(K + 1)])))
        r_k, phi_k = ck[K, 0].clone(), ck[K, 1].clone()
        ctx.params, ctx.stream, ctx.ck = p, s, ck
        ctx.save_for_backward(frames)
        return r_k, phi_k

    @staticmethod
    def backward(ctx, r_bar, phi_bar):
        (frames,) = ctx.saved_tensors
        p, s, ck = ctx.params, ctx.stream, ctx.ck
        n, K = p.n, frames.shape[0]
        L = ddh.lib()
        wsb = L.ddh_unrolled_workspace_bytes(n)
        ws = torch.empty(wsb // 4, dtype=torch.float32, device="cuda")
        grads = torch.zeros(3, dtype=torch.float32, device="cuda")
        rb = (r_bar if r_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        pb = (phi_bar if phi_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        r0b, p0b = torch.empty_like(rb), torch.empty_like(pb)
        ys = [frames[k] for k in range(K)]
        ddh.check(L.ddh_unrolled_backward(s._h, K, _ptrs(ys), _ptrs([ck[k, 0] for k in range(K + 1)]),
                                          _ptrs([ck[k, 1] for k in range(K + 1)]), c_void_p(rb.data_ptr()),
                                          c_void_p(pb.data_ptr()), c_void_p(r0b.data_ptr()), c_void_p(p0b.data_ptr()),
                                          c_void_p(grads.data_ptr()), c_void_p(ws.data_ptr()), wsb))
        s.sync()
        g = grads.to(torch.float64)
        return r0b, p0b, g[0], g[1], g[2], None, None


def unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params):
    return UnrolledDDH.apply(r0, phi0, prior_sigma, prior_p, noise_var, frames, params)
