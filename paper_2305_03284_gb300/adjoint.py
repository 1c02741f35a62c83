"""K unrolled DDH-MBIR frame steps as a ``torch.autograd.Function`` (forward and adjoint
kernels of libddh).

``unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params)`` runs ``len(frames)``
frame steps from the state ``(r0, phi0)`` and returns the final ``(r_K, phi_K)``.  The
forward pass keeps one checkpoint of the state per frame; the backward pass recomputes each
frame's intermediates from its checkpoint (``ddh_step_trace``) and runs the hand-written
adjoint (``ddh_step_backward``), giving gradients with respect to ``r0``, ``phi0`` and the
scalar tensors ``prior_sigma``, ``prior_p`` and ``noise_var``.
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


class UnrolledDDH(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r0, phi0, prior_sigma, prior_p, noise_var, frames, params):
        p = _with(params, prior_sigma, prior_p, noise_var)
        s = ddh.Stream(p)
        s.set_state(r0.detach().contiguous(), phi0.detach().contiguous(), 0)
        ckpts = []
        for k in range(frames.shape[0]):
            ckpts.append((s.reflectance().clone(), s.phase().clone()))
            s.step(frames[k])
        r_k, phi_k = s.reflectance().clone(), s.phase().clone()
        s.sync()
        ctx.params = p
        ctx.ckpts = ckpts
        ctx.save_for_backward(frames)
        return r_k, phi_k

    @staticmethod
    def backward(ctx, r_bar, phi_bar):
        (frames,) = ctx.saved_tensors
        p, n = ctx.params, ctx.params.n
        L = ddh.lib()
        s = ddh.Stream(p)
        ws = torch.empty(L.ddh_backward_workspace_bytes(n) // 4, dtype=torch.float32, device="cuda")
        trace = torch.zeros(L.ddh_trace_floats(n), dtype=torch.float32, device="cuda")
        grads = torch.zeros(3, dtype=torch.float32, device="cuda")
        rb = (r_bar if r_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        pb = (phi_bar if phi_bar is not None else torch.zeros((n, n), device="cuda")).contiguous().float()
        for k in range(frames.shape[0] - 1, -1, -1):
            r_prev, phi_prev = ctx.ckpts[k]
            s.set_state(r_prev, phi_prev, k)
            y = frames[k]
            ddh.check(L.ddh_step_trace(s._h, c_void_p(y.data_ptr()), c_void_p(trace.data_ptr())))
            r_new = s.reflectance()
            out_r = torch.empty_like(rb)
            out_p = torch.empty_like(pb)
            ddh.check(L.ddh_step_backward(s._h, c_void_p(y.data_ptr()), c_void_p(r_prev.data_ptr()),
                                          c_void_p(phi_prev.data_ptr()), c_void_p(trace.data_ptr()),
                                          c_void_p(r_new.data_ptr()), c_void_p(rb.data_ptr()),
                                          c_void_p(pb.data_ptr()), c_void_p(out_r.data_ptr()),
                                          c_void_p(out_p.data_ptr()), c_void_p(grads.data_ptr()),
                                          c_void_p(ws.data_ptr()), ws.numel() * 4))
            rb, pb = out_r, out_p
        s.sync()
        g = grads.to(torch.float64)
        return rb, pb, g[0], g[1], g[2], None, None


def unrolled(r0, phi0, prior_sigma, prior_p, noise_var, frames, params):
    return UnrolledDDH.apply(r0, phi0, prior_sigma, prior_p, noise_var, frames, params)
