"""The allocation-free adjoint entry point (ddh_step_backward_noalloc).

Callers such as a real-time beam-control loop cannot afford a device allocation while a
frame is being processed (cudaMalloc may take unbounded time and may synchronise the whole
device), so the library offers a variant of the frame-step adjoint whose scratch lives in a
static device array instead of a caller workspace.  These tests call it through the C ABI
and check it against ddh_step_backward on two calls in a row (the shared scratch keeps the
previous call's contents, which must not leak into the next result).  This file is named to
be collected last.
"""
import numpy as np
import pytest
import torch

from oracle import ddh_oracle as o
from synth import ddh_synth as sy

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the adjoint tests' per-frame tolerance


@pytest.fixture(scope="module")
def ddh():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import ddh as mod
    assert torch.cuda.is_available()
    return mod


def _ptr(ddh, t):
    return ddh.c_void_p(t.data_ptr())


def _inputs(ddh, s, n, y, r_prev, phi_prev, seed):
    """Trace of the frame from (r_prev, phi_prev), its output r, and random output gradients."""
    L = ddh.lib()
    s.set_state(r_prev, phi_prev, 0)
    trace = torch.zeros(L.ddh_trace_floats(n), dtype=torch.float32, device="cuda")
    ddh.check(L.ddh_step_trace(s._h, _ptr(ddh, y), _ptr(ddh, trace)))
    r_new = s.reflectance().clone()
    g = torch.Generator(device="cuda").manual_seed(seed)
    r_bar = torch.randn((n, n), device="cuda", generator=g)
    phi_bar = torch.randn((n, n), device="cuda", generator=g)
    return trace, r_new, r_bar, phi_bar


@pytest.mark.parametrize("n", [64, 128])
def test_noalloc_backward_matches_workspace_backward_twice(ddh, n):
    L = ddh.lib()
    cfg = sy.config_single_64(3) if n == 64 else sy.config_batched(3)[0]
    ys, _ = sy.Stream(cfg).frames(3)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
    s = ddh.Stream(p)
    frames = torch.from_numpy(ys).cuda()
    # a realistic entering state: the state after one frame
    s.step(frames[0])
    r1, phi1 = s.reflectance().clone(), s.phase().clone()
    ws = torch.empty(L.ddh_backward_workspace_bytes(n) // 4, dtype=torch.float32, device="cuda")
    for call, k in enumerate((1, 2)):  # two calls in a row, different frames and gradients
        trace, r_new, r_bar, phi_bar = _inputs(ddh, s, n, frames[k], r1, phi1, seed=call)
        outs = []
        for noalloc in (False, True):
            out_r = torch.full((n, n), float("nan"), device="cuda")
            out_p = torch.full((n, n), float("nan"), device="cuda")
            grads = torch.zeros(3, device="cuda")
            args = [s._h, _ptr(ddh, frames[k]), _ptr(ddh, r1), _ptr(ddh, phi1), _ptr(ddh, trace), _ptr(ddh, r_new),
                    _ptr(ddh, r_bar), _ptr(ddh, phi_bar), _ptr(ddh, out_r), _ptr(ddh, out_p), _ptr(ddh, grads)]
            if noalloc:
                ddh.check(L.ddh_step_backward_noalloc(*args))
            else:
                ddh.check(L.ddh_step_backward(*args, _ptr(ddh, ws), ws.numel() * 4))
            s.sync()
            outs.append((out_r.cpu().numpy(), out_p.cpu().numpy(), grads.cpu().numpy()))
        (ra, pa, ga), (rb, pb, gb) = outs
        assert np.all(np.isfinite(rb)) and np.all(np.isfinite(pb))
        assert np.linalg.norm(rb - ra) <= TOL * np.linalg.norm(ra)
        assert np.linalg.norm(pb - pa) <= TOL * np.linalg.norm(pa)
        assert np.all(np.abs(gb - ga) <= TOL * np.abs(ga))


def test_noalloc_backward_rejects_grids_above_its_scratch(ddh):
    L = ddh.lib()
    p = ddh.default_params(256, 128.0, 5.0)
    s = ddh.Stream(p)
    z = torch.zeros((256, 256), device="cuda")
    y = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
    tr = torch.zeros(L.ddh_trace_floats(256), device="cuda")
    g = torch.zeros(3, device="cuda")
    rc = L.ddh_step_backward_noalloc(s._h, _ptr(ddh, y), _ptr(ddh, z), _ptr(ddh, z), _ptr(ddh, tr), _ptr(ddh, z),
                                     _ptr(ddh, z), _ptr(ddh, z), _ptr(ddh, z), _ptr(ddh, z), _ptr(ddh, g))
    assert rc == -1
    assert b"128" in L.ddh_last_cuda_error()
