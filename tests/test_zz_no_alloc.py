"""The allocation-free adjoint entry point (ddh_step_backward_noalloc).

Callers such as a real-time beam-control loop cannot afford a device allocation while a
frame is being processed (cudaMalloc may take unbounded time and may synchronise the whole
device), and a host whose device memory is fully budgeted up front has none to give, so the
library offers a variant of the frame-step adjoint whose scratch lives in a static device
array instead of a caller workspace.  These tests call it through the C ABI and check it
against ddh_step_backward on two calls in a row, bit for bit: both run the same kernels on
scratch of the same layout, so any difference would mean the shared array kept something of
an earlier call that leaked into the next result.  They also check that the calls allocate no
device memory.  This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from synth import ddh_synth as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddh():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import ddh as mod
    assert torch.cuda.is_available()
    return mod


def _ptr(ddh, t):
    return ddh.c_void_p(t.data_ptr())


def _config(n):
    if n == 32:
        return sy.config_adjoint(small=True, streams=1, frames=3)[0]
    if n == 64:
        return sy.config_single_64(3)
    return sy.config_batched(3)[0]  # a 128 x 128 stream


class _Case:
    """One stream of grid n: an entering state after one frame, and per call a frame's trace,
    its output r and random output gradients (all on the device, made before any timed call)."""

    def __init__(self, ddh, n, seed):
        L = ddh.lib()
        cfg = _config(n)
        assert cfg.n == n
        ys, _ = sy.Stream(cfg).frames(3)
        self.n = n
        self.s = ddh.Stream(ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr))
        self.frames = torch.from_numpy(ys).cuda()
        self.s.step(self.frames[0])
        self.r1, self.phi1 = self.s.reflectance().clone(), self.s.phase().clone()
        self.ws = torch.empty(L.ddh_backward_workspace_bytes(n) // 4, dtype=torch.float32, device="cuda")
        self.calls = []
        for k in (1, 2):
            self.s.set_state(self.r1, self.phi1, 0)
            trace = torch.zeros(L.ddh_trace_floats(n), dtype=torch.float32, device="cuda")
            ddh.check(L.ddh_step_trace(self.s._h, _ptr(ddh, self.frames[k]), _ptr(ddh, trace)))
            r_new = self.s.reflectance().clone()
            g = torch.Generator(device="cuda").manual_seed(seed + k)
            self.calls.append((k, trace, r_new, torch.randn((n, n), device="cuda", generator=g),
                               torch.randn((n, n), device="cuda", generator=g)))
        self.s.sync()

    def run(self, ddh, call, noalloc):
        L = ddh.lib()
        n = self.n
        k, trace, r_new, r_bar, phi_bar = self.calls[call]
        out_r = torch.full((n, n), float("nan"), device="cuda")
        out_p = torch.full((n, n), float("nan"), device="cuda")
        grads = torch.zeros(3, device="cuda")
        args = [self.s._h, _ptr(ddh, self.frames[k]), _ptr(ddh, self.r1), _ptr(ddh, self.phi1), _ptr(ddh, trace),
                _ptr(ddh, r_new), _ptr(ddh, r_bar), _ptr(ddh, phi_bar), _ptr(ddh, out_r), _ptr(ddh, out_p),
                _ptr(ddh, grads)]
        if noalloc:
            ddh.check(L.ddh_step_backward_noalloc(*args))
        else:
            ddh.check(L.ddh_step_backward(*args, _ptr(ddh, self.ws), self.ws.numel() * 4))
        self.s.sync()
        return out_r.cpu().numpy(), out_p.cpu().numpy(), grads.cpu().numpy()


def _assert_same(a, b):
    for x, y in zip(a, b):
        assert np.all(np.isfinite(y))
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("n", [32, 64, 128])
def test_noalloc_backward_equals_workspace_backward_twice(ddh, n):
    case = _Case(ddh, n, seed=10 * n)
    for call in (0, 1):  # two calls in a row, different frames and gradients
        _assert_same(case.run(ddh, call, noalloc=False), case.run(ddh, call, noalloc=True))


def test_noalloc_backward_larger_grid_then_smaller(ddh):
    """The shared array first holds a 128 x 128 call's scratch, then serves a 64 x 64 call."""
    big, small = _Case(ddh, 128, seed=7), _Case(ddh, 64, seed=8)
    ref_big, ref_small = big.run(ddh, 0, noalloc=False), small.run(ddh, 0, noalloc=False)
    _assert_same(ref_big, big.run(ddh, 0, noalloc=True))
    _assert_same(ref_small, small.run(ddh, 0, noalloc=True))


def test_noalloc_backward_allocates_no_device_memory(ddh):
    case = _Case(ddh, 64, seed=3)
    case.run(ddh, 0, noalloc=True)  # first call on the device: the array's address lookup
    torch.cuda.synchronize()
    L = ddh.lib()
    k, trace, r_new, r_bar, phi_bar = case.calls[1]
    n = case.n
    out_r = torch.empty((n, n), device="cuda")
    out_p = torch.empty((n, n), device="cuda")
    grads = torch.zeros(3, device="cuda")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used1 = torch.cuda.memory_allocated()
    for _ in range(20):
        ddh.check(L.ddh_step_backward_noalloc(case.s._h, _ptr(ddh, case.frames[k]), _ptr(ddh, case.r1),
                                              _ptr(ddh, case.phi1), _ptr(ddh, trace), _ptr(ddh, r_new),
                                              _ptr(ddh, r_bar), _ptr(ddh, phi_bar), _ptr(ddh, out_r),
                                              _ptr(ddh, out_p), _ptr(ddh, grads)))
    case.s.sync()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, f"device free memory changed by {free1 - free2} bytes over 20 calls"
    assert torch.cuda.memory_allocated() == used1


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
