"""GPU adjoint (ddh_step_backward, the autograd Function) against the FP64 oracle gradient
and FP64 finite differences."""
from ctypes import c_void_p

import numpy as np
import pytest
import torch

from oracle import ddh_adjoint as adj
from oracle import ddh_oracle as o
from synth import ddh_synth as sy

pytestmark = pytest.mark.gpu

TOL_FRAME = 1e-4   # one frame: FP32 adjoint vs FP64 adjoint at the same (float32) inputs (measured <= 2.3e-5)
TOL_UNROLLED = 1e-3  # K = 8 frames: trajectories differ by FP32 rounding amplified per frame (measured <= 4e-5)


@pytest.fixture(scope="module")
def mods():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import adjoint, ddh
    return ddh, adjoint


def _oracle_params(p):
    return o.Params(n=p.n, aperture_diam=float(p.aperture_diam), lam=float(p.lam), alpha=float(p.alpha),
                    n_k=p.n_k, noise_var=float(p.noise_var), prior_p=float(p.prior_p), prior_q=float(p.prior_q),
                    prior_T=float(p.prior_T), prior_sigma=float(p.prior_sigma), r_floor=float(p.r_floor),
                    tilt_mode=p.tilt_mode, phase_block=p.phase_block)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("n,tilt", [(32, 1), (64, 1), (64, 0), (256, 1)])
def test_frame_backward_matches_oracle(mods, n, tilt):
    ddh, _ = mods
    cfg = {32: sy.config_adjoint(small=True, streams=1, frames=3)[0], 64: sy.config_single_64(3),
           256: sy.config_adjoint(streams=1, frames=3)[0]}[n]
    ys, _ = sy.Stream(cfg).frames(3)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr, tilt_mode=tilt)
    prm = _oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    st = o.init_state(cfg.n)
    for y in ys[:2]:
        st, _ = o.step(st, y, prm)
    r32, p32 = st.r.astype(np.float32), st.phi.astype(np.float32)
    rng = np.random.default_rng(n)
    rbar = rng.standard_normal((n, n)).astype(np.float32)
    pbar = np.where(a, rng.standard_normal((n, n)), 0.0).astype(np.float32)
    ref_r, ref_p, ref_g, _ = adj.frame_backward(r32.astype(np.float64), p32.astype(np.float64), ys[2], prm,
                                                rbar.astype(np.float64), pbar.astype(np.float64))
    L = ddh.lib()
    s = ddh.Stream(p)
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    r_prev, phi_prev, y = cu(r32), cu(p32), cu(ys[2])
    s.set_state(r_prev, phi_prev, 2)
    tr = torch.zeros(L.ddh_trace_floats(n), dtype=torch.float32, device="cuda")
    ddh.check(L.ddh_step_trace(s._h, ddh.c_void_p(y.data_ptr()), ddh.c_void_p(tr.data_ptr())))
    r_new = s.reflectance()
    ws = torch.empty(L.ddh_backward_workspace_bytes(n) // 4, dtype=torch.float32, device="cuda")
    g = torch.zeros(3, dtype=torch.float32, device="cuda")
    out_r, out_p = torch.empty((n, n), device="cuda"), torch.empty((n, n), device="cuda")
    rb_t, pb_t = cu(rbar), cu(pbar)
    ptr = lambda t: ddh.c_void_p(t.data_ptr())
    ddh.check(L.ddh_step_backward(s._h, ptr(y), ptr(r_prev), ptr(phi_prev), ptr(tr), ptr(r_new), ptr(rb_t), ptr(pb_t),
                                  ptr(out_r), ptr(out_p), ptr(g), ptr(ws), ws.numel() * 4))
    torch.cuda.synchronize()
    er, ep = _rel(out_r.cpu().numpy(), ref_r), _rel(out_p.cpu().numpy(), ref_p)
    eg = np.abs(g.cpu().numpy().astype(np.float64) - ref_g) / np.maximum(np.abs(ref_g), 1e-12)
    print(f"n={n} tilt={tilt} r_bar {er:.2e} phi_bar {ep:.2e} grads {eg}")
    assert er < TOL_FRAME and ep < TOL_FRAME and np.all(eg < TOL_FRAME), (er, ep, eg)


def test_unrolled_autograd_matches_oracle_and_fd(mods):
    """K = 8 frames on the 32x32 copy of the differentiation workload, through
    torch.autograd: gradients in sigma_r, p, sigma^2, phi0 and r0."""
    ddh, adjoint = mods
    K = 8
    cfg = sy.config_adjoint(small=True, streams=1, frames=K)[0]
    ys, _ = sy.Stream(cfg).frames(K)
    p = ddh.default_params(32, 16.0, cfg.snr)
    prm = _oracle_params(p)
    a = o.aperture(32, 16.0)
    rng = np.random.default_rng(4)
    phi0 = np.where(a, 0.3 * rng.standard_normal((32, 32)), 0.0).astype(np.float32)
    r0 = (0.05 + 0.02 * rng.random((32, 32))).astype(np.float32)
    c = rng.standard_normal((3, 32, 32))
    frames = torch.from_numpy(ys).cuda()
    at = torch.from_numpy(a).cuda()
    ct = torch.from_numpy(c).cuda()
    r0t = torch.from_numpy(r0).cuda().requires_grad_(True)
    p0t = torch.from_numpy(phi0).cuda().requires_grad_(True)
    sig = torch.tensor(float(p.prior_sigma), dtype=torch.float64, requires_grad=True)
    pp = torch.tensor(float(p.prior_p), dtype=torch.float64, requires_grad=True)
    s2 = torch.tensor(float(p.noise_var), dtype=torch.float64, requires_grad=True)
    rK, phiK = adjoint.unrolled(r0t, p0t, sig, pp, s2, frames, p)
    loss = (at * (ct[0] * torch.cos(phiK) + ct[1] * torch.sin(phiK))).sum() + (ct[2] * rK).sum()
    loss.backward()
    gpu = np.array([sig.grad.item(), pp.grad.item(), s2.grad.item()])
    # oracle gradient along the oracle's own FP64 trajectory from the same float32 start
    st = o.State(r=r0.astype(np.float64), phi=phi0.astype(np.float64))
    for y in ys:
        st, _ = o.step(st, y, prm)
    phib = a * (-c[0] * np.sin(st.phi) + c[1] * np.cos(st.phi))
    rb, pb, g, _ = adj.unrolled_grad(r0.astype(np.float64), phi0.astype(np.float64), ys, prm, c[2], phib)
    eg = np.abs(gpu - g) / np.abs(g)
    ephi = _rel(p0t.grad.cpu().numpy(), pb)
    er = _rel(r0t.grad.cpu().numpy(), rb)
    print(f"unrolled K=8: grads rel {eg}, phi0 {ephi:.2e}, r0 {er:.2e}")
    assert np.all(eg < TOL_UNROLLED) and ephi < TOL_UNROLLED and er < TOL_UNROLLED
    # FP64 central finite difference of the oracle in sigma_r (h = 1e-6)
    from dataclasses import replace

    def L(prm_):
        s_ = o.State(r=r0.astype(np.float64), phi=phi0.astype(np.float64))
        for y in ys:
            s_, _ = o.step(s_, y, prm_)
        return float(np.sum(a * (c[0] * np.cos(s_.phi) + c[1] * np.sin(s_.phi))) + np.sum(c[2] * s_.r))
    h = 1e-6
    fd = (L(replace(prm, prior_sigma=prm.prior_sigma + h)) - L(replace(prm, prior_sigma=prm.prior_sigma - h))) / (2 * h)
    assert abs(gpu[0] - fd) < TOL_UNROLLED * abs(fd), (gpu[0], fd)


def test_config4_sixteen_streams_256(mods):
    """16 streams at 256^2, K = 8 unrolled steps each: finite gradients for every stream."""
    ddh, adjoint = mods
    cfgs = sy.config_adjoint(streams=16, frames=8)
    for cfg in cfgs[:16]:
        ys, _ = sy.Stream(cfg).frames(8)
        p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
        r0 = torch.zeros((256, 256), device="cuda", requires_grad=True)
        phi0 = torch.zeros((256, 256), device="cuda", requires_grad=True)
        sig = torch.tensor(float(p.prior_sigma), dtype=torch.float64, requires_grad=True)
        pp = torch.tensor(float(p.prior_p), dtype=torch.float64, requires_grad=True)
        s2 = torch.tensor(float(p.noise_var), dtype=torch.float64, requires_grad=True)
        rK, phiK = adjoint.unrolled(r0, phi0, sig, pp, s2, torch.from_numpy(ys).cuda(), p)
        (torch.cos(phiK).sum() + rK.sum()).backward()
        for t in (sig.grad, pp.grad, s2.grad, r0.grad, phi0.grad):
            assert torch.isfinite(t).all()
        if cfg.stream_id == 0:
            # the first stream against the FP64 oracle gradient at full size (same loss)
            prm = _oracle_params(p)
            a = o.aperture(256, cfg.aperture_diam)
            st = o.init_state(256)
            for y in ys:
                st, _ = o.step(st, y, prm)
            rb, pb, g, _ = adj.unrolled_grad(np.zeros((256, 256)), np.zeros((256, 256)), ys, prm,
                                             np.ones((256, 256)), a * -np.sin(st.phi))
            gpu = np.array([sig.grad.item(), pp.grad.item(), s2.grad.item()])
            eg = np.abs(gpu - g) / np.abs(g)
            er, ep = _rel(r0.grad.cpu().numpy(), rb), _rel(phi0.grad.cpu().numpy() * a, pb * a)
            print(f"256^2 K=8 stream 0: grads rel {eg}, r0 {er:.2e}, phi0 {ep:.2e}")
            assert np.all(eg < TOL_UNROLLED) and er < TOL_UNROLLED and ep < TOL_UNROLLED, (eg, er, ep)


def _window_grads(ddh, adjoint, cfg, ys_dev):
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
    r0 = torch.full((cfg.n, cfg.n), 1e-3, device="cuda", requires_grad=True)
    phi0 = torch.zeros((cfg.n, cfg.n), device="cuda", requires_grad=True)
    sig = torch.tensor(float(p.prior_sigma), dtype=torch.float64, requires_grad=True)
    pp = torch.tensor(float(p.prior_p), dtype=torch.float64, requires_grad=True)
    s2 = torch.tensor(float(p.noise_var), dtype=torch.float64, requires_grad=True)
    rK, phiK = adjoint.unrolled(r0, phi0, sig, pp, s2, ys_dev, p)
    (rK.sum() + phiK.square().sum()).backward()
    return [sig.grad, pp.grad, s2.grad, r0.grad, phi0.grad]


def test_windows_on_concurrent_streams_equal_sequential_windows(mods):
    """Unrolled windows issued on four CUDA streams at once (the library keeps one state per
    stream) give bit for bit the gradients of the same windows run one after another."""
    ddh, adjoint = mods
    cfgs = sy.config_adjoint(streams=8, frames=8)
    ys = [torch.from_numpy(sy.Stream(c).frames(8)[0]).cuda() for c in cfgs]
    seq = [[t.detach().clone() for t in _window_grads(ddh, adjoint, c, y)] for c, y in zip(cfgs, ys)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(4)]
    conc = []
    for i, (c, y) in enumerate(zip(cfgs, ys)):
        st = streams[i % 4]
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            conc.append(_window_grads(ddh, adjoint, c, y))
    torch.cuda.synchronize()
    for a, b in zip(seq, conc):
        for x, y in zip(a, b):
            assert torch.equal(x, y.to(x.device))


def test_unrolled_calls_equal_per_frame_calls(mods):
    """ddh_unrolled_forward / ddh_unrolled_backward (the K-frame loops inside the library)
    give bit for bit what the per-frame calls give: ddh_step from each checkpoint, then
    ddh_step_trace + ddh_step_backward frame by frame in reverse."""
    ddh, adjoint = mods
    cfg = sy.config_adjoint(small=True, streams=1, frames=5)[0]
    K, n = 5, 32
    ys = torch.from_numpy(sy.Stream(cfg).frames(K)[0]).cuda()
    p = ddh.default_params(n, 16.0, cfg.snr)
    L = ddh.lib()
    rng = np.random.default_rng(3)
    r0 = torch.from_numpy((0.05 + rng.random((n, n))).astype(np.float32)).cuda()
    phi0 = torch.zeros((n, n), device="cuda")
    rbar = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda()
    pbar = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda()
    ptrs = lambda ts: (c_void_p * len(ts))(*[c_void_p(t.data_ptr()) for t in ts])
    # library loops
    s = ddh.Stream(p)
    s.set_state(r0, phi0, 0)
    ck = torch.empty((K + 1, 2, n, n), device="cuda")
    ddh.check(L.ddh_unrolled_forward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck[k, 0] for k in range(K + 1)]),
                                     ptrs([ck[k, 1] for k in range(K + 1)]), None))
    wsb = L.ddh_unrolled_workspace_bytes(n)
    ws = torch.empty(wsb // 4, device="cuda")
    r0b, p0b, g = torch.empty((n, n), device="cuda"), torch.empty((n, n), device="cuda"), torch.zeros(3, device="cuda")
    ddh.check(L.ddh_unrolled_backward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck[k, 0] for k in range(K + 1)]),
                                      ptrs([ck[k, 1] for k in range(K + 1)]), None, c_void_p(rbar.data_ptr()),
                                      c_void_p(pbar.data_ptr()), c_void_p(r0b.data_ptr()), c_void_p(p0b.data_ptr()),
                                      c_void_p(g.data_ptr()), c_void_p(ws.data_ptr()), wsb))
    s.sync()
    # the same with the forward's stored traces instead of recomputing each frame
    s.set_state(r0, phi0, 0)
    ck2 = torch.empty((K + 1, 2, n, n), device="cuda")
    trs = torch.empty((K, L.ddh_trace_floats(n)), device="cuda")
    ddh.check(L.ddh_unrolled_forward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck2[k, 0] for k in range(K + 1)]),
                                     ptrs([ck2[k, 1] for k in range(K + 1)]), ptrs([trs[k] for k in range(K)])))
    r0b2, p0b2, gt = torch.empty((n, n), device="cuda"), torch.empty((n, n), device="cuda"), torch.zeros(3, device="cuda")
    ddh.check(L.ddh_unrolled_backward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck2[k, 0] for k in range(K + 1)]),
                                      ptrs([ck2[k, 1] for k in range(K + 1)]), ptrs([trs[k] for k in range(K)]),
                                      c_void_p(rbar.data_ptr()), c_void_p(pbar.data_ptr()), c_void_p(r0b2.data_ptr()),
                                      c_void_p(p0b2.data_ptr()), c_void_p(gt.data_ptr()), c_void_p(ws.data_ptr()), wsb))
    s.sync()
    assert torch.equal(ck, ck2) and torch.equal(r0b, r0b2) and torch.equal(p0b, p0b2) and torch.equal(g, gt)
    # the same through per-frame calls
    t = ddh.Stream(p)
    t.set_state(r0, phi0, 0)
    states = [(r0.clone(), phi0.clone())]
    for k in range(K):
        t.step(ys[k])
        states.append((t.reflectance().clone(), t.phase().clone()))
    for k in range(K + 1):
        assert torch.equal(ck[k, 0], states[k][0]) and torch.equal(ck[k, 1], states[k][1]), k
    bws = torch.empty(L.ddh_backward_workspace_bytes(n) // 4, device="cuda")
    trace = torch.zeros(L.ddh_trace_floats(n), device="cuda")
    g2 = torch.zeros(3, device="cuda")
    rb, pb = rbar, pbar
    for k in range(K - 1, -1, -1):
        t.set_state(states[k][0], states[k][1], k)
        ddh.check(L.ddh_step_trace(t._h, c_void_p(ys[k].data_ptr()), c_void_p(trace.data_ptr())))
        out_r, out_p = torch.empty_like(rb), torch.empty_like(pb)
        ddh.check(L.ddh_step_backward(t._h, c_void_p(ys[k].data_ptr()), c_void_p(states[k][0].data_ptr()),
                                      c_void_p(states[k][1].data_ptr()), c_void_p(trace.data_ptr()),
                                      c_void_p(states[k + 1][0].data_ptr()), c_void_p(rb.data_ptr()),
                                      c_void_p(pb.data_ptr()), c_void_p(out_r.data_ptr()), c_void_p(out_p.data_ptr()),
                                      c_void_p(g2.data_ptr()), c_void_p(bws.data_ptr()), bws.numel() * 4))
        rb, pb = out_r, out_p
    t.sync()
    assert torch.equal(r0b, rb) and torch.equal(p0b, pb) and torch.equal(g, g2)
    with pytest.raises(ddh.DdhError):   # workspace too small
        ddh.check(L.ddh_unrolled_backward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck[k, 0] for k in range(K + 1)]),
                                          ptrs([ck[k, 1] for k in range(K + 1)]), None, c_void_p(rbar.data_ptr()),
                                          c_void_p(pbar.data_ptr()), c_void_p(r0b.data_ptr()), c_void_p(p0b.data_ptr()),
                                          c_void_p(g.data_ptr()), c_void_p(ws.data_ptr()), wsb - 4))


def test_set_params_and_the_reused_adjoint_state(mods):
    """ddh_set_params: a state whose prior/noise parameters are replaced steps bit for bit like
    a fresh state built with them; a different grid size is refused.  The autograd Function
    reuses one state per stream through it, so a call after a call with other parameters
    gives bit for bit what it gave before."""
    ddh, adjoint = mods
    K, n = 4, 32
    cfg = sy.config_adjoint(small=True, streams=1, frames=K)[0]
    ys = torch.from_numpy(sy.Stream(cfg).frames(K)[0]).cuda()
    p1 = ddh.default_params(n, 16.0, cfg.snr)
    p2 = ddh.default_params(n, 16.0, cfg.snr)
    p2.prior_sigma, p2.prior_p, p2.noise_var = 2.0 * p1.prior_sigma, 1.5, 0.5 * p1.noise_var
    a, b = ddh.Stream(p1), ddh.Stream(p2)
    a.set_params(p2)
    for k in range(K):
        a.step(ys[k])
        b.step(ys[k])
    assert torch.equal(a.phase(), b.phase()) and torch.equal(a.reflectance(), b.reflectance())
    with pytest.raises(ddh.DdhError):
        a.set_params(ddh.default_params(64, 32.0, cfg.snr))

    def grads(p):
        r0 = torch.full((n, n), 0.05, device="cuda", requires_grad=True)
        phi0 = torch.zeros((n, n), device="cuda", requires_grad=True)
        ts = [torch.tensor(float(v), dtype=torch.float64, requires_grad=True)
              for v in (p.prior_sigma, p.prior_p, p.noise_var)]
        rK, phiK = adjoint.unrolled(r0, phi0, *ts, ys, p)
        (rK.sum() + torch.sin(phiK).sum()).backward()
        return [r0.grad.clone(), phi0.grad.clone()] + [t.grad.clone() for t in ts]

    g1, g2, g3 = grads(p1), grads(p2), grads(p1)
    assert all(torch.equal(x, y) for x, y in zip(g1, g3))
    assert not torch.equal(g1[0], g2[0])


def test_autograd_stored_and_recomputed_traces_agree(mods):
    """UnrolledDDH with the forward's stored intermediates and with per-frame recomputation:
    the same gradients bit for bit."""
    ddh, adjoint = mods
    K, n = 4, 64
    cfg = sy.config_single_64(K)
    ys = torch.from_numpy(sy.Stream(cfg).frames(K)[0]).cuda()
    p = ddh.default_params(n, cfg.aperture_diam, cfg.snr)

    def grads(store):
        r0 = torch.full((n, n), 0.05, device="cuda", requires_grad=True)
        phi0 = torch.zeros((n, n), device="cuda", requires_grad=True)
        ts = [torch.tensor(float(v), dtype=torch.float64, requires_grad=True)
              for v in (p.prior_sigma, p.prior_p, p.noise_var)]
        rK, phiK = adjoint.unrolled(r0, phi0, *ts, ys, p, store_traces=store)
        (rK.sum() + torch.cos(phiK).sum()).backward()
        return [r0.grad, phi0.grad] + [t.grad for t in ts]

    a, b = grads(True), grads(False)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_unrolled_forward_dropped_frame_keeps_checkpoints(mods):
    """A non-finite frame inside the unrolled forward leaves the state, so the next checkpoint
    equals the previous one (the step writes the checkpoints itself)."""
    ddh, adjoint = mods
    K, n = 3, 32
    cfg = sy.config_adjoint(small=True, streams=1, frames=K)[0]
    ys_np = sy.Stream(cfg).frames(K)[0]
    ys_np[1, 2, 2] = np.nan
    ys = torch.from_numpy(ys_np).cuda()
    p = ddh.default_params(n, 16.0, cfg.snr)
    L = ddh.lib()
    ptrs = lambda ts: (c_void_p * len(ts))(*[c_void_p(t.data_ptr()) for t in ts])
    s = ddh.Stream(p)
    ck = torch.full((K + 1, 2, n, n), -7.0, device="cuda")
    ddh.check(L.ddh_unrolled_forward(s._h, K, ptrs([ys[k] for k in range(K)]), ptrs([ck[k, 0] for k in range(K + 1)]),
                                     ptrs([ck[k, 1] for k in range(K + 1)]), None))
    with pytest.raises(ddh.DdhError):
        s.sync()
    assert torch.equal(ck[2], ck[1]) and not torch.equal(ck[3], ck[2])
