"""GPU parity: libddh's CUDA path against the FP64 oracle on seeded synthetic streams.

Tolerance: relative L2 error 2e-5 on phi (wrapped difference over the aperture), r and the
per-frame Strehl ratio, the figure the design targets for complex64/FP32 arithmetic against
an FP64 reference.  Every call goes through the C ABI (the ctypes binding).
"""
import math

import numpy as np
import pytest
import torch

from oracle import ddh_oracle as o
from synth import ddh_synth as sy

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def ddh():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import ddh as mod
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return mod


def oracle_params(p) -> o.Params:
    """The oracle runs on exactly the (float32) parameter values the library received."""
    return o.Params(n=p.n, aperture_diam=float(p.aperture_diam), lam=float(p.lam), alpha=float(p.alpha),
                    n_k=p.n_k, noise_var=float(p.noise_var), prior_p=float(p.prior_p),
                    prior_q=float(p.prior_q), prior_T=float(p.prior_T), prior_sigma=float(p.prior_sigma),
                    r_floor=float(p.r_floor), tilt_mode=p.tilt_mode, phase_block=p.phase_block,
                    phase_prior=float(p.phase_prior), phase_sweeps=p.phase_sweeps or 2,
                    noise_update=p.noise_update)


def rel_l2(a, b):
    a = np.asarray(a)
    a = a.astype(np.complex128 if np.iscomplexobj(a) else np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_l2_phase(a, b, ap):
    d = o.wrap(np.asarray(a, np.float64) - b)[ap]
    return float(np.linalg.norm(d) / np.linalg.norm(b[ap]))


def cu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def np32(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def make(ddh, cfg, frames, **over):
    st = sy.Stream(sy.with_frames(cfg, frames))
    ys, ph = st.frames(frames)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr, **over)
    return st, ys, ph, p


# ------------------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n", [64, 128, 256])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2_matches_oracle(ddh, n, inverse):
    rng = np.random.default_rng(n + inverse)
    x = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    got = np32(ddh.fft2(cu(x), inverse=inverse))
    ref = (o.ifft2u if inverse else o.fft2u)(x.astype(np.complex128))
    assert rel_l2(got, ref) < 2e-6


def test_fft2_in_place(ddh):
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))).astype(np.complex64)
    t = cu(x)
    ddh.fft2(t, out=t)
    assert rel_l2(np32(t), o.fft2u(x.astype(np.complex128))) < 2e-6


# ----------------------------------------------------------------- one frame, stage by stage
def test_first_frame_intermediates_64(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 2)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    s.step(cu(ys[0]))
    tr = s.step_trace(cu(ys[1]))  # second frame: nonzero phase, tilt and r history
    st0, _ = o.step(o.init_state(cfg.n), ys[0], prm)
    _, ot = o.step(st0, ys[1], prm)
    stats = np32(tr["stats"])
    assert abs(stats[0] + 1j * stats[1] - ot.stats["mean"]) < 1e-5 / ot.stats["scale"]
    assert math.isclose(stats[2], ot.stats["scale"], rel_tol=1e-5)
    assert abs(stats[3] - ot.stats["tx"]) < 1e-6 and abs(stats[4] - ot.stats["ty"]) < 1e-6
    assert rel_l2(np32(tr["b"]), ot.b) < TOL
    assert rel_l2(np32(tr["r_init"]), ot.r_init) < TOL
    assert rel_l2(np32(tr["mu"]), ot.mu) < TOL
    assert rel_l2(np32(tr["s"]), ot.s) < TOL
    assert rel_l2(np32(tr["z"])[a], ot.z[a]) < TOL


# ------------------------------------------------------------------- multi-frame parity
def _run_free(ddh, p, ys, ph, with_strehl=True):
    s = ddh.Stream(p)
    phis, rs, S = [], [], []
    for i in range(len(ys)):
        s.step(cu(ys[i]))
        phis.append(np32(s.phase()))
        rs.append(np32(s.reflectance()))
        if with_strehl:
            S.append(s.strehl(cu(ph[i].astype(np.float32))))
    s.sync()
    return np.array(phis), np.array(rs), np.array(S)


def _run_oracle(prm, ys, ph):
    a = o.aperture(prm.n, prm.aperture_diam)
    st = o.init_state(prm.n)
    phis, rs, S = [], [], []
    for i in range(len(ys)):
        st, _ = o.step(st, ys[i], prm)
        phis.append(st.phi)
        rs.append(st.r)
        S.append(o.strehl(st.phi, ph[i], a))
    return np.array(phis), np.array(rs), np.array(S)


def test_free_running_parity_64_100_frames_tiled_phase(ddh):
    """Parity bar (phi, r, Strehl within 2e-5 after 100 frames): 64x64 stream (32 px pupil,
    D/r0 10, 0.5 px/frame, SNR 10), 100 free-running frames of one EM iteration each, phase
    held constant on 2x2 tiles.  With
    tiles the iteration contracts (the oracle's own 1e-7 perturbations decay), so GPU and
    oracle trajectories can agree after 100 frames."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 100, phase_block=2)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, gS = _run_free(ddh, p, ys, ph)
    ophi, orr, oS = _run_oracle(prm, ys, ph)
    e = (rel_l2_phase(gphi[-1], ophi[-1], a), rel_l2(gr[-1], orr[-1]), rel_l2(gS, oS))
    print(f"100 frames, tiled phase: phi {e[0]:.2e}, r {e[1]:.2e}, Strehl trace {e[2]:.2e}")
    assert e[0] < TOL and e[1] < TOL and e[2] < TOL, e
    assert np.all(gphi[:, ~a] == 0.0)


@pytest.mark.parametrize("stream", ["paper", "bench"])
def test_free_running_parity_256_100_frames_tiled_phase_both_paths(ddh, stream):
    """The same parity bar at the realistic size: 100 free-running 256^2 frames with the phase
    held constant on 2x2 tiles, on the cluster kernel and on the L2-staged kernels, against one
    FP64 oracle trajectory: the paper's Sec. 5.A stream (bar chart, D/r0 10, SNR 10 dB; sigma_r
    0.03, alpha 0.0125) and the benchmark's stream (D/r0 15, 1 px/frame, SNR 5; defaults)."""
    from paper_2305_03284_gb300 import _lib
    frames = 100
    if stream == "paper":
        cfg = sy.config_paper_256(0, frames)
        mk = lambda path: ddh.tracking_params(256, 128.0, 10.0, phase_prior=0.0, exec_path=path)
    else:
        cfg = sy.with_frames(sy.config_single_256(), frames)
        mk = lambda path: ddh.default_params(256, 128.0, 5.0, phase_block=2, exec_path=path)
    ys, ph = sy.Stream(cfg).frames(frames)
    ph = ph.astype(np.float32).astype(np.float64)
    a = o.aperture(256, 128.0)
    ophi, orr, oS = _run_oracle(oracle_params(mk(_lib.DDH_PATH_CLUSTER)), ys, ph)
    for path in (_lib.DDH_PATH_CLUSTER, _lib.DDH_PATH_STAGED):
        s = ddh.Stream(mk(path))
        yd = cu(ys)
        gS = []
        for k in range(frames):
            s.step(yd[k])
            gS.append(s.strehl(cu(ph[k].astype(np.float32))))
        e = (rel_l2_phase(np32(s.phase()), ophi[-1], a), rel_l2(np32(s.reflectance()), orr[-1]), rel_l2(gS, oS))
        s.close()
        print(f"256^2 {stream} stream, path {path}, 100 frames, tiled phase: phi {e[0]:.2e}, r {e[1]:.2e}, "
              f"Strehl trace {e[2]:.2e}")
        assert e[0] < TOL and e[1] < TOL and e[2] < TOL, (path, e)


def test_free_running_parity_64_per_pixel_phase_short(ddh):
    """Per-pixel phase: the iteration amplifies any perturbation (the FP64 oracle against
    itself grows 1e-7 to O(1) within ~30 frames), so free-running agreement is checked over
    the first 8 frames, and frame-by-frame agreement over 100 frames teacher-forced below."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 8)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, gS = _run_free(ddh, p, ys, ph)
    ophi, orr, oS = _run_oracle(prm, ys, ph)
    assert rel_l2_phase(gphi[-1], ophi[-1], a) < TOL
    assert rel_l2(gr[-1], orr[-1]) < TOL
    assert rel_l2(gS, oS) < TOL


@pytest.mark.parametrize("block", [1, 2])
def test_teacher_forced_parity_64_100_frames(ddh, block):
    """Each frame starts the GPU from the oracle's previous state (rounded to float32): the
    one-step map agrees to the tolerance along the whole 100-frame trajectory."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 100, phase_block=block)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    worst_phi = worst_r = 0.0
    for i in range(100):
        r32, p32 = ost.r.astype(np.float32), ost.phi.astype(np.float32)
        s.set_state(cu(r32), cu(p32), i)
        s.step(cu(ys[i]))
        nxt, _ = o.step(o.State(r=r32.astype(np.float64), phi=p32.astype(np.float64), n=i), ys[i], prm)
        worst_phi = max(worst_phi, rel_l2_phase(np32(s.phase()), nxt.phi, a))
        worst_r = max(worst_r, rel_l2(np32(s.reflectance()), nxt.r))
        ost, _ = o.step(ost, ys[i], prm)
    assert worst_phi < TOL and worst_r < TOL, (worst_phi, worst_r)


@pytest.mark.parametrize("which", ["128", "256", "256-tiled"])
def test_parity_larger_grids(ddh, which):
    if which.startswith("256"):
        cfg = sy.config_single_256(frames=6)
    else:
        cfg = sy.config_batched(frames=6)[0]  # a 128^2 stream of the batched workload
    st, ys, ph, p = make(ddh, cfg, 6, phase_block=2 if which.endswith("tiled") else 1)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, gS = _run_free(ddh, p, ys, ph)
    ophi, orr, oS = _run_oracle(prm, ys, ph)
    assert rel_l2_phase(gphi[-1], ophi[-1], a) < TOL
    assert rel_l2(gr[-1], orr[-1]) < TOL
    assert rel_l2(gS, oS) < TOL


def test_parity_256_every_frame_long_run(ddh):
    """The benchmark's workload and launch configuration (single 256^2 stream, one launch per
    frame) over 300 free-running frames; at every frame the oracle takes one step from the
    GPU's own state, and phi, r and the frame's Strehl ratio (GPU Strehl kernel against the
    oracle's Strehl of its one-step phase) are compared."""
    cfg = sy.config_single_256(frames=300)
    st = sy.Stream(cfg)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    worst = [0.0, 0.0, 0.0]
    r0 = np.zeros((256, 256))
    p0 = np.zeros((256, 256))
    for i in range(300):
        y, ph = st.frame(i)
        s.step(cu(y))
        nxt, _ = o.step(o.State(r=r0, phi=p0, n=i), y, prm)
        gphi = np32(s.phase()).astype(np.float64)
        gr = np32(s.reflectance()).astype(np.float64)
        g_s = s.strehl(cu(ph.astype(np.float32)))
        o_s = o.strehl(nxt.phi, ph.astype(np.float32).astype(np.float64), a)
        e = (rel_l2_phase(gphi, nxt.phi, a), rel_l2(gr, nxt.r), abs(g_s - o_s) / o_s)
        worst = [max(w, v) for w, v in zip(worst, e)]
        assert e[0] < TOL and e[1] < TOL and e[2] < TOL, (i, e)
        r0, p0 = gr, gphi
    s.sync()
    print(f"300 frames at 256^2, worst one-step error: phi {worst[0]:.2e}, r {worst[1]:.2e}, Strehl {worst[2]:.2e}")


def test_parity_256_full_1000_frame_stream_every_tenth_frame(ddh):
    """The whole 1000-frame 256^2 stream of the benchmark workload, free-running on the GPU;
    at every tenth frame the oracle takes one step from the GPU's own state and phi, r and
    that frame's Strehl ratio are compared."""
    cfg = sy.config_single_256(frames=1000)
    st = sy.Stream(cfg)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    worst = [0.0, 0.0, 0.0]
    for i in range(1000):
        y, ph = st.frame(i)
        check = i % 10 == 9
        if check:
            r0 = np32(s.reflectance()).astype(np.float64)
            p0 = np32(s.phase()).astype(np.float64)
        s.step(cu(y))
        if check:
            nxt, _ = o.step(o.State(r=r0, phi=p0, n=i), y, prm)
            g_s = s.strehl(cu(ph.astype(np.float32)))
            o_s = o.strehl(nxt.phi, ph.astype(np.float32).astype(np.float64), a)
            e = (rel_l2_phase(np32(s.phase()), nxt.phi, a), rel_l2(np32(s.reflectance()), nxt.r), abs(g_s - o_s) / o_s)
            worst = [max(w, v) for w, v in zip(worst, e)]
            assert e[0] < TOL and e[1] < TOL and e[2] < TOL, (i, e)
    s.sync()
    print(f"1000 frames at 256^2, every tenth frame: phi {worst[0]:.2e}, r {worst[1]:.2e}, Strehl {worst[2]:.2e}")


@pytest.mark.parametrize("over", [{"n_k": 2}, {"n_k": 3}, {"n_k": 4}, {"n_k": 8}, {"tilt_mode": 0},
                                  {"aperture_diam": 31.3},
                                  {"prior_sigma": 0.05, "prior_p": 1.5}, {"phase_block": 4},
                                  {"phase_block": 2, "n_k": 2}])
def test_parity_variants_64(ddh, over):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 12, **over)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, float(p.aperture_diam))
    gphi, gr, _ = _run_free(ddh, p, ys[:5], ph[:5], with_strehl=False)
    ophi, orr, _ = _run_oracle(prm, ys[:5], ph[:5])
    assert rel_l2_phase(gphi[-1], ophi[-1], a) < TOL
    assert rel_l2(gr[-1], orr[-1]) < TOL
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    for i in range(12):
        r32, p32 = ost.r.astype(np.float32), ost.phi.astype(np.float32)
        s.set_state(cu(r32), cu(p32), i)
        s.step(cu(ys[i]))
        nxt, _ = o.step(o.State(r=r32.astype(np.float64), phi=p32.astype(np.float64), n=i), ys[i], prm)
        assert rel_l2_phase(np32(s.phase()), nxt.phi, a) < TOL
        assert rel_l2(np32(s.reflectance()), nxt.r) < TOL
        ost = nxt


def test_empty_aperture(ddh):
    """A pupil that contains no pixel: phase stays zero, r follows the prior-only EM."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 3, aperture_diam=0.5)
    prm = oracle_params(p)
    gphi, gr, _ = _run_free(ddh, p, ys, ph, with_strehl=False)
    ophi, orr, _ = _run_oracle(prm, ys, ph)
    assert np.all(gphi == 0.0)
    assert rel_l2(gr[-1], orr[-1]) < TOL


def test_strehl_matches_oracle(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 1)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    rng = np.random.default_rng(3)
    est = np.where(a, ph[0] + 0.3 * rng.standard_normal(ph[0].shape), 0.0).astype(np.float32)
    s.set_state(cu(np.zeros((64, 64), np.float32)), cu(est), 0)
    got = s.strehl(cu(ph[0].astype(np.float32)))
    ref = o.strehl(est.astype(np.float64), ph[0].astype(np.float32).astype(np.float64), a)
    assert abs(got - ref) < 1e-5 * ref
    s.set_state(cu(np.zeros((64, 64), np.float32)), cu(ph[0].astype(np.float32) * a), 0)
    assert abs(s.strehl(cu(ph[0].astype(np.float32))) - 1.0) < 1e-5


@pytest.mark.parametrize("n", [256, 512])
def test_strehl_matches_oracle_large_grids(ddh, n):
    """The Strehl evaluation at 256^2 (cluster kernel) and 512^2 (row and column launches through
    the staged stream's scratch) against the oracle's, for a perturbed estimate and for the true
    phase (Strehl 1)."""
    cfg = sy.config_single_256() if n == 256 else sy.config_batched(frames=1)[56]
    assert cfg.n == n
    st, ys, ph, p = make(ddh, cfg, 1)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    rng = np.random.default_rng(5)
    est = np.where(a, ph[0] + 0.3 * rng.standard_normal(ph[0].shape), 0.0).astype(np.float32)
    zeros = cu(np.zeros((n, n), np.float32))
    s.set_state(zeros, cu(est), 0)
    got = s.strehl(cu(ph[0].astype(np.float32)))
    ref = o.strehl(est.astype(np.float64), ph[0].astype(np.float32).astype(np.float64), a)
    print(f"{n}^2 Strehl: library {got:.6f}, oracle {ref:.6f}")
    assert abs(got - ref) < 1e-5 * ref
    s.set_state(zeros, cu(ph[0].astype(np.float32) * a), 0)
    assert abs(s.strehl(cu(ph[0].astype(np.float32))) - 1.0) < 1e-5
    s.close()


# -------------------------------------------------------------------------- API behaviour
def test_batch_equals_individual_steps(ddh):
    cfgs = [sy.config_single_64(), sy.config_batched(4)[0], sy.config_single_256(4), sy.config_batched(4)[1]]
    data = [make(ddh, c, 4) for c in cfgs]
    solo = [ddh.Stream(d[3]) for d in data]
    batch = [ddh.Stream(d[3]) for d in data]
    for f in range(4):
        ys = [cu(d[1][f]) for d in data]
        for s, y in zip(solo, ys):
            s.step(y)
        ddh.step_batch(batch, ys)
    for s1, s2 in zip(solo, batch):
        assert torch.equal(s1.phase(), s2.phase())
        assert torch.equal(s1.reflectance(), s2.reflectance())
    with pytest.raises(ddh.DdhError):
        ddh.step_batch([batch[0], batch[0]], [cu(data[0][1][0])] * 2)
    ddh.step_batch([], [])


def test_step_host_equals_device(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 3)
    a, b = ddh.Stream(p), ddh.Stream(p)
    out = torch.empty((64, 64), dtype=torch.float32).pin_memory()
    for i in range(3):
        a.step(cu(ys[i]))
        b.step_host(torch.from_numpy(ys[i]).pin_memory(), out)
    assert torch.equal(a.phase().cpu(), out)
    assert b.frame_index == 3


@pytest.mark.parametrize("n", [64, 256])
def test_pipelined_host_steps_equal_device_steps(ddh, n):
    """ddh_step_host_async: every frame's phase arrives in its own pinned buffer, equal to the
    device-resident steps bitwise, with several frames in flight."""
    cfg = sy.config_single_64() if n == 64 else sy.config_single_256(frames=10)
    st, ys, ph, p = make(ddh, cfg, 10)
    a, b = ddh.Stream(p), ddh.Stream(p)
    hy = [torch.from_numpy(y).pin_memory() for y in ys]
    outs = [torch.full((n, n), -7.0, dtype=torch.float32).pin_memory() for _ in range(10)]
    tickets = [b.step_host_async(hy[i], outs[i]) for i in range(6)]
    b.host_wait(tickets[1])
    tickets += [b.step_host_async(hy[i], outs[i]) for i in range(6, 10)]
    assert tickets == list(range(10))
    b.host_wait(tickets[9])
    b.sync()
    for i in range(10):
        a.step(cu(ys[i]))
        assert torch.equal(a.phase().cpu(), outs[i]), i
    assert b.frame_index == 10
    with pytest.raises(ddh.DdhError):
        b.host_wait(10)          # not issued
    with pytest.raises(ddh.DdhError):
        b.host_wait(-1)


def test_host_step_in_place_dropped_frame(ddh):
    """A non-finite frame through the in-place host path: the pinned output receives the
    unchanged phase (as the staged copy of the kept state would), and the error surfaces."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 3)
    s = ddh.Stream(p)
    out = torch.full((64, 64), -7.0, dtype=torch.float32).pin_memory()
    s.host_wait(s.step_host_async(torch.from_numpy(ys[0]).pin_memory(), out))
    before = out.clone()
    bad = ys[1].copy()
    bad[5, 9] = np.inf
    out2 = torch.full((64, 64), -7.0, dtype=torch.float32).pin_memory()
    s.host_wait(s.step_host_async(torch.from_numpy(bad).pin_memory(), out2))
    with pytest.raises(ddh.DdhError):
        s.sync()
    assert torch.equal(out2, before) and torch.equal(s.phase().cpu(), before)


@pytest.mark.parametrize("over", [{}, {"noise_update": 1}, {"phase_block": 2, "phase_prior": 20.0}])
def test_host_steps_staged_fallbacks(ddh, over):
    """Pinned buffers take the in-place path (the kernel reads the frame and writes phi over the
    CPU-GPU link); pageable buffers, and streams whose phi a post-step kernel changes, take the
    staged copies.  Every combination equals the device-resident steps bitwise."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 6, **over)
    a, b, c = ddh.Stream(p), ddh.Stream(p), ddh.Stream(p)
    for i in range(6):
        a.step(cu(ys[i]))
        out_b = torch.full((64, 64), -7.0, dtype=torch.float32)           # pageable
        b.step_host(torch.from_numpy(ys[i]).clone(), out_b)
        out_c = torch.full((64, 64), -7.0, dtype=torch.float32).pin_memory()
        t = c.step_host_async(torch.from_numpy(ys[i]).pin_memory(), out_c)
        c.host_wait(t)
        ref = a.phase().cpu()
        assert torch.equal(ref, out_b) and torch.equal(ref, out_c), i
    c.sync()


def test_checkpoint_roundtrip(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 6)
    s = ddh.Stream(p)
    for i in range(3):
        s.step(cu(ys[i]))
    blob = s.save()
    for i in range(3, 6):
        s.step(cu(ys[i]))
    ref = s.phase().clone()
    t = ddh.Stream(p)
    t.load(blob)
    assert t.frame_index == 3
    for i in range(3, 6):
        t.step(cu(ys[i]))
    assert torch.equal(t.phase(), ref)


def test_nonfinite_frame_is_rejected_and_state_kept(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 3)
    s = ddh.Stream(p)
    s.step(cu(ys[0]))
    s.sync()
    phi0, r0 = s.phase().clone(), s.reflectance().clone()
    bad = ys[1].copy()
    bad[10, 20] = np.nan
    s.step(cu(bad))
    with pytest.raises(ddh.DdhError) as e:
        s.sync()
    assert e.value.code == -5
    assert torch.equal(s.phase(), phi0) and torch.equal(s.reflectance(), r0)
    const = np.full((64, 64), 1 + 1j, np.complex64)  # zero variance: Normalize undefined
    s.step(cu(const))
    with pytest.raises(ddh.DdhError):
        s.sync()
    s.step(cu(ys[1]))
    s.sync()
    assert not torch.equal(s.phase(), phi0)


def test_bounded_device_wait_expires_and_state_stays_usable(ddh):
    """Failure detection without a fault: a device wait that nothing completes gives up after
    its time limit and latches the timeout status, the host reads DDH_ETIMEOUT, and the same
    state then steps exactly like a fresh one."""
    import ctypes
    import time
    from paper_2305_03284_gb300._lib import DDH_EINVAL, DDH_ETIMEOUT
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 2)
    s, ref = ddh.Stream(p), ddh.Stream(p)
    t0 = time.perf_counter()
    assert ddh.lib().ddh_selftest_wait(s._h, ctypes.c_double(0.002)) == DDH_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.002
    assert ddh.lib().ddh_selftest_wait(s._h, ctypes.c_double(5.0)) == DDH_EINVAL  # limit above 1 s
    s.sync()  # the latched status was cleared by the self-test call
    for i in range(2):
        s.step(cu(ys[i]))
        ref.step(cu(ys[i]))
    assert torch.equal(s.phase(), ref.phase()) and torch.equal(s.reflectance(), ref.reflectance())


def test_argument_errors(ddh):
    p = ddh.default_params(64, 32.0, 10.0)
    s = ddh.Stream(p)
    buf = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device="cuda")
    rc = ddh.lib().ddh_step(s._h, ddh.c_void_p(buf.data_ptr() + 8))
    assert rc == -1  # misaligned frame
    for bad in ({"prior_q": 1.5}, {"n_k": 0}, {"noise_var": 0.0}, {"aperture_diam": 65.0}, {"n": 100}):
        q = ddh.default_params(64, 32.0, 10.0, **bad)
        with pytest.raises(ddh.DdhError):
            ddh.Stream(q)


# ------------------------------------------------------------------- static DH-MBIR mode
@pytest.mark.parametrize("reset_every,cycles,block", [(10, 1, 1), (200, 1, 2), (50, 2, 2)])
def test_static_mode_parity_64(ddh, reset_every, cycles, block):
    """Static DH-MBIR (Sec. 3) through the frame step: EM iterated on one frame, r reset to
    the back-projection every `reset_every` iterations (each step is one bootstrap period).
    With the per-pixel phase the static iteration first amplifies perturbations (~20x within
    ~50 iterations on the FP64 oracle itself), so it is compared within that horizon; with
    tiled phase the full 200-iteration period and two shorter periods in a row."""
    cfg = sy.config_single_64()
    st, ys, ph, _ = make(ddh, cfg, 2)
    p = ddh.static_params(cfg.n, cfg.aperture_diam, cfg.snr, reset_every, phase_block=block)
    assert (p.n_k, p.tilt_mode) == (reset_every, 0) and p.lam == 1.0 and p.alpha == 1.0
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    for _ in range(cycles):
        s.step(cu(ys[1]))
        ost, _ = o.step(ost, ys[1], prm)
    e = (rel_l2_phase(np32(s.phase()), ost.phi, a), rel_l2(np32(s.reflectance()), ost.r))
    print(f"static mode, {cycles} x {reset_every} EM iterations, G = {block}: phi {e[0]:.2e}, r {e[1]:.2e}")
    assert e[0] < TOL and e[1] < TOL, e


# -------------------------------------------------------------- 512 x 512 (L2-staged path)
@pytest.mark.parametrize("over", [{}, {"phase_block": 2}, {"n_k": 2}])
def test_parity_512_l2_staged(ddh, over):
    cfg = sy.config_batched(frames=3)[56]  # a 512^2 stream of the 64-stream workload
    assert cfg.n == 512
    st, ys, ph, p = make(ddh, cfg, 3 if not over else 2, **over)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, _ = _run_free(ddh, p, ys, ph, with_strehl=False)
    ophi, orr, _ = _run_oracle(prm, ys, ph)
    assert rel_l2_phase(gphi[-1], ophi[-1], a) < TOL
    assert rel_l2(gr[-1], orr[-1]) < TOL
    assert np.all(gphi[-1][~a] == 0.0)


def test_parity_512_free_running_30_frames_tiled_phase(ddh):
    """A 512^2 stream of the 64-stream workload (L2-staged kernels, the only path at this size)
    free-running for 30 frames with 2x2 phase tiles: phi, r and the Strehl trace against the
    FP64 oracle."""
    cfg = sy.config_batched(frames=30)[56]
    assert cfg.n == 512
    st, ys, ph, p = make(ddh, cfg, 30, phase_block=2)
    ph = ph.astype(np.float32).astype(np.float64)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, gS = _run_free(ddh, p, ys, ph)
    ophi, orr, oS = _run_oracle(oracle_params(p), ys, ph)
    e = (rel_l2_phase(gphi[-1], ophi[-1], a), rel_l2(gr[-1], orr[-1]), rel_l2(gS, oS))
    print(f"512^2, 30 free-running frames, tiled phase: phi {e[0]:.2e}, r {e[1]:.2e}, Strehl trace {e[2]:.2e}")
    assert e[0] < TOL and e[1] < TOL and e[2] < TOL, e


# ------------------------------------------- 128^2 and 256^2 on the L2-staged path (exec_path)
@pytest.mark.parametrize("which", ["128", "256", "256-tiled", "256-nk2"])
def test_parity_staged_path_smaller_grids(ddh, which):
    """The staged kernels (the throughput path of large batches) on the cluster kernel's grid
    sizes: free-running against the oracle, then teacher-forced frame by frame."""
    cfg = sy.config_single_256(frames=8) if which.startswith("256") else sy.config_batched(frames=8)[0]
    over = {"exec_path": 2}
    if which.endswith("tiled"):
        over["phase_block"] = 2
    if which.endswith("nk2"):
        over["n_k"] = 2
    st, ys, ph, p = make(ddh, cfg, 8, **over)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    gphi, gr, gS = _run_free(ddh, p, ys[:5], ph[:5])
    ophi, orr, oS = _run_oracle(prm, ys[:5], ph[:5])
    assert rel_l2_phase(gphi[-1], ophi[-1], a) < TOL
    assert rel_l2(gr[-1], orr[-1]) < TOL
    assert rel_l2(gS, oS) < TOL
    assert np.all(gphi[-1][~a] == 0.0)
    s = ddh.Stream(p)
    ost = o.State(r=orr[-1], phi=ophi[-1], n=5)
    for i in range(5, 8):
        r32, p32 = ost.r.astype(np.float32), ost.phi.astype(np.float32)
        s.set_state(cu(r32), cu(p32), i)
        s.step(cu(ys[i]))
        nxt, _ = o.step(o.State(r=r32.astype(np.float64), phi=p32.astype(np.float64), n=i), ys[i], prm)
        assert rel_l2_phase(np32(s.phase()), nxt.phi, a) < TOL
        assert rel_l2(np32(s.reflectance()), nxt.r) < TOL
        ost = nxt


def test_staged_and_cluster_paths_agree_and_batches_keep_each_path(ddh):
    """A 256^2 stream on either path gives the same estimate within the tolerance; in a batch
    that mixes both paths (and a 512^2 and a 128^2 stream), every stream equals its solo run
    bit for bit."""
    cfgs = [sy.config_single_256(4), sy.config_single_256(4), sy.config_batched(4)[0], sy.config_batched(4)[56]]
    paths = [1, 2, 2, 0]
    data = [make(ddh, c, 4, exec_path=pa) for c, pa in zip(cfgs, paths)]
    solo = [ddh.Stream(d[3]) for d in data]
    batch = [ddh.Stream(d[3]) for d in data]
    for f in range(4):
        ys = [cu(d[1][f]) for d in data]
        for s_, y in zip(solo, ys):
            s_.step(y)
        ddh.step_batch(batch, ys)
    for s1, s2 in zip(solo, batch):
        assert torch.equal(s1.phase(), s2.phase())
        assert torch.equal(s1.reflectance(), s2.reflectance())
    a = o.aperture(256, 128.0)
    p_cl, p_st = np32(solo[0].phase()).astype(np.float64), np32(solo[1].phase()).astype(np.float64)
    assert rel_l2_phase(p_st, p_cl, a) < TOL
    assert rel_l2(np32(solo[1].reflectance()), np32(solo[0].reflectance()).astype(np.float64)) < TOL
    # the path is fixed for the state's lifetime
    with pytest.raises(ddh.DdhError):
        solo[0].set_params(ddh.default_params(256, 128.0, 5.0, exec_path=2))
    # the staged path has no trace output and no adjoint
    tr = torch.zeros(ddh.lib().ddh_trace_floats(256), device="cuda")
    assert ddh.lib().ddh_step_trace(solo[1]._h, ddh.c_void_p(cu(data[1][1][0]).data_ptr()),
                                    ddh.c_void_p(tr.data_ptr())) == -1
    with pytest.raises(ddh.DdhError):
        ddh.Stream(ddh.default_params(64, 32.0, 10.0, exec_path=2))
    with pytest.raises(ddh.DdhError):
        ddh.Stream(ddh.default_params(512, 256.0, 10.0, exec_path=1))


def test_512_rejects_nonfinite_frame(ddh):
    cfg = sy.config_batched(frames=2)[56]
    st, ys, ph, p = make(ddh, cfg, 2)
    s = ddh.Stream(p)
    s.step(cu(ys[0]))
    s.sync()
    phi0 = s.phase().clone()
    bad = ys[1].copy()
    bad[3, 5] = np.inf
    s.step(cu(bad))
    with pytest.raises(ddh.DdhError):
        s.sync()
    assert torch.equal(s.phase(), phi0)
