"""GPU tile-phase prior and sigma^2 M-step against the FP64 oracle (the post-step kernel and
the step kernel's side outputs)."""
import numpy as np
import pytest
import torch

from oracle import ddh_oracle as o
from synth import ddh_synth as sy
from test_gpu_parity import TOL, cu, make, np32, oracle_params, rel_l2, rel_l2_phase

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddh():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import ddh as mod
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return mod


CASES = [  # (phase_block, phase_prior, noise_update)
    (2, 20.0, 0), (4, 60.0, 0), (2, 20.0, 1), (1, 0.0, 1), (4, 0.0, 1),
]


@pytest.mark.parametrize("block,lam,upd", CASES)
def test_teacher_forced_parity_64(ddh, block, lam, upd):
    """Every frame starts both sides from the oracle's state (r, phi and the sigma^2 estimate,
    rounded to float32); the one-frame map agrees along a 40-frame trajectory."""
    from dataclasses import replace
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 40, phase_block=block, phase_prior=lam, noise_update=upd)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    worst = [0.0, 0.0, 0.0]
    for i in range(40):
        r32, p32 = ost.r.astype(np.float32), ost.phi.astype(np.float32)
        nv32 = np.float32(ost.noise_var if ost.noise_var is not None else p.noise_var)
        s.set_params(ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr, phase_block=block, phase_prior=lam,
                                        noise_update=upd, noise_var=float(nv32)))
        s.set_state(cu(r32), cu(p32), i)
        s.step(cu(ys[i]))
        start = o.State(r=r32.astype(np.float64), phi=p32.astype(np.float64), n=i, noise_var=float(nv32))
        nxt, _ = o.step(start, ys[i], replace(prm, noise_var=float(nv32)))
        worst[0] = max(worst[0], rel_l2_phase(np32(s.phase()), nxt.phi, a))
        worst[1] = max(worst[1], rel_l2(np32(s.reflectance()), nxt.r))
        if upd:
            worst[2] = max(worst[2], abs(s.noise_estimate() - nxt.noise_var) / nxt.noise_var)
        ost, _ = o.step(ost, ys[i], prm)
    print(f"G {block} lam {lam} noise {upd}: phi {worst[0]:.2e} r {worst[1]:.2e} sigma^2 {worst[2]:.2e}")
    assert worst[0] < TOL and worst[1] < TOL and worst[2] < TOL, worst


@pytest.mark.parametrize("block,lam,upd", [(2, 20.0, 1), (4, 60.0, 1)])
def test_free_running_parity_64(ddh, block, lam, upd):
    """Free-running, 100 frames (tiled phase, so the iteration contracts): phase, reflectance,
    Strehl trace and the sigma^2 estimate against the oracle's own trajectory."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 100, phase_block=block, phase_prior=lam, noise_update=upd)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    gS, oS, gnv, onv = [], [], [], []
    for i in range(100):
        s.step(cu(ys[i]))
        gS.append(s.strehl(cu(ph[i].astype(np.float32))))
        gnv.append(s.noise_estimate())
        ost, _ = o.step(ost, ys[i], prm)
        oS.append(o.strehl(ost.phi, ph[i], a))
        onv.append(ost.noise_var)
    e = (rel_l2_phase(np32(s.phase()), ost.phi, a), rel_l2(np32(s.reflectance()), ost.r),
         rel_l2(np.array(gS), np.array(oS)), rel_l2(np.array(gnv), np.array(onv)))
    print(f"100 frames G {block} lam {lam}: phi {e[0]:.2e} r {e[1]:.2e} Strehl {e[2]:.2e} sigma^2 {e[3]:.2e}")
    assert max(e) < TOL, e


def test_prior_256_one_frame(ddh):
    """256^2 (16-CTA clusters, the largest tile box): one frame from a seeded state."""
    cfg = sy.config_adjoint(streams=1, frames=2)[0]
    st, ys, ph, p = make(ddh, cfg, 2, phase_block=2, phase_prior=20.0, noise_update=1)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    ost = o.init_state(cfg.n)
    ost, _ = o.step(ost, ys[0], prm)
    r32, p32 = ost.r.astype(np.float32), ost.phi.astype(np.float32)
    from dataclasses import replace
    nv = float(np.float32(ost.noise_var))
    q = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr, phase_block=2, phase_prior=20.0, noise_update=1,
                           noise_var=nv)
    s = ddh.Stream(q)
    s.set_state(cu(r32), cu(p32), 1)
    s.step(cu(ys[1]))
    nxt, _ = o.step(o.State(r=r32.astype(np.float64), phi=p32.astype(np.float64), n=1, noise_var=nv), ys[1],
                    replace(prm, noise_var=nv))
    e = (rel_l2_phase(np32(s.phase()), nxt.phi, a), rel_l2(np32(s.reflectance()), nxt.r),
         abs(s.noise_estimate() - nxt.noise_var) / nxt.noise_var)
    assert max(e) < TOL, e


def test_dropped_frame_leaves_phase_and_sigma2(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 3, phase_block=2, phase_prior=20.0, noise_update=1)
    s = ddh.Stream(p)
    s.step(cu(ys[0]))
    s.sync()
    phi0, r0, nv0 = np32(s.phase()), np32(s.reflectance()), s.noise_estimate()
    bad = ys[1].copy()
    bad[3, 3] = np.nan
    s.step(cu(bad))
    with pytest.raises(ddh.DdhError):
        s.sync()
    assert np.array_equal(np32(s.phase()), phi0) and np.array_equal(np32(s.reflectance()), r0)
    assert s.noise_estimate() == nv0


def test_checkpoint_carries_the_sigma2_estimate(ddh):
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 6, noise_update=1)
    s = ddh.Stream(p)
    for i in range(3):
        s.step(cu(ys[i]))
    blob = s.save()
    nv = s.noise_estimate()
    assert nv != float(np.float32(p.noise_var))
    t = ddh.Stream(p)
    t.load(blob)
    assert t.noise_estimate() == nv
    for i in range(3, 6):
        s.step(cu(ys[i]))
        t.step(cu(ys[i]))
    assert np.array_equal(np32(s.phase()), np32(t.phase())) and s.noise_estimate() == t.noise_estimate()


def test_refused_where_unsupported(ddh):
    """The adjoint refuses the post-step M-steps; so do a prior without tiles, with n_k > 1, or
    whose tile box exceeds the post kernel's 128 x 128 (a 512 px pupil in 2x2 tiles)."""
    cfg = sy.config_single_64()
    st, ys, ph, p = make(ddh, cfg, 1, noise_update=1)
    for over in ({"phase_prior": 1.0}, {"phase_prior": 1.0, "phase_block": 2, "n_k": 2},
                 {"phase_sweeps": 17}, {"noise_update": 2}, {"phase_prior": -1.0}):
        with pytest.raises(ddh.DdhError):
            ddh.Stream(ddh.default_params(64, 32.0, 10.0, **over))
    with pytest.raises(ddh.DdhError):
        ddh.Stream(ddh.default_params(512, 512.0, 10.0, phase_block=2, phase_prior=5.0))
    s = ddh.Stream(p)
    L = ddh.lib()
    z = torch.zeros((64, 64), device="cuda")
    tr = torch.zeros(L.ddh_trace_floats(64), device="cuda")
    g = torch.zeros(3, device="cuda")
    y = cu(ys[0])
    args = [s._h] + [ddh.c_void_p(t.data_ptr()) for t in (y, z, z, tr, z, z, z, z, z, g)]
    assert L.ddh_step_backward_noalloc(*args) == -1


def test_batches_and_service_equal_solo_steps_with_the_post_step_m_steps(ddh):
    """Streams with the tile-phase prior and/or the sigma^2 M-step inside a batch (mixed with
    plain streams and grid sizes), in a captured graph and in the service: every stream's phi,
    r and sigma^2 equal its solo run bit for bit."""
    from paper_2305_03284_gb300 import serve
    cfgs = [sy.config_single_64(), sy.config_single_256(6), sy.config_batched(6)[0], sy.config_single_64()]
    overs = [{"phase_block": 2, "phase_prior": 20.0, "noise_update": 1},
             {"phase_block": 2, "phase_prior": 10.0},
             {"noise_update": 1},
             {}]
    data = [make(ddh, c, 6, **o_) for c, o_ in zip(cfgs, overs)]
    solo = [ddh.Stream(d[3]) for d in data]
    for f in range(6):
        for s_, d in zip(solo, data):
            s_.step(cu(d[1][f]))
    batch = [ddh.Stream(d[3]) for d in data]
    graph = [ddh.Stream(d[3]) for d in data]
    g = ddh.BatchGraph(graph)
    for f in range(6):
        ys = [cu(d[1][f]) for d in data]
        ddh.step_batch(batch, ys)
        g.run(ys)
    torch.cuda.synchronize()
    for k, s1 in enumerate(solo):
        for s2 in (batch[k], graph[k]):
            assert torch.equal(s1.phase(), s2.phase()), k
            assert torch.equal(s1.reflectance(), s2.reflectance()), k
            assert s1.noise_estimate() == s2.noise_estimate(), k
    g.close()
    svc = serve.NativeService(mem_budget_bytes=1 << 34)
    for i, d in enumerate(data):
        svc.admit(i, d[3])
    frames = [cu(d[1]) for d in data]
    rng = np.random.default_rng(9)
    arrivals = sorted((float(t), i, frames[i][k]) for i in range(len(data))
                      for k, t in enumerate(np.cumsum(rng.exponential(1e-4, 6))))
    assert len(svc.drive(arrivals)) == 24
    for k, s1 in enumerate(solo):
        assert torch.equal(s1.phase(), svc.phase(k)), k
        assert torch.equal(s1.reflectance(), svc.reflectance(k)), k
    svc.close()


@pytest.mark.parametrize("n,frames,over", [
    (256, 30, {"phase_block": 2, "phase_prior": 10.0, "noise_update": 1}),
    (512, 10, {"phase_block": 2, "phase_prior": 20.0, "noise_update": 1}),
    (256, 4, {"noise_update": 1}),
])
def test_staged_kernels_with_the_post_step_m_steps(ddh, n, frames, over):
    """The L2-staged kernels' side outputs (tile sums, residual and posterior-variance partials
    per 8-row / 8-column block) feed the same post-step kernel: free-running against the oracle
    (phase, reflectance, Strehl trace and the sigma^2 estimate); per-pixel phase only over a few
    frames, where the iteration does not contract."""
    from paper_2305_03284_gb300 import _lib
    cfg = sy.config_single_256() if n == 256 else sy.config_batched(frames=frames)[56]
    assert cfg.n == n
    st, ys, ph, p = make(ddh, cfg, frames, exec_path=_lib.DDH_PATH_STAGED, **over)
    ph = ph.astype(np.float32).astype(np.float64)
    prm = oracle_params(p)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    s = ddh.Stream(p)
    ost = o.init_state(cfg.n)
    gS, oS, gnv, onv = [], [], [], []
    for i in range(frames):
        s.step(cu(ys[i]))
        gS.append(s.strehl(cu(ph[i].astype(np.float32))))
        gnv.append(s.noise_estimate())
        ost, _ = o.step(ost, ys[i], prm)
        oS.append(o.strehl(ost.phi, ph[i], a))
        onv.append(ost.noise_var)
    e = (rel_l2_phase(np32(s.phase()), ost.phi, a), rel_l2(np32(s.reflectance()), ost.r),
         rel_l2(np.array(gS), np.array(oS)), rel_l2(np.array(gnv), np.array(onv)))
    print(f"staged {n}^2 {over}, {frames} frames: phi {e[0]:.2e} r {e[1]:.2e} Strehl {e[2]:.2e} sigma^2 {e[3]:.2e}")
    assert max(e) < TOL, e
    s.close()


def test_staged_batches_and_graphs_equal_solo_steps_with_the_post_step_m_steps(ddh):
    """Staged streams with the prior and/or the sigma^2 M-step beside plain staged and cluster
    streams, in one batch and in a captured graph: phi, r and sigma^2 equal the solo runs bit
    for bit."""
    from paper_2305_03284_gb300 import _lib
    S = _lib.DDH_PATH_STAGED
    cfgs = [sy.config_single_256(6), sy.config_single_256(6), sy.config_batched(6)[56], sy.config_single_256(6)]
    overs = [{"phase_block": 2, "phase_prior": 10.0, "noise_update": 1, "exec_path": S},
             {"exec_path": S},
             {"phase_block": 2, "phase_prior": 20.0, "exec_path": S},
             {"phase_block": 2, "phase_prior": 10.0, "noise_update": 1}]
    data = [make(ddh, c, 6, **o_) for c, o_ in zip(cfgs, overs)]
    solo = [ddh.Stream(d[3]) for d in data]
    for f in range(6):
        for s_, d in zip(solo, data):
            s_.step(cu(d[1][f]))
    batch = [ddh.Stream(d[3]) for d in data]
    graph = [ddh.Stream(d[3]) for d in data]
    g = ddh.BatchGraph(graph)
    for f in range(6):
        ys = [cu(d[1][f]) for d in data]
        ddh.step_batch(batch, ys)
        g.run(ys)
    torch.cuda.synchronize()
    for k, s1 in enumerate(solo):
        for s2 in (batch[k], graph[k]):
            assert torch.equal(s1.phase(), s2.phase()), k
            assert torch.equal(s1.reflectance(), s2.reflectance()), k
            assert s1.noise_estimate() == s2.noise_estimate(), k
    g.close()
