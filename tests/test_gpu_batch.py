"""GPU: batched steps (concurrent grid-size groups, captured CUDA graph) and FFT schedules."""
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
    assert torch.cuda.is_available()
    return mod


def _cfgs():
    b = sy.config_batched(4)
    # interleaved grid sizes, so that equal sizes are not adjacent
    return [sy.config_single_64(4), b[0], sy.config_single_256(4), b[57], b[1], sy.config_single_64(4).__class__(
        **{**sy.config_single_64(4).__dict__, "stream_id": 7}), b[33], b[58]]


def _data(ddh, cfgs, frames):
    out = []
    for c in cfgs:
        ys, _ = sy.Stream(sy.with_frames(c, frames)).frames(frames)
        out.append((torch.from_numpy(ys).cuda(), ddh.default_params(c.n, c.aperture_diam, c.snr)))
    return out


def test_batch_graph_equals_solo_steps(ddh):
    data = _data(ddh, _cfgs(), 4)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        solo = [ddh.Stream(p, stream=stream) for _, p in data]
        grouped = [ddh.Stream(p, stream=stream) for _, p in data]
        g = ddh.BatchGraph(grouped)
        for f in range(4):
            for s, (ys, _) in zip(solo, data):
                s.step(ys[f])
            g.run([ys[f] for ys, _ in data])
        stream.synchronize()
        for a, b in zip(solo, grouped):
            assert torch.equal(a.phase(), b.phase()) and torch.equal(a.reflectance(), b.reflectance())
            assert b.frame_index == 4
        g.close()


def test_step_batch_interleaved_sizes_equals_solo(ddh):
    data = _data(ddh, _cfgs(), 3)
    solo = [ddh.Stream(p) for _, p in data]
    grouped = [ddh.Stream(p) for _, p in data]
    for f in range(3):
        for s, (ys, _) in zip(solo, data):
            s.step(ys[f])
        ddh.step_batch(grouped, [ys[f] for ys, _ in data])
    for a, b in zip(solo, grouped):
        assert torch.equal(a.phase(), b.phase()) and torch.equal(a.reflectance(), b.reflectance())


def test_batch_graph_argument_errors(ddh):
    data = _data(ddh, _cfgs()[:2], 1)
    sts = [ddh.Stream(p) for _, p in data]
    with pytest.raises(ddh.DdhError):
        ddh.BatchGraph([sts[0], sts[0]])
    g = ddh.BatchGraph(sts)
    buf = torch.zeros(64 * 64 + 2, dtype=torch.complex64, device="cuda")
    ptrs = (ddh.c_void_p * 2)(ddh.c_void_p(buf.data_ptr() + 8), ddh.c_void_p(data[1][0][0].data_ptr()))
    assert ddh.lib().ddh_batch_run(g._h, ptrs) == -1  # misaligned frame
    g.close()


@pytest.mark.parametrize("n", [64, 128, 256])
def test_every_fft_schedule_matches_oracle(ddh, n):
    cfg = {64: sy.config_single_64(3), 128: sy.config_batched(3)[0], 256: sy.config_single_256(3)}[n]
    ys, _ = sy.Stream(cfg).frames(3)
    p = ddh.default_params(cfg.n, cfg.aperture_diam, cfg.snr)
    prm = o.Params(n=p.n, aperture_diam=float(p.aperture_diam), lam=float(p.lam), alpha=float(p.alpha),
                   n_k=p.n_k, noise_var=float(p.noise_var), prior_p=float(p.prior_p), prior_q=float(p.prior_q),
                   prior_T=float(p.prior_T), prior_sigma=float(p.prior_sigma), r_floor=float(p.r_floor),
                   tilt_mode=p.tilt_mode, phase_block=p.phase_block)
    a = o.aperture(cfg.n, cfg.aperture_diam)
    ost = o.init_state(cfg.n)
    for y in ys:
        ost, _ = o.step(ost, y, prm)
    old = ddh.get_fft_schedule(n)
    try:
        for sched in range(ddh.fft_schedule_count(n)):
            ddh.set_fft_schedule(n, sched)
            s = ddh.Stream(p)
            for y in ys:
                s.step(torch.from_numpy(y).cuda())
            s.sync()
            phi = s.phase().cpu().numpy().astype(np.float64)
            r = s.reflectance().cpu().numpy().astype(np.float64)
            assert np.linalg.norm(o.wrap(phi - ost.phi)[a]) / np.linalg.norm(ost.phi[a]) < TOL, sched
            assert np.linalg.norm(r - ost.r) / np.linalg.norm(ost.r) < TOL, sched
    finally:
        ddh.set_fft_schedule(n, old)
    with pytest.raises(ddh.DdhError):
        ddh.set_fft_schedule(n, ddh.fft_schedule_count(n))


def test_autotune_small(ddh, tmp_path):
    """The tuner on a reduced search (128^2: FFT schedules, two staged chunks, the path at two
    batch sizes) writes a table whose winners it leaves selected and that apply() restores."""
    from paper_2305_03284_gb300 import autotune
    L = ddh.lib()
    old_s, old_c = ddh.get_fft_schedule(128), L.ddh_get_staged_chunk(128)
    try:
        out = str(tmp_path / "t.json")
        table = autotune.tune(path=out, sizes=(128,), batch_sizes=(1, 4), big={128: 4}, chunks=(2, 4),
                              schedule_streams={128: 2}, persistent_mix=False)
        row = table["128"]
        assert 0 <= row["schedule"] < ddh.fft_schedule_count(128)
        assert row["staged_chunk"] in (2, 4) and set(row["path_us_per_step"]) == {"1", "4"}
        assert ddh.get_fft_schedule(128) == row["schedule"]
        assert L.ddh_get_staged_chunk(128) == row["staged_chunk"]
        ddh.set_fft_schedule(128, old_s)
        L.ddh_set_staged_chunk(128, 3)
        assert autotune.apply(out)["128"]["staged_chunk"] == row["staged_chunk"]
        assert L.ddh_get_staged_chunk(128) == row["staged_chunk"] and ddh.get_fft_schedule(128) == row["schedule"]
        start = row["staged_from_streams"]
        assert autotune.recommend_path(128, 1000, out) == (2 if start is not None else 1)
        assert autotune.recommend_path(512, 3, out) == 0
        assert L.ddh_set_staged_chunk(64, 4) == -1 and L.ddh_set_staged_chunk(256, 65) == -1
    finally:
        ddh.set_fft_schedule(128, old_s)
        L.ddh_set_staged_chunk(128, old_c)


@pytest.mark.parametrize("n_k", [1, 2])
def test_persistent_staged_launch_equals_chained_launches(ddh, n_k):
    """A batch whose staged streams (128^2, 256^2 and 512^2 runs, with a cluster-kernel stream
    between them) run as one persistent launch per step gives, bit for bit, what the chained
    stage launches give -- by ddh_step_batch and through a captured graph."""
    from synth import ddh_synth as sy
    L = ddh.lib()
    b = sy.config_batched(3)
    cfgs = [b[0], b[1], b[2], sy.config_single_256(3), b[30], sy.config_single_256(3), b[56], b[57]]
    paths = [2, 2, 2, 2, 1, 2, 0, 0]
    data = []
    for c, pa in zip(cfgs, paths):
        ys, _ = sy.Stream(sy.with_frames(c, 3)).frames(3)
        data.append((torch.from_numpy(ys).cuda(), ddh.default_params(c.n, c.aperture_diam, c.snr, exec_path=pa,
                                                                     n_k=n_k)))
    old = L.ddh_get_staged_persistent()
    results = {}
    try:
        for mode in (0, 1):
            assert L.ddh_set_staged_persistent(mode) == 0
            direct = [ddh.Stream(p) for _, p in data]
            graphed = [ddh.Stream(p) for _, p in data]
            g = ddh.BatchGraph(graphed)
            for f in range(3):
                ys = [y[f] for y, _ in data]
                ddh.step_batch(direct, ys)
                g.run(ys)
            torch.cuda.synchronize()
            for s_ in direct + graphed:
                s_.sync()
            results[mode] = [(s_.phase().clone(), s_.reflectance().clone()) for s_ in direct + graphed]
            g.close()
    finally:
        L.ddh_set_staged_persistent(old)
    for (p0, r0), (p1, r1) in zip(results[0], results[1]):
        assert torch.equal(p0, p1) and torch.equal(r0, r1)
    # direct and graph agree too
    k = len(data)
    for i in range(k):
        assert torch.equal(results[1][i][0], results[1][k + i][0])
    assert L.ddh_set_staged_persistent(2) == -1
