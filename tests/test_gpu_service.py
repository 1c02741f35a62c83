"""GPU: the continuous-batching service on libddh."""
import numpy as np
import pytest
import torch

from synth import ddh_synth as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2305_03284_gb300 import build
    build.build()
    from paper_2305_03284_gb300 import ddh, serve
    assert torch.cuda.is_available()
    return ddh, serve


def _sensors():
    b = sy.config_batched(6)
    return [sy.config_single_256(6), b[0], b[40], sy.config_single_64(6), b[1], b[41]]


def test_native_background_loop_delivers_in_order(mods):
    """Frames submitted while the library thread runs complete in order, and the sensor's
    phase then equals a plain stream's after the same frames."""
    ddh, serve = mods
    cfg = sy.config_single_64(4)
    frames = torch.from_numpy(sy.Stream(cfg).frames(4)[0]).cuda()
    svc = serve.NativeService(mem_budget_bytes=1 << 32)
    svc.admit(7, ddh.default_params(64, 32.0, 10.0))
    ref = ddh.Stream(ddh.default_params(64, 32.0, 10.0))
    svc.start()
    done = []
    try:
        for k in range(4):
            svc.submit(7, frames[k], tag=k)
        t0 = svc.now()
        while len(done) < 4 and svc.now() - t0 < 30:
            done.extend(svc.poll())
    finally:
        svc.stop()
    for k in range(4):
        ref.step(frames[k])
    assert [c[0] for c in done] == [0, 1, 2, 3] and [c[2] for c in done] == [1, 2, 3, 4]
    assert torch.equal(svc.phase(7), ref.phase())
    svc.close()


def test_native_staged_sensors_alone_equal_in_mix(mods):
    """Sensors on the staged kernels (exec_path 2) mixed with cluster-path sensors: each
    result equals the same sensor served alone, under both policies."""
    ddh, serve = mods
    b = sy.config_batched(5)
    cfgs = [sy.config_single_256(5), b[1], sy.config_single_256(5), b[2]]
    paths = [2, 2, 1, 1]
    frames = [torch.from_numpy(sy.Stream(c).frames(5)[0]).cuda() for c in cfgs]
    params = [ddh.default_params(c.n, c.aperture_diam, c.snr, exec_path=pa) for c, pa in zip(cfgs, paths)]
    alone = serve.NativeService(mem_budget_bytes=1 << 34)
    alone.admit(0, params[0])
    alone.drive([(0.0, 0, frames[0][k]) for k in range(5)])
    rng = np.random.default_rng(2)
    arrivals = sorted((float(t), i, frames[i][k]) for i in range(len(cfgs))
                      for k, t in enumerate(np.cumsum(rng.exponential(1e-4, 5))))
    for flags in (0, 3):
        mix = serve.NativeService(mem_budget_bytes=1 << 34)
        mix.set_policy(flags)
        for i, p in enumerate(params):
            mix.admit(i, p)
        res = mix.drive(arrivals)
        assert len(res) == 20
        assert torch.equal(alone.phase(0), mix.phase(0)) and torch.equal(alone.reflectance(0), mix.reflectance(0))
        mix.close()
    alone.close()


# ------------------------------------------------------------------ native scheduler
def test_native_alone_equals_mix_and_per_frame_mode(mods):
    ddh, serve = mods
    cfgs = _sensors()
    frames = [torch.from_numpy(sy.Stream(c).frames(6)[0]).cuda() for c in cfgs]
    params = [ddh.default_params(c.n, c.aperture_diam, c.snr) for c in cfgs]
    alone = serve.NativeService(mem_budget_bytes=1 << 34)
    alone.admit(0, params[0])
    res = alone.drive([(0.0, 0, frames[0][k]) for k in range(6)])
    assert sorted(r[2] for r in res) == [1, 2, 3, 4, 5, 6]
    rng = np.random.default_rng(1)
    arrivals = sorted((float(t), i, frames[i][k]) for i in range(len(cfgs))
                      for k, t in enumerate(np.cumsum(rng.exponential(2e-4, 6))))
    outs = {}
    for mode in (False, True):
        mix = serve.NativeService(mem_budget_bytes=1 << 34, per_frame_launch=mode)
        for i, p in enumerate(params):
            mix.admit(i, p)
        res = mix.drive(arrivals)
        assert len(res) == 36 and all(r[4] >= r[3] for r in res)
        for i in range(len(cfgs)):  # per-sensor completion order follows arrival order
            idx = [r[0] for r in res if r[1] == i]
            assert [r[2] for r in res if r[1] == i] == list(range(1, 7)) and idx == sorted(idx)
        outs[mode] = (mix.phase(0), mix.reflectance(0), mix.stats())
        mix.close()
    assert outs[False][2]["batches"] < 36   # frames shared launches
    for mode in (False, True):
        assert torch.equal(alone.phase(0), outs[mode][0]) and torch.equal(alone.reflectance(0), outs[mode][1])
    alone.close()


def test_native_admission_budget(mods):
    ddh, serve = mods
    p256 = ddh.default_params(256, 128.0, 5.0)
    need = ddh.lib().ddh_state_bytes(256)
    svc = serve.NativeService(mem_budget_bytes=2 * need + 10)
    svc.admit(1, p256)
    svc.admit(2, p256)
    with pytest.raises(serve.AdmissionError):
        svc.admit(3, p256)
    svc.release(1)
    svc.admit(3, p256)
    assert svc.stats()["used_bytes"] == 2 * need
    svc.close()
