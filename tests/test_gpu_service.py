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


def test_result_alone_equals_result_in_mix(mods):
    ddh, serve = mods
    cfgs = _sensors()
    frames = [torch.from_numpy(sy.Stream(c).frames(6)[0]).cuda() for c in cfgs]
    params = [ddh.default_params(c.n, c.aperture_diam, c.snr) for c in cfgs]
    alone = serve.Service(mem_budget_bytes=1 << 34)
    alone.admit("x", params[0])
    for f in range(6):
        alone.submit("x", frames[0][f])
    alone.drain()
    mix = serve.Service(mem_budget_bytes=1 << 34)
    for i, p in enumerate(params):
        mix.admit(i, p)
    rng = np.random.default_rng(0)
    arrivals = sorted((float(t), i, frames[i][k]) for i in range(len(cfgs))
                      for k, t in enumerate(np.cumsum(rng.exponential(2e-4, 6))))
    res = mix.drive(arrivals)
    assert len(res) == 36
    assert max(mix.batch_sizes) > 1
    a, m = alone.state("x"), mix.state(0)
    assert torch.equal(a.phase(), m.phase()) and torch.equal(a.reflectance(), m.reflectance())
    assert m.frame_index == 6


def test_admission_against_memory_budget(mods):
    ddh, serve = mods
    p256 = ddh.default_params(256, 128.0, 5.0)
    be = serve.LibddhBackend()
    need = be.state_bytes(p256)
    svc = serve.Service(backend=be, mem_budget_bytes=2 * need + 10)
    svc.admit("a", p256)
    svc.admit("b", p256)
    with pytest.raises(serve.AdmissionError):
        svc.admit("c", p256)
    svc.release("a")
    svc.admit("c", p256)
    assert svc.used_bytes == 2 * need


def test_background_loop_and_phase_delivery(mods):
    ddh, serve = mods
    cfg = sy.config_single_64(4)
    frames = torch.from_numpy(sy.Stream(cfg).frames(4)[0]).cuda()
    svc = serve.Service(mem_budget_bytes=1 << 32)
    svc.admit("s", ddh.default_params(64, 32.0, 10.0))
    ref = ddh.Stream(ddh.default_params(64, 32.0, 10.0))
    svc.start()
    try:
        futs = [svc.submit("s", frames[k]) for k in range(4)]
        res = [f.result(timeout=30) for f in futs]
    finally:
        svc.stop()
    for k in range(4):
        ref.step(frames[k])
    assert [r.frame_index for r in res] == [1, 2, 3, 4]
    assert torch.equal(res[-1].phase, ref.phase())


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
