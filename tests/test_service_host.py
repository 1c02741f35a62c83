"""Host-side logic of the continuous-batching service (no GPU): the native batch-formation
policy ``ddh_sched_pick`` through the C ABI, case by case and inside a discrete-event
simulation of the 32-sensor Poisson workload on a modelled device."""
import ctypes

import numpy as np
import pytest

from paper_2305_03284_gb300 import _lib
from synth import ddh_synth as sy

BACKLOG, AGE = _lib.DDH_SCHED_BACKLOG, _lib.DDH_SCHED_AGE


@pytest.fixture(scope="module")
def lib():
    from paper_2305_03284_gb300 import build
    build.build()
    return _lib.lib()


def _pick(lib, queued, oldest=None, in_flight=0, max_in_flight=2, now=0.0, age=1e-3, flags=BACKLOG | AGE):
    n = len(queued)
    view = (_lib.DdhSchedSensor * max(n, 1))()
    for i, q in enumerate(queued):
        view[i].queued = q
        view[i].oldest_arrival_s = oldest[i] if oldest is not None else 0.0
    pick = (ctypes.c_ubyte * max(n, 1))()
    rc = lib.ddh_sched_pick(view, n, in_flight, max_in_flight, now, age, flags, pick)
    return rc, [pick[i] for i in range(n)]


def test_idle_device_launches_every_ready_sensor(lib):
    rc, pick = _pick(lib, [0, 1, 3, 0, 1])
    assert rc == 3 and pick == [0, 1, 1, 0, 1]
    assert _pick(lib, [0, 0, 0])[0] == 0
    assert _pick(lib, [])[0] == 0


def test_nothing_beyond_max_in_flight(lib):
    assert _pick(lib, [1, 1, 1, 1], in_flight=2, max_in_flight=2) == (0, [0, 0, 0, 0])
    assert _pick(lib, [5, 5], in_flight=3, max_in_flight=2)[0] == 0


def test_behind_a_running_batch_half_the_sensors(lib):
    # 2 of 6 ready, none backlogged or old: wait for the running batch
    assert _pick(lib, [1, 1, 0, 0, 0, 0], in_flight=1, flags=0)[0] == 0
    assert _pick(lib, [1, 1, 0, 0, 0, 0], in_flight=1)[0] == 0
    # 3 of 6 ready: launch behind it
    assert _pick(lib, [1, 1, 1, 0, 0, 0], in_flight=1, flags=0) == (3, [1, 1, 1, 0, 0, 0])


def test_backlogged_sensor_launches_behind_a_running_batch(lib):
    q = [2, 0, 0, 0, 1, 0]  # sensor 0 has a second frame waiting
    assert _pick(lib, q, in_flight=1, flags=0)[0] == 0
    assert _pick(lib, q, in_flight=1, flags=BACKLOG) == (2, [1, 0, 0, 0, 1, 0])


def test_old_frame_launches_behind_a_running_batch(lib):
    q, oldest = [1, 0, 0, 0], [0.010, 0, 0, 0]
    assert _pick(lib, q, oldest, in_flight=1, now=0.0105, age=1e-3, flags=AGE)[0] == 0
    assert _pick(lib, q, oldest, in_flight=1, now=0.0111, age=1e-3, flags=AGE)[0] == 1
    assert _pick(lib, q, oldest, in_flight=1, now=0.0111, age=1e-3, flags=0)[0] == 0


def test_policy_rejects_bad_arguments(lib):
    assert lib.ddh_sched_pick(None, 3, 0, 2, 0.0, 1e-3, 0, None) == -1
    assert _pick(lib, [1], max_in_flight=0)[0] == -1
    assert lib.ddh_service_set_policy(None, 0, 1e-3) == -1


# ------------------------------------------------------------------ simulated workload
# Device model of one batched step, from GB300 measurements of the library's kernels: a fixed
# 12 us per batch plus the per-frame cost of each grid size in a large batch (512^2 on the
# staged kernels 12.4 us, 256^2 on the cluster kernel 5.1 us, 128^2 2.0 us); batches run one
# after another in launch order; the scheduler spends 15 us of host time per launch and polls
# every 5 us otherwise.
COST = {512: 12.4e-6, 256: 5.1e-6, 128: 2.0e-6}


def _trace(seed=5, total=10_000):
    cfgs = sy.config_service(frames_total=total)
    rates = np.array([c.rate_khz * 1e3 for c in cfgs])
    horizon = total / rates.sum()
    rng = np.random.default_rng(seed)
    arr = []
    for i in range(len(cfgs)):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rates[i])
            if t > horizon:
                break
            arr.append((t, i))
    arr.sort()
    return [c.n for c in cfgs], arr, horizon


def _simulate(lib, sizes, arr, flags, age=1e-3, max_in_flight=2, c0=12e-6, host=15e-6, poll=5e-6):
    n = len(sizes)
    queues = [[] for _ in range(n)]
    view = (_lib.DdhSchedSensor * n)()
    pick = (ctypes.c_ubyte * n)()
    in_flight, lat = [], []
    dev_t = t = done_t = 0.0
    i = 0
    order = []  # (sensor, frame number) in completion order
    launched = [0] * n
    while i < len(arr) or in_flight or any(queues):
        while i < len(arr) and arr[i][0] <= t:
            queues[arr[i][1]].append(arr[i][0])
            i += 1
        while in_flight and in_flight[0][0] <= t:
            _, items = in_flight.pop(0)
            for s, a, k in items:
                lat.append(t - a)
                order.append((s, k))
            done_t = t
        for k in range(n):
            view[k].queued = len(queues[k])
            view[k].oldest_arrival_s = queues[k][0] if queues[k] else 0.0
        rc = lib.ddh_sched_pick(view, n, len(in_flight), max_in_flight, t, age, flags, pick)
        assert rc >= 0
        if rc > 0:
            items = []
            for k in range(n):
                if pick[k]:
                    items.append((k, queues[k].pop(0), launched[k]))
                    launched[k] += 1
            dev_t = max(t + host, dev_t) + c0 + sum(COST[sizes[k]] for k, _, _ in items)
            in_flight.append((dev_t, items))
            t += host
        elif any(queues):
            t += poll
        else:
            nxt = ([arr[i][0]] if i < len(arr) else []) + ([in_flight[0][0]] if in_flight else [])
            t = max(t + poll, min(nxt)) if nxt else t + poll
    lat = np.sort(np.array(lat))
    return len(lat) / done_t, lat[len(lat) // 2], lat[int(0.99 * len(lat))], order


def test_simulated_service_keeps_up_and_keeps_each_sensor_in_order(lib):
    sizes, arr, horizon = _trace()
    offered = len(arr) / horizon
    fps, p50, p99, order = _simulate(lib, sizes, arr, BACKLOG | AGE)
    assert len(order) == len(arr)
    for s in range(len(sizes)):  # each sensor's frames complete in arrival order, one at a time
        ks = [k for x, k in order if x == s]
        assert ks == sorted(ks) == list(range(len(ks)))
    assert fps >= 0.99 * offered
    assert p50 < 1e-3


def test_simulated_backlog_rule_shortens_the_tail(lib):
    """With a sensor whose frames outpace full batches, the backlog rule lets it advance behind
    a running batch: the simulated p99 falls against the half-the-sensors rule alone."""
    sizes, arr, _ = _trace()
    _, _, p99_old, _ = _simulate(lib, sizes, arr, 0)
    _, _, p99_new, _ = _simulate(lib, sizes, arr, BACKLOG | AGE)
    assert p99_new < p99_old
