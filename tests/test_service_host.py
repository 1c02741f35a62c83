"""Host-side logic of the continuous-batching service, on a fake backend (no GPU)."""
import pytest

from paper_2305_03284_gb300.serve import AdmissionError, Service


class FakeEvent:
    def __init__(self, backend):
        self.backend = backend
        self.polls = 0

    def query(self):
        self.polls += 1
        return self.polls > self.backend.latency_polls


class FakeState:
    def __init__(self, params):
        self.params = params
        self.frames = []
        self.closed = False


class Params:
    def __init__(self, n):
        self.n = n


class FakeBackend:
    def __init__(self, latency_polls=1, bytes_per_state=100):
        self.latency_polls = latency_polls
        self.bytes_per_state = bytes_per_state
        self.batches = []

    def state_bytes(self, params):
        return self.bytes_per_state

    def new_state(self, params):
        return FakeState(params)

    def new_outputs(self, params):
        return [f"out{i}" for i in range(3)]

    def step_batch(self, states, frames):
        for s, f in zip(states, frames):
            s.frames.append(f)
        self.batches.append(list(frames))

    def phase(self, state, out):
        pass

    def record(self):
        return FakeEvent(self)

    def close_state(self, state):
        state.closed = True


def make(**kw):
    be = FakeBackend(**{k: v for k, v in kw.items() if k in ("latency_polls", "bytes_per_state")})
    svc = Service(backend=be, mem_budget_bytes=kw.get("budget", 10_000), max_in_flight=kw.get("max_in_flight", 2),
                  clock=lambda: 0.0)
    return be, svc


def test_fifo_per_sensor_and_one_frame_per_sensor_per_batch():
    be, svc = make(latency_polls=3)
    svc.admit("a", Params(64))
    svc.admit("b", Params(128))
    fa = [svc.submit("a", f"a{i}") for i in range(3)]
    fb = [svc.submit("b", f"b{i}") for i in range(2)]
    svc.drain()
    assert svc.state("a").frames == ["a0", "a1", "a2"]
    assert svc.state("b").frames == ["b0", "b1"]
    # no batch ever held two frames of one sensor
    for batch in be.batches:
        assert len({f[0] for f in batch}) == len(batch)
    assert [f.result().frame_index for f in fa] == [1, 2, 3]
    assert fb[-1].result().phase == "out1"


def test_frames_arriving_while_a_batch_runs_join_the_next_launch():
    be, svc = make(latency_polls=5, max_in_flight=2)
    for s in "abc":
        svc.admit(s, Params(64))
    svc.submit("a", "a0")
    assert svc.poll() == 1            # batch 1 in flight: {a}
    svc.submit("b", "b0")
    svc.submit("c", "c0")
    assert svc.poll() == 2            # batch 2 launched while batch 1 still runs: {b, c}
    svc.submit("a", "a1")
    assert svc.poll() == 0            # two batches are in flight
    svc.drain()
    assert be.batches == [["a0"], ["b0", "c0"], ["a1"]]


def test_next_frame_of_a_sensor_joins_the_next_batch_while_its_previous_runs():
    be, svc = make(latency_polls=5, max_in_flight=3)
    svc.admit("a", Params(64))
    svc.admit("b", Params(64))
    fa = [svc.submit("a", "a0"), svc.submit("a", "a1")]
    assert svc.poll() == 1            # {a0}: one frame per sensor per batch
    assert svc.poll() == 1            # {a1} launched while a0 still runs (batches run in order)
    fb = svc.submit("b", "b0")
    fa.append(svc.submit("a", "a2"))
    assert svc.poll() == 2            # {a2, b0}
    assert svc.poll() == 0            # three batches in flight
    svc.drain()
    assert be.batches == [["a0"], ["a1"], ["a2", "b0"]]
    assert svc.state("a").frames == ["a0", "a1", "a2"]
    assert [f.result().frame_index for f in fa] == [1, 2, 3]
    assert [f.result().phase for f in fa] == ["out0", "out1", "out2"]
    assert fb.result().frame_index == 1


def test_admission_by_budget_and_release():
    be, svc = make(bytes_per_state=400, budget=1000)
    svc.admit("a", Params(64))
    svc.admit("b", Params(64))
    with pytest.raises(AdmissionError) as e:
        svc.admit("c", Params(64))
    assert e.value.code == -6
    svc.submit("a", "a0")
    svc.poll()
    svc.release("a")                  # frame still in flight: not freed yet
    assert svc.used_bytes == 800
    svc.drain()
    svc.poll()
    assert svc.used_bytes == 400 and "a" not in svc.sensors()
    svc.admit("c", Params(64))
    with pytest.raises(ValueError):
        svc.admit("c", Params(64))


def test_drive_replays_arrivals_and_reports_latency():
    be = FakeBackend(latency_polls=2)
    t = [0.0]

    def clock():
        t[0] += 1e-4
        return t[0]
    svc = Service(backend=be, mem_budget_bytes=10_000, clock=clock)
    for s in range(4):
        svc.admit(s, Params(128))
    arrivals = sorted((0.001 * k + 0.0002 * s, s, (s, k)) for s in range(4) for k in range(5))
    res = svc.drive(arrivals)
    assert len(res) == 20 and all(r.latency_s >= 0 for r in res)
    for s in range(4):
        assert svc.state(s).frames == [(s, k) for k in range(5)]
    assert max(svc.batch_sizes) > 1   # frames of different sensors shared launches


def test_a_batch_behind_a_running_one_needs_half_of_the_sensors():
    be, svc = make(latency_polls=5, max_in_flight=2)
    for x in "abcd":
        svc.admit(x, Params(64))
    svc.submit("a", "a0")
    assert svc.poll() == 1            # nothing in flight: any batch goes
    svc.submit("a", "a1")
    assert svc.poll() == 0            # 1 of 4 sensors ready behind a running batch: wait
    svc.submit("b", "b0")
    assert svc.poll() == 2            # 2 of 4: {a1, b0}
    svc.drain()
    assert be.batches == [["a0"], ["a1", "b0"]]
