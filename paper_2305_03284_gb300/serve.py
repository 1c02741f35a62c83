"""Continuous-batching streaming service over libddh.

Sensors are admitted against a device-memory budget (free HBM minus a reserve, or a cap the
caller sets); each keeps its state ``(n, r, phi)`` resident on the device.  Frames arrive at
any time into per-sensor FIFOs.  The scheduler loop repeatedly

1. resolves finished batches (an event per batch), delivering each frame's phase and latency;
2. forms a batch from the next queued frame of every sensor that has one (at most one frame per
   sensor per batch) and launches it with ``ddh_step_batch`` without waiting for batches
   already in flight (up to ``max_in_flight``), so frames that arrive while the GPU works join
   the next launch.  Frames n and n+1 of one sensor depend on each other; they may sit in
   consecutive batches on the device at once because the batches execute in order on one
   stream (a backend must keep that order).  A batch starts behind a running one only if it
   holds at least half of the sensors, so that a backlog keeps the device busy while light
   traffic still gathers into full batches.

Each sensor's result is independent of which other sensors share its launches (one cluster per
stream, no cross-stream arithmetic), so a frame's output is the same alone and in the mix.
The scheduling logic is backend-agnostic: ``Service(backend=...)`` takes any object with
``new_state(params)``, ``step_batch(states, frames)``, ``record() -> event`` (an object with
``query()``), ``phase(state, out)`` and ``state_bytes(params)``; the default drives libddh.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

from ._lib import DDH_EBUDGET


class AdmissionError(RuntimeError):
    """Admission refused: the sensor's state would exceed the device-memory budget."""
    code = DDH_EBUDGET


@dataclass
class FrameResult:
    sensor: object
    frame_index: int
    latency_s: float
    phase: object = None   # device tensor (a slot of the sensor's output ring) or None


@dataclass
class _Sensor:
    sid: object
    state: object
    params: object
    nbytes: int
    queue: collections.deque = field(default_factory=collections.deque)
    in_flight: int = 0        # frames in batches on the device
    frames_done: int = 0
    frames_launched: int = 0
    out_ring: list = field(default_factory=list)
    closing: bool = False


class LibddhBackend:
    """libddh on one CUDA stream (torch supplies the stream and the output tensors)."""

    def __init__(self, cuda_stream=None, out_ring: int = 4):
        import torch
        from . import ddh
        self.torch = torch
        self.ddh = ddh
        self.stream = cuda_stream if cuda_stream is not None else torch.cuda.Stream()
        self.out_ring = out_ring

    def state_bytes(self, params) -> int:
        n = int(params.n)
        img = 4 * n * n
        # libddh: r, phi, a 2 N^2 float staging buffer, status and scalar words; plus the
        # service's output ring of phase images
        return 4 * img + 512 + self.out_ring * img

    def new_state(self, params):
        with self.torch.cuda.stream(self.stream):
            return self.ddh.Stream(params, stream=self.stream)

    def new_outputs(self, params):
        n = int(params.n)
        return [self.torch.empty((n, n), dtype=self.torch.float32, device="cuda") for _ in range(self.out_ring)]

    def step_batch(self, states, frames) -> None:
        self.ddh.step_batch(states, frames)

    def phase(self, state, out) -> None:
        state.phase(out)

    def record(self):
        ev = self.torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info()
        return int(free)

    def close_state(self, state) -> None:
        state.close()


class PerFrameLaunchBackend(LibddhBackend):
    """Comparison path: the same scheduler, but every frame is its own ``ddh_step`` launch."""

    def step_batch(self, states, frames) -> None:
        for st, y in zip(states, frames):
            st.step(y)


class Service:
    def __init__(self, backend=None, mem_budget_bytes: int | None = None, reserve_bytes: int = 1 << 30,
                 max_in_flight: int = 2, deliver_phase: bool = True, clock=time.perf_counter):
        self.backend = backend if backend is not None else LibddhBackend()
        self.max_in_flight = max_in_flight
        self.deliver_phase = deliver_phase
        self.clock = clock
        self._sensors: dict = {}
        self._in_flight = collections.deque()   # (event, [(sensor, future, arrival, slot)])
        self._lock = threading.RLock()
        self._used = 0
        if mem_budget_bytes is None:
            free = getattr(self.backend, "free_bytes", lambda: 1 << 62)()
            mem_budget_bytes = max(0, free - reserve_bytes)
        self.budget = int(mem_budget_bytes)
        self.batches_launched = 0
        self.batch_sizes: list[int] = []
        self._thread = None
        self._stop = threading.Event()

    # -- admission ----------------------------------------------------------------------
    def admit(self, sid, params) -> None:
        """Admit a sensor if its resident state fits the memory budget."""
        need = int(self.backend.state_bytes(params))
        with self._lock:
            if sid in self._sensors:
                raise ValueError(f"sensor {sid!r} already admitted")
            if self._used + need > self.budget:
                raise AdmissionError(f"sensor {sid!r} needs {need} B; {self.budget - self._used} B of budget left")
            state = self.backend.new_state(params)
            s = _Sensor(sid=sid, state=state, params=params, nbytes=need)
            if self.deliver_phase:
                s.out_ring = self.backend.new_outputs(params)
            self._sensors[sid] = s
            self._used += need

    def release(self, sid) -> None:
        """Drop a sensor once its queued and in-flight frames are done (frees its budget)."""
        with self._lock:
            self._sensors[sid].closing = True
            self._reap()

    @property
    def used_bytes(self) -> int:
        return self._used

    def sensors(self):
        return list(self._sensors)

    def state(self, sid):
        return self._sensors[sid].state

    # -- frames -------------------------------------------------------------------------
    def submit(self, sid, frame, arrival: float | None = None) -> Future:
        """Queue one frame (a device tensor the caller keeps valid until its future resolves)."""
        fut = Future()
        with self._lock:
            s = self._sensors[sid]
            if s.closing:
                raise ValueError(f"sensor {sid!r} is being released")
            s.queue.append((frame, self.clock() if arrival is None else arrival, fut))
        return fut

    def pending(self) -> int:
        with self._lock:
            return sum(len(s.queue) for s in self._sensors.values()) + sum(len(b) for _, b in self._in_flight)

    # -- scheduler ----------------------------------------------------------------------
    def poll(self) -> int:
        """Resolve finished batches and launch the next one; returns frames launched."""
        with self._lock:
            while self._in_flight and self._in_flight[0][0].query():
                _, items = self._in_flight.popleft()
                now = self.clock()
                for s, fut, arrival, slot in items:
                    s.in_flight -= 1
                    s.frames_done += 1
                    out = s.out_ring[slot] if slot is not None else None
                    fut.set_result(FrameResult(s.sid, s.frames_done, now - arrival, out))
            self._reap()
            if len(self._in_flight) >= self.max_in_flight:
                return 0
            ready = [s for s in self._sensors.values() if s.queue]
            if not ready:
                return 0
            if self._in_flight and 2 * len(ready) < len(self._sensors):
                return 0          # behind a running batch only a batch of half the sensors
            frames, states, items = [], [], []
            for s in ready:
                frame, arrival, fut = s.queue.popleft()
                frames.append(frame)
                states.append(s.state)
                s.in_flight += 1
                items.append((s, fut, arrival, None))
            self.backend.step_batch(states, frames)
            if self.deliver_phase:
                for i, (s, fut, arrival, _) in enumerate(items):
                    slot = s.frames_launched % len(s.out_ring)
                    self.backend.phase(s.state, s.out_ring[slot])
                    items[i] = (s, fut, arrival, slot)
            for s, *_ in items:
                s.frames_launched += 1
            self._in_flight.append((self.backend.record(), items))
            self.batches_launched += 1
            self.batch_sizes.append(len(items))
            return len(items)

    def _reap(self) -> None:
        for sid in [k for k, s in self._sensors.items() if s.closing and not s.queue and s.in_flight == 0]:
            s = self._sensors.pop(sid)
            self.backend.close_state(s.state)
            self._used -= s.nbytes

    def drain(self, timeout_s: float = 60.0) -> None:
        t0 = time.perf_counter()
        while self.pending():
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("service did not drain")

    def start(self) -> None:
        """Run the scheduler loop on a background thread (for submit() from other threads)."""
        self._stop.clear()

        def loop():
            while not self._stop.is_set():
                if self.poll() == 0:
                    time.sleep(20e-6)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self) -> None:
        self._stop.set()
        if self._thread is not None:
            self._thread.join()
            self._thread = None

    def drive(self, arrivals) -> list[FrameResult]:
        """Replay ``arrivals`` = sorted ``(t_seconds, sensor, frame)`` against the clock in the
        calling thread; each frame's latency runs from its scheduled arrival to completion."""
        futs = []
        t0 = self.clock()
        i = 0
        while i < len(arrivals) or self.pending():
            now = self.clock() - t0
            while i < len(arrivals) and arrivals[i][0] <= now:
                t, sid, frame = arrivals[i]
                futs.append(self.submit(sid, frame, arrival=t0 + t))
                i += 1
            self.poll()
        return [f.result() for f in futs]


class NativeService:
    """The continuous-batching scheduler of libddh (a C++ thread inside the library).

    ``admit`` / ``release`` sensors (int ids) against a device-memory budget, ``submit`` device
    frames, collect ``(tag, sensor, frame_index, arrival_s, done_s)`` completions with
    ``poll``.  ``per_frame_launch=True`` is the comparison mode that launches every frame alone.
    """

    def __init__(self, cuda_stream=None, mem_budget_bytes: int = 0, max_in_flight: int = 2,
                 per_frame_launch: bool = False):
        import ctypes
        import torch
        from . import _lib
        self._ct = ctypes
        self._L = _lib
        self.torch = torch
        self.stream = cuda_stream if cuda_stream is not None else torch.cuda.Stream()
        self._h = ctypes.c_void_p()
        _lib.check(_lib.lib().ddh_service_create(ctypes.byref(self._h), ctypes.c_void_p(self.stream.cuda_stream),
                                                 int(mem_budget_bytes), int(max_in_flight),
                                                 1 if per_frame_launch else 0))
        self._buf = (_lib.DdhCompletion * 4096)()
        self._n = ctypes.c_int()
        self._sizes = {}

    def admit(self, sid: int, params) -> None:
        rc = self._L.lib().ddh_service_admit(self._h, int(sid), self._ct.byref(params))
        if rc == self._L.DDH_EBUDGET:
            raise AdmissionError(f"sensor {sid} does not fit the memory budget")
        self._L.check(rc)
        self._sizes[int(sid)] = int(params.n)

    def release(self, sid: int) -> None:
        self._L.check(self._L.lib().ddh_service_release(self._h, int(sid)))

    def phase(self, sid: int, out=None):
        """Copy of the sensor's current phase (valid between its frames)."""
        st = self._L.lib().ddh_service_state(self._h, int(sid))
        if not st:
            raise KeyError(sid)
        n = self._sizes[int(sid)]
        out = out if out is not None else self.torch.empty((n, n), dtype=self.torch.float32, device="cuda")
        self._L.check(self._L.lib().ddh_phase(self._ct.c_void_p(st), self._ct.c_void_p(out.data_ptr())))
        self._join_state(st)
        return out

    def _join_state(self, st) -> None:
        # the copy runs on the sensor's stream: order torch's current stream after it
        sst = self._L.lib().ddh_state_stream(self._ct.c_void_p(st))
        self.torch.cuda.current_stream().wait_stream(self.torch.cuda.ExternalStream(sst))

    def reflectance(self, sid: int, out=None):
        st = self._L.lib().ddh_service_state(self._h, int(sid))
        if not st:
            raise KeyError(sid)
        n = self._sizes[int(sid)]
        out = out if out is not None else self.torch.empty((n, n), dtype=self.torch.float32, device="cuda")
        self._L.check(self._L.lib().ddh_reflectance(self._ct.c_void_p(st), self._ct.c_void_p(out.data_ptr())))
        self._join_state(st)
        return out

    def submit(self, sid: int, frame, arrival_s: float = -1.0, tag: int = 0) -> None:
        self._L.check(self._L.lib().ddh_service_submit(self._h, int(sid), self._ct.c_void_p(frame.data_ptr()),
                                                       float(arrival_s), int(tag)))

    def poll(self) -> list:
        self._L.check(self._L.lib().ddh_service_poll(self._h, self._buf, len(self._buf), self._ct.byref(self._n)))
        return [(c.tag, c.sensor, c.frame_index, c.arrival_s, c.done_s) for c in self._buf[: self._n.value]]

    def pending(self) -> int:
        return int(self._L.lib().ddh_service_pending(self._h))

    def stats(self) -> dict:
        b, f, u = self._ct.c_int64(), self._ct.c_int64(), self._ct.c_size_t()
        self._L.check(self._L.lib().ddh_service_stats(self._h, self._ct.byref(b), self._ct.byref(f),
                                                      self._ct.byref(u)))
        return {"batches": b.value, "frames": f.value, "used_bytes": u.value}

    def now(self) -> float:
        return float(self._L.lib().ddh_service_now())

    def start(self) -> None:
        self._L.check(self._L.lib().ddh_service_start(self._h))

    def stop(self) -> None:
        self._L.check(self._L.lib().ddh_service_stop(self._h))

    def drive(self, arrivals, timeout_s: float = 120.0) -> list:
        """Replay ``arrivals`` = sorted ``(t_seconds, sensor, frame)`` on the library thread;
        returns completions (tag = index into ``arrivals``)."""
        self.start()
        done = []
        try:
            t0 = self.now()
            i = 0
            while i < len(arrivals):
                now = self.now() - t0
                while i < len(arrivals) and arrivals[i][0] <= now:
                    t, sid, frame = arrivals[i]
                    self.submit(sid, frame, arrival_s=t0 + t, tag=i)
                    i += 1
                done.extend(self.poll())
            while len(done) < len(arrivals):
                done.extend(self.poll())
                if self.now() - t0 > timeout_s:
                    raise TimeoutError("service did not finish the trace")
        finally:
            self.stop()
        return done

    def close(self) -> None:
        if self._h:
            self._L.lib().ddh_service_free(self._h)
            self._h = self._ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
