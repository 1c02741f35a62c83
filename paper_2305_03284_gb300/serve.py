"""Continuous-batching streaming service: the Python handle of libddh's native scheduler.

Sensors are admitted against a device-memory budget (free HBM minus a reserve, or a cap the
caller sets); each keeps its state ``(n, r, phi)`` resident on the device.  Frames arrive at
any time into per-sensor FIFOs.  The scheduler (a C++ thread inside libddh) repeatedly resolves
finished batches (an event per batch) and, when its batch-formation policy (``ddh_sched_pick``,
a pure host function that the host tests also drive in a simulation) says so, launches the next
queued frame of every sensor that has one as one batched step, without waiting for batches
already on the device.  Frames n and n+1 of one sensor depend on each other; they may sit in
consecutive batches on the device at once because the batches execute in order on one stream.

Each sensor's result is independent of which other sensors share its launches (no cross-stream
arithmetic, the kernels are fixed per stream), so a frame's output is the same alone and in
the mix.
"""
from __future__ import annotations

from ._lib import DDH_EBUDGET


class AdmissionError(RuntimeError):
    """Admission refused: the sensor's state would exceed the device-memory budget."""
    code = DDH_EBUDGET


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
        self._running = False
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

    def set_policy(self, flags: int, age_limit_s: float = 1e-3) -> None:
        """Select the batch-formation rules (``DDH_SCHED_*`` flags of the C header)."""
        self._L.check(self._L.lib().ddh_service_set_policy(self._h, int(flags), float(age_limit_s)))

    def start(self) -> None:
        self._L.check(self._L.lib().ddh_service_start(self._h))
        self._running = True

    def stop(self) -> None:
        self._running = False
        self._L.check(self._L.lib().ddh_service_stop(self._h))

    def drive(self, arrivals, timeout_s: float = 120.0, keep_running: bool = False) -> list:
        """Replay ``arrivals`` = sorted ``(t_seconds, sensor, frame)`` on the library thread;
        returns completions (tag = index into ``arrivals``).  The library thread is started if
        it is not running; ``keep_running`` leaves it running afterwards (a later replay then
        does not pay for starting it).  The replaying Python loop runs
        with the garbage collector paused: a collection pass over a large heap stops this
        thread for tens of milliseconds, which would delay submissions past their scheduled
        arrival times and be counted as service latency."""
        import gc
        gc_was_on = gc.isenabled()
        gc.disable()
        if not self._running:
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
            if not keep_running:
                self.stop()
            if gc_was_on:
                gc.enable()
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
