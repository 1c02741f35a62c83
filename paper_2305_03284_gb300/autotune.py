"""Autotuner for libddh's per-grid-size FFT radix schedule.

For each grid size it times every schedule on seeded synthetic frames in the configuration
that matters for throughput (as many streams per launch as clusters of that size can be
resident), keeps the fastest, and writes a table ``{"<n>": {"schedule": s, "us_per_frame": t,
...}}``.  ``apply(table)`` selects those schedules in the library for the current device.
Schedules differ only in rounding, and a given grid size always uses the same schedule
whatever the batch mix, so results do not depend on which streams share a launch.
"""
from __future__ import annotations

import json
import os

import torch

from . import ddh

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def _frames(n: int, streams: int, frames: int):
    from synth import ddh_synth as sy  # seeded inputs only
    out = []
    for s in range(streams):
        cfg = sy.StreamConfig(n=n, aperture_diam=n / 2, d_over_r0=10.0, wind=0.5, wind_angle=0.7, snr=10.0,
                              frames=frames, config_id=6, stream_id=s)
        ys, _ = sy.Stream(cfg).frames(frames)
        out.append(torch.from_numpy(ys).cuda())
    return out


def time_schedule(n: int, schedule: int, streams: int, frames: int = 8, reps: int = 50, rings=None) -> float:
    """Microseconds per timestep for `streams` streams of size n, one batched launch per step."""
    ddh.set_fft_schedule(n, schedule)
    cuda_stream = torch.cuda.Stream()
    with torch.cuda.stream(cuda_stream):
        sts = [ddh.Stream(ddh.default_params(n, n / 2, 10.0), stream=cuda_stream) for _ in range(streams)]
        rings = rings if rings is not None else _frames(n, streams, frames)
        for t in range(5):
            ddh.step_batch(sts, [rings[i][t % frames] for i in range(streams)])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cuda_stream)
        for t in range(reps):
            ddh.step_batch(sts, [rings[i][t % frames] for i in range(streams)])
        e1.record(cuda_stream)
        e1.synchronize()
        for s in sts:
            s.sync()
    return e0.elapsed_time(e1) * 1e3 / reps


def tune(sizes=(64, 128, 256), streams_for=None, path: str | None = DEFAULT_TABLE) -> dict:
    streams_for = streams_for or {64: 32, 128: 16, 256: 7}
    table = {}
    for n in sizes:
        k = streams_for.get(n, 8)
        rings = _frames(n, k, 8)
        times = [time_schedule(n, s, k, rings=rings) for s in range(ddh.fft_schedule_count(n))]
        best = min(range(len(times)), key=lambda i: times[i])
        table[str(n)] = {"schedule": best, "us_per_step": times[best], "streams": k,
                         "all_us_per_step": times}
        ddh.set_fft_schedule(n, best)
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


def apply(table: dict | str | None = DEFAULT_TABLE) -> dict:
    """Select the tabled schedules (a dict, or the path of a JSON table) on the current device."""
    if isinstance(table, str) or table is None:
        if table is None or not os.path.exists(table):
            return {}
        with open(table) as f:
            table = json.load(f)
    for n, row in table.items():
        ddh.set_fft_schedule(int(n), int(row["schedule"]))
    return table


if __name__ == "__main__":
    print(json.dumps(tune(), indent=1))
