"""Autotuner of libddh's launch shapes on the current GPU.

Knobs, per grid size N:
* the FFT radix schedule of the cluster kernel (N <= 256);
* the launch chunk of the L2-staged kernels (streams per launch sequence, N = 128, 256, 512):
  small chunks keep a chunk's working images in L2 between its stages, large ones launch fewer
  kernels;
* which kernels a batch of B streams of size N should run on (``exec_path``): the cluster
  kernel (one thread-block cluster per stream; at most 7 resident 16-CTA clusters at 256^2, so
  112 of the 152 SMs) or the staged kernels (every stage spread over all SMs), timed at
  several batch sizes; ``recommend_path(n, streams)`` reads the result;
* whether a batch's staged streams run as chained stage launches or as one persistent launch
  per step (``ddh_set_staged_persistent``), timed on the 64-stream mix of 128^2, 256^2 and
  512^2 streams all on the staged kernels, and on 32 streams of 256^2.

Each candidate is timed on seeded synthetic frames with CUDA events, one batched step per time
step, after warm-up.  The table (``{"<n>": {...}}``) is committed as ``tuning_gb300.json``;
``apply()`` selects its schedules and chunks in the library for the current device.  A stream's
result never depends on the batch it runs in: the FFT schedule is fixed per grid size, the path
is fixed per stream at creation, and the chunking only groups streams into launches.
"""
from __future__ import annotations

import json
import os

import torch

from . import ddh
from ._lib import DDH_PATH_CLUSTER, DDH_PATH_DEFAULT, DDH_PATH_STAGED, check, lib

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
STAGED_SIZES = (128, 256, 512)
CLUSTER_SIZES = (64, 128, 256)


def _frames(n: int, streams: int, frames: int):
    from synth import ddh_synth as sy  # seeded inputs only
    out = []
    for s in range(streams):
        cfg = sy.StreamConfig(n=n, aperture_diam=n / 2, d_over_r0=10.0, wind=0.5, wind_angle=0.7, snr=10.0,
                              frames=frames, config_id=6, stream_id=s)
        ys, _ = sy.Stream(cfg).frames(frames)
        out.append(torch.from_numpy(ys).cuda())
    return out


def time_batch(n: int, streams: int, path: int = DDH_PATH_DEFAULT, frames: int = 4, reps: int = 40,
               rings=None) -> float:
    """Microseconds per time step for `streams` streams of size n on `path`, every stream
    advanced one frame per step by one captured-graph batch."""
    cuda_stream = torch.cuda.Stream()
    rings = rings if rings is not None else _frames(n, min(streams, 8), frames)
    with torch.cuda.stream(cuda_stream):
        sts = [ddh.Stream(ddh.default_params(n, n / 2, 10.0, exec_path=path), stream=cuda_stream)
               for _ in range(streams)]
        g = ddh.BatchGraph(sts)
        k = len(rings)
        for t in range(3):
            g.run([rings[i % k][t % frames] for i in range(streams)])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cuda_stream)
        for t in range(reps):
            g.run([rings[i % k][t % frames] for i in range(streams)])
        e1.record(cuda_stream)
        e1.synchronize()
        g.close()
        for s in sts:
            s.sync()
            s.close()
    return e0.elapsed_time(e1) * 1e3 / reps


def tune(path: str | None = DEFAULT_TABLE, sizes=(64, 128, 256, 512), batch_sizes=(1, 2, 4, 7, 8, 16, 32, 64),
         big: dict | None = None, chunks=(4, 8, 16, 32), schedule_streams: dict | None = None,
         persistent_mix: bool = True) -> dict:
    """Time every knob; `big` gives the batch size (per N) the staged chunk is tuned at and
    `schedule_streams` the batch the FFT schedules are compared at (as many clusters as can
    be resident).  Leaves the winners selected in the library."""
    big = big or {64: 64, 128: 64, 256: 32, 512: 16}
    schedule_streams = schedule_streams or {64: 32, 128: 16, 256: 7}
    table: dict = {}
    for n in sizes:
        row: dict = {}
        rings = _frames(n, 8, 4)
        if n in CLUSTER_SIZES:
            t = []
            for sch in range(ddh.fft_schedule_count(n)):
                ddh.set_fft_schedule(n, sch)
                t.append(time_batch(n, schedule_streams[n], DDH_PATH_CLUSTER, rings=rings))
            row["schedule"] = min(range(len(t)), key=lambda i: t[i])
            row["schedule_us_per_step"] = t
            ddh.set_fft_schedule(n, row["schedule"])
        if n in STAGED_SIZES:
            t = {}
            for c in chunks:
                check(lib().ddh_set_staged_chunk(n, c))
                t[str(c)] = time_batch(n, big[n], DDH_PATH_STAGED, rings=rings)
            row["staged_chunk"] = int(min(t, key=t.get))
            row["staged_chunk_us_per_step"] = t
            row["staged_chunk_streams"] = big[n]
            check(lib().ddh_set_staged_chunk(n, row["staged_chunk"]))
        if n in CLUSTER_SIZES and n in STAGED_SIZES:
            cmp = {}
            for b in batch_sizes:
                cmp[str(b)] = {"cluster": time_batch(n, b, DDH_PATH_CLUSTER, rings=rings),
                               "staged": time_batch(n, b, DDH_PATH_STAGED, rings=rings)}
            row["path_us_per_step"] = cmp
            wins = [int(b) for b, v in cmp.items() if v["staged"] < v["cluster"]]
            # the smallest batch size from which the staged kernels win at every measured size
            start = None
            for b in sorted(int(x) for x in cmp):
                if all(w in wins for w in (int(x) for x in cmp if int(x) >= b)):
                    start = b
                    break
            row["staged_from_streams"] = start
        table[str(n)] = row
    if persistent_mix:
        table["persistent"] = tune_persistent()
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


def time_mixed(sizes, persistent: int, frames: int = 4, reps: int = 30) -> float:
    """Microseconds per time step of a captured-graph batch of staged streams of the given grid
    sizes, with the persistent launch on or off."""
    check(lib().ddh_set_staged_persistent(int(persistent)))
    cuda_stream = torch.cuda.Stream()
    rings = {n: _frames(n, 4, frames) for n in set(sizes)}
    with torch.cuda.stream(cuda_stream):
        sts = [ddh.Stream(ddh.default_params(n, n / 2, 10.0, exec_path=DDH_PATH_STAGED), stream=cuda_stream)
               for n in sizes]
        g = ddh.BatchGraph(sts)
        ys = lambda t: [rings[n][i % 4][t % frames] for i, n in enumerate(sizes)]
        for t in range(3):
            g.run(ys(t))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cuda_stream)
        for t in range(reps):
            g.run(ys(t))
        e1.record(cuda_stream)
        e1.synchronize()
        g.close()
        for s in sts:
            s.sync()
            s.close()
    return e0.elapsed_time(e1) * 1e3 / reps


def tune_persistent() -> dict:
    mix = [128] * 32 + [256] * 24 + [512] * 8
    out = {}
    for name, sizes in (("mix64", mix), ("256x32", [256] * 32)):
        out[name] = {"chained_us_per_step": time_mixed(sizes, 0), "persistent_us_per_step": time_mixed(sizes, 1)}
    # persistent only where it wins on both workloads
    out["persistent"] = int(all(v["persistent_us_per_step"] < v["chained_us_per_step"] for v in out.values()))
    check(lib().ddh_set_staged_persistent(out["persistent"]))
    return out


def _load(table):
    if isinstance(table, str) or table is None:
        if table is None or not os.path.exists(table):
            return {}
        with open(table) as f:
            return json.load(f)
    return table


def apply(table: dict | str | None = DEFAULT_TABLE) -> dict:
    """Select the tabled FFT schedules and staged chunks (a dict, or the path of a JSON table)
    on the current device."""
    table = _load(table)
    for n, row in table.items():
        if n == "persistent":
            check(lib().ddh_set_staged_persistent(int(row.get("persistent", 0))))
            continue
        if "schedule" in row:
            ddh.set_fft_schedule(int(n), int(row["schedule"]))
        if "staged_chunk" in row:
            check(lib().ddh_set_staged_chunk(int(n), int(row["staged_chunk"])))
    return table


def recommend_path(n: int, streams: int, table: dict | str | None = DEFAULT_TABLE) -> int:
    """The exec_path to create `streams` streams of grid n with, for the fastest batched step:
    the staged kernels from the tabled batch size on, else the cluster kernel."""
    row = _load(table).get(str(n), {})
    start = row.get("staged_from_streams")
    if n not in CLUSTER_SIZES:
        return DDH_PATH_DEFAULT
    if start is not None and streams >= int(start):
        return DDH_PATH_STAGED
    return DDH_PATH_CLUSTER


if __name__ == "__main__":
    print(json.dumps(tune(), indent=1))
