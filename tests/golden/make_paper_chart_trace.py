"""Writes paper_chart_strehl.txt: the FP64 oracle's per-frame Strehl ratio over 150 frames of
the paper-parameter stream (Sec. 5.A: N 256, D/r0 10, v = (0.421, 0.421) px/frame, SNR 10 dB,
a bar-chart object), simulations 0-9, with the tracking parameter set (2 x 2 phase tiles under
the tile prior of precision 10, sigma_r 0.03, alpha 0.0125, lambda 0.45, one EM iteration per
frame).  Calls only oracle/ and synth/; the parameters are rounded to float32, the precision in
which the library receives them.  Run from the repository root:

    python tests/golden/make_paper_chart_trace.py
"""
import math
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_chart_strehl.txt")
FRAMES = 150
SIMS = 10


def params():
    sys.path.insert(0, ROOT)
    from oracle import ddh_oracle as o
    f32 = lambda v: float(np.float32(v))
    a = o.aperture(256, 128.0)
    nv = f32(1.0 / (1.0 + float(a.mean()) * 10.0))
    return o.Params(n=256, aperture_diam=128.0, lam=f32(0.45), alpha=f32(0.0125), n_k=1, noise_var=nv,
                    prior_p=f32(1.1), prior_q=2.0, prior_T=1.0, prior_sigma=f32(0.03), r_floor=f32(1e-10),
                    tilt_mode=1, phase_block=2, phase_prior=10.0, phase_sweeps=2, noise_update=0)


def one(sim):
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import ddh_oracle as o
    from synth import ddh_synth as sy
    prm = params()
    st = sy.Stream(sy.config_paper_256(sim, FRAMES))
    a = o.aperture(256, 128.0)
    state = o.init_state(256)
    out = []
    for k in range(FRAMES):
        y, ph = st.frame(k)
        state, _ = o.step(state, y, prm)
        out.append(o.strehl(state.phi, ph.astype(np.float32).astype(np.float64), a))
    return sim, out


if __name__ == "__main__":
    with mp.get_context("spawn").Pool(min(SIMS, os.cpu_count() or 1)) as pool:
        res = dict(pool.map(one, range(SIMS)))
    with open(OUT, "w") as f:
        f.write("# FP64 oracle Strehl ratio per frame (rows: frames 0-149; columns: simulations 0-9) of\n")
        f.write("# the paper-parameter bar-chart stream with the tracking parameter set; written by\n")
        f.write("# tests/golden/make_paper_chart_trace.py (oracle/ and synth/ only)\n")
        for k in range(FRAMES):
            f.write(" ".join(f"{res[s][k]:.10e}" for s in range(SIMS)) + "\n")
    best = [max(np.convolve(res[s], np.ones(10) / 10, mode="valid")) for s in range(SIMS)]
    print("best 10-frame mean per simulation:", " ".join(f"{b:.3f}" for b in best))
