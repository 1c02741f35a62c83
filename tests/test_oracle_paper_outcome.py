"""The oracle's multi-frame trajectory against the paper's reported outcome (Sec. 5.C: at the
Sec. 5.A simulation parameters the loop reaches a Strehl ratio of 0.8 within 150 frames at one
EM iteration per frame).  One simulation of the bar-chart stream with the tracking parameter
set, run on the CPU: its per-frame Strehl ratios equal the stored oracle trace
(tests/golden/paper_chart_strehl.txt, written by tests/golden/make_paper_chart_trace.py), and its
10-frame mean reaches 0.8 within the first 40 frames."""
import os
import sys

import numpy as np

from oracle import ddh_oracle as o
from synth import ddh_synth as sy

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_paper_chart_trace as gold  # noqa: E402  (the script's parameter set, oracle-only)

SIM, FRAMES = 2, 40


def test_oracle_trajectory_reaches_the_papers_strehl_and_matches_the_stored_trace():
    prm = gold.params()
    st = sy.Stream(sy.config_paper_256(SIM, gold.FRAMES))
    a = o.aperture(256, 128.0)
    state = o.init_state(256)
    trace = []
    for k in range(FRAMES):
        y, ph = st.frame(k)
        state, _ = o.step(state, y, prm)
        trace.append(o.strehl(state.phi, ph.astype(np.float32).astype(np.float64), a))
    trace = np.array(trace)
    stored = np.loadtxt(os.path.join(HERE, "golden", "paper_chart_strehl.txt"))[:FRAMES, SIM]
    assert np.allclose(trace, stored, rtol=1e-9, atol=0.0), float(np.max(np.abs(trace - stored)))
    mean10 = np.convolve(trace, np.ones(10) / 10, mode="valid")
    assert trace[0] < 0.2  # the loop starts from the uncorrected phase
    assert mean10.max() >= 0.8, mean10.max()
