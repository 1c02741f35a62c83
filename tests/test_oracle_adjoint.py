"""Pins of the oracle gradient (FP64 reverse mode through K frame steps) to FP64 central
finite differences (h = 1e-6) on the 32x32 copy of the differentiation workload."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import ddh_adjoint as adj
from oracle import ddh_oracle as o
from synth import ddh_synth as sy


def _setup(tilt_mode=1, frames=3):
    cfg = sy.config_adjoint(small=True, streams=1, frames=frames)[0]
    ys, _ = sy.Stream(cfg).frames(frames)
    prm = o.default_params(32, 16.0, cfg.snr, tilt_mode=tilt_mode)
    a = o.aperture(32, 16.0)
    rng = np.random.default_rng(tilt_mode)
    phi0 = np.where(a, 0.3 * rng.standard_normal((32, 32)), 0.0)
    r0 = 0.05 + 0.02 * rng.random((32, 32))
    c = rng.standard_normal((3, 32, 32))
    return ys, prm, a, phi0, r0, c


def _loss(ys, prm, a, c, r0, phi0):
    st = o.State(r=r0.copy(), phi=phi0.copy())
    for y in ys:
        st, _ = o.step(st, y, prm)
    return float(np.sum(a * (c[0] * np.cos(st.phi) + c[1] * np.sin(st.phi))) + np.sum(c[2] * st.r)), st


@pytest.mark.parametrize("tilt_mode", [1, 0])
def test_oracle_gradient_matches_finite_differences(tilt_mode):
    ys, prm, a, phi0, r0, c = _setup(tilt_mode)
    _, stK = _loss(ys, prm, a, c, r0, phi0)
    phib = a * (-c[0] * np.sin(stK.phi) + c[1] * np.cos(stK.phi))
    rb, pb, g, _ = adj.unrolled_grad(r0, phi0, ys, prm, c[2], phib)
    h = 1e-6
    for k, field in enumerate(["prior_sigma", "prior_p", "noise_var"]):
        v = getattr(prm, field)
        fd = (_loss(ys, replace(prm, **{field: v + h}), a, c, r0, phi0)[0]
              - _loss(ys, replace(prm, **{field: v - h}), a, c, r0, phi0)[0]) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * abs(fd) + 1e-9, (field, g[k], fd)
    rng = np.random.default_rng(9)
    d = np.where(a, rng.standard_normal((32, 32)), 0.0)
    fd = (_loss(ys, prm, a, c, r0, phi0 + h * d)[0] - _loss(ys, prm, a, c, r0, phi0 - h * d)[0]) / (2 * h)
    assert abs(np.sum(pb * d) - fd) <= 1e-5 * abs(fd)
    d = 0.01 * rng.standard_normal((32, 32))
    fd = (_loss(ys, prm, a, c, r0 + h * d, phi0)[0] - _loss(ys, prm, a, c, r0 - h * d, phi0)[0]) / (2 * h)
    assert abs(np.sum(rb * d) - fd) <= 1e-5 * abs(fd)


def test_weight_derivatives_match_finite_differences():
    prm = o.Params(n=4, aperture_diam=2, prior_p=1.2, prior_T=1.4, prior_sigma=0.2)
    d = np.array([-0.7, -0.05, 0.003, 0.2, 1.5])
    w, dd, ds, dp = adj.weight_and_derivs(d, prm)
    assert np.allclose(w, o.qggmrf_weight(d, prm), rtol=1e-13)
    h = 1e-7
    assert np.allclose(dd, (o.qggmrf_weight(d + h, prm) - o.qggmrf_weight(d - h, prm)) / (2 * h), rtol=1e-6)
    fs = lambda s: o.qggmrf_weight(d, replace(prm, prior_sigma=s))
    assert np.allclose(ds, (fs(0.2 + h) - fs(0.2 - h)) / (2 * h), rtol=1e-6)
    fp = lambda p: o.qggmrf_weight(d, replace(prm, prior_p=p))
    assert np.allclose(dp, (fp(1.2 + h) - fp(1.2 - h)) / (2 * h), rtol=1e-6)


def test_adjoint_rejects_unsupported_variants():
    ys, prm, a, phi0, r0, c = _setup()
    with pytest.raises(ValueError):
        adj.frame_backward(r0, phi0, ys[0], replace(prm, n_k=2), r0, phi0)
