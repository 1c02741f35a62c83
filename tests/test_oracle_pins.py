"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (no GPU).

Each test checks one oracle function against something other than itself: a naive DFT,
Parseval, the adjoint identity, the exact Gaussian posterior, a dense scan, a brute-force
ICD, the closed-form limits of the q-GGMRF potential, a dense-matrix MAP objective, or a value
printed in the paper (tests/golden/paper_values.txt).
"""
import math
import os

import numpy as np
import pytest

from oracle import ddh_oracle as o
from synth import ddh_synth as sy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def _dft_matrix_2d(n):
    """Dense unitary 2D DFT on row-major n x n images, written from the definition."""
    k = np.arange(n)
    f1 = np.exp(-2j * math.pi * np.outer(k, k) / n) / math.sqrt(n)
    return np.kron(f1, f1)


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out[key] = [float(v) for v in vals]
    return out


# ---------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("n", [8, 16])
def test_fft_matches_naive_dft(n):
    rng = _rng(n)
    x = _crandn(rng, n, n)
    X = np.zeros((n, n), complex)
    for ky in range(n):
        for kx in range(n):
            acc = 0j
            for yy in range(n):
                for xx in range(n):
                    acc += x[yy, xx] * np.exp(-2j * math.pi * (ky * yy + kx * xx) / n)
            X[ky, kx] = acc / n
    assert np.allclose(o.fft2u(x), X, atol=1e-12)
    assert np.allclose(o.ifft2u(X), x, atol=1e-12)


def test_parseval_and_inverse():
    rng = _rng(1)
    x = _crandn(rng, 32, 32)
    assert math.isclose(np.linalg.norm(o.fft2u(x)), np.linalg.norm(x), rel_tol=1e-13)
    assert np.allclose(o.ifft2u(o.fft2u(x)), x, atol=1e-13)


def test_adjoint_identity():
    rng = _rng(2)
    n = 16
    a = o.aperture(n, 8.0)
    x, y = _crandn(rng, n, n), _crandn(rng, n, n)
    phi = rng.uniform(-math.pi, math.pi, (n, n))
    lhs = np.vdot(y, o.forward_op(x, phi, a))
    rhs = np.vdot(o.adjoint_op(y, phi, a), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_operator_matches_dense_matrix():
    """A_phi = D_a D(exp(j phi)) F as an explicit matrix (Sec. 2)."""
    rng = _rng(3)
    n = 8
    a = o.aperture(n, 4.0)
    phi = rng.uniform(-math.pi, math.pi, (n, n))
    A = np.diag(a.ravel().astype(float)) @ np.diag(np.exp(1j * phi.ravel())) @ _dft_matrix_2d(n)
    g = _crandn(rng, n, n)
    assert np.allclose(o.forward_op(g, phi, a).ravel(), A @ g.ravel(), atol=1e-12)
    y = _crandn(rng, n, n)
    assert np.allclose(o.adjoint_op(y, phi, a).ravel(), A.conj().T @ y.ravel(), atol=1e-12)


def test_aperture_geometry():
    a = o.aperture(256, 128.0)
    # disc of radius 64 about (127.5, 127.5): pi r^2 to within the pixelation
    assert abs(a.sum() - math.pi * 64 ** 2) < 2 * math.pi * 64
    assert a[127, 127] and a[128, 128] and not a[0, 0]
    assert np.array_equal(a, a[::-1, :]) and np.array_equal(a, a.T)


# ---------------------------------------------------------------------------- Normalize
def test_normalize_eq4():
    rng = _rng(4)
    y = _crandn(rng, 32, 32) * 3.0 + (1.5 - 2j)
    yt, st = o.normalize(y)
    assert abs(yt.mean()) < 1e-13
    assert math.isclose(np.sum(np.abs(yt) ** 2), y.size, rel_tol=1e-13)
    # invariant to affine rescaling up to the phase of the scale
    c = 3.0 * np.exp(0.7j)
    yt2, _ = o.normalize(c * y + (2.0 + 1.0j))
    assert np.allclose(yt2, np.exp(0.7j) * yt, atol=1e-12)


# ---------------------------------------------------------------------------- RemoveTipTilt
def test_tip_tilt_removes_wrapped_plane():
    n, d = 32, 16.0
    a = o.aperture(n, d)
    c = (n - 1) / 2
    yy, xx = np.mgrid[0:n, 0:n]
    tx, ty, piston = 0.9, -1.3, 2.5
    phi = o.wrap(tx * (xx - c) + ty * (yy - c) + piston)
    ex, ey = o.tip_tilt(phi, a)
    assert math.isclose(ex, tx, rel_tol=1e-12) and math.isclose(ey, ty, rel_tol=1e-12)
    out, _ = o.remove_tip_tilt(phi, a)
    assert np.allclose(o.wrap(out[a] - piston), 0.0, atol=1e-12)
    assert np.all(out[~a] == 0.0)


def test_tip_tilt_zero_phase():
    a = o.aperture(16, 8.0)
    assert o.tip_tilt(np.zeros((16, 16)), a) == (0.0, 0.0)


# ---------------------------------------------------------------------------- E-step
def test_estep_equals_exact_posterior_for_constant_r():
    """For constant r the A^H A ~ I posterior mean is exact: F^H D_a F is a projection and
    A^H y lies in its range.  Compare with D(r) A^H (A D(r) A^H + s2 I)^-1 y."""
    rng = _rng(5)
    n = 8
    a = o.aperture(n, 4.0)
    phi = rng.uniform(-math.pi, math.pi, (n, n))
    A = np.diag(a.ravel().astype(float)) @ np.diag(np.exp(1j * phi.ravel())) @ _dft_matrix_2d(n)
    y = _crandn(rng, n, n)
    r0, s2 = 0.7, 0.3
    prm = o.Params(n=n, aperture_diam=4.0, noise_var=s2)
    R = r0 * np.eye(n * n)
    mu_exact = R @ A.conj().T @ np.linalg.solve(A @ R @ A.conj().T + s2 * np.eye(n * n), y.ravel())
    b = o.adjoint_op(y, phi, a)
    mu, s, w = o.estep(np.full((n, n), r0), b, prm)
    assert np.allclose(mu.ravel(), mu_exact, atol=1e-12)
    # the variance term is the exact one when a == 1 everywhere (A unitary)
    Au = np.diag(np.exp(1j * phi.ravel())) @ _dft_matrix_2d(n)
    cov = np.linalg.inv(np.eye(n * n) / r0 + Au.conj().T @ Au / s2)
    assert np.allclose(np.real(np.diag(cov)), (s - np.abs(mu) ** 2).ravel(), atol=1e-12)


# ---------------------------------------------------------------------------- prior
def test_qggmrf_closed_forms():
    prm = o.Params(n=4, aperture_diam=2, prior_p=1.1, prior_q=2.0, prior_T=1.0, prior_sigma=0.3)
    # p = q = 2: u = 1 and rho = D^2 / (4 sigma^2)
    prm22 = o.Params(n=4, aperture_diam=2, prior_p=2.0, prior_q=2.0, prior_T=1.0, prior_sigma=0.3)
    d = np.linspace(-2, 2, 41)
    assert np.allclose(o.qggmrf_rho(d, prm22), d ** 2 / (4 * 0.3 ** 2), rtol=1e-13)
    # small |D|: rho ~ D^2 / (p sigma^2 T^(2-p)); large |D|: rho ~ |D|^p/(p sigma^p)
    small = 1e-7
    assert math.isclose(float(o.qggmrf_rho(small, prm)), small ** 2 / (1.1 * 0.3 ** 2), rel_tol=1e-5)
    big = 1e7
    assert math.isclose(float(o.qggmrf_rho(big, prm)), big ** 1.1 / (1.1 * 0.3 ** 1.1), rel_tol=1e-5)


def test_qggmrf_weight_is_derivative_over_delta():
    prm = o.Params(n=4, aperture_diam=2, prior_p=1.1, prior_q=2.0, prior_T=1.3, prior_sigma=0.2)
    d = np.concatenate([np.linspace(-3, -1e-3, 50), np.linspace(1e-3, 3, 50)])
    h = 1e-6
    deriv = (o.qggmrf_rho(d + h, prm) - o.qggmrf_rho(d - h, prm)) / (2 * h)
    assert np.allclose(o.qggmrf_weight(d, prm), deriv / d, rtol=1e-6)
    # the value at zero is the limit
    lim = float(o.qggmrf_weight(np.array([0.0]), prm)[0])
    assert math.isclose(lim, float(o.qggmrf_weight(np.array([1e-9]), prm)[0]), rel_tol=1e-6)


def test_symmetric_bound_majorises():
    prm = o.Params(n=4, aperture_diam=2, prior_p=1.1, prior_q=2.0, prior_T=1.0, prior_sigma=0.1)
    dp = np.linspace(-2, 2, 81)
    dd = np.linspace(-3, 3, 241)
    for x0 in dp:
        bound = o.qggmrf_rho(x0, prm) + 0.5 * o.qggmrf_weight(np.array([x0]), prm)[0] * (dd ** 2 - x0 ** 2)
        assert np.all(o.qggmrf_rho(dd, prm) <= bound + 1e-12)


def test_prior_energy_bruteforce():
    rng = _rng(6)
    n = 5
    prm = o.Params(n=n, aperture_diam=2, prior_sigma=0.2)
    r = rng.uniform(0, 1, (n, n))
    e = 0.0
    pix = [(y, x) for y in range(n) for x in range(n)]
    for i, (y0, x0) in enumerate(pix):
        for (y1, x1) in pix[i + 1:]:
            dy, dx = abs(y1 - y0), abs(x1 - x0)
            if max(dy, dx) != 1:
                continue
            bij = 1 / (4 + 2 * math.sqrt(2)) / (math.sqrt(2) if dy and dx else 1.0)
            e += bij * float(o.qggmrf_rho(r[y0, x0] - r[y1, x1], prm))
    assert math.isclose(o.prior_energy(r, prm), e, rel_tol=1e-12)


# ---------------------------------------------------------------------------- cubic / ICD
def _h(r, W, C, s):
    return np.log(r) + s / r + 0.5 * W * r ** 2 - C * r


def test_cubic_argmin_is_global_minimiser():
    rng = _rng(7)
    cases = []
    for _ in range(300):  # generic coefficients
        W = 10 ** rng.uniform(-1, 3)
        C = W * 10 ** rng.uniform(-3, 0.5)
        s = 10 ** rng.uniform(-4, 0)
        cases.append((W, C, s))
    for _ in range(300):  # three positive roots by construction
        x = np.sort(10 ** rng.uniform(-3, 1, 3))
        W = 1.0 / (x[0] * x[1] + x[0] * x[2] + x[1] * x[2])
        cases.append((W, W * x.sum(), W * x.prod()))
    W, C, s = (np.array(v) for v in zip(*cases))
    r = o.cubic_argmin(W, C, s)
    grid = np.logspace(-7, 3, 200_001)
    for i in range(len(cases)):
        f = W[i] * r[i] ** 3 - C[i] * r[i] ** 2 + r[i] - s[i]
        scale = W[i] * r[i] ** 3 + C[i] * r[i] ** 2 + r[i] + s[i]
        assert abs(f) <= 1e-9 * scale
        hs = _h(grid, W[i], C[i], s[i])
        hr = _h(r[i], W[i], C[i], s[i])
        assert hr <= hs.min() + 1e-9 * max(1.0, abs(hr))


def test_cubic_w_zero_gives_s():
    s = np.array([0.3, 2.0])
    assert np.array_equal(o.cubic_argmin(np.zeros(2), np.zeros(2), s), s)


def test_icd_sweep_bruteforce_small_grid():
    """4-colour sweep on a 5x5 grid vs a pixel-by-pixel dense minimisation of the surrogate,
    with neighbours and weights enumerated explicitly."""
    rng = _rng(8)
    n = 5
    prm = o.Params(n=n, aperture_diam=2, prior_sigma=0.1, r_floor=1e-10)
    r0 = rng.uniform(0.01, 0.5, (n, n))
    s = rng.uniform(0.01, 0.5, (n, n))
    got = o.icd_sweep(r0, s, prm)
    r = r0.copy()
    grid = np.logspace(-6, 1, 70_001)
    for cx, cy in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        for yy in range(n):
            for xx in range(n):
                if xx % 2 != cx or yy % 2 != cy:
                    continue
                terms = []
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if (dy, dx) == (0, 0):
                            continue
                        y1, x1 = yy + dy, xx + dx
                        if not (0 <= y1 < n and 0 <= x1 < n):
                            continue
                        bij = 1 / (4 + 2 * math.sqrt(2)) / (math.sqrt(2) if dy and dx else 1.0)
                        beta = bij * float(o.qggmrf_weight(np.array([r0[yy, xx] - r0[y1, x1]]), prm)[0])
                        terms.append((beta, r[y1, x1]))
                hv = np.log(grid) + s[yy, xx] / grid
                for beta, rj in terms:
                    hv = hv + 0.5 * beta * (grid - rj) ** 2
                k = int(np.argmin(hv))
                lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
                for _ in range(200):  # golden-section refinement
                    m1, m2 = lo + 0.382 * (hi - lo), hi - 0.382 * (hi - lo)
                    f1 = np.log(m1) + s[yy, xx] / m1 + sum(0.5 * b_ * (m1 - rj) ** 2 for b_, rj in terms)
                    f2 = np.log(m2) + s[yy, xx] / m2 + sum(0.5 * b_ * (m2 - rj) ** 2 for b_, rj in terms)
                    lo, hi = (lo, m2) if f1 < f2 else (m1, hi)
                r[yy, xx] = 0.5 * (lo + hi)
    assert np.allclose(got, r, rtol=1e-7)


# ---------------------------------------------------------------------------- phase M-step
def test_phase_mstep_exact_recovery_noiseless():
    rng = _rng(9)
    n = 16
    a = o.aperture(n, 8.0)
    g = _crandn(rng, n, n)
    phi = np.where(a, rng.uniform(-math.pi, math.pi, (n, n)), 0.0)
    y = o.forward_op(g, phi, a)
    est, z = o.phase_mstep(y, g, np.zeros((n, n)), a)
    assert np.allclose(o.wrap(est - phi)[a], 0.0, atol=1e-12)
    assert np.all(est[~a] == 0.0)


def test_phase_mstep_minimises_data_term():
    rng = _rng(10)
    n = 8
    a = o.aperture(n, 6.0)
    y, mu = _crandn(rng, n, n), _crandn(rng, n, n)
    est, z = o.phase_mstep(y, mu, np.zeros((n, n)), a)
    base = np.abs(y - np.exp(1j * est) * z) ** 2
    for dphi in (0.01, -0.01, 0.5, 3.0):
        assert np.all((base <= np.abs(y - np.exp(1j * (est + dphi)) * z) ** 2 + 1e-12)[a])


# ---------------------------------------------------------------------------- EM objective
def _dense_map_cost(r, phi, y, prm):
    n = prm.n
    A = np.diag(np.exp(1j * phi.ravel())) @ _dft_matrix_2d(n)
    cov = A @ np.diag(r.ravel()) @ A.conj().T + prm.noise_var * np.eye(n * n)
    sign, logdet = np.linalg.slogdet(cov)
    quad = np.real(np.vdot(y.ravel(), np.linalg.solve(cov, y.ravel())))
    return logdet + quad + o.prior_energy(r, prm)


def test_em_objective_matches_dense_likelihood():
    rng = _rng(11)
    n = 8
    prm = o.Params(n=n, aperture_diam=1e6, noise_var=0.3, prior_sigma=0.2)
    r = rng.uniform(0.05, 1.0, (n, n))
    phi = rng.uniform(-1, 1, (n, n))
    y = _crandn(rng, n, n)
    assert math.isclose(o.em_objective_unit_aperture(r, phi, y, prm), _dense_map_cost(r, phi, y, prm),
                        rel_tol=1e-11)


def test_static_em_is_monotone_with_unit_aperture():
    """With a == 1 the operator is unitary, the E-step exact, and each EM iteration cannot
    increase the MAP cost of Eq. 2 (evaluated with a dense covariance)."""
    rng = _rng(12)
    n = 8
    prm = o.Params(n=n, aperture_diam=1e6, noise_var=0.2, prior_sigma=0.1)
    a = o.aperture(n, prm.aperture_diam)
    assert a.all()
    g = np.sqrt(rng.uniform(0, 1, (n, n))) * _crandn(rng, n, n)
    y = np.exp(1j * rng.uniform(-1, 1, (n, n))) * o.fft2u(g) + math.sqrt(0.2) * _crandn(rng, n, n)
    y, _ = o.normalize(y)
    r = np.maximum(np.abs(o.adjoint_op(y, np.zeros((n, n)), a)) ** 2, 1e-3)
    phi = np.zeros((n, n))
    costs = [_dense_map_cost(r, phi, y, prm)]
    for _ in range(50):
        r, phi = o.em_static_step(r, phi, y, prm, a)
        costs.append(_dense_map_cost(r, phi, y, prm))
    diffs = np.diff(costs)
    assert np.all(diffs <= 1e-9 * np.abs(costs[:-1])), diffs.max()
    assert costs[-1] < costs[0]


# ---------------------------------------------------------------------------- Strehl
def test_strehl_properties():
    rng = _rng(13)
    n = 64
    a = o.aperture(n, 32.0)
    phi = np.where(a, rng.uniform(-math.pi, math.pi, (n, n)), 0.0)
    assert math.isclose(o.strehl(phi, phi, a), 1.0, rel_tol=1e-12)
    assert math.isclose(o.strehl(phi + 1.234, phi, a), 1.0, rel_tol=1e-12)
    yy, xx = np.mgrid[0:n, 0:n]
    tilt = 2 * math.pi * (3 * xx - 2 * yy) / n   # integer-cycle tilt shifts the PSF by pixels
    assert math.isclose(o.strehl(phi + tilt, phi, a), 1.0, rel_tol=1e-12)
    # Marechal: small Gaussian residual sigma -> S ~ exp(-sigma^2)
    sig = 0.1
    err = sig * rng.standard_normal((n, n))
    S = o.strehl(phi + err, phi, a)
    assert abs(S - math.exp(-sig ** 2)) < 0.005


# ---------------------------------------------------------------------------- step
def test_first_frame_from_zero_state():
    cfg = sy.config_single_64(2)
    st = sy.Stream(cfg)
    y, _ = st.frame(0)
    prm = o.default_params(64, 32.0, cfg.snr, prior_sigma=0.1)
    s1, tr = o.step(o.init_state(64), y, prm)
    assert tr.stats["tx"] == 0.0 and tr.stats["ty"] == 0.0
    assert np.allclose(tr.r_init, np.maximum(prm.lam * prm.alpha * np.abs(tr.b) ** 2, prm.r_floor))
    a = o.aperture(64, 32.0)
    assert np.all(s1.phi[~a] == 0) and np.all(np.abs(s1.phi) <= math.pi)
    assert np.all(s1.r >= prm.r_floor) and np.all(np.isfinite(s1.r))


# ---------------------------------------------------------------------------- generator
def test_velocity_matches_paper():
    gold = _golden()
    vx, vy = sy.paper_velocity()
    fg, fs, nn, dr0 = gold["velocity_inputs_fg_fs_N_Dr0"]
    assert sy.velocity_magnitude(fg, fs, int(nn), dr0) == pytest.approx(math.hypot(vx, vy))
    assert vx == pytest.approx(gold["velocity_px_per_step"][0], abs=5e-4)
    assert vy == pytest.approx(gold["velocity_px_per_step"][1], abs=5e-4)


def test_default_weights_match_paper():
    gold = _golden()
    prm = o.Params(n=8, aperture_diam=4)
    assert prm.alpha == gold["alpha"][0] and prm.lam == gold["lambda"][0]


def test_phase_screen_structure_function():
    """Kolmogorov D(rho) = 6.88 (rho/r0)^(5/3); the sampled spectral method with subharmonics
    keeps the 5/3 law and loses part of the power at 1 px sampling."""
    cfg = sy.config_single_64(20)
    ratios = {2: [], 4: []}
    for sid in range(24):
        st = sy.Stream(sy.with_frames(cfg, 20).__class__(**{**cfg.__dict__, "stream_id": sid}))
        ph = st.screen(0)
        for rho in ratios:
            d = 0.5 * (np.mean((ph[:, rho:] - ph[:, :-rho]) ** 2) + np.mean((ph[rho:, :] - ph[:-rho, :]) ** 2))
            ratios[rho].append(d / (6.88 * (rho / st.r0_px) ** (5 / 3)))
    r2, r4 = np.mean(ratios[2]), np.mean(ratios[4])
    assert 0.6 < r2 < 1.1 and 0.6 < r4 < 1.1
    assert abs(r2 - r4) < 0.15  # the 5/3 exponent holds between the two separations


# ---------------------------------------------------------------------------- tiled phase
def test_tiled_phase_mstep_recovers_tile_constant_phase():
    rng = _rng(14)
    n, G = 16, 2
    a = o.aperture(n, 12.0)
    g = _crandn(rng, n, n)
    tiles = rng.uniform(-math.pi, math.pi, (n // G, n // G))
    phi = np.where(a, np.kron(tiles, np.ones((G, G))), 0.0)
    y = o.forward_op(g, phi, a)
    est, _ = o.phase_mstep(y, g, np.zeros((n, n)), a, block=G)
    assert np.allclose(o.wrap(est - phi)[a], 0.0, atol=1e-12)


def test_tiled_phase_mstep_minimises_tile_data_term():
    rng = _rng(15)
    n, G = 8, 4
    a = o.aperture(n, 7.0)
    y, mu = _crandn(rng, n, n), _crandn(rng, n, n)
    est, z = o.phase_mstep(y, mu, np.zeros((n, n)), a, block=G)
    for ty in range(n // G):
        for tx in range(n // G):
            sl = (slice(ty * G, ty * G + G), slice(tx * G, tx * G + G))
            m = a[sl]
            if not m.any():
                continue
            ph0 = est[sl][m][0]
            assert np.allclose(est[sl][m], ph0)  # constant on the tile
            cost = lambda t: float(np.sum(np.abs(y[sl][m] - np.exp(1j * t) * z[sl][m]) ** 2))
            grid = np.linspace(-math.pi, math.pi, 20001)
            assert cost(ph0) <= min(cost(t) for t in grid) + 1e-9


def test_tiled_block_one_is_per_pixel():
    rng = _rng(16)
    a = o.aperture(16, 10.0)
    y, mu = _crandn(rng, 16, 16), _crandn(rng, 16, 16)
    e1, _ = o.phase_mstep(y, mu, np.zeros((16, 16)), a)
    e2, _ = o.phase_mstep(y, mu, np.zeros((16, 16)), a, block=1)
    assert np.array_equal(e1, e2)


def test_static_em_monotone_with_tiled_phase():
    rng = _rng(17)
    n = 8
    prm = o.Params(n=n, aperture_diam=1e6, noise_var=0.2, prior_sigma=0.1, phase_block=2)
    a = o.aperture(n, prm.aperture_diam)
    g = np.sqrt(rng.uniform(0, 1, (n, n))) * _crandn(rng, n, n)
    y = np.exp(1j * rng.uniform(-1, 1, (n, n))) * o.fft2u(g) + math.sqrt(0.2) * _crandn(rng, n, n)
    y, _ = o.normalize(y)
    r = np.maximum(np.abs(o.adjoint_op(y, np.zeros((n, n)), a)) ** 2, 1e-3)
    phi = np.zeros((n, n))
    costs = [_dense_map_cost(r, phi, y, prm)]
    for _ in range(30):
        r, phi = o.em_static_step(r, phi, y, prm, a)
        costs.append(_dense_map_cost(r, phi, y, prm))
    assert np.all(np.diff(costs) <= 1e-9 * np.abs(costs[:-1]))


# ---------------------------------------------------------------------------- sensitivity
def _divergence(block, frames):
    cfg = sy.config_single_64(frames)
    ys, _ = sy.Stream(cfg).frames(frames)
    prm = o.default_params(64, 32.0, cfg.snr, phase_block=block)
    a = o.aperture(64, 32.0)
    A, B = o.init_state(64), o.init_state(64)
    rng = _rng(18)
    out = []
    for i in range(frames):
        A, _ = o.step(A, ys[i], prm)
        B, _ = o.step(B, ys[i], prm)
        if i == 0:
            B.r = B.r * (1 + 1e-7 * rng.standard_normal(B.r.shape))
            B.phi = np.where(a, B.phi + 1e-7 * rng.standard_normal(B.phi.shape), 0.0)
        out.append(np.linalg.norm(o.wrap(A.phi - B.phi)[a]) / np.linalg.norm(A.phi[a]))
    return np.array(out)


def test_per_pixel_phase_iteration_amplifies_perturbations():
    """Property of the per-pixel reading on this workload: a 1e-7 change of the state grows by
    orders of magnitude within 40 frames (bounds any free-running comparison horizon)."""
    d = _divergence(1, 40)
    assert d[-1] > 1e-3


def test_tiled_phase_iteration_contracts():
    d = _divergence(2, 40)
    assert d.max() < 1e-5 and d[-1] < 1e-6


def test_static_mode_is_the_frame_step_with_unit_blend():
    """Static DH-MBIR (Sec. 3): EM iterated on one frame with r reset to the back-projected
    estimate |A_phi^H y~|^2 at the start of each bootstrap period.  The frame step with
    lambda = alpha = 1, n_k = K and no tip/tilt removal is exactly that period: its r-init is
    the reset (Eq. 3 with lambda = alpha = 1) and its K EM iterations are the plain loop."""
    cfg = sy.config_single_64(3)
    ys, _ = sy.Stream(cfg).frames(3)
    K = 6
    prm = o.default_params(64, cfg.aperture_diam, cfg.snr, lam=1.0, alpha=1.0, n_k=K, tilt_mode=0)
    a = o.aperture(64, cfg.aperture_diam)
    st = o.init_state(64)
    r, phi = st.r, st.phi
    yt, _ = o.normalize(ys[1])
    for cycle in range(2):
        st, _ = o.step(st, ys[1], prm)
        # the static loop written out: reset, then K plain EM iterations
        b = o.adjoint_op(yt, phi, a)
        r = np.maximum(np.abs(b) ** 2, prm.r_floor)
        for _ in range(K):
            r, phi = o.em_static_step(r, phi, yt, prm, a)
        assert np.allclose(st.r, r, rtol=1e-12, atol=0) and np.allclose(st.phi, phi, rtol=0, atol=1e-12)


# ---- tile-phase M-step under the GMRF phase prior, sigma^2 M-step ----------------------------
def _phase_case(seed=5, n=64, d=32.0):
    rng = _rng(seed)
    a = o.aperture(n, d)
    yt = _crandn(rng, n, n)
    mu = 0.7 * o.ifft2u(yt) + 0.3 * _crandn(rng, n, n)  # z = F mu correlated with y
    return a, yt, mu


def test_phase_prior_zero_precision_is_the_tile_angle_step():
    a, yt, mu = _phase_case()
    phi_old = _rng(1).uniform(-1, 1, a.shape) * a
    for G in (2, 4):
        p0, z0 = o.phase_mstep(yt, mu, phi_old, a, G)
        p1, z1 = o.phase_mstep_prior(yt, mu, phi_old, a, G, 0.0, 0.3, 3)
        assert np.array_equal(p0, p1) and np.array_equal(z0, z1)


def test_phase_prior_sweeps_do_not_increase_the_map_cost():
    """Each majorised ICD sweep lowers (never raises) the phase M-step's cost, evaluated per
    pixel from its definition (data term over the aperture pixels, prior on the tile values)."""
    a, yt, mu = _phase_case()
    z = o.fft2u(mu)
    for G, lam in ((2, 4.0), (4, 40.0)):
        vt, has_ap = o.phase_tile_sums(yt, z, a, G)
        active = has_ap & (vt != 0)
        costs = []
        for k in range(7):
            phi, _ = o.phase_mstep_prior(yt, mu, np.zeros_like(yt.real), a, G, lam, 0.3, k)
            costs.append(o.phase_map_objective(phi, yt, z, a, 0.3, G, lam, active))
        assert all(c1 <= c0 + 1e-9 * abs(c0) for c0, c1 in zip(costs, costs[1:])), costs
        assert costs[-1] < costs[0] - 1e-4 * abs(costs[0])  # the prior moves the estimate


def test_phase_prior_fixed_point_is_stationary():
    """After many sweeps every active tile sits where the cost's derivative in its phase (a
    central difference of the per-pixel cost, all the tile's aperture pixels moved) is zero."""
    a, yt, mu = _phase_case(seed=7)
    z = o.fft2u(mu)
    G, lam, s2 = 4, 20.0, 0.3
    vt, has_ap = o.phase_tile_sums(yt, z, a, G)
    active = has_ap & (vt != 0)
    phi, _ = o.phase_mstep_prior(yt, mu, np.zeros_like(yt.real), a, G, lam, s2, 400)
    h = 1e-5
    nt = a.shape[0] // G
    worst = 0.0
    for T in range(nt):
        for X in range(nt):
            if not active[T, X]:
                continue
            m = np.zeros(a.shape, bool)
            m[T * G:(T + 1) * G, X * G:(X + 1) * G] = True
            m &= a
            fp = o.phase_map_objective(np.where(m, phi + h, phi), yt, z, a, s2, G, lam, active)
            fm = o.phase_map_objective(np.where(m, phi - h, phi), yt, z, a, s2, G, lam, active)
            scale = 2.0 * abs(vt[T, X]) / s2 + lam
            worst = max(worst, abs(fp - fm) / (2 * h) / scale)
    assert worst < 1e-5, worst


def test_phase_prior_two_tiles_closed_form():
    """Two active neighbouring tiles with equal |v| and angles +-alpha: the symmetric optimum
    phi = (beta, -beta) solves K sin(beta - alpha) + 2 lam b beta = 0, K = 2|v|/s2 (a scalar
    root found by bracketing, independent of the sweep's update formula)."""
    from scipy.optimize import brentq
    nt, alpha, m, s2, lam = 4, 1.0, 1.0, 0.5, 3.0
    vt = np.zeros((nt, nt), complex)
    vt[1, 1] = m * np.exp(1j * alpha)
    vt[1, 2] = m * np.exp(-1j * alpha)
    active = vt != 0
    pt = o.phase_prior_icd(vt, active, s2, lam, 500, np.angle(vt))
    K = 2 * m / s2
    beta = brentq(lambda b: K * math.sin(b - alpha) + 2 * lam * o.B_NN * b, 0.0, alpha)
    assert abs(pt[1, 1] - beta) < 1e-10 and abs(pt[1, 2] + beta) < 1e-10, (pt[1, 1], pt[1, 2], beta)
    assert np.all(pt[~active] == 0.0)


def test_noise_mstep_exact_fit_leaves_the_posterior_variance():
    rng = _rng(11)
    n = 32
    a = o.aperture(n, 16.0)
    z = _crandn(rng, n, n)
    phi = rng.uniform(-3, 3, (n, n))
    y = np.where(a, np.exp(1j * phi) * z, _crandn(rng, n, n))  # exact fit on the pupil only
    cvar = rng.uniform(0.01, 0.2, (n, n))
    assert abs(o.noise_mstep(y, z, phi, a, cvar) - cvar.mean()) < 1e-15


def test_noise_mstep_em_reaches_the_ml_variance():
    """Full aperture, phi = 0, constant r: y ~ CN(0, (r + s2) I) marginally, so the ML noise
    variance is mean|y|^2 - r; EM iterations of (E-step, sigma^2 M-step) must converge there."""
    rng = _rng(12)
    n = 32
    a = np.ones((n, n), bool)
    y = 1.1 * _crandn(rng, n, n)
    r0 = 0.4
    r = np.full((n, n), r0)
    phi = np.zeros((n, n))
    s2 = 2.0
    for _ in range(5000):
        prm = o.Params(n=n, aperture_diam=float(n), noise_var=s2)
        b = o.adjoint_op(y, phi, a)
        mu, _, w = o.estep(r, b, prm)
        s2_new = o.noise_mstep(y, o.fft2u(mu), phi, a, s2 * w)
        if abs(s2_new - s2) < 1e-15:
            break
        s2 = s2_new
    target = float(np.mean(np.abs(y) ** 2)) - r0
    assert target > 0.1 and abs(s2 - target) < 1e-9 * target, (s2, target)


def test_noise_mstep_residual_is_the_pupil_noise_power():
    """With the posterior variance zero and y = e^{j phi} z + w on the pupil (w ~ CN(0, v0)),
    the update is the sample noise power over the pupil pixels only: within 4 standard errors
    of v0 (about 6,400 pixels), whatever the data off the pupil."""
    rng = _rng(13)
    n = 128
    a = o.aperture(n, 90.0)
    z = _crandn(rng, n, n)
    phi = rng.uniform(-3, 3, (n, n))
    v0 = 0.37
    y = np.where(a, np.exp(1j * phi) * z + math.sqrt(v0) * _crandn(rng, n, n), 5.0 * _crandn(rng, n, n))
    est = o.noise_mstep(y, z, phi, a, np.zeros((n, n)))
    assert abs(est - v0) < 4 * v0 / math.sqrt(a.sum()), (est, v0)


# ---------------------------------------------------------------------------- Eq. 3 blend
def test_r_init_blend_with_previous_state_hand_values():
    """Eq. 3 with r_{n-1} != 0: (1 - lambda) r_{n-1} + lambda alpha |b|^2, floored.  Expected
    values computed by hand for lambda 0.45 / alpha 0.025 (the paper's, Sec. 5.B) and for
    lambda 0.3 / alpha 0.5."""
    r_prev = np.array([[0.2, 1.0], [0.0, 3.0]])
    b = np.array([[1 + 1j, 0.5], [2j, 0.0]])  # |b|^2 = 2, 0.25, 4, 0
    got = o.r_init(r_prev, b, o.Params(n=2, aperture_diam=2, lam=0.45, alpha=0.025, r_floor=1e-10))
    # 0.55*0.2 + 0.01125*2 = 0.1325; 0.55*1 + 0.01125*0.25 = 0.5528125; 0.01125*4 = 0.045; 0.55*3 = 1.65
    assert np.allclose(got, [[0.1325, 0.5528125], [0.045, 1.65]], rtol=0, atol=1e-15)
    got = o.r_init(r_prev, b, o.Params(n=2, aperture_diam=2, lam=0.3, alpha=0.5, r_floor=1e-10))
    # 0.7*0.2 + 0.15*2 = 0.44; 0.7 + 0.15*0.25 = 0.7375; 0.15*4 = 0.6; 0.7*3 = 2.1
    assert np.allclose(got, [[0.44, 0.7375], [0.6, 2.1]], rtol=0, atol=1e-15)
    # the floor applies where both terms vanish
    got = o.r_init(np.zeros((1, 2)), np.array([[0.0, 1.0]]), o.Params(n=2, aperture_diam=2, r_floor=1e-6))
    assert got[0, 0] == 1e-6 and got[0, 1] == pytest.approx(0.45 * 0.025)


# ---------------------------------------------------------------------------- phase M-step branch
def test_phase_mstep_keeps_old_phase_where_the_product_is_zero():
    """Where y~_i conj(z_i) = 0 the angle is undefined and the old phase stays (per pixel), and
    a tile whose summed product is 0 keeps its pixels' old phases (tiled)."""
    rng = _rng(31)
    n = 8
    a = o.aperture(n, 8.0)
    y = _crandn(rng, n, n)
    mu = _crandn(rng, n, n)
    old = np.where(a, rng.uniform(-3, 3, (n, n)), 0.0)
    zero = np.zeros((n, n), bool)
    zero[2, 3] = zero[4, 4] = zero[5, 1] = True
    assert np.all(a[zero])
    y0 = np.where(zero, 0.0, y)
    phi, z = o.phase_mstep(y0, mu, old, a)
    assert np.array_equal(phi[zero], old[zero])
    expect = np.angle(y0 * np.conj(np.fft.fft2(mu, norm="ortho")))
    on = a & ~zero
    assert np.allclose(phi[on], expect[on], atol=1e-12)
    # tiled: zero the whole 2x2 tile (rows 2-3, cols 2-3) of y
    y1 = y.copy()
    y1[2:4, 2:4] = 0.0
    phi_t, _ = o.phase_mstep(y1, mu, old, a, block=2)
    assert np.array_equal(phi_t[2:4, 2:4], old[2:4, 2:4])
    assert not np.array_equal(phi_t[0:2, 2:4][a[0:2, 2:4]], old[0:2, 2:4][a[0:2, 2:4]])


# ---------------------------------------------------------------------------- frame orchestration
def _icd_bruteforce(r0, s, prm):
    """One 4-colour ICD sweep by dense scan plus golden-section refinement of every pixel's
    surrogate, neighbours and weights enumerated explicitly (weights at the sweep's entry
    values, neighbour values as updated so far)."""
    n = r0.shape[0]
    r = r0.copy()
    grid = np.logspace(-8, 2, 100_001)
    for cx, cy in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        for yy in range(n):
            for xx in range(n):
                if xx % 2 != cx or yy % 2 != cy:
                    continue
                terms = []
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        y1, x1 = yy + dy, xx + dx
                        if (dy, dx) == (0, 0) or not (0 <= y1 < n and 0 <= x1 < n):
                            continue
                        bij = 1 / (4 + 2 * math.sqrt(2)) / (math.sqrt(2) if dy and dx else 1.0)
                        beta = bij * float(o.qggmrf_weight(np.array([r0[yy, xx] - r0[y1, x1]]), prm)[0])
                        terms.append((beta, r[y1, x1]))

                def h(v):
                    return np.log(v) + s[yy, xx] / v + sum(0.5 * b_ * (v - rj) ** 2 for b_, rj in terms)
                k = int(np.argmin(h(grid)))
                lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
                for _ in range(200):
                    m1, m2 = lo + 0.382 * (hi - lo), hi - 0.382 * (hi - lo)
                    lo, hi = (lo, m2) if h(m1) < h(m2) else (m1, hi)
                r[yy, xx] = max(0.5 * (lo + hi), prm.r_floor)
    return r


def _hand_frame(r_prev, phi_prev, y, prm, s2):
    """One frame of Fig. 1 unrolled by hand on a tiny grid with dense matrices: Normalize
    (Eq. 4), the tip/tilt fit over explicitly enumerated aperture pairs, the back-projection
    through the dense operator, Eq. 3, then N_k EM iterations in which the first E-step uses
    the r-init back-projection and later ones recompute it with the current phase, the phase
    M-step uses that iteration's E-step mean (not the updated r), and the r M-step is the ICD
    sweep from the iteration's entry r.  Returns (r, phi, z and C of the last iteration)."""
    n = prm.n
    M = n * n
    Fm = _dft_matrix_2d(n)
    c = (n - 1) / 2.0
    a = np.array([[(x - c) ** 2 + (yy - c) ** 2 <= (prm.aperture_diam / 2) ** 2 for x in range(n)]
                  for yy in range(n)])
    d = y - y.sum() / M
    yt = math.sqrt(M) * d / math.sqrt(float(np.sum(np.abs(d) ** 2)))
    dxs, dys = [], []
    for yy in range(n):
        for x in range(n):
            if x + 1 < n and a[yy, x] and a[yy, x + 1]:
                dxs.append(math.remainder(phi_prev[yy, x + 1] - phi_prev[yy, x], 2 * math.pi))
            if yy + 1 < n and a[yy, x] and a[yy + 1, x]:
                dys.append(math.remainder(phi_prev[yy + 1, x] - phi_prev[yy, x], 2 * math.pi))
    tx, ty = float(np.mean(dxs)), float(np.mean(dys))
    phi = np.zeros((n, n))
    for yy in range(n):
        for x in range(n):
            if a[yy, x]:
                phi[yy, x] = math.remainder(phi_prev[yy, x] - tx * (x - c) - ty * (yy - c), 2 * math.pi)

    def backproject(ph):
        A = np.diag((a * np.exp(1j * ph)).ravel()) @ Fm
        return (A.conj().T @ yt.ravel()).reshape(n, n)
    b = backproject(phi)
    r = np.maximum((1 - prm.lam) * r_prev + prm.lam * prm.alpha * np.abs(b) ** 2, prm.r_floor)
    for it in range(prm.n_k):
        if it > 0:
            b = backproject(phi)
        w = r / (r + s2)
        mu = w * b
        cvar = s2 * w
        s = np.abs(mu) ** 2 + cvar
        z = (Fm @ mu.ravel()).reshape(n, n)
        v = yt * np.conj(z)
        phi = np.where(a & (v != 0), np.angle(v), phi)
        r = _icd_bruteforce(r, s, prm)
    return r, phi, z, cvar, yt, a


@pytest.mark.parametrize("n_k", [1, 2])
def test_frame_step_matches_a_hand_unrolled_dense_frame(n_k):
    rng = _rng(40 + n_k)
    n = 8
    prm = o.Params(n=n, aperture_diam=6.0, n_k=n_k, noise_var=0.4, prior_sigma=0.3)
    a = o.aperture(n, 6.0)
    y = (3.0 * _crandn(rng, n, n) + 0.5).astype(np.complex64).astype(np.complex128)
    r_prev = rng.uniform(0.05, 1.5, (n, n))
    phi_prev = np.where(a, rng.uniform(-math.pi, math.pi, (n, n)), 0.0)
    st, _ = o.step(o.State(r=r_prev.copy(), phi=phi_prev.copy(), n=3), y, prm)
    r_h, phi_h, _, _, _, _ = _hand_frame(r_prev, phi_prev, y, prm, prm.noise_var)
    assert st.n == 4
    assert np.allclose(st.r, r_h, rtol=2e-7)
    assert np.allclose(o.wrap(st.phi - phi_h)[a], 0.0, atol=1e-7)  # r by golden section: ~1e-8
    assert np.all(st.phi[~a] == 0.0)
    if n_k == 1:
        # the discriminating power of this pin: phi from the updated r's posterior mean differs
        yt, _ = o.normalize(y)
        phi_t, _ = o.remove_tip_tilt(phi_prev, a)
        b = o.adjoint_op(yt, phi_t, a)
        alt, _ = o.phase_mstep(yt, st.r / (st.r + prm.noise_var) * b, phi_t, a)
        assert np.max(np.abs(o.wrap(alt - phi_h)[a])) > 1e-3


def test_noise_mstep_runs_after_the_last_em_iteration_and_feeds_the_next_frame():
    """With the sigma^2 M-step on: after frame 1's last EM iteration sigma^2 becomes
    mean_P |y~ - e^{j phi} z|^2 + mean(C) at the new phase (z, C of that iteration), and
    frame 2's E-steps use it."""
    rng = _rng(50)
    n = 8
    prm = o.Params(n=n, aperture_diam=6.0, n_k=2, noise_var=0.4, prior_sigma=0.3, noise_update=1)
    a = o.aperture(n, 6.0)
    ys = [(3.0 * _crandn(rng, n, n) + 0.5) for _ in range(2)]
    r_prev = rng.uniform(0.05, 1.5, (n, n))
    phi_prev = np.where(a, rng.uniform(-math.pi, math.pi, (n, n)), 0.0)
    st1, _ = o.step(o.State(r=r_prev.copy(), phi=phi_prev.copy(), n=0), ys[0], prm)
    r1, phi1, z1, c1, yt1, a1 = _hand_frame(r_prev, phi_prev, ys[0], prm, prm.noise_var)
    s2 = float(np.sum(np.abs(yt1 - np.exp(1j * phi1) * z1)[a1] ** 2)) / float(a1.sum()) + float(c1.mean())
    assert st1.noise_var == pytest.approx(s2, rel=1e-7)  # r by golden section: ~1e-8
    st2, _ = o.step(st1, ys[1], prm)
    r2, phi2, _, _, _, _ = _hand_frame(st1.r, st1.phi, ys[1], prm, s2)
    assert np.allclose(st2.r, r2, rtol=2e-7)
    assert np.allclose(o.wrap(st2.phi - phi2)[a], 0.0, atol=1e-7)
