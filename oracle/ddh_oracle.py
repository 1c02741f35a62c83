"""FP64 CPU oracle for the per-frame Dynamic DH-MBIR step.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct statement of what
the GPU path computes; only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import it.  It shares no code with the CUDA library and imports nothing from it.

Every function follows one passage of the paper (Sheikh, Pellizzari, Kisner, Buzzard, Bouman,
"Dynamic DH-MBIR for Phase-Error Estimation from Streaming Digital-Holography Data",
arXiv:2305.03284).  The paper defers the EM equations and both priors to earlier work, so the
E-step, the two M-steps and the reflectance prior below are the standard Gaussian-posterior EM
reading of its forward model (Eq. 1, Sec. 2) and MAP objective (Eq. 2):

* operator: ``A_phi = D_a D(exp(j phi)) F`` (Sec. 2, Fresnel factor taken as identity because a
  diagonal unitary is absorbed by the circularly-symmetric reflection coefficients);
* E-step with ``A^H A ~ I``: ``w = r/(r+s2)``, ``mu = w b``, ``C = s2 w``, ``s = |mu|^2 + C``;
* reflectance M-step: one 4-colour ICD sweep of ``sum_i log r_i + s_i/r_i`` plus a q-GGMRF
  8-neighbour prior, majorised by the symmetric-bound quadratic surrogate formed once at the
  sweep's entry values; each pixel minimises a 1-D function whose stationarity condition is the
  cubic ``W r^3 - C r^2 + r - s = 0``;
* phase M-step: ``phi_i = angle(y_i conj(z_i))`` on the aperture, ``z = F mu`` (or, with the
  phase held constant on G x G tiles, the angle of the tile sum of ``y conj(z)``; optionally
  under a Gaussian MRF prior on the wrapped differences of neighbouring tiles, minimised by
  majorised ICD sweeps);
* optional sigma^2 M-step, once per frame after its last EM iteration: ``E||y - A g||^2 / |P|``
  over the posterior of g; the next frame's E-steps use the new value;
* loop (Fig. 1): Normalize (Eq. 4), RemoveTipTilt, r-init (Eq. 3), ``N_k`` EM iterations.

Arithmetic is float64 throughout; the input frame is the complex64 frame promoted to complex128.

Parity status: the FFT, operator, Normalize, RemoveTipTilt, E-step, cubic/ICD, surrogate,
phase M-step and Strehl functions are each pinned by tests against closed forms, brute force or
the exact posterior (see the oracle tests).  The prior-weighted tile-phase M-step is pinned by
monotone descent of its per-pixel cost, stationarity at its fixed point (finite differences)
and a two-tile closed form; the sigma^2 M-step by the exact-fit case, the sample noise power
over the pupil, and convergence of EM to the maximum-likelihood variance.  The r-init blend is
pinned by hand-computed values with a non-zero previous state; one whole frame (Normalize,
tip/tilt, back-projection, Eq. 3, N_k = 1 and 2 EM iterations, the sigma^2 M-step and its use
in the next frame) by a hand-unrolled dense-matrix frame on an 8 x 8 grid.  The multi-frame
trajectory has no printed per-frame values in the paper; it is pinned to the paper's reported
outcome only (Sec. 5.C: Strehl 0.8 reached within 150 frames at the Sec. 5.A parameters, which
the oracle's trajectory reproduces on the bar-chart stream with the tracking parameter set);
beyond that and the pins above it is *parity unpinned*.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

# 8-neighbour weights summing to one: orthogonal 1/(4 + 2 sqrt 2), diagonal that / sqrt 2
B_NN = 1.0 / (4.0 + 2.0 * math.sqrt(2.0))
B_DIAG = B_NN / math.sqrt(2.0)
NEIGHBOURS = [(-1, 0, B_NN), (1, 0, B_NN), (0, -1, B_NN), (0, 1, B_NN),
              (-1, -1, B_DIAG), (-1, 1, B_DIAG), (1, -1, B_DIAG), (1, 1, B_DIAG)]  # (dy, dx, b)
COLOURS = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (x % 2, y % 2) in sweep order


@dataclass(frozen=True)
class Params:
    """Mirror of the C ``ddh_params`` struct (all quantities in normalised units)."""
    n: int
    aperture_diam: float
    lam: float = 0.45            # Eq. 3 lambda (Sec. 5.B)
    alpha: float = 0.025         # Eq. 3 alpha (Sec. 5.B)
    n_k: int = 1                 # EM iterations per frame (Fig. 1)
    noise_var: float = 0.3       # sigma^2 after Normalize
    prior_p: float = 1.1
    prior_q: float = 2.0
    prior_T: float = 1.0
    prior_sigma: float = 0.1
    r_floor: float = 1e-10
    tilt_mode: int = 1           # 1: RemoveTipTilt each frame, 0: skip
    phase_block: int = 1         # 1: per-pixel phase; G > 1: phase constant on G x G blocks
    phase_prior: float = 0.0     # precision 1/sigma_phi^2 of the tile-phase GMRF (0: flat prior)
    phase_sweeps: int = 2        # ICD sweeps of the tile-phase M-step under that prior
    noise_update: int = 0        # 1: sigma^2 is re-estimated by an M-step every frame


@dataclass
class State:
    r: np.ndarray                # reflectance, N x N
    phi: np.ndarray              # phase, N x N (zero off the aperture)
    n: int = 0
    noise_var: float | None = None  # current sigma^2 estimate (noise_update); None: the parameter


@dataclass
class Trace:
    """Intermediates of one frame (for per-stage comparisons)."""
    stats: dict = field(default_factory=dict)
    y_norm: np.ndarray | None = None
    phi_tilt: np.ndarray | None = None
    b: np.ndarray | None = None
    r_init: np.ndarray | None = None
    mu: np.ndarray | None = None
    s: np.ndarray | None = None
    z: np.ndarray | None = None


def init_state(n: int) -> State:
    """Fig. 1: n <- 0, r <- 0, phi <- 0."""
    return State(r=np.zeros((n, n)), phi=np.zeros((n, n)), n=0)


# ---------------------------------------------------------------------------------------
# geometry, transforms, operator (Sec. 2)
# ---------------------------------------------------------------------------------------
def aperture(n: int, diam: float) -> np.ndarray:
    """Binary disc ``D_a``: centre ((n-1)/2, (n-1)/2), diameter ``diam`` px (Sec. 2)."""
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    return ((xx - c) ** 2 + (yy - c) ** 2) <= (diam / 2.0) ** 2


def fft2u(x: np.ndarray) -> np.ndarray:
    """Normalised (unitary) 2D DFT ``F`` (Sec. 2), kernel exp(-j 2 pi k.x / N) / N."""
    return np.fft.fft2(np.asarray(x, np.complex128), norm="ortho")


def ifft2u(x: np.ndarray) -> np.ndarray:
    """``F^H``, the inverse of the unitary DFT."""
    return np.fft.ifft2(np.asarray(x, np.complex128), norm="ortho")


def forward_op(g: np.ndarray, phi: np.ndarray, a: np.ndarray) -> np.ndarray:
    """``A_phi g = D_a D(exp(j phi)) F g`` (Eq. 1 and Sec. 2)."""
    return a * np.exp(1j * phi) * fft2u(g)


def adjoint_op(y: np.ndarray, phi: np.ndarray, a: np.ndarray) -> np.ndarray:
    """``A_phi^H y = F^H D(exp(-j phi)) D_a y``."""
    return ifft2u(a * np.exp(-1j * phi) * y)


def wrap(d: np.ndarray) -> np.ndarray:
    """Map angles into (-pi, pi]."""
    w = np.mod(d + math.pi, 2.0 * math.pi) - math.pi
    return np.where(w == -math.pi, math.pi, w)


# ---------------------------------------------------------------------------------------
# per-frame pre-conditioning (Fig. 1, Eq. 4, Sec. 4)
# ---------------------------------------------------------------------------------------
def normalize(y: np.ndarray) -> tuple[np.ndarray, dict]:
    """Eq. 4: ``sqrt(p) (y - mu)/||y - mu||`` with ``mu`` the mean over all ``p`` entries."""
    y = np.asarray(y, np.complex128)
    p = y.size
    mu = y.mean()
    d = y - mu
    nrm = math.sqrt(float(np.sum(np.abs(d) ** 2)))
    scale = math.sqrt(p) / nrm
    return scale * d, {"mean": mu, "scale": scale}


def tip_tilt(phi: np.ndarray, a: np.ndarray) -> tuple[float, float]:
    """Least-squares constant gradient of the wrapped neighbour phase differences over the
    aperture pairs (the RemoveTipTilt regression, Sec. 4): the mean x- and y-difference."""
    px = a[:, :-1] & a[:, 1:]
    py = a[:-1, :] & a[1:, :]
    dx = wrap(phi[:, 1:] - phi[:, :-1])[px]
    dy = wrap(phi[1:, :] - phi[:-1, :])[py]
    tx = float(dx.mean()) if dx.size else 0.0
    ty = float(dy.mean()) if dy.size else 0.0
    return tx, ty


def remove_tip_tilt(phi: np.ndarray, a: np.ndarray) -> tuple[np.ndarray, tuple[float, float]]:
    """RemoveTipTilt (Fig. 1): subtract the fitted plane about the pupil centre, re-wrap, and
    keep the phase zero off the aperture.  Piston is left alone."""
    n = phi.shape[0]
    tx, ty = tip_tilt(phi, a)
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    out = wrap(phi - tx * (xx - c) - ty * (yy - c))
    return np.where(a, out, 0.0), (tx, ty)


# ---------------------------------------------------------------------------------------
# r-init and E-step (Eq. 3; EM of Sec. 3)
# ---------------------------------------------------------------------------------------
def r_init(r_prev: np.ndarray, b: np.ndarray, prm: Params) -> np.ndarray:
    """Eq. 3: ``(1 - lambda) r_{n-1} + lambda alpha |A^H y|^2``, floored at ``r_floor``."""
    r = (1.0 - prm.lam) * r_prev + prm.lam * prm.alpha * np.abs(b) ** 2
    return np.maximum(r, prm.r_floor)


def estep(r: np.ndarray, b: np.ndarray, prm: Params):
    """Posterior of g given y under A^H A ~ I: mean ``w b``, variance ``s2 w``,
    and second moment ``s = |mu|^2 + C``."""
    w = r / (r + prm.noise_var)
    mu = w * b
    cvar = prm.noise_var * w
    s = np.abs(mu) ** 2 + cvar
    return mu, s, w


# ---------------------------------------------------------------------------------------
# reflectance prior and M-step
# ---------------------------------------------------------------------------------------
def qggmrf_rho(delta, prm: Params):
    """q-GGMRF potential ``|D|^p/(p s^p) * u/(1+u)``, ``u = |D/(T s)|^(q-p)``."""
    p, q, T, sg = prm.prior_p, prm.prior_q, prm.prior_T, prm.prior_sigma
    ad = np.abs(np.asarray(delta, np.float64))
    u = (ad / (T * sg)) ** (q - p)
    return ad ** p / (p * sg ** p) * u / (1.0 + u)


def qggmrf_weight(delta, prm: Params):
    """``rho'(D)/D = |D|^(p-2) s^(-p) u (q/p + u)/(1+u)^2``; at D = 0 (q = 2) its limit
    ``2/(p s^2 T^(2-p))``.  Twice the symmetric-bound surrogate coefficient."""
    p, q, T, sg = prm.prior_p, prm.prior_q, prm.prior_T, prm.prior_sigma
    ad = np.abs(np.asarray(delta, np.float64))
    out = np.empty_like(ad)
    nz = ad > 0
    u = (ad[nz] / (T * sg)) ** (q - p)
    out[nz] = ad[nz] ** (p - 2.0) * sg ** (-p) * u * (q / p + u) / (1.0 + u) ** 2
    if q != 2.0 and np.any(~nz):
        raise ValueError("the surrogate weight at zero difference is finite only for q = 2")
    out[~nz] = 2.0 / (p * sg ** 2 * T ** (2.0 - p))
    return out


def prior_energy(r: np.ndarray, prm: Params) -> float:
    """``sum over unordered 8-neighbour pairs of b_ij rho(r_i - r_j)`` (free boundary)."""
    e = 0.0
    for dy, dx, bij in [(0, 1, B_NN), (1, 0, B_NN), (1, 1, B_DIAG), (1, -1, B_DIAG)]:
        a_, b_ = _pair_views(r, dy, dx)
        e += bij * float(np.sum(qggmrf_rho(a_ - b_, prm)))
    return e


def _pair_views(x, dy, dx):
    """(x[i], x[i + (dy, dx)]) for all i whose neighbour lies inside the grid."""
    n0, n1 = x.shape
    ys0, ys1 = (slice(0, n0 - dy), slice(dy, n0)) if dy >= 0 else (slice(-dy, n0), slice(0, n0 + dy))
    xs0, xs1 = (slice(0, n1 - dx), slice(dx, n1)) if dx >= 0 else (slice(-dx, n1), slice(0, n1 + dx))
    return x[ys0, xs0], x[ys1, xs1]


def _neighbour(x, dy, dx, fill=0.0):
    """Array whose entry i is x[i + (dy, dx)] (``fill`` where that lies off the grid)."""
    n0, n1 = x.shape
    out = np.full_like(x, fill)
    ys_dst = slice(max(0, -dy), n0 - max(0, dy))
    xs_dst = slice(max(0, -dx), n1 - max(0, dx))
    ys_src = slice(max(0, dy), n0 - max(0, -dy))
    xs_src = slice(max(0, dx), n1 - max(0, -dx))
    out[ys_dst, xs_dst] = x[ys_src, xs_src]
    return out


def _inside(n, dy, dx):
    m = np.zeros((n, n), bool)
    m[max(0, -dy): n - max(0, dy), max(0, -dx): n - max(0, dx)] = True
    return m


def cubic_argmin(W, C, s, E=None):
    """Per pixel: the positive real root of ``W r^3 - C r^2 + r - s`` that minimises
    ``h(r) = log r + s/r + W r^2/2 - C r`` (ties: the smaller root); ``r = s`` where W = 0.

    Roots come from the eigenvalues of the monic companion matrix (a library eigen-solver
    serves as the root finder).  ``E`` (the r-independent part of h) does not affect the
    choice and is ignored.
    """
    W = np.asarray(W, np.float64)
    C = np.asarray(C, np.float64)
    s = np.asarray(s, np.float64)
    out = s.copy()
    pos = W > 0
    if not np.any(pos):
        return out
    w, c, sv = W[pos], C[pos], s[pos]
    comp = np.zeros((w.size, 3, 3))
    comp[:, 0, 0] = c / w          # -a2
    comp[:, 0, 1] = -1.0 / w       # -a1
    comp[:, 0, 2] = sv / w         # -a0
    comp[:, 1, 0] = 1.0
    comp[:, 2, 1] = 1.0
    roots = np.linalg.eigvals(comp)
    real = np.abs(roots.imag) <= 1e-7 * np.maximum(1.0, np.abs(roots.real))
    rr = roots.real
    ok = real & (rr > 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.log(np.where(ok, rr, 1.0)) + sv[:, None] / np.where(ok, rr, 1.0) \
            + 0.5 * w[:, None] * rr ** 2 - c[:, None] * rr
    h = np.where(ok, h, np.inf)
    # ties go to the smaller root: sort candidates by value first, argmin takes the first
    order = np.argsort(np.where(ok, rr, np.inf), axis=1)
    h_sorted = np.take_along_axis(h, order, axis=1)
    r_sorted = np.take_along_axis(rr, order, axis=1)
    pick = np.argmin(h_sorted, axis=1)
    best = r_sorted[np.arange(w.size), pick]
    if not np.all(np.isfinite(np.min(h_sorted, axis=1))):
        raise FloatingPointError("cubic without a positive real root (s must be > 0)")
    out[pos] = best
    return out


def icd_sweep(r_entry: np.ndarray, s: np.ndarray, prm: Params) -> np.ndarray:
    """One 4-colour ICD sweep of the r M-step.

    The surrogate weights ``beta_ij = b_ij rho'(D)/D`` are formed once from the entry values;
    pixels of one colour (x%2, y%2) are updated together from the current neighbour values
    (colours (0,0), (1,0), (0,1), (1,1) in that order); each takes the minimiser of
    ``log r + s_i/r + sum_j beta_ij/2 (r - r_j)^2`` and is floored at ``r_floor``.
    """
    n = r_entry.shape[0]
    yy, xx = np.mgrid[0:n, 0:n]
    betas = []
    for dy, dx, bij in NEIGHBOURS:
        inside = _inside(n, dy, dx)
        rn = _neighbour(r_entry, dy, dx)
        beta = np.where(inside, bij * qggmrf_weight(r_entry - rn, prm), 0.0)
        betas.append(beta)
    W = np.sum(betas, axis=0)
    r = r_entry.copy()
    for cx, cy in COLOURS:
        sel = (xx % 2 == cx) & (yy % 2 == cy)
        Cn = np.zeros((n, n))
        for (dy, dx, _), beta in zip(NEIGHBOURS, betas):
            Cn += beta * _neighbour(r, dy, dx)
        root = cubic_argmin(W[sel], Cn[sel], s[sel])
        r[sel] = np.maximum(root, prm.r_floor)
    return r


# ---------------------------------------------------------------------------------------
# phase M-step
# ---------------------------------------------------------------------------------------
def phase_mstep(y_norm: np.ndarray, mu: np.ndarray, phi_old: np.ndarray, a: np.ndarray, block: int = 1):
    """Minimise ``sum_i a_i |y_i - exp(j phi_i) z_i|^2`` with ``z = F mu``.

    Per-pixel phase (``block == 1``): ``phi_i = angle(y_i conj(z_i))`` on the aperture.
    Phase constant on aligned ``block x block`` tiles: ``phi_B = angle(sum_{i in B} a_i y_i
    conj(z_i))``, the exact minimiser over one tile.  Where the (summed) product is 0 the old
    value is kept; the phase is zero off the aperture.  Returns (phi, z)."""
    z = fft2u(mu)
    v = np.where(a, y_norm * np.conj(z), 0.0)
    if block > 1:
        n = v.shape[0]
        vb = v.reshape(n // block, block, n // block, block).sum(axis=(1, 3))
        v = np.kron(vb, np.ones((block, block)))
    phi = np.where(v != 0, np.angle(v), phi_old)
    return np.where(a, phi, 0.0), z


# ---------------------------------------------------------------------------------------
# tile-phase M-step under a GMRF phase prior, and the sigma^2 M-step (extensions: the paper
# names p(phi) in Eq. 2 but defers its form; the noise variance is a parameter of Eq. 1)
# ---------------------------------------------------------------------------------------
NOISE_FLOOR = 1e-6  # lower bound on the re-estimated sigma^2 (normalised units)


def phase_tile_sums(y_norm: np.ndarray, z: np.ndarray, a: np.ndarray, block: int):
    """Per aligned ``block x block`` tile t: ``v_t = sum_{i in t} a_i y_i conj(z_i)`` and
    whether the tile holds an aperture pixel."""
    n = y_norm.shape[0]
    nt = n // block
    v = np.where(a, y_norm * np.conj(z), 0.0)
    vt = v.reshape(nt, block, nt, block).sum(axis=(1, 3))
    has_ap = np.asarray(a, bool).reshape(nt, block, nt, block).any(axis=(1, 3))
    return vt, has_ap


def phase_prior_icd(vt: np.ndarray, active: np.ndarray, s2: float, lam: float, sweeps: int,
                    start: np.ndarray) -> np.ndarray:
    """Minimise over the active tiles' phases
        f(phi) = -(2/s2) sum_t |v_t| cos(phi_t - angle v_t)
                 + (lam/2) sum_{t~s} b_ts wrap(phi_t - phi_s)^2
    (the EM data term of Eq. 1 with ``A^H A`` independent of phi, and a Gaussian MRF on the
    wrapped differences of 8-neighbour active tiles, weights as the reflectance prior's) by
    ``sweeps`` 4-colour ICD sweeps from ``start``.  Each tile minimises a quadratic majoriser
    of its 1-D function at the current value: ``1 - cos x`` by its symmetric bound
    ``sin(x0)/(2 x0) x^2`` (+ const) about ``x0 = wrap(phi_t - angle v_t)``, and each
    ``wrap(d)^2`` by ``(d - 2 pi k)^2`` with k its current branch; the minimiser is wrapped
    into (-pi, pi].  A tile whose majoriser has zero curvature keeps its value."""
    nt = vt.shape[0]
    kap = 2.0 * np.abs(vt) / s2
    th = np.angle(vt)
    pt = np.array(start, np.float64, copy=True)
    for _ in range(sweeps):
        for cx, cy in COLOURS:
            for T in range(cy, nt, 2):
                for X in range(cx, nt, 2):
                    if not active[T, X]:
                        continue
                    p0 = pt[T, X]
                    x0 = float(wrap(p0 - th[T, X]))
                    c0 = 0.5 if x0 == 0.0 else math.sin(x0) / (2.0 * x0)
                    wsum = ssum = 0.0
                    for dy, dx, bij in NEIGHBOURS:
                        T2, X2 = T + dy, X + dx
                        if 0 <= T2 < nt and 0 <= X2 < nt and active[T2, X2]:
                            wsum += bij
                            ssum += bij * (p0 - float(wrap(p0 - pt[T2, X2])))
                    den = 2.0 * kap[T, X] * c0 + lam * wsum
                    if den > 0.0:
                        pt[T, X] = float(wrap((2.0 * kap[T, X] * c0 * (p0 - x0) + lam * ssum) / den))
    return pt


def phase_map_objective(phi: np.ndarray, y_norm: np.ndarray, z: np.ndarray, a: np.ndarray, s2: float,
                        block: int, lam: float, active: np.ndarray) -> float:
    """The phase M-step's cost, per pixel: ``-(2/s2) sum_{i in P} Re(conj(y_i) e^{j phi_i} z_i)``
    plus the prior of ``phase_prior_icd`` on the tile values of ``phi`` (constant on tiles)."""
    ab = np.asarray(a, bool)
    data = -2.0 / s2 * float(np.sum(np.real(np.conj(y_norm) * np.exp(1j * phi) * z)[ab]))
    nt = phi.shape[0] // block
    cnt = ab.reshape(nt, block, nt, block).sum(axis=(1, 3))
    tot = np.where(ab, phi, 0.0).reshape(nt, block, nt, block).sum(axis=(1, 3))
    pt = np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0)  # the tile value at its aperture pixels
    e = 0.0
    for dy, dx, bij in [(0, 1, B_NN), (1, 0, B_NN), (1, 1, B_DIAG), (1, -1, B_DIAG)]:
        p1, p2 = _pair_views(pt, dy, dx)
        m1, m2 = _pair_views(active, dy, dx)
        e += bij * float(np.sum(np.where(m1 & m2, wrap(p1 - p2) ** 2, 0.0)))
    return data + 0.5 * lam * e


def phase_mstep_prior(y_norm: np.ndarray, mu: np.ndarray, phi_old: np.ndarray, a: np.ndarray, block: int,
                      lam: float, s2: float, sweeps: int):
    """Tile-phase M-step under the GMRF phase prior: start from the prior-free tile angles
    (``phase_mstep``), then ``phase_prior_icd`` over the tiles that hold an aperture pixel and a
    non-zero tile sum; their aperture pixels take the tile value.  ``lam = 0`` is
    ``phase_mstep``.  Returns (phi, z)."""
    phi, z = phase_mstep(y_norm, mu, phi_old, a, block)
    if lam <= 0.0:
        return phi, z
    vt, has_ap = phase_tile_sums(y_norm, z, a, block)
    active = has_ap & (vt != 0)
    pt = phase_prior_icd(vt, active, s2, lam, sweeps, np.angle(vt))
    on = np.kron(active, np.ones((block, block), bool)) & np.asarray(a, bool)
    return np.where(on, np.kron(pt, np.ones((block, block))), phi), z


def noise_mstep(y_norm: np.ndarray, z: np.ndarray, phi: np.ndarray, a: np.ndarray, cvar: np.ndarray) -> float:
    """EM update of sigma^2 under Eq. 1 (noise CN(0, sigma^2) on the P measured pupil pixels):
    ``E||y - A g||^2 / |P|`` over the posterior of g, with ``A = D_a D(e^{j phi}) F``:
    ``(1/|P|) sum_{i in P} |y_i - e^{j phi_i} z_i|^2 + (1/M) sum_j C_jj`` (diagonal posterior
    covariance C, unitary F), floored at ``NOISE_FLOOR``."""
    ab = np.asarray(a, bool)
    res = float(np.sum(np.abs(y_norm - np.exp(1j * phi) * z)[ab] ** 2)) / float(ab.sum())
    return max(res + float(np.mean(cvar)), NOISE_FLOOR)


# ---------------------------------------------------------------------------------------
# one frame of DDH-MBIR (Fig. 1)
# ---------------------------------------------------------------------------------------
def step(state: State, y: np.ndarray, prm: Params) -> tuple[State, Trace]:
    """ReadData -> Normalize -> RemoveTipTilt -> r-init (Eq. 3) -> N_k x EM -> WriteData."""
    a = aperture(prm.n, prm.aperture_diam)
    tr = Trace()
    yt, st = normalize(y)
    tr.stats = dict(st)
    tr.y_norm = yt
    if prm.tilt_mode:
        phi, (tx, ty) = remove_tip_tilt(state.phi, a)
    else:
        phi, (tx, ty) = np.where(a, state.phi, 0.0), (0.0, 0.0)
    tr.stats.update(tx=tx, ty=ty)
    tr.phi_tilt = phi
    b = adjoint_op(yt, phi, a)
    tr.b = b
    r = r_init(state.r, b, prm)
    tr.r_init = r
    s2 = state.noise_var if (prm.noise_update and state.noise_var is not None) else prm.noise_var
    pe = replace(prm, noise_var=s2)
    for it in range(prm.n_k):
        if it > 0:
            b = adjoint_op(yt, phi, a)
        mu, s, w = estep(r, b, pe)
        r_new = icd_sweep(r, s, pe)
        if prm.phase_prior > 0.0:
            phi, z = phase_mstep_prior(yt, mu, phi, a, prm.phase_block, prm.phase_prior, s2, prm.phase_sweeps)
        else:
            phi, z = phase_mstep(yt, mu, phi, a, prm.phase_block)
        if prm.noise_update and it == prm.n_k - 1:  # once per frame, after its last EM iteration
            s2 = noise_mstep(yt, z, phi, a, s2 * w)
        r = r_new
        if it == 0:
            tr.mu, tr.s, tr.z = mu, s, z
    nv = s2 if prm.noise_update else state.noise_var
    return State(r=r, phi=phi, n=state.n + 1, noise_var=nv), tr


def run(y_frames, prm: Params, state: State | None = None):
    """Run a stream of frames; returns the final state and the per-frame (r, phi)."""
    st = state if state is not None else init_state(prm.n)
    rs, phis = [], []
    for y in y_frames:
        st, _ = step(st, y, prm)
        rs.append(st.r)
        phis.append(st.phi)
    return st, np.array(rs), np.array(phis)


# ---------------------------------------------------------------------------------------
# evaluation (Sec. 5.B)
# ---------------------------------------------------------------------------------------
def strehl(phi_hat: np.ndarray, phi_true: np.ndarray, a: np.ndarray) -> float:
    """Peak Strehl ratio: ``max |F^H(a exp(j(phi - phi_hat)))|^2 / max |F^H a|^2``."""
    num = np.max(np.abs(ifft2u(a * np.exp(1j * (phi_true - phi_hat)))) ** 2)
    den = np.max(np.abs(ifft2u(a.astype(np.float64))) ** 2)
    return float(num / den)


def em_objective_unit_aperture(r, phi, y_norm, prm: Params) -> float:
    """MAP cost of Eq. 2 (up to constants) when the aperture is the whole grid, so that A is
    unitary: ``sum log(r + s2) + |b|^2/(r + s2) + prior``, ``b = F^H(exp(-j phi) y)``."""
    b = ifft2u(np.exp(-1j * phi) * y_norm)
    v = r + prm.noise_var
    return float(np.sum(np.log(v) + np.abs(b) ** 2 / v)) + prior_energy(r, prm)


def em_static_step(r, phi, y_norm, prm: Params, a=None):
    """One plain EM iteration ``EM(r, phi; y)`` of the static DH-MBIR loop (Sec. 3)."""
    if a is None:
        a = aperture(prm.n, prm.aperture_diam)
    b = adjoint_op(y_norm, phi, a)
    mu, s, _ = estep(r, b, prm)
    r_new = np.maximum(icd_sweep(r, s, prm), prm.r_floor)
    phi_new, _ = phase_mstep(y_norm, mu, phi, a, prm.phase_block)
    return r_new, phi_new


def default_params(n: int, aperture_diam: float, snr: float, **kw) -> Params:
    """Parameters with ``noise_var = 1/(1 + f SNR)``, f the aperture fill fraction."""
    f = float(aperture(n, aperture_diam).mean())
    return replace(Params(n=n, aperture_diam=aperture_diam, noise_var=1.0 / (1.0 + f * snr)), **kw)
