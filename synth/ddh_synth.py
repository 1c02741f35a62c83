"""Seeded synthetic streams of single-shot digital-holography frames.

This module only *produces inputs*: it holds none of the EM method's arithmetic and is
imported by both the FP64 oracle tests and the GPU path's tests/benchmarks, never by either
implementation.  It stands in for the paper's simulation (Sec. 5.A), whose reflectance (the
1951 USAF chart) is replaced by a seeded smooth random field or a seeded bar chart:

* reflectance ``r_true``: the image plane is zero-padded 2x, so the object occupies the central
  ``N/2 x N/2`` block: a periodic Gaussian filter (sigma = 3 px) of U[0, 1] noise on that block,
  rescaled to [0, 1], and zero elsewhere (``obj="smooth"``); or (``obj="bars"``) a seeded bar
  chart on that block, the structure of the paper's resolution-chart object: ``bars`` bright
  rectangles (reflectance 1; widths 2 to N/32 px, lengths N/20 to N/6 px, horizontal or
  vertical at seeded positions) on a dark (0) background;
* phase: a Kolmogorov screen made by the spectral (FFT) method on an ``L x L`` periodic grid,
  phase PSD ``0.023 r0^(-5/3) f^(-11/3)`` (f in cycles/px, r0 in px), structure function
  ``6.88 (rho/r0)^(5/3)``;
* frozen flow: the screen is shifted by ``n * v`` px at frame ``n`` (Fourier shift), cropped to
  ``N x N``, and piston/tip/tilt are removed by least squares over the aperture (Sec. 5.A);
* frames: ``g_n ~ CN(0, r_true)`` drawn independently per frame, and
  ``y_n = a * exp(j phi_n) * F g_n + w_n`` with ``F`` the unitary 2D DFT (Eq. 1 and the
  isoplanatic decomposition of Sec. 2, the Fresnel factor taken as identity), ``w_n ~ CN(0,
  mean(r_true)/SNR)`` on the whole grid (SNR is a linear power ratio: ``mean(r_true)`` over the
  whole grid is the signal power per pupil pixel);
* frozen-flow speed: ``|v| = (1/0.43) (f_g/f_s) N/(D/r0)`` px/frame (Sec. 5.A).

Seeding: configuration ``k``, stream ``s``: static parts (reflectance, screen, wind angle) use
``SeedSequence([k, s, 0])``; frame ``n`` uses ``SeedSequence([k, s, n + 1])``.  Frames are
returned as complex64 (the single cast both implementations start from) and the true phase as
float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

try:  # scipy's FFT is multithreaded; numpy's is the fallback on hosts without scipy
    import scipy.fft as _fft

    def _irfft2(x, s):
        return _fft.irfft2(x, s=s, workers=-1)

    def _fft2u(x):
        return _fft.fft2(x, norm="ortho", workers=-1)
except ImportError:  # pragma: no cover
    def _irfft2(x, s):
        return np.fft.irfft2(x, s=s)

    def _fft2u(x):
        return np.fft.fft2(x, norm="ortho")


KOLMOGOROV_PSD = 0.023  # phase PSD constant (f in cycles per unit length)


@dataclass(frozen=True)
class StreamConfig:
    n: int                      # grid side N
    aperture_diam: float        # pupil diameter in px
    d_over_r0: float            # turbulence strength D/r0
    wind: float                 # frozen-flow speed |v| in px/frame
    wind_angle: float | None    # direction (rad, x right / y down); None = seeded
    snr: float                  # linear signal-to-noise power ratio over the aperture
    frames: int                 # frames the stream must be able to produce
    config_id: int
    stream_id: int = 0
    refl_sigma_px: float = 3.0
    rate_khz: float = 0.0       # frame arrival rate (streaming-service workload only)
    obj: str = "smooth"         # reflectance: "smooth" random field or "bars" (a bar chart)
    bars: int = 16              # bright bars of the "bars" object
    obj_seed: int | None = None # seed of the object; None: the stream's static seed


def config_single_64(frames: int = 20) -> StreamConfig:
    """Single stream, 64x64 grid, 32 px pupil, D/r0 = 10, 0.5 px/frame down-right, SNR 10."""
    return StreamConfig(n=64, aperture_diam=32.0, d_over_r0=10.0, wind=0.5,
                        wind_angle=math.pi / 4, snr=10.0, frames=frames, config_id=1)


def config_single_256(frames: int = 1000) -> StreamConfig:
    """Single stream, 256x256 grid, 128 px pupil, D/r0 = 15, 1 px/frame seeded angle, SNR 5."""
    return StreamConfig(n=256, aperture_diam=128.0, d_over_r0=15.0, wind=1.0,
                        wind_angle=None, snr=5.0, frames=frames, config_id=2)


def config_batched(frames: int = 200) -> list[StreamConfig]:
    """64 independent streams: 32 x 128^2, 24 x 256^2, 8 x 512^2, pupil = grid/2.

    Per stream (seeded): D/r0 ~ U[5, 20], wind ~ U[0.25, 2] px/frame, angle ~ U[0, 2 pi).
    SNR is the paper's 10 (Sec. 5.A).
    """
    rng = np.random.default_rng(np.random.SeedSequence([3, 999_999]))
    sizes = [128] * 32 + [256] * 24 + [512] * 8
    out = []
    for s, n in enumerate(sizes):
        out.append(StreamConfig(n=n, aperture_diam=n / 2, d_over_r0=float(rng.uniform(5, 20)),
                                wind=float(rng.uniform(0.25, 2.0)),
                                wind_angle=float(rng.uniform(0, 2 * math.pi)), snr=10.0,
                                frames=frames, config_id=3, stream_id=s))
    return out


def config_adjoint(small: bool = False, streams: int = 16, frames: int = 8) -> list[StreamConfig]:
    """Differentiation workload: 16 streams at 256^2 (or the 32^2, 16 px pupil copy)."""
    n, d = (32, 16.0) if small else (256, 128.0)
    return [StreamConfig(n=n, aperture_diam=d, d_over_r0=10.0, wind=0.5, wind_angle=math.pi / 4,
                         snr=10.0, frames=frames, config_id=4, stream_id=s)
            for s in range(streams)]


def config_service(sensors: int = 32, frames_total: int = 10_000) -> list[StreamConfig]:
    """Streaming-service workload: grids drawn from {128, 256, 512}, rates ~ U[0.5, 5] kHz."""
    rng = np.random.default_rng(np.random.SeedSequence([5, 999_999]))
    out = []
    per = max(1, frames_total // sensors)
    for s in range(sensors):
        n = int(rng.choice([128, 256, 512]))
        out.append(StreamConfig(n=n, aperture_diam=n / 2, d_over_r0=float(rng.uniform(5, 20)),
                                wind=float(rng.uniform(0.25, 2.0)),
                                wind_angle=float(rng.uniform(0, 2 * math.pi)), snr=10.0,
                                frames=per, config_id=5, stream_id=s,
                                rate_khz=float(rng.uniform(0.5, 5.0))))
    return out


def config_paper_256(sim: int = 0, frames: int = 150) -> StreamConfig:
    """The paper's simulation parameters (Sec. 5.A): N = 256, D/r0 = 10, frozen flow
    v = (0.421, 0.421) px/frame (down and to the right), SNR 10 dB (linear 10), the pupil of
    diameter N/2 on the 2x zero-padded grid, and a bar-chart object standing in for the 1951
    USAF chart (one chart for every simulation; `sim` seeds the turbulence, speckle and noise)."""
    vx, vy = paper_velocity()
    return StreamConfig(n=256, aperture_diam=128.0, d_over_r0=10.0, wind=math.hypot(vx, vy),
                        wind_angle=math.atan2(vy, vx), snr=10.0, frames=frames, config_id=7, stream_id=sim,
                        obj="bars", bars=16, obj_seed=7_000)


def velocity_magnitude(f_g: float, f_s: float, n: int, d_over_r0: float) -> float:
    """Frozen-flow displacement per sample in px (Sec. 5.A, scaled Tyson Eq. 4.15)."""
    return (1.0 / 0.43) * (f_g / f_s) * (n / d_over_r0)


def paper_velocity() -> tuple[float, float]:
    """Displacement for the paper's parameters (N=256, f_g=100 Hz, f_s=10 kHz, D/r0=10),
    flowing down and to the right: equal x and y components."""
    m = velocity_magnitude(100.0, 10_000.0, 256, 10.0)
    return (m / math.sqrt(2.0), m / math.sqrt(2.0))


def _bar_chart(m: int, bars: int, seed) -> np.ndarray:
    """An m x m bar chart: `bars` bright (1) rectangles on a dark (0) background, each of width
    2 .. m/16 px and length m/10 .. m/3 px, horizontal or vertical, at seeded positions."""
    rng = seed if isinstance(seed, np.random.Generator) else np.random.default_rng(np.random.SeedSequence([seed]))
    r = np.zeros((m, m))
    for _ in range(bars):
        w = int(rng.integers(2, max(3, m // 16)))
        h = int(rng.integers(m // 10, m // 3))
        x0 = int(rng.integers(0, m - w))
        y0 = int(rng.integers(0, m - h))
        if rng.random() < 0.5:
            r[y0:y0 + h, x0:x0 + w] = 1.0
        else:
            r[x0:x0 + w, y0:y0 + h] = 1.0
    return r


def _pupil(n: int, diam: float) -> np.ndarray:
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    return ((xx - c) ** 2 + (yy - c) ** 2) <= (diam / 2.0) ** 2


def _next_pow2(v: float) -> int:
    p = 1
    while p < v:
        p *= 2
    return p


class Stream:
    """One seeded synthetic sensor stream; frames are produced on demand."""

    def __init__(self, cfg: StreamConfig):
        self.cfg = cfg
        n = cfg.n
        rng = np.random.default_rng(np.random.SeedSequence([cfg.config_id, cfg.stream_id, 0]))
        # reflectance on the 2x zero-padded image plane: periodic Gaussian filter of U[0,1]
        # noise on the central N/2 x N/2 block, min-max to [0, 1]; zero outside the block
        m = n // 2
        u = rng.uniform(0.0, 1.0, size=(m, m))
        f = np.fft.fftfreq(m)
        g = np.exp(-2.0 * math.pi ** 2 * cfg.refl_sigma_px ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
        sm = np.real(np.fft.ifft2(np.fft.fft2(u) * g))
        self.r_true = np.zeros((n, n))
        if cfg.obj == "bars":
            self.r_true[n // 4: n // 4 + m, n // 4: n // 4 + m] = _bar_chart(m, cfg.bars, cfg.obj_seed
                                                                            if cfg.obj_seed is not None else rng)
        else:
            self.r_true[n // 4: n // 4 + m, n // 4: n // 4 + m] = (sm - sm.min()) / (sm.max() - sm.min())
        self.pupil = _pupil(n, cfg.aperture_diam)
        self.noise_var_raw = float(self.r_true.mean() / cfg.snr)
        angle = cfg.wind_angle if cfg.wind_angle is not None else float(rng.uniform(0, 2 * math.pi))
        self.velocity = (cfg.wind * math.cos(angle), cfg.wind * math.sin(angle))  # (x, y) px/frame
        # Kolmogorov screen on an L x L periodic grid (spectral method, Hermitian half-plane)
        L = _next_pow2(max(4 * n, n + cfg.wind * cfg.frames + 1))
        self.L = L
        self.r0_px = cfg.aperture_diam / cfg.d_over_r0
        fy = np.fft.fftfreq(L)[:, None]
        fx = np.fft.rfftfreq(L)[None, :]
        fr = np.sqrt(fx ** 2 + fy ** 2)
        with np.errstate(divide="ignore"):
            psd = KOLMOGOROV_PSD * self.r0_px ** (-5.0 / 3.0) * fr ** (-11.0 / 3.0)
        psd[0, 0] = 0.0
        # phi(x) = Re sum_k A_k xi_k exp(i 2 pi f.x) with |A_k|^2 = 2 PSD df^2 and
        # xi ~ CN(0,1) gives D(rho) = 2 int PSD (1 - cos 2 pi f.rho) d^2f.  The real part is
        # a Hermitian sum with E|H_k|^2 = |A_k|^2 / 2, which irfft2 synthesises from the half
        # plane (scaled by L^2).  irfft2 keeps only the Hermitian part of the kx = 0 and
        # kx = L/2 columns, halving their variance, so those columns are scaled by sqrt(2).
        xi = (rng.standard_normal(psd.shape) + 1j * rng.standard_normal(psd.shape)) / math.sqrt(2)
        amp = np.sqrt(2.0 * psd) / L
        amp[:, 0] *= math.sqrt(2.0)
        amp[:, -1] *= math.sqrt(2.0)
        self._spec_half = xi * amp * (L * L) / math.sqrt(2.0)
        self._fx = fx
        self._fy = fy
        # Low-frequency compensation (subharmonics, Lane et al. 1992): three levels of 3 x 3
        # frequency grids with spacing 1/(3^p L), centre excluded, same PSD and amplitudes.
        sh_f, sh_c = [], []
        for p in (1, 2, 3):
            dfp = 1.0 / (3 ** p * L)
            for iy in (-1, 0, 1):
                for ix in (-1, 0, 1):
                    if ix == 0 and iy == 0:
                        continue
                    fxy = (ix * dfp, iy * dfp)
                    ps = KOLMOGOROV_PSD * self.r0_px ** (-5.0 / 3.0) * math.hypot(*fxy) ** (-11.0 / 3.0)
                    zeta = (rng.standard_normal() + 1j * rng.standard_normal()) / math.sqrt(2)
                    sh_f.append(fxy)
                    sh_c.append(zeta * math.sqrt(2.0 * ps) * dfp)
        self._sh_f = sh_f
        self._sh_c = np.array(sh_c)
        # least-squares basis for piston/tip/tilt removal over the pupil
        c = (n - 1) / 2.0
        yy, xx = np.mgrid[0:n, 0:n]
        self._basis = np.stack([np.ones(n * n), (xx - c).ravel(), (yy - c).ravel()], axis=1)

    # -- phase -------------------------------------------------------------------------
    def screen(self, n_frame: int) -> np.ndarray:
        """Full-grid turbulent phase at frame ``n_frame`` before piston/tip/tilt removal."""
        sx, sy = n_frame * self.velocity[0], n_frame * self.velocity[1]
        ramp = np.exp(-2j * math.pi * (self._fx * sx + self._fy * sy))
        big = _irfft2(self._spec_half * ramp, s=(self.L, self.L))
        n = self.cfg.n
        x = np.arange(n, dtype=np.float64)
        lo = np.zeros((n, n), np.complex128)
        for (fxs, fys), c in zip(self._sh_f, self._sh_c):
            lo += c * np.outer(np.exp(2j * math.pi * fys * (x - sy)), np.exp(2j * math.pi * fxs * (x - sx)))
        return big[:n, :n] + lo.real

    def true_phase(self, n_frame: int) -> np.ndarray:
        phi = self.screen(n_frame)
        m = self.pupil.ravel()
        coef, *_ = np.linalg.lstsq(self._basis[m], phi.ravel()[m], rcond=None)
        return phi - (self._basis @ coef).reshape(phi.shape)

    # -- frames ------------------------------------------------------------------------
    def frame(self, n_frame: int) -> tuple[np.ndarray, np.ndarray]:
        """(y_n as complex64 N x N, true phase as float64 N x N) for frame ``n_frame``."""
        cfg = self.cfg
        n = cfg.n
        phi = self.true_phase(n_frame)
        rng = np.random.default_rng(np.random.SeedSequence([cfg.config_id, cfg.stream_id,
                                                            n_frame + 1]))
        g = np.sqrt(self.r_true / 2.0) * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        w = math.sqrt(self.noise_var_raw / 2.0) * (rng.standard_normal((n, n))
                                                    + 1j * rng.standard_normal((n, n)))
        y = self.pupil * np.exp(1j * phi) * _fft2u(g) + w
        return y.astype(np.complex64), phi

    def frames(self, count: int, start: int = 0) -> tuple[np.ndarray, np.ndarray]:
        ys = np.empty((count, self.cfg.n, self.cfg.n), np.complex64)
        ph = np.empty((count, self.cfg.n, self.cfg.n), np.float64)
        for i in range(count):
            ys[i], ph[i] = self.frame(start + i)
        return ys, ph

    def default_noise_var(self) -> float:
        """Post-normalisation noise power 1/(1 + f SNR), f = pupil fill fraction."""
        f = self.pupil.mean()
        return 1.0 / (1.0 + f * self.cfg.snr)


def make_stream(cfg: StreamConfig) -> Stream:
    return Stream(cfg)


def with_frames(cfg: StreamConfig, frames: int) -> StreamConfig:
    return replace(cfg, frames=frames)
