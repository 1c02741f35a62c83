"""FP64 reverse-mode derivative of K unrolled DDH-MBIR frame steps (oracle gradient).

TEST INFRASTRUCTURE ONLY (same rules as ``ddh_oracle``): imported by the tests and nothing in
the GPU library.  It differentiates ``ddh_oracle.step`` (one EM iteration per frame, per-pixel
phase) with respect to the state entering each frame, the q-GGMRF scale ``sigma_r`` and shape
``p``, and the noise variance ``sigma^2``, by the chain rule through each stage in reverse:

* phase M-step ``phi = angle(v)``, ``v = y~ conj(z)``: ``v_bar = phi_bar i v/|v|^2``,
  ``z_bar = y~ conj(v_bar)``, ``mu_bar = F^H z_bar``;
* ICD sweep, colours in reverse: the update ``r_i = root(W_i, C_i, s_i)`` differentiated
  implicitly (``g = W r^3 - C r^2 + r - s = 0``, ``g' = 3W r^2 - 2C r + 1``), the neighbour sums
  ``W = sum beta``, ``C = sum beta r_j`` and the weights ``beta = b_ij w(r0_i - r0_j; sigma_r, p)``;
* E-step ``w = r/(r+s2)``, ``mu = w b``, ``s = |mu|^2 + s2 w``; r-init (Eq. 3) with its floor;
* back-projection ``b = F^H(a e^{-j phi'} y~)`` and RemoveTipTilt ``phi' = phi - plane(phi)``.

Complex quantities carry the gradient ``dL/dRe + i dL/dIm``.  The weight's derivative in the
difference is singular at zero difference when p > 1 (a cusp of order 2 - p); there the
subgradient 0 is used.  Floors and root-branch switches are treated as locally constant.
"""
from __future__ import annotations

import math

import numpy as np

from . import ddh_oracle as o


def weight_and_derivs(delta, prm: o.Params):
    """w(D) = rho'(D)/D for q = 2 and its partial derivatives in D, sigma_r and p."""
    p, q, T, sg = prm.prior_p, prm.prior_q, prm.prior_T, prm.prior_sigma
    if q != 2.0:
        raise ValueError("derivatives implemented for q = 2")
    d = np.asarray(delta, np.float64)
    ad = np.abs(d)
    t = ad / (T * sg)
    with np.errstate(divide="ignore", invalid="ignore"):
        lt = np.where(t > 0, np.log(np.where(t > 0, t, 1.0)), 0.0)
    u = np.where(t > 0, np.exp((q - p) * lt), 0.0)
    A = q / p + u
    B = 1.0 + u
    w = (T * sg) ** (p - 2.0) * sg ** (-p) * A / B ** 2
    k = 1.0 / A - 2.0 / B          # d ln w / du
    # du/dD = (q-p) u / D  (D != 0); subgradient 0 at D = 0
    with np.errstate(divide="ignore", invalid="ignore"):
        du_dd = np.where(ad > 0, (q - p) * u / np.where(ad > 0, d, 1.0), 0.0)
    dw_dd = w * k * du_dd
    du_ds = -(q - p) * u / sg
    dw_ds = w * ((p - 2.0) / sg - p / sg + k * du_ds)
    du_dp = -u * lt
    dw_dp = w * (math.log(T) + (-q / p ** 2 + du_dp) / A - 2.0 * du_dp / B)
    return w, dw_dd, dw_ds, dw_dp


def _plane_coords(n):
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    return xx - c, yy - c


def frame_backward(r_prev, phi_prev, y, prm: o.Params, r_bar, phi_bar):
    """Adjoint of one frame step: given dL/dr_n and dL/dphi_n, return dL/dr_{n-1},
    dL/dphi_{n-1} and the frame's contributions to dL/dsigma_r, dL/dp, dL/dsigma^2."""
    if prm.n_k != 1 or prm.phase_block != 1:
        raise ValueError("the adjoint covers one EM iteration per frame with per-pixel phase")
    n = prm.n
    a = o.aperture(n, prm.aperture_diam)
    s2 = prm.noise_var
    # ---- forward recompute ----------------------------------------------------------------
    yt, _ = o.normalize(y)
    if prm.tilt_mode:
        phi1, (tx, ty) = o.remove_tip_tilt(phi_prev, a)
    else:
        phi1 = np.where(a, phi_prev, 0.0)
    u = a * np.exp(-1j * phi1) * yt
    b = o.ifft2u(u)
    pre = (1.0 - prm.lam) * r_prev + prm.lam * prm.alpha * np.abs(b) ** 2
    r0 = np.maximum(pre, prm.r_floor)
    w = r0 / (r0 + s2)
    mu = w * b
    s = np.abs(mu) ** 2 + s2 * w
    z = o.fft2u(mu)
    v = yt * np.conj(z)
    # ICD forward recompute with the per-colour values kept
    yy, xx = np.mgrid[0:n, 0:n]
    colour = (xx % 2) + 2 * (yy % 2)          # sweep order index of (x%2, y%2): (0,0),(1,0),(0,1),(1,1)
    betas, dbd, dbs, dbp, inside = [], [], [], [], []
    for dy, dx, bij in o.NEIGHBOURS:
        ins = o._inside(n, dy, dx)
        rn = o._neighbour(r0, dy, dx)
        wv, wd, ws, wp = weight_and_derivs(r0 - rn, prm)
        betas.append(np.where(ins, bij * wv, 0.0))
        dbd.append(np.where(ins, bij * wd, 0.0))
        dbs.append(np.where(ins, bij * ws, 0.0))
        dbp.append(np.where(ins, bij * wp, 0.0))
        inside.append(ins)
    W = np.sum(betas, axis=0)
    r = r0.copy()
    roots = np.zeros_like(r0)
    for cidx in range(4):
        sel = colour == cidx
        Cn = np.zeros((n, n))
        for (dy, dx, _), beta in zip(o.NEIGHBOURS, betas):
            Cn += beta * o._neighbour(r, dy, dx)
        rt = o.cubic_argmin(W[sel], Cn[sel], s[sel])
        roots[sel] = rt
        r[sel] = np.maximum(rt, prm.r_floor)
    r_new = r
    # value of neighbour j seen by pixel i at i's update: updated if colour(j) < colour(i)
    # ---- reverse: phase M-step ------------------------------------------------------------
    g_sigma = g_p = g_s2 = 0.0
    absv2 = np.abs(v) ** 2
    live = a & (absv2 > 0)
    vbar = np.where(live, phi_bar * 1j * v / np.where(live, absv2, 1.0), 0.0)
    zbar = yt * np.conj(vbar)
    mubar = o.ifft2u(zbar)
    # ---- reverse: ICD -----------------------------------------------------------------------
    abar = np.array(r_bar, np.float64).copy()       # adjoint of the current value of each pixel
    r0bar = np.zeros((n, n))
    sbar = np.zeros((n, n))
    clamped = roots < prm.r_floor
    for cidx in (3, 2, 1, 0):
        sel = colour == cidx
        # neighbour values seen at this colour's update
        cur = np.where(colour < cidx, r_new, r0)
        Cn = np.zeros((n, n))
        for (dy, dx, _), beta in zip(o.NEIGHBOURS, betas):
            Cn += beta * o._neighbour(cur, dy, dx)
        rt = roots
        gp = 3.0 * W * rt ** 2 - 2.0 * Cn * rt + 1.0
        gbar = np.where(sel & ~clamped, abar, 0.0)
        abar = np.where(sel, 0.0, abar)
        Wbar = -gbar * rt ** 3 / gp
        Cbar = gbar * rt ** 2 / gp
        sbar += gbar / gp
        for k, ((dy, dx, _), beta) in enumerate(zip(o.NEIGHBOURS, betas)):
            rj = o._neighbour(cur, dy, dx)
            betabar = np.where(sel, Cbar * rj + Wbar, 0.0)
            # C_i = sum beta_ij r_j: the neighbour's value receives Cbar_i beta_ij
            contrib = np.where(sel, Cbar * beta, 0.0)
            abar += _shift_back(contrib, dy, dx)
            # beta_ij = b_ij w(r0_i - r0_j; sigma, p)
            g_sigma += float(np.sum(betabar * dbs[k]))
            g_p += float(np.sum(betabar * dbp[k]))
            r0bar += betabar * dbd[k]
            r0bar -= _shift_back(betabar * dbd[k], dy, dx)
    r0bar += abar  # what is left is the adjoint of the entry values through neighbour sums
    # ---- reverse: E-step --------------------------------------------------------------------
    mubar_t = mubar + 2.0 * sbar * mu
    wbar = np.real(mubar_t * np.conj(b)) + sbar * s2
    bbar = w * mubar_t
    g_s2 += float(np.sum(sbar * w + wbar * (-r0 / (r0 + s2) ** 2)))
    r0bar = r0bar + wbar * s2 / (r0 + s2) ** 2
    # ---- reverse: r-init --------------------------------------------------------------------
    live_r = pre > prm.r_floor
    r_prev_bar = np.where(live_r, (1.0 - prm.lam) * r0bar, 0.0)
    bbar = bbar + np.where(live_r, 2.0 * prm.lam * prm.alpha * r0bar, 0.0) * b
    # ---- reverse: back-projection and RemoveTipTilt ----------------------------------------
    ubar = o.fft2u(bbar)
    phi1bar = np.where(a, np.imag(np.conj(ubar) * u), 0.0)
    phi_prev_bar = phi1bar.copy()
    if prm.tilt_mode:
        X, Y = _plane_coords(n)
        txbar = -float(np.sum(phi1bar * X))
        tybar = -float(np.sum(phi1bar * Y))
        px = a[:, :-1] & a[:, 1:]
        py = a[:-1, :] & a[1:, :]
        if px.sum():
            gx = txbar / px.sum()
            phi_prev_bar[:, 1:] += np.where(px, gx, 0.0)
            phi_prev_bar[:, :-1] -= np.where(px, gx, 0.0)
        if py.sum():
            gy = tybar / py.sum()
            phi_prev_bar[1:, :] += np.where(py, gy, 0.0)
            phi_prev_bar[:-1, :] -= np.where(py, gy, 0.0)
    phi_prev_bar = np.where(a, phi_prev_bar, 0.0)
    return r_prev_bar, phi_prev_bar, np.array([g_sigma, g_p, g_s2]), (r_new, np.where(a & (absv2 > 0), np.angle(v), np.where(a, phi1, 0.0)))


def _shift_back(x, dy, dx):
    """Array whose entry j is x[j - (dy, dx)]: moves a value computed at pixel i onto its
    neighbour j = i + (dy, dx) (zero where that neighbour is off the grid)."""
    return o._neighbour(x, -dy, -dx)


def unrolled_grad(r0, phi0, ys, prm: o.Params, r_bar_K, phi_bar_K):
    """Gradients of L through K frames (L's gradient given at the final state): returns
    (dL/dr0, dL/dphi0, [dL/dsigma_r, dL/dp, dL/dsigma^2]) and the final state."""
    states = [(np.array(r0, np.float64), np.array(phi0, np.float64))]
    st = o.State(r=states[0][0].copy(), phi=states[0][1].copy())
    for y in ys:
        st, _ = o.step(st, y, prm)
        states.append((st.r, st.phi))
    rb, pb = np.array(r_bar_K, np.float64), np.array(phi_bar_K, np.float64)
    g = np.zeros(3)
    for k in range(len(ys) - 1, -1, -1):
        rb, pb, gk, _ = frame_backward(states[k][0], states[k][1], ys[k], prm, rb, pb)
        g += gk
    return rb, pb, g, states[-1]
