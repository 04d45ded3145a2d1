"""Gradient of a z-stack loss through the Bessel strategy (FP64, test-only).

Per emitter with slices z_s the forward (Eq. 10-11, see :mod:`oracle.bessel`)
is

    F_s(theta_j)   = A_j exp(i W(theta_j)) exp(i k z_s cos theta_j)
    P_n(r_i, z_s)  = sum_j B_n[i, j] F_s(theta_j),
                     B_n[i, j] = w_j g_n(theta_j) J_n(k r_i sin theta_j)  (real)
    v_n(pixel)     = (1 - f) P_n(r_c) + f P_n(r_{c+1})                    (interp.)
    E_c(pixel)     = C_B sum_n M_cn(pixel) v_n                            (Eq. 10)
    I(pixel)       = sum_c |E_c|^2

with W = W_GL(t_s) + sum over m = 0 Noll terms c_q Z_q(sin theta / s_max)
+ W_0(theta).  For a real loss L and a complex quantity X the gradient is
g_X = dL/dRe X + i dL/dIm X, so a complex-linear map X -> a X sends g back as
conj(a) g.  The adjoint runs the same steps backwards:

    g_E_c   = 2 (dL/dI) E_c
    g_v_n   = sum_c conj(C_B M_cn) g_E_c
    g_P_n   = transpose of the interpolation applied to g_v_n
    g_F_s   = sum_n B_n^H g_P_n
    Q_j     = sum_s conj(g_F_s(theta_j)) F_s(theta_j)
    dL/dW_0(theta_j) = Re(i Q_j) = -Im Q_j
    dL/dc_q          = sum_j Z_q(sin theta_j / s_max) dL/dW_0(theta_j)     (Eq. 15)
    dL/dt_s          = sum_j Re(i D_j Q_j),  D_j = dW_GL/dt_s (complex where a
                       layer is evanescent; Eq. 13 with t_i(t_s) from Eq. 14)

Non-axisymmetric (m != 0) Noll terms do not enter the spherical form, so their
gradient is zero.  The tests pin this adjoint with central finite differences
of :func:`oracle.bessel.psf_bessel_batch` and with the piston invariance
(dL/dc_1 = sum_j dL/dW_0 = 0: a constant phase leaves every intensity alone).
"""
import math

import numpy as np
from scipy.special import jv

from .bessel import (C_BESSEL, angular_weights, gl_rule, interpolate, model_pol,
                     pixel_polar, pupil_function, radial_grid)
from .optics import _layer_root, noll_to_nm
from .optics import zernike as zernike_poly


def depth_derivative(opt, sin_t):
    """D = dW_GL/dt_s [rad/um]: the sample layer contributes n_s cos theta_s and
    the immersion layer (t_i = t_s (1 - n_i/n_s) + const by Eq. 14) its share."""
    k0 = 2.0 * math.pi / opt.lam
    return k0 * (_layer_root(opt.n_s, opt.n_i, sin_t)
                 + (1.0 - opt.n_i / opt.n_s) * _layer_root(opt.n_i, opt.n_i, sin_t))


def field_matrix(cos_p, sin_p, pol):
    """M[c][n] of Eq. 10 (E_c = C_B sum_n M_cn v_n), each an array over pixels."""
    px, py = pol
    cos2 = cos_p * cos_p - sin_p * sin_p
    sin2 = 2.0 * sin_p * cos_p
    zero = np.zeros_like(cos_p, dtype=np.complex128)
    return [[px + zero, zero, -(px * cos2 + py * sin2)],
            [py + zero, zero, py * cos2 - px * sin2],
            [zero, -2j * (px * cos_p + py * sin_p), zero]]


def emitter_loss_and_grads(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike=None,
                           w0=None, project=False, target=None, grad_intensity=None):
    """One emitter.  Loss sum (I - T)^2 if ``target`` is given (else the
    linear functional sum grad_intensity * I).  Returns
    (L, dL/dW_0 [n_theta], dL/dc [n_zern], dL/dt_s, I [nz, nx, ny])."""
    th, wt = gl_rule(n_theta, opt.theta_max)
    sin_t, cos_t = np.sin(th), np.cos(th)
    g = angular_weights(opt, sin_t, cos_t)
    f0 = pupil_function(opt, th, zernike, project, w0)
    r, r_max = radial_grid(n_r, nx, ny, dx, dy)
    B = [jv(n, opt.k * np.outer(r, sin_t)) * (wt * g[n])[None, :] for n in range(3)]
    rho, cos_p, sin_p = pixel_polar(nx, ny, dx, dy)
    M = field_matrix(cos_p, sin_p, model_pol(opt))
    # interpolation cell and weight of every pixel (same rule as the forward)
    t = rho * ((n_r - 1) / r_max) if r_max > 0 else np.zeros_like(rho)
    c0 = np.clip(np.floor(t).astype(np.int64), 0, n_r - 2)
    f = t - c0
    zs = np.asarray(zs, dtype=np.float64)
    Q = np.zeros(n_theta, dtype=np.complex128)
    I_all = np.empty((len(zs), nx, ny))
    L = 0.0
    for iz, z in enumerate(zs):
        F = f0 * np.exp(1j * opt.k * z * cos_t)
        P = [B[n] @ F for n in range(3)]
        v = [interpolate(P[n], r_max, rho) for n in range(3)]
        E = [C_BESSEL * sum(M[c][n] * v[n] for n in range(3)) for c in range(3)]
        I = sum(e.real ** 2 + e.imag ** 2 for e in E)
        I_all[iz] = I
        if target is not None:
            d = I - target[iz]
            L += float(np.sum(d * d))
            gI = 2.0 * d
        else:
            L += float(np.sum(grad_intensity[iz] * I))
            gI = grad_intensity[iz]
        gE = [2.0 * gI * E[c] for c in range(3)]
        gP = []
        for n in range(3):
            gv = sum(np.conj(C_BESSEL * M[c][n]) * gE[c] for c in range(3))
            acc = np.zeros(n_r, dtype=np.complex128)
            np.add.at(acc, c0.ravel(), ((1.0 - f) * gv).ravel())
            np.add.at(acc, c0.ravel() + 1, (f * gv).ravel())
            gP.append(acc)
        gF = sum(np.conj(B[n]).T @ gP[n] for n in range(3))     # B^H (complex with Fresnel)
        Q += np.conj(gF) * F
    gW = -Q.imag
    D = depth_derivative(opt, sin_t)
    g_depth = float(np.sum(np.real(1j * D * Q)))
    n_zern = 0 if zernike is None else len(zernike)
    gc = np.zeros(n_zern)
    for q in range(n_zern):
        if noll_to_nm(q + 1)[1] == 0:
            gc[q] = np.sum(zernike_poly(q + 1, sin_t / opt.s_max, np.zeros_like(th)) * gW)
    return L, gW, gc, g_depth, I_all


def loss_and_grads_batch(opt, depths, zernikes, z_offsets, zs, n_theta, n_r, nx,
                         ny, dx, dy, phase_theta=None, project=False, target=None,
                         grad_intensity=None, emitters=None):
    """Batched emitters with packed slices (the layout of the library call).
    Returns per-emitter arrays (L [n], gW [n, n_theta], gc [n, n_zern],
    g_depth [n]) for the listed ``emitters`` (default: all)."""
    z_offsets = np.asarray(z_offsets)
    zs = np.asarray(zs, dtype=np.float64)
    sel = list(range(len(depths))) if emitters is None else list(emitters)
    out = ([], [], [], [])
    for e in sel:
        a, b = z_offsets[e], z_offsets[e + 1]
        T = None if target is None else np.asarray(target[a:b], dtype=np.float64)
        G = None if grad_intensity is None else np.asarray(grad_intensity[a:b],
                                                           dtype=np.float64)
        res = emitter_loss_and_grads(
            opt.with_depth(depths[e]), n_theta, n_r, nx, ny, dx, dy, zs[a:b],
            None if zernikes is None else zernikes[e],
            None if phase_theta is None else phase_theta[e], project, T, G)
        for k in range(4):
            out[k].append(res[k])
    return (np.array(out[0]), np.array(out[1]), np.array(out[2]), np.array(out[3]))
