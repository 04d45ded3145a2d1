"""Continuum oracle: Eq. 9 with Eq. 12 corrections by direct double quadrature.

E(x, y, z) = -i/(2 pi) int_0^theta_max dtheta int_0^2pi dphi
             A(theta) e^{i W(theta, phi)} e_inf(theta, phi)
             e^{i k (x sin(theta) cos(phi) + y sin(theta) sin(phi) + z cos(theta))}
             sin(theta)

theta: Gauss-Legendre on [0, theta_max]; phi: trapezoid rule with n_phi
equispaced nodes (spectrally accurate for the periodic phi integrand).  No
Bessel identity and no Cartesian grid is used, so this pins both strategies.
W may be any Zernike combination (not only axisymmetric).  Test-only, FP64.
"""
import math

import numpy as np

from .bessel import gl_rule
from .optics import amplitude, far_field_model, gibson_lanni_phase, zernike_phase

C_CONT = -1j / (2.0 * math.pi)


def field_points(opt, xs, ys, zs, zernike=None, n_theta=512, n_phi=256):
    """E [3, npts] at the points (xs[i], ys[i], zs[i])."""
    th, wt = gl_rule(n_theta, opt.theta_max)
    ph = np.arange(n_phi, dtype=np.float64) * (2.0 * math.pi / n_phi)
    wph = 2.0 * math.pi / n_phi
    TH, PH = np.meshgrid(th, ph, indexing="ij")          # [nth, nph]
    sin_t, cos_t = np.sin(TH), np.cos(TH)
    cos_p, sin_p = np.cos(PH), np.sin(PH)
    w = gibson_lanni_phase(opt, sin_t)
    if zernike is not None and len(zernike):
        w = w + zernike_phase(np.asarray(zernike, dtype=np.float64),
                              sin_t / opt.s_max, PH)
    base = (amplitude(opt, cos_t, sin_t) * np.exp(1j * w) * sin_t
            * (wt[:, None] * wph))
    ef = far_field_model(opt, cos_t, sin_t, cos_p, sin_p)
    terms = [(base * e).ravel() for e in ef]              # 3 x [nodes]
    sx = (sin_t * cos_p).ravel()
    sy = (sin_t * sin_p).ravel()
    sz = cos_t.ravel()
    xs = np.atleast_1d(np.asarray(xs, dtype=np.float64))
    ys = np.atleast_1d(np.asarray(ys, dtype=np.float64))
    zs = np.atleast_1d(np.asarray(zs, dtype=np.float64))
    out = np.empty((3, len(xs)), dtype=np.complex128)
    for i in range(len(xs)):
        e = np.exp(1j * opt.k * (sx * xs[i] + sy * ys[i] + sz * zs[i]))
        for c in range(3):
            out[c, i] = C_CONT * np.dot(terms[c], e)
    return out
