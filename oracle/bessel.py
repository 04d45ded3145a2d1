"""Spherical (Bessel) strategy: Eq. 10 with the integrals of Eq. 11.

For an axisymmetric pupil the incident field is e_inc^a(theta) = p_a F0(theta)
with F0 = A(theta) exp(i W(theta)) (Eq. 12 correction factors, W = W_GL +
the m = 0 Zernike terms), so Eq. 11 needs only three complex profiles

    I_n(rho, z) = int_0^theta_max g_n(theta) J_n(k rho sin theta)
                  F0(theta) exp(i k z cos theta) dtheta,
    g_0 = sin(1 + cos), g_1 = sin^2, g_2 = sin(cos - 1),

and I_n^a = p_a I_n.  The theta integral uses Gauss-Legendre nodes on
[0, theta_max].  Profiles are sampled on r_i = i r_max / (N_r - 1), r_max the
corner radius of the output grid, and linearly interpolated (complex) at each
pixel radius before Eq. 10 is applied.  FP64; test infrastructure only.
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import jv

from .fourier import grid_coords
from .optics import (amplitude, fresnel_coefficients, gibson_lanni_phase, noll_to_nm,
                     zernike_phase)

C_BESSEL = -0.5j                     # -i f k / 2 with f k = 1 (Eq. 10)


class NotAxisymmetric(ValueError):
    pass


def gl_rule(n_theta, theta_max):
    """Gauss-Legendre nodes/weights mapped from [-1, 1] to [0, theta_max]."""
    x, w = leggauss(n_theta)
    return 0.5 * theta_max * (x + 1.0), 0.5 * theta_max * w


def simpson_rule(n_intervals, theta_max):
    """Composite Simpson nodes/weights (n_intervals even) on [0, theta_max]."""
    if n_intervals % 2:
        raise ValueError("Simpson needs an even number of intervals")
    h = theta_max / n_intervals
    th = np.arange(n_intervals + 1) * h
    w = np.full(n_intervals + 1, 2.0)
    w[1::2] = 4.0
    w[0] = w[-1] = 1.0
    return th, w * h / 3.0


def riemann_rule(n_intervals, theta_max):
    """Left Riemann sum nodes/weights on [0, theta_max]."""
    h = theta_max / n_intervals
    return np.arange(n_intervals) * h, np.full(n_intervals, h)


def axisymmetric_coeffs(zernike, project):
    """Keep only m = 0 Noll terms; others must be zero unless projected away."""
    if zernike is None:
        return None
    z = np.asarray(zernike, dtype=np.float64).copy()
    for idx in range(len(z)):
        if noll_to_nm(idx + 1)[1] != 0 and z[idx] != 0.0:
            if not project:
                raise NotAxisymmetric(
                    "Noll j=%d has m != 0; the spherical form needs an "
                    "axisymmetric pupil" % (idx + 1))
            z[idx] = 0.0
    return z


def pupil_function(opt, theta, zernike=None, project=False, w0=None):
    """F0(theta) = A(theta) exp(i W(theta)), W = W_GL + m=0 Zernike terms
    (+ an optional free radial phase w0(theta) at the nodes, radians)."""
    sin_t = np.sin(theta)
    cos_t = np.cos(theta)
    w = gibson_lanni_phase(opt, sin_t)
    z = axisymmetric_coeffs(zernike, project)
    if z is not None and len(z):
        w = w + zernike_phase(z, sin_t / opt.s_max, np.zeros_like(theta))
    if w0 is not None:
        w = w + np.asarray(w0, dtype=np.float64)
    return amplitude(opt, cos_t, sin_t) * np.exp(1j * w)


def angular_weights(opt, sin_t, cos_t):
    """g_0, g_1, g_2 of Eq. 11 for the model: q_s = q_p = 1 (the printed
    form); with Fresnel coefficients the phi integrals of Eq. 6 give
    g_0 = sin (q_s + q_p cos), g_1 = q_p sin^2, g_2 = sin (q_p cos - q_s);
    the scalar model (Eq. 5) is carried by g_0 = 2 sin (so that
    E_x = -(i/2) I_0 is Eq. 5 with x polarisation), g_1 = g_2 = 0."""
    if opt.scalar:
        z = 0.0 * sin_t
        return (2.0 * sin_t, z, z)
    if opt.fresnel:
        qs, qp = fresnel_coefficients(opt, sin_t)
        return (sin_t * (qs + qp * cos_t), qp * sin_t * sin_t, sin_t * (qp * cos_t - qs))
    return (sin_t * (1.0 + cos_t), sin_t * sin_t, sin_t * (cos_t - 1.0))


def model_pol(opt):
    """Jones vector the spherical form uses (x for the scalar model)."""
    return (1.0 + 0j, 0j) if opt.scalar else opt.pol


def profiles(opt, n_theta, r, zs, zernike=None, project=False, rule="gl",
             w0=None):
    """I_n(r_i, z) of Eq. 11 for n = 0, 1, 2 -> complex array [nz, 3, len(r)]."""
    if rule == "gl":
        th, wt = gl_rule(n_theta, opt.theta_max)
    elif rule == "simpson":
        th, wt = simpson_rule(n_theta, opt.theta_max)
    else:
        th, wt = riemann_rule(n_theta, opt.theta_max)
    sin_t, cos_t = np.sin(th), np.cos(th)
    g = angular_weights(opt, sin_t, cos_t)
    f0 = pupil_function(opt, th, zernike, project, w0)
    arg = opt.k * np.outer(np.asarray(r, dtype=np.float64), sin_t)  # [nr, nth]
    zs = np.asarray(zs, dtype=np.float64)
    out = np.empty((len(zs), 3, arg.shape[0]), dtype=np.complex128)
    for n in range(3):
        kern = jv(n, arg) * (wt * g[n])[None, :]                      # [nr, nth]
        for iz, z in enumerate(zs):
            out[iz, n] = kern @ (f0 * np.exp(1j * opt.k * z * cos_t))
    return out


def radial_grid(n_r, nx, ny, dx, dy):
    """r_i = i r_max/(N_r - 1), r_max the corner radius of the output grid."""
    r_max = math.hypot(0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dy)
    return np.arange(n_r, dtype=np.float64) * (r_max / (n_r - 1)), r_max


def interpolate(prof, r_max, rho):
    """Linear interpolation of complex profiles [..., n_r] at radii rho."""
    n_r = prof.shape[-1]
    # r_max = 0 (a single pixel on the axis): every r_i is 0, use cell 0
    t = rho * ((n_r - 1) / r_max) if r_max > 0 else np.zeros_like(rho)
    i0 = np.clip(np.floor(t).astype(np.int64), 0, n_r - 2)
    f = t - i0
    return prof[..., i0] * (1.0 - f) + prof[..., i0 + 1] * f


def field_from_profiles(I0, I1, I2, cos_p, sin_p, pol):
    """Eq. 10 with I_n^a = p_a I_n -> [E_x, E_y, E_z]."""
    px, py = pol
    cos2 = cos_p * cos_p - sin_p * sin_p
    sin2 = 2.0 * sin_p * cos_p
    ex = (px * I0 - px * I2 * cos2) - py * I2 * sin2
    ey = -px * I2 * sin2 + (py * I0 + py * I2 * cos2)
    ez = -2j * px * I1 * cos_p - 2j * py * I1 * sin_p
    return [C_BESSEL * ex, C_BESSEL * ey, C_BESSEL * ez]


def pixel_polar(nx, ny, dx, dy):
    xs = grid_coords(nx, dx)
    ys = grid_coords(ny, dy)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    rho = np.hypot(X, Y)
    safe = rho > 0
    cos_p = np.where(safe, X / np.where(safe, rho, 1.0), 1.0)
    sin_p = np.where(safe, Y / np.where(safe, rho, 1.0), 0.0)
    return rho, cos_p, sin_p


def field_bessel(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike=None,
                 project=False, w0=None):
    """E [nz, 3, nx, ny] by profiles on the radial grid + interpolation."""
    r, r_max = radial_grid(n_r, nx, ny, dx, dy)
    prof = profiles(opt, n_theta, r, zs, zernike, project, w0=w0)
    rho, cos_p, sin_p = pixel_polar(nx, ny, dx, dy)
    E = np.empty((len(zs), 3, nx, ny), dtype=np.complex128)
    for iz in range(len(zs)):
        In = [interpolate(prof[iz, n], r_max, rho) for n in range(3)]
        E[iz] = np.stack(field_from_profiles(*In, cos_p, sin_p, model_pol(opt)))
    return E


def field_bessel_direct(opt, n_theta, nx, ny, dx, dy, zs, zernike=None,
                        project=False, rule="gl"):
    """E [nz, 3, nx, ny] with Eq. 11 evaluated at every pixel radius."""
    rho, cos_p, sin_p = pixel_polar(nx, ny, dx, dy)
    prof = profiles(opt, n_theta, rho.ravel(), zs, zernike, project, rule)
    E = np.empty((len(zs), 3, nx, ny), dtype=np.complex128)
    for iz in range(len(zs)):
        In = [prof[iz, n].reshape(nx, ny) for n in range(3)]
        E[iz] = np.stack(field_from_profiles(*In, cos_p, sin_p, model_pol(opt)))
    return E


def psf_bessel(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike=None,
               project=False, w0=None):
    E = field_bessel(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike, project, w0)
    return np.sum(E.real ** 2 + E.imag ** 2, axis=1)


def psf_bessel_batch(opt, depths, zernikes, z_offsets, zs, n_theta, n_r, nx,
                     ny, dx, dy, project=False, emitters=None, phase_theta=None):
    """Batched emitters (each its own depth, Zernike row and z sub-list; with
    ``phase_theta`` [n_em, n_theta] also a free radial phase at the nodes).

    Returns the packed intensity [z_offsets[-1], nx, ny] (or only the slices of
    the listed ``emitters``, concatenated in that order).
    """
    z_offsets = np.asarray(z_offsets)
    zs = np.asarray(zs, dtype=np.float64)
    sel = range(len(depths)) if emitters is None else emitters
    out = []
    for e in sel:
        o = opt.with_depth(depths[e])
        zc = None if zernikes is None else zernikes[e]
        w0 = None if phase_theta is None else phase_theta[e]
        out.append(psf_bessel(o, n_theta, n_r, nx, ny, dx, dy,
                              zs[z_offsets[e]:z_offsets[e + 1]], zc, project, w0))
    return np.concatenate(out, axis=0)


def profiles_batch(opt, depths, zernikes, z_offsets, zs, n_theta, n_r, nx, ny,
                   dx, dy, project=False, emitters=None, phase_theta=None):
    """Complex profiles [sum z, 3, n_r] of the batched emitters (packed)."""
    r, _ = radial_grid(n_r, nx, ny, dx, dy)
    z_offsets = np.asarray(z_offsets)
    zs = np.asarray(zs, dtype=np.float64)
    sel = range(len(depths)) if emitters is None else emitters
    out = []
    for e in sel:
        o = opt.with_depth(depths[e])
        zc = None if zernikes is None else zernikes[e]
        w0 = None if phase_theta is None else phase_theta[e]
        out.append(profiles(o, n_theta, r, zs[z_offsets[e]:z_offsets[e + 1]],
                            zc, project, w0=w0))
    return np.concatenate(out, axis=0)
