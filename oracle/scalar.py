"""Scalar models (Sec. 3.2) and the paraxial forms of the Airy benchmark.

Scalar propagators, e_far = e_inc = A(theta) e^{iW} (the correction factors
of Eq. 12 apply to the scalar model as well), f k = 1:
    Eq. 3 (Cartesian):  E = -i/(2 pi) sum_disk ds^2 e_inc e^{i k s_z z} / s_z
                            e^{i k (s_x x + s_y y)}      (midpoint rule)
    Eq. 5 (spherical):  E = -i int_0^theta_max e_inc(theta) J_0(k rho sin)
                            e^{i k z cos} sin dtheta     (Gauss-Legendre)

Paraxial forms for the Airy benchmark of Sec. 5.2.2 (Eq. 18):

With e_inc = 1 and the extra factor s_z = cos(theta) the paper introduces for
this benchmark, Eq. 5 at focus becomes
    E(rho) = -i int_0^theta_max J_0(k rho sin t) sin t cos t dt
and Eq. 3 becomes the 2D Fourier transform of the uniform disk,
    E(x, y) = -i/(2 pi) sum_disk ds^2 exp(i k (s_x x + s_y y)).
Both equal -i s_max^2 J_1(v)/v, v = k s_max rho, i.e. the Airy pattern
2 J_1(v)/v of Eq. 18 up to the constant -i s_max^2 / 2.  Test-only, FP64.
"""
import math

import numpy as np
from scipy.special import jv

from .bessel import gl_rule, riemann_rule, simpson_rule
from .fourier import grid_coords
from .optics import pupil_mask, pupil_nodes


def scalar_bessel_paraxial(opt, rho, n_nodes, rule="gl"):
    if rule == "gl":
        th, wt = gl_rule(n_nodes, opt.theta_max)
    elif rule == "simpson":
        th, wt = simpson_rule(n_nodes, opt.theta_max)
    else:
        th, wt = riemann_rule(n_nodes, opt.theta_max)
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    kern = jv(0, opt.k * np.outer(rho, np.sin(th)))
    return -1j * kern @ (wt * np.sin(th) * np.cos(th))


def scalar_fourier_paraxial(opt, n_pupil, nx, dx):
    """E on the x axis (y = 0 is not a node for even n_x; use the full grid)."""
    mask = pupil_mask(n_pupil)
    u = pupil_nodes(n_pupil)
    ds = 2.0 * opt.s_max / n_pupil
    xs = grid_coords(nx, dx)
    A = np.exp(1j * opt.k * opt.s_max * np.outer(xs, u))
    E = -1j / (2.0 * math.pi) * ds * ds * (A @ mask.astype(np.float64) @ A.T)
    return E, xs


def scalar_spherical(opt, n_theta, rho, zs, zernike=None, project=False):
    """Eq. 5 at radii rho -> E [nz, len(rho)] (axisymmetric pupil)."""
    from .bessel import pupil_function
    th, wt = gl_rule(n_theta, opt.theta_max)
    sin_t, cos_t = np.sin(th), np.cos(th)
    e_inc = pupil_function(opt, th, zernike, project)
    kern = jv(0, opt.k * np.outer(np.asarray(rho, dtype=np.float64), sin_t))
    out = []
    for z in np.atleast_1d(np.asarray(zs, dtype=np.float64)):
        out.append(-1j * kern @ (wt * sin_t * e_inc * np.exp(1j * opt.k * z * cos_t)))
    return np.array(out)


def scalar_spherical_psf(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike=None,
                         project=False):
    """Eq. 5 on the radial grid r_i = i r_max / (N_r - 1), linearly
    interpolated at the pixel radii, |E|^2 -> [nz, nx, ny]."""
    from .bessel import interpolate, pixel_polar, radial_grid
    r, r_max = radial_grid(n_r, nx, ny, dx, dy)
    prof = scalar_spherical(opt, n_theta, r, zs, zernike, project)
    rho, _, _ = pixel_polar(nx, ny, dx, dy)
    E = np.stack([interpolate(prof[iz], r_max, rho) for iz in range(prof.shape[0])])
    return E.real ** 2 + E.imag ** 2


def scalar_cartesian(opt, n_pupil, grid, zernike=None, phase_map=None):
    """Eq. 3 by the midpoint rule on the pupil grid -> E [nz, nx, ny]."""
    from .fourier import pupil_phase, zoom_matrix
    from .optics import amplitude, pupil_geometry
    sin_t, cos_t, _, _, _, _ = pupil_geometry(opt, n_pupil)
    mask = pupil_mask(n_pupil)
    safe = np.where(mask, cos_t, 1.0)
    e_inc = amplitude(opt, cos_t, sin_t) * np.exp(1j * pupil_phase(opt, n_pupil, zernike,
                                                                   phase_map))
    P = np.where(mask, e_inc / safe, 0.0)
    ds = 2.0 * opt.s_max / n_pupil
    Ax = zoom_matrix(opt, n_pupil, grid["nx"], grid["dx"])
    Ay = zoom_matrix(opt, n_pupil, grid["ny"], grid["dy"])
    out = []
    for z in np.asarray(grid["z"], dtype=np.float64):
        out.append(-1j / (2.0 * math.pi) * ds * ds *
                   (Ax @ (P * np.exp(1j * opt.k * z * cos_t)) @ Ay.T))
    return np.array(out)
