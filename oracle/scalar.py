"""Scalar paraxial forms used for the Airy benchmark of Sec. 5.2.2 (Eq. 18).

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
