"""Cartesian (Fourier) strategy: Eq. 8 with the correction factors of Eq. 12.

E(x, y, z) = -i/(2 pi) * sum over disk nodes (p, q) of
    ds^2 * A(theta) e^{iW} e_inf(theta, phi) / s_z * e^{i k s_z z}
         * e^{i k (s_x x + s_y y)},
with s_x = s_max u_p, s_y = s_max v_q, ds = 2 s_max / N (midpoint rule on the
N x N cell-centred grid; no fractional edge weights).  W = W_GL (Eq. 13-14)
+ sum_j c_j Z_j (Eq. 15) + W_0 (the free phase map of Eq. 15).

Output grid: x_a = (a - (n_x - 1)/2) dx, y_b = (b - (n_y - 1)/2) dy; fields
are returned as [z, channel, x, y] (Sec. 4.1 tensor layout).
FP64 / complex128 throughout; test infrastructure only.
"""
import math

import numpy as np

from .optics import (amplitude, far_field_model, gibson_lanni_phase, pupil_geometry,
                     pupil_mask, pupil_nodes, zernike_phase)

C_FOURIER = -1j / (2.0 * math.pi)          # -i f k / (2 pi) with f k = 1


def grid_coords(n, d):
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * d


def pupil_phase(opt, n_pupil, zernike=None, phase_map=None):
    """W(s) on the pupil grid in radians (complex where Gibson-Lanni decays)."""
    sin_t, cos_t, cos_p, sin_p, rn, phi = pupil_geometry(opt, n_pupil)
    w = gibson_lanni_phase(opt, sin_t)
    if zernike is not None and len(zernike):
        w = w + zernike_phase(np.asarray(zernike, dtype=np.float64), rn, phi)
    if phase_map is not None:
        w = w + np.asarray(phase_map, dtype=np.float64)
    return w


def pupil_field(opt, n_pupil, zernike=None, phase_map=None):
    """P_c[p, q] = A e^{iW} e_inf,c / cos(theta) on the disk, 0 outside.

    Returns (P [3, N, N] complex128, cos_theta [N, N]).
    """
    sin_t, cos_t, cos_p, sin_p, rn, phi = pupil_geometry(opt, n_pupil)
    mask = pupil_mask(n_pupil)
    amp = amplitude(opt, cos_t, sin_t)
    w = pupil_phase(opt, n_pupil, zernike, phase_map)
    ef = far_field_model(opt, cos_t, sin_t, cos_p, sin_p)
    safe_cos = np.where(mask, cos_t, 1.0)
    P = np.stack([np.where(mask, amp * np.exp(1j * w) * e / safe_cos, 0.0)
                  for e in ef])
    return P, cos_t


def zoom_matrix(opt, n_pupil, n_out, d):
    """A[a, p] = exp(i k s_max u_p x_a) = exp(2 pi i (NA/lambda) u_p x_a)."""
    u = pupil_nodes(n_pupil)
    x = grid_coords(n_out, d)
    return np.exp(1j * opt.k * opt.s_max * np.outer(x, u))


def field_separable(opt, n_pupil, grid, zernike=None, phase_map=None):
    """Eq. 8 evaluated as E_c(z) = C ds^2 A_x (P_c e^{ik z cos}) A_y^T."""
    P, cos_t = pupil_field(opt, n_pupil, zernike, phase_map)
    ds = 2.0 * opt.s_max / n_pupil
    Ax = zoom_matrix(opt, n_pupil, grid["nx"], grid["dx"])
    Ay = zoom_matrix(opt, n_pupil, grid["ny"], grid["dy"])
    zs = np.asarray(grid["z"], dtype=np.float64)
    E = np.empty((len(zs), 3, grid["nx"], grid["ny"]), dtype=np.complex128)
    for iz, z in enumerate(zs):
        defocus = np.exp(1j * opt.k * z * cos_t)
        for c in range(3):
            E[iz, c] = C_FOURIER * ds * ds * (Ax @ (P[c] * defocus) @ Ay.T)
    return E


def field_brute(opt, n_pupil, grid, zernike=None, phase_map=None):
    """Eq. 8 as a direct double sum, one exponent k s.rho per term (tiny sizes)."""
    P, cos_t = pupil_field(opt, n_pupil, zernike, phase_map)
    mask = pupil_mask(n_pupil)
    u = pupil_nodes(n_pupil)
    U, V = np.meshgrid(u, u, indexing="ij")
    sx = (opt.s_max * U)[mask]
    sy = (opt.s_max * V)[mask]
    sz = cos_t[mask]
    Pm = P[:, mask]                                    # [3, n_nodes]
    ds = 2.0 * opt.s_max / n_pupil
    xs = grid_coords(grid["nx"], grid["dx"])
    ys = grid_coords(grid["ny"], grid["dy"])
    zs = np.asarray(grid["z"], dtype=np.float64)
    E = np.empty((len(zs), 3, len(xs), len(ys)), dtype=np.complex128)
    for iz, z in enumerate(zs):
        for a, x in enumerate(xs):
            ph = opt.k * (sx[None, :] * x + sy[None, :] * ys[:, None]
                          + sz[None, :] * z)                # [ny, n_nodes]
            E[iz, :, a, :] = C_FOURIER * ds * ds * (np.exp(1j * ph) @ Pm.T).T
    return E


def intensity(E):
    """|E_x|^2 + |E_y|^2 + |E_z|^2 over the channel axis of [z, c, x, y]."""
    return np.sum(E.real ** 2 + E.imag ** 2, axis=1)


def psf_fourier(opt, n_pupil, grid, zernike=None, phase_map=None):
    """Intensity z-stack [nz, nx, ny] of the Fourier strategy (separable form)."""
    return intensity(field_separable(opt, n_pupil, grid, zernike, phase_map))
