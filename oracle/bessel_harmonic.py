"""Spherical (Bessel) strategy for a pupil without axial symmetry, by
azimuthal harmonics.  Test infrastructure only (FP64; imported by tests/,
the smoke check and the benchmark's CPU baseline, never by the library).

The spherical form of Sec. 3.4 / Eq. 10-11 needs W(theta) alone.  For any
W(theta, phi) (Zernike terms with m != 0, Eq. 15) expand the pupil in
azimuthal harmonics,

    A(theta) e^{i W(theta, phi)} = sum_m P_m(theta) e^{i m phi},

and the far field of Eq. 6 likewise (harmonics n = -2 .. 2).  With
u = q_s + q_p cos, v = q_p cos - q_s, s = q_p sin (q = 1 without Fresnel):

    e_x = p_x u/2 + (p_x - i p_y) v/4 e^{2i phi} + (p_x + i p_y) v/4 e^{-2i phi}
    e_y = p_y u/2 + (-i p_x - p_y) v/4 e^{2i phi} + (i p_x - p_y) v/4 e^{-2i phi}
    e_z = -(p_x - i p_y) s/2 e^{i phi} - (p_x + i p_y) s/2 e^{-i phi}.

The phi integral of Eq. 9 is done exactly by the Jacobi-Anger expansion,
int_0^{2 pi} e^{i l phi} e^{i x cos(phi - phi_p)} dphi = 2 pi i^l J_l(x) e^{i l phi_p},
so with f k = 1 (the prefactor -i/(2 pi) of Eq. 9)

    E_c(rho, phi_p, z) = -i sum_l i^l e^{i l phi_p} I_{c,l}(rho, z),
    I_{c,l} = int g-weighted combinations of P_{l-n}(theta) J_l(k rho sin theta)
              e^{i k z cos theta} dtheta,

with the g_n of Eq. 11 (g_0 = sin u, g_1 = sin s, g_2 = sin v) carrying the
sin(theta) of the measure.  For P_0 alone this is Eq. 10-11 term by term.

Discretisation (the method this oracle fixes):
* P_m(theta_j) = (1 / N_phi) sum_k A e^{i W(theta_j, phi_k)} e^{-i m phi_k},
  phi_k = 2 pi k / N_phi, N_phi = 4 * (smallest power of two >= M + 1),
  kept for |m| <= M (orders l = -(M+2) .. M+2);
* theta: Gauss-Legendre on [0, theta_max] (as the axisymmetric path);
* radial grid r_i = i r_max / (N_r - 1), complex linear interpolation of
  I_{c,l} at each pixel radius.

Truncation: if the m != 0 part of W is a trigonometric polynomial of degree
d in phi whose coefficients have l1 norm alpha (alpha <= sum |c_j| N_j over
the m != 0 Noll terms, N_j the Zernike normalisation, |R| <= 1), then
e^{i W} = sum_k (i W)^k / k! has no harmonic beyond k d from its first k
terms, so the harmonics |m| > K d carry at most alpha^{K+1} / (K+1)! e^alpha
(l1).  `harmonic_order` returns the smallest M = K d with that below tol;
aliasing in the DFT only folds harmonics |m| >= N_phi - M > 3 M, bounded by
the same tail.

Adaptive order (tail_tol > 0): the bound is pessimistic; with the computed
harmonics (|m| <= m_max) each emitter keeps M_e = the largest |m| with
max_theta |P_m| > tail_tol max_theta |P_0| (0 if none), and the harmonics
beyond it are dropped.  Past the few harmonics that carry W, |P_m| falls
faster than geometrically (as J_k(a) ~ (a/2)^k / k!), so the dropped tail is
about its first term, below tail_tol; a per-harmonic test (not the summed
tail) keeps the decision clear of the rounding floor of an FP32 DFT, a few
1e-8 of P_0 on every harmonic.
"""
import math

import numpy as np
from scipy.special import jv

from .bessel import (angular_weights, gl_rule, interpolate, model_pol, pixel_polar,
                     radial_grid)
from .optics import amplitude, gibson_lanni_phase, noll_to_nm, zernike_phase


def n_phi_for(m_max):
    p = 1
    while p < m_max + 1:
        p *= 2
    return 4 * p


def zernike_norm(n, m):
    return math.sqrt(n + 1.0) if m == 0 else math.sqrt(2.0 * (n + 1.0))


def harmonic_order(zernike, tol=1e-7):
    """Smallest M = K d with alpha^{K+1} / (K+1)! e^alpha <= tol (see above);
    0 without m != 0 terms."""
    if zernike is None:
        return 0
    alpha, d = 0.0, 0
    for idx, c in enumerate(np.asarray(zernike, dtype=np.float64)):
        n, m = noll_to_nm(idx + 1)
        if m != 0 and c != 0.0:
            alpha += abs(c) * zernike_norm(n, m)
            d = max(d, abs(m))
    if d == 0:
        return 0
    K, term = 0, alpha        # term = alpha^{K+1} / (K+1)!
    while term * math.exp(alpha) > tol:
        K += 1
        term *= alpha / (K + 1)
    return max(K, 1) * d


def pupil_harmonics(opt, theta, zernike, m_max, w0=None):
    """P_m(theta_j) for m = -M .. M -> complex [2M+1, n_theta] (row m + M)."""
    nphi = n_phi_for(m_max)
    phi = np.arange(nphi, dtype=np.float64) * (2.0 * math.pi / nphi)
    TH, PH = np.meshgrid(theta, phi, indexing="ij")
    sin_t, cos_t = np.sin(TH), np.cos(TH)
    w = gibson_lanni_phase(opt, sin_t)
    if zernike is not None and len(zernike):
        w = w + zernike_phase(np.asarray(zernike, dtype=np.float64), sin_t / opt.s_max, PH)
    if w0 is not None:
        w = w + np.asarray(w0, dtype=np.float64)[:, None]
    f = amplitude(opt, cos_t, sin_t) * np.exp(1j * w)
    spec = np.fft.fft(f, axis=1) / nphi          # spec[:, k] = sum f e^{-2 pi i k n / N}
    m = np.arange(-m_max, m_max + 1)
    return spec[:, m % nphi].T


def channel_coeffs(pol):
    """coef[c][kind] for the kinds (g_0, P_l), (g_2, P_{l-2}), (g_2, P_{l+2}),
    (g_1, P_{l-1}), (g_1, P_{l+1})."""
    px, py = pol
    return np.array([
        [0.5 * px, 0.25 * (px - 1j * py), 0.25 * (px + 1j * py), 0.0, 0.0],
        [0.5 * py, 0.25 * (-1j * px - py), 0.25 * (1j * px - py), 0.0, 0.0],
        [0.0, 0.0, 0.0, -0.5 * (px - 1j * py), -0.5 * (px + 1j * py)]], dtype=np.complex128)


KIND_G = (0, 2, 2, 1, 1)         # which g_n
KIND_SHIFT = (0, -2, 2, -1, 1)   # P index = l + shift


def adaptive_order(P, m_max, tail_tol):
    """Largest |m| <= m_max with max_theta |P_m| > tail_tol max_theta |P_0|,
    0 if none (P [2 m_max + 1, n_theta], row m + m_max)."""
    amax = np.max(np.abs(P), axis=1)
    lim = tail_tol * amax[m_max]
    for M in range(m_max, 0, -1):
        if amax[m_max + M] > lim or amax[m_max - M] > lim:
            return M
    return 0


def harmonic_profiles(opt, n_theta, r, zs, zernike, m_max, w0=None, tail_tol=0.0):
    """I_{c,l}(r_i, z) -> complex [nz, 3, 2M+5, len(r)] (order index l + M + 2).
    With tail_tol > 0 the harmonics beyond the emitter's adaptive order
    (adaptive_order) are dropped (set to zero) first."""
    th, wt = gl_rule(n_theta, opt.theta_max)
    sin_t, cos_t = np.sin(th), np.cos(th)
    g = angular_weights(opt, sin_t, cos_t)
    P = pupil_harmonics(opt, th, zernike, m_max, w0)
    if tail_tol > 0.0:
        M = adaptive_order(P, m_max, tail_tol)
        keep = np.abs(np.arange(-m_max, m_max + 1)) <= M
        P = np.where(keep[:, None], P, 0.0)
    coef = channel_coeffs(model_pol(opt))
    arg = opt.k * np.outer(np.asarray(r, dtype=np.float64), sin_t)
    zs = np.asarray(zs, dtype=np.float64)
    L = m_max + 2
    out = np.zeros((len(zs), 3, 2 * L + 1, arg.shape[0]), dtype=np.complex128)
    for li, l in enumerate(range(-L, L + 1)):
        kern = jv(l, arg) * wt[None, :]
        F = np.zeros((3, len(th)), dtype=np.complex128)
        for kind in range(5):
            mi = l + KIND_SHIFT[kind]
            if abs(mi) > m_max:
                continue
            gp = g[KIND_G[kind]] * P[mi + m_max]
            for c in range(3):
                if coef[c, kind] != 0:
                    F[c] += coef[c, kind] * gp
        for iz, z in enumerate(zs):
            dz = np.exp(1j * opt.k * z * cos_t)
            out[iz, :, li] = (kern @ (F * dz[None, :]).T).T
    return out


def field_from_harmonics(I, cos_p, sin_p):
    """E_c = -i sum_l i^l e^{i l phi} I_{c,l} for I [3, 2L+1, ...]."""
    L = (I.shape[1] - 1) // 2
    e1 = cos_p + 1j * sin_p
    out = []
    for c in range(3):
        acc = 0.0
        for li, l in enumerate(range(-L, L + 1)):
            acc = acc + (1j ** l) * (e1 ** l) * I[c, li]
        out.append(-1j * acc)
    return out


def field_harmonic(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike, m_max, w0=None,
                   tail_tol=0.0):
    """E [nz, 3, nx, ny]: profiles on the radial grid, interpolated."""
    r, r_max = radial_grid(n_r, nx, ny, dx, dy)
    prof = harmonic_profiles(opt, n_theta, r, zs, zernike, m_max, w0, tail_tol)
    rho, cos_p, sin_p = pixel_polar(nx, ny, dx, dy)
    E = np.empty((len(zs), 3, nx, ny), dtype=np.complex128)
    for iz in range(len(zs)):
        Ii = interpolate(prof[iz], r_max, rho)          # [3, 2L+1, nx, ny]
        E[iz] = np.stack(field_from_harmonics(Ii, cos_p, sin_p))
    return E


def field_harmonic_direct(opt, n_theta, nx, ny, dx, dy, zs, zernike, m_max):
    """E [nz, 3, nx, ny] with the radial integrals at every pixel radius."""
    rho, cos_p, sin_p = pixel_polar(nx, ny, dx, dy)
    prof = harmonic_profiles(opt, n_theta, rho.ravel(), zs, zernike, m_max)
    E = np.empty((len(zs), 3, nx, ny), dtype=np.complex128)
    for iz in range(len(zs)):
        Ii = prof[iz].reshape(3, prof.shape[2], nx, ny)
        E[iz] = np.stack(field_from_harmonics(Ii, cos_p, sin_p))
    return E


def psf_harmonic(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike, m_max, w0=None,
                 tail_tol=0.0):
    E = field_harmonic(opt, n_theta, n_r, nx, ny, dx, dy, zs, zernike, m_max, w0, tail_tol)
    return np.sum(E.real ** 2 + E.imag ** 2, axis=1)


def psf_harmonic_batch(opt, depths, zernikes, z_offsets, zs, n_theta, n_r, nx, ny,
                       dx, dy, m_max, emitters=None, tail_tol=0.0):
    """Batched emitters, packed [z_offsets[-1], nx, ny] (or the listed ones)."""
    z_offsets = np.asarray(z_offsets)
    zs = np.asarray(zs, dtype=np.float64)
    sel = range(len(depths)) if emitters is None else emitters
    out = []
    for e in sel:
        o = opt.with_depth(depths[e])
        out.append(psf_harmonic(o, n_theta, n_r, nx, ny, dx, dy,
                                zs[z_offsets[e]:z_offsets[e + 1]],
                                None if zernikes is None else zernikes[e], m_max,
                                tail_tol=tail_tol))
    return np.concatenate(out, axis=0)
