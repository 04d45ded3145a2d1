"""Optical model pieces shared by every oracle strategy (FP64, test-only).

Conventions (each is a reading of the paper where it is silent or
ambiguous):

* k = 2*pi*n_i/lambda: theta is defined in the immersion medium (Sec. 3.1).
* The prefactor f*k of Eq. 1 is set to 1, so the Cartesian form carries
  -i/(2*pi) and the spherical form -i/2 (Eq. 8 / Eq. 10).
* The pupil coordinates of the Gibson-Lanni / Zernike footnote (Sec. 3.4) are
  normalised: sin(theta) = (NA/n_i) * sqrt(u^2 + v^2) with u, v in [-1, 1];
  the Zernike radius is sqrt(u^2 + v^2) = sin(theta)/s_max.
* Fresnel coefficients q_s = q_p = 1 (Eq. 7 is not applied).
* Zernike polynomials follow Noll's ordering and RMS normalisation, phi measured
  from +x (pupil index p) towards +y (pupil index q), coefficients in radians.
"""
import math

import numpy as np


class Optics:
    """Physical parameters of Eq. 1, Eq. 13-14 and Eq. 16-17 (lengths in um)."""

    def __init__(self, NA, lam, n_i, n_s=None, n_g=None, n_i_design=None,
                 n_g_design=None, t_g=170.0, t_g_design=None, t_i_design=150.0,
                 depth=0.0, pol=(1.0, 0.0), apodize=True, s_env=0.0,
                 scalar=False, fresnel=False):
        self.NA = float(NA)
        self.lam = float(lam)
        self.n_i = float(n_i)
        self.n_s = float(n_i if n_s is None else n_s)
        self.n_g = float(1.5 if n_g is None else n_g)
        self.n_i_design = float(self.n_i if n_i_design is None else n_i_design)
        self.n_g_design = float(self.n_g if n_g_design is None else n_g_design)
        self.t_g = float(t_g)
        self.t_g_design = float(self.t_g if t_g_design is None else t_g_design)
        self.t_i_design = float(t_i_design)
        self.depth = float(depth)
        self.pol = (complex(pol[0]), complex(pol[1]))
        self.apodize = bool(apodize)
        self.s_env = float(s_env)
        self.scalar = bool(scalar)        # Eq. 3 / Eq. 5: e_far = e_inc, one channel
        self.fresnel = bool(fresnel)      # Eq. 6 with the q_s, q_p of Eq. 7

    @classmethod
    def from_dict(cls, d):
        keys = ("NA", "lam", "n_i", "n_s", "n_g", "n_i_design", "n_g_design",
                "t_g", "t_g_design", "t_i_design", "depth", "pol", "apodize",
                "s_env", "scalar", "fresnel")
        return cls(**{k: d[k] for k in keys if k in d})

    def with_depth(self, depth):
        o = Optics.__new__(Optics)
        o.__dict__.update(self.__dict__)
        o.depth = float(depth)
        return o

    # Sec. 3.1: k = 2 pi n / lambda with n the immersion index; s_max = NA/n_i.
    @property
    def k(self):
        return 2.0 * math.pi * self.n_i / self.lam

    @property
    def s_max(self):
        return self.NA / self.n_i

    @property
    def theta_max(self):
        return math.asin(self.s_max)


# ----------------------------------------------------------------------------
# Pupil grid (Cartesian parameterisation, Eq. 8): cell-centred midpoint nodes.
# ----------------------------------------------------------------------------
def pupil_nodes(n_pupil):
    """Normalised node coordinates u_p = (2p+1-N)/N, p = 0..N-1."""
    p = np.arange(n_pupil, dtype=np.float64)
    return (2.0 * p + 1.0 - n_pupil) / n_pupil


def pupil_mask(n_pupil):
    """Disk s_x^2 + s_y^2 <= s_max^2 tested exactly on integers:
    (2p+1-N)^2 + (2q+1-N)^2 <= N^2 (mask[p, q], p along x, q along y)."""
    m = 2 * np.arange(n_pupil, dtype=np.int64) + 1 - n_pupil
    return (m[:, None] ** 2 + m[None, :] ** 2) <= n_pupil * n_pupil


def pupil_geometry(opt, n_pupil):
    """sin(theta), cos(theta), cos(phi), sin(phi) on the pupil grid.

    Returns arrays [N, N] indexed [p, q]; outside the disk the values are
    meaningless (the mask removes them).  At the exact centre (odd N) phi is
    undefined; cos(phi)=1, sin(phi)=0 is used there, which is harmless because
    every phi-dependent term of Eq. 6 is multiplied by sin(theta) or
    (1 - cos(theta)), both zero at the centre.
    """
    u = pupil_nodes(n_pupil)
    U, V = np.meshgrid(u, u, indexing="ij")
    rn = np.sqrt(U * U + V * V)
    sin_t = opt.s_max * rn
    cos_t = np.sqrt(np.clip(1.0 - sin_t * sin_t, 0.0, None))
    safe = rn > 0
    cos_p = np.where(safe, U / np.where(safe, rn, 1.0), 1.0)
    sin_p = np.where(safe, V / np.where(safe, rn, 1.0), 0.0)
    return sin_t, cos_t, cos_p, sin_p, rn, np.arctan2(V, U)


# ----------------------------------------------------------------------------
# Eq. 6: far field on the Gaussian reference sphere, q_s = q_p = 1.
# ----------------------------------------------------------------------------
def far_field(cos_t, sin_t, cos_p, sin_p, pol, q_s=1.0, q_p=1.0):
    """e_inf = [x, y, z] components for an incident field (pol_x, pol_y).

    Written as the two columns of Eq. 6 (the e_inc^x and e_inc^y columns),
    each divided by two as in the paper.
    """
    px, py = pol
    cos2 = cos_p * cos_p - sin_p * sin_p
    sin2 = 2.0 * sin_p * cos_p
    # column multiplying e_inc^x / 2
    cx = (q_s * (1.0 - cos2) + q_p * (1.0 + cos2) * cos_t,
          (-q_s + q_p * cos_t) * sin2,
          -2.0 * q_p * cos_p * sin_t)
    # column multiplying e_inc^y / 2
    cy = ((-q_s + q_p * cos_t) * sin2,
          q_s * (1.0 + cos2) + q_p * (1.0 - cos2) * cos_t,
          -2.0 * q_p * sin_p * sin_t)
    return [0.5 * (cx[i] * px + cy[i] * py) for i in range(3)]


def fresnel_coefficients(opt, sin_t):
    """q_s, q_p of Eq. 7: products over the interfaces sample -> coverslip ->
    immersion.  The angle in medium m follows from Snell's law,
    n_m sin(theta_m) = n_i sin(theta), with cos(theta_m) the principal complex
    root (Im >= 0) where medium m is evanescent."""
    media = [opt.n_s, opt.n_g, opt.n_i]
    nis = opt.n_i * np.asarray(sin_t, dtype=np.float64)
    cos_m = [np.sqrt((1.0 - (nis / n) ** 2).astype(np.complex128) + 0j) for n in media]
    qs = np.ones_like(cos_m[0])
    qp = np.ones_like(cos_m[0])
    for m in range(len(media) - 1):
        n1, n2, c1, c2 = media[m], media[m + 1], cos_m[m], cos_m[m + 1]
        qs = qs * (2.0 * n1 * c1 / (n1 * c1 + n2 * c2))
        qp = qp * (2.0 * n1 * c1 / (n2 * c1 + n1 * c2))
    return qs, qp


def far_field_model(opt, cos_t, sin_t, cos_p, sin_p):
    """The far field the model uses: scalar (Sec. 3.2: e_far = e_inc = 1 in
    channel 0), vectorial with q_s = q_p = 1, or vectorial with the Fresnel
    coefficients of Eq. 7."""
    if opt.scalar:
        one = np.ones(np.shape(cos_t), dtype=np.complex128)
        return [one, 0.0 * one, 0.0 * one]
    if opt.fresnel:
        qs, qp = fresnel_coefficients(opt, sin_t)
        return far_field(cos_t, sin_t, cos_p, sin_p, opt.pol, qs, qp)
    return far_field(cos_t, sin_t, cos_p, sin_p, opt.pol)


# ----------------------------------------------------------------------------
# Eq. 16-17: amplitude correction factors.
# ----------------------------------------------------------------------------
def amplitude(opt, cos_t, sin_t):
    a = np.ones_like(cos_t)
    if opt.apodize:
        a = a * np.sqrt(cos_t)                       # Eq. 16
    if opt.s_env > 0:
        a = a * np.exp(-(sin_t * sin_t) / (opt.s_env * opt.s_env))   # Eq. 17
    return a


# ----------------------------------------------------------------------------
# Eq. 13-14: Gibson-Lanni phase (radians, complex: Im > 0 is decay).
# ----------------------------------------------------------------------------
def immersion_thickness(opt):
    """Eq. 14 as printed: t_i = t_s + n_i(-t_s/n_s - t_g/n_g + t_g*/n_g* + t_i*/n_i*)."""
    t_s = opt.depth
    return t_s + opt.n_i * (-t_s / opt.n_s - opt.t_g / opt.n_g
                            + opt.t_g_design / opt.n_g_design
                            + opt.t_i_design / opt.n_i_design)


def _layer_root(n, n_i, sin_t):
    """sqrt(n^2 - n_i^2 sin^2 theta), principal complex root (Im >= 0)."""
    arg = n * n - (n_i * sin_t) ** 2
    return np.sqrt(arg.astype(np.complex128) + 0j)


def gibson_lanni_phase(opt, sin_t):
    """W(s) of Eq. 13 in radians, complex where a layer is evanescent."""
    t_i = immersion_thickness(opt)
    n_i = opt.n_i
    opl = (opt.depth * _layer_root(opt.n_s, n_i, sin_t)
           + t_i * _layer_root(n_i, n_i, sin_t)
           - opt.t_i_design * _layer_root(opt.n_i_design, n_i, sin_t)
           + opt.t_g * _layer_root(opt.n_g, n_i, sin_t)
           - opt.t_g_design * _layer_root(opt.n_g_design, n_i, sin_t))
    return (2.0 * math.pi / opt.lam) * opl


# ----------------------------------------------------------------------------
# Eq. 15: Zernike polynomials, Noll ordering and normalisation.
# ----------------------------------------------------------------------------
def noll_to_nm(j):
    """Noll index j >= 1 -> (n, m); m > 0 is cos(m phi), m < 0 is sin(|m| phi).

    Within radial order n the index runs over increasing |m|; for m != 0 an
    even j takes the cosine and an odd j the sine (Noll 1976).
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    k = j - n * (n + 1) // 2 - 1          # 0-based position within order n
    if n % 2 == 0:
        am = 2 * ((k + 1) // 2)
    else:
        am = 2 * (k // 2) + 1
    if am == 0:
        return n, 0
    return (n, am) if j % 2 == 0 else (n, -am)


def zernike_radial(n, am, rho):
    """R_n^{|m|}(rho) = sum_s (-1)^s (n-s)! / (s! ((n+m)/2-s)! ((n-m)/2-s)!) rho^(n-2s)."""
    out = np.zeros_like(rho, dtype=np.float64)
    for s in range((n - am) // 2 + 1):
        c = ((-1) ** s * math.factorial(n - s)
             / (math.factorial(s) * math.factorial((n + am) // 2 - s)
                * math.factorial((n - am) // 2 - s)))
        out = out + c * rho ** (n - 2 * s)
    return out


def zernike(j, rho, phi):
    """Z_j(rho, phi), RMS-normalised on the unit disk."""
    n, m = noll_to_nm(j)
    r = zernike_radial(n, abs(m), rho)
    if m == 0:
        return math.sqrt(n + 1.0) * r
    norm = math.sqrt(2.0 * (n + 1.0))
    if m > 0:
        return norm * r * np.cos(m * phi)
    return norm * r * np.sin(-m * phi)


def zernike_phase(coeffs, rho, phi, axisymmetric_only=False):
    """sum_j c_j Z_j (coeffs[j-1] multiplies Noll index j), radians."""
    w = np.zeros_like(rho, dtype=np.float64)
    for idx, c in enumerate(coeffs):
        if c == 0.0:
            continue
        j = idx + 1
        if axisymmetric_only and noll_to_nm(j)[1] != 0:
            continue
        w = w + c * zernike(j, rho, phi)
    return w
