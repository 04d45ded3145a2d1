"""Pins of the azimuthal-harmonic (non-axisymmetric) Bessel oracle, CPU only.

* With an axisymmetric pupil it is Eq. 10-11 term by term: equal to the
  axisymmetric oracle to round-off for every polarisation and model.
* With m != 0 Zernike terms, evaluated at the pixel radii, it equals the
  direct quadrature of Eq. 9 (same Gauss-Legendre theta nodes, trapezoid in
  phi): the harmonic algebra, the Jacobi-Anger signs and the far-field
  harmonics are fixed by an independent computation.
* The truncation order from the tail bound keeps the error below the bound.
"""
import numpy as np
import pytest

from oracle import bessel, bessel_harmonic as bh, continuum
from oracle.optics import Optics
from paper_2502_03170_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def opt_of(**kw):
    d = W.optics_gibson_lanni(1.5)
    d.update(kw)
    return Optics.from_dict(d)


def nonaxial_zernike():
    z = np.zeros(21)
    z[4], z[5] = 0.12, -0.08      # astigmatism (Noll 5, 6)
    z[6], z[7] = 0.05, 0.09       # coma (7, 8)
    z[8] = -0.06                  # trefoil (9)
    z[10] = 0.1                   # spherical (11, m = 0)
    z[3] = 0.2                    # defocus (4, m = 0)
    return z


@pytest.mark.parametrize("kw", [dict(pol=W.CIRCULAR), dict(pol=(1.0, 0.0)),
                                dict(pol=(0.6, 0.48 + 0.64j)), dict(scalar=True),
                                dict(fresnel=True, pol=W.CIRCULAR)])
def test_axisymmetric_pupil_is_eq10(kw):
    o = opt_of(**kw)
    zc = np.zeros(11)
    zc[3], zc[10] = 0.3, -0.2
    args = (40, 48, 9, 11, 0.04, 0.035, [-0.4, 0.3])
    Eb = bessel.field_bessel(o, *args, zernike=zc)
    for m_max in (0, 3):
        Eh = bh.field_harmonic(o, *args, zc, m_max)
        assert np.max(np.abs(Eh - Eb)) <= 1e-13 * np.max(np.abs(Eb)), m_max


@pytest.mark.parametrize("kw", [dict(pol=W.CIRCULAR), dict(pol=(0.6, 0.48 + 0.64j)),
                                dict(scalar=True), dict(fresnel=True, pol=(1.0, 0.0))])
def test_harmonics_equal_direct_quadrature(kw):
    o = opt_of(**kw)
    zc = nonaxial_zernike()
    m_max = bh.harmonic_order(zc, tol=1e-12)
    nx, ny, dx, dy = 5, 4, 0.07, 0.06
    zs = [0.35]
    Eh = bh.field_harmonic_direct(o, 60, nx, ny, dx, dy, zs, zc, m_max)[0]
    xs = (np.arange(nx) - (nx - 1) / 2) * dx
    ys = (np.arange(ny) - (ny - 1) / 2) * dy
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    Ec = continuum.field_points(o, X.ravel(), Y.ravel(), np.full(nx * ny, zs[0]), zernike=zc,
                                n_theta=60, n_phi=256).reshape(3, nx, ny)
    assert np.max(np.abs(Eh - Ec)) <= 1e-10 * np.max(np.abs(Ec))
    # the m != 0 terms matter: dropping them changes the field at the 1e-2 level
    z0 = zc.copy()
    for j in (4, 5, 6, 7, 8):
        z0[j] = 0.0
    E0 = bh.field_harmonic_direct(o, 60, nx, ny, dx, dy, zs, z0, m_max)[0]
    assert np.max(np.abs(E0 - Ec)) > 1e-2 * np.max(np.abs(Ec))


def test_truncation_bound():
    o = opt_of(pol=W.CIRCULAR)
    zc = nonaxial_zernike()
    args = (50, 5, 5, 0.06, 0.06, [0.1])
    ref = bh.field_harmonic_direct(o, *args, zc, bh.harmonic_order(zc, tol=1e-13))[0]
    errs = {}
    for tol in (1e-3, 1e-5, 1e-7):
        m_max = bh.harmonic_order(zc, tol=tol)
        E = bh.field_harmonic_direct(o, *args, zc, m_max)[0]
        errs[tol] = np.max(np.abs(E - ref)) / np.max(np.abs(ref))
        assert errs[tol] <= tol, (tol, m_max, errs[tol])
    assert errs[1e-7] < errs[1e-3]
    # no m != 0 term: order 0
    assert bh.harmonic_order(np.array([0, 0, 0, 0.3, 0, 0, 0, 0, 0, 0, 0.1])) == 0


def test_pupil_harmonics_are_the_fourier_series():
    """P_m for a single pure harmonic term: e^{i a cos(2 phi)} has the
    Jacobi-Anger coefficients i^k J_k(a) at m = 2k (A = 1 without GL)."""
    d = dict(W.optics_plain(), apodize=0)
    o = Optics.from_dict(d)
    th = np.array([0.3, 0.7, 1.0])
    zc = np.zeros(6)
    zc[5] = 0.4                           # Noll 6: sqrt(6) rho^2 cos 2 phi
    P = bh.pupil_harmonics(o, th, zc, 12)
    a = 0.4 * np.sqrt(6.0) * (np.sin(th) / o.s_max) ** 2
    from scipy.special import jv
    for m in range(-12, 13):
        expect = (1j ** (m // 2)) * jv(m // 2, a) if m % 2 == 0 else 0.0 * a
        assert np.allclose(P[m + 12], expect, atol=1e-13), m


def test_adaptive_order_keeps_the_error_within_the_tolerance():
    """The adaptive order from the computed harmonics is far below the bound
    order, and the field it gives stays within the tolerance of the
    bound-order field (and of the direct quadrature of Eq. 9)."""
    o = opt_of(pol=W.CIRCULAR)
    zc = nonaxial_zernike()
    m_bound = bh.harmonic_order(zc, tol=1e-7)
    th, _ = bessel.gl_rule(50, o.theta_max)
    P = bh.pupil_harmonics(o, th, zc, m_bound)
    m_eff = bh.adaptive_order(P, m_bound, 1e-7)
    assert 0 < m_eff < m_bound
    args = (50, 5, 5, 0.06, 0.06, [0.1, -0.3])
    ref = bh.field_harmonic_direct(o, *args, zc, m_bound)
    Eb = np.stack([bh.field_harmonic_direct(o, *args, zc, m_eff)])[0]
    assert np.max(np.abs(Eb - ref)) <= 1e-6 * np.max(np.abs(ref))
    # the same through the profile path with the adaptive switch
    Ia = bh.psf_harmonic(o, 40, 48, 9, 11, 0.04, 0.035, [0.2], zc, m_bound, tail_tol=1e-7)
    Ib = bh.psf_harmonic(o, 40, 48, 9, 11, 0.04, 0.035, [0.2], zc, m_bound)
    assert np.max(np.abs(Ia - Ib)) <= 2e-6 * np.max(Ib)
