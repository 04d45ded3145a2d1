"""Pins of the scalar model (Eq. 3, Eq. 5) and of the Fresnel transmission
coefficients (Eq. 6-7) in the oracle (CPU only)."""
import numpy as np
import pytest

from oracle import bessel, bessel_adjoint, continuum, fourier, scalar
from oracle.optics import Optics, fresnel_coefficients
from paper_2502_03170_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def opt_of(base, **kw):
    d = dict(base)
    d.update(kw)
    return Optics.from_dict(d)


# ---------------------------------------------------------------- scalar model
def test_scalar_spherical_equals_continuum():
    """Eq. 5 is the phi integral of Eq. 4 done exactly: equal theta nodes give
    the same sum as the direct (theta, phi) quadrature."""
    zc = np.zeros(11)
    zc[3], zc[10] = 0.3, -0.2
    o = opt_of(W.optics_gibson_lanni(1.0), scalar=True)
    rho = np.array([0.0, 0.05, 0.2, 0.37])
    zs = [-0.3, 0.4]
    E = scalar.scalar_spherical(o, 200, rho, zs, zc)
    C = np.array([continuum.field_points(o, rho, 0 * rho, np.full(4, z), zernike=zc,
                                         n_theta=200, n_phi=64)[0] for z in zs])
    assert np.max(np.abs(E - C)) <= 1e-12 * np.max(np.abs(C))


def test_scalar_through_the_vectorial_profiles():
    """The spherical machinery with g_0 = 2 sin, g_1 = g_2 = 0 and x polarisation
    reproduces Eq. 5 on the radial grid (same interpolation)."""
    o = opt_of(W.optics_gibson_lanni(2.0), scalar=True)
    zc = np.zeros(11)
    zc[3] = 0.25
    args = (48, 40, 11, 12, 0.04, 0.035, [-0.5, 0.2])
    I1 = bessel.psf_bessel(o, *args, zernike=zc)
    I2 = scalar.scalar_spherical_psf(o, *args, zernike=zc)
    assert np.max(np.abs(I1 - I2)) <= 1e-12 * np.max(I2)


def test_scalar_cartesian_equals_fourier_oracle_and_converges():
    o = opt_of(W.optics_gibson_lanni(1.0), scalar=True)
    zc = np.zeros(21)
    zc[5] = 0.2                                   # m != 0 is fine on this path
    grid = dict(nx=6, ny=6, dx=0.06, dy=0.06, z=[0.25])
    E3 = scalar.scalar_cartesian(o, 48, grid, zc)
    Ef = fourier.field_separable(o, 48, grid, zc)
    assert np.max(np.abs(Ef[:, 1:])) == 0.0
    assert np.max(np.abs(Ef[:, 0] - E3)) <= 1e-12 * np.max(np.abs(E3))
    xs = fourier.grid_coords(6, 0.06)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    ec = continuum.field_points(o, X.ravel(), Y.ravel(), np.full(36, 0.25), zernike=zc,
                                n_theta=300, n_phi=256)[0].reshape(6, 6)
    errs = []
    for N in (32, 64, 128):
        E = scalar.scalar_cartesian(o, N, grid, zc)[0]
        errs.append(np.max(np.abs(E - ec)) / np.max(np.abs(ec)))
    assert errs[2] < errs[0] and errs[2] < 2e-2


def test_scalar_is_the_low_na_limit_of_the_vectorial_model():
    """abs(I_vec - I_scalar) / max I = O(NA^2) for x polarisation."""
    errs = []
    for NA in (0.2, 0.1):
        base = dict(W.optics_plain(), NA=NA, pol=(1.0, 0.0))
        ov, os_ = opt_of(base), opt_of(base, scalar=True)
        args = (64, 32, 9, 9, 0.3, 0.3, [0.0, 1.0])
        Iv = bessel.psf_bessel(ov, *args)
        Is = bessel.psf_bessel(os_, *args)
        errs.append(np.max(np.abs(Iv - Is)) / np.max(Is))
    assert errs[1] < errs[0] / 3.0 and errs[1] < 1e-2


# -------------------------------------------------------------- Fresnel (Eq. 7)
def test_fresnel_index_matched_is_identity():
    base = dict(W.optics_plain(), n_s=1.518, n_g=1.518, pol=W.CIRCULAR)
    o1, o2 = opt_of(base), opt_of(base, fresnel=True)
    st = np.linspace(0, 0.92, 7)
    qs, qp = fresnel_coefficients(o2, st)
    assert np.allclose(qs, 1.0, atol=1e-15) and np.allclose(qp, 1.0, atol=1e-15)
    grid = dict(nx=8, ny=7, dx=0.05, dy=0.05, z=[0.1])
    I1 = fourier.psf_fourier(o1, 32, grid)
    assert np.max(np.abs(I1 - fourier.psf_fourier(o2, 32, grid))) <= 1e-14 * np.max(I1)


def test_fresnel_normal_incidence_closed_form():
    o = opt_of(W.optics_gibson_lanni(1.0), fresnel=True)
    qs, qp = fresnel_coefficients(o, np.array([0.0]))
    ref = (2 * o.n_s / (o.n_s + o.n_g)) * (2 * o.n_g / (o.n_g + o.n_i))
    assert abs(qs[0] - ref) < 1e-15 and abs(qp[0] - ref) < 1e-15


def test_fresnel_energy_conservation_single_interface():
    """Sample -> immersion with a matched coverslip: with the Stokes relations
    r_s = t_s - 1, r_p = (n_2/n_1) t_p - 1, reflectance + transmittance = 1 for
    both polarisations at every sub-critical angle."""
    o = opt_of(dict(W.optics_gibson_lanni(1.0), n_g=1.518), fresnel=True)
    n1, n2 = o.n_s, o.n_i
    st = np.linspace(0.0, 0.99 * n1 / n2, 9)          # immersion-side sin(theta)
    ts, tp = fresnel_coefficients(o, st)
    c2 = np.sqrt(1 - st ** 2)
    c1 = np.sqrt(1 - (n2 * st / n1) ** 2)
    factor = (n2 * c2) / (n1 * c1)
    rs, rp = ts - 1.0, (n2 / n1) * tp - 1.0
    assert np.allclose(np.abs(rs) ** 2 + factor * np.abs(ts) ** 2, 1.0, atol=1e-13)
    assert np.allclose(np.abs(rp) ** 2 + factor * np.abs(tp) ** 2, 1.0, atol=1e-13)


@pytest.mark.parametrize("pol", [W.CIRCULAR, (1.0, 0.0)])
def test_fresnel_bessel_equals_continuum(pol):
    """Eq. 10-11 with the Fresnel weights g_n equals the direct quadrature of
    Eq. 9 with the Fresnel far field (NA 1.4 > n_s: complex q past the
    critical angle)."""
    o = opt_of(dict(W.optics_gibson_lanni(1.0), pol=pol), fresnel=True)
    zc = np.zeros(11)
    zc[10] = 0.2
    xs = np.array([0.0, 0.07, -0.15, 0.21])
    ys = np.array([0.0, 0.11, 0.05, -0.3])
    zs = np.array([0.0, 0.3, -0.2, 0.5])
    ec = continuum.field_points(o, xs, ys, zs, zernike=zc, n_theta=300, n_phi=128)
    rho = np.hypot(xs, ys)
    eb = np.empty((3, 4), dtype=np.complex128)
    for i in range(4):
        prof = bessel.profiles(o, 300, [rho[i]], [zs[i]], zc)[0, :, 0]
        c = xs[i] / rho[i] if rho[i] > 0 else 1.0
        s = ys[i] / rho[i] if rho[i] > 0 else 0.0
        eb[:, i] = bessel.field_from_profiles(*prof, c, s, o.pol)
    assert np.max(np.abs(eb - ec)) <= 1e-12 * np.max(np.abs(ec))


def test_fresnel_fourier_converges_to_continuum():
    o = opt_of(dict(W.optics_gibson_lanni(1.0), pol=W.CIRCULAR), fresnel=True)
    xs = fourier.grid_coords(6, 0.06)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    ec = continuum.field_points(o, X.ravel(), Y.ravel(), np.full(36, 0.25),
                                n_theta=300, n_phi=256).reshape(3, 6, 6)
    grid = dict(nx=6, ny=6, dx=0.06, dy=0.06, z=[0.25])
    errs = []
    for N in (32, 64, 128):
        E = fourier.field_separable(o, N, grid)[0]
        errs.append(np.max(np.abs(E - ec)) / np.max(np.abs(ec)))
    assert errs[2] < errs[0] and errs[2] < 2e-2


def test_adjoint_with_fresnel_and_scalar_fd():
    """The Bessel adjoint oracle (B^H for the complex Fresnel operand) against
    central differences of the forward oracle."""
    geo = dict(n_theta=20, n_r=24, nx=9, ny=8, dx=0.06, dy=0.05)
    zs = np.array([-0.3, 0.4])
    for kw in (dict(fresnel=True), dict(scalar=True)):
        o = opt_of(dict(W.optics_gibson_lanni(0.0), pol=W.CIRCULAR), **kw).with_depth(2.0)
        T = np.random.default_rng(3).uniform(0, 1e-3, (2, geo["nx"], geo["ny"]))
        w0 = 0.2 * np.cos(np.arange(20))
        L, gW, _, gd, _ = bessel_adjoint.emitter_loss_and_grads(
            o, geo["n_theta"], geo["n_r"], geo["nx"], geo["ny"], geo["dx"], geo["dy"], zs,
            None, w0, True, T, None)

        def loss(w, depth):
            I = bessel.psf_bessel(o.with_depth(depth), geo["n_theta"], geo["n_r"], geo["nx"],
                                  geo["ny"], geo["dx"], geo["dy"], zs, None, True, w)
            return float(np.sum((I - T) ** 2))
        h = 1e-5
        for j in (0, 11):
            wp, wm = w0.copy(), w0.copy()
            wp[j] += h
            wm[j] -= h
            fd = (loss(wp, 2.0) - loss(wm, 2.0)) / (2 * h)
            assert abs(fd - gW[j]) <= 1e-6 * np.max(np.abs(gW)), (kw, j)
        fd = (loss(w0, 2.0 + h) - loss(w0, 2.0 - h)) / (2 * h)
        assert abs(fd - gd) <= 1e-6 * abs(fd), kw
