"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: a closed
form (Airy, Eq. 18), an independent parameterisation of the same integral
(continuum quadrature of Eq. 9 vs the Bessel form Eq. 10-11 vs the Cartesian
form Eq. 8), exact invariants (Parseval, symmetry), convergence orders printed
in Sec. 5.2.2, Zernike orthonormality, Gauss-Legendre exactness, the paraxial
expansion of Eq. 13-14, and finite differences for the adjoint.
"""
import math

import numpy as np
import pytest
from scipy.special import j1

from oracle import adjoint, bessel, continuum, fourier, scalar
from oracle.optics import (Optics, far_field, gibson_lanni_phase, noll_to_nm,
                           pupil_geometry, pupil_mask, zernike)
from paper_2502_03170_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def airy(opt, rho):
    v = opt.k * opt.s_max * np.asarray(rho, dtype=np.float64)
    safe = np.where(v > 0, v, 1.0)
    return np.where(v > 0, -1j * opt.s_max ** 2 * j1(safe) / safe,
                    -0.5j * opt.s_max ** 2)


def slope(h, e):
    return np.polyfit(np.log(h), np.log(e), 1)[0]


# ---------------------------------------------------------------- Eq. 18 ----
def test_airy_closed_form_bessel_gl():
    opt = Optics.from_dict(W.optics_plain())
    rho = np.linspace(0.0, 1.5, 61)
    e = scalar.scalar_bessel_paraxial(opt, rho, 64, "gl")
    assert np.max(np.abs(e - airy(opt, rho))) < 1e-13


def test_airy_convergence_orders():
    """Sec. 5.2.2: Riemann first order, Simpson fourth order, Cartesian
    between first and second order (delta = L2 norm against Eq. 18)."""
    opt = Optics.from_dict(W.optics_plain())
    rho = np.linspace(0.0, 1.0, 101)
    ref = airy(opt, rho)
    ns = (16, 32, 64, 128, 256)
    h = [opt.theta_max / n for n in ns]
    er = [np.linalg.norm(scalar.scalar_bessel_paraxial(opt, rho, n, "riemann")
                         - ref) for n in ns]
    es = [np.linalg.norm(scalar.scalar_bessel_paraxial(opt, rho, n, "simpson")
                         - ref) for n in ns]
    assert 0.9 < slope(h, er) < 1.1
    assert 3.8 < slope(h, es) < 4.3
    ef, hf = [], []
    for n in (16, 32, 64, 128, 256):
        E, xs = scalar.scalar_fourier_paraxial(opt, n, 33, 0.02)
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        ef.append(np.linalg.norm(E - airy(opt, np.hypot(X, Y))))
        hf.append(2.0 / n)
    assert 1.0 < slope(hf, ef) < 2.0


# --------------------------------------------- equivalence theorem (Sec 4.1) -
POINTS = [(0.0, 0.0, 0.0), (0.1, 0.05, 0.3), (0.25, -0.1, -0.5),
          (0.03, 0.2, 0.0), (-0.31, 0.12, 0.8)]


@pytest.mark.parametrize("pol", [(1.0, 0.0), W.CIRCULAR, (0.6, 0.8j * 0.5 + 0.3)])
@pytest.mark.parametrize("aberr", ["none", "gl_zernike"])
def test_bessel_equals_continuum(pol, aberr):
    """Eq. 10-11 (Bessel) = Eq. 9 (direct theta-phi quadrature)."""
    d = W.optics_plain() if aberr == "none" else W.optics_gibson_lanni(2.0)
    d["pol"] = pol
    opt = Optics.from_dict(d)
    zc = np.zeros(21)
    if aberr != "none":
        zc[3], zc[10], zc[21 - 1] = 0.3, -0.2, 0.0
    xs, ys, zs = map(np.array, zip(*POINTS))
    ec = continuum.field_points(opt, xs, ys, zs, zernike=zc, n_theta=400,
                                n_phi=96)
    for i, (x, y, z) in enumerate(POINTS):
        r = math.hypot(x, y)
        cp, sp = (x / r, y / r) if r > 0 else (1.0, 0.0)
        prof = bessel.profiles(opt, 400, [r], [z], zernike=zc)
        eb = np.array(bessel.field_from_profiles(
            prof[0, 0, 0], prof[0, 1, 0], prof[0, 2, 0], cp, sp, opt.pol))
        assert np.max(np.abs(eb - ec[:, i])) < 1e-12 * np.max(np.abs(ec))


def test_fourier_converges_to_continuum():
    """Eq. 8 midpoint sum -> Eq. 9 as the pupil grid refines (any W)."""
    opt = Optics.from_dict(W.optics_gibson_lanni(1.0))
    zc = np.zeros(21)
    zc[3], zc[5], zc[7], zc[10] = 0.2, 0.3, -0.15, -0.1   # incl. m != 0
    grid = dict(nx=6, ny=6, dx=0.06, dy=0.06, z=[0.25])
    xg = fourier.grid_coords(6, 0.06)
    X, Y = np.meshgrid(xg, xg, indexing="ij")
    ec = continuum.field_points(opt, X.ravel(), Y.ravel(), np.full(36, 0.25),
                                zernike=zc, n_theta=300, n_phi=256)
    errs = []
    for n in (32, 64, 128, 256):
        E = fourier.field_separable(opt, n, grid, zernike=zc)
        errs.append(np.max(np.abs(E[0].reshape(3, -1) - ec)) / np.max(np.abs(ec)))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 2e-2


def test_fourier_bessel_agree_axisymmetric():
    """The two strategies give the same stack for an axisymmetric pupil."""
    opt = Optics.from_dict(W.optics_gibson_lanni(0.5))
    zc = np.zeros(21)
    zc[3], zc[10] = 0.2, 0.1
    zs = [-0.4, 0.0, 0.4]
    If = fourier.psf_fourier(opt, 512, dict(nx=8, ny=8, dx=0.05, dy=0.05, z=zs),
                             zernike=zc)
    Eb = bessel.field_bessel_direct(opt, 200, 8, 8, 0.05, 0.05, zs, zernike=zc)
    Ib = np.sum(np.abs(Eb) ** 2, axis=1)
    assert np.max(np.abs(If - Ib)) / np.max(Ib) < 1e-2


# ------------------------------------------------------- discrete structure --
def test_brute_equals_separable():
    opt = Optics.from_dict(W.optics_gibson_lanni(1.0))
    zc = np.zeros(21)
    zc[4], zc[6] = 0.3, -0.2
    g = np.random.default_rng(1)
    pm = g.normal(0, 0.5, (16, 16))
    grid = dict(nx=6, ny=5, dx=0.04, dy=0.05, z=[-0.3, 0.0, 0.6])
    Eb = fourier.field_brute(opt, 16, grid, zc, pm)
    Es = fourier.field_separable(opt, 16, grid, zc, pm)
    assert np.max(np.abs(Eb - Es)) < 1e-12 * np.max(np.abs(Es))


def test_parseval_full_period():
    """On the unzoomed full-period grid (dx = lambda/(2 NA), N_out = N_p) the
    zoom matrices are sqrt(N)-unitary: sum |E_c|^2 dx^2 =
    |C|^2 ds^2 (2 pi/k)^2 sum |P_c|^2, for every z."""
    opt = Optics.from_dict(W.optics_gibson_lanni(1.0))
    n = 24
    dx = opt.lam / (2 * opt.NA)
    E = fourier.field_separable(opt, n, dict(nx=n, ny=n, dx=dx, dy=dx,
                                             z=[-0.7, 0.0, 1.3]))
    P, _ = fourier.pupil_field(opt, n)
    ds = 2 * opt.s_max / n
    for iz in range(3):
        for c in range(3):
            lhs = np.sum(np.abs(E[iz, c]) ** 2) * dx * dx
            rhs = (ds * 2 * math.pi / opt.k / (2 * math.pi)) ** 2 * np.sum(
                np.abs(P[c]) ** 2)
            assert abs(lhs / rhs - 1) < 1e-12


def test_far_field_is_unitary():
    """Eq. 6 with q_s = q_p = 1 preserves |e|^2 = |e_inc|^2 (no energy change
    in the basis change; the energy factor is the apodization of Eq. 16)."""
    g = np.random.default_rng(2)
    th = g.uniform(0, 1.2, 50)
    ph = g.uniform(0, 2 * math.pi, 50)
    for pol in [(1, 0), (0, 1), W.CIRCULAR, (0.3 + 0.2j, -0.5j)]:
        ef = far_field(np.cos(th), np.sin(th), np.cos(ph), np.sin(ph), pol)
        n2 = sum(np.abs(e) ** 2 for e in ef)
        assert np.allclose(n2, abs(pol[0]) ** 2 + abs(pol[1]) ** 2, atol=1e-14)


@pytest.mark.parametrize("pol", [(1.0, 0.0), W.CIRCULAR])
def test_axial_symmetry_aberration_free(pol):
    d = W.optics_plain()
    d["pol"] = pol
    opt = Optics.from_dict(d)
    zs = np.linspace(-1, 1, 6)
    I = fourier.psf_fourier(opt, 32, dict(nx=12, ny=12, dx=0.03, dy=0.03, z=zs))
    if pol == (1.0, 0.0):
        assert np.max(np.abs(I - I[::-1])) < 1e-12 * I.max()
    else:
        # circular light changes handedness under z -> -z: on the discrete
        # grid (only 90-degree rotational symmetry) the reflected stack is the
        # mirror image I(x, -y, -z) = I(x, y, z), exactly.
        assert np.max(np.abs(I - I[::-1, :, ::-1])) < 1e-12 * I.max()
        assert np.max(np.abs(I - I[::-1])) < 1e-3 * I.max()
    Ib = bessel.psf_bessel(opt, 64, 64, 12, 12, 0.03, 0.03, zs)
    assert np.max(np.abs(Ib - Ib[::-1])) < 1e-12 * Ib.max()
    # Gibson-Lanni breaks it (Sec. 5.1: spherical aberration)
    og = Optics.from_dict(dict(W.optics_gibson_lanni(1.0), pol=pol))
    Ig = fourier.psf_fourier(og, 32, dict(nx=12, ny=12, dx=0.03, dy=0.03, z=zs))
    assert np.max(np.abs(Ig - Ig[::-1, :, ::-1])) > 1e-2 * Ig.max()


def test_rotational_symmetry_circular():
    opt = Optics.from_dict(W.optics_gibson_lanni(1.0))
    zc = np.zeros(21)
    zc[3], zc[10] = 0.3, 0.2
    I = fourier.psf_fourier(opt, 32, dict(nx=10, ny=10, dx=0.04, dy=0.04,
                                          z=[-0.3, 0.4]), zernike=zc)
    for iz in range(2):
        # 90-degree rotations map the pupil grid onto itself; a mirror would
        # flip the handedness of circular light, so only rotations are exact.
        assert np.max(np.abs(I[iz] - np.rot90(I[iz]))) < 1e-12 * I.max()
        assert np.max(np.abs(I[iz] - np.rot90(I[iz], 2))) < 1e-12 * I.max()
    ol = Optics.from_dict(dict(W.optics_plain(), pol=(1.0, 0.0)))
    Il = fourier.psf_fourier(ol, 32, dict(nx=10, ny=10, dx=0.04, dy=0.04,
                                          z=[0.0]))[0]
    assert np.max(np.abs(Il - Il[::-1, :])) < 1e-12 * Il.max()   # mirror x
    assert np.max(np.abs(Il - Il.T)) > 1e-3 * Il.max()           # not round


def test_low_na_limit():
    """At low NA the vectorial intensity tends to the scalar one (Sec. 3.3)."""
    diffs = []
    for na in (0.1, 0.2):
        d = dict(W.optics_plain(), NA=na, pol=(1.0, 0.0), apodize=False)
        opt = Optics.from_dict(d)
        g = dict(nx=8, ny=8, dx=0.3, dy=0.3, z=[0.0, 1.0])
        Iv = fourier.psf_fourier(opt, 48, g)
        # scalar model of Eq. 3 with the same 1/s_z weighting: the x channel
        # of a far field equal to the incident field.
        P, cos_t = fourier.pupil_field(opt, 48)
        mask = pupil_mask(48)
        Ps = np.where(mask, 1.0 / np.where(mask, cos_t, 1.0), 0.0)
        ds = 2 * opt.s_max / 48
        Ax = fourier.zoom_matrix(opt, 48, 8, 0.3)
        Is = []
        for z in g["z"]:
            E = fourier.C_FOURIER * ds * ds * (
                Ax @ (Ps * np.exp(1j * opt.k * z * cos_t)) @ Ax.T)
            Is.append(np.abs(E) ** 2)
        Is = np.array(Is)
        diffs.append(np.max(np.abs(Iv - Is)) / Is.max())
    assert diffs[0] < 1e-2
    assert 2.5 < diffs[1] / diffs[0] < 6.0            # O(NA^2)


# ------------------------------------------------------------- Zernike -------
def test_zernike_orthonormal():
    """Noll RMS normalisation: (1/pi) int_disk Z_i Z_j = delta_ij."""
    x, w = np.polynomial.legendre.leggauss(40)
    r = 0.5 * (x + 1)
    wr = 0.5 * w
    nph = 64
    ph = np.arange(nph) * 2 * math.pi / nph
    R, PH = np.meshgrid(r, ph, indexing="ij")
    wgt = (wr[:, None] * R) * (2 * math.pi / nph) / math.pi
    Z = np.array([zernike(j, R, PH) for j in range(1, 29)])
    G = np.einsum("iab,jab,ab->ij", Z, Z, wgt)
    assert np.max(np.abs(G - np.eye(28))) < 1e-12


def test_zernike_noll_conventions():
    u = np.linspace(-0.9, 0.9, 8)
    U, V = np.meshgrid(u, u, indexing="ij")
    rho, phi = np.hypot(U, V), np.arctan2(V, U)
    # tip/tilt are linear in x / y; j even -> cosine, j odd -> sine
    assert np.allclose(zernike(2, rho, phi) / U, zernike(2, rho, phi)[-1, 0] / U[-1, 0])
    assert np.allclose(zernike(3, rho, phi) / V, zernike(3, rho, phi)[0, -1] / V[0, -1])
    for j in range(2, 40):
        n, m = noll_to_nm(j)
        assert (n - abs(m)) % 2 == 0 and abs(m) <= n
        if m != 0:
            assert (m > 0) == (j % 2 == 0)
        # every radial polynomial is 1 at the rim
        assert abs(zernike(j, np.array(1.0), np.array(0.0 if m >= 0 else math.pi / (2 * abs(m))))
                   - math.sqrt((2.0 if m else 1.0) * (n + 1))) < 1e-12
    # the ordering visits each (n, m) once
    seen = {noll_to_nm(j) for j in range(1, 67)}
    assert len(seen) == 66


# ------------------------------------------------------- Gibson-Lanni ---------
def test_gibson_lanni_zero_depth_is_zero():
    opt = Optics.from_dict(W.optics_gibson_lanni(0.0))
    s = np.linspace(0, opt.s_max, 50)
    assert np.max(np.abs(gibson_lanni_phase(opt, s))) < 1e-9


def test_gibson_lanni_paraxial_defocus():
    """Eq. 13 with t_i from Eq. 14: W(s) - W(0) ~ -(k0 n_i t_s / 2) s^2 for
    small s (the s^2 terms of all layers combine into one defocus)."""
    for depth in (0.5, 2.0, 7.0):
        opt = Optics.from_dict(W.optics_gibson_lanni(depth))
        s = np.array([1e-3, 2e-3])
        w = gibson_lanni_phase(opt, s) - gibson_lanni_phase(opt, np.zeros(1))
        c = (w / s ** 2).real
        expect = -(2 * math.pi / opt.lam) * opt.n_i * depth / 2
        assert np.allclose(c, expect, rtol=1e-5)


def test_gibson_lanni_evanescent():
    opt = Optics.from_dict(W.optics_gibson_lanni(2.0))
    s = np.linspace(0, opt.s_max, 200)
    w = gibson_lanni_phase(opt, s)
    ev = opt.n_i * s > opt.n_s
    assert np.all(np.abs(w.imag[~ev]) < 1e-12)
    assert np.all(w.imag[ev] > 0)                       # decay, |e^{iW}| < 1
    assert np.all(np.abs(np.exp(1j * w[ev])) < 1)


# --------------------------------------------------- quadrature / interp -----
def test_gauss_legendre_exactness():
    th, w = bessel.gl_rule(10, 1.3)
    for deg in range(20):
        assert abs(np.sum(w * th ** deg) - 1.3 ** (deg + 1) / (deg + 1)) < 1e-12 * max(1, 1.3 ** deg)


def test_radial_interpolation_second_order():
    opt = Optics.from_dict(W.optics_plain())
    Ed = bessel.field_bessel_direct(opt, 128, 16, 16, 0.03, 0.03, [0.2])
    errs = []
    for nr in (32, 64, 128, 256):
        E = bessel.field_bessel(opt, 128, nr, 16, 16, 0.03, 0.03, [0.2])
        errs.append(np.linalg.norm(E - Ed))
    assert 1.8 < slope([1.0 / 32, 1.0 / 64, 1.0 / 128, 1.0 / 256], errs) < 2.2


def test_not_axisymmetric_rejected():
    opt = Optics.from_dict(W.optics_plain())
    zc = np.zeros(21)
    zc[5] = 0.1
    with pytest.raises(bessel.NotAxisymmetric):
        bessel.profiles(opt, 16, [0.1], [0.0], zernike=zc)
    p1 = bessel.profiles(opt, 16, [0.1], [0.0], zernike=zc, project=True)
    p0 = bessel.profiles(opt, 16, [0.1], [0.0])
    assert np.allclose(p1, p0)


# ------------------------------------------------------------- adjoint -------
def test_adjoint_matches_finite_differences():
    opt = Optics.from_dict(W.optics_gibson_lanni(1.0))
    n = 16
    grid = dict(nx=8, ny=8, dx=0.05, dy=0.05, z=[-0.4, 0.3])
    g = np.random.default_rng(3)
    zc = np.zeros(21)
    zc[3:9] = g.normal(0, 0.2, 6)
    pm = np.where(pupil_mask(n), g.normal(0, 0.3, (n, n)), 0.0)
    target = g.uniform(0, 1e-3, (2, 8, 8))
    L, gW, gc, _ = adjoint.loss_and_grad(opt, n, grid, zc, pm, target)
    h = 1e-6
    mask = pupil_mask(n)
    idx = [(p, q) for p in range(n) for q in range(n) if mask[p, q]]
    for k in g.choice(len(idx), 12, replace=False):
        p, q = idx[k]
        d = np.zeros((n, n))
        d[p, q] = h
        lp = adjoint.loss(fourier.psf_fourier(opt, n, grid, zc, pm + d), target)
        lm = adjoint.loss(fourier.psf_fourier(opt, n, grid, zc, pm - d), target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gW[p, q]) <= 1e-6 * np.max(np.abs(gW)) + 1e-7 * abs(fd)
    for j in range(21):
        d = np.zeros(21)
        d[j] = h
        lp = adjoint.loss(fourier.psf_fourier(opt, n, grid, zc + d, pm), target)
        lm = adjoint.loss(fourier.psf_fourier(opt, n, grid, zc - d, pm), target)
        assert abs((lp - lm) / (2 * h) - gc[j]) <= 1e-6 * np.max(np.abs(gc))
    # Taylor remainder of a random direction decays as h^2
    dirn = np.where(mask, g.normal(0, 1, (n, n)), 0.0)
    rem = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        le = adjoint.loss(fourier.psf_fourier(opt, n, grid, zc, pm + eps * dirn),
                          target)
        rem.append(abs(le - L - eps * np.sum(gW * dirn)))
    assert 3.0 < rem[0] / rem[1] < 5.0 and 3.0 < rem[1] / rem[2] < 5.0


def test_noll_table_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "noll_table.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 22
    for j, n, m in rows:
        assert noll_to_nm(int(j)) == (int(n), int(m))
