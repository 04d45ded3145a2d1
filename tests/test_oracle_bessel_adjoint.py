"""Pins of the Bessel-strategy adjoint oracle (CPU only).

Every gradient is checked against central finite differences of the forward
oracle (:func:`oracle.bessel.psf_bessel_batch`), which shares none of the
adjoint's backward steps: a dropped conjugate, a wrong sign of the Eq. 10
matrix, a transposed interpolation or a missing evanescent part of
dW_GL/dt_s each fail one of these."""
import numpy as np
import pytest

from oracle import bessel as ob
from oracle import bessel_adjoint as oa
from oracle.optics import Optics
from paper_2502_03170_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

# small, ragged case: odd/even grid, pixel on no axis, 3 planes
CASE = dict(n_theta=20, n_r=24, nx=9, ny=8, dx=0.06, dy=0.05)
ZS = np.array([-0.4, 0.1, 0.7])


def optics(pol=(1.0, 1j), depth=2.0):
    d = W.optics_gibson_lanni(depth)
    d["pol"] = (pol[0] / np.sqrt(2.0), pol[1] / np.sqrt(2.0))
    return Optics.from_dict(d)


def coeffs():
    c = np.zeros(12)
    c[3] = 0.3      # Z_4 defocus (m = 0)
    c[10] = -0.2    # Z_11 spherical (m = 0)
    c[4] = 0.25     # Z_5 astigmatism (m != 0): dropped by the projection
    return c


def loss_fn(opt, depth, c, w0, T=None, G=None):
    I = ob.psf_bessel(opt.with_depth(depth), CASE["n_theta"], CASE["n_r"], CASE["nx"],
                      CASE["ny"], CASE["dx"], CASE["dy"], ZS, c, project=True, w0=w0)
    if T is not None:
        return float(np.sum((I - T) ** 2))
    return float(np.sum(G * I))


def reference_target(opt):
    g = np.random.default_rng(5)
    I = ob.psf_bessel(opt.with_depth(1.5), CASE["n_theta"], CASE["n_r"], CASE["nx"],
                      CASE["ny"], CASE["dx"], CASE["dy"], ZS, None)
    return I * (1.0 + 0.1 * g.normal(size=I.shape))


def analytic(opt, depth, c, w0, T=None, G=None):
    return oa.emitter_loss_and_grads(opt.with_depth(depth), CASE["n_theta"], CASE["n_r"],
                                     CASE["nx"], CASE["ny"], CASE["dx"], CASE["dy"], ZS,
                                     c, w0, True, T, G)


@pytest.mark.parametrize("pol", [(1.0, 1j), (1.0, 0.0), (0.6, -0.8j)])
def test_phase_gradient_fd(pol):
    opt = optics(pol)
    T = reference_target(opt)
    w0 = 0.3 * np.sin(np.arange(CASE["n_theta"]))
    L, gW, _, _, _ = analytic(opt, 2.0, coeffs(), w0, T=T)
    assert abs(L - loss_fn(opt, 2.0, coeffs(), w0, T=T)) <= 1e-12 * L
    h = 1e-5
    for j in (0, 7, CASE["n_theta"] - 1):
        wp, wm = w0.copy(), w0.copy()
        wp[j] += h
        wm[j] -= h
        fd = (loss_fn(opt, 2.0, coeffs(), wp, T=T) - loss_fn(opt, 2.0, coeffs(), wm, T=T)) / (2 * h)
        assert abs(fd - gW[j]) <= 1e-6 * np.max(np.abs(gW)), (j, fd, gW[j])


def test_zernike_and_depth_gradient_fd():
    opt = optics()
    T = reference_target(opt)
    c = coeffs()
    _, gW, gc, gd, _ = analytic(opt, 2.0, c, None, T=T)
    h = 1e-5
    for q in (3, 10):                                   # m = 0 terms
        cp, cm = c.copy(), c.copy()
        cp[q] += h
        cm[q] -= h
        fd = (loss_fn(opt, 2.0, cp, None, T=T) - loss_fn(opt, 2.0, cm, None, T=T)) / (2 * h)
        assert abs(fd - gc[q]) <= 1e-6 * abs(fd), (q, fd, gc[q])
    assert gc[4] == 0.0                                 # projected m != 0 term
    # depth: NA 1.4 > n_s 1.33, so the sample layer is evanescent near the rim
    # and dW_GL/dt_s is complex there
    fd = (loss_fn(opt, 2.0 + h, c, None, T=T) - loss_fn(opt, 2.0 - h, c, None, T=T)) / (2 * h)
    assert abs(fd - gd) <= 1e-6 * abs(fd), (fd, gd)
    assert np.any(np.imag(oa.depth_derivative(opt, np.sin(
        ob.gl_rule(CASE["n_theta"], opt.theta_max)[0]))) != 0)


def test_piston_invariance():
    opt = optics()
    T = reference_target(opt)
    c = coeffs()
    c[0] = 0.4
    _, gW, gc, _, _ = analytic(opt, 2.0, c, None, T=T)
    assert abs(gc[0]) <= 1e-9 * np.sum(np.abs(gW))
    assert abs(np.sum(gW)) <= 1e-9 * np.sum(np.abs(gW))


def test_linear_functional_mode_fd():
    opt = optics((1.0, 0.3 + 0.2j))
    G = np.random.default_rng(9).normal(size=(len(ZS), CASE["nx"], CASE["ny"]))
    c = coeffs()
    L, gW, gc, gd, I = analytic(opt, 3.0, c, None, G=G)
    assert abs(L - np.sum(G * I)) <= 1e-12 * np.sum(np.abs(G * I))
    h = 1e-5
    fd = (loss_fn(opt, 3.0 + h, c, None, G=G) - loss_fn(opt, 3.0 - h, c, None, G=G)) / (2 * h)
    assert abs(fd - gd) <= 1e-6 * abs(fd)
    w = np.zeros(CASE["n_theta"])
    w[5] = h
    fd = (loss_fn(opt, 3.0, c, w, G=G) - loss_fn(opt, 3.0, c, -w, G=G)) / (2 * h)
    assert abs(fd - gW[5]) <= 1e-6 * np.max(np.abs(gW))


def test_batch_layout_matches_single():
    opt = optics()
    depths = np.array([0.5, 2.0])
    zc = np.stack([coeffs(), 0.5 * coeffs()])
    offs = np.array([0, 2, 5])
    zs = np.array([-0.2, 0.3, -0.5, 0.0, 0.6])
    T = np.random.default_rng(2).uniform(0, 1e-3, (5, CASE["nx"], CASE["ny"]))
    L, gW, gc, gd = oa.loss_and_grads_batch(opt, depths, zc, offs, zs, CASE["n_theta"],
                                            CASE["n_r"], CASE["nx"], CASE["ny"], CASE["dx"],
                                            CASE["dy"], project=True, target=T)
    r = oa.emitter_loss_and_grads(opt.with_depth(2.0), CASE["n_theta"], CASE["n_r"],
                                  CASE["nx"], CASE["ny"], CASE["dx"], CASE["dy"], zs[2:5],
                                  zc[1], None, True, T[2:5], None)
    assert L[1] == r[0] and np.array_equal(gW[1], r[1]) and gd[1] == r[3]
