"""Scalar propagators (Eq. 3, Eq. 5) and Fresnel transmission (Eq. 6-7) on
the GPU, through the C ABI, against the FP64 oracle (pinned on the CPU).

Tolerances as for the vectorial model: intensity max-rel 1e-5 (FP32 and
split FP16), 1e-4 (split BF16); gradients relative L2 1e-4."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import bessel as ob
from oracle import bessel_adjoint as oba
from oracle import fourier as of
from oracle import scalar as osc
from oracle.optics import pupil_mask
from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import max_rel, oracle_optics, rel_l2

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "split_fp16": 1e-5, "split_bf16": 1e-5}


def model(base, **kw):
    d = dict(base)
    d.update(kw)
    return d


@pytest.mark.parametrize("prec", ["fp32", "split_fp16", "split_bf16"])
def test_fourier_scalar(lib, prec):
    d = model(W.optics_gibson_lanni(1.5), scalar=True)
    zc = np.zeros(21)
    zc[3:12] = np.random.default_rng(2).normal(0, 0.15, 9)
    grid = dict(nx=40, ny=24, dx=0.03, dy=0.035, z=np.linspace(-0.6, 0.6, 5))
    I = api.fourier(d, 64, grid, zernike=zc, precision=prec).cpu().numpy()
    E = osc.scalar_cartesian(oracle_optics(d), 64, grid, zc)
    assert max_rel(I, E.real ** 2 + E.imag ** 2) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "split_fp16", "split_bf16"])
@pytest.mark.parametrize("pol", [W.CIRCULAR, (0.6, 0.48 + 0.64j)])
def test_fourier_fresnel(lib, prec, pol):
    d = model(W.optics_gibson_lanni(1.5), fresnel=True, pol=pol)
    zc = np.zeros(21)
    zc[3:12] = np.random.default_rng(3).normal(0, 0.15, 9)
    grid = dict(nx=32, ny=40, dx=0.03, dy=0.03, z=np.linspace(-0.5, 0.7, 4))
    I = api.fourier(d, 64, grid, zernike=zc, precision=prec).cpu().numpy()
    Ir = of.psf_fourier(oracle_optics(d), 64, grid, zc)
    assert max_rel(I, Ir) <= TOL[prec]
    # the coefficients change the PSF (NA 1.4 crosses the sample's critical angle)
    I0 = of.psf_fourier(oracle_optics(model(d, fresnel=False)), 64, grid, zc)
    assert max_rel(I0, Ir) > 1e-2


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_bessel_scalar(lib, prec):
    d = model(W.optics_gibson_lanni(0.0), scalar=True)
    g = np.random.default_rng(4)
    depth = np.array([0.5, 3.0, 7.0])
    zern = np.zeros((3, 11))
    zern[:, 3] = g.normal(0, 0.2, 3)
    zern[:, 10] = g.normal(0, 0.1, 3)
    offs = np.array([0, 2, 3, 6], dtype=np.int32)
    z = np.array([-0.4, 0.3, 0.0, -0.8, 0.1, 0.9])
    geo = (64, 48, 20, 18, 0.03, 0.025)
    I = api.bessel(d, depth, zern, offs, z, *geo, precision=prec).cpu().numpy()
    o = oracle_optics(d)
    for e in range(3):
        a, b = offs[e], offs[e + 1]
        Ir = osc.scalar_spherical_psf(o.with_depth(depth[e]), *geo, z[a:b], zern[e])
        assert max_rel(I[a:b], Ir) <= TOL[prec], e


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
@pytest.mark.parametrize("geo,nz", [((80, 48, 17, 20, 0.03, 0.03), (3, 2)),
                                    ((200, 300, 64, 61, 0.02, 0.02), (40, 1, 57, 9))])
def test_bessel_fresnel(lib, prec, geo, nz):
    """Complex angular weights (Eq. 7 in Eq. 11).  Split FP16 runs the radial
    contraction per order n with g_n on the F operand; the second case spans
    several radius tiles (300 radii), slice tiles straddling the order planes
    and a ragged theta tail (200 nodes)."""
    d = model(W.optics_gibson_lanni(0.0), fresnel=True, pol=W.CIRCULAR)
    g = np.random.default_rng(len(nz))
    n_em = len(nz)
    depth = g.uniform(0.5, 5.0, n_em)
    zern = np.zeros((n_em, 11))
    zern[:, 10] = g.normal(0, 0.15, n_em)
    zern[:, 3] = g.normal(0, 0.2, n_em)
    offs = np.concatenate([[0], np.cumsum(nz)]).astype(np.int32)
    z = g.uniform(-0.8, 0.8, int(offs[-1]))
    I = api.bessel(d, depth, zern, offs, z, *geo, precision=prec).cpu().numpy()
    opt = oracle_optics(d)
    for e in range(n_em):
        a, b = offs[e], offs[e + 1]
        Ir = ob.psf_bessel_batch(opt, depth, zern, offs, z, *geo, emitters=[e])
        assert max_rel(I[a:b], Ir) <= 1e-5, e


@pytest.mark.parametrize("kw", [dict(fresnel=True), dict(scalar=True)])
def test_fourier_backward_models(lib, kw):
    from .test_gpu_backward import gpu_backward
    rng = np.random.default_rng(9)
    d = model(W.optics_gibson_lanni(1.0), pol=W.CIRCULAR, **kw)
    N, nx, ny, nz = 32, 16, 24, 3
    grid = dict(nx=nx, ny=ny, dx=0.03, dy=0.035, z=np.linspace(-0.4, 0.5, nz))
    zern = np.zeros((1, 21))
    zern[0, 3:12] = rng.normal(0, 0.2, 9)
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (1, N, N)), 0.0)
    T = rng.uniform(0, 2e-4, (1, nz, nx, ny))
    L, gWr, gcr, _ = oadj.loss_and_grad(oracle_optics(d), N, grid, zern[0], pm[0], T[0])
    for prec in ("fp32", "split_fp16"):
        loss, gW, gc = gpu_backward(d, N, grid, zern, pm, target=T, prec=prec)
        assert rel_l2(gW[0], gWr) <= 1e-4, prec
        assert rel_l2(gc[0], gcr) <= 1e-4, prec


def test_bessel_backward_scalar(lib):
    d = model(W.optics_gibson_lanni(0.0), scalar=True)
    g = np.random.default_rng(5)
    depth = np.array([1.0, 5.0])
    zern = np.zeros((2, 11))
    zern[:, 3] = g.normal(0, 0.2, 2)
    offs = np.array([0, 3, 5], dtype=np.int32)
    z = np.array([-0.3, 0.1, 0.5, -0.6, 0.2])
    w0 = 0.3 * g.normal(size=(2, 24))
    geo = dict(n_theta=24, n_r=40, nx=12, ny=12, dx=0.04, dy=0.04)
    o = oracle_optics(d)
    T = ob.psf_bessel_batch(o, depth + 0.5, zern, offs, z, geo["n_theta"], geo["n_r"],
                            geo["nx"], geo["ny"], geo["dx"], geo["dy"])
    for prec in ("fp32", "split_fp16"):
        res = api.bessel_backward(d, depth, zern, offs, z, target=T, phase_theta=w0,
                                  precision=prec, **geo)
        ref = oba.loss_and_grads_batch(o, depth, zern, offs, z, phase_theta=w0, target=T,
                                       **geo)
        torch.cuda.synchronize()
        assert rel_l2(res["grad_phase_theta"].cpu().numpy(), ref[1]) <= 1e-4, prec
        assert rel_l2(res["grad_depth"].cpu().numpy(), ref[3]) <= 1e-4, prec
