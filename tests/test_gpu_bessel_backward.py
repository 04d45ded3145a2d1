"""Adjoint of the Bessel strategy on the GPU (through the C ABI) against the
FP64 adjoint oracle, which the CPU tests pin with finite differences.

Tolerance: relative L2 <= 1e-4 for every gradient (the gradient bound of the
workloads); the loss to 1e-5 relative.  Each gradient is compared over the
whole batch (per-emitter depth gradients are sums of terms of both signs, so
one emitter's value can be small against its terms)."""
import numpy as np
import pytest
import torch

from oracle import bessel as ob
from oracle import bessel_adjoint as oa
from paper_2502_03170_gb300 import _lib, api, autograd
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import oracle_optics, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4
PRECS = ["fp32", "split_fp16", "split_bf16"]


def batch(seed=3, nz=(3, 1, 4, 2), n_theta=24):
    g = np.random.default_rng(seed)
    n_em = len(nz)
    depth = g.uniform(0.0, 6.0, n_em)
    zern = np.zeros((n_em, 15))
    zern[:, 3] = g.normal(0, 0.3, n_em)      # Z_4
    zern[:, 10] = g.normal(0, 0.2, n_em)     # Z_11
    zern[:, 5] = g.normal(0, 0.2, n_em)      # Z_6 (m != 0, projected away)
    offs = np.zeros(n_em + 1, dtype=np.int32)
    offs[1:] = np.cumsum(nz)
    z = np.concatenate([np.sort(g.uniform(-1.0, 1.0, n)) for n in nz])
    w0 = 0.4 * g.normal(size=(n_em, n_theta))
    return depth, zern, offs, z, w0


def target_for(opt, depth, zern, offs, z, geo, seed=11):
    """A synthetic measured stack: the oracle's PSFs of shifted emitters with
    5 % multiplicative noise."""
    g = np.random.default_rng(seed)
    I = ob.psf_bessel_batch(opt, depth + 0.4, 0.5 * zern, offs, z, geo["n_theta"],
                            geo["n_r"], geo["nx"], geo["ny"], geo["dx"], geo["dy"],
                            project=True)
    return I * (1.0 + 0.05 * g.normal(size=I.shape))


class SampledSlices:
    """dL/dI of a few emitters' slices, indexed like the packed stack."""

    def __init__(self, chunks):
        self.chunks = chunks

    def __getitem__(self, sl):
        return self.chunks[(int(sl.start), int(sl.stop))]


def compare(res, ref, loss=True):
    L, gW, gc, gd = ref
    torch.cuda.synchronize()
    if loss:
        assert rel_l2(res["loss"].cpu().numpy(), L) <= 1e-5
    assert rel_l2(res["grad_phase_theta"].cpu().numpy(), gW) <= TOL
    assert rel_l2(res["grad_zernike"].cpu().numpy(), gc) <= TOL
    assert rel_l2(res["grad_depth"].cpu().numpy(), gd) <= TOL


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("pol", [W.CIRCULAR, (1.0, 0.0), (0.6, 0.48 + 0.64j)])
@pytest.mark.parametrize("nx,ny", [(9, 8), (16, 16), (13, 21)])
def test_target_loss_parity(lib, pol, nx, ny, prec):
    geo = dict(n_theta=24, n_r=40, nx=nx, ny=ny, dx=0.05, dy=0.045)
    d = dict(W.optics_gibson_lanni(0.0), pol=pol)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch()
    T = target_for(opt, depth, zern, offs, z, geo)
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=True,
                              phase_theta=w0, precision=prec, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T, **geo)
    compare(res, ref)
    # m != 0 terms do not enter the spherical form
    assert torch.all(res["grad_zernike"][:, 5] == 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nx,ny,n_r", [(16, 16, 40), (13, 21, 40), (180, 177, 256)])
def test_fresnel_weights(lib, prec, nx, ny, n_r):
    """Complex g_n (Fresnel coefficients, Eq. 7 in Eq. 11): the adjoint
    contracts with B^H.  16 x 16 and 13 x 21 take the sorted epilogue and
    (split modes) the tensor-core contraction with the (Re, Im) row pairs;
    180 x 177 the one-pass epilogue and the FP32 contraction."""
    geo = dict(n_theta=24, n_r=n_r, nx=nx, ny=ny, dx=0.05 * 16 / nx, dy=0.045 * 16 / ny)
    d = dict(W.optics_gibson_lanni(0.0), pol=(0.6, 0.48 + 0.64j), fresnel=True)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=21)
    T = target_for(opt, depth, zern, offs, z, geo)
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=True,
                              phase_theta=w0, precision=prec, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T, **geo)
    compare(res, ref)


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_grad_intensity_mode_and_determinism(lib, prec):
    geo = dict(n_theta=48, n_r=96, nx=40, ny=34, dx=0.03, dy=0.03)
    d = W.optics_gibson_lanni(0.0)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=8, nz=(7, 1, 12, 5, 9, 3), n_theta=48)
    G = np.random.default_rng(4).normal(size=(len(z), geo["nx"], geo["ny"]))
    r1 = api.bessel_backward(d, depth, zern, offs, z, grad_intensity=G, project=True,
                             phase_theta=w0, precision=prec, **geo)
    r2 = api.bessel_backward(d, depth, zern, offs, z, grad_intensity=G, project=True,
                             phase_theta=w0, precision=prec, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, grad_intensity=G, **geo)
    compare(r1, ref, loss=False)
    for k in ("grad_phase_theta", "grad_zernike", "grad_depth"):
        assert torch.equal(r1[k], r2[k]), k          # fixed-order reductions


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_several_tiles_ragged(lib, prec):
    """More slices than one contraction tile (64) and theta nodes spanning
    several 32-wide tiles with a ragged tail."""
    geo = dict(n_theta=70, n_r=64, nx=24, ny=24, dx=0.04, dy=0.04)
    d = W.optics_gibson_lanni(0.0)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=5, nz=(40, 3, 33, 1, 29), n_theta=70)
    T = target_for(opt, depth, zern, offs, z, geo, seed=2)
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=True,
                              phase_theta=w0, precision=prec, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T, **geo)
    compare(res, ref)


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_large_grid_generic_path(lib, prec):
    """A grid whose mirror groups do not fit in shared memory takes the
    one-pass epilogue and the FP32 contraction."""
    geo = dict(n_theta=20, n_r=256, nx=180, ny=177, dx=0.012, dy=0.012)
    d = W.optics_gibson_lanni(0.0)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=12, nz=(2, 1), n_theta=20)
    T = target_for(opt, depth, zern, offs, z, geo)
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=True,
                              phase_theta=w0, precision=prec, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T, **geo)
    compare(res, ref)


def test_empty_stack_and_rejected_emitter(lib):
    geo = dict(n_theta=16, n_r=24, nx=8, ny=8, dx=0.05, dy=0.05)
    d = W.optics_gibson_lanni(0.0)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=9, nz=(2, 0, 3), n_theta=16)
    T = target_for(opt, depth, zern, offs, z, geo)
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=True,
                              phase_theta=w0, **geo)
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T, **geo)
    compare(res, ref)
    assert torch.all(res["grad_phase_theta"][1] == 0) and res["loss"][1] == 0
    # without projection an m != 0 coefficient rejects the emitter: zero gradients
    ws = api.Workspace()
    res = api.bessel_backward(d, depth, zern, offs, z, target=T, project=False,
                              phase_theta=w0, workspace=ws, **geo)
    torch.cuda.synchronize()
    assert ws.status() == _lib.PSF_ERR_NOT_AXISYMMETRIC
    assert torch.all(res["grad_phase_theta"] == 0)


def test_autograd_matches_backward(lib):
    geo = dict(n_theta=24, n_r=40, nx=12, ny=12, dx=0.05, dy=0.05)
    d = W.optics_gibson_lanni(0.0)
    opt = oracle_optics(d)
    depth, zern, offs, z, w0 = batch(seed=6)
    T = torch.as_tensor(target_for(opt, depth, zern, offs, z, geo), device="cuda",
                        dtype=torch.float32)
    dep = torch.tensor(depth, device="cuda", requires_grad=True)
    zc = torch.tensor(zern, device="cuda", requires_grad=True)
    ph = torch.tensor(w0, device="cuda", dtype=torch.float32, requires_grad=True)
    I = autograd.bessel_psf(dep, zc, ph, d, offs, z, geo["n_theta"], geo["n_r"],
                            geo["nx"], geo["ny"], geo["dx"], geo["dy"])
    ((I - T) ** 2).sum().backward()
    ref = oa.loss_and_grads_batch(opt, depth, zern, offs, z, phase_theta=w0,
                                  project=True, target=T.cpu().numpy().astype(np.float64),
                                  **geo)
    assert rel_l2(ph.grad.cpu().numpy(), ref[1]) <= TOL
    assert rel_l2(zc.grad.cpu().numpy(), ref[2]) <= TOL
    assert rel_l2(dep.grad.cpu().numpy(), ref[3]) <= TOL


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_bessel_backward_full_size_sampled(lib, prec):
    """The batched workload (4096 emitters, 147k slices of 128^2 px, 200 theta
    nodes, 256 radii) in one backward call with a seeded dL/dI; sampled
    emitters recomputed by the oracle."""
    c = W.bessel()
    n_sl = int(c["z_offsets"][-1])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    G = torch.randn((n_sl, c["nx"], c["ny"]), device="cuda", generator=gen)
    res = api.bessel_backward(c["optics"], c["depth"], c["zernike"], c["z_offsets"],
                              c["z"], c["n_theta"], c["n_r"], c["nx"], c["ny"], c["dx"],
                              c["dy"], grad_intensity=G, project=True, precision=prec)
    torch.cuda.synchronize()
    opt = oracle_optics(c["optics"])
    offs = c["z_offsets"]
    sample = (0, 1733, 4095)
    Gs = SampledSlices({(int(offs[e]), int(offs[e + 1])):
                        G[int(offs[e]):int(offs[e + 1])].cpu().numpy() for e in sample})
    del G
    ref = oa.loss_and_grads_batch(opt, c["depth"], c["zernike"], offs, c["z"],
                                  c["n_theta"], c["n_r"], c["nx"], c["ny"], c["dx"],
                                  c["dy"], project=True, grad_intensity=Gs,
                                  emitters=sample)
    gw = res["grad_phase_theta"].cpu().numpy()[list(sample)]
    gc = res["grad_zernike"].cpu().numpy()[list(sample)]
    gd = res["grad_depth"].cpu().numpy()[list(sample)]
    assert rel_l2(gw, ref[1]) <= TOL
    assert rel_l2(gc, ref[2]) <= TOL
    assert rel_l2(gd, ref[3]) <= TOL
    torch.cuda.empty_cache()
