"""Bessel strategy on the GPU (through the C ABI) against the FP64 oracle.

Tolerance per stack: max |I - I_ref| / max |I_ref| <= 1e-5 for the FP32 and
split-fp16 radial contractions; the complex profiles are held to the same
bound.  Split BF16 (16 significant bits per operand) measured 5.2e-5 on the
workload: the forward refuses it (PSF_ERR_PRECISION), as it refuses split
FP16 beyond 448 theta nodes."""
import numpy as np
import pytest
import torch

from oracle import bessel as ob
from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import max_rel, oracle_optics

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "split_fp16": 1e-5}
PRECS = ["fp32", "split_fp16"]


def small_batch(seed=7, nz=(3, 1, 4, 2, 5), with_m_nonzero=True):
    g = np.random.default_rng(seed)
    n_em = len(nz)
    depth = g.uniform(0.0, 5.0, n_em)
    zern = np.zeros((n_em, 21))
    zern[:, 3] = g.normal(0, 0.2, n_em)
    zern[:, 10] = g.normal(0, 0.1, n_em)
    if with_m_nonzero:
        zern[:, 5] = g.normal(0, 0.1, n_em)
    offs = np.zeros(n_em + 1, dtype=np.int32)
    offs[1:] = np.cumsum(nz)
    z = np.concatenate([np.sort(g.uniform(-1.2, 1.2, n)) for n in nz])
    return depth, zern, offs, z


def per_stack_max_rel(I, Ir, offs):
    return max(max_rel(I[a:b], Ir[a:b]) for a, b in zip(offs[:-1], offs[1:]) if b > a)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("pol", [W.CIRCULAR, (1.0, 0.0), (0.6, 0.48 + 0.64j)])
def test_small_batch_parity(lib, pol, prec):
    d = dict(W.optics_gibson_lanni(0.0), pol=pol)
    depth, zern, offs, z = small_batch()
    nt, nr, nx, ny, dx, dy = 64, 48, 20, 17, 0.03, 0.025
    I, P = api.bessel(d, depth, zern, offs, z, nt, nr, nx, ny, dx, dy,
                      project=True, profiles=True, precision=prec)
    torch.cuda.synchronize()
    I, P = I.cpu().numpy(), P.cpu().numpy()
    opt = oracle_optics(d)
    Ir = ob.psf_bessel_batch(opt, depth, zern, offs, z, nt, nr, nx, ny, dx, dy,
                             project=True)
    Pr = ob.profiles_batch(opt, depth, zern, offs, z, nt, nr, nx, ny, dx, dy,
                           project=True)
    assert per_stack_max_rel(I, Ir, offs) <= TOL[prec]
    assert max_rel(P, Pr) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
@pytest.mark.parametrize("nx,ny,nr,nt", [(21, 15, 32, 40), (1, 1, 2, 40),
                                         (9, 40, 300, 40), (24, 40, 64, 40),
                                         (2, 8, 2, 7), (16, 8, 1024, 130)])
def test_odd_grids_and_centre_pixel(lib, nx, ny, nr, nt, prec):
    """Odd grids put a pixel on the axis (r = 0, J_1 = J_2 = 0) and make the
    interpolation use the first radial cell; n_r = 2 is the smallest grid.
    Even grids with ny % 8 == 0 take the mirror-symmetric epilogue (an
    elliptical Jones vector makes its sin 2phi sign flips visible); theta
    counts that are not multiples of the 64-wide K tile leave a ragged tail."""
    d = dict(W.optics_gibson_lanni(0.0), pol=(0.6, 0.48 + 0.64j))
    depth, zern, offs, z = small_batch(seed=3, nz=(2, 3))
    I, P = api.bessel(d, depth, zern, offs, z, nt, nr, nx, ny, 0.021, 0.019,
                      project=True, profiles=True, precision=prec)
    torch.cuda.synchronize()
    I, P = I.cpu().numpy(), P.cpu().numpy()
    assert np.all(np.isfinite(P))
    opt = oracle_optics(d)
    Ir = ob.psf_bessel_batch(opt, depth, zern, offs, z, nt, nr, nx, ny, 0.021,
                             0.019, project=True)
    Pr = ob.profiles_batch(opt, depth, zern, offs, z, nt, nr, nx, ny, 0.021,
                           0.019, project=True)
    assert per_stack_max_rel(I, Ir, offs) <= TOL[prec]
    assert max_rel(P, Pr) <= TOL[prec]


def test_not_axisymmetric_status(lib):
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = small_batch()
    zern[:, 5] = 0.0
    zern[2, 5] = 0.1                      # emitter 2 has an m != 0 term
    ws = api.Workspace()
    I = api.bessel(d, depth, zern, offs, z, 32, 32, 8, 8, 0.03, 0.03,
                   project=False, workspace=ws)
    assert ws.status() == _lib.PSF_ERR_NOT_AXISYMMETRIC
    I2 = api.bessel(d, depth, zern, offs, z, 32, 32, 8, 8, 0.03, 0.03,
                    project=True, workspace=ws)
    assert ws.status() == _lib.PSF_OK
    I, I2 = I.cpu().numpy(), I2.cpu().numpy()
    for e in (0, 1, 3, 4):
        a, b = offs[e], offs[e + 1]
        assert np.array_equal(I[a:b], I2[a:b])


@pytest.mark.parametrize("prec", PRECS)
def test_bessel_config_full_size_sampled(lib, prec):
    """The batched workload (4096 emitters, uneven stacks, 200 theta nodes,
    256 radii, 128^2 px) in one call; sampled emitters recomputed by the
    oracle."""
    c = W.bessel()
    I = api.bessel(c["optics"], c["depth"], c["zernike"], c["z_offsets"], c["z"],
                   c["n_theta"], c["n_r"], c["nx"], c["ny"], c["dx"], c["dy"],
                   project=True, precision=prec)
    torch.cuda.synchronize()
    opt = oracle_optics(c["optics"])
    offs = c["z_offsets"]
    for e in (0, 1733, 4095):
        a, b = int(offs[e]), int(offs[e + 1])
        Ie = I[a:b].cpu().numpy()
        Ir = ob.psf_bessel_batch(opt, c["depth"], c["zernike"], offs, c["z"],
                                 c["n_theta"], c["n_r"], c["nx"], c["ny"],
                                 c["dx"], c["dy"], project=True, emitters=[e])
        assert max_rel(Ie, Ir) <= TOL[prec], e
    del I
    torch.cuda.empty_cache()


def test_bessel_outputs_to_pinned_host_memory(lib):
    """Both spherical entry points write straight into pinned host memory:
    bitwise the device results."""
    c = W.bessel(n_emitters=6, n_theta=48, n_r=40, nx=20, nz_lo=2, nz_hi=5)
    args = (c["optics"], c["depth"], c["zernike"], c["z_offsets"], c["z"], 48, 40, 20, 20,
            c["dx"], c["dy"])
    n = int(c["z_offsets"][-1])
    I_dev = api.bessel(*args, project=True)
    I_pin = torch.empty((n, 20, 20), dtype=torch.float32, pin_memory=True)
    api.bessel(*args, project=True, out=I_pin)
    H_dev = api.bessel_harmonic(*args, m_max=5)
    H_pin = torch.empty((n, 20, 20), dtype=torch.float32, pin_memory=True)
    api.bessel_harmonic(*args, m_max=5, out=H_pin)
    torch.cuda.synchronize()
    assert np.array_equal(I_pin.numpy(), I_dev.cpu().numpy())
    assert np.array_equal(H_pin.numpy(), H_dev.cpu().numpy())


def test_split_modes_outside_the_envelope_are_refused(lib):
    """Split BF16, and split FP16 beyond 448 theta nodes, are refused before
    any launch; "auto" takes split FP16 inside the envelope (bitwise the
    same stack) and FP32 beyond it."""
    d = W.optics_gibson_lanni(0.0)
    depth, zern, offs, z = small_batch(seed=5, nz=(2, 3))
    geo = (200, 48, 12, 12, 0.03, 0.03)
    with pytest.raises(_lib.PsfError) as e:
        api.bessel(d, depth, zern, offs, z, *geo, project=True, precision="split_bf16")
    assert e.value.code == _lib.PSF_ERR_PRECISION
    with pytest.raises(_lib.PsfError) as e:
        api.bessel(d, depth, zern, offs, z, 600, *geo[1:], project=True,
                   precision="split_fp16")
    assert e.value.code == _lib.PSF_ERR_PRECISION
    a = api.bessel(d, depth, zern, offs, z, *geo, project=True, precision="auto")
    f = api.bessel(d, depth, zern, offs, z, *geo, project=True, precision="split_fp16")
    a6 = api.bessel(d, depth, zern, offs, z, 600, *geo[1:], project=True, precision="auto")
    f6 = api.bessel(d, depth, zern, offs, z, 600, *geo[1:], project=True, precision="fp32")
    torch.cuda.synchronize()
    assert torch.equal(a, f) and torch.equal(a6, f6)
