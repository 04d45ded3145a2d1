"""Chirp-Z (Bluestein) evaluation of the Fourier strategy's zoom DFTs on the
GPU, through the C ABI, against the FP64 oracle.

The chirp-Z form computes the same discrete sum as the dense matrix-DFT
(Eq. 8 by the midpoint rule on the pupil grid), so the oracle is the plain
separable FP64 sum; the bound is the forward one, max-rel 1e-5 for the
intensity and the complex fields.  The cases span every FFT length the
kernels are built for (256 ... 4096), ragged pupil sizes and line counts,
different lengths per direction, and the models and aberrations of the
other Fourier tests."""
import numpy as np
import pytest
import torch

from oracle import fourier as of
from oracle.optics import pupil_mask
from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import max_rel, oracle_optics

pytestmark = pytest.mark.gpu
TOL = 1e-5


def fft_len(N, n):
    L = 256
    while L < N + n - 1:
        L *= 2
    return L


def aberrated(N, seed, **kw):
    g = np.random.default_rng(seed)
    d = W.optics_gibson_lanni(1.5)
    d["pol"] = (0.8, 0.36 + 0.48j)
    d.update(kw)
    zern = np.zeros(21)
    zern[3:21] = g.normal(0, 0.15, 18)
    pm = np.where(pupil_mask(N), g.normal(0, 0.2, (N, N)), 0.0)
    return d, zern, pm


# (N, nx, ny, nz): FFT lengths per direction in the comments
CASES = [
    (64, 64, 64, 3),      # 256 / 256
    (63, 37, 29, 4),      # 256 / 256, odd pupil, ragged lines
    (128, 300, 77, 2),    # 512 / 256
    (256, 512, 200, 2),   # 1024 / 512
    (100, 1000, 20, 1),   # 2048 / 256
    (40, 2100, 9, 1),     # 4096 / 256
    (33, 5, 1000, 2),     # 256 / 2048
]


@pytest.mark.parametrize("N,nx,ny,nz", CASES)
def test_chirpz_matches_oracle(lib, N, nx, ny, nz):
    d, zern, pm = aberrated(N, N * 7 + nx)
    grid = dict(nx=nx, ny=ny, dx=0.013, dy=0.021, z=np.linspace(-0.9, 1.3, nz))
    assert fft_len(N, nx) <= 4096 and fft_len(N, ny) <= 4096
    I, F = api.fourier(d, N, grid, zernike=zern, phase_map=pm, precision="chirpz_fp32",
                       fields=True)
    torch.cuda.synchronize()
    E = of.field_separable(oracle_optics(d), N, grid, zern, pm)
    assert max_rel(F.cpu().numpy(), E) <= TOL
    assert max_rel(I.cpu().numpy(), of.intensity(E)) <= TOL


@pytest.mark.parametrize("kw", [dict(scalar=True), dict(fresnel=True)])
def test_chirpz_models(lib, kw):
    N = 96
    d, zern, pm = aberrated(N, 5, **kw)
    grid = dict(nx=70, ny=51, dx=0.02, dy=0.02, z=[-0.5, 0.0, 0.8])
    I = api.fourier(d, N, grid, zernike=zern, phase_map=pm, precision="chirpz_fp32")
    torch.cuda.synchronize()
    Iref = of.psf_fourier(oracle_optics(d), N, grid, zern, pm)
    assert max_rel(I.cpu().numpy(), Iref) <= TOL


def test_chirpz_full_workload_sampled_planes(lib):
    """The 256^2-pupil, 512^2-pixel, 128-plane stack in the launch
    configuration the benchmark times; the oracle checks four planes
    (first, last, two inside the chunking)."""
    c = W.fourier()
    I = api.fourier(c["optics"], c["n_pupil"], c["grid"], zernike=c["zernike"],
                    precision="chirpz_fp32")
    torch.cuda.synchronize()
    I = I.cpu().numpy()
    sel = [0, 37, 64, 127]
    g = dict(c["grid"], z=c["grid"]["z"][sel])
    Iref = of.psf_fourier(oracle_optics(c["optics"]), c["n_pupil"], g, c["zernike"])
    assert max_rel(I[sel], Iref) <= TOL
    assert np.all(np.isfinite(I))


def test_chirpz_large_pupil(lib):
    """N_p = 1024 (FFT length 2048 along both directions) on two planes."""
    c = W.fourier()
    N = 1024
    g = dict(c["grid"], z=np.array([-1.1, 0.6]))
    I = api.fourier(c["optics"], N, g, zernike=c["zernike"], precision="chirpz_fp32")
    torch.cuda.synchronize()
    Iref = of.psf_fourier(oracle_optics(c["optics"]), N, g, c["zernike"])
    assert max_rel(I.cpu().numpy(), Iref) <= TOL


def test_chirpz_agrees_with_the_dense_paths(lib):
    """Same sum three ways on the GPU: chirp-Z, FP32 matrix-DFT, split FP16."""
    c = W.fourier()
    g = dict(c["grid"], z=c["grid"]["z"][::16])
    out = {p: api.fourier(c["optics"], c["n_pupil"], g, zernike=c["zernike"],
                          precision=p).cpu().numpy()
           for p in ("chirpz_fp32", "fp32", "split_fp16")}
    assert max_rel(out["chirpz_fp32"], out["fp32"]) <= 2 * TOL
    assert max_rel(out["chirpz_fp32"], out["split_fp16"]) <= 2 * TOL


def test_chirpz_limits(lib):
    d = W.optics_plain()
    with pytest.raises(_lib.PsfError) as e:
        api.fourier(d, 2048, dict(nx=2050, ny=8, dx=0.02, dy=0.02, z=[0.0]),
                    precision="chirpz_fp32")
    assert e.value.code == _lib.PSF_ERR_PRECISION
    # smallest sizes: one pixel, two pupil nodes
    I = api.fourier(d, 2, dict(nx=1, ny=1, dx=0.02, dy=0.02, z=[0.0]),
                    precision="chirpz_fp32").cpu().numpy()
    Iref = of.psf_fourier(oracle_optics(d), 2, dict(nx=1, ny=1, dx=0.02, dy=0.02, z=[0.0]))
    assert max_rel(I, Iref) <= TOL
