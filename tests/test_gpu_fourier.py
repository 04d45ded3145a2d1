"""Fourier strategy on the GPU (through the C ABI) against the FP64 oracle.

Tolerance: max |I - I_ref| / max |I_ref| <= 1e-5 per stack for intensity and
the same for the complex fields (the forward target of the spec)."""
import math

import numpy as np
import pytest
import torch

from oracle import fourier as of
from paper_2502_03170_gb300 import api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import max_rel, oracle_optics

pytestmark = pytest.mark.gpu
TOL = 1e-5


def run_case(lib, d, N, grid, zern=None, pm=None, precision="fp32", fields=True):
    res = api.fourier(d, N, grid, zernike=zern, phase_map=pm,
                      precision=precision, fields=fields)
    torch.cuda.synchronize()
    if fields:
        I, F = res
        return I.cpu().numpy(), F.cpu().numpy()
    return res.cpu().numpy(), None


def test_plain_stack_full(lib):
    c = W.plain()
    I, F = run_case(lib, c["optics"], c["n_pupil"], c["grid"])
    opt = oracle_optics(c["optics"])
    E = of.field_separable(opt, c["n_pupil"], c["grid"])
    Ir = of.intensity(E)
    assert max_rel(I, Ir) <= TOL
    assert max_rel(F, E) <= TOL


@pytest.mark.parametrize("N,nx,ny,nz", [(40, 37, 29, 5), (33, 16, 65, 3),
                                        (2, 1, 1, 1), (65, 70, 3, 2)])
def test_ragged_aberrated(lib, N, nx, ny, nz):
    g = np.random.default_rng(N * 1000 + nx)
    d = W.optics_gibson_lanni(1.5)
    d["pol"] = (0.8, 0.36 + 0.48j)
    d["s_env"] = 0.9
    zern = np.zeros(21)
    zern[1:21] = g.normal(0, 0.15, 20)
    pm = g.normal(0, 0.4, (N, N))
    grid = dict(nx=nx, ny=ny, dx=0.017, dy=0.023,
                z=np.sort(g.uniform(-1.3, 0.9, nz)))
    I, F = run_case(lib, d, N, grid, zern, pm)
    opt = oracle_optics(d)
    E = of.field_separable(opt, N, grid, zernike=zern, phase_map=pm)
    assert max_rel(I, of.intensity(E)) <= TOL
    assert max_rel(F, E) <= TOL


def test_fourier_config_full_size_sampled(lib):
    """The benchmark workload (256^2 pupil, 512^2 px, 128 planes) in one call;
    three planes recomputed by the oracle."""
    c = W.fourier()
    I, _ = run_case(lib, c["optics"], c["n_pupil"], c["grid"], c["zernike"],
                    fields=False)
    assert np.all(np.isfinite(I))
    opt = oracle_optics(c["optics"])
    zs = np.asarray(c["grid"]["z"])
    for iz in (0, 61, 127):
        g1 = dict(c["grid"], z=[zs[iz]])
        Ir = of.psf_fourier(opt, c["n_pupil"], g1, zernike=c["zernike"])[0]
        assert max_rel(I[iz], Ir) <= TOL, iz


def test_rejects_bad_arguments(lib):
    c = W.plain()
    d = dict(c["optics"], NA=1.6)
    with pytest.raises(Exception):
        api.fourier(d, 64, c["grid"])
