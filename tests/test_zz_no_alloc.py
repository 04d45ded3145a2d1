"""psf_fourier_vectorial_noalloc: the Fourier forward for callers that cannot
allocate device memory (their host application owns all device memory, or
cudaMalloc is not allowed in their loop).  It must give the same stack as
psf_fourier_vectorial with a caller workspace, on consecutive calls that reuse
the library's fixed scratch array, and must reject sizes the array cannot
hold.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, d, N, grid, zern, pm):
    o = api.make_optics(d)
    g = api.Grid(grid)
    I = torch.full((g.c.nz, g.c.nx, g.c.ny), float("nan"), device="cuda")
    F = torch.full((g.c.nz, 3, g.c.nx, g.c.ny), float("nan"),
                   dtype=torch.complex64, device="cuda")
    zh = np.ascontiguousarray(zern, dtype=np.float64)
    _lib.check(lib, lib.psf_fourier_vectorial_noalloc(
        ctypes.byref(o), N, ctypes.byref(g.c),
        zh.ctypes.data_as(ctypes.c_void_p), len(zh), api._ptr(pm), api._ptr(I),
        api._ptr(F), api._stream()))
    torch.cuda.synchronize()
    return I.cpu().numpy(), F.cpu().numpy()


def test_noalloc_matches_workspace_entry_point(lib):
    rng = np.random.default_rng(17)
    cases = []
    for N, nx, ny, nz in ((64, 64, 64, 16), (40, 37, 29, 5)):
        d = W.optics_gibson_lanni(1.0)
        zern = np.zeros(21)
        zern[3:21] = rng.normal(0, 0.1, 18)
        pm = torch.as_tensor(rng.normal(0, 0.3, (N, N)).astype(np.float32)).cuda()
        grid = dict(nx=nx, ny=ny, dx=0.02, dy=0.021, z=np.linspace(-1, 1, nz))
        cases.append((d, N, grid, zern, pm))
    # two calls in a row per case, alternating cases so the shared array
    # always holds the other problem's data when a call starts
    for rep in range(2):
        for d, N, grid, zern, pm in cases:
            I_ref, F_ref = api.fourier(d, N, grid, zernike=zern, phase_map=pm,
                                       fields=True)
            I_ref, F_ref = I_ref.cpu().numpy(), F_ref.cpu().numpy()
            I, F = _noalloc(lib, d, N, grid, zern, pm)
            assert np.all(np.isfinite(I)), rep
            # the same kernels and per-plane arithmetic (only the z-chunk
            # length differs, which no plane's result depends on): bitwise
            assert np.array_equal(I, I_ref), rep
            assert np.array_equal(F, F_ref), rep


def test_noalloc_runs_large_stacks_in_short_chunks(lib):
    """The 256^2-pupil, 512^2-pixel stack needs far more than the 24 MiB array
    in one launch; the forward shortens its z-chunks to the array and gives
    the stack of the workspace entry point."""
    c = W.fourier(nz=6)
    o = api.make_optics(c["optics"])
    g = api.Grid(c["grid"])
    need = lib.psf_fourier_workspace_size(ctypes.byref(o), c["n_pupil"], ctypes.byref(g.c), 0)
    assert need > (24 << 20)
    pm = torch.zeros((c["n_pupil"], c["n_pupil"]), device="cuda")
    I, F = _noalloc(lib, c["optics"], c["n_pupil"], c["grid"], c["zernike"], pm)
    I_ref, F_ref = api.fourier(c["optics"], c["n_pupil"], c["grid"], zernike=c["zernike"],
                               fields=True)
    I_ref, F_ref = I_ref.cpu().numpy(), F_ref.cpu().numpy()
    assert np.array_equal(I, I_ref)
    assert np.array_equal(F, F_ref)


def test_noalloc_rejects_sizes_beyond_the_array(lib):
    """A 1024^2 pupil does not fit the array even one plane at a time."""
    c = W.fourier(nz=2)
    N = 1024
    o = api.make_optics(c["optics"])
    g = api.Grid(c["grid"])
    I = torch.zeros(1, device="cuda")
    r = lib.psf_fourier_vectorial_noalloc(
        ctypes.byref(o), N, ctypes.byref(g.c), None, 0, None,
        api._ptr(I), None, api._stream())
    assert r == _lib.PSF_ERR_WORKSPACE
    msg = lib.psf_last_error().decode()
    assert "one plane at a time" in msg and str(24 << 20) in msg
