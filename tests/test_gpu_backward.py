"""Adjoint of the Fourier strategy on the GPU against the FP64 oracle adjoint
(gradients within 1e-4 relative L2) and finite differences."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import adjoint as oa
from oracle.optics import pupil_mask
from paper_2502_03170_gb300 import _lib, api
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import oracle_optics, rel_l2

pytestmark = pytest.mark.gpu
TOL_G = 1e-4


def gpu_backward(d, N, grid, zern, pm, target=None, grad_I=None):
    lib = _lib.load()
    o = api.make_optics(d)
    g = api.Grid(grid)
    batch = zern.shape[0]
    need = lib.psf_fourier_backward_workspace_size(ctypes.byref(o), N,
                                                   ctypes.byref(g.c), 0)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    pm_d = dev(pm)
    T = dev(target) if target is not None else None
    G = dev(grad_I) if grad_I is not None else None
    loss = torch.zeros(batch, device="cuda")
    gW = torch.zeros((batch, N, N), device="cuda")
    gc = torch.zeros((batch, zern.shape[1]), device="cuda")
    zh = np.ascontiguousarray(zern, dtype=np.float64)
    p = lambda t: ctypes.c_void_p(0 if t is None else t.data_ptr())
    _lib.check(lib, lib.psf_fourier_vectorial_backward(
        ctypes.byref(o), N, ctypes.byref(g.c), batch,
        zh.ctypes.data_as(ctypes.c_void_p), zern.shape[1], p(pm_d), 0, p(T),
        p(G), p(loss) if T is not None else None, p(gW), p(gc), p(ws),
        ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    return loss.cpu().numpy(), gW.cpu().numpy(), gc.cpu().numpy()


@pytest.mark.parametrize("N,nx,ny,nz", [(24, 13, 11, 3), (32, 16, 16, 4)])
def test_backward_matches_oracle(lib, N, nx, ny, nz):
    rng = np.random.default_rng(11 + N)
    d = W.optics_gibson_lanni(1.0)
    grid = dict(nx=nx, ny=ny, dx=0.04, dy=0.05, z=np.linspace(-0.6, 0.5, nz))
    batch = 2
    zern = np.zeros((batch, 21))
    zern[:, 3:15] = rng.normal(0, 0.2, (batch, 12))
    mask = pupil_mask(N)
    pm = np.where(mask, rng.normal(0, 0.3, (batch, N, N)), 0.0)
    opt = oracle_optics(d)
    refs, targets = [], []
    for b in range(batch):
        T = rng.uniform(0, 2e-4, (nz, nx, ny))
        targets.append(T)
        refs.append(oa.loss_and_grad(opt, N, grid, zern[b], pm[b], T))
    loss, gW, gc = gpu_backward(d, N, grid, zern, pm, target=np.stack(targets))
    for b in range(batch):
        L, gWr, gcr, _ = refs[b]
        assert abs(loss[b] - L) <= 1e-5 * abs(L)
        assert rel_l2(gW[b], gWr) <= TOL_G
        assert rel_l2(gc[b], gcr) <= TOL_G


def test_backward_upstream_gradient(lib):
    """dL/dI supplied by the caller (autograd path)."""
    rng = np.random.default_rng(5)
    N, nx, ny, nz = 20, 10, 12, 2
    d = W.optics_plain()
    grid = dict(nx=nx, ny=ny, dx=0.04, dy=0.04, z=[-0.3, 0.2])
    zern = np.zeros((1, 21))
    zern[0, 4:9] = rng.normal(0, 0.2, 5)
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (1, N, N)), 0.0)
    gI = rng.normal(0, 1.0, (1, nz, nx, ny))
    _, gW, gc = gpu_backward(d, N, grid, zern, pm, grad_I=gI)
    opt = oracle_optics(d)
    from oracle import fourier as of
    I = of.psf_fourier(opt, N, grid, zern[0], pm[0])
    # dL/dI = 2 (I - T)  <=>  T = I - gI / 2
    _, gWr, gcr, _ = oa.loss_and_grad(opt, N, grid, zern[0], pm[0], I - gI[0] / 2)
    assert rel_l2(gW[0], gWr) <= TOL_G
    assert rel_l2(gc[0], gcr) <= TOL_G
