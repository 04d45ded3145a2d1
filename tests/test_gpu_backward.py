"""Adjoint of the Fourier strategy on the GPU against the FP64 oracle adjoint
(gradients within 1e-4 relative L2; the oracle adjoint is pinned by finite
differences on the CPU).  FP32 contractions and the tensor-core split path
(forward recomputed in split FP16 / BF16, adjoint contractions in split
BF16)."""
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


PREC = {"fp32": 0, "split_fp16": 1, "split_bf16": 2}


def gpu_backward(d, N, grid, zern, pm, target=None, grad_I=None, prec="fp32", ws_bytes=None):
    lib = _lib.load()
    o = api.make_optics(d)
    g = api.Grid(grid)
    batch = zern.shape[0]
    need = ws_bytes or lib.psf_fourier_backward_workspace_size(ctypes.byref(o), N,
                                                               ctypes.byref(g.c), PREC[prec])
    assert need > 0, lib.psf_last_error()
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
        zh.ctypes.data_as(ctypes.c_void_p), zern.shape[1], p(pm_d), PREC[prec], p(T),
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


@pytest.mark.parametrize("prec", ["split_fp16", "split_bf16"])
@pytest.mark.parametrize("N,nx,ny,nz", [(32, 16, 24, 5), (48, 72, 64, 3)])
def test_split_backward_matches_oracle(lib, N, nx, ny, nz, prec):
    """Tensor-core adjoint: several m/n tiles with a ragged tail (72 = 64 + 8)."""
    rng = np.random.default_rng(7 + N)
    d = W.optics_gibson_lanni(1.0)
    grid = dict(nx=nx, ny=ny, dx=0.03, dy=0.035, z=np.linspace(-0.5, 0.6, nz))
    batch = 2
    zern = np.zeros((batch, 21))
    zern[:, 3:15] = rng.normal(0, 0.2, (batch, 12))
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (batch, N, N)), 0.0)
    opt = oracle_optics(d)
    refs, targets = [], []
    for b in range(batch):
        T = rng.uniform(0, 2e-4, (nz, nx, ny))
        targets.append(T)
        refs.append(oa.loss_and_grad(opt, N, grid, zern[b], pm[b], T))
    loss, gW, gc = gpu_backward(d, N, grid, zern, pm, target=np.stack(targets), prec=prec)
    loss2, gW2, gc2 = gpu_backward(d, N, grid, zern, pm, target=np.stack(targets), prec=prec)
    assert np.array_equal(gW, gW2) and np.array_equal(loss, loss2)   # fixed order
    for b in range(batch):
        L, gWr, gcr, _ = refs[b]
        assert abs(loss[b] - L) <= 1e-4 * abs(L)
        assert rel_l2(gW[b], gWr) <= TOL_G
        assert rel_l2(gc[b], gcr) <= TOL_G


def test_split_backward_upstream_gradient(lib):
    rng = np.random.default_rng(15)
    N, nx, ny, nz = 32, 16, 16, 2
    d = W.optics_plain()
    grid = dict(nx=nx, ny=ny, dx=0.04, dy=0.04, z=[-0.3, 0.2])
    zern = np.zeros((1, 21))
    zern[0, 4:9] = rng.normal(0, 0.2, 5)
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (1, N, N)), 0.0)
    gI = rng.normal(0, 1.0, (1, nz, nx, ny))
    _, gW, gc = gpu_backward(d, N, grid, zern, pm, grad_I=gI, prec="split_fp16")
    opt = oracle_optics(d)
    from oracle import fourier as of
    I = of.psf_fourier(opt, N, grid, zern[0], pm[0])
    _, gWr, gcr, _ = oa.loss_and_grad(opt, N, grid, zern[0], pm[0], I - gI[0] / 2)
    assert rel_l2(gW[0], gWr) <= TOL_G
    assert rel_l2(gc[0], gcr) <= TOL_G


def test_split_backward_adjoint_config_sampled(lib):
    """The phase-retrieval workload (batch 64, 256^2 pupil, 128^2 px, 32
    planes) in one split-FP16 call; two batch elements recomputed by the
    oracle.  The target is the oracle PSF of the true phases with 1 % noise."""
    c = W.adjoint()
    N, grid, B = c["n_pupil"], c["grid"], c["batch"]
    d = c["optics"]
    opt = oracle_optics(d)
    from oracle import fourier as of
    rng = np.random.default_rng(c["noise_seed"])
    sample = (0, 37)
    nz, nx, ny = len(grid["z"]), grid["nx"], grid["ny"]
    T = np.zeros((B, nz, nx, ny), dtype=np.float32)
    for b in sample:
        I = of.psf_fourier(opt, N, grid, c["c_true"][b], c["w_true"][b])
        T[b] = I + rng.normal(0, 0.01 * I.max(), I.shape)
    zern = np.zeros((B, 21))
    pm = np.zeros((B, N, N))
    loss, gW, gc = gpu_backward(d, N, grid, zern, pm, target=T, prec="split_fp16")
    for b in sample:
        L, gWr, gcr, _ = oa.loss_and_grad(opt, N, grid, zern[b], pm[b], T[b].astype(np.float64))
        assert abs(loss[b] - L) <= 1e-4 * abs(L)
        assert rel_l2(gW[b], gWr) <= TOL_G
        assert rel_l2(gc[b], gcr) <= TOL_G


@pytest.mark.parametrize("N,nx,ny,nz,batch", [(64, 72, 56, 5, 3), (48, 136, 40, 4, 2)])
@pytest.mark.parametrize("use_target", [True, False])
def test_backward_cta_pair_matches_single_cta(lib, N, nx, ny, nz, batch, use_target,
                                              monkeypatch):
    """The adjoint's four contractions on the CTA-pair kernel (default) and on
    the single-CTA kernel give bitwise equal loss and gradients (odd numbers
    of 64-row output tiles included: the last pair's peer tile is empty)."""
    rng = np.random.default_rng(5 + N)
    d = W.optics_gibson_lanni(1.0)
    grid = dict(nx=nx, ny=ny, dx=0.03, dy=0.035, z=np.linspace(-0.5, 0.6, nz))
    zern = np.zeros((batch, 21))
    zern[:, 3:12] = rng.normal(0, 0.15, (batch, 9))
    pm = rng.normal(0, 0.2, (batch, N, N))
    T = rng.uniform(0, 2e-4, (batch, nz, nx, ny))
    G = rng.normal(0, 1.0, (batch, nz, nx, ny))
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PSF_TC_PAIR", mode)
        out[mode] = gpu_backward(d, N, grid, zern, pm,
                                 target=T if use_target else None,
                                 grad_I=None if use_target else G, prec="split_fp16")
    for a, b in zip(out["1"], out["0"]):
        assert np.array_equal(a, b)
    if use_target:   # and the pair result is the adjoint the oracle computes
        L, gWr, gcr, _ = oa.loss_and_grad(oracle_optics(d), N, grid, zern[0], pm[0], T[0])
        assert rel_l2(out["1"][1][0], gWr) <= 1e-4
        assert rel_l2(out["1"][2][0], gcr) <= 1e-4


@pytest.mark.parametrize("use_target", [True, False])
def test_backward_chunking_is_invisible(lib, use_target):
    """Six pupils of 32 planes: with the default workspace the adjoint runs
    two groups (128-plane chunks: 4 + 2 pupils), with the batch-sized one a
    single 192-plane group.  Each plane's arithmetic and every summation
    order are the same, so loss and gradients are bitwise equal."""
    rng = np.random.default_rng(21)
    d = W.optics_gibson_lanni(1.0)
    N, nx, ny, nz, B = 32, 16, 24, 32, 6
    grid = dict(nx=nx, ny=ny, dx=0.03, dy=0.035, z=np.linspace(-0.8, 0.8, nz))
    zern = np.zeros((B, 21))
    zern[:, 3:15] = rng.normal(0, 0.15, (B, 12))
    pm = rng.normal(0, 0.2, (B, N, N))
    T = rng.uniform(0, 2e-4, (B, nz, nx, ny))
    G = rng.normal(0, 1.0, (B, nz, nx, ny))
    lib_ = _lib.load()
    o = api.make_optics(d)
    g = api.Grid(grid)
    small = lib_.psf_fourier_backward_workspace_size(ctypes.byref(o), N, ctypes.byref(g.c), 1)
    big = lib_.psf_fourier_backward_workspace_size_batch(ctypes.byref(o), N, ctypes.byref(g.c),
                                                         1, B)
    assert big > small
    out = []
    for ws_bytes in (small, big):
        out.append(gpu_backward(d, N, grid, zern, pm, target=T if use_target else None,
                                grad_I=None if use_target else G, prec="split_fp16",
                                ws_bytes=ws_bytes))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "split_fp16", "split_bf16"])
def test_fourier_autograd_function(lib, prec):
    """torch.autograd through fourier_psf for a batch of two pupils: the
    gradient of sum (I - T)^2 with respect to the phase maps and the Zernike
    rows against the FP64 oracle adjoint (pinned by finite differences on the
    CPU), in the forward's precision; the forward stack against the oracle
    forward."""
    from paper_2502_03170_gb300 import autograd as ag

    from .gpu_helpers import max_rel
    rng = np.random.default_rng(3)
    N, nx, ny, nz, B = 32, 16, 24, 3, 2
    d = W.optics_gibson_lanni(1.0)
    grid = dict(nx=nx, ny=ny, dx=0.04, dy=0.035, z=np.linspace(-0.5, 0.4, nz))
    zern = np.zeros((B, 21))
    zern[:, 3:15] = rng.normal(0, 0.2, (B, 12))
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (B, N, N)), 0.0)
    T = rng.uniform(0, 2e-4, (B, nz, nx, ny))
    pm_t = torch.tensor(pm, dtype=torch.float32, device="cuda", requires_grad=True)
    zc_t = torch.tensor(zern, dtype=torch.float64, device="cuda", requires_grad=True)
    I = ag.fourier_psf(pm_t, zc_t, d, N, grid, precision=prec)
    L = ((I - torch.tensor(T, dtype=torch.float32, device="cuda")) ** 2).sum()
    gW, gc = torch.autograd.grad(L, (pm_t, zc_t))
    opt = oracle_optics(d)
    tol_f = 1e-5
    for b in range(B):
        _, gWr, gcr, Ir = oa.loss_and_grad(opt, N, grid, zern[b], pm[b], T[b])
        assert max_rel(I[b].detach().cpu().numpy(), Ir) <= tol_f
        assert rel_l2(gW[b].cpu().numpy(), gWr) <= TOL_G
        assert rel_l2(gc[b].cpu().numpy(), gcr) <= TOL_G


@pytest.mark.parametrize("prec", ["fp32", "split_fp16"])
def test_fourier_autograd_without_zernike_terms(lib, prec):
    """An unbatched pupil with an empty Zernike vector: the phase-map
    gradient against the oracle adjoint, a zero-length Zernike gradient."""
    from paper_2502_03170_gb300 import autograd as ag
    rng = np.random.default_rng(9)
    N, nx, ny, nz = 32, 16, 16, 2
    d = W.optics_plain()
    grid = dict(nx=nx, ny=ny, dx=0.04, dy=0.04, z=[-0.3, 0.25])
    pm = np.where(pupil_mask(N), rng.normal(0, 0.3, (N, N)), 0.0)
    T = rng.uniform(0, 2e-4, (nz, nx, ny))
    pm_t = torch.tensor(pm, dtype=torch.float32, device="cuda", requires_grad=True)
    zc_t = torch.zeros(0, dtype=torch.float64, device="cuda", requires_grad=True)
    I = ag.fourier_psf(pm_t, zc_t, d, N, grid, precision=prec)
    L = ((I - torch.tensor(T, dtype=torch.float32, device="cuda")) ** 2).sum()
    gW, gc = torch.autograd.grad(L, (pm_t, zc_t))
    assert gc.shape == (0,)
    _, gWr, _, _ = oa.loss_and_grad(oracle_optics(d), N, grid, None, pm, T, n_zern=0)
    assert rel_l2(gW.cpu().numpy(), gWr) <= TOL_G
