"""Differentiable PSFs: torch.autograd.Functions over the libpsf forwards
(Eq. 8, Eq. 10-11) and their hand-written adjoints.

Fourier strategy: gradients flow to the pupil phase map W_0 and to the
Zernike coefficients of Eq. 15; the backward recomputes each z-plane instead
of storing pupil fields.  Bessel strategy: gradients flow to a free radial
phase W_0(theta) at the Gauss-Legendre nodes, the m = 0 Zernike coefficients
and the emitter depths (Eq. 13-14); the backward recomputes the radial
profiles.
"""
import ctypes

import numpy as np
import torch

from . import _lib, api


def _backward_call(optics, n_pupil, grid, zernike, phase_map, target=None,
                   grad_I=None, precision="fp32", want_loss=True,
                   workspace=None, stream=None):
    """Runs psf_fourier_vectorial_backward; all tensors on the current device.

    zernike   [B, n_zern] (host copy taken), phase_map [B, N, N] or None,
    target / grad_I [B, nz, nx, ny].  Returns (loss [B] or None, gW, gc)."""
    lib = _lib.load()
    o = optics if isinstance(optics, _lib.PsfOptics) else api.make_optics(optics)
    g = grid if isinstance(grid, api.Grid) else api.Grid(grid)
    prec = api.PRECISIONS[precision] if isinstance(precision, str) else precision
    zh = np.ascontiguousarray(np.asarray(
        zernike.detach().cpu() if torch.is_tensor(zernike) else zernike,
        dtype=np.float64))
    if zh.ndim == 1:
        zh = zh[None, :]
    B, nzern = zh.shape
    dev = torch.device("cuda", torch.cuda.current_device())
    # a workspace for the whole batch in one pass (the call falls back to
    # shorter chunks when a smaller workspace is handed in)
    need = lib.psf_fourier_backward_workspace_size_batch(ctypes.byref(o), n_pupil,
                                                         ctypes.byref(g.c), prec, B)
    if need == 0:
        raise _lib.PsfError(_lib.PSF_ERR_ARG, lib.psf_last_error().decode())
    ws = (workspace or api.Workspace(dev)).get(need)

    def f32(t):
        if t is None:
            return None
        t = t if torch.is_tensor(t) else torch.as_tensor(np.asarray(t))
        return t.to(device=dev, dtype=torch.float32).contiguous()

    pm, T, G = f32(phase_map), f32(target), f32(grad_I)
    loss = torch.empty(B, device=dev) if (want_loss and T is not None) else None
    gW = torch.empty((B, n_pupil, n_pupil), device=dev)
    gc = torch.empty((B, nzern), device=dev) if nzern > 0 else None
    p = api._ptr
    _lib.check(lib, lib.psf_fourier_vectorial_backward(
        ctypes.byref(o), n_pupil, ctypes.byref(g.c), B,
        zh.ctypes.data_as(ctypes.c_void_p) if nzern else None, nzern, p(pm),
        prec, p(T), p(G), p(loss), p(gW), p(gc), p(ws), ws.numel(),
        api._stream(stream)))
    return loss, gW, gc


def fourier_loss_grad(optics, n_pupil, grid, zernike, phase_map, target,
                      precision="fp32"):
    """L2 loss sum (I - T)^2 per batch element and its gradients (numpy)."""
    loss, gW, gc = _backward_call(optics, n_pupil, grid, zernike, phase_map,
                                  target=target, precision=precision)
    torch.cuda.synchronize()
    return (loss.cpu().numpy(), gW.cpu().numpy(),
            None if gc is None else gc.cpu().numpy())


class FourierPSF(torch.autograd.Function):
    """I = psf(W_0, c) for a batch of pupils, differentiable in W_0 and c.

    phase_map [B, N, N] (or [N, N]) in radians on the device, zernike
    [B, n_zern] (or [n_zern]; n_zern may be 0).  Returns I [B, nz, nx, ny]
    (or [nz, nx, ny] for unbatched inputs).  The backward runs the adjoint of
    Eq. 8 in the forward's precision: the split modes recompute each plane's
    fields with the tensor-core contractions of the forward and contract the
    adjoint on the tensor cores as well; fp32 runs both in FP32."""

    @staticmethod
    def forward(ctx, phase_map, zernike, optics, n_pupil, grid, precision):
        batched = phase_map.dim() == 3
        pm = phase_map.detach() if batched else phase_map.detach()[None]
        zc = zernike.detach() if zernike.dim() == 2 else zernike.detach()[None]
        if zc.shape[0] != pm.shape[0]:
            raise ValueError("zernike and phase_map batch sizes differ")
        B = pm.shape[0]
        g = grid if isinstance(grid, api.Grid) else api.Grid(grid)
        zh = np.ascontiguousarray(zc.cpu().numpy(), dtype=np.float64)
        I = torch.empty((B, g.c.nz, g.c.nx, g.c.ny), dtype=torch.float32, device=pm.device)
        ws = api.Workspace(pm.device)
        for b in range(B):
            api.fourier(optics, n_pupil, g, zernike=zh[b] if zh.shape[1] else None,
                        phase_map=pm[b], precision=precision, out=I[b], workspace=ws)
        ctx.save_for_backward(pm, zc)
        ctx.cfg = (optics, n_pupil, g, precision, batched, zernike.dim())
        return I if batched else I[0]

    @staticmethod
    def backward(ctx, grad_I):
        pm, zc = ctx.saved_tensors
        optics, n_pupil, g, precision, batched, zdim = ctx.cfg
        G = (grad_I if batched else grad_I[None]).to(torch.float32).contiguous()
        _, gW, gc = _backward_call(optics, n_pupil, g, zc, pm, grad_I=G,
                                   precision=precision, want_loss=False)
        gz = torch.zeros_like(zc) if gc is None else gc.to(dtype=zc.dtype, device=zc.device)
        gp = gW.to(pm.dtype)
        if not batched:
            gp = gp[0]
        if zdim == 1:
            gz = gz[0]
        return gp, gz, None, None, None, None


def fourier_psf(phase_map, zernike, optics, n_pupil, grid, precision="fp32"):
    return FourierPSF.apply(phase_map, zernike, optics, n_pupil, grid, precision)


class BesselPSF(torch.autograd.Function):
    """I = psf(depth, c, W_0(theta)) for batched emitters (packed slices);
    differentiable in all three."""

    @staticmethod
    def forward(ctx, depth, zernike, phase_theta, optics, z_offsets, z, n_theta,
                n_r, nx, ny, dx, dy):
        I = api.bessel(optics, depth.detach(), zernike.detach(), z_offsets, z,
                       n_theta, n_r, nx, ny, dx, dy, project=True,
                       phase_theta=phase_theta.detach())
        ctx.save_for_backward(depth, zernike, phase_theta)
        ctx.cfg = (optics, z_offsets, z, n_theta, n_r, nx, ny, dx, dy)
        return I

    @staticmethod
    def backward(ctx, grad_I):
        depth, zernike, phase_theta = ctx.saved_tensors
        optics, z_offsets, z, n_theta, n_r, nx, ny, dx, dy = ctx.cfg
        g = api.bessel_backward(optics, depth, zernike, z_offsets, z, n_theta, n_r, nx,
                                ny, dx, dy, grad_intensity=grad_I.contiguous(),
                                project=True, phase_theta=phase_theta)
        return (g["grad_depth"].to(depth.dtype), g["grad_zernike"].to(zernike.dtype),
                g["grad_phase_theta"].to(phase_theta.dtype),
                None, None, None, None, None, None, None, None, None)


def bessel_psf(depth, zernike, phase_theta, optics, z_offsets, z, n_theta, n_r, nx, ny,
               dx, dy):
    return BesselPSF.apply(depth, zernike, phase_theta, optics, z_offsets, z, n_theta,
                           n_r, nx, ny, dx, dy)
