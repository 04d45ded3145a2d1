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
    """I = psf(W_0, c) for one pupil; differentiable in W_0 and c."""

    @staticmethod
    def forward(ctx, phase_map, zernike, optics, n_pupil, grid, precision):
        I = api.fourier(optics, n_pupil, grid,
                        zernike=zernike.detach().cpu().numpy(),
                        phase_map=phase_map.detach(), precision=precision)
        ctx.save_for_backward(phase_map, zernike)
        ctx.cfg = (optics, n_pupil, grid, precision)
        return I

    @staticmethod
    def backward(ctx, grad_I):
        phase_map, zernike = ctx.saved_tensors
        optics, n_pupil, grid, precision = ctx.cfg
        _, gW, gc = _backward_call(optics, n_pupil, grid, zernike[None, :],
                                   phase_map[None], grad_I=grad_I[None],
                                   precision="fp32", want_loss=False)
        gz = gc[0].to(dtype=zernike.dtype, device=zernike.device)
        return gW[0].to(phase_map.dtype), gz, None, None, None, None


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
