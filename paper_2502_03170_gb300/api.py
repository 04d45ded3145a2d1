"""Python API over libpsf: torch tensors in, torch tensors out.

PyTorch supplies device memory and the current CUDA stream only; every step
of the PSF computation runs in libpsf's kernels (no fallback path exists).
"""
import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import PsfGrid, PsfOptics, check

PRECISIONS = {"fp32": _lib.PSF_PREC_FP32, "split_fp16": _lib.PSF_PREC_SPLIT_FP16,
              "split_bf16": _lib.PSF_PREC_SPLIT_BF16,
              "chirpz_fp32": _lib.PSF_PREC_FP32_CHIRPZ, "auto": _lib.PSF_PREC_AUTO,
              "split_tf32": _lib.PSF_PREC_SPLIT_TF32, "tf32": _lib.PSF_PREC_TF32}


def make_optics(d, flags=0):
    """psf_optics from a parameter dict (keys as in ``workloads``; optional
    booleans ``scalar`` and ``fresnel`` select the model)."""
    o = PsfOptics()
    o.NA = d["NA"]
    o.lambda_ = d["lam"]
    o.n_i = d["n_i"]
    o.n_s = d.get("n_s", d["n_i"])
    o.n_g = d.get("n_g", 1.5)
    o.n_i_design = d.get("n_i_design", o.n_i)
    o.n_g_design = d.get("n_g_design", o.n_g)
    o.t_g = d.get("t_g", 170.0)
    o.t_g_design = d.get("t_g_design", o.t_g)
    o.t_i_design = d.get("t_i_design", 150.0)
    o.depth = d.get("depth", 0.0)
    px, py = d.get("pol", (1.0, 0.0))
    px, py = complex(px), complex(py)
    o.pol[0], o.pol[1], o.pol[2], o.pol[3] = px.real, px.imag, py.real, py.imag
    o.apodize = 1 if d.get("apodize", True) else 0
    o.s_env = d.get("s_env", 0.0)
    if d.get("scalar"):
        flags |= _lib.PSF_SCALAR
    if d.get("fresnel"):
        flags |= _lib.PSF_FRESNEL
    if d.get("outside_envelope"):
        flags |= _lib.PSF_OUTSIDE_ENVELOPE
    o.flags = flags
    return o


class Grid:
    """psf_grid plus the host z array it points to (kept alive here)."""

    def __init__(self, g):
        self.z = np.ascontiguousarray(np.asarray(g["z"], dtype=np.float64))
        self.c = PsfGrid()
        self.c.nx, self.c.ny = int(g["nx"]), int(g["ny"])
        self.c.dx, self.c.dy = float(g["dx"]), float(g["dy"])
        self.c.nz = len(self.z)
        self.c.z = self.z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _raise_code(lib, code):
    """Raises the error of a call that was refused before any launch."""
    raise _lib.PsfError(code if code else _lib.PSF_ERR_ARG, lib.psf_last_error().decode())


def _zern_host(zernike):
    if zernike is None:
        return None, 0
    z = np.ascontiguousarray(np.asarray(zernike, dtype=np.float64))
    return z, z.shape[-1]


class Workspace:
    """Device workspace (torch-allocated bytes) reused across calls."""

    def __init__(self, device=None):
        self.buf = None
        self.device = device or torch.device("cuda", torch.cuda.current_device())

    def get(self, nbytes):
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                                   device=self.device)
        return self.buf

    def status(self, stream=None):
        lib = _lib.load()
        return lib.psf_workspace_status(_ptr(self.buf), _stream(stream))


def fourier(optics, n_pupil, grid, zernike=None, phase_map=None,
            precision="fp32", fields=False, out=None, workspace=None,
            stream=None):
    """Vectorial PSF z-stack by the Fourier strategy (Eq. 8).

    Returns intensity [nz, nx, ny] (float32, cuda) or (intensity, fields) with
    fields complex64 [nz, 3, nx, ny].
    """
    lib = _lib.load()
    o = optics if isinstance(optics, PsfOptics) else make_optics(optics)
    g = grid if isinstance(grid, Grid) else Grid(grid)
    prec = PRECISIONS[precision] if isinstance(precision, str) else precision
    zh, nzern = _zern_host(zernike)
    ws = workspace or Workspace()
    need = lib.psf_fourier_workspace_size(ctypes.byref(o), n_pupil,
                                          ctypes.byref(g.c), prec)
    if need == 0:
        # validation failed: the call without a workspace returns its code
        # (arguments are checked before anything is launched)
        code = lib.psf_fourier_vectorial(
            ctypes.byref(o), n_pupil, ctypes.byref(g.c), None, 0, None, prec,
            ctypes.c_void_p(16), None, None, 0, None)
        raise _lib.PsfError(code if code else _lib.PSF_ERR_ARG,
                            lib.psf_last_error().decode())
    buf = ws.get(need)
    dev = buf.device
    I = out if out is not None else torch.empty(
        (g.c.nz, g.c.nx, g.c.ny), dtype=torch.float32, device=dev)
    F = torch.empty((g.c.nz, 3, g.c.nx, g.c.ny), dtype=torch.complex64,
                    device=dev) if fields else None
    pm = None
    if phase_map is not None:
        pm = phase_map if torch.is_tensor(phase_map) else torch.as_tensor(
            np.asarray(phase_map, dtype=np.float32))
        pm = pm.to(device=dev, dtype=torch.float32).contiguous()
    check(lib, lib.psf_fourier_vectorial(
        ctypes.byref(o), n_pupil, ctypes.byref(g.c),
        None if zh is None else zh.ctypes.data_as(ctypes.c_void_p), nzern,
        _ptr(pm), prec, _ptr(I), _ptr(F), _ptr(buf), buf.numel(),
        _stream(stream)))
    return (I, F) if fields else I


def harmonic_order(zernike, tol=1e-7):
    """Azimuthal truncation order M for the harmonic Bessel path: the largest
    over the emitters of the tail bound (host computation in the library).
    zernike: [n_em, n_zern] (host array or tensor)."""
    lib = _lib.load()
    zh = np.ascontiguousarray(
        (zernike.detach().cpu().numpy() if torch.is_tensor(zernike) else np.asarray(zernike)),
        dtype=np.float64)
    if zh.ndim == 1:
        zh = zh[None, :]
    m = lib.psf_bessel_harmonic_order(zh.ctypes.data_as(ctypes.c_void_p), zh.shape[0],
                                      zh.shape[1], float(tol))
    if m < 0:
        raise _lib.PsfError(m, lib.psf_last_error().decode())
    return m


def bessel_harmonic(optics, depth, zernike, z_offsets, z, n_theta, n_r, nx, ny, dx, dy,
                    m_max=None, tol=1e-7, tail_tol=None, precision="fp32", workspace=None,
                    stream=None, out=None):
    """Batched vectorial PSFs by the spherical strategy for pupils without
    axial symmetry (azimuthal harmonics |m| <= m_max of the pupil; m != 0
    Zernike terms enter exactly).  m_max defaults to harmonic_order(zernike,
    tol); each emitter then keeps the harmonics up to its adaptive order for
    tail_tol (default tol; 0 keeps m_max for all).  precision "fp32" or
    "split_fp16" (the radial contraction on the tensor cores).  Same array
    conventions as bessel(); returns [n_slices, nx, ny]."""
    lib = _lib.load()
    if m_max is None:
        m_max = 0 if zernike is None else harmonic_order(zernike, tol)
    if tail_tol is None:
        tail_tol = tol
    a = _BesselArgs(optics, depth, zernike, z_offsets, z, False, None)
    o, dev = a.o, a.dev
    ws = workspace or Workspace(dev)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    need = lib.psf_bessel_harmonic_workspace_size(ctypes.byref(o), a.n_em, a.n_slices,
                                                  n_theta, n_r, nx, ny, int(m_max), prec)

    def call(I, buf, nbytes):
        return lib.psf_bessel_vectorial_harmonic(
            ctypes.byref(o), a.n_em, _ptr(a.depth), _ptr(a.zern), a.n_zern, _ptr(a.offs),
            _ptr(a.z), a.n_slices, n_theta, n_r, nx, ny, float(dx), float(dy), int(m_max),
            float(tail_tol), prec, _ptr(I), _ptr(buf), nbytes, _stream(stream))
    if need == 0:
        _raise_code(lib, call(None, None, 0))
    buf = ws.get(need)
    I = out if out is not None else torch.empty((a.n_slices, nx, ny), dtype=torch.float32,
                                                device=dev)
    check(lib, call(I, buf, buf.numel()))
    return I


class _BesselArgs:
    """Device copies of the per-emitter inputs of a Bessel call."""

    def __init__(self, optics, depth, zernike, z_offsets, z, project, phase_theta):
        flags = _lib.PSF_PROJECT_AXISYMMETRIC if project else 0
        o = optics if isinstance(optics, PsfOptics) else make_optics(optics, flags)
        if isinstance(optics, PsfOptics):
            o.flags = (o.flags & ~_lib.PSF_PROJECT_AXISYMMETRIC) | flags
        self.o = o
        self.dev = torch.device("cuda", torch.cuda.current_device())

        def dv(a, dt):
            if a is None:
                return None
            t = a if torch.is_tensor(a) else torch.as_tensor(np.asarray(a))
            return t.detach().to(device=self.dev, dtype=dt).contiguous()

        self.depth = dv(depth, torch.float64)
        self.zern = dv(zernike, torch.float64)
        self.offs = dv(z_offsets, torch.int32)
        self.z = dv(z, torch.float64)
        self.phase = dv(phase_theta, torch.float32)
        self.n_em = self.depth.numel()
        self.n_zern = 0 if self.zern is None else self.zern.shape[-1]
        self.n_slices = int(self.z.numel())


def bessel(optics, depth, zernike, z_offsets, z, n_theta, n_r, nx, ny, dx, dy,
           project=False, profiles=False, precision="fp32", workspace=None,
           stream=None, intensity=True, phase_theta=None, out=None):
    """Batched vectorial PSFs by the Bessel strategy (Eq. 10-11).

    depth [n_em], zernike [n_em, n_zern], z_offsets [n_em + 1] (int32),
    z [n_slices]: torch tensors on the device (or arrays, copied there);
    phase_theta [n_em, n_theta] (optional): free radial phase at the
    Gauss-Legendre nodes, radians.
    Returns intensity [n_slices, nx, ny] (and profiles [n_slices, 3, n_r]);
    ``out`` (device or pinned host float32 [n_slices, nx, ny]) receives it.
    """
    lib = _lib.load()
    a = _BesselArgs(optics, depth, zernike, z_offsets, z, project, phase_theta)
    o, dev = a.o, a.dev
    prec = PRECISIONS[precision] if isinstance(precision, str) else precision
    depth_d, zern_d, offs_d, z_d = a.depth, a.zern, a.offs, a.z
    n_em, n_zern, n_slices = a.n_em, a.n_zern, a.n_slices
    ws = workspace or Workspace(dev)
    need = lib.psf_bessel_workspace_size(ctypes.byref(o), n_em, n_slices,
                                         n_theta, n_r, nx, ny, prec)

    def call(I, P, buf, nbytes):
        return lib.psf_bessel_vectorial(
            ctypes.byref(o), n_em, _ptr(depth_d), _ptr(zern_d), n_zern,
            _ptr(a.phase), _ptr(offs_d), _ptr(z_d), n_slices, n_theta, n_r, nx, ny,
            float(dx), float(dy), prec, _ptr(I), _ptr(P), _ptr(buf), nbytes,
            _stream(stream))
    if need == 0:
        # invalid arguments: the call without a workspace returns their code
        # (validated before anything is launched)
        _raise_code(lib, call(None, None, None, 0))
    buf = ws.get(need)
    I = (out if out is not None else torch.empty((n_slices, nx, ny), dtype=torch.float32,
                                                 device=dev)) if intensity else None
    P = torch.empty((n_slices, 3, n_r), dtype=torch.complex64,
                    device=dev) if profiles else None
    check(lib, call(I, P, buf, buf.numel()))
    if not intensity:
        return P
    return (I, P) if profiles else I


def bessel_backward(optics, depth, zernike, z_offsets, z, n_theta, n_r, nx, ny, dx,
                    dy, target=None, grad_intensity=None, project=False,
                    phase_theta=None, precision="fp32", workspace=None, stream=None):
    """Gradients of a Bessel-strategy z-stack loss (adjoint of Eq. 10-11).

    With ``target`` [n_slices, nx, ny] the loss per emitter is sum (I - T)^2;
    otherwise ``grad_intensity`` = dL/dI.  Returns a dict with ``loss`` [n_em]
    (target only), ``grad_phase_theta`` [n_em, n_theta], ``grad_zernike``
    [n_em, n_zern] (zero for m != 0 terms) and ``grad_depth`` [n_em].
    ``precision`` selects the recomputation (and, for the split modes, the
    tensor-core adjoint contraction)."""
    lib = _lib.load()
    a = _BesselArgs(optics, depth, zernike, z_offsets, z, project, phase_theta)
    dev = a.dev
    prec = PRECISIONS[precision] if isinstance(precision, str) else precision
    need = lib.psf_bessel_backward_workspace_size(
        ctypes.byref(a.o), a.n_em, a.n_slices, n_theta, n_r, nx, ny, prec)
    if need == 0:
        raise _lib.PsfError(_lib.PSF_ERR_ARG, lib.psf_last_error().decode())
    buf = (workspace or Workspace(dev)).get(need)

    def f32(t):
        if t is None:
            return None
        t = t if torch.is_tensor(t) else torch.as_tensor(np.asarray(t))
        return t.detach().to(device=dev, dtype=torch.float32).contiguous()

    T, G = f32(target), f32(grad_intensity)
    loss = torch.empty(a.n_em, device=dev) if T is not None else None
    gW = torch.empty((a.n_em, n_theta), device=dev)
    gc = torch.empty((a.n_em, a.n_zern), device=dev) if a.n_zern else None
    gd = torch.empty(a.n_em, device=dev)
    check(lib, lib.psf_bessel_vectorial_backward(
        ctypes.byref(a.o), a.n_em, _ptr(a.depth), _ptr(a.zern), a.n_zern,
        _ptr(a.phase), _ptr(a.offs), _ptr(a.z), a.n_slices, n_theta, n_r, nx, ny,
        float(dx), float(dy), prec, _ptr(T), _ptr(G), _ptr(loss), _ptr(gW), _ptr(gc),
        _ptr(gd), _ptr(buf), buf.numel(), _stream(stream)))
    return dict(loss=loss, grad_phase_theta=gW, grad_zernike=gc, grad_depth=gd)
