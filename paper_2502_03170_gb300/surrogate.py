"""Learned surrogate of the Bessel-path profiles (Python side).

The network, its training step, inference and the fallback to the Bessel
kernel all run in libpsf (see the MLP section of include/psf.h); this module
owns the device buffers and drives training with targets produced on the fly
by the Bessel path itself.
"""
import ctypes

import numpy as np
import torch

from . import _lib, api
from . import workloads as W

N_R = 256


class Surrogate:
    def __init__(self, seed=0, device=None):
        self.lib = _lib.load()
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.state = torch.zeros(self.lib.psf_mlp_state_bytes(), dtype=torch.uint8,
                                 device=self.dev)
        self.n_params = self.lib.psf_mlp_param_count()
        self._ws = api.Workspace(self.dev)
        self.step = 0
        _lib.check(self.lib, self.lib.psf_mlp_init(api._ptr(self.state), seed,
                                                   api._stream()))

    def _f32(self, a):
        t = a if torch.is_tensor(a) else torch.as_tensor(np.asarray(a))
        return t.to(device=self.dev, dtype=torch.float32).contiguous()

    def params(self):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        _lib.check(self.lib, self.lib.psf_mlp_get_params(api._ptr(self.state),
                                                         api._ptr(p), api._stream()))
        return p

    def set_params(self, p):
        p = self._f32(p)
        _lib.check(self.lib, self.lib.psf_mlp_set_params(api._ptr(self.state),
                                                         api._ptr(p), api._stream()))

    def _work(self, B):
        need = self.lib.psf_mlp_workspace_size(B)
        if need == 0:
            raise _lib.PsfError(_lib.PSF_ERR_ARG, "batch outside [1, 2^20]")
        return self._ws.get(need)

    def train_step(self, query, target, lr):
        """One Adam step; returns device loss [2] (trunk, error head)."""
        q, t = self._f32(query), self._f32(target).reshape(-1, 1536)
        B = q.shape[0]
        ws = self._work(B)
        loss = torch.empty(2, dtype=torch.float32, device=self.dev)
        self.step += 1
        _lib.check(self.lib, self.lib.psf_mlp_train_step(
            api._ptr(self.state), api._ptr(q), api._ptr(t), B, ctypes.c_float(lr),
            self.step, api._ptr(loss), api._ptr(ws), ws.numel(), api._stream()))
        return loss

    def gradients(self, query, target):
        q, t = self._f32(query), self._f32(target).reshape(-1, 1536)
        B = q.shape[0]
        ws = self._work(B)
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        loss = torch.empty(2, dtype=torch.float32, device=self.dev)
        _lib.check(self.lib, self.lib.psf_mlp_gradients(
            api._ptr(self.state), api._ptr(q), api._ptr(t), B, api._ptr(g),
            api._ptr(loss), api._ptr(ws), ws.numel(), api._stream()))
        return g, loss

    def forward(self, query, error_head=True):
        """The network's profiles [B][1536] (on-axis phase divided out:
        axis_phase(query, out, optics, +1) restores them, as profiles() does)
        and the error head's log10 relative error [B] (None with
        error_head=False: the network alone)."""
        q = self._f32(query)
        B = q.shape[0]
        ws = self._work(B)
        out = torch.empty((B, 1536), dtype=torch.float32, device=self.dev)
        err = torch.empty(B, dtype=torch.float32, device=self.dev) if error_head else None
        _lib.check(self.lib, self.lib.psf_mlp_forward(
            api._ptr(self.state), api._ptr(q), B, api._ptr(out),
            api._ptr(err) if error_head else None, api._ptr(ws), ws.numel(), api._stream()))
        return out, err

    def profiles(self, query, optics, max_rel_err, n_theta, nx, ny, dx, dy,
                 precision="split_fp16"):
        """Surrogate profiles with Bessel fallback: (out [B][1536], n_fallback)."""
        q = self._f32(query)
        B = q.shape[0]
        o = optics if isinstance(optics, _lib.PsfOptics) else api.make_optics(optics)
        prec = api.PRECISIONS[precision] if isinstance(precision, str) else precision
        need = self.lib.psf_surrogate_workspace_size(ctypes.byref(o), B, n_theta, nx,
                                                     ny, prec)
        if need == 0:
            raise _lib.PsfError(_lib.PSF_ERR_ARG, self.lib.psf_last_error().decode())
        ws = self._ws.get(need)
        out = torch.empty((B, 1536), dtype=torch.float32, device=self.dev)
        nfb = ctypes.c_int(0)
        _lib.check(self.lib, self.lib.psf_surrogate_profiles(
            api._ptr(self.state), ctypes.byref(o), api._ptr(q), B, float(max_rel_err),
            n_theta, nx, ny, float(dx), float(dy), prec, api._ptr(out),
            ctypes.byref(nfb), api._ptr(ws), ws.numel(), api._stream()))
        return out, nfb.value


def axis_phase(query, data, optics, direction):
    """In place: the complex profiles data [B][1536] times e^{direction 2 pi i
    phi}, phi the on-axis phase of each query (psf_surrogate_phase).  The
    network learns the profiles with the phase divided out (direction -1)."""
    lib = _lib.load()
    q = query if torch.is_tensor(query) else torch.as_tensor(np.asarray(query))
    q = q.to(device=data.device, dtype=torch.float32).contiguous()
    o = optics if isinstance(optics, _lib.PsfOptics) else api.make_optics(optics)
    _lib.check(lib, lib.psf_surrogate_phase(ctypes.byref(o), api._ptr(q), q.shape[0],
                                            api._ptr(data), int(direction), api._stream()))
    return data


def residual_targets(query, targets, optics):
    """Training targets in the form the network learns: the Bessel-path
    profiles with their on-axis phase divided out (a copy)."""
    return axis_phase(query, targets.clone(), optics, -1)


def bessel_targets(query, optics, n_theta, nx, ny, dx, dy, precision="split_fp16",
                   workspace=None):
    """Profiles [B][1536] of the queries by the Bessel path (one emitter and
    one defocus plane per query, m != 0 Zernike terms projected out)."""
    q = query if torch.is_tensor(query) else torch.as_tensor(np.asarray(query))
    q = q.to(device="cuda", dtype=torch.float64)
    B = q.shape[0]
    offs = torch.arange(B + 1, dtype=torch.int32, device=q.device)
    P = api.bessel(optics, q[:, 21].contiguous(), q[:, :21].contiguous(), offs,
                   q[:, 22].contiguous(), n_theta, N_R, nx, ny, dx, dy, project=True,
                   profiles=True, precision=precision, workspace=workspace,
                   intensity=False)
    return torch.view_as_real(P).reshape(B, 1536)


def queries(n, seed_salt=0):
    """Surrogate queries as float [n][23] (c_1..c_21, depth, z)."""
    c, depth, z = W.surrogate_queries(n, seed_salt)
    return np.concatenate([c, depth[:, None], z[:, None]], axis=1).astype(np.float32)
