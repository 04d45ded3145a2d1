"""Seeded synthetic inputs shaped like the paper's PSF workloads.

This module holds only parameter sets and random draws (numpy
``default_rng(20250203 + config)``); it contains none of the PSF arithmetic,
so both the CUDA path and the FP64 oracle can be fed from it.

Workloads (lengths in um, lambda = 0.532):

* ``plain``   - NA 1.4, n_i 1.518, aberration-free, circular polarisation,
  64 x 64 pixels at 0.020, 16 slices over [-1, 1]; Fourier pupil 64^2,
  Bessel 128 theta nodes / 128 radii.
* ``fourier`` - 256^2 pupil, 512 x 512 pixels at 0.010, 128 slices over
  [-2, 2], Gibson-Lanni (n_s 1.33, n_g 1.5, t_g 170, t_i* 150, depth 2) and
  Noll c_4..c_21 ~ N(0, 0.1) rad.
* ``bessel``  - 4096 emitters, depth ~ U(0, 10), Noll c_4..c_11 ~ N(0, 0.05)
  (projected onto m = 0), n_z ~ U{8..64} slices over [-1, 1] each,
  256 radii, 200 theta nodes, 128 x 128 pixels at 0.020.
* ``adjoint`` - batch of 64 phase-retrieval problems: 256^2 pupil,
  128 x 128 pixels at 0.020, 32 slices over [-1, 1]; true phase =
  Noll c_4..c_21 ~ N(0, 0.1) + a smooth random map.
* ``surrogate`` - (c_1..c_21 with c_4..c_11 ~ N(0, 0.05), depth U(0, 10),
  z U(-2, 2)) query vectors for the MLP surrogate.
"""
import math

import numpy as np

SEED_BASE = 20250203
N_ZERN = 21
CIRCULAR = (1.0 / math.sqrt(2.0), 1j / math.sqrt(2.0))


def rng(config, salt=0):
    return np.random.default_rng(SEED_BASE + config + 1000 * salt)


def optics_plain():
    return dict(NA=1.4, lam=0.532, n_i=1.518, n_s=1.518, n_g=1.5,
                n_i_design=1.518, n_g_design=1.5, t_g=170.0, t_g_design=170.0,
                t_i_design=150.0, depth=0.0, pol=CIRCULAR, apodize=True,
                s_env=0.0)


def optics_gibson_lanni(depth=2.0):
    d = optics_plain()
    d.update(n_s=1.33, n_g=1.5, n_g_design=1.5, t_g=170.0, t_g_design=170.0,
             t_i_design=150.0, depth=float(depth))
    return d


def linspace_z(lo, hi, n):
    return np.linspace(lo, hi, n)


def plain(n_pupil=64, nx=64, nz=16):
    """Aberration-free stack (64^2 px at 20 nm, 16 slices over +-1 um)."""
    return dict(optics=optics_plain(), n_pupil=n_pupil,
                grid=dict(nx=nx, ny=nx, dx=0.020, dy=0.020,
                          z=linspace_z(-1.0, 1.0, nz)),
                zernike=np.zeros(N_ZERN), n_theta=128, n_r=128)


def fourier(n_pupil=256, nx=512, nz=128, z_range=2.0, seed_salt=0):
    """Fourier strategy at scale (Gibson-Lanni + Noll 4..21 ~ N(0, 0.1))."""
    g = rng(2, seed_salt)
    c = np.zeros(N_ZERN)
    c[3:21] = g.normal(0.0, 0.1, size=18)
    return dict(optics=optics_gibson_lanni(2.0), n_pupil=n_pupil,
                grid=dict(nx=nx, ny=nx, dx=0.010, dy=0.010,
                          z=linspace_z(-z_range, z_range, nz)),
                zernike=c)


def bessel(n_emitters=4096, n_theta=200, n_r=256, nx=128, nz_lo=8, nz_hi=64,
           seed_salt=0):
    """Batched emitters with uneven z-stacks (packed z list + offsets)."""
    g = rng(3, seed_salt)
    depth = g.uniform(0.0, 10.0, size=n_emitters)
    zc = np.zeros((n_emitters, N_ZERN))
    zc[:, 3:11] = g.normal(0.0, 0.05, size=(n_emitters, 8))
    nz = g.integers(nz_lo, nz_hi + 1, size=n_emitters)
    offs = np.zeros(n_emitters + 1, dtype=np.int32)
    offs[1:] = np.cumsum(nz)
    z = np.concatenate([linspace_z(-1.0, 1.0, int(n)) for n in nz])
    return dict(optics=optics_gibson_lanni(0.0), n_emitters=n_emitters,
                depth=depth, zernike=zc, z_offsets=offs, z=z,
                n_theta=n_theta, n_r=n_r, nx=nx, ny=nx, dx=0.020, dy=0.020)


def smooth_map(g, n_pupil, n_modes=6, amp=0.3):
    """Random smooth phase map: a few low-frequency cosines on [-1, 1]^2."""
    u = (2.0 * np.arange(n_pupil) + 1.0 - n_pupil) / n_pupil
    U, V = np.meshgrid(u, u, indexing="ij")
    out = np.zeros((n_pupil, n_pupil))
    for _ in range(n_modes):
        fx, fy = g.uniform(-1.5, 1.5, size=2)
        out += g.normal(0.0, amp / math.sqrt(n_modes)) * np.cos(
            math.pi * (fx * U + fy * V) + g.uniform(0, 2 * math.pi))
    return out


def adjoint(batch=64, n_pupil=256, nx=128, nz=32):
    """Phase retrieval problems: true phases and the start point (zero)."""
    g = rng(4)
    c_true = np.zeros((batch, N_ZERN))
    c_true[:, 3:21] = g.normal(0.0, 0.1, size=(batch, 18))
    w_true = np.stack([smooth_map(g, n_pupil) for _ in range(batch)])
    return dict(optics=optics_plain(), n_pupil=n_pupil, batch=batch,
                grid=dict(nx=nx, ny=nx, dx=0.020, dy=0.020,
                          z=linspace_z(-1.0, 1.0, nz)),
                c_true=c_true, w_true=w_true, noise_seed=SEED_BASE + 40)


def surrogate_queries(n, seed_salt=0, z_range=2.0):
    """MLP inputs: 21 Zernike coefficients, depth, z."""
    g = rng(5, seed_salt)
    c = np.zeros((n, N_ZERN))
    c[:, 3:11] = g.normal(0.0, 0.05, size=(n, 8))
    depth = g.uniform(0.0, 10.0, size=n)
    z = g.uniform(-z_range, z_range, size=n)
    return c, depth, z
