"""Surrogate MLP on the GPU: gradients and the Adam step against the FP64
oracle (BF16 storage emulated), the fallback to the Bessel path, and what a
trained network gains over the Bessel kernel alone.

Gradient tolerance: the oracle rounds to BF16 where the kernels store BF16,
but a value that lands within FP32 accumulation noise of a BF16 rounding
boundary can round the other way (one BF16 ulp, 2^-8 relative); these flips
compound through the four stored hidden gradients, measured at 6e-5 (output
layer) to 9e-4 (input layer) relative L2 -> 1e-3."""
import time

import numpy as np
import pytest
import torch

from oracle import mlp as om
from paper_2502_03170_gb300 import surrogate as sg
from paper_2502_03170_gb300 import workloads as W

from .gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL_BF16 = 1e-3
GEOM = dict(n_theta=200, nx=128, ny=128, dx=0.020, dy=0.020)


def host_params(seed, scale=0.06):
    g = np.random.default_rng(seed)
    lay = om.param_layout()
    p = g.normal(0, scale, lay["total"]).astype(np.float32)
    W0 = p[lay["W"][0]:lay["W"][0] + 256 * om.IN_PAD].reshape(256, om.IN_PAD)
    W0[:, om.IN_FEAT:] = 0.0
    return p


def test_gradients_match_oracle(lib):
    s = sg.Surrogate(seed=1)
    p = host_params(5)
    s.set_params(p)
    g = np.random.default_rng(6)
    q = sg.queries(300, seed_salt=9)
    t = g.normal(0, 0.3, (300, 1536)).astype(np.float32)
    grads, loss = s.gradients(q, t)
    torch.cuda.synchronize()
    L, Le, gr = om.loss_and_grads(p.astype(np.float64), q, t, emulate=True)
    loss = loss.cpu().numpy()
    assert abs(loss[0] - L) <= 1e-4 * abs(L)
    assert abs(loss[1] - Le) <= 1e-3 * abs(Le) + 1e-6
    gpu = grads.cpu().numpy()
    lay = om.param_layout()
    for l in range(om.NLAYER):
        sl = slice(lay["W"][l], lay["b"][l] + om.layer_out(l))
        assert rel_l2(gpu[sl], gr[sl]) <= TOL_BF16, l
    sl = slice(lay["We"], lay["total"])
    assert rel_l2(gpu[sl], gr[sl]) <= TOL_BF16


def test_adam_step_matches_oracle(lib):
    s = sg.Surrogate(seed=2)
    p = host_params(7)
    s.set_params(p)
    q = sg.queries(128, seed_salt=3)
    t = np.random.default_rng(8).normal(0, 0.3, (128, 1536)).astype(np.float32)
    grads, _ = s.gradients(q, t)
    gpu_g = grads.cpu().numpy().astype(np.float64)
    s.train_step(q, t, lr=1e-3)
    p1 = s.params().cpu().numpy().astype(np.float64)
    ref, _, _ = om.adam(p.astype(np.float64), 0.0, 0.0, gpu_g, lr=1e-3, step=1)
    assert rel_l2(p1 - p, ref - p) <= 1e-4


def test_fallback_paths(lib):
    d = W.optics_gibson_lanni(0.0)
    s = sg.Surrogate(seed=3)
    q = sg.queries(257, seed_salt=4)
    ref = sg.bessel_targets(q, d, **GEOM).cpu().numpy()
    out, nfb = s.profiles(q, d, max_rel_err=1e-30, **GEOM)   # everything falls back
    assert nfb == 257
    assert np.array_equal(out.cpu().numpy(), ref)
    out2, nfb2 = s.profiles(q, d, max_rel_err=1e30, **GEOM)  # nothing falls back
    mo, _ = s.forward(q)
    sg.axis_phase(q, mo, d, +1)                              # the same restore
    assert nfb2 == 0
    assert torch.equal(out2, mo)


def test_axis_phase_against_oracle(lib):
    """The on-axis phase against its definition evaluated by the oracle's own
    Gibson-Lanni path (Eq. 13-14) and Zernike polynomials (Eq. 15) at rho = 0
    plus k z; and the -1 / +1 round trip."""
    import math

    from oracle.optics import Optics, gibson_lanni_phase, zernike
    d = W.optics_gibson_lanni(0.0)
    opt = Optics.from_dict(d)
    q = sg.queries(64, seed_salt=5)
    q[:, 0] = 0.3                                            # piston enters as well
    ones = torch.zeros((64, 1536), device="cuda")
    ones[:, 0::2] = 1.0
    ph = sg.axis_phase(q, ones.clone(), d, +1).cpu().numpy()
    got = ph[:, 0::2] + 1j * ph[:, 1::2]
    for b in range(64):
        phi = float(np.real(gibson_lanni_phase(opt.with_depth(float(q[b, 21])),
                                               np.zeros(1)))[0])
        phi += sum(float(q[b, j - 1]) * float(zernike(j, np.zeros(1), np.zeros(1))[0])
                   for j in range(1, 22))
        phi += opt.k * float(q[b, 22])
        ref = complex(math.cos(phi), math.sin(phi))
        assert np.max(np.abs(got[b] - ref)) <= 2e-6, b
    t = torch.randn((64, 1536), device="cuda")
    back = sg.axis_phase(q, sg.residual_targets(q, t, d), d, +1)
    assert rel_l2(back.cpu().numpy(), t.cpu().numpy()) <= 1e-6


def train_surrogate(d, n_train=1 << 20, B=4096, steps=20000, lr0=2e-3, seed=12):
    """Adam with a cosine schedule on n_train Bessel-path samples."""
    q_all = torch.as_tensor(sg.queries(n_train, seed_salt=11), device="cuda")
    t_all = torch.empty((n_train, 1536), device="cuda")
    for k in range(0, n_train, 131072):
        t_all[k:k + 131072] = sg.bessel_targets(q_all[k:k + 131072], d, **GEOM)
    sg.axis_phase(q_all, t_all, d, -1)              # the form the network learns
    s = sg.Surrogate(seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    losses = []
    for it in range(steps):
        if it % (n_train // B) == 0:
            perm = torch.randperm(n_train, device="cuda", generator=gen)
        k = (it % (n_train // B)) * B
        lr = lr0 * 0.5 * (1 + np.cos(np.pi * it / steps)) + 1e-6
        loss = s.train_step(q_all[perm[k:k + B]], t_all[perm[k:k + B]], lr)
        if it in (0, steps - 1):
            losses.append(loss.clone())
    torch.cuda.synchronize()
    return s, [x.cpu().numpy() for x in losses]


def test_training_gain(lib):
    """Train on 1M Bessel-path samples generated on the GPU, then answer 100k
    fresh queries: report accuracy, the accepted fraction and the error head's
    honesty at the 1e-3 bound of the workload and at 3e-2, and the time against
    the Bessel kernel alone."""
    d = W.optics_gibson_lanni(0.0)
    s, (first, last) = train_surrogate(d)
    assert last[0] < 1e-3 * first[0]
    nq = 100000
    q = torch.as_tensor(sg.queries(nq, seed_salt=99), device="cuda")
    ref = sg.bessel_targets(q, d, **GEOM)
    out, err_pred = s.forward(q)
    sg.axis_phase(q, out, d, +1)
    true = (torch.linalg.norm(out - ref, dim=1) / torch.linalg.norm(ref, dim=1)).cpu().numpy()
    pred = err_pred.cpu().numpy()
    for thr in (1e-3, 3e-2, 1e-1):
        for _ in range(2):
            sg.bessel_targets(q, d, **GEOM)
            s.profiles(q, d, thr, **GEOM)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sg.bessel_targets(q, d, **GEOM)
        torch.cuda.synchronize()
        t_bessel = time.perf_counter() - t0
        t0 = time.perf_counter()
        out_s, nfb = s.profiles(q, d, thr, **GEOM)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t0
        final = (torch.linalg.norm(out_s - ref, dim=1) /
                 torch.linalg.norm(ref, dim=1)).cpu().numpy()
        acc = np.ones(nq, dtype=bool)
        acc[:] = False
        fb = final <= 1e-6                       # exact Bessel answers
        acc = ~fb
        mis = (final[acc] > thr).mean() if acc.any() else 0.0
        print("surrogate thr %.0e: loss %.3e -> %.3e, median err %.2e, accepted %.3f, "
              "accepted over the bound %.4f, bessel %.2f ms, surrogate+fallback %.2f ms "
              "(%d fallbacks)" % (thr, first[0], last[0], np.median(true), acc.mean(),
                                  mis, 1e3 * t_bessel, 1e3 * t_sur, nfb))
        assert nfb >= int(fb.sum()) - 5
        assert mis <= 0.05                       # honest where it answers
