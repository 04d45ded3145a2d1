"""Small, self-contained invocations of single hot kernels for profiling.

    python profile_cases.py <case> [--precision P] [--nz NZ]

Each case runs one warm-up call and one measured call of the library on
cuda:0 with sizes small enough for a full ncu capture (well under a few GB on
the device), then exits.  Cases:

* ``fourier``  - 256^2 pupil (``--pupil`` to change it), 512^2 px at 10 nm,
  16 planes, Gibson-Lanni + Zernike (one z-chunk of the benchmark stack).
* ``bessel``   - ``--emitters`` (default 256) emitters of the batched Bessel
  workload (about 600 MB of output for 256, above the 126 MB L2).
* ``bessel_backward`` - the adjoint of the same emitters with a seeded dL/dI
  (about 600 MB of input for 256 emitters).
* ``fourier_backward`` - the phase-retrieval adjoint (256^2 pupil, 128^2 px,
  32 planes) for ``--batch`` pupils against a seeded target.
* ``bessel_harmonic`` - ``--emitters`` emitters of the batched workload with
  every Zernike term, by azimuthal harmonics at the tail-bound order
  (``--mmax`` to set it) with the adaptive per-emitter order
  (``--tail-tol``, default 1e-7; 0 keeps the bound order); ``--precision
  split_fp16`` puts the radial contraction on the tensor cores.
* ``surrogate`` - the surrogate network (seeded initial weights) on
  ``--batch`` queries: the forward with the error head (one BF16 tcgen05 GEMM
  per layer).
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2502_03170_gb300 import _lib, api  # noqa: E402
from paper_2502_03170_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fourier", "bessel", "bessel_backward",
                                     "fourier_backward", "bessel_harmonic", "surrogate"])
    ap.add_argument("--mmax", type=int, default=-1)
    ap.add_argument("--tail-tol", type=float, default=1e-7)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--emitters", type=int, default=256)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--nz", type=int, default=16)
    ap.add_argument("--pupil", type=int, default=0, help="pupil size (0: the workload's)")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    if args.case == "fourier":
        c = W.fourier(nz=args.nz)
        g = api.Grid(c["grid"])
        ws = api.Workspace()
        out = torch.empty((g.c.nz, g.c.nx, g.c.ny), device="cuda")
        n_pupil = args.pupil or c["n_pupil"]
        for _ in range(2):
            api.fourier(c["optics"], n_pupil, g, zernike=c["zernike"],
                        precision=args.precision, out=out, workspace=ws)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
    elif args.case == "fourier_backward":
        from paper_2502_03170_gb300 import autograd
        c = W.adjoint(batch=args.batch)
        g = c["grid"]
        nz, nx, ny = len(g["z"]), g["nx"], g["ny"]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(11)
        T = 1e-3 * torch.rand((args.batch, nz, nx, ny), device="cuda", generator=gen)
        zern = np.zeros((args.batch, 21))
        for _ in range(2):
            loss, gW, gc = autograd._backward_call(
                c["optics"], c["n_pupil"], g, zern, None, target=T,
                precision=args.precision)
        torch.cuda.synchronize()
        assert torch.isfinite(gW).all()
    elif args.case == "surrogate":
        from paper_2502_03170_gb300 import surrogate as sg
        s = sg.Surrogate(seed=3)
        q = torch.as_tensor(sg.queries(args.batch, seed_salt=99), device="cuda")
        for _ in range(2):
            out, err = s.forward(q)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
    elif args.case == "bessel_harmonic":
        c = W.bessel(n_emitters=args.emitters)
        m = args.mmax if args.mmax >= 0 else api.harmonic_order(c["zernike"], 1e-7)
        for _ in range(2):
            I = api.bessel_harmonic(c["optics"], c["depth"], c["zernike"], c["z_offsets"],
                                    c["z"], c["n_theta"], c["n_r"], c["nx"], c["ny"],
                                    c["dx"], c["dy"], m_max=m, tail_tol=args.tail_tol,
                                    precision=args.precision)
        torch.cuda.synchronize()
        assert torch.isfinite(I).all()
    elif args.case == "bessel_backward":
        c = W.bessel(n_emitters=args.emitters)
        n_sl = int(c["z_offsets"][-1])
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        G = torch.randn((n_sl, c["nx"], c["ny"]), device="cuda", generator=gen)
        for _ in range(2):
            r = api.bessel_backward(c["optics"], c["depth"], c["zernike"],
                                    c["z_offsets"], c["z"], c["n_theta"], c["n_r"],
                                    c["nx"], c["ny"], c["dx"], c["dy"],
                                    grad_intensity=G, project=True,
                                    precision=args.precision)
        torch.cuda.synchronize()
        assert torch.isfinite(r["grad_phase_theta"]).all()
    else:
        c = W.bessel(n_emitters=args.emitters)
        for _ in range(2):
            I = api.bessel(c["optics"], c["depth"], c["zernike"], c["z_offsets"],
                           c["z"], c["n_theta"], c["n_r"], c["nx"], c["ny"],
                           c["dx"], c["dy"], project=True, precision=args.precision)
        torch.cuda.synchronize()
        assert torch.isfinite(I).all()
    print("ok")


if __name__ == "__main__":
    main()
