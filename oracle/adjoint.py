"""Gradient of a z-stack L2 loss through the Fourier strategy (FP64, test-only).

Loss L = sum_{z,x,y} (I - T)^2 with I = sum_c |E_c|^2 and E_c from Eq. 8/12.
Every pupil factor carries e^{iW}, W = W_GL + sum_j c_j Z_j + W_0 (Eq. 15), so
dP_c/dW = i P_c at each node.  Writing E_c(z) = M(P~_c,z) with
M(X) = C ds^2 A_x X A_y^T and P~ = P e^{i k z cos(theta)}:

    dL/dW_0[p, q] = sum_{z, c} 2 Re( conj(G^_{c,z}[p, q]) * i * P~_{c,z}[p, q] ),
    G^ = M^H(R) = conj(C ds^2) A_x^H R conj(A_y),  R = 2 (I - T) E_c,
    dL/dc_j      = sum_{p, q} Z_j[p, q] dL/dW_0[p, q]   (chain rule, Eq. 15).

This is the analytic adjoint of the separable oracle; the tests pin it with
central finite differences of :func:`loss`.
"""
import numpy as np

from .fourier import C_FOURIER, pupil_field, zoom_matrix
from .optics import pupil_geometry, pupil_mask, zernike


def loss(I, T):
    d = I - T
    return float(np.sum(d * d))


def loss_and_grad(opt, n_pupil, grid, zernike_coeffs, phase_map, target,
                  n_zern=None):
    """Returns (L, dL/dW_0 [N, N], dL/dc [n_zern], I [nz, nx, ny])."""
    P, cos_t = pupil_field(opt, n_pupil, zernike_coeffs, phase_map)
    ds = 2.0 * opt.s_max / n_pupil
    cfac = C_FOURIER * ds * ds
    Ax = zoom_matrix(opt, n_pupil, grid["nx"], grid["dx"])
    Ay = zoom_matrix(opt, n_pupil, grid["ny"], grid["dy"])
    zs = np.asarray(grid["z"], dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    gW = np.zeros((n_pupil, n_pupil))
    I_all = np.empty((len(zs), grid["nx"], grid["ny"]))
    L = 0.0
    for iz, z in enumerate(zs):
        defocus = np.exp(1j * opt.k * z * cos_t)
        Pt = [P[c] * defocus for c in range(3)]
        E = [cfac * (Ax @ Pt[c] @ Ay.T) for c in range(3)]
        I = sum(e.real ** 2 + e.imag ** 2 for e in E)
        I_all[iz] = I
        d = I - target[iz]
        L += float(np.sum(d * d))
        for c in range(3):
            R = 2.0 * d * E[c]
            Gh = np.conj(cfac) * (Ax.conj().T @ R @ Ay.conj())
            gW += 2.0 * np.real(np.conj(Gh) * 1j * Pt[c])
    gW = np.where(pupil_mask(n_pupil), gW, 0.0)
    nz_ = n_zern if n_zern is not None else (
        0 if zernike_coeffs is None else len(zernike_coeffs))
    _, _, _, _, rn, phi = pupil_geometry(opt, n_pupil)
    gc = np.array([np.sum(zernike(j + 1, rn, phi) * gW) for j in range(nz_)])
    return L, gW, gc, I_all
