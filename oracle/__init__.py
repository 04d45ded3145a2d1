"""FP64 CPU oracle for the vectorial Richards-Wolf PSF hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (``paper_2502_03170_gb300``) and imports
nothing from it.

Everything here is plain numpy/scipy in float64 / complex128, written from the
paper's equations in the order the paper states them:

* :mod:`oracle.optics`     pupil geometry, Eq. 6 (far field, q_s = q_p = 1),
                           Eq. 13-14 (Gibson-Lanni), Eq. 15 (Noll Zernike),
                           Eq. 16 (apodization), Eq. 17 (Gaussian envelope).
* :mod:`oracle.fourier`    Eq. 8 + Eq. 12 by the midpoint rule on the pupil
                           grid (brute-force double sum and separable form).
* :mod:`oracle.bessel`     Eq. 10-11 by Gauss-Legendre in theta, radial
                           profiles, linear radial interpolation.
* :mod:`oracle.continuum`  Eq. 9 + Eq. 12 by direct double quadrature in
                           (theta, phi), no Bessel identities.
* :mod:`oracle.scalar`     Eq. 3 / Eq. 5 in the paraxial form of Sec. 5.2.2
                           (Airy check, Eq. 18).
* :mod:`oracle.adjoint`    gradient of the z-stack L2 loss w.r.t. the pupil
                           phase map W_0 and Zernike coefficients (Eq. 15).
* :mod:`oracle.mlp`        the surrogate MLP's forward/backward/Adam in FP64.

Library primitives used as steps: ``numpy`` matmul / exp,
``numpy.polynomial.legendre.leggauss`` (Gauss-Legendre nodes),
``scipy.special.jv`` (Bessel J_n).

Pins (tests marked ``not gpu``) tie every function to something other than
itself: the Airy closed form (Eq. 18), the Fourier-Bessel equivalence theorem
(Sec. 4.1), the continuum quadrature, axial / rotational symmetry, discrete
Parseval energy, Zernike orthonormality, Gauss-Legendre exactness, the
paraxial Gibson-Lanni expansion and finite differences for the gradient.
The MLP oracle is pinned by finite differences, PyTorch's FP64 autograd and
torch.optim.Adam; its agreement with the paper is "parity unpinned" (the
paper has no surrogate).
"""
