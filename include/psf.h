/*
 * psf.h - C ABI of the GB300 vectorial PSF library (libpsf.so).
 *
 * Computes vectorial high-NA point-spread-function z-stacks from the
 * Richards-Wolf integral (Eq. 1) with the correction factors of Eq. 12
 * (apodization Eq. 16, Gaussian envelope Eq. 17, Gibson-Lanni Eq. 13-14,
 * Zernike + free phase mask Eq. 15) by the two strategies of Sec. 3:
 *   - Cartesian / Fourier (Eq. 8): pupil fields mapped to a zoomed focal grid
 *     by per-z separable matrix-DFT contractions;
 *   - spherical / Bessel (Eq. 10-11): theta quadrature of J_0/J_1/J_2 as a
 *     [r x theta] x [theta x z] contraction, then radial interpolation.
 *
 * Conventions shared by every entry point
 *   - Lengths in micrometres.  k = 2 pi n_i / lambda (Sec. 3.1), f k = 1, so
 *     E carries -i/(2 pi) (Eq. 8) or -i/2 (Eq. 10); both strategies return
 *     fields on the same absolute scale.
 *   - Pupil grid (Fourier): N x N cell-centred nodes u_p = (2p+1-N)/N, disk
 *     (2p+1-N)^2 + (2q+1-N)^2 <= N^2, sin(theta) = (NA/n_i) sqrt(u^2+v^2)
 *     (footnote of Sec. 3.4), weight ds^2 with ds = 2 NA / (n_i N).
 *     Index p runs along x, q along y.
 *   - Output grid: x_a = (a - (nx-1)/2) dx, y_b = (b - (ny-1)/2) dy.
 *   - Layout (Sec. 4.1): row-major (z, channel, x, y).  Intensity is
 *     float [nz][nx][ny]; fields are interleaved complex64 [nz][3][nx][ny].
 *   - Zernike coefficients: Noll index j = 1..n_zern stored at [j-1], radians,
 *     RMS-normalised on the unit pupil (Noll 1976); phi from +x towards +y.
 *   - Fresnel coefficients q_s = q_p = 1 (Eq. 7 not applied) unless the
 *     PSF_FRESNEL flag is set; PSF_SCALAR selects the scalar model.
 *
 * Ownership and execution
 *   - Every device buffer is owned by the caller.  The library allocates no
 *     device memory: each call takes a caller-provided device workspace whose
 *     size the matching *_workspace_size() query returns.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous with respect to the host.  Host arrays
 *     passed in (z lists, Zernike rows) are read before the call returns.
 *   - Calls that share a workspace must not overlap on the GPU.
 *
 * Errors
 *   - Arguments are validated on the host before anything is enqueued; on
 *     error nothing is launched and outputs are untouched.  The return value
 *     is PSF_OK or a negative PSF_ERR_* code; psf_last_error() gives a
 *     message (thread-local, valid until the next call on the thread).
 *   - Conditions only the device can see (a bounded wait that gave up, a
 *     non-axisymmetric Zernike row inside device data) are recorded in a
 *     status word at the start of the workspace; psf_workspace_status()
 *     synchronises the stream and returns it.  A kernel that records an
 *     error returns early without trapping.
 */
#ifndef PSF_H
#define PSF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define PSF_OK                    0
#define PSF_ERR_ARG              -1  /* bad size / pointer / NA >= n_i ...     */
#define PSF_ERR_NOT_AXISYMMETRIC -2  /* m != 0 Zernike term on the Bessel path */
#define PSF_ERR_WORKSPACE        -3  /* workspace missing or too small         */
#define PSF_ERR_PRECISION        -4  /* precision mode not supported here      */
#define PSF_ERR_CUDA             -5  /* a CUDA runtime call failed             */
#define PSF_ERR_DEVICE_TIMEOUT   -6  /* a bounded device wait gave up          */

/* ---- precision of the contractions ---------------------------------------
 * Phases are always formed in extended precision (FP64 host/device for the
 * per-call pupil and twiddle tables, double-float for per-(node, z) defocus)
 * and reduced modulo one cycle before sin/cos.                              */
#define PSF_PREC_FP32        0  /* plain FP32 FMA complex contractions        */
#define PSF_PREC_SPLIT_FP16  1  /* tcgen05 kind::f16, operands split hi+lo
                                   fp16 (power-of-two scaled), 3 products,
                                   FP32 accumulation in TMEM                  */
#define PSF_PREC_SPLIT_BF16  2  /* same with bf16 hi+lo operands              */
#define PSF_PREC_FP32_CHIRPZ 3  /* Fourier forward only: the zoom DFTs of
                                   Eq. 8 by Bluestein's chirp-Z transform
                                   (Sec. 4: FFT-based zoom for arbitrary pixel
                                   size), FP32 shared-memory FFTs of length
                                   L = 2^k >= max(256, n_pupil + n_out - 1),
                                   L <= 4096 per direction; same discrete sum
                                   as PSF_PREC_FP32, O(L log L) per line      */
#define PSF_PREC_SPLIT_TF32  5  /* Fourier forward: tcgen05 kind::tf32, operands
                                   split hi + lo TF32 (FP32 storage), 3
                                   products, FP32 accumulation in TMEM       */
#define PSF_PREC_TF32        6  /* Fourier forward: one TF32 product per MAC
                                   (10-bit operand mantissas: 1.3e-4 to
                                   3.4e-4; outside the accuracy envelope,
                                   accepted only with PSF_OUTSIDE_ENVELOPE)   */
#define PSF_PREC_AUTO        4  /* the fastest mode inside the accuracy
                                   envelope below: Fourier forward split FP16
                                   (n_pupil <= 512), else split BF16 (<= 1024),
                                   else chirp-Z when its FFT length fits, else
                                   FP32; spherical forwards split FP16 (n_theta
                                   <= 448), else FP32; adjoints split FP16
                                   where the tensor-core adjoint runs, else
                                   FP32                                       */

/* ---- accuracy envelope of the split modes ---------------------------------
 * Every forward call is meant to stay within 1e-5 (max |I - I_ref| over max
 * |I_ref| of the stack) of the FP64 oracle of the same discrete sums.  The
 * split modes round each operand to hi + lo 16-bit parts and accumulate in
 * FP32 on the tensor cores; their error grows with the length of each
 * contraction.  A forward call in a split mode is refused with
 * PSF_ERR_PRECISION (before any launch) outside the sizes where the error
 * measured on the benchmark workloads (Gibson-Lanni + Noll 4..21, 512^2 px)
 * stays within half the bound:
 *   Fourier   split FP16  n_pupil <= 512   (4.3e-6 at 512; 8.7e-6 at 1024)
 *             split BF16  n_pupil <= 1024  (4.2e-6 at 1024; 7.6e-6 at 2048)
 *             split TF32  n_pupil <= 256   (3.0e-6 at 256; 6.1e-6 at 512)
 *             TF32        refused          (one product: 1.3e-4 to 3.4e-4)
 *   Bessel /  split FP16  n_theta <= 448   (5.2e-6 at 448; 9.9e-6 at 880)
 *   harmonic  split BF16  refused          (5.2e-5 on the Bessel workload)
 * The flag PSF_OUTSIDE_ENVELOPE lifts these refusals.
 * FP32 and chirp-Z stay below 2e-6 at every size.  The adjoints (gradient
 * bound 1e-4 relative L2) take every mode they support.                      */

/* ---- flags ---------------------------------------------------------------- */
#define PSF_PROJECT_AXISYMMETRIC 1  /* Bessel path: drop m != 0 Zernike terms
                                       instead of reporting an error (Sec. 3.4:
                                       the spherical form needs an
                                       axisymmetric pupil)                     */
#define PSF_SCALAR               2  /* scalar model (Sec. 3.2): e_far = e_inc,
                                       Eq. 3 (Cartesian) / Eq. 5 (spherical);
                                       the field is channel 0 (x), the Jones
                                       vector is not used; every path          */
#define PSF_FRESNEL              4  /* vectorial model with the Fresnel
                                       transmission coefficients q_s, q_p of
                                       Eq. 7 in Eq. 6, over the interfaces
                                       sample -> coverslip -> immersion (Snell
                                       angles, principal root where evanescent).
                                       Every path and adjoint; the split Bessel
                                       contraction then runs per order n with
                                       the complex g_n on the F operand, and
                                       the Bessel adjoint contracts with B^H    */
#define PSF_OUTSIDE_ENVELOPE     8  /* accept a precision mode outside the
                                       accuracy envelope below (results may miss
                                       the 1e-5 bound; for comparisons)        */

/* Physical parameters (Eq. 1, Eq. 13-14, Eq. 16-17). */
typedef struct {
  double NA;          /* numerical aperture, 0 < NA < n_i                      */
  double lambda;      /* vacuum wavelength, um                                 */
  double n_i;         /* immersion index (propagation medium, Sec. 3.1)        */
  double n_s;         /* sample index                                          */
  double n_g;         /* coverslip index                                       */
  double n_i_design;  /* design (starred) immersion index                      */
  double n_g_design;  /* design coverslip index                                */
  double t_g;         /* coverslip thickness, um                               */
  double t_g_design;  /* design coverslip thickness, um                        */
  double t_i_design;  /* design immersion thickness t_i*, um                   */
  double depth;       /* emitter depth t_s, um (Fourier path; the Bessel path
                         takes one depth per emitter)                          */
  double pol[4];      /* Jones vector (p_x.re, p_x.im, p_y.re, p_y.im)         */
  int    apodize;     /* 1: A = sqrt(cos theta) (Eq. 16); 0: A = 1            */
  double s_env;       /* > 0: Gaussian envelope exp(-sin^2/s_env^2) (Eq. 17)   */
  int    flags;       /* PSF_PROJECT_AXISYMMETRIC | PSF_SCALAR | PSF_FRESNEL   */
} psf_optics;

/* Output grid of the Fourier strategy. */
typedef struct {
  int nx, ny;         /* pixels along x and y                                 */
  double dx, dy;      /* pixel pitch, um                                       */
  int nz;             /* number of defocus planes                              */
  const double* z;    /* host [nz] defocus distances, um                       */
} psf_grid;

/* ========================================================================== */
/* Fourier (Cartesian) strategy, Eq. 8 with Eq. 12.                           */
/* ========================================================================== */

/* Bytes of device workspace psf_fourier_vectorial() needs for these sizes
 * (0 on invalid arguments). */
size_t psf_fourier_workspace_size(const psf_optics* opt, int n_pupil,
                                  const psf_grid* grid, int precision);

/* E_c(x_a, y_b, z) = -i/(2 pi) ds^2 sum_{p,q in disk} A e^{iW} e_inf,c / cos
 *                    e^{i k z cos} e^{i k s_max (u_p x_a + v_q y_b)},
 * I = |E_x|^2 + |E_y|^2 + |E_z|^2 (Eq. 8, Eq. 6, Eq. 12-17).
 *   zernike    host [n_zern] (may be NULL if n_zern == 0), 0 <= n_zern <= 66
 *   phase_map  device float [n_pupil][n_pupil] W_0 in radians, or NULL
 *   intensity  float [nz][nx][ny] (required), device memory or pinned host
 *              memory; host memory that is not pinned gives PSF_ERR_ARG
 *              before any launch.  A pinned host intensity without fields
 *              on the split precisions is streamed: the stack is computed
 *              in eight z-chunks into a staging area of the workspace (when
 *              it has room beyond the chunk layout) and each chunk is copied
 *              to the host while the next one runs; the call completes on
 *              `stream` once the stack is on the host.  Otherwise the
 *              kernels store through the host memory's device alias.
 *   fields     complex64 [nz][3][nx][ny], or NULL (same memory rules)
 * Sizes: 2 <= n_pupil <= 4096, nx, ny, nz >= 1. */
int psf_fourier_vectorial(const psf_optics* opt, int n_pupil,
                          const psf_grid* grid, const double* zernike,
                          int n_zern, const float* phase_map, int precision,
                          float* intensity, void* fields, void* workspace,
                          size_t ws_bytes, void* stream);

/* Fixed size of the library-owned scratch array used by
 * psf_fourier_vectorial_noalloc() (24 MiB). */
#define PSF_NOALLOC_SCRATCH_BYTES (24u << 20)

/* psf_fourier_vectorial() for callers that cannot allocate device memory.
 * The paper has no counterpart: this is a deployment convenience.
 *
 * Some callers cannot hand the library a workspace: their host application
 * owns all device memory through its own allocator (a framework's caching
 * allocator, an imaging application that gives plug-ins a fixed budget), or
 * they run latency-critical loops in which cudaMalloc, which can synchronise
 * the device, is not allowed.  This entry point allocates nothing: it uses a
 * file-scope device array of PSF_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library keeps until the process exits.  The caller still owns
 * and passes the inputs and outputs (same meaning as in
 * psf_fourier_vectorial(); contractions in PSF_PREC_FP32).
 *   - Sizes whose workspace would exceed the array are rejected with
 *     PSF_ERR_WORKSPACE and a message giving both sizes; nothing is launched.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: a cudaDeviceReset() between calls is not supported (the
 *     array's memory would be gone while the library still holds its
 *     address).
 *   - All calls share the one array and it keeps the previous call's
 *     contents; every call rewrites what it reads.  Calls whose executions
 *     overlap on the GPU (other streams, other host threads) race on the
 *     array and give undefined results: serialise them.
 *   - Device-side status (psf_workspace_status) is not available here. */
int psf_fourier_vectorial_noalloc(const psf_optics* opt, int n_pupil,
                                  const psf_grid* grid, const double* zernike,
                                  int n_zern, const float* phase_map,
                                  float* intensity, void* fields, void* stream);

/* Workspace for psf_fourier_vectorial_backward(). */
size_t psf_fourier_backward_workspace_size(const psf_optics* opt, int n_pupil,
                                           const psf_grid* grid, int precision);

/* Workspace with which psf_fourier_vectorial_backward() handles `batch`
 * pupils in one pass over all their planes (at most 2048 planes and 16 GB;
 * split precisions).  The backward call takes the largest chunk of planes
 * that fits the workspace it is given, from this size down to the one of
 * psf_fourier_backward_workspace_size() (128 planes); longer chunks run the
 * contractions in fewer, fuller launches. */
size_t psf_fourier_backward_workspace_size_batch(const psf_optics* opt, int n_pupil,
                                                 const psf_grid* grid, int precision,
                                                 int batch);

/* Gradient of L_b = sum_{z,x,y} g(I_b) for `batch` independent pupils, by the
 * adjoint of Eq. 8 with per-z recomputation (no pupil field is stored):
 *   dL/dW_0[p,q] = sum_{z,c} 2 Re(conj(G^_{c,z}[p,q]) i P_{c,z}[p,q]),
 *   G^ = conj(C ds^2) A_x^H R conj(A_y),  R = (dL/dI) E_c,
 *   dL/dc_j = sum_{p,q} Z_j[p,q] dL/dW_0[p,q]   (chain rule through Eq. 15).
 * With target != NULL the loss is sum (I - T)^2 (dL/dI = 2 (I - T));
 * otherwise dL/dI = grad_intensity.
 *   zernike         host [batch][n_zern]
 *   phase_map       device [batch][n_pupil][n_pupil] or NULL (zero)
 *   target          device [batch][nz][nx][ny] or NULL
 *   grad_intensity  device [batch][nz][nx][ny] (used iff target == NULL)
 *   loss            device float [batch] or NULL (only with target)
 *   grad_phase_map  device float [batch][n_pupil][n_pupil] or NULL
 *   grad_zernike    device float [batch][n_zern] or NULL                    */
int psf_fourier_vectorial_backward(const psf_optics* opt, int n_pupil,
                                   const psf_grid* grid, int batch,
                                   const double* zernike, int n_zern,
                                   const float* phase_map, int precision,
                                   const float* target,
                                   const float* grad_intensity, float* loss,
                                   float* grad_phase_map, float* grad_zernike,
                                   void* workspace, size_t ws_bytes,
                                   void* stream);

/* ========================================================================== */
/* Bessel (spherical) strategy, Eq. 10-11, batched emitters.                  */
/* ========================================================================== */

/* Workspace for psf_bessel_vectorial(). */
size_t psf_bessel_workspace_size(const psf_optics* base, int n_emitters,
                                 int n_slices, int n_theta, int n_r, int nx,
                                 int ny, int precision);

/* Every emitter e has depth t_s = depth[e], Zernike row zernike[e][0..n_zern)
 * (only m = 0 terms enter, Sec. 3.4), an optional free radial phase
 * phase_theta[e][j] at the theta nodes and defocus planes
 * z[z_offsets[e] .. z_offsets[e+1]).  Per slice:
 *   I_n(r_i, z) = sum_j w_j g_n(theta_j) J_n(k r_i sin theta_j)
 *                 A(theta_j) e^{i(W_e(theta_j) + k z cos theta_j)},
 * W_e = W_GL(t_s) (Eq. 13-14) + sum_{m=0} c_j Z_j (Eq. 15) + phase_theta[e],
 * g_0 = sin(1+cos), g_1 = sin^2, g_2 = sin(cos-1) (Eq. 11), Gauss-Legendre
 * nodes theta_j on [0, asin(NA/n_i)]; r_i = i r_max/(n_r-1) with r_max the
 * corner radius of the output grid; complex linear interpolation of I_n at
 * each pixel radius; E from Eq. 10 with the Jones vector of `base`.
 *   depth, zernike, z_offsets, z : DEVICE arrays (double, double, int, double)
 *   phase_theta  device float [n_emitters][n_theta] (radians) or NULL
 *   n_slices   = z_offsets[n_emitters] (host copy, for sizing)
 *   intensity  float [n_slices][nx][ny] (packed; device or pinned host
 *              memory, as for psf_fourier_vectorial); may be NULL when
 *              profiles is given (profiles only, no Cartesian epilogue)
 *   profiles   device complex64 [n_slices][3][n_r] (I_0, I_1, I_2) or NULL
 * A non-zero m != 0 coefficient without PSF_PROJECT_AXISYMMETRIC marks the
 * workspace status PSF_ERR_NOT_AXISYMMETRIC and that emitter's slices are not
 * written.  Sizes: n_theta in [2, 880], n_r in [2, 4096].                 */
int psf_bessel_vectorial(const psf_optics* base, int n_emitters,
                         const double* depth, const double* zernike, int n_zern,
                         const float* phase_theta, const int* z_offsets,
                         const double* z, int n_slices, int n_theta, int n_r,
                         int nx, int ny, double dx, double dy, int precision,
                         float* intensity, void* profiles, void* workspace,
                         size_t ws_bytes, void* stream);

/* ========================================================================== */
/* Spherical strategy without axial symmetry: azimuthal harmonics.            */
/* ========================================================================== */

/* The spherical form (Sec. 3.4, Eq. 10-11) needs an axisymmetric pupil.  For
 * any W(theta, phi) the pupil is expanded in azimuthal harmonics,
 *   A e^{i W(theta, phi)} = sum_{|m| <= M} P_m(theta) e^{i m phi},
 * P_m by a DFT over N_phi = 4 * (smallest power of two >= M + 1) azimuths;
 * the far field of Eq. 6 has harmonics n = -2 .. 2, and the phi integral of
 * Eq. 9 is exact by the Jacobi-Anger expansion:
 *   E_c(rho, phi, z) = -i sum_{|l| <= M+2} i^l e^{i l phi} I_{c,l}(rho, z),
 *   I_{c,l} = int sum_kinds coef_c g_n(theta) P_{l-n'}(theta)
 *             J_l(k rho sin theta) e^{i k z cos theta} dtheta
 * (g_n of Eq. 11 and its Fresnel / scalar forms; Gauss-Legendre in theta;
 * I_{c,l} on the radial grid r_i = i r_max / (N_r - 1), linearly
 * interpolated).  With m = 0 terms only this is Eq. 10-11.  Cost grows with
 * the 2M + 5 orders.                                                         */

/* Truncation order: the largest over the emitters of the smallest M = K d
 * with alpha^{K+1} / (K+1)! e^alpha <= tol, alpha = sum |c_j| N_j and d =
 * max |m| over the emitter's m != 0 Noll terms (the l1 tail of the
 * harmonics of e^{i W} beyond M).  zernike: HOST [n_em][n_zern].  Returns
 * M >= 0, or a negative PSF_ERR_* code. */
int psf_bessel_harmonic_order(const double* zernike, int n_em, int n_zern, double tol);

/* Workspace for psf_bessel_vectorial_harmonic() (0 on invalid arguments). */
size_t psf_bessel_harmonic_workspace_size(const psf_optics* base, int n_emitters,
                                          int n_slices, int n_theta, int n_r,
                                          int nx, int ny, int m_max, int precision);

/* Batched PSFs with every Zernike term (any m) by the azimuthal harmonics
 * |m| <= m_max (0 <= m_max <= 64).  Arguments as psf_bessel_vectorial()
 * (device arrays depth [n_em], zernike [n_em][n_zern], z_offsets [n_em+1],
 * z [n_slices]; intensity device or pinned host [n_slices][nx][ny]); no free
 * radial phase, no profiles output; the flags PSF_SCALAR / PSF_FRESNEL select
 * the model (PSF_PROJECT_AXISYMMETRIC is ignored: no term is dropped).
 * tail_tol in [0, 1): with tail_tol > 0 each emitter keeps only the
 * harmonics |m| <= M_e, M_e the largest |m| <= m_max with
 * max_theta |P_m(theta)| > tail_tol max_theta |P_0(theta)| (0 if none; the
 * harmonics past those that carry W fall faster than geometrically, so the
 * dropped tail is about tail_tol; the tail bound of
 * psf_bessel_harmonic_order() is pessimistic and the adaptive order
 * typically halves the orders); 0 keeps m_max for every emitter.
 * PSF_ERR_ARG for tail_tol outside [0, 1).
 * precision: PSF_PREC_FP32 (the per-order radial contraction in FP32 FMA)
 * or PSF_PREC_SPLIT_FP16 (the contraction on the tensor cores: w_j J_|l|
 * and D Bh split into FP16 hi + lo, three products, FP32 accumulation);
 * other modes give PSF_ERR_PRECISION (BF16 parts keep too few bits for
 * the 1e-5 bound here). */
int psf_bessel_vectorial_harmonic(const psf_optics* base, int n_emitters,
                                  const double* depth, const double* zernike,
                                  int n_zern, const int* z_offsets, const double* z,
                                  int n_slices, int n_theta, int n_r, int nx, int ny,
                                  double dx, double dy, int m_max, double tail_tol,
                                  int precision, float* intensity, void* workspace,
                                  size_t ws_bytes, void* stream);

/* Workspace for psf_bessel_vectorial_backward() (0 if the arguments are
 * invalid; the backward takes nx, ny <= 4096). */
size_t psf_bessel_backward_workspace_size(const psf_optics* base, int n_emitters,
                                          int n_slices, int n_theta, int n_r,
                                          int nx, int ny, int precision);

/* Gradient of L = sum_{slices, pixels} g(I) through Eq. 10-11 (same inputs as
 * psf_bessel_vectorial; the profiles are recomputed, nothing is stored).
 * With target != NULL the loss is sum (I - T)^2 per emitter, otherwise
 * dL/dI = grad_intensity.  The adjoint, with G = dL/dI and the complex
 * gradient g_X = dL/dRe X + i dL/dIm X:
 *   g_E_c = 2 G E_c;  g_I_n through the conjugate of Eq. 10 and the transposed
 *   radial interpolation;  g_F = sum_n B_n^H g_I_n (B_n the J_n operand,
 *   complex with PSF_FRESNEL);
 *   Q_j = sum_{z of e} conj(g_F(theta_j, z)) F(theta_j, z);
 *   dL/dW_0(theta_j) = -Im Q_j,
 *   dL/dc_q  = sum_j Z_q(sin theta_j / s_max) dL/dW_0(theta_j)  (m = 0 Noll q;
 *              0 for m != 0, which do not enter the spherical form),
 *   dL/dt_s  = sum_j Re(i D_j Q_j), D_j = dW_GL/dt_s (Eq. 13 with t_i from
 *              Eq. 14; complex where a layer is evanescent).
 * Every reduction runs in a fixed order (bitwise reproducible).
 *   target, grad_intensity  device float [n_slices][nx][ny] (one non-NULL)
 *   loss              device float [n_emitters] or NULL (target only)
 *   grad_phase_theta  device float [n_emitters][n_theta] or NULL
 *   grad_zernike      device float [n_emitters][n_zern] or NULL
 *   grad_depth        device float [n_emitters] or NULL  (per um)
 * precision: PSF_PREC_FP32 runs the recomputation and the adjoint contraction
 * in FP32; the split modes recompute the profiles on tensor cores in that
 * split and, where the grid's mirror groups fit in shared memory (up to about
 * 150 x 150 pixels), contract g_F on tensor cores in split BF16 (hi + lo,
 * FP32 accumulation).  An emitter rejected as non-axisymmetric (workspace
 * status) gets zero gradients. */
int psf_bessel_vectorial_backward(const psf_optics* base, int n_emitters,
                                  const double* depth, const double* zernike,
                                  int n_zern, const float* phase_theta,
                                  const int* z_offsets, const double* z,
                                  int n_slices, int n_theta, int n_r, int nx,
                                  int ny, double dx, double dy, int precision,
                                  const float* target,
                                  const float* grad_intensity, float* loss,
                                  float* grad_phase_theta, float* grad_zernike,
                                  float* grad_depth, void* workspace,
                                  size_t ws_bytes, void* stream);

/* ========================================================================== */
/* Learned surrogate of the Bessel profiles (not in the paper; motivated by   */
/* its learning-based applications, Sec. 6).                                  */
/* ========================================================================== */
/* An MLP 23 -> 256 -> 256 -> 256 -> 256 -> 1536 with SiLU on the hidden
 * layers maps a query q = (c_1..c_21 [rad], depth t_s [um], defocus z [um])
 * to the complex profiles I_0, I_1, I_2 of Eq. 11 at the 256 radii of the
 * Bessel path (out[b] = complex64 [3][256] viewed as float [1536]); an error
 * head 256 -> 1 on the last hidden layer predicts log10 of the relative L2
 * error of out[b].  The network sees q as c / 0.05, d = t_s / 5 - 1,
 * u = z / 2 and the Fourier features sin/cos(2 pi f_k u), f_k = 0.5 16^(k/23),
 * and sin/cos(2 pi g_k d), g_k = 0.5 40^(k/23), k = 0..23 (119 inputs padded
 * to 120).  Weights live in FP32 (master) with BF16 copies; every GEMM runs on
 * tcgen05 in BF16 with FP32 accumulation; hidden activations and
 * pre-activations are stored in BF16.
 *
 * state: caller-owned device block of psf_mlp_state_bytes() bytes holding the
 *   FP32 parameters (packed W_0 [256][120] (input padded), b_0, W_1, b_1,
 *   W_2, b_2, W_3, b_3, W_4 [1536][256], b_4, error head w_e [256], b_e),
 *   the Adam moments and the BF16 weight copies.
 * query [B][23], target / out [B][1536]: device float. */
#define PSF_MLP_IN 23
#define PSF_MLP_OUT 1536
size_t psf_mlp_param_count(void);
size_t psf_mlp_state_bytes(void);
/* Deterministic initialisation from seed (uniform fan-in scaled weights,
 * zero biases, zero moments). */
int psf_mlp_init(void* state, unsigned long long seed, void* stream);
size_t psf_mlp_workspace_size(int batch);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step = 1, 2, ... for the
 * bias correction) on L = (1/B) sum_b |out_b - t_b|^2 / |t_b|^2 for the
 * trunk and (1/B) sum_b (e_b - log10(rel_err_b))^2 for the error head (whose
 * gradient does not flow into the trunk).  loss: device float [2] or NULL. */
int psf_mlp_train_step(void* state, const float* query, const float* target,
                       int batch, float lr, int step, float* loss, void* ws,
                       size_t ws_bytes, void* stream);
/* Gradients of the same losses at the current parameters (packed like the
 * parameters, device float [param_count]); the state is not changed. */
int psf_mlp_gradients(void* state, const float* query, const float* target,
                      int batch, float* grads, float* loss, void* ws,
                      size_t ws_bytes, void* stream);
/* Inference: out [B][1536]; err_log10 [B] (predicted log10 relative error)
 * or NULL.  Sizes: 1 <= batch <= 1048576. */
int psf_mlp_forward(const void* state, const float* query, int batch, float* out,
                    float* err_log10, void* ws, size_t ws_bytes, void* stream);
int psf_mlp_get_params(const void* state, float* params, void* stream);
int psf_mlp_set_params(void* state, const float* params, void* stream);

/* The profiles' on-axis phase phi (theta = 0 of Eq. 10-11): the Gibson-Lanni
 * path of Eq. 13 at the query's depth t_s, the m = 0 Zernike terms of Eq. 15
 * at rho = 0 (query coefficients c_1..c_21) and the defocus n_i z / lambda,
 * in cycles (FP64, reduced mod 1).  Multiplies the complex profiles data
 * [batch][3 x 256] (the interleaved re / im [batch][1536] layout) in place
 * by e^{direction 2 pi i phi}.  The network is trained on targets with the
 * phase divided out (direction -1: a smoother function of z and t_s) and
 * psf_mlp_forward returns that form; psf_surrogate_profiles restores the
 * phase (direction +1).  query: device float [batch][23]; data: device.
 * PSF_ERR_ARG for NULL pointers, direction not +-1 or batch outside
 * [0, 1048576]. */
int psf_surrogate_phase(const psf_optics* base, const float* query, int batch,
                        float* data, int direction, void* stream);

/* Profiles of `batch` queries by the surrogate, with the Bessel path as the
 * fallback: the network's answer with its on-axis phase restored
 * (psf_surrogate_phase), and queries whose predicted relative error, doubled
 * as a safety margin, exceeds max_rel_err (or is not finite) are
 * recomputed by psf_bessel_vectorial (geometry of `base`, n_theta Gauss-
 * Legendre nodes, 256 radii up to the corner radius of the nx x ny grid at
 * dx, dy) and their outputs replaced.  Synchronises the stream once (to size
 * the fallback batch); *n_fallback receives its size. */
size_t psf_surrogate_workspace_size(const psf_optics* base, int batch,
                                    int n_theta, int nx, int ny, int precision);
int psf_surrogate_profiles(const void* state, const psf_optics* base,
                           const float* query, int batch, double max_rel_err,
                           int n_theta, int nx, int ny, double dx, double dy,
                           int precision, float* out, int* n_fallback, void* ws,
                           size_t ws_bytes, void* stream);

/* ========================================================================== */
/* Status and diagnostics.                                                    */
/* ========================================================================== */

/* Synchronises `stream` and returns the device status word of `workspace`
 * (PSF_OK, PSF_ERR_NOT_AXISYMMETRIC or PSF_ERR_DEVICE_TIMEOUT), or
 * PSF_ERR_CUDA if the stream itself reports an error. */
int psf_workspace_status(const void* workspace, void* stream);

/* Kernel timing for benchmarks.  While enabled, every hot kernel launch is
 * bracketed by a pair of CUDA events recorded on the launching stream (the
 * events are created once and reused; enabling clears previous records).
 * psf_kernel_timing_read() synchronises on the recorded events and returns
 * the number of launches and their summed device time for one kernel class:
 *   0 pupil fields, 1 stage-1 contraction, 2 stage-2 contraction + |E|^2,
 *   3 Bessel radial contraction, 4 Bessel radial-to-Cartesian epilogue,
 *   5 adjoint recomputation + contractions, 6 per-call set-up kernels
 *   (pupil node table, zoom matrices, J_n operand, emitter tables).
 * Returns PSF_OK, or PSF_ERR_ARG for an unknown class.  Not thread-safe. */
int psf_kernel_timing(int enable);
int psf_kernel_timing_read(int kernel_class, int* launches, double* total_ms);

/* Message of the last error on this thread ("" if none). */
const char* psf_last_error(void);

/* ABI version (major * 100 + minor). */
int psf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSF_H */
