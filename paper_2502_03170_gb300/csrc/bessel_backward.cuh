// Adjoint kernels of the Bessel (spherical) strategy (Eq. 10-11).
#pragma once

#include "bessel_kernels.cuh"

namespace psf {

// Pixels that share one radius: (a, b) and its mirrors (nx-1-a, b),
// (a, ny-1-b), (nx-1-a, ny-1-b) (index -1 where a mirror coincides with an
// earlier one).  f is the interpolation weight in cell `cell`; the
// polarisation factor of mirror k is gc + gs for k = 0, 3 and gc - gs for
// k = 1, 2 (S1 cos 2phi + S2 sin 2phi; sin 2phi changes sign under one flip).
// The table is sorted by cell; cell_start[c] .. cell_start[c+1] are cell c's.
struct __align__(16) PixGroup {
  int pix[4];
  float f, gc, gs;
  int cell;
};

size_t bessel_adj_epilogue_smem(const BesselParams& p, bool stage);
bool bessel_adj_stage_fits(const BesselParams& p);
// g_P (in place of the profiles) and, with target, the per-slice loss
void launch_bessel_adj_epilogue(const BesselParams& p, float2* prof, const int* slice_em,
                                const int* valid, const PixGroup* groups,
                                const int* cell_start, const float* target,
                                const float* grad_intensity, float* loss_slice,
                                cudaStream_t s);
// Sorted two-pass form for grids whose mirror groups fit in shared memory:
// gpc[g] = (position of natural group g in the cell-sorted order, cell),
// gfg[g] = (f, gc, gs, 0), sorted_f[k] = f of the k-th sorted group.
// With g_hi != NULL, g_P is written as BF16 hi/lo planes [2 n_slices][kp]
// (rows (s, re), (s, im)) for the tensor-core contraction, else in place.
bool bessel_adj_sorted_fits(const BesselParams& p);
void launch_bessel_adj_epilogue_sorted(const BesselParams& p, float2* prof,
                                       const int* slice_em, const int* valid,
                                       const int2* gpc, const float4* gfg,
                                       const float* sorted_f, const int* cell_start,
                                       const float* target, const float* grad_intensity,
                                       float* loss_slice, uint16_t* g_hi, uint16_t* g_lo,
                                       int kp, cudaStream_t s);
// Staged form of the sorted epilogue (slices streamed into shared memory by
// the TMA engine): grids with <= 4096 mirror groups, nx * ny % 4 == 0, even
// n_r and a 16-byte aligned dL/dI (or target).
bool bessel_adj_staged_fits(const BesselParams& p, const void* src);
void launch_bessel_adj_epilogue_staged(const BesselParams& p, float2* prof,
                                       const int* slice_em, const int* valid,
                                       const int2* gpc, const float4* gfg,
                                       const float* sorted_f, const int* cell_start,
                                       const float* target, const float* grad_intensity,
                                       float* loss_slice, uint16_t* g_hi, uint16_t* g_lo,
                                       int kp, int* status, cudaStream_t s);
// g_F[s][j] = sum_row conj(B[j][row]) g_P[s][row], B = Bt (real) or, when
// BtC is non-null, the complex operand of the Fresnel weights
void launch_bessel_adj_contract(const BesselParams& p, const float* Bt, const float2* BtC,
                                const float2* gP, float2* gF, cudaStream_t s);
// per-emitter gradients and loss
void launch_bessel_adj_reduce(const BesselParams& p, ThetaTable t, EmitterTable et,
                              const int* z_offsets, const float2* zz, const float2* gF,
                              const float* loss_slice, float* loss, float* grad_w,
                              float* grad_zern, float* grad_depth, cudaStream_t s);

}  // namespace psf
