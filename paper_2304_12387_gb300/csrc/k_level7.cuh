// Kernels of a 7-point face-weight lattice level (LevelT) shared by the
// unsmoothed (k_lattice.cu) and smoothed-aggregation (k_amg.cu) hierarchies,
// and the dense coarsest-level solve.
#pragma once
#include "hd_internal.h"

namespace {

// residual b - S x at cell (I,J,Z) given the x value there
template <typename T>
__device__ __forceinline__ T stencil_res(const LevelT<T>& lv, const T* __restrict__ x, T bc, T xc, int I, int J,
                                         int Z, int64_t c) {
  int64_t xl = I + (int64_t)(lv.X + 1) * (J + (int64_t)lv.Y * Z);
  int64_t yl = I + (int64_t)lv.X * (J + (int64_t)(lv.Y + 1) * Z);
  int64_t zl = I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z);
  int64_t XY = (int64_t)lv.X * lv.Y;
  T r = fma(-lv.diag[c], xc, bc);
  if (I > 0) r = fma(lv.wx[xl], x[c - 1], r);
  if (I < lv.X - 1) r = fma(lv.wx[xl + 1], x[c + 1], r);
  if (J > 0) r = fma(lv.wy[yl], x[c - lv.X], r);
  if (J < lv.Y - 1) r = fma(lv.wy[yl + lv.X], x[c + lv.X], r);
  if (Z > 0) r = fma(lv.wz[zl], x[c - XY], r);
  if (Z < lv.Z - 1) r = fma(lv.wz[zl + XY], x[c + XY], r);
  return r;
}

// first pre-smoothing sweep from a zero guess: x = D_l1^-1 b
template <typename T>
__global__ void k_vc_scale(LevelT<T> lv, const T* __restrict__ b, T* __restrict__ x) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  x[c] = lv.dinv[c] * b[c];
}

template <typename T>
__global__ void k_vc_jacobi(LevelT<T> lv, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  T xc = x[c];
  xo[c] = fma(lv.dinv[c], stencil_res<T>(lv, x, b[c], xc, I, J, Z, c), xc);
}

// coarsest level: x = A^-1 b with the stored FP64 dense inverse (n <= a few hundred);
// FP64 accumulation for either vector type (the coarsest solve stays FP64)
template <typename T>
__global__ void k_vc_coarse(int n, const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x) {
  // one warp per output row; the inverse is symmetric, so row i is contiguous
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* row = Ainv + (int64_t)i * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(row[j], (double)b[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[i] = (T)s;
}

}  // namespace
