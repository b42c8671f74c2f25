// Kernels of a 7-point face-weight lattice level (LevelT) shared by the
// unsmoothed (k_lattice.cu) and smoothed-aggregation (k_amg.cu) hierarchies,
// and the dense coarsest-level solve.
#pragma once
#include "hd_internal.h"

namespace {

// Rounding the operator of a level to FP32 loses its row sums (the mass of S~, C~ =
// W~^-1, and the boundary faces) where they are small against the diagonal: with a
// 10^6 coefficient contrast the FP32 W-cycle then differs from the FP64 one by tens of
// percent (its second coarse correction amplifies the inconsistency). The FP32 copies
// therefore keep, in place of the diagonal, the row sum computed in FP64, and apply
// (S x)_c = rs_c x_c + sum_nbr w (x_c - x_nbr): the zero-row-sum part acts on
// differences, the small part is exact to FP32 rounding.
template <typename T>
constexpr bool rowsum_form() { return sizeof(T) == 4; }
// x - o on the row-sum levels; x on the others, where o is zero (a double-float
// subtraction of zero would still cost a full TwoSum)
template <typename T>
__device__ __forceinline__ T rs_diff(T x, T o) {
  if constexpr (rowsum_form<T>()) return x - o;
  else return x;
}

// residual b - S x at cell (I,J,Z) given the x value there (FP32 levels: diag holds the
// row sum, see rowsum_form)
template <typename T>
__device__ __forceinline__ T stencil_res(const LevelT<T>& lv, const T* __restrict__ x, T bc, T xc, int I, int J,
                                         int Z, int64_t c) {
  int64_t xl = I + (int64_t)(lv.X + 1) * (J + (int64_t)lv.Y * Z);
  int64_t yl = I + (int64_t)lv.X * (J + (int64_t)(lv.Y + 1) * Z);
  int64_t zl = I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z);
  int64_t XY = (int64_t)lv.X * lv.Y;
  // Face weights exist for boundary faces too, so all six are loaded; a missing
  // neighbour reads x at the own cell and gets a zero weight. No branch: the
  // loads overlap instead of waiting one after another.
  const bool ml = I > 0, mh = I < lv.X - 1, nl = J > 0, nh = J < lv.Y - 1, ol = Z > 0, oh = Z < lv.Z - 1;
  const T w0 = lv.wx[xl], w1 = lv.wx[xl + 1], w2 = lv.wy[yl], w3 = lv.wy[yl + lv.X], w4 = lv.wz[zl],
          w5 = lv.wz[zl + XY];
  const T x0 = x[ml ? c - 1 : c], x1 = x[mh ? c + 1 : c], x2 = x[nl ? c - lv.X : c], x3 = x[nh ? c + lv.X : c],
          x4 = x[ol ? c - XY : c], x5 = x[oh ? c + XY : c];
  T r = fma(-lv.diag[c], xc, bc);
  if constexpr (rowsum_form<T>()) {
    r = fma(ml ? w0 : (T)0, x0 - xc, r);
    r = fma(mh ? w1 : (T)0, x1 - xc, r);
    r = fma(nl ? w2 : (T)0, x2 - xc, r);
    r = fma(nh ? w3 : (T)0, x3 - xc, r);
    r = fma(ol ? w4 : (T)0, x4 - xc, r);
    r = fma(oh ? w5 : (T)0, x5 - xc, r);
    return r;
  }
  r = fma(ml ? w0 : (T)0, x0, r);
  r = fma(mh ? w1 : (T)0, x1, r);
  r = fma(nl ? w2 : (T)0, x2, r);
  r = fma(nh ? w3 : (T)0, x3, r);
  r = fma(ol ? w4 : (T)0, x4, r);
  r = fma(oh ? w5 : (T)0, x5, r);
  return r;
}

// row sums of a FP64 7-point level (diag minus the weights of the faces that have a
// neighbour), the diagonal slot of its FP32 copy
__global__ void k_level_rowsum(LevelT<double> lv, float* __restrict__ out) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  const int64_t xl = I + (int64_t)(lv.X + 1) * (J + (int64_t)lv.Y * Z);
  const int64_t yl = I + (int64_t)lv.X * (J + (int64_t)(lv.Y + 1) * Z);
  const int64_t zl = c, XY = (int64_t)lv.X * lv.Y;
  double s = lv.diag[c];
  if (I > 0) s -= lv.wx[xl];
  if (I < lv.X - 1) s -= lv.wx[xl + 1];
  if (J > 0) s -= lv.wy[yl];
  if (J < lv.Y - 1) s -= lv.wy[yl + lv.X];
  if (Z > 0) s -= lv.wz[zl];
  if (Z < lv.Z - 1) s -= lv.wz[zl + XY];
  out[c] = (float)s;
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
