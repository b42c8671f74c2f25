// Per-element building blocks on the L2 space (k^3 histopolation DOFs per element, Sec.
// 2.1), for kernels that give one CTA to each element: block sums, the lattice index of an
// element-local cell, the change of basis between Gauss-Legendre nodal values and
// histopolation coefficients, and the sum-factorised passes between the DOFs and the q^3
// Gauss points. Degree and point count are run-time values; the element's data sits in
// shared memory. Layouts: element-local index a = a1 + k (a2 + k a3), point p = p1 +
// q (p2 + q p3), tables B[p k + a] (a basis at the points) and TT[j k + m] (histopolation
// coefficient j of the Gauss-Legendre Lagrange function m).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

// sum of v over the CTA (every thread gets it); red: one double per warp
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// global lattice index of element-local cell a of element e
__device__ __forceinline__ int64_t mi_cell(int64_t e, int a, int k, int nx, int ny) {
  const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
  const int a1 = a % k, a2 = (a / k) % k, a3 = a / (k * k);
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k;
  return (ex * k + a1) + X * ((ey * k + a2) + Y * (ez * k + a3));
}

// out = (M x M x M) in with M(j, m) = TT[j k + m] (tr = true: the transpose TT^T acting on
// histopolation data) or TT[m k + j] (tr = false: TT acting on GL nodal data); u, v scratch
template <typename T>
__device__ void mi_tt3(int k, const T* TT, bool tr, const T* in, T* u, T* v, T* out) {
  const int n = k * k * k;
  auto M = [&](int j, int m) { return tr ? TT[j * k + m] : TT[m * k + j]; };
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int m1 = i % k, r = i / k;
    T s = T(0);
    for (int j = 0; j < k; ++j) s = fma(M(j, m1), in[j + k * r], s);
    u[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int m1 = i % k, m2 = (i / k) % k, j3 = i / (k * k);
    T s = T(0);
    for (int j = 0; j < k; ++j) s = fma(M(j, m2), u[m1 + k * (j + k * j3)], s);
    v[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = i % (k * k), m3 = i / (k * k);
    T s = T(0);
    for (int j = 0; j < k; ++j) s = fma(M(j, m3), v[r + k * k * j], s);
    out[i] = s;
  }
  __syncthreads();
}

// T3[p] = wd[p] sum_a B(p1,a1) B(p2,a2) B(p3,a3) P[a] (wd NULL: 1): B (q x k) to the points
// along x, y, z (T1: q k k, T2: q q k scratch)
template <typename T>
__device__ void mi_to_points(int k, int q, const T* B, const T* P, T* T1, T* T2, T* T3, const T* wd) {
  const int kk = k * k, qq = q * q;
  for (int i = threadIdx.x; i < q * kk; i += blockDim.x) {  // T1[p1 + q r], r = a2 + k a3
    const int p1 = i % q, r = i / q;
    T s = T(0);
    for (int a = 0; a < k; ++a) s = fma(B[p1 * k + a], P[a + k * r], s);
    T1[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < qq * k; i += blockDim.x) {  // T2[p1 + q (p2 + q a3)]
    const int p1 = i % q, p2 = (i / q) % q, a3 = i / qq;
    T s = T(0);
    for (int a = 0; a < k; ++a) s = fma(B[p2 * k + a], T1[p1 + q * (a + k * a3)], s);
    T2[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < qq * q; i += blockDim.x) {  // T3[p], scaled by the point weight
    const int r = i % qq, p3 = i / qq;
    T s = T(0);
    for (int a = 0; a < k; ++a) s = fma(B[p3 * k + a], T2[r + qq * a], s);
    T3[i] = wd ? s * wd[i] : s;
  }
  __syncthreads();
}

// W[a] = sum_p B(p1,a1) B(p2,a2) B(p3,a3) T3[p]: back from the points along z, y, x
// (T2, T1 scratch)
template <typename T>
__device__ void mi_from_points(int k, int q, const T* B, const T* T3, T* T2, T* T1, T* W) {
  const int kk = k * k, qq = q * q;
  for (int i = threadIdx.x; i < qq * k; i += blockDim.x) {  // back along z
    const int r = i % qq, a3 = i / qq;
    T s = T(0);
    for (int p = 0; p < q; ++p) s = fma(B[p * k + a3], T3[r + qq * p], s);
    T2[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < q * kk; i += blockDim.x) {  // back along y
    const int p1 = i % q, a2 = (i / q) % k, a3 = i / (q * k);
    T s = T(0);
    for (int p = 0; p < q; ++p) s = fma(B[p * k + a2], T2[p1 + q * (p + q * a3)], s);
    T1[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kk * k; i += blockDim.x) {  // back along x
    const int a1 = i % k, r = i / k;
    T s = T(0);
    for (int p = 0; p < q; ++p) s = fma(B[p * k + a1], T1[p + q * r], s);
    W[i] = s;
  }
  __syncthreads();
}

// w = W_e p by sum factorisation: to the points, the point weights wd, and back
// (T1: q k k, T2: q q k, T3: q^3 values)
template <typename T>
__device__ void mi_apply_w(int k, int q, const T* B, const T* __restrict__ wd, const T* P, T* W, T* T1, T* T2,
                           T* T3) {
  mi_to_points(k, q, B, P, T1, T2, T3, wd);
  mi_from_points(k, q, B, T3, T2, T1, W);
}

}  // namespace
