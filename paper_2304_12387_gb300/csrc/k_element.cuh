// Element kernels of the block operator, templated on the scalar type, the
// degree K (subcells per direction) and the number Q of Gauss-Legendre points
// per direction. One translation unit per K instantiates them (k_elem_k*.cu).
//
// Data layouts (element e = ex + nx (ey + ny ez)):
//   G     [E][6][Q^3]      w_p b_e (J^T J)_{ab} / det J at point p, ab in 00,01,02,11,12,22
//   winv  [E][K^3][K^3]    unweighted W_e^-1 (symmetric; element (b,a) read as (a,b))
//   wdet  [E][Q^3]         w_p / det J
// Local RT dof order: x-component i + (K+1)(j + K l); y-component
// NX1 + i + K (j + (K+1) l); z-component 2 NX1 + i + K (j + K l), NX1 = (K+1) K^2.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "dfloat.cuh"
#include "hd_internal.h"
#include "tc_ptx.cuh"

namespace hdk {

template <typename T>
struct TabT {
  T BI[HD_MAXQ * (HD_MAXK + 1)];
  T BH[HD_MAXQ * HD_MAXK];
  T BG[HD_MAXQ * HD_MAXK];
  T TT[HD_MAXK * HD_MAXK];
  T GW[HD_MAXQ];             // 1D Gauss-Legendre weights on [0,1]
  T HI[HD_MAXK * HD_MAXK];   // inverse 1D histopolation mass
  T BIp[16], BIn[16], BHp[16], BHn[16], BITp[16], BITn[16], BHTp[16], BHTn[16];  // even-odd forms
};

template <typename T>
inline T tab_cast(double v) { return (T)v; }
template <>
inline dfloat tab_cast<dfloat>(double v) { return df_split_host(v); }

template <typename T>
inline TabT<T> make_tab(const ElemTables& t) {
  TabT<T> o;
  for (int i = 0; i < HD_MAXQ * (HD_MAXK + 1); ++i) o.BI[i] = tab_cast<T>(t.BI[i]);
  for (int i = 0; i < HD_MAXQ * HD_MAXK; ++i) o.BH[i] = tab_cast<T>(t.BH[i]);
  for (int i = 0; i < HD_MAXQ * HD_MAXK; ++i) o.BG[i] = tab_cast<T>(t.BG[i]);
  for (int i = 0; i < HD_MAXK * HD_MAXK; ++i) o.TT[i] = tab_cast<T>(t.TT[i]);
  for (int i = 0; i < HD_MAXQ; ++i) o.GW[i] = tab_cast<T>(t.gw[i]);
  for (int i = 0; i < HD_MAXK * HD_MAXK; ++i) o.HI[i] = tab_cast<T>(t.HI[i]);
  for (int i = 0; i < 16; ++i) {
    o.BIp[i] = tab_cast<T>(t.BIp[i]);
    o.BIn[i] = tab_cast<T>(t.BIn[i]);
    o.BHp[i] = tab_cast<T>(t.BHp[i]);
    o.BHn[i] = tab_cast<T>(t.BHn[i]);
    o.BITp[i] = tab_cast<T>(t.BITp[i]);
    o.BITn[i] = tab_cast<T>(t.BITn[i]);
    o.BHTp[i] = tab_cast<T>(t.BHTp[i]);
    o.BHTn[i] = tab_cast<T>(t.BHTn[i]);
  }
  return o;
}

// Local CG parameters (Sec. 2.5 / 3.1: W^-1 by a fused per-element CG in the
// Gauss-Legendre nodal basis, no global reductions).
template <typename T>
struct CgArgs {
  const T* wdet;     // [E][Q^3] w_p / det J, or null: use the dense W_e^-1
  const T* diag;     // [E][K^3] Jacobi diagonal of W_e in the basis the CG works in
  int maxit;
  T tol2;            // stop when ||r||^2 <= tol2 ||b||^2 (per element)
  int hist;          // 0: CG in the GL nodal basis (Sec. 2.5); 1: in the histopolation basis
  int chol;          // 1 (and wdet null): W_e^-1 q_e by the stored Cholesky factor passed as winv
  int* err = nullptr;  // error word: bit 2 = a bounded wait for staged W_e^-1 rows ran out
};

// Sum of products as one FMA chain (one type per arithmetic: double, float or
// double-float with its renormalised FMA).
template <typename T>
struct Acc {
  T s;
  __device__ __forceinline__ void init(T b, T x) { s = b * x; }
  __device__ __forceinline__ void add(T b, T x) { s = fma(b, x, s); }
  __device__ __forceinline__ T get() const { return s; }
};

// out[o*SO] = sum_i B[o*NI + i] in[i*SI], o < NO   (B row-major NO x NI)
template <typename T, int NI, int NO, int SI, int SO>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out, const T* B) {
  T x[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) x[i] = in[i * SI];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    Acc<T> s;
    s.init(B[o * NI], x[0]);
#pragma unroll
    for (int i = 1; i < NI; ++i) s.add(B[o * NI + i], x[i]);
    out[o * SO] = s.get();
  }
}

// out[o*SO] = sum_i B[i*NO + o] in[i*SI], o < NO   (transposed use of a NI x NO table)
template <typename T, int NI, int NO, int SI, int SO>
__device__ __forceinline__ void contractT(const T* __restrict__ in, T* __restrict__ out, const T* B) {
  T x[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) x[i] = in[i * SI];
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    Acc<T> s;
    s.init(B[o], x[0]);
#pragma unroll
    for (int i = 1; i < NI; ++i) s.add(B[i * NO + o], x[i]);
    out[o * SO] = s.get();
  }
}

// out[o*SO] = sum_i M[o][i] in[i*SI], o < NO, for a centrosymmetric NO x NI matrix M in
// its even-odd form P, N (see ElemTables): sums and differences of mirrored inputs, then
// each pair of mirrored outputs from one even and one odd partial sum. About half the
// multiply-adds of contract, and chains of at most ceil(NI / 2) terms.
template <typename T, int NI, int NO, int SI, int SO>
__device__ __forceinline__ void contract_eo(const T* __restrict__ in, T* __restrict__ out, const T* P, const T* N) {
  constexpr int EI = (NI + 1) / 2, HI = NI / 2, EO = (NO + 1) / 2, HO = NO / 2;
  T ev[EI], od[HI > 0 ? HI : 1];
#pragma unroll
  for (int i = 0; i < HI; ++i) {
    const T a = in[i * SI], b = in[(NI - 1 - i) * SI];
    ev[i] = a + b;
    od[i] = a - b;
  }
  if constexpr (NI % 2 == 1) ev[HI] = in[HI * SI];
#pragma unroll
  for (int o = 0; o < EO; ++o) {
    Acc<T> e;
    e.init(P[o * EI], ev[0]);
#pragma unroll
    for (int i = 1; i < EI; ++i) e.add(P[o * EI + i], ev[i]);
    if (o < HO) {
      Acc<T> d;
      d.init(N[o * HI], od[0]);
#pragma unroll
      for (int i = 1; i < HI; ++i) d.add(N[o * HI + i], od[i]);
      out[o * SO] = e.get() + d.get();
      out[(NO - 1 - o) * SO] = e.get() - d.get();
    } else {
      out[o * SO] = e.get();  // the middle output of an odd NO
    }
  }
}

template <int K, int Q>
struct Sizes {
  static constexpr int NX1 = (K + 1) * K * K;
  static constexpr int NRT = 3 * NX1;
  static constexpr int NL2 = K * K * K;
  static constexpr int NQ = Q * Q * Q;
  static constexpr int T1 = 3 * Q * K * (K + 1);
  static constexpr int UQ = 3 * NQ;
  static constexpr int R1 = (T1 > UQ ? T1 : UQ);   // T1 and the point values share a region
  static constexpr int R2 = 3 * Q * Q * (K + 1);  // T2
  static constexpr int PER_ELEM = NRT + NL2 + R1 + R2;
};

// global RT id and essential flag of local dof n of element (ex,ey,ez)
template <int K>
__device__ __forceinline__ int rt_global(const LatticeDims& L, int ex, int ey, int ez, int n, bool& ess) {
  constexpr int NX1 = (K + 1) * K * K;
  int I, J, Z;
  if (n < NX1) {
    int i = n % (K + 1), r = n / (K + 1);
    I = ex * K + i; J = ey * K + r % K; Z = ez * K + r / K;
    ess = (I == 0 && (L.ess & 1)) || (I == L.X && (L.ess & 2));
    return I + (L.X + 1) * (J + L.Y * Z);
  } else if (n < 2 * NX1) {
    int m = n - NX1;
    int i = m % K, r = m / K;
    I = ex * K + i; J = ey * K + r % (K + 1); Z = ez * K + r / (K + 1);
    ess = (J == 0 && (L.ess & 4)) || (J == L.Y && (L.ess & 8));
    return L.n_xf + I + L.X * (J + (L.Y + 1) * Z);
  } else {
    int m = n - 2 * NX1;
    int i = m % K, r = m / K;
    I = ex * K + i; J = ey * K + r % K; Z = ez * K + r / K;
    ess = (Z == 0 && (L.ess & 16)) || (Z == L.Z && (L.ess & 32));
    return L.n_xf + L.n_yf + I + L.X * (J + L.Y * Z);
  }
}

// own-cell part of (D^T q) at local face n (q: element-local L2 values)
template <typename T, int K>
__device__ __forceinline__ T dt_local(const T* sq, int n) {
  constexpr int NX1 = (K + 1) * K * K;
  T v = (T)0;
  if (n < NX1) {
    int i = n % (K + 1), r = n / (K + 1);  // r = j + K l
    if (i > 0) v += sq[(i - 1) + K * r];
    if (i < K) v -= sq[i + K * r];
  } else if (n < 2 * NX1) {
    int m = n - NX1;
    int i = m % K, r = m / K;
    int j = r % (K + 1), l = r / (K + 1);
    if (j > 0) v += sq[i + K * ((j - 1) + K * l)];
    if (j < K) v -= sq[i + K * (j + K * l)];
  } else {
    int m = n - 2 * NX1;
    int i = m % K, r = m / K;
    int j = r % K, l = r / K;
    if (l > 0) v += sq[i + K * (j + K * (l - 1))];
    if (l < K) v -= sq[i + K * (j + K * l)];
  }
  return v;
}

// (D u)_cell for local cell a = i + K (j + K l) from the element-local RT values
template <typename T, int K>
__device__ __forceinline__ T div_local(const T* su, int a) {
  constexpr int NX1 = (K + 1) * K * K;
  int i = a % K, j = (a / K) % K, l = a / (K * K);
  T v = su[(i + 1) + (K + 1) * (j + K * l)] - su[i + (K + 1) * (j + K * l)];
  v += su[NX1 + i + K * ((j + 1) + (K + 1) * l)] - su[NX1 + i + K * (j + (K + 1) * l)];
  v += su[2 * NX1 + i + K * (j + K * (l + 1))] - su[2 * NX1 + i + K * (j + K * l)];
  return v;
}

// ---------------------------------------------------------------------------
// Per-element 3D application of the K x K map TT (or its transpose) to EB
// element-local L2 vectors: in -> t1 -> t2 -> out, one direction per stage.
template <typename T, int K, int EB, bool TRANS>
__device__ __forceinline__ void apply_tt(const TabT<T>& tab, const T* in, int in_stride, T* t1, T* t2, T* out,
                                         int buf_stride, int out_stride) {
  constexpr int KK = K * K;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int t = tid; t < EB * KK; t += nth) {  // x: lines (m2, m3)
    int el = t / KK, r = t - el * KK;
    if (TRANS) contractT<T, K, K, 1, 1>(in + el * in_stride + K * r, t1 + el * buf_stride + K * r, tab.TT);
    else contract<T, K, K, 1, 1>(in + el * in_stride + K * r, t1 + el * buf_stride + K * r, tab.TT);
  }
  __syncthreads();
  for (int t = tid; t < EB * KK; t += nth) {  // y: lines (i1, m3)
    int el = t / KK, r = t - el * KK, i1 = r % K, m3 = r / K;
    if (TRANS) contractT<T, K, K, K, K>(t1 + el * buf_stride + i1 + KK * m3, t2 + el * buf_stride + i1 + KK * m3, tab.TT);
    else contract<T, K, K, K, K>(t1 + el * buf_stride + i1 + KK * m3, t2 + el * buf_stride + i1 + KK * m3, tab.TT);
  }
  __syncthreads();
  for (int t = tid; t < EB * KK; t += nth) {  // z: lines (i1, i2)
    int el = t / KK, r = t - el * KK;
    if (TRANS) contractT<T, K, K, KK, KK>(t2 + el * buf_stride + r, out + el * out_stride + r, tab.TT);
    else contract<T, K, K, KK, KK>(t2 + el * buf_stride + r, out + el * out_stride + r, tab.TT);
  }
  __syncthreads();
}

// w = W p for EB elements in the GL nodal basis (GLB: tables BG) or the
// histopolation basis (tables BH): basis -> quadrature points (three stages),
// times w_p / det J, and back (three transposed stages). Scratch s1.
template <typename T, int K, int Q, int EB, bool GLB>
__device__ __forceinline__ void apply_wgl(const TabT<T>& tab, const T* p, int vstride, T* w, T* s1, int s1stride,
                                          const T* __restrict__ wdet, int e0, int n_elem) {
  constexpr int KK = K * K, NQ = Q * Q * Q;
  const int tid = threadIdx.x, nth = blockDim.x;
  const T* B = GLB ? tab.BG : tab.BH;
  T* t1b = s1;                       // [Q K K]
  T* t2b = s1 + Q * KK;              // [Q Q K]
  T* vb = s1 + Q * KK + Q * Q * K;   // [Q^3]
  for (int t = tid; t < EB * KK; t += nth) {
    int el = t / KK, r = t - el * KK;
    contract<T, K, Q, 1, 1>(p + el * vstride + K * r, t1b + el * s1stride + Q * r, B);
  }
  __syncthreads();
  for (int t = tid; t < EB * Q * K; t += nth) {
    int el = t / (Q * K), r = t - el * Q * K, px = r % Q, m3 = r / Q;
    contract<T, K, Q, Q, Q>(t1b + el * s1stride + px + Q * K * m3, t2b + el * s1stride + px + Q * Q * m3, B);
  }
  __syncthreads();
  for (int t = tid; t < EB * Q * Q; t += nth) {
    int el = t / (Q * Q), r = t - el * Q * Q;
    contract<T, K, Q, Q * Q, Q * Q>(t2b + el * s1stride + r, vb + el * s1stride + r, B);
  }
  __syncthreads();
  for (int t = tid; t < EB * NQ; t += nth) {
    int el = t / NQ, pt = t - el * NQ, e = e0 + el;
    vb[el * s1stride + pt] *= (e < n_elem) ? wdet[(size_t)e * NQ + pt] : (T)0;
  }
  __syncthreads();
  for (int t = tid; t < EB * Q * Q; t += nth) {
    int el = t / (Q * Q), r = t - el * Q * Q;
    contractT<T, Q, K, Q * Q, Q * Q>(vb + el * s1stride + r, t2b + el * s1stride + r, B);
  }
  __syncthreads();
  for (int t = tid; t < EB * Q * K; t += nth) {
    int el = t / (Q * K), r = t - el * Q * K, px = r % Q, m3 = r / Q;
    contractT<T, Q, K, Q, Q>(t2b + el * s1stride + px + Q * Q * m3, t1b + el * s1stride + px + Q * K * m3, B);
  }
  __syncthreads();
  for (int t = tid; t < EB * KK; t += nth) {
    int el = t / KK, r = t - el * KK;
    contractT<T, Q, K, 1, 1>(t1b + el * s1stride + Q * r, w + el * vstride + K * r, B);
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// W_e^-1 q_e for EB elements by the local CG of Sec. 2.5: b = TT^T q (GL nodal
// right-hand side), Jacobi-preconditioned CG on W_GL from a = 0, result TT a in
// s1 (returned). GLB = false: the same CG on W in the histopolation basis itself
// (b = q, result a; the comparison of the two bases in Sec. 3.1). One warp per
// element for the vector operations; the loop runs until every element of the
// CTA meets its tolerance or maxit is reached.
template <typename T, int K, int Q, int EB, bool GLB>
__device__ T* local_cg(const TabT<T>& tab, const T* sq, T* s1, int s1stride, T* s2, int s2stride,
                       const CgArgs<T>& cg, int e0, int n_elem) {
  constexpr int NL2 = K * K * K;
  __shared__ T sc_rz[EB], sc_bb[EB];
  __shared__ int sc_active[EB];
  __shared__ int sc_any;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // per element in s2: a, r, p, w (NL2 each)
  T* A = s2;
  T* R = s2 + NL2;
  T* P = s2 + 2 * NL2;
  T* W = s2 + 3 * NL2;
  if (GLB) {
    apply_tt<T, K, EB, true>(tab, sq, NL2, s1, s1 + NL2, R, s1stride, s2stride);  // r = b = TT^T q
  } else {
    for (int t = threadIdx.x; t < EB * NL2; t += blockDim.x) R[(t / NL2) * s2stride + t % NL2] = sq[t];
    __syncthreads();
  }
  for (int el = warp; el < EB; el += nw) {
    const int e = e0 + el;
    const T* D = cg.diag + (size_t)(e < n_elem ? e : 0) * NL2;
    T rz = 0, bb = 0;
    for (int i = lane; i < NL2; i += 32) {
      T r = R[el * s2stride + i];
      T z = (e < n_elem) ? r / D[i] : (T)0;
      A[el * s2stride + i] = 0;
      P[el * s2stride + i] = z;
      rz += r * z;
      bb += r * r;
    }
    rz = warp_allsum(rz);
    bb = warp_allsum(bb);
    if (lane == 0) {
      sc_rz[el] = rz;
      sc_bb[el] = bb;
      sc_active[el] = (e < n_elem) && (bb > (T)0);
    }
  }
  __syncthreads();
  for (int it = 0; it < cg.maxit; ++it) {
    apply_wgl<T, K, Q, EB, GLB>(tab, P, s2stride, W, s1, s1stride, cg.wdet, e0, n_elem);
    for (int el = warp; el < EB; el += nw) {
      if (!sc_active[el]) continue;
      T pw = 0;
      for (int i = lane; i < NL2; i += 32) pw += P[el * s2stride + i] * W[el * s2stride + i];
      pw = warp_allsum(pw);
      const T alpha = sc_rz[el] / pw;
      T rr = 0;
      for (int i = lane; i < NL2; i += 32) {
        A[el * s2stride + i] += alpha * P[el * s2stride + i];
        T r = R[el * s2stride + i] - alpha * W[el * s2stride + i];
        R[el * s2stride + i] = r;
        rr += r * r;
      }
      rr = warp_allsum(rr);
      __syncwarp();
      if (lane == 0) sc_active[el] = (rr > cg.tol2 * sc_bb[el]) && (pw > (T)0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int el = 0; el < EB; ++el) any |= sc_active[el];
      sc_any = any;
    }
    __syncthreads();
    if (!sc_any) break;
    for (int el = warp; el < EB; el += nw) {
      if (!sc_active[el]) continue;
      const T* D = cg.diag + (size_t)(e0 + el) * NL2;
      T rz = 0;
      for (int i = lane; i < NL2; i += 32) {
        T z = R[el * s2stride + i] / D[i];
        W[el * s2stride + i] = z;
        rz += R[el * s2stride + i] * z;
      }
      rz = warp_allsum(rz);
      const T beta = rz / sc_rz[el];
      for (int i = lane; i < NL2; i += 32) P[el * s2stride + i] = W[el * s2stride + i] + beta * P[el * s2stride + i];
      __syncwarp();
      if (lane == 0) sc_rz[el] = rz;
    }
    __syncthreads();
  }
  T* out = s1 + 2 * NL2;
  if (GLB) {
    apply_tt<T, K, EB, false>(tab, A, s2stride, s1, s1 + NL2, out, s1stride, s1stride);  // TT a
  } else {
    for (int t = threadIdx.x; t < EB * NL2; t += blockDim.x)
      out[(t / NL2) * s1stride + t % NL2] = A[(t / NL2) * s2stride + t % NL2];
    __syncthreads();
  }
  return out;
}

// W_e^-1 q_e for EB elements by the Cholesky factor of W_e (the factorisation
// approach of Sec. 3.1: W_e = L L^T stored [NL2][NL2] row-major, zero above the
// diagonal, the diagonal entries stored as their reciprocals). One warp per
// element: forward L y = q by rows (a warp sum per row), back L^T z = y by the
// columns of L^T, which are the rows of L (an axpy per step): every read of L is a
// contiguous row. Result in s1 (returned).
template <typename T, int K, int EB>
__device__ T* local_chol(const T* __restrict__ Lg, const T* sq, T* s1, int s1stride, int e0, int n_elem) {
  constexpr int NL2 = K * K * K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int el = warp; el < EB; el += nw) {
    const int e = e0 + el;
    T* y = s1 + el * s1stride;
    for (int i = lane; i < NL2; i += 32) y[i] = sq[el * NL2 + i];
    __syncwarp();
    if (e >= n_elem) continue;
    const T* L = Lg + (size_t)e * NL2 * NL2;
    for (int i = 0; i < NL2; ++i) {
      T sum = (T)0;
      for (int j = lane; j < i; j += 32) sum = fma(L[i * NL2 + j], y[j], sum);
      sum = warp_allsum(sum);
      const T yi = (y[i] - sum) * L[i * NL2 + i];
      __syncwarp();
      if (lane == 0) y[i] = yi;
      __syncwarp();
    }
    for (int i = NL2 - 1; i >= 0; --i) {
      const T zi = y[i] * L[i * NL2 + i];
      __syncwarp();
      if (lane == 0) y[i] = zi;
      for (int j = lane; j < i; j += 32) y[j] = fma(-L[i * NL2 + j], zi, y[j]);
      __syncwarp();
    }
  }
  __syncthreads();
  return s1;
}

// ---------------------------------------------------------------------------
// Fused block-operator kernel: EB elements per CTA.
//   OP_M : y_u += M_e u_e (sum factorisation: interpolation to the Q^3 points,
//          the 3x3 geometric factor, transposed interpolation)
//   OP_DT: y_u += own-cell D^T q
//   OP_D : y_q  = D u on the element's cells
//   OP_C : y_q -= c_e W_e^-1 q  (OP_CPOS: +)
// AFF (affine meshes, q = k+1): Ga[e][8] holds b_e J^T J / det J (6 entries) and
// det J; the point factor is w_p times that matrix, and W_e^-1 q = det J
// (H^-1 x H^-1 x H^-1) q by three K x K contractions, so the kernel reads 64 B of
// element data instead of 8 (6 Q^3 + K^6) B.
// Essential faces: with OP_M the owning element adds u_g (constrained
// identity); otherwise nothing. y_u receives one atomic add per element and
// face: a shared face gets exactly two addends on a zeroed vector, so the
// result does not depend on their order.
// Launch configuration per arithmetic type (elements per CTA, threads per CTA),
// measured on GB300 at k = 4: FP64 is bound by its pipe and prefers 8/256;
// double-float is latency-bound and gains from more resident warps (8/512);
// FP32 is HBM-bound and prefers 4/256. The HD_*_EB / HD_*_THREADS macros
// override them for tuning builds.
#ifndef HD_F64_EB
#define HD_F64_EB 8
#endif
#ifndef HD_F64_THREADS
#define HD_F64_THREADS 256
#endif
#ifndef HD_DF_EB
#define HD_DF_EB 8
#endif
#ifndef HD_DF_THREADS
#define HD_DF_THREADS 512
#endif
#ifndef HD_F32_EB
#define HD_F32_EB 4
#endif
#ifndef HD_F32_THREADS
#define HD_F32_THREADS 256
#endif
#ifndef HD_F64_PREFETCH
#define HD_F64_PREFETCH 0
#endif
#ifndef HD_DF_PREFETCH
#define HD_DF_PREFETCH 0
#endif
#ifndef HD_F32_PREFETCH
#define HD_F32_PREFETCH 3
#endif
// PREFETCH: bit 1 asks the copy engine to stage the CTA's contiguous G block,
// bit 2 its W^-1 block, in L2 as the CTA starts (cp.async.bulk.prefetch). The
// HBM-bound FP32 kernel gains about 10 % at k = 4; the FP64 and double-float
// kernels, whose loads already overlap their arithmetic, lose.
#ifndef HD_DFA_EB
#define HD_DFA_EB 8
#endif
#ifndef HD_DFA_THREADS
#define HD_DFA_THREADS 512
#endif
// The W_e^-1 rows read from global memory (one thread per row): the unrolled batch sets the
// loads in flight per thread (ElemCfg::WINV_UNROLL). Measured at 64^3, k = 4: double-float
// kernel 8 -> 3.69 ms, 16 -> 3.60, 32 -> 3.58, 64 -> 3.67; two or four partial sums per row
// instead of one chain: 3.93 and 4.30 ms (the chain is not the limit, the load latency is).
// The FP32 kernel, bound by HBM, keeps 8 (1.44 ms, 1.46 with 32); FP64 is the same either way.
#ifndef HD_WINV_UNROLL
#define HD_WINV_UNROLL 32
#endif
// POINTS: quadrature points per thread and pass of the pointwise stage, whose geometric
// factors are all loaded before any is used (more loads in flight). Double-float kernel at
// 64^3, k = 4: 1 -> 3.58 ms, 3 -> 3.44, 4 -> 3.48 (two, written as a pair of named points:
// 3.44; as the loop below: 3.79, where the compiler kept fewer loads in flight). The same
// batching of the gather of u (3 or 5 loads per pass) measured 3.46 ms, and 1.55 against
// 1.46 ms for the FP32 kernel: not kept.
#ifndef HD_DF_POINTS
#define HD_DF_POINTS 3
#endif

template <typename T, bool AFF = false>
struct ElemCfg {
  static constexpr int EB = HD_F64_EB, THREADS = HD_F64_THREADS, PREFETCH = HD_F64_PREFETCH, POINTS = 1,
                       WINV_UNROLL = HD_WINV_UNROLL;
};
template <>
struct ElemCfg<dfloat, false> {
  static constexpr int EB = HD_DF_EB, THREADS = HD_DF_THREADS, PREFETCH = HD_DF_PREFETCH, POINTS = HD_DF_POINTS,
                       WINV_UNROLL = HD_WINV_UNROLL;
};
template <>
struct ElemCfg<dfloat, true> {  // the affine fast path (no per-element arrays to stream)
  static constexpr int EB = HD_DFA_EB, THREADS = HD_DFA_THREADS, PREFETCH = 0, POINTS = 1, WINV_UNROLL = 8;
};
template <>
struct ElemCfg<float, false> {
  static constexpr int EB = HD_F32_EB, THREADS = HD_F32_THREADS, PREFETCH = HD_F32_PREFETCH, POINTS = 1,
                       WINV_UNROLL = 8;
};

// Staging of the dense W_e^-1 rows by the copy engine (double-float kernel): the
// sum-factorisation buffers T1/T2 are idle while the L2 rows are computed, so they
// hold two buffers of NB rows of W_e^-1 for each element of the CTA. One thread asks
// for a chunk with one bulk copy per element (cp.async.bulk, completion counted on
// the buffer's mbarrier), the first two before the gather; the rows' threads then
// read W from shared memory instead of waiting on HBM loads. Needs an even NL2 (the
// per-element blocks and chunks start on 16-byte boundaries) and one thread per row.
#ifndef HD_DF_STAGE
#define HD_DF_STAGE 0
#endif
template <typename T, int K, int Q, int EB, bool AFF>
struct StageW {
  using S = Sizes<K, Q>;
  static constexpr int NL2 = S::NL2;
  static constexpr int FIT = EB * (S::R1 + S::R2) / (2 * EB * NL2);  // rows per buffer that fit
  static constexpr int NB = FIT >= NL2 ? NL2 : FIT >= 32 ? 32 : FIT >= 16 ? 16 : FIT >= 8 ? 8 : FIT >= 4 ? 4 : 2;
  static constexpr bool ON = HD_DF_STAGE != 0 && std::is_same<T, dfloat>::value && !AFF && NL2 % 2 == 0 &&
                             NL2 % NB == 0 && FIT >= 2 && EB * NL2 <= ElemCfg<T, AFF>::THREADS;
  static constexpr int NCH = NL2 / NB;
  static constexpr int BAR_BYTES = ON ? 16 : 0;
};

// L2 prefetch of [p, p + bytes) in 16 KB pieces, one piece per lane; the range
// is trimmed to whole 16-byte units and skipped when p is not 16-byte aligned.
__device__ __forceinline__ void prefetch_l2_block(const void* p, size_t bytes, int lane) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if (a & 15) return;
  bytes &= ~(size_t)15;
  constexpr size_t CH = 16384;
  for (size_t off = (size_t)lane * CH; off < bytes; off += 32 * CH) {
    const uint32_t sz = (uint32_t)(bytes - off < CH ? bytes - off : CH);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a + off), "r"(sz) : "memory");
  }
}

template <typename T, typename IO, int K, int Q, int EB, bool AFF = false>
__global__ void __launch_bounds__(ElemCfg<T, AFF>::THREADS)
k_elem_op(const TabT<T> tab, const LatticeDims L, const int mode, const int n_elem, const int e_first,
          const T* __restrict__ G, const T* __restrict__ winv, const T* __restrict__ cscale,
          const CgArgs<T> cg, const IO* __restrict__ u, const IO* __restrict__ q, IO* __restrict__ yu,
          IO* __restrict__ yq, const T* __restrict__ Ga) {
  using S = Sizes<K, Q>;
  constexpr int NX1 = S::NX1, NRT = S::NRT, NL2 = S::NL2, NQ = S::NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* su = sm;                         // [EB][NRT]  u_e, later y_e
  T* sq = su + EB * NRT;              // [EB][NL2]
  T* s1 = sq + EB * NL2;              // [EB][R1]   T1 / point values
  T* s2 = s1 + EB * S::R1;            // [EB][R2]   T2
  const int e0 = e_first + blockIdx.x * EB;  // elements [e_first, n_elem) of this launch
  const int tid = threadIdx.x, nth = blockDim.x;
  const bool needu = (mode & (OP_M | OP_D)) != 0;
  const bool needq = (mode & (OP_DT | OP_C)) != 0;
  const bool use_cg = !AFF && (mode & OP_C) && cg.wdet != nullptr;
  const bool use_chol = !AFF && (mode & OP_C) && !use_cg && cg.chol != 0;
  using SW = StageW<T, K, Q, EB, AFF>;
  [[maybe_unused]] const bool stage_w = SW::ON && (mode & OP_C) && !use_cg && !use_chol;
  [[maybe_unused]] uint64_t* wbar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)EB * S::PER_ELEM * sizeof(T));
  [[maybe_unused]] const int ne_cta = (n_elem - e0 < EB) ? n_elem - e0 : EB;
  // chunk c (rows [c NB, (c + 1) NB) of every element's W_e^-1) into buffer c & 1
  [[maybe_unused]] auto w_issue = [&](int c) {
    T* buf = s1 + (c & 1) * (EB * SW::NB * NL2);
    const uint32_t bar = tc::smem_u32(&wbar[c & 1]);
    tc::mbar_arrive_expect_tx(bar, (uint32_t)(ne_cta * SW::NB * NL2 * sizeof(T)));
    for (int el = 0; el < ne_cta; ++el)
      tc::bulk_g2s(tc::smem_u32(buf + el * SW::NB * NL2),
                   winv + ((size_t)(e0 + el) * NL2 + (size_t)c * SW::NB) * NL2, SW::NB * NL2 * sizeof(T), bar);
  };
  if constexpr (SW::ON) {
    if (stage_w && tid == 0) {  // the barrier after the gather publishes the initialisation
      tc::mbar_init(tc::smem_u32(&wbar[0]), 1);
      tc::mbar_init(tc::smem_u32(&wbar[1]), 1);
      tc::fence_mbar_init();
      w_issue(0);
      if (SW::NCH > 1) w_issue(1);
    }
  }
  if constexpr (ElemCfg<T, AFF>::PREFETCH != 0) {
    if (tid < 32 && e0 < n_elem) {
      const int ne = (n_elem - e0 < EB) ? n_elem - e0 : EB;
      if ((ElemCfg<T, AFF>::PREFETCH & 1) && (mode & OP_M))
        prefetch_l2_block(G + (size_t)e0 * 6 * NQ, (size_t)ne * 6 * NQ * sizeof(T), tid);
      if ((ElemCfg<T, AFF>::PREFETCH & 2) && (mode & OP_C) && !use_cg)
        prefetch_l2_block(winv + (size_t)e0 * NL2 * NL2, (size_t)ne * NL2 * NL2 * sizeof(T), tid);
    }
  }

  // -- gather -----------------------------------------------------------------
  if (needu) {
    for (int t = tid; t < EB * NRT; t += nth) {
      int el = t / NRT, n = t - el * NRT, e = e0 + el;
      T v = (T)0;
      if (e < n_elem) {
        int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
        bool ess;
        int g = rt_global<K>(L, ex, ey, ez, n, ess);
        v = ess ? (T)0 : Cvt<T, IO>::in(u[g]);
      }
      su[t] = v;
    }
  }
  if (needq) {
    for (int t = tid; t < EB * NL2; t += nth) {
      int el = t / NL2, a = t - el * NL2, e = e0 + el;
      T v = (T)0;
      if (e < n_elem) {
        int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
        int i = a % K, j = (a / K) % K, l = a / (K * K);
        v = Cvt<T, IO>::in(q[(ex * K + i) + L.X * ((ey * K + j) + L.Y * (ez * K + l))]);
      }
      sq[t] = v;
    }
  }
  __syncthreads();

  // -- L2 rows: y_q = D u - C q ------------------------------------------------
  const T* cgres = nullptr;
  if constexpr (!std::is_same<T, dfloat>::value && !AFF) {
    if (use_cg) {
      if constexpr (std::is_same<T, double>::value)  // the histopolation-basis CG: FP64 only
        if (cg.hist) cgres = local_cg<T, K, Q, EB, false>(tab, sq, s1, S::R1, s2, S::R2, cg, e0, n_elem);
      if (!cgres) cgres = local_cg<T, K, Q, EB, true>(tab, sq, s1, S::R1, s2, S::R2, cg, e0, n_elem);
    }
    if constexpr (std::is_same<T, double>::value)  // the Cholesky factor: FP64 only
      if (use_chol) cgres = local_chol<T, K, EB>(winv, sq, s1, S::R1, e0, n_elem);
  }
  if constexpr (AFF) {
    if (mode & OP_C) {  // H^-1 along x (sq -> s1), y (s1 -> s2), z (s2 -> s1)
      constexpr int KK = K * K;
      for (int t = tid; t < EB * KK; t += nth) {
        const int el = t / KK, r = t - el * KK;
        contract<T, K, K, 1, 1>(sq + el * NL2 + K * r, s1 + el * S::R1 + K * r, tab.HI);
      }
      __syncthreads();
      for (int t = tid; t < EB * KK; t += nth) {
        const int el = t / KK, r = t - el * KK, i = r % K, l = r / K;
        contract<T, K, K, K, K>(s1 + el * S::R1 + i + KK * l, s2 + el * S::R2 + i + KK * l, tab.HI);
      }
      __syncthreads();
      for (int t = tid; t < EB * KK; t += nth) {
        const int el = t / KK, r = t - el * KK;
        contract<T, K, K, KK, KK>(s2 + el * S::R2 + r, s1 + el * S::R1 + r, tab.HI);
      }
      __syncthreads();
    }
  }
  // one L2 row (element-local cell t), given its D u part v
  auto l2_row = [&](int t, T v) {
    const int el = t / NL2, a = t - el * NL2, e = e0 + el;
    if (mode & OP_C) {
      T s = (T)0;
      if constexpr (AFF) {
        s = s1[el * S::R1 + a] * Ga[(size_t)e * 8 + 6];
      } else if (use_cg || use_chol) {
        s = cgres[el * S::R1 + a];
      } else {
        const T* W = winv + (size_t)e * NL2 * NL2;
        const T* qe = sq + el * NL2;
        Acc<T> acc;
        acc.init(W[a], qe[0]);
#pragma unroll ElemCfg<T, AFF>::WINV_UNROLL
        for (int b = 1; b < NL2; ++b) acc.add(W[b * NL2 + a], qe[b]);
        s = acc.get();
      }
      s *= cscale[e];
      v = (mode & OP_CPOS) ? v + s : v - s;
    }
    int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
    int i = a % K, j = (a / K) % K, l = a / (K * K);
    yq[(ex * K + i) + L.X * ((ey * K + j) + L.Y * (ez * K + l))] = Cvt<T, IO>::out(v);
  };
  bool rows_done = false;
  if constexpr (SW::ON) {
    if (stage_w) {  // the rows from the staged chunks (one thread per row)
      const int el = tid / NL2, a = tid - el * NL2;
      const bool mine = tid < EB * NL2 && el < ne_cta;
      const T* qe = sq + el * NL2;
      Acc<T> acc;
      for (int c = 0; c < SW::NCH; ++c) {
        if (mine) {
          if (!tc::mbar_wait(tc::smem_u32(&wbar[c & 1]), (uint32_t)((c >> 1) & 1)) && cg.err) atomicOr(cg.err, 2);
          const T* Wc = s1 + (c & 1) * (EB * SW::NB * NL2) + el * SW::NB * NL2 + a;
          if (c == 0) {
            acc.init(Wc[0], qe[0]);
#pragma unroll
            for (int bb = 1; bb < SW::NB; ++bb) acc.add(Wc[bb * NL2], qe[bb]);
          } else {
#pragma unroll
            for (int bb = 0; bb < SW::NB; ++bb) acc.add(Wc[bb * NL2], qe[c * SW::NB + bb]);
          }
        }
        if (SW::NCH > 2) {  // buffer c & 1 takes chunk c + 2 once every row has read it
          __syncthreads();
          if (tid == 0 && c + 2 < SW::NCH) {
            tc::fence_proxy_async_smem();
            w_issue(c + 2);
          }
        }
      }
      if (mine) {
        const int e = e0 + el;
        T v = (mode & OP_D) ? div_local<T, K>(su + el * NRT, a) : (T)0;
        const T s = acc.get() * cscale[e];
        v = (mode & OP_CPOS) ? v + s : v - s;
        const int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
        const int i = a % K, j = (a / K) % K, l = a / (K * K);
        yq[(ex * K + i) + L.X * ((ey * K + j) + L.Y * (ez * K + l))] = Cvt<T, IO>::out(v);
      }
      rows_done = true;
    }
  }
  if ((mode & (OP_D | OP_C)) && !rows_done) {
    for (int t = tid; t < EB * NL2; t += nth) {
      if (e0 + t / NL2 >= n_elem) continue;
      l2_row(t, (mode & OP_D) ? div_local<T, K>(su + (t / NL2) * NRT, t % NL2) : (T)0);
    }
  }
  if (use_cg || use_chol || rows_done || (AFF && (mode & OP_C))) __syncthreads();

  if (mode & OP_M) {
    // -- interpolation to the points: stage A (contract along x) ----------------
    {
      constexpr int LX = K * K, LY = (K + 1) * K, LZ = K * (K + 1);
      for (int t = tid; t < EB * (LX + LY + LZ); t += nth) {
        if (t < EB * LX) {
          int el = t / LX, r = t - el * LX;  // r = j + K l
          contract_eo<T, K + 1, Q, 1, 1>(su + el * NRT + (K + 1) * r, s1 + el * S::R1 + Q * r, tab.BIp, tab.BIn);
        } else if (t < EB * (LX + LY)) {
          int tt = t - EB * LX, el = tt / LY, r = tt - el * LY;  // r = j + (K+1) l
          contract_eo<T, K, Q, 1, 1>(su + el * NRT + NX1 + K * r, s1 + el * S::R1 + Q * K * K + Q * r, tab.BHp, tab.BHn);
        } else {
          int tt = t - EB * (LX + LY), el = tt / LZ, r = tt - el * LZ;  // r = j + K l
          contract_eo<T, K, Q, 1, 1>(su + el * NRT + 2 * NX1 + K * r,
                                  s1 + el * S::R1 + Q * K * K + Q * (K + 1) * K + Q * r, tab.BHp, tab.BHn);
        }
      }
    }
    __syncthreads();
    // stage B (contract along y): T2[px + Q (py + Q l)]
    {
      constexpr int LX = Q * K, LY = Q * K, LZ = Q * (K + 1);
      for (int t = tid; t < EB * (LX + LY + LZ); t += nth) {
        if (t < EB * LX) {
          int el = t / LX, r = t - el * LX, px = r % Q, l = r / Q;
          contract_eo<T, K, Q, Q, Q>(s1 + el * S::R1 + px + Q * K * l, s2 + el * S::R2 + px + Q * Q * l, tab.BHp, tab.BHn);
        } else if (t < EB * (LX + LY)) {
          int tt = t - EB * LX, el = tt / LY, r = tt - el * LY, px = r % Q, l = r / Q;
          contract_eo<T, K + 1, Q, Q, Q>(s1 + el * S::R1 + Q * K * K + px + Q * (K + 1) * l,
                                      s2 + el * S::R2 + Q * Q * K + px + Q * Q * l, tab.BIp, tab.BIn);
        } else {
          int tt = t - EB * (LX + LY), el = tt / LZ, r = tt - el * LZ, px = r % Q, l = r / Q;
          contract_eo<T, K, Q, Q, Q>(s1 + el * S::R1 + Q * K * K + Q * (K + 1) * K + px + Q * K * l,
                                  s2 + el * S::R2 + 2 * Q * Q * K + px + Q * Q * l, tab.BHp, tab.BHn);
        }
      }
    }
    __syncthreads();
    // stage C (contract along z): point values U_c[px + Q (py + Q pz)] in s1
    {
      constexpr int LL = Q * Q;
      for (int t = tid; t < EB * 3 * LL; t += nth) {
        int c = t / (EB * LL), tt = t - c * EB * LL, el = tt / LL, r = tt - el * LL;
        T* out = s1 + el * S::R1 + c * NQ + r;
        const T* in = s2 + el * S::R2 + c * Q * Q * K + r;
        if (c == 2)
          contract_eo<T, K + 1, Q, Q * Q, Q * Q>(in, out, tab.BIp, tab.BIn);
        else
          contract_eo<T, K, Q, Q * Q, Q * Q>(in, out, tab.BHp, tab.BHn);
      }
    }
    __syncthreads();
    // -- pointwise: v = G u --------------------------------------------------------
    // NPT points per pass (see ElemCfg); from k = 4 on, where shared memory already keeps
    // two CTAs per SM and the extra registers cost no occupancy
    if constexpr (!AFF && ElemCfg<T, AFF>::POINTS > 1 && K >= 4) {
      constexpr int NPT = ElemCfg<T, AFF>::POINTS;
      auto point = [&](T* U, const T* gg) {
        const T ux = U[0], uy = U[NQ], uz = U[2 * NQ];
        Acc<T> v0, v1, v2;
        v0.init(gg[2], uz); v0.add(gg[1], uy); v0.add(gg[0], ux);
        v1.init(gg[4], uz); v1.add(gg[3], uy); v1.add(gg[1], ux);
        v2.init(gg[5], uz); v2.add(gg[4], uy); v2.add(gg[2], ux);
        U[0] = v0.get();
        U[NQ] = v1.get();
        U[2 * NQ] = v2.get();
      };
      for (int t = tid; t < EB * NQ; t += NPT * nth) {
        T gv[NPT][6];
        int off[NPT];
        bool okv[NPT];
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
          const int tj = t + j * nth, el = tj / NQ, p = tj - el * NQ, e = e0 + el;
          okv[j] = tj < EB * NQ && e < n_elem;
          off[j] = el * S::R1 + p;
          const T* g = G + (size_t)(okv[j] ? e : 0) * 6 * NQ + (okv[j] ? p : 0);
#pragma unroll
          for (int c = 0; c < 6; ++c) gv[j][c] = g[c * NQ];
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j)
          if (okv[j]) point(s1 + off[j], gv[j]);
      }
    } else {
      for (int t = tid; t < EB * NQ; t += nth) {
        int el = t / NQ, p = t - el * NQ, e = e0 + el;
        if (e >= n_elem) continue;
        T g00, g01, g02, g11, g12, g22;
        T* U = s1 + el * S::R1 + p;
        T ux = U[0], uy = U[NQ], uz = U[2 * NQ];
        if constexpr (AFF) {
          const T* g = Ga + (size_t)e * 8;
          g00 = g[0]; g01 = g[1]; g02 = g[2]; g11 = g[3]; g12 = g[4]; g22 = g[5];
          const int px = p % Q, py = (p / Q) % Q, pz = p / (Q * Q);
          const T w = tab.GW[px] * tab.GW[py] * tab.GW[pz];
          ux = ux * w; uy = uy * w; uz = uz * w;
        } else {
          const T* g = G + (size_t)e * 6 * NQ + p;
          g00 = g[0]; g01 = g[NQ]; g02 = g[2 * NQ]; g11 = g[3 * NQ]; g12 = g[4 * NQ]; g22 = g[5 * NQ];
        }
        Acc<T> v0, v1, v2;
        v0.init(g02, uz); v0.add(g01, uy); v0.add(g00, ux);
        v1.init(g12, uz); v1.add(g11, uy); v1.add(g01, ux);
        v2.init(g22, uz); v2.add(g12, uy); v2.add(g02, ux);
        U[0] = v0.get();
        U[NQ] = v1.get();
        U[2 * NQ] = v2.get();
      }
    }
    __syncthreads();
    // -- transposed interpolation: stage C^T (z) -------------------------------
    {
      constexpr int LL = Q * Q;
      for (int t = tid; t < EB * 3 * LL; t += nth) {
        int c = t / (EB * LL), tt = t - c * EB * LL, el = tt / LL, r = tt - el * LL;
        const T* in = s1 + el * S::R1 + c * NQ + r;
        T* out = s2 + el * S::R2 + c * Q * Q * K + r;
        if (c == 2)
          contract_eo<T, Q, K + 1, Q * Q, Q * Q>(in, out, tab.BITp, tab.BITn);
        else
          contract_eo<T, Q, K, Q * Q, Q * Q>(in, out, tab.BHTp, tab.BHTn);
      }
    }
    __syncthreads();
    // stage B^T (y): T1 from T2
    {
      constexpr int LX = Q * K, LY = Q * K, LZ = Q * (K + 1);
      for (int t = tid; t < EB * (LX + LY + LZ); t += nth) {
        if (t < EB * LX) {
          int el = t / LX, r = t - el * LX, px = r % Q, l = r / Q;
          contract_eo<T, Q, K, Q, Q>(s2 + el * S::R2 + px + Q * Q * l, s1 + el * S::R1 + px + Q * K * l, tab.BHTp, tab.BHTn);
        } else if (t < EB * (LX + LY)) {
          int tt = t - EB * LX, el = tt / LY, r = tt - el * LY, px = r % Q, l = r / Q;
          contract_eo<T, Q, K + 1, Q, Q>(s2 + el * S::R2 + Q * Q * K + px + Q * Q * l,
                                       s1 + el * S::R1 + Q * K * K + px + Q * (K + 1) * l, tab.BITp, tab.BITn);
        } else {
          int tt = t - EB * (LX + LY), el = tt / LZ, r = tt - el * LZ, px = r % Q, l = r / Q;
          contract_eo<T, Q, K, Q, Q>(s2 + el * S::R2 + 2 * Q * Q * K + px + Q * Q * l,
                                   s1 + el * S::R1 + Q * K * K + Q * (K + 1) * K + px + Q * K * l, tab.BHTp, tab.BHTn);
        }
      }
    }
    __syncthreads();
    // stage A^T (x): y_e into su
    {
      constexpr int LX = K * K, LY = (K + 1) * K, LZ = K * (K + 1);
      for (int t = tid; t < EB * (LX + LY + LZ); t += nth) {
        if (t < EB * LX) {
          int el = t / LX, r = t - el * LX;
          contract_eo<T, Q, K + 1, 1, 1>(s1 + el * S::R1 + Q * r, su + el * NRT + (K + 1) * r, tab.BITp, tab.BITn);
        } else if (t < EB * (LX + LY)) {
          int tt = t - EB * LX, el = tt / LY, r = tt - el * LY;
          contract_eo<T, Q, K, 1, 1>(s1 + el * S::R1 + Q * K * K + Q * r, su + el * NRT + NX1 + K * r, tab.BHTp, tab.BHTn);
        } else {
          int tt = t - EB * (LX + LY), el = tt / LZ, r = tt - el * LZ;
          contract_eo<T, Q, K, 1, 1>(s1 + el * S::R1 + Q * K * K + Q * (K + 1) * K + Q * r,
                                   su + el * NRT + 2 * NX1 + K * r, tab.BHTp, tab.BHTn);
        }
      }
    }
    __syncthreads();
  }

  // -- scatter to y_u ------------------------------------------------------------
  if (mode & (OP_M | OP_DT)) {
    for (int t = tid; t < EB * NRT; t += nth) {
      int el = t / NRT, n = t - el * NRT, e = e0 + el;
      if (e >= n_elem) continue;
      int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
      bool ess;
      int g = rt_global<K>(L, ex, ey, ez, n, ess);
      IO o;
      if (ess) {
        if (!(mode & OP_M)) continue;
        o = u[g];
      } else {
        T v = (mode & OP_M) ? su[t] : (T)0;
        if (mode & OP_DT) v += dt_local<T, K>(sq + el * NL2, n);
        o = Cvt<T, IO>::out(v);
      }
      atomicAdd(yu + g, o);
    }
  }
}

// ---------------------------------------------------------------------------
// Setup: geometric factors at the Q^3 points of each element (one thread per
// element and point). Trilinear map from the 8 corner vertices.
template <int Q>
__global__ void k_geom(const ElemTables tab, const LatticeDims L, const int n_elem,
                       const double* __restrict__ vx, const double* __restrict__ vy,
                       const double* __restrict__ vz, const double* __restrict__ bcoef,
                       double* __restrict__ G, double* __restrict__ wdet, int* __restrict__ bad) {
  constexpr int NQ = Q * Q * Q;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_elem * NQ) return;
  int e = (int)(t / NQ), p = (int)(t - (int64_t)e * NQ);
  int px = p % Q, py = (p / Q) % Q, pz = p / (Q * Q);
  double x1 = tab.gx[px], x2 = tab.gx[py], x3 = tab.gx[pz];
  double w = tab.gw[px] * tab.gw[py] * tab.gw[pz];
  int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        int64_t vid = (ex + a) + (int64_t)(L.nx + 1) * ((ey + b) + (int64_t)(L.ny + 1) * (ez + c));
        double Na = a ? x1 : 1.0 - x1, Nb = b ? x2 : 1.0 - x2, Nc = c ? x3 : 1.0 - x3;
        double da = a ? 1.0 : -1.0, db = b ? 1.0 : -1.0, dc = c ? 1.0 : -1.0;
        double g0 = da * Nb * Nc, g1 = Na * db * Nc, g2 = Na * Nb * dc;
        double X[3] = {vx[vid], vy[vid], vz[vid]};
        for (int i = 0; i < 3; ++i) {
          J[i][0] += X[i] * g0;
          J[i][1] += X[i] * g1;
          J[i][2] += X[i] * g2;
        }
      }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det > 0.0)) {
    atomicExch(bad, 1);
    det = 1.0;
  }
  double s = w * bcoef[e] / det;
  double JtJ[6];
  int idx = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) JtJ[idx++] = J[0][a] * J[0][b] + J[1][a] * J[1][b] + J[2][a] * J[2][b];
  double* g = G + (size_t)e * 6 * NQ + p;
  for (int c = 0; c < 6; ++c) g[c * NQ] = s * JtJ[c];
  wdet[(size_t)e * NQ + p] = w / det;
}

// Setup: W_e = sum_p wdet_p psi_a psi_b by sum factorisation over the tensor
// structure, then W_e^-1 by Gauss-Jordan elimination in shared memory (W_e is
// SPD: no pivoting), symmetrised. One CTA per element.
template <int K, int Q>
struct WinvSmem {
  static constexpr int NL2 = K * K * K, KK = K * K, NQ = Q * Q * Q;
  static constexpr int OFF_HH = NQ;
  static constexpr int OFF_T1 = OFF_HH + Q * KK;
  static constexpr int OFF_T2 = OFF_T1 + Q * Q * KK;
  static constexpr int OFF_A = OFF_T2 + Q * KK * KK;
  static constexpr int OFF_COL = OFF_A + NL2 * NL2;
  static constexpr int TOTAL = OFF_COL + NL2;
};

template <int K, int Q, bool CHOL = false>
__global__ void __launch_bounds__(128)
k_winv(const ElemTables tab, const int n_elem, const double* __restrict__ wdet,
       double* __restrict__ winv, double* __restrict__ wdiag) {
  using S = WinvSmem<K, Q>;
  constexpr int NL2 = S::NL2, KK = S::KK, NQ = S::NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sw = reinterpret_cast<double*>(smem_raw);
  double* HH = sw + S::OFF_HH;     // HH[p][(a,b)] = h_a(g_p) h_b(g_p)
  double* T1 = sw + S::OFF_T1;     // [p1][p2][(a3,b3)]
  double* T2 = sw + S::OFF_T2;     // [p1][(a2,b2)][(a3,b3)]
  double* A = sw + S::OFF_A;       // [NL2][NL2]
  double* colp = sw + S::OFF_COL;  // pivot column
  const int e = blockIdx.x;
  if (e >= n_elem) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int t = tid; t < NQ; t += nth) sw[t] = wdet[(size_t)e * NQ + t];
  for (int t = tid; t < Q * KK; t += nth) {
    int p = t / KK, ab = t % KK, a = ab % K, b = ab / K;
    HH[t] = tab.BH[p * K + a] * tab.BH[p * K + b];
  }
  __syncthreads();
  for (int t = tid; t < Q * Q * KK; t += nth) {
    int p12 = t / KK, ab = t % KK;
    double s = 0.0;
    for (int p3 = 0; p3 < Q; ++p3) s += sw[p12 + Q * Q * p3] * HH[p3 * KK + ab];
    T1[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < Q * KK * KK; t += nth) {
    int p1 = t / (KK * KK), r = t % (KK * KK), ab2 = r / KK, ab3 = r % KK;
    double s = 0.0;
    for (int p2 = 0; p2 < Q; ++p2) s += HH[p2 * KK + ab2] * T1[(p1 + Q * p2) * KK + ab3];
    T2[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < NL2 * NL2; t += nth) {
    int A_ = t / NL2, B_ = t % NL2;  // row (a1,a2,a3), col (b1,b2,b3)
    int a1 = A_ % K, a2 = (A_ / K) % K, a3 = A_ / KK;
    int b1 = B_ % K, b2 = (B_ / K) % K, b3 = B_ / KK;
    int ab1 = a1 + K * b1, ab2 = a2 + K * b2, ab3 = a3 + K * b3;
    double s = 0.0;
    for (int p1 = 0; p1 < Q; ++p1) s += HH[p1 * KK + ab1] * T2[(p1 * KK + ab2) * KK + ab3];
    A[t] = s;
  }
  __syncthreads();
  for (int t = tid; t < NL2; t += nth) wdiag[(size_t)e * NL2 + t] = A[t * NL2 + t];
  if constexpr (CHOL) {
    // W_e = L L^T (right-looking, in place in the lower triangle; SPD: no pivoting);
    // stored with zeros above the diagonal and the reciprocal on it
    for (int p = 0; p < NL2; ++p) {
      __syncthreads();
      const double d = sqrt(A[p * NL2 + p]);
      for (int i = p + 1 + tid; i < NL2; i += nth) A[i * NL2 + p] /= d;
      __syncthreads();
      if (tid == 0) A[p * NL2 + p] = d;
      const int m = NL2 - p - 1;  // trailing lower triangle, row-wise
      for (int t = tid; t < m * m; t += nth) {
        const int i = p + 1 + t / m, j = p + 1 + t % m;
        if (j <= i) A[i * NL2 + j] = fma(-A[i * NL2 + p], A[j * NL2 + p], A[i * NL2 + j]);
      }
    }
    __syncthreads();
    double* out = winv + (size_t)e * NL2 * NL2;
    for (int t = tid; t < NL2 * NL2; t += nth) {
      const int i = t / NL2, j = t % NL2;
      out[t] = j < i ? A[t] : (j == i ? 1.0 / A[t] : 0.0);
    }
    return;
  }
  // Gauss-Jordan elimination in place (W_e is SPD: no pivoting). After step p,
  // column p holds column p of the inverse.
  for (int p = 0; p < NL2; ++p) {
    __syncthreads();
    for (int i = tid; i < NL2; i += nth) colp[i] = A[i * NL2 + p];
    __syncthreads();
    const double piv = 1.0 / colp[p];
    for (int j = tid; j < NL2; j += nth) A[p * NL2 + j] = (j == p) ? piv : A[p * NL2 + j] * piv;
    __syncthreads();
    for (int t = tid; t < NL2 * NL2; t += nth) {
      int i = t / NL2, j = t - i * NL2;
      if (i == p) continue;
      double f = colp[i];
      A[t] = (j == p) ? -f * piv : fma(-f, A[p * NL2 + j], A[t]);
    }
  }
  __syncthreads();
  double* out = winv + (size_t)e * NL2 * NL2;
  for (int t = tid; t < NL2 * NL2; t += nth) {
    int i = t / NL2, j = t % NL2;
    out[t] = 0.5 * (A[i * NL2 + j] + A[j * NL2 + i]);
  }
}

// Setup: diag(M_e) by sum factorisation with squared 1D tables, added to the
// global diagonal (two addends on shared faces). One thread per element and
// local dof (direct sum over the Q^3 points: setup only).
template <int K, int Q>
__global__ void k_diagM(const ElemTables tab, const LatticeDims L, const int n_elem,
                        const double* __restrict__ G, double* __restrict__ mt) {
  constexpr int NX1 = (K + 1) * K * K, NRT = 3 * NX1, NQ = Q * Q * Q;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_elem * NRT) return;
  int e = (int)(t / NRT), n = (int)(t - (int64_t)e * NRT);
  int c, i, j, l;
  if (n < NX1) { c = 0; i = n % (K + 1); j = (n / (K + 1)) % K; l = n / ((K + 1) * K); }
  else if (n < 2 * NX1) { int m = n - NX1; c = 1; i = m % K; j = (m / K) % (K + 1); l = m / (K * (K + 1)); }
  else { int m = n - 2 * NX1; c = 2; i = m % K; j = (m / K) % K; l = m / (K * K); }
  const double* g = G + (size_t)e * 6 * NQ + (c == 0 ? 0 : (c == 1 ? 3 : 5)) * NQ;
  double s = 0.0;
  for (int pz = 0; pz < Q; ++pz) {
    double bz = (c == 2) ? tab.BI[pz * (K + 1) + l] : tab.BH[pz * K + l];
    for (int py = 0; py < Q; ++py) {
      double by = (c == 1) ? tab.BI[py * (K + 1) + j] : tab.BH[py * K + j];
      for (int px = 0; px < Q; ++px) {
        double bx = (c == 0) ? tab.BI[px * (K + 1) + i] : tab.BH[px * K + i];
        double v = bx * by * bz;
        s += g[px + Q * (py + Q * pz)] * v * v;
      }
    }
  }
  int ex = e % L.nx, ey = (e / L.nx) % L.ny, ez = e / (L.nx * L.ny);
  bool ess;
  int gid = rt_global<K>(L, ex, ey, ez, n, ess);
  atomicAdd(mt + gid, s);
}

// Setup: diag of W_e = sum_p wdet_p B(p,a)^2 for the tensor basis B = B1 x B1 x B1
// (BH: the histopolation basis; BG: the GL nodal basis of the local CG).
template <int K, int Q>
__global__ void k_diag_tensor(const ElemTables tab, const int n_elem, const bool gl, const double* __restrict__ wdet,
                              double* __restrict__ out) {
  constexpr int NL2 = K * K * K, NQ = Q * Q * Q;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_elem * NL2) return;
  const int e = (int)(t / NL2), a = (int)(t % NL2);
  const int a1 = a % K, a2 = (a / K) % K, a3 = a / (K * K);
  const double* B = gl ? tab.BG : tab.BH;
  double s = 0.0;
  for (int p3 = 0; p3 < Q; ++p3) {
    double b3 = B[p3 * K + a3];
    for (int p2 = 0; p2 < Q; ++p2) {
      double b2 = B[p2 * K + a2];
      for (int p1 = 0; p1 < Q; ++p1) {
        double b = B[p1 * K + a1] * b2 * b3;
        s += wdet[(size_t)e * NQ + p1 + Q * (p2 + Q * p3)] * b * b;
      }
    }
  }
  out[t] = s;
}

template <typename T, typename IO, int K, int Q, bool AFF>
hd_status launch_elem_op(hd_op* h, int mode, const T* G, const T* winv, const T* cs, const CgArgs<T>& cg,
                         const IO* u, const IO* q, IO* yu, IO* yq, const T* Ga) {
  constexpr int EB = ElemCfg<T, AFF>::EB, THREADS = ElemCfg<T, AFF>::THREADS;
  using S = Sizes<K, Q>;
  size_t smem = (size_t)EB * S::PER_ELEM * sizeof(T) + StageW<T, K, Q, EB, AFF>::BAR_BYTES;
  auto kern = k_elem_op<T, IO, K, Q, EB, AFF>;
  static bool attr_set[HD_MAX_DEVICES] = {};
  bool* done = device_flag(attr_set);
  if (!done || !*done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return hd_cuda_check(h, e, "cudaFuncSetAttribute(k_elem_op)");
    if (done) *done = true;
  }
  TabT<T> tab = make_tab<T>(h->tab);
  const int64_t e_end = h->e_end < 0 ? h->n_elem : h->e_end, e_first = h->e_end < 0 ? 0 : h->e_first;
  int blocks = (int)((e_end - e_first + EB - 1) / EB);
  prof_mark(h, true);
  if (blocks > 0)
    kern<<<blocks, THREADS, smem, h->stream>>>(tab, h->L, mode, (int)e_end, (int)e_first, G, winv, cs, cg, u, q,
                                               yu, yq, Ga);
  prof_mark(h, false);
  HD_LAUNCH_CK(h, "k_elem_op");
  return HD_OK;
}

// Ga: the affine factors (or null: the general kernel). The affine kernel is built for
// q = k+1 and the FP64 / double-float arithmetic only.
template <typename T, typename IO, int K, int Q>
hd_status run_elem_op(hd_op* h, int mode, const T* G, const T* winv, const T* cs, const CgArgs<T>& cg,
                      const IO* u, const IO* q, IO* yu, IO* yq, const T* Ga = nullptr) {
  constexpr bool HAS_AFF = Q == K + 1 && !std::is_same<T, float>::value;
  if (HAS_AFF && Ga != nullptr)
    return launch_elem_op<T, IO, K, Q, HAS_AFF>(h, mode, G, winv, cs, cg, u, q, yu, yq, Ga);
  return launch_elem_op<T, IO, K, Q, false>(h, mode, G, winv, cs, cg, u, q, yu, yq, Ga);
}

template <int K, int Q>
hd_status run_elem_setup(hd_op* h, const double* bcoef, int* d_bad) {
  constexpr int NQ = Q * Q * Q, NRT = 3 * (K + 1) * K * K;
  // phase times (setup_ms[0..2]): geometric factors; W^-1 data (dense inverses, or
  // the Jacobi diagonals of the local CG); diag(M)
  cudaEvent_t ev[4];
  for (auto& x : ev) cudaEventCreate(&x);
  cudaEventRecord(ev[0], h->stream);
  int64_t n = h->n_elem * NQ;
  if (n > 0) k_geom<Q><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      h->tab, h->L, (int)h->n_elem, h->d_vx, h->d_vy, h->d_vz, bcoef, h->d_G, h->d_wdet, d_bad);
  HD_LAUNCH_CK(h, "k_geom");
  cudaEventRecord(ev[1], h->stream);
  if (h->n_elem > 0) {
    constexpr int NL2 = K * K * K;
    unsigned nb = (unsigned)((h->n_elem * NL2 + 255) / 256);
    k_diag_tensor<K, Q><<<nb, 256, 0, h->stream>>>(h->tab, (int)h->n_elem, true, h->d_wdet, h->d_wgldiag);
    if (h->winv_mode == HD_WINV_CG || h->winv_mode == HD_WINV_CG_HIST)  // else diag(W_e) comes from k_winv
      k_diag_tensor<K, Q><<<nb, 256, 0, h->stream>>>(h->tab, (int)h->n_elem, false, h->d_wdet, h->d_wdiag);
    HD_LAUNCH_CK(h, "k_diag_tensor");
  }
  if (h->winv_mode == HD_WINV_DENSE && h->n_elem > 0) {
    size_t smem = (size_t)WinvSmem<K, Q>::TOTAL * sizeof(double);
    cudaError_t err = cudaFuncSetAttribute(k_winv<K, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return hd_cuda_check(h, err, "cudaFuncSetAttribute(k_winv)");
    k_winv<K, Q><<<(unsigned)h->n_elem, 128, smem, h->stream>>>(h->tab, (int)h->n_elem, h->d_wdet, h->d_winv,
                                                                 h->d_wdiag);
    HD_LAUNCH_CK(h, "k_winv");
  }
  if (h->winv_mode == HD_WINV_CHOL && h->n_elem > 0) {
    size_t smem = (size_t)WinvSmem<K, Q>::TOTAL * sizeof(double);
    cudaError_t err =
        cudaFuncSetAttribute(k_winv<K, Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return hd_cuda_check(h, err, "cudaFuncSetAttribute(k_winv chol)");
    k_winv<K, Q, true><<<(unsigned)h->n_elem, 128, smem, h->stream>>>(h->tab, (int)h->n_elem, h->d_wdet,
                                                                       h->d_wchol, h->d_wdiag);
    HD_LAUNCH_CK(h, "k_winv chol");
  }
  cudaEventRecord(ev[2], h->stream);
  int64_t m = h->n_elem * NRT;
  if (m > 0) k_diagM<K, Q><<<(unsigned)((m + 255) / 256), 256, 0, h->stream>>>(h->tab, h->L, (int)h->n_elem,
                                                                          h->d_G, h->d_mt);
  HD_LAUNCH_CK(h, "k_diagM");
  cudaEventRecord(ev[3], h->stream);
  if (cudaEventSynchronize(ev[3]) == cudaSuccess)
    for (int i = 0; i < 3; ++i) cudaEventElapsedTime(&h->setup_ms[i], ev[i], ev[i + 1]);
  for (auto& x : ev) cudaEventDestroy(x);
  return HD_OK;
}

}  // namespace hdk

// Per-K entry points defined in k_elem_k*.cu
#define HD_DECLARE_K(KK)                                                                          \
  hd_status elem_op_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu,       \
                          double* yq);                                                            \
  hd_status elem_op_df_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu,    \
                             double* yq);                                                         \
  hd_status elem_op_f32_k##KK(hd_op* h, int mode, const float* u, const float* q, float* yu,      \
                              float* yq);                                                         \
  hd_status elem_op_f32io64_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu, \
                                  double* yq);                                                    \
  hd_status elem_setup_k##KK(hd_op* h, const double* bcoef, int* d_bad);

HD_DECLARE_K(2)
HD_DECLARE_K(3)
HD_DECLARE_K(4)
HD_DECLARE_K(5)

// FP64: the dense W_e^-1, or the local CG to a relative residual of 1e-14 in the GL nodal
// basis (HD_WINV_CG, at most 40 iterations) or the histopolation basis (HD_WINV_CG_HIST,
// at most 100: its Jacobi-scaled W is worse conditioned).
// FP32 (inner solves): the dense W_e^-1 in FP32 when the handle has one (faster on
// this GPU than the CG's barrier-bound iterations), else the local CG to 1e-6.
#define HD_DEFINE_K(KK)                                                                                   \
  hd_status elem_op_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq) { \
    const bool hi = h->winv_mode == HD_WINV_CG_HIST, ch = h->winv_mode == HD_WINV_CHOL;                   \
    const bool cgm = h->winv_mode == HD_WINV_CG || hi;                                                    \
    hdk::CgArgs<double> cg{cgm ? h->d_wdet : nullptr, hi ? h->d_wdiag : h->d_wgldiag, hi ? 100 : 40, 1e-28, \
                           hi ? 1 : 0, ch ? 1 : 0};                                                       \
    const double* wi = ch ? h->d_wchol : h->d_winv;                                                       \
    if (h->q == KK + 1)                                                                                   \
      return hdk::run_elem_op<double, double, KK, KK + 1>(h, mode, h->d_G, wi, h->d_cscale, cg, u, q, yu, \
                                                          yq, h->d_Ga);                                   \
    return hdk::run_elem_op<double, double, KK, KK + 2>(h, mode, h->d_G, wi, h->d_cscale, cg, u, q, yu, yq); \
  }                                                                                                       \
  hd_status elem_op_df_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu,            \
                             double* yq) {                                                                \
    hdk::CgArgs<dfloat> cg{nullptr, nullptr, 0, dfloat(0), 0, 0, h->d_kerr};                              \
    if (h->q == KK + 1)                                                                                   \
      return hdk::run_elem_op<dfloat, double, KK, KK + 1>(h, mode, h->x_G, h->x_winv, h->x_cscale, cg, u, \
                                                          q, yu, yq, h->x_Ga);                            \
    return hdk::run_elem_op<dfloat, double, KK, KK + 2>(h, mode, h->x_G, h->x_winv, h->x_cscale, cg, u, q, \
                                                        yu, yq);                                          \
  }                                                                                                       \
  hd_status elem_op_f32_k##KK(hd_op* h, int mode, const float* u, const float* q, float* yu,              \
                              float* yq) {                                                                \
    hdk::CgArgs<float> cg{h->f_winv ? nullptr : h->f_wdet, h->f_wgldiag, 20, 1e-12f, 0, 0};               \
    if (h->q == KK + 1)                                                                                   \
      return hdk::run_elem_op<float, float, KK, KK + 1>(h, mode, h->f_G, h->f_winv, h->f_cscale, cg, u, q, \
                                                        yu, yq);                                          \
    return hdk::run_elem_op<float, float, KK, KK + 2>(h, mode, h->f_G, h->f_winv, h->f_cscale, cg, u, q,  \
                                                      yu, yq);                                            \
  }                                                                                                       \
  hd_status elem_op_f32io64_k##KK(hd_op* h, int mode, const double* u, const double* q, double* yu,       \
                                  double* yq) {                                                           \
    hdk::CgArgs<float> cg{h->f_winv ? nullptr : h->f_wdet, h->f_wgldiag, 20, 1e-12f, 0, 0};               \
    if (h->q == KK + 1)                                                                                   \
      return hdk::run_elem_op<float, double, KK, KK + 1>(h, mode, h->f_G, h->f_winv, h->f_cscale, cg, u,  \
                                                         q, yu, yq);                                      \
    return hdk::run_elem_op<float, double, KK, KK + 2>(h, mode, h->f_G, h->f_winv, h->f_cscale, cg, u, q, \
                                                       yu, yq);                                           \
  }                                                                                                       \
  hd_status elem_setup_k##KK(hd_op* h, const double* bcoef, int* d_bad) {                                 \
    if (h->q == KK + 1) return hdk::run_elem_setup<KK, KK + 1>(h, bcoef, d_bad);                          \
    return hdk::run_elem_setup<KK, KK + 2>(h, bcoef, d_bad);                                              \
  }
