// Tensor-core block apply on affine meshes (inner operator of the mixed-precision
// solves).
//
// On a parallelepiped element the Jacobian J is constant, so the Piola-mapped RT mass
// (Eq. matrices) is M_e = sum_ab G_ab K_ab with G = beta J^T J / det J (3 x 3 per
// element) and K_ab = int phi_hat_a phi_hat_b^T the reference-cube blocks between
// velocity components a and b, shared by all elements (each a Kronecker product of 1D
// mass matrices). With the elements of a tile as the M dimension of a GEMM, the nine
// products U_b K_ab^T are dense contractions for the 5th-generation tensor cores:
// tcgen05.mma, operands in shared memory, FP32 accumulators in tensor memory, one
// element per TMEM lane. FP16 holds 11 significant bits, so both operands are split
// into FP16 pairs (v = hi + lo, each scaled by a power of two into FP16's range) and
// each block takes three products, U_hi K_hi + U_lo K_hi + U_hi K_lo (the lo*lo term
// is below FP32 rounding): about 22-bit operands and FP32 accumulation, an FP32-class
// operator. The rest of the block apply is element-local and cheap and runs on the
// CUDA cores in FP32: D u and the own-cell D^T q of the lattice divergence (Sec. 2.1)
// and C q = c_e det J (H^-1 x H^-1 x H^-1) q (the affine W_e^-1, Sec. 2.5).
//
// Kernel structure (persistent, one CTA per SM, 288 threads): eight element warps own
// the 128 elements of a tile, two threads per element (element t & 127, half t >> 7):
// they stage the tile's L2 coefficients q~ in shared memory with coalesced loads,
// gather each half of the element's RT coefficients, split them into the FP16 pairs
// of the A operand (a per-element, per-component power of two from the maximum the two
// halves exchange through shared memory), compute y_q = D u - C q for half of the
// element's cells while the tensor core works, and read half of the accumulator
// columns from TMEM lane t & 127 in the epilogue. Warp 8 allocates TMEM, and its lane
// 0 streams the nine K_ab blocks (hi + lo, pre-laid-out in global memory) through a
// two-stage shared-memory ring with bulk copies (cp.async.bulk, mbarrier transaction
// counts) and issues the MMAs, signalling with tcgen05.commit. Every wait is bounded;
// a timeout sets the error word, the CTA drains what it has in flight and frees its
// TMEM.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "hd_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_TILE = 128;          // elements per tile = TMEM lanes
constexpr int TC_EW = 8;              // element warps: two threads per element
constexpr int TC_ET = 32 * TC_EW;     // element threads
constexpr int TC_THREADS = TC_ET + 32;  // and the control warp
constexpr int TC_STAGES = 2;          // K_ab ring depth
constexpr int TC_TMEM_COLS = 512;

template <int K>
struct TcShape {
  static constexpr int NC = (K + 1) * K * K;             // RT dofs per component
  static constexpr int NP = (NC + 15) / 16 * 16;         // padded to the MMA's N and K granules
  static constexpr int NH = (NC + 1) / 2;                // dofs per thread of an element's pair
  static constexpr int NL2 = K * K * K;
  static constexpr int QP = NL2 + 1;                     // staged q~ row (odd: no bank conflicts)
  static constexpr uint32_t U_BYTES = TC_TILE * NP * 2;  // one component, one half of the pair
  static constexpr uint32_t Q_BYTES = (TC_TILE * QP * 4 + 15) / 16 * 16;
  static constexpr uint32_t KB_BYTES = NP * NP * 2;      // one K_ab block, one half of the pair
  static constexpr uint32_t EF_BYTES = TC_TILE * 8 * 4;    // a tile's element factors
  static constexpr uint32_t SMEM = 6 * U_BYTES + Q_BYTES + 2 * EF_BYTES + TC_STAGES * 2 * KB_BYTES;
  // accumulator regions of 3 NP columns: a = 2 reuses a = 0's when nine do not fit
  static constexpr bool REUSE = 9 * NP > TC_TMEM_COLS;
  static_assert(3 * NP * (REUSE ? 2 : 3) <= TC_TMEM_COLS, "accumulators exceed TMEM");
  static_assert(SMEM <= 227 * 1024 - 4096, "shared memory");
};

struct TcParams {
  float HI[HD_MAXK * HD_MAXK];  // inverse of the 1D histopolation mass (row-major)
  float kscale[9];              // 2^-p_ab: undoes the power-of-two scaling of block (a, b)
};

enum { B_KFULL = 0, B_KEMPTY = TC_STAGES, B_UFULL = 2 * TC_STAGES, B_UEMPTY, B_ACC, B_REG = B_ACC + 3, B_FIN = B_REG + 3,
       B_EF, B_COUNT = B_EF + 2 };

// local dof n of component a -> (i, j, l) along x, y, z (the component's node index
// runs along its own axis, interval indices along the others)
template <int K>
__device__ __forceinline__ void tc_dof_ijl(int a, int n, int& i, int& j, int& l) {
  if (a == 0) {
    i = n % (K + 1); j = (n / (K + 1)) % K; l = n / ((K + 1) * K);
  } else if (a == 1) {
    i = n % K; j = (n / K) % (K + 1); l = n / (K * (K + 1));
  } else {
    i = n % K; j = (n / K) % K; l = n / (K * K);
  }
}

// global RT id and essential flag of dof (i, j, l) of component a of element (ex, ey, ez)
template <int K>
__device__ __forceinline__ int tc_rt_global(const LatticeDims& L, int a, int ex, int ey, int ez, int i, int j, int l,
                                            bool& ess) {
  const int I = ex * K + i, J = ey * K + j, Z = ez * K + l;
  if (a == 0) {
    ess = (I == 0 && (L.ess & 1)) || (I == L.X && (L.ess & 2));
    return I + (L.X + 1) * (J + L.Y * Z);
  }
  if (a == 1) {
    ess = (J == 0 && (L.ess & 4)) || (J == L.Y && (L.ess & 8));
    return L.n_xf + I + L.X * (J + (L.Y + 1) * Z);
  }
  ess = (Z == 0 && (L.ess & 16)) || (Z == L.Z && (L.ess & 32));
  return L.n_xf + L.n_yf + I + L.X * (J + L.Y * Z);
}

template <typename IO>
__device__ __forceinline__ float tc_in(IO v);
template <>
__device__ __forceinline__ float tc_in<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tc_in<double>(double v) { return Cvt<float, double>::in(v); }
template <typename IO>
__device__ __forceinline__ IO tc_out(float v);
template <>
__device__ __forceinline__ float tc_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ double tc_out<double>(float v) { return Cvt<float, double>::out(v); }

// power of two s with max|v| / s in [2^13, 2^14] (1 for max = 0)
__device__ __forceinline__ float tc_scale_for(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  int ex;
  frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
  return ldexpf(1.f, ex - 14);
}

// waits with a bound, giving up early once another thread has aborted
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

// barrier among the element threads only (the control warp does not take part)
__device__ __forceinline__ void tc_elem_sync() { asm volatile("bar.sync 1, %0;" ::"n"(TC_ET) : "memory"); }

// Gather of component B of the tile's RT coefficients into the FP16 pairs of the A
// operand (see the kernel). Essential faces and elements past the end give 0.
// Gather of component B of element el's RT coefficients, half HF of them (dofs
// [HF*NH, min(NC, (HF+1)*NH))), into the FP16 pairs of the A operand: the two threads of
// the element exchange their maxima through shared memory (smax[half][element]) and
// take the same power-of-two scale. Essential faces and elements past the end give 0.
template <typename IO, int K, int B, int HF>
__device__ __forceinline__ float tc_gather_half(const LatticeDims& L, bool valid, int ex, int ey, int ez,
                                                const IO* __restrict__ x, unsigned char* sU, float (*smax)[TC_TILE],
                                                int el) {
  using S = TcShape<K>;
  constexpr int NC = S::NC, NP = S::NP, NH = S::NH, N0 = HF * NH, N1 = HF ? NC : NH;
  float v[NH];
  float m = 0.f;
#pragma unroll
  for (int jj = 0; jj < NH; ++jj) {
    const int n = N0 + jj;
    v[jj] = 0.f;
    if (n < N1 && valid) {
      int i, j, l;
      tc_dof_ijl<K>(B, n, i, j, l);
      bool ess;
      const int g = tc_rt_global<K>(L, B, ex, ey, ez, i, j, l, ess);
      if (!ess) v[jj] = tc_in<IO>(x[g]);
    }
    m = fmaxf(m, fabsf(v[jj]));
  }
  smax[HF][el] = m;
  tc_elem_sync();
  const float sc = tc_scale_for(fmaxf(smax[0][el], smax[1][el]));
  const float inv = 1.f / sc;
  unsigned char* hi = sU + B * S::U_BYTES;
  unsigned char* lo = sU + (3 + B) * S::U_BYTES;
#pragma unroll
  for (int jj = 0; jj < NH; ++jj) {
    const int n = N0 + jj;
    if (n >= N1) continue;
    const float w = v[jj] * inv;
    const __half h = __float2half_rn(w);
    const uint32_t off = tc::kmajor_offset(el, n, NP);
    *reinterpret_cast<__half*>(hi + off) = h;
    *reinterpret_cast<__half*>(lo + off) = __float2half_rn(w - __half2float(h));
  }
  return sc;
}

// value of local dof n of component b of tile element el from its FP16 pair (times the scale)
template <int K>
__device__ __forceinline__ float tc_u_smem(const unsigned char* sU, int b, int el, int n, float sc) {
  using S = TcShape<K>;
  const uint32_t off = tc::kmajor_offset(el, n, S::NP);
  const float h = __half2float(*reinterpret_cast<const __half*>(sU + b * S::U_BYTES + off));
  const float l = __half2float(*reinterpret_cast<const __half*>(sU + (3 + b) * S::U_BYTES + off));
  return (h + l) * sc;
}

// y_q = D u - C q on the cells a3 in [HF ? ceil(K/2) : 0, HF ? K : ceil(K/2)) of one element:
// C q = sC (H^-1 x H^-1 x H^-1) q with the z contraction first (it alone mixes a3), D u
// from the element's FP16 pairs in shared memory (essential faces were gathered as 0)
template <typename IO, int K, int HF>
__device__ __forceinline__ void tc_yq(const LatticeDims& L, const TcParams& P, int ex, int ey, int ez, float sC,
                                      const float* q, const unsigned char* sU, int el, const float sc[3],
                                      IO* __restrict__ yq) {
  constexpr int A3H = (K + 1) / 2, A3LO = HF ? A3H : 0, A3HI = HF ? K : A3H;
#pragma unroll
  for (int a3 = A3LO; a3 < A3HI; ++a3) {
    float t1[K * K], t2[K * K];
#pragma unroll
    for (int c = 0; c < K * K; ++c) {
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < K; ++m) s = fmaf(P.HI[a3 * K + m], q[c + K * K * m], s);
      t1[c] = s;  // c = a1 + K a2
    }
#pragma unroll
    for (int c = 0; c < K * K; ++c) {
      const int a1 = c % K, a2 = c / K;
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < K; ++m) s = fmaf(P.HI[a2 * K + m], t1[a1 + K * m], s);
      t2[c] = s;
    }
#pragma unroll
    for (int c = 0; c < K * K; ++c) {
      const int a1 = c % K, a2 = c / K;
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < K; ++m) s = fmaf(P.HI[a1 * K + m], t2[m + K * a2], s);
      // x-faces i = a1, a1 + 1; y-faces j = a2, a2 + 1; z-faces l = a3, a3 + 1
      const float du = tc_u_smem<K>(sU, 0, el, a1 + 1 + (K + 1) * (a2 + K * a3), sc[0]) -
                       tc_u_smem<K>(sU, 0, el, a1 + (K + 1) * (a2 + K * a3), sc[0]) +
                       tc_u_smem<K>(sU, 1, el, a1 + K * (a2 + 1 + (K + 1) * a3), sc[1]) -
                       tc_u_smem<K>(sU, 1, el, a1 + K * (a2 + (K + 1) * a3), sc[1]) +
                       tc_u_smem<K>(sU, 2, el, a1 + K * (a2 + K * (a3 + 1)), sc[2]) -
                       tc_u_smem<K>(sU, 2, el, a1 + K * (a2 + K * a3), sc[2]);
      yq[(ex * K + a1) + (int64_t)L.X * ((ey * K + a2) + (int64_t)L.Y * (ez * K + a3))] = tc_out<IO>(du - sC * s);
    }
  }
}

// epilogue of component a on this thread's chunks of 16 accumulator columns (chunk c16
// with c16 % 2 == HF): y_u += g_a0 D_a0 + g_a1 D_a1 + g_a2 D_a2 + own-cell D^T q, one
// atomic per face (a shared face gets exactly two, from its two elements); essential
// faces get x (the constrained identity)
template <typename IO, int K, int HF>
__device__ __forceinline__ void tc_epilogue(const LatticeDims& L, int a, uint32_t base, float ga0, float ga1, float ga2,
                                            bool valid, int ex, int ey, int ez, const float* q,
                                            const IO* __restrict__ x, IO* __restrict__ y) {
  using S = TcShape<K>;
  constexpr int NC = S::NC, NP = S::NP;
#pragma unroll 1
  for (int c0 = 16 * HF; c0 < NC; c0 += 32) {
    float d0[16], d1[16], d2[16];
    tc::tmem_ld16(base + c0, d0);
    tc::tmem_ld16(base + NP + c0, d1);
    tc::tmem_ld16(base + 2 * NP + c0, d2);
    tc::tmem_wait_ld();
    if (!valid) continue;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int n = c0 + jj;
      if (n >= NC) continue;
      int i, j, l;
      tc_dof_ijl<K>(a, n, i, j, l);
      bool ess;
      const int gid = tc_rt_global<K>(L, a, ex, ey, ez, i, j, l, ess);
      if (ess) {
        atomicAdd(y + gid, x[gid]);
        continue;
      }
      float v = ga0 * d0[jj] + ga1 * d1[jj] + ga2 * d2[jj];
      // own-cell D^T q: + q of the cell whose high face this is, - q of the cell whose low face
      const int node = a == 0 ? i : (a == 1 ? j : l);
      const int st = a == 0 ? 1 : (a == 1 ? K : K * K);
      const int c = i + K * (j + K * l);  // the cell on the face's high side (when node < K)
      if (node > 0) v += q[c - st];
      if (node < K) v -= q[c];
      atomicAdd(y + gid, tc_out<IO>(v));
    }
  }
}

template <typename IO, int K>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_op_tc(const LatticeDims L, const int n_elem, const TcParams P, const __half* __restrict__ kblocks,
            const float* __restrict__ ef, const IO* __restrict__ x, IO* __restrict__ y, int* __restrict__ err) {
  using S = TcShape<K>;
  constexpr int NC = S::NC, NP = S::NP, NH = S::NH, NL2 = S::NL2, QP = S::QP;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[B_COUNT];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;                   // any thread: others stop polling early
  __shared__ int elem_abort;                   // element threads: written before, read after a barrier
  __shared__ float smax[3][2][TC_TILE];        // per-half maxima of |u| per component and element
  unsigned char* sU = smem;                    // [part][component] A operands, K-major
  float* sQ = reinterpret_cast<float*>(smem + 6 * S::U_BYTES);                   // [element][QP]
  float* sEF = reinterpret_cast<float*>(smem + 6 * S::U_BYTES + S::Q_BYTES);      // [2][element][8]
  unsigned char* sK = smem + 6 * S::U_BYTES + S::Q_BYTES + 2 * S::EF_BYTES;       // [stage][part]
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t n_tiles = ((int64_t)n_elem + TC_TILE - 1) / TC_TILE;
  const int64_t off_q = (int64_t)L.n_xf + L.n_yf + (int64_t)L.X * L.Y * (L.Z + 1);  // = n_rt
  volatile int* abort_v = &abort_flag;
  auto bar = [&](int i) { return tc::smem_u32(&bars[i]); };

  if (tid == 0) {
    abort_flag = 0;
    elem_abort = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      tc::mbar_init(bar(B_KFULL + s), 1);
      tc::mbar_init(bar(B_KEMPTY + s), 1);
    }
    tc::mbar_init(bar(B_UFULL), TC_ET);
    tc::mbar_init(bar(B_UEMPTY), 1);
    for (int a = 0; a < 3; ++a) {
      tc::mbar_init(bar(B_ACC + a), 1);
      tc::mbar_init(bar(B_REG + a), TC_ET);
    }
    tc::mbar_init(bar(B_FIN), 1);
    tc::mbar_init(bar(B_EF), 1);
    tc::mbar_init(bar(B_EF + 1), 1);
    tc::fence_mbar_init();
  }
  if (warp == TC_EW) {
    tc::tmem_alloc(tc::smem_u32(&tmem_slot), TC_TMEM_COLS);
    tc::tmem_relinquish();
  } else {
    // zero the A operands once: the padding columns stay zero (finite) for every tile
    for (uint32_t o = tid * 16; o < 6 * S::U_BYTES; o += TC_ET * 16)
      *reinterpret_cast<uint4*>(sU + o) = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async_smem();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = tmem_slot;

  if (warp == TC_EW) {
    // ---- control warp: the K_ab ring and the MMAs (lane 0) ------------------------
    if ((tid & 31) == 0) {
      const uint32_t idesc = tc::idesc_f16_f32(TC_TILE, NP);
      uint32_t issued = 0, blk = 0;
      int uses[3] = {0, 0, 0};
      bool ok = true;
      int64_t ef_last = -1;  // last tile iteration whose element factors were requested
      for (int64_t tile = blockIdx.x, it = 0; ok && tile < n_tiles; tile += gridDim.x, ++it) {
        // the tile's element factors by the copy engine into buffer it & 1 (its previous
        // user, tile it - 2, finished before the element threads signalled tile it - 1)
        {
          const int64_t e0 = tile * TC_TILE;
          const uint32_t bytes = (uint32_t)((n_elem - e0 < TC_TILE ? n_elem - e0 : TC_TILE) * 32);
          tc::mbar_arrive_expect_tx(bar(B_EF + (int)(it & 1)), bytes);
          tc::bulk_g2s(tc::smem_u32(sEF + (it & 1) * TC_TILE * 8), ef + e0 * 8, bytes, bar(B_EF + (int)(it & 1)));
          ef_last = it;
        }
        if (!(ok = tc_wait(bar(B_UFULL), (uint32_t)(it & 1), abort_v))) break;
        tc::fence_after_sync();
        for (int a = 0; ok && a < 3; ++a) {
          const int r = (S::REUSE && a == 2) ? 0 : a;
          if (uses[r] > 0 && !(ok = tc_wait(bar(B_REG + r), (uint32_t)((uses[r] - 1) & 1), abort_v))) break;
          tc::fence_after_sync();
          ++uses[r];
          const uint32_t dcol = tbase + (uint32_t)(r * 3 * NP);
          for (int b = 0; ok && b < 3; ++b) {
            while (ok && issued < blk + TC_STAGES) {
              const uint32_t s = issued % TC_STAGES;
              if (issued >= TC_STAGES && !(ok = tc_wait(bar(B_KEMPTY + s), ((issued / TC_STAGES) - 1) & 1, abort_v)))
                break;
              tc::mbar_arrive_expect_tx(bar(B_KFULL + s), 2 * S::KB_BYTES);
              tc::bulk_g2s(tc::smem_u32(sK + s * 2 * S::KB_BYTES), kblocks + (size_t)(issued % 9) * NP * NP * 2,
                           2 * S::KB_BYTES, bar(B_KFULL + s));
              ++issued;
            }
            const uint32_t s = blk % TC_STAGES;
            if (!ok || !(ok = tc_wait(bar(B_KFULL + s), (blk / TC_STAGES) & 1, abort_v))) break;
            tc::fence_after_sync();
            const uint32_t uhi = tc::smem_u32(sU + b * S::U_BYTES), ulo = tc::smem_u32(sU + (3 + b) * S::U_BYTES);
            const uint32_t khi = tc::smem_u32(sK + s * 2 * S::KB_BYTES), klo = khi + S::KB_BYTES;
            const uint32_t d = dcol + (uint32_t)(b * NP);
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              const uint32_t A = (p == 1) ? ulo : uhi, B = (p == 2) ? klo : khi;
#pragma unroll
              for (int ks = 0; ks < NP / 16; ++ks)
                tc::mma_f16(d, tc::smem_desc(A + ks * 256, 128, NP * 16), tc::smem_desc(B + ks * 256, 128, NP * 16),
                            idesc, p > 0 || ks > 0);
            }
            tc::mma_commit(bar(B_KEMPTY + s));  // the stage is free once these MMAs are done
            ++blk;
          }
          if (ok) tc::mma_commit(bar(B_ACC + a));
        }
        if (ok) tc::mma_commit(bar(B_UEMPTY));
      }
      if (!ok) {
        atomicOr(err, 1);
        abort_flag = 1;
      }
      // drain: every MMA issued by this thread, then every bulk copy still in flight
      tc::mma_commit(bar(B_FIN));
      if (!tc::mbar_wait(bar(B_FIN), 0)) atomicOr(err, 2);
      for (uint32_t c = blk; c < issued; ++c)
        if (!tc::mbar_wait(bar(B_KFULL + c % TC_STAGES), (c / TC_STAGES) & 1)) atomicOr(err, 2);
      for (int64_t i = ef_last - 1; i <= ef_last; ++i)  // the element-factor copies of the last two tiles
        if (i >= 0 && !tc::mbar_wait(bar(B_EF + (int)(i & 1)), (uint32_t)((i >> 1) & 1))) atomicOr(err, 2);
    }
    __syncwarp();
  } else {
    // ---- element warps ---------------------------------------------------------------
    // Every exit decision is uniform over the element threads (they share a named
    // barrier): a failed wait sets elem_abort, and all threads test it after a barrier.
    const int el = tid & (TC_TILE - 1), hf = tid >> 7;  // own element (epilogue, y_q) and half
    for (int64_t tile = blockIdx.x, it = 0; tile < n_tiles; tile += gridDim.x, ++it) {
      if (it > 0 && !tc_wait(bar(B_UEMPTY), (uint32_t)((it - 1) & 1), abort_v)) elem_abort = 1;
      tc_elem_sync();
      if (elem_abort) break;
      const int64_t e0 = tile * TC_TILE;
      // q~ of the tile's elements into shared memory, consecutive threads on consecutive cells
      for (int s = tid; s < TC_TILE * NL2; s += TC_ET) {
        const int a1 = s % K, r = s / K, e2 = r % TC_TILE, o = r / TC_TILE;  // o = a2 + K a3
        float v = 0.f;
        if (e0 + e2 < n_elem) {
          const int f = (int)(e0 + e2), fx = f % L.nx, fy = (f / L.nx) % L.ny, fz = f / (L.nx * L.ny);
          const int a2 = o % K, a3 = o / K;
          v = tc_in<IO>(x[off_q + (fx * K + a1) + (int64_t)L.X * ((fy * K + a2) + (int64_t)L.Y * (fz * K + a3))]);
        }
        sQ[e2 * QP + a1 + K * o] = v;
      }
      // this thread's half of the element's RT coefficients, per component: FP16 pairs
      const int64_t e = e0 + el;
      const bool valid = e < n_elem;
      const int ee = valid ? (int)e : 0;
      const int ex = ee % L.nx, ey = (ee / L.nx) % L.ny, ez = ee / (L.nx * L.ny);
      float sc[3];
      if (hf) {
        sc[0] = tc_gather_half<IO, K, 0, 1>(L, valid, ex, ey, ez, x, sU, smax[0], el);
        sc[1] = tc_gather_half<IO, K, 1, 1>(L, valid, ex, ey, ez, x, sU, smax[1], el);
        sc[2] = tc_gather_half<IO, K, 2, 1>(L, valid, ex, ey, ez, x, sU, smax[2], el);
      } else {
        sc[0] = tc_gather_half<IO, K, 0, 0>(L, valid, ex, ey, ez, x, sU, smax[0], el);
        sc[1] = tc_gather_half<IO, K, 1, 0>(L, valid, ex, ey, ez, x, sU, smax[1], el);
        sc[2] = tc_gather_half<IO, K, 2, 0>(L, valid, ex, ey, ez, x, sU, smax[2], el);
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(bar(B_UFULL));
      tc_elem_sync();  // sQ and U complete for every element thread
      // the element factors staged by the control warp's bulk copy (warp-uniform wait)
      if (!__all_sync(0xffffffffu, tc_wait(bar(B_EF + (int)(it & 1)), (uint32_t)((it >> 1) & 1), abort_v)))
        elem_abort = 1;
      const float* f = sEF + (it & 1) * TC_TILE * 8 + el * 8;
      const float* q = sQ + el * QP;
      // while the tensor core works: y_q = D u - C q on this thread's half of the cells
      if (valid) {
        if (hf)
          tc_yq<IO, K, 1>(L, P, ex, ey, ez, f[6], q, sU, el, sc, y + off_q);
        else
          tc_yq<IO, K, 0>(L, P, ex, ey, ez, f[6], q, sU, el, sc, y + off_q);
      }
      // epilogue: y_u += sum_b G_ab s_b K_ab u_b + own-cell D^T q on this thread's chunks of
      // 16 columns, from TMEM lane el
      float g[3][3];
      {
        const float G00 = valid ? f[0] : 0.f, G01 = valid ? f[1] : 0.f, G02 = valid ? f[2] : 0.f;
        const float G11 = valid ? f[3] : 0.f, G12 = valid ? f[4] : 0.f, G22 = valid ? f[5] : 0.f;
        const float Gm[3][3] = {{G00, G01, G02}, {G01, G11, G12}, {G02, G12, G22}};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) g[a][b] = Gm[a][b] * P.kscale[a * 3 + b] * sc[b];
      }
      const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int r = (S::REUSE && a == 2) ? 0 : a;
        // warp-uniform: the TMEM loads are warp-collective
        const bool ready = __all_sync(0xffffffffu, tc_wait(bar(B_ACC + a), (uint32_t)(it & 1), abort_v));
        if (!ready) {
          elem_abort = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t base = tlane + (uint32_t)(r * 3 * NP);
        if (hf)
          tc_epilogue<IO, K, 1>(L, a, base, g[a][0], g[a][1], g[a][2], valid, ex, ey, ez, q, x, y);
        else
          tc_epilogue<IO, K, 0>(L, a, base, g[a][0], g[a][1], g[a][2], valid, ex, ey, ez, q, x, y);
        tc::fence_before_sync();
        tc::mbar_arrive(bar(B_REG + r));
      }
      tc_elem_sync();
      if (elem_abort) break;
    }
    if (elem_abort && tid == 0) {
      atomicOr(err, 4);
      abort_flag = 1;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == TC_EW) tc::tmem_dealloc(tbase, TC_TMEM_COLS);
}

}  // namespace

// ---- host side ------------------------------------------------------------------------

struct TcState {
  __half* kblocks = nullptr;  // [9][2][NP x NP] K-major canonical layout
  float* ef = nullptr;        // [E][8] G00 G01 G02 G11 G12 G22, c_e det J, 0
  int* err = nullptr;
  TcParams P;
  int grid = 0;
};

namespace {

__global__ void k_tc_elemdata(int64_t E, const double* __restrict__ Ga, const double* __restrict__ cs,
                              float* __restrict__ ef) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  for (int i = 0; i < 6; ++i) ef[e * 8 + i] = (float)Ga[e * 8 + i];
  ef[e * 8 + 6] = (float)(cs[e] * Ga[e * 8 + 6]);
  ef[e * 8 + 7] = 0.f;
}

// reference blocks K_ab as Kronecker products of the 1D matrices int l_i l_i', int l_i h_j,
// int h_j h_j' (Gauss rule of the handle's tables, q = k + 1: exact), each scaled by a
// power of two into FP16's range and split into hi + lo, written in the MMA's K-major
// layout (rows: dofs n of component a = N; columns: dofs m of component b = K)
template <int K>
void tc_build_blocks(const ElemTables& tab, int q, std::vector<__half>& out, float kscale[9]) {
  using S = TcShape<K>;
  constexpr int NC = S::NC, NP = S::NP;
  double MII[K + 1][K + 1], MIH[K + 1][K], MHH[K][K];
  for (int i = 0; i <= K; ++i)
    for (int i2 = 0; i2 <= K; ++i2) {
      double s = 0;
      for (int p = 0; p < q; ++p) s += tab.gw[p] * tab.BI[p * (K + 1) + i] * tab.BI[p * (K + 1) + i2];
      MII[i][i2] = s;
    }
  for (int i = 0; i <= K; ++i)
    for (int j = 0; j < K; ++j) {
      double s = 0;
      for (int p = 0; p < q; ++p) s += tab.gw[p] * tab.BI[p * (K + 1) + i] * tab.BH[p * K + j];
      MIH[i][j] = s;
    }
  for (int j = 0; j < K; ++j)
    for (int j2 = 0; j2 < K; ++j2) {
      double s = 0;
      for (int p = 0; p < q; ++p) s += tab.gw[p] * tab.BH[p * K + j] * tab.BH[p * K + j2];
      MHH[j][j2] = s;
    }
  auto ijl = [](int a, int n, int idx[3]) {
    if (a == 0) { idx[0] = n % (K + 1); idx[1] = (n / (K + 1)) % K; idx[2] = n / ((K + 1) * K); }
    else if (a == 1) { idx[0] = n % K; idx[1] = (n / K) % (K + 1); idx[2] = n / (K * (K + 1)); }
    else { idx[0] = n % K; idx[1] = (n / K) % K; idx[2] = n / (K * K); }
  };
  out.assign((size_t)9 * 2 * NP * NP, __float2half(0.f));
  std::vector<double> blk((size_t)NC * NC);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double mx = 0;
      for (int n = 0; n < NC; ++n)
        for (int m = 0; m < NC; ++m) {
          int ia[3], ib[3];
          ijl(a, n, ia);
          ijl(b, m, ib);
          double v = 1.0;
          for (int d = 0; d < 3; ++d) {
            const bool na = d == a, nb = d == b;
            v *= na ? (nb ? MII[ia[d]][ib[d]] : MIH[ia[d]][ib[d]]) : (nb ? MIH[ib[d]][ia[d]] : MHH[ia[d]][ib[d]]);
          }
          blk[(size_t)n * NC + m] = v;
          mx = std::fmax(mx, std::fabs(v));
        }
      int ex = 0;
      std::frexp(mx > 0 ? mx : 1.0, &ex);
      const double sc = std::ldexp(1.0, 14 - ex);
      kscale[a * 3 + b] = (float)std::ldexp(1.0, ex - 14);
      __half* hi = out.data() + (size_t)(a * 3 + b) * 2 * NP * NP;
      __half* lo = hi + NP * NP;
      for (int n = 0; n < NC; ++n)
        for (int m = 0; m < NC; ++m) {
          const float v = (float)(blk[(size_t)n * NC + m] * sc);
          const __half h = __float2half_rn(v);
          const size_t o = tc::kmajor_offset(n, m, NP) / 2;
          hi[o] = h;
          lo[o] = __float2half_rn(v - __half2float(h));
        }
    }
}

template <typename IO, int K>
hd_status tc_launch(hd_op* h, const IO* x, IO* y) {
  using S = TcShape<K>;
  TcState* st = h->tc;
  // at least 120 KB of shared memory per CTA: one CTA per SM, so that no CTA waits for
  // another's 512 TMEM columns
  constexpr uint32_t smem = S::SMEM > 120u * 1024u ? S::SMEM : 120u * 1024u;
  static bool configured[HD_MAX_DEVICES] = {};
  bool* cfg = device_flag(configured);
  if (!cfg || !*cfg) {
    cudaError_t e = cudaFuncSetAttribute(k_op_tc<IO, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return hd_cuda_check(h, e, "cudaFuncSetAttribute(k_op_tc)");
    if (cfg) *cfg = true;
  }
  HD_CK(h, cudaMemsetAsync(y, 0, sizeof(IO) * h->n_rt, h->stream));
  if (h->n_elem == 0) return HD_OK;
  const int64_t tiles = (h->n_elem + TC_TILE - 1) / TC_TILE;
  const int grid = (int)(tiles < st->grid ? tiles : st->grid);
  k_op_tc<IO, K><<<grid, TC_THREADS, smem, h->stream>>>(h->L, (int)h->n_elem, st->P, st->kblocks, st->ef, x, y,
                                                           st->err);
  HD_LAUNCH_CK(h, "k_op_tc");
  return HD_OK;
}

template <typename IO>
hd_status tc_dispatch(hd_op* h, const IO* x, IO* y) {
  switch (h->k) {
    case 2: return tc_launch<IO, 2>(h, x, y);
    case 3: return tc_launch<IO, 3>(h, x, y);
    case 4: return tc_launch<IO, 4>(h, x, y);
  }
  return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "tensor-core operator: k = 2..4");
}

}  // namespace

// Builds the tensor-core operator's data on first use: the split reference blocks, the
// FP32 per-element factors and the error word.
hd_status tc_setup(hd_op* h) {
  if (h->tc) return HD_OK;
  if (!h->d_Ga)
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED,
                   "tensor-core operator: affine meshes only (hd_create with affine = 1, q = k + 1, dense W^-1, "
                   "every element a parallelepiped)");
  if (h->k < 2 || h->k > 4) return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "tensor-core operator: k = 2..4");
  int dev = 0, major = 0, sms = 0;
  HD_CK(h, cudaGetDevice(&dev));
  HD_CK(h, cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  HD_CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (major != 10) return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "tensor-core operator: sm_100 family (tcgen05) only");
  TcState* st = new (std::nothrow) TcState();
  if (!st) return hd_fail(h, HD_ERR_OOM, "tensor-core state");
  std::memset(&st->P, 0, sizeof(st->P));
  std::vector<__half> blocks;
  switch (h->k) {
    case 2: tc_build_blocks<2>(h->tab, h->q, blocks, st->P.kscale); break;
    case 3: tc_build_blocks<3>(h->tab, h->q, blocks, st->P.kscale); break;
    case 4: tc_build_blocks<4>(h->tab, h->q, blocks, st->P.kscale); break;
  }
  for (int i = 0; i < h->k * h->k; ++i) st->P.HI[i] = (float)h->tab.HI[i];
  st->grid = sms;
  hd_status s = HD_OK;
  if (cudaMalloc(&st->kblocks, blocks.size() * sizeof(__half)) != cudaSuccess ||
      cudaMalloc(&st->ef, sizeof(float) * 8 * (h->n_elem > 0 ? h->n_elem : 1)) != cudaSuccess ||
      cudaMalloc(&st->err, sizeof(int)) != cudaSuccess) {
    s = hd_fail(h, HD_ERR_OOM, "tensor-core operator data");
  } else if (cudaMemcpy(st->kblocks, blocks.data(), blocks.size() * sizeof(__half), cudaMemcpyHostToDevice) !=
                 cudaSuccess ||
             cudaMemset(st->err, 0, sizeof(int)) != cudaSuccess) {
    s = hd_fail(h, HD_ERR_CUDA, "tensor-core operator upload");
  } else if (h->n_elem > 0) {
    k_tc_elemdata<<<(unsigned)((h->n_elem + 255) / 256), 256, 0, h->stream>>>(h->n_elem, h->d_Ga, h->d_cscale, st->ef);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) s = hd_fail(h, HD_ERR_CUDA, "tensor-core operator setup");
  }
  if (s != HD_OK) {
    cudaFree(st->kblocks);
    cudaFree(st->ef);
    cudaFree(st->err);
    delete st;
    return s;
  }
  h->tc = st;
  return HD_OK;
}

void tc_free(hd_op* h) {
  if (!h->tc) return;
  cudaFree(h->tc->kblocks);
  cudaFree(h->tc->ef);
  cudaFree(h->tc->err);
  delete h->tc;
  h->tc = nullptr;
}

hd_status tc_apply(hd_op* h, const double* x, double* y) {
  hd_status s = tc_setup(h);
  if (s != HD_OK) return s;
  return tc_dispatch<double>(h, x, y);
}
hd_status tc_apply_f32(hd_op* h, const float* x, float* y) {
  hd_status s = tc_setup(h);
  if (s != HD_OK) return s;
  return tc_dispatch<float>(h, x, y);
}

// error word of the tensor-core kernel (bounded waits that ran out); cleared on read
hd_status tc_check(hd_op* h) {
  // the element kernel's word (its W_e^-1 staging, when built with it) and the tensor-core kernel's
  int e = 0, ek = 0;
  if (h->d_kerr) HD_CK(h, cudaMemcpyAsync(&ek, h->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (h->tc) HD_CK(h, cudaMemcpyAsync(&e, h->tc->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  if (ek) {
    HD_CK(h, cudaMemsetAsync(h->d_kerr, 0, sizeof(int), h->stream));
    return hd_fail(h, HD_ERR_CUDA, std::string("a bounded wait ran out: ") +
                                       ((ek & 16) ? "tensor-core convolution" : "staged W^-1 rows"));
  }
  if (e) {
    HD_CK(h, cudaMemsetAsync(h->tc->err, 0, sizeof(int), h->stream));
    return hd_fail(h, HD_ERR_CUDA, "tensor-core operator: a bounded wait ran out (error word " + std::to_string(e) + ")");
  }
  return HD_OK;
}

extern "C" hd_status hd_apply_op_tc(hd_handle h, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  return tc_apply(h, x, y);
}
extern "C" hd_status hd_apply_op_tc_f32(hd_handle h, const float* x, float* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  return tc_apply_f32(h, x, y);
}
extern "C" hd_status hd_tc_status(hd_handle h) {
  if (!h) return HD_ERR_INVALID_ARG;
  return tc_check(h);
}
extern "C" hd_status hd_set_inner_operator(hd_handle h, int32_t mode) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (mode == 0) {
    h->inner_op = 0;
    return HD_OK;
  }
  if (mode != 1) return hd_fail(h, HD_ERR_INVALID_ARG, "inner operator: 0 (CUDA cores) or 1 (tensor cores)");
  hd_status s = tc_setup(h);
  if (s != HD_OK) return s;
  h->inner_op = 1;
  return HD_OK;
}
