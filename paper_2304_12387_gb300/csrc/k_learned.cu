// Learned Schur-complement preconditioner: a linear, symmetric-by-construction
// convolutional network on the L2 cell lattice added to the V/W-cycle on S~ (the
// paper uses one AMG V-cycle, Sec. 3.2):
//
//   P r = V r + s (C1^T C2^T C2 C1 (s r)) + delta r / d,    s = d^-1/2, d = diag(S~),
//
// V the handle's V/W-cycle (the hierarchy it was created with), C1: 3x3x3 conv
// 1 -> 32, C2: 3x3x3 conv 32 -> 32 (no bias, no activation), ^T the adjoint
// convolutions. The network term is positive semi-definite for any weights, so P
// stays SPD and, with small initial weights, starts at the plain cycle: training
// can only add to it what the energy-norm loss says the cycle misses.
//
// Activations are FP16 with 32 channels per cell ([cell][32], 64 B), weights FP16
// for compute with an FP32 master copy, accumulation FP32. The 32 -> 32
// convolutions (forward and adjoint) run on the tensor cores: tcgen05.mma with
// accumulators in tensor memory (k_conv2_tc, the default), or mma.sync m16n8k16
// (k_conv2); the 1 -> 32 / 32 -> 1 convolutions and the weight gradients on the
// CUDA cores. Input fields are normalised to unit RMS before the network and the
// output rescaled (exactly linear), which keeps FP16 in range.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hd_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int NC = 32;
constexpr int NT = 27;
constexpr int TPB = 256;
constexpr int RED_BLOCKS = 512;
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// ---- small reductions --------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum_d(double v, double* sh) {
  v = warp_sum_d(v);
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (ln < (int)(blockDim.x >> 5)) ? sh[ln] : 0.0;
    s = warp_sum_d(s);
  }
  __syncthreads();
  return s;
}

// partial[b] = sum over block b's chunk of (a_i w_i)^2  (w may be float or null)
template <typename TA>
__global__ void k_sumsq_partial(int64_t n, const TA* __restrict__ a, const float* __restrict__ w,
                                double* __restrict__ partial) {
  __shared__ double sh[32];
  int64_t chunk = (n + RED_BLOCKS - 1) / RED_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double v = (double)a[i] * (w ? (double)w[i] : 1.0);
    s = fma(v, v, s);
  }
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
// partial[b] = sum over block b's chunk of a_i b_i
__global__ void k_dot_partial_l(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ partial) {
  __shared__ double sh[32];
  int64_t chunk = (n + RED_BLOCKS - 1) / RED_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
__global__ void k_final_sum(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = block_sum_d(partial[threadIdx.x], sh);  // blockDim.x == RED_BLOCKS
  if (threadIdx.x == 0) out[0] = s;
}
// scal[0] = sum of squares; scal[1] = sigma = sqrt(scal[0]/n) (1 if zero); scal[8] = 1/sigma
__global__ void k_sigma(const double* __restrict__ partial, double* __restrict__ scal, int64_t n) {
  __shared__ double sh[32];
  double s = block_sum_d(partial[threadIdx.x], sh);
  if (threadIdx.x == 0) {
    double sigma = sqrt(s / (double)n);
    if (!(sigma > 0.0)) sigma = 1.0;
    scal[0] = s;
    scal[1] = sigma;
    scal[8] = 1.0 / sigma;
  }
}

// ---- element-wise kernels ----------------------------------------------------
__global__ void k_sq(int64_t n, const double* __restrict__ diag, float* __restrict__ sq, double* __restrict__ dinv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  sq[i] = (float)(1.0 / sqrt(diag[i]));
  dinv[i] = 1.0 / diag[i];
}
// u = s r / sigma (1/sigma at scal[8])
__global__ void k_make_u(int64_t n, const double* __restrict__ r, const float* __restrict__ sq,
                         const double* __restrict__ scal, float* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  u[i] = (float)r[i] * sq[i] * (float)scal[8];
}

// ---- 1 -> 32 and 32 -> 1 convolutions (one warp per cell, lane = channel) ----
__device__ __forceinline__ void cell_ijk(int64_t c, int X, int Y, int& I, int& J, int& K) {
  I = (int)(c % X);
  J = (int)((c / X) % Y);
  K = (int)(c / ((int64_t)X * Y));
}

// out[c][co] = sum_t W1[co,t] in(c + off_t) (zero outside): one thread per cell,
// all 32 channels, W1 (as W1h[t][co]) in shared memory
__global__ void __launch_bounds__(256) k_conv1(int X, int Y, int Z, const __half* __restrict__ W1h,
                                               const float* __restrict__ in, __half* __restrict__ out) {
  __shared__ float w[NT * NC];
  for (int i = threadIdx.x; i < NT * NC; i += blockDim.x) w[i] = __half2float(W1h[i]);
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= (int64_t)X * Y * Z) return;
  int I, J, K;
  cell_ijk(c, X, Y, I, J, K);
  float acc[NC];
#pragma unroll
  for (int co = 0; co < NC; ++co) acc[co] = 0.f;
#pragma unroll 1
  for (int t = 0; t < NT; ++t) {
    const int i = I + t % 3 - 1, j = J + (t / 3) % 3 - 1, k = K + t / 9 - 1;
    if (i < 0 || i >= X || j < 0 || j >= Y || k < 0 || k >= Z) continue;
    const float v = in[i + (int64_t)X * (j + (int64_t)Y * k)];
#pragma unroll
    for (int co = 0; co < NC; ++co) acc[co] = fmaf(w[t * NC + co], v, acc[co]);
  }
  uint4* o = reinterpret_cast<uint4*>(out + c * NC);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __half2 h0 = __floats2half2_rn(acc[8 * q + 0], acc[8 * q + 1]), h1 = __floats2half2_rn(acc[8 * q + 2], acc[8 * q + 3]);
    __half2 h2 = __floats2half2_rn(acc[8 * q + 4], acc[8 * q + 5]), h3 = __floats2half2_rn(acc[8 * q + 6], acc[8 * q + 7]);
    uint4 v;
    v.x = *reinterpret_cast<uint32_t*>(&h0);
    v.y = *reinterpret_cast<uint32_t*>(&h1);
    v.z = *reinterpret_cast<uint32_t*>(&h2);
    v.w = *reinterpret_cast<uint32_t*>(&h3);
    o[q] = v;
  }
}

// s = sum_{t,co} W1[co,t] g[c - off_t][co]; mode 0: z = sq sigma s + delta r / d (FP64);
// mode 1: outf = s (FP32); mode 2: z += sq sigma s + delta r / d. One thread per cell.
__global__ void __launch_bounds__(256) k_conv1T(int X, int Y, int Z, const __half* __restrict__ W1h,
                                                const __half* __restrict__ g, int mode, const float* __restrict__ sq,
                                                const double* __restrict__ scal, double delta,
                                                const double* __restrict__ r, const double* __restrict__ dinv,
                                                double* __restrict__ z, float* __restrict__ outf) {
  __shared__ float w[NT * NC];
  for (int i = threadIdx.x; i < NT * NC; i += blockDim.x) w[i] = __half2float(W1h[i]);
  __syncthreads();
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= (int64_t)X * Y * Z) return;
  int I, J, K;
  cell_ijk(c, X, Y, I, J, K);
  float acc = 0.f;
#pragma unroll 1
  for (int t = 0; t < NT; ++t) {
    const int i = I - (t % 3 - 1), j = J - ((t / 3) % 3 - 1), k = K - (t / 9 - 1);
    if (i < 0 || i >= X || j < 0 || j >= Y || k < 0 || k >= Z) continue;
    const uint4* src = reinterpret_cast<const uint4*>(g + (i + (int64_t)X * (j + (int64_t)Y * k)) * NC);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 v = src[q];
      const __half2* hv = reinterpret_cast<const __half2*>(&v);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        float2 f = __half22float2(hv[p]);
        acc = fmaf(w[t * NC + 8 * q + 2 * p], f.x, acc);
        acc = fmaf(w[t * NC + 8 * q + 2 * p + 1], f.y, acc);
      }
    }
  }
  if (mode == 0)
    z[c] = (double)sq[c] * scal[1] * (double)acc + delta * r[c] * dinv[c];
  else if (mode == 2)
    z[c] += (double)sq[c] * scal[1] * (double)acc + delta * r[c] * dinv[c];
  else
    outf[c] = acc;
}

// ---- 32 -> 32 convolution on the tensor cores --------------------------------
// Tile of 16 x 4 x 4 output cells per CTA iteration (persistent CTAs), halo
// 18 x 6 x 6 cells in shared memory, weights W[t][o][i] (27 x 32 x 32 halves) in
// shared memory. 16-byte channel chunks are XOR-swizzled by (row >> 1) & 3 so
// that the fragment loads of 8 consecutive rows hit distinct banks.
constexpr int CTX = 16, CTY = 4, CTZ = 4;
constexpr int HX = CTX + 2, HY = CTY + 2, HZ = CTZ + 2, HCELLS = HX * HY * HZ;

__device__ __forceinline__ int swz(int row, int ch) { return row * NC + ((((ch >> 3) ^ ((row >> 1) & 3))) << 3) + (ch & 7); }

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256) k_conv2(int X, int Y, int Z, const __half* __restrict__ Wg,
                                               const __half* __restrict__ in, __half* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half* ws = reinterpret_cast<__half*>(smem_raw);  // [27*32][32]
  __half* hs = ws + NT * NC * NC;                    // [HCELLS][32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  // weights once per CTA
  for (int i = tid; i < NT * NC * 4; i += blockDim.x) {
    int row = i >> 2, ch = (i & 3) * 8;
    *reinterpret_cast<uint4*>(ws + swz(row, ch)) = *reinterpret_cast<const uint4*>(Wg + row * NC + ch);
  }
  const int ntx = (X + CTX - 1) / CTX, nty = (Y + CTY - 1) / CTY, ntz = (Z + CTZ - 1) / CTZ;
  const int64_t ntiles = (int64_t)ntx * nty * ntz;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = (int)(tile % ntx), ty = (int)((tile / ntx) % nty), tz = (int)(tile / ((int64_t)ntx * nty));
    const int x0 = tx * CTX, y0 = ty * CTY, z0 = tz * CTZ;
    __syncthreads();  // previous tile's fragments are consumed (and weights are in place)
    for (int i = tid; i < HCELLS * 4; i += blockDim.x) {
      int cell = i >> 2, ch = (i & 3) * 8;
      int hx = cell % HX, hy = (cell / HX) % HY, hz = cell / (HX * HY);
      int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gx >= 0 && gx < X && gy >= 0 && gy < Y && gz >= 0 && gz < Z)
        v = *reinterpret_cast<const uint4*>(in + (gx + (int64_t)X * (gy + (int64_t)Y * gz)) * NC + ch);
      *reinterpret_cast<uint4*>(hs + swz(cell, ch)) = v;
    }
    __syncthreads();
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
      const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int ch0 = ks * 16 + 2 * t4;
        uint32_t bf[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int row = t * NC + nt * 8 + g;
          bf[nt][0] = *reinterpret_cast<const uint32_t*>(ws + swz(row, ch0));
          bf[nt][1] = *reinterpret_cast<const uint32_t*>(ws + swz(row, ch0 + 8));
        }
#pragma unroll
        for (int mr = 0; mr < 2; ++mr) {
          const int rr = 2 * warp + mr, y = rr % CTY, z = rr / CTY;
          const int cA = ((z + dz) * HY + (y + dy)) * HX + (g + dx), cB = cA + 8;
          uint32_t af[4];
          af[0] = *reinterpret_cast<const uint32_t*>(hs + swz(cA, ch0));
          af[1] = *reinterpret_cast<const uint32_t*>(hs + swz(cB, ch0));
          af[2] = *reinterpret_cast<const uint32_t*>(hs + swz(cA, ch0 + 8));
          af[3] = *reinterpret_cast<const uint32_t*>(hs + swz(cB, ch0 + 8));
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma16816(acc[mr][nt], af, bf[nt]);
        }
      }
    }
#pragma unroll
    for (int mr = 0; mr < 2; ++mr) {
      const int rr = 2 * warp + mr, y = y0 + rr % CTY, z = z0 + rr / CTY;
      if (y >= Y || z >= Z) continue;
#pragma unroll
      for (int half_ = 0; half_ < 2; ++half_) {
        const int x = x0 + g + 8 * half_;
        if (x >= X) continue;
        __half* o = out + (x + (int64_t)X * (y + (int64_t)Y * z)) * NC;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          *reinterpret_cast<__half2*>(o + nt * 8 + 2 * t4) =
              __floats2half2_rn(acc[mr][nt][2 * half_], acc[mr][nt][2 * half_ + 1]);
      }
    }
  }
}

// ---- 32 -> 32 convolution on the 5th-generation tensor cores (tcgen05) ----------------
// Implicit GEMM: a tile is 128 consecutive cells of one x-line (M = 128), N = 32 output
// channels, K = 27 taps x 32 input channels, per tap two tcgen05.mma.kind::f16 (K = 16)
// into an FP32 accumulator of 32 TMEM columns. The A operand of tap (dx, dy, dz) is the
// halo line (y + dy - 1, z + dz - 1) shifted by dx, read in place: the halo is stored
// channel-chunk-major (16 bytes = 8 channels of one cell, consecutive cells contiguous),
// so 8 consecutive cells form a core matrix (128 bytes) at any shift, row groups sit 128
// bytes apart and the two chunks of a K step one chunk slab apart. Weights W[t][o][i] are
// staged once per CTA as core matrices (8 o x 8 i).
// Work unit: one x-tile and one z, for a run of CT_YRUN consecutive y. The CTA walks y
// through a ring of 5 halo slabs (a slab: the lines z - 1, z, z + 1 at one y), so each
// tile loads one new slab (3 lines) instead of 9 lines. Slabs are loaded by 16-byte
// cp.async copies (zero fill outside the lattice) two tiles ahead, one commit group per
// tile, so a slab has a whole tile's MMAs and epilogue to arrive;
// accumulators are double-buffered, so a tile's epilogue (8 warps: TMEM lane = cell,
// 16 channels per warp half) overlaps the next tile's MMAs. Every wait is bounded
// (error word bit 4).
constexpr int CT_M = 128;                          // cells per tile
constexpr int CT_H = CT_M + 2;                     // halo cells per line
constexpr int CT_RING = 5;                         // slabs in the ring
constexpr int CT_SLOTS = 3 * CT_RING;              // halo lines
constexpr int CT_CHUNK = CT_SLOTS * CT_H * 16;     // bytes of one 8-channel slab of the ring
constexpr int CT_HALO = 4 * CT_CHUNK;              // 124,800 bytes
constexpr int CT_W = NT * 4 * 4 * 128;             // 55,296 bytes of weights
constexpr int CT_SMEM = CT_HALO + CT_W + 64;
constexpr int CT_THREADS = 256;
constexpr int CT_YRUN = 48;                        // y per work unit

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the most recent committed group complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ int ring_slot(int y) { return ((y % CT_RING) + CT_RING) % CT_RING; }

__global__ void __launch_bounds__(CT_THREADS, 1)
k_conv2_tc(int X, int Y, int Z, const __half* __restrict__ Wg, const __half* __restrict__ in,
           __half* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* wsm = smem_raw + CT_HALO;                  // [27 taps][4 o-groups][4 i-chunks][8 o][8 i]
  uint64_t* bar = reinterpret_cast<uint64_t*>(wsm + CT_W);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < NT * NC * 4; i += CT_THREADS) {  // 16-byte pieces: (t, o, i-chunk)
    const int t = i / (NC * 4), o = (i / 4) % NC, c = i % 4;
    const uint4 v = *reinterpret_cast<const uint4*>(Wg + ((size_t)t * NC + o) * NC + c * 8);
    *reinterpret_cast<uint4*>(wsm + ((t * 4 + (o >> 3)) * 4 + c) * 128 + (o & 7) * 16) = v;
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(&bar[0]), 1);
    tc::mbar_init(tc::smem_u32(&bar[1]), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), 64);  // two accumulators of 32 columns
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();  // the staged weights, for the tensor core
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot, hbase = tc::smem_u32(smem_raw), wbase = tc::smem_u32(wsm);
  const int ntx = (X + CT_M - 1) / CT_M, nyr = (Y + CT_YRUN - 1) / CT_YRUN;
  const int64_t nunits = (int64_t)ntx * Z * nyr;
  constexpr uint32_t IDESC = tc::idesc_f16_f32(CT_M, NC);
  // slab y' (lines z - 1, z, z + 1) of the x-tile at x0 into its ring slot
  auto load_slab = [&](int x0, int yp, int z) {
    const int sl = ring_slot(yp);
    for (int i = tid; i < 3 * CT_H * 4; i += CT_THREADS) {
      const int c = i & 3, h = (i >> 2) % CT_H, zl = (i >> 2) / CT_H;
      const int gx = x0 - 1 + h, gz = z - 1 + zl;
      const bool ok = gx >= 0 && gx < X && yp >= 0 && yp < Y && gz >= 0 && gz < Z;
      const __half* src = ok ? in + (gx + (int64_t)X * (yp + (int64_t)Y * gz)) * NC + c * 8 : in;
      cp_async16(hbase + c * CT_CHUNK + ((sl * 3 + zl) * CT_H + h) * 16, src, ok);
    }
  };
  // one thread: 27 taps x 2 K steps into accumulator b. A descriptor's address field is
  // the shared-memory address in 16-byte units, so every operand's descriptor is a base
  // descriptor plus a constant offset (the ring slots of the three y-slabs of the tile
  // are the only run-time part).
  const uint64_t adesc0 = tc::smem_desc(hbase, CT_CHUNK, 128), bdesc0 = tc::smem_desc(wbase, 128, 512);
  auto issue = [&](int y, int b) {
    const int lofs[3] = {ring_slot(y - 1) * 3 * CT_H, ring_slot(y) * 3 * CT_H, ring_slot(y + 1) * 3 * CT_H};
    const uint32_t d = tmem + 32 * b;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;  // the order of W[t]
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ad = adesc0 + (uint64_t)(2 * ks * (CT_CHUNK / 16) + lofs[dy] + dz * CT_H + dx);
        const uint64_t bd = bdesc0 + (uint64_t)((t * 16 + 2 * ks) * 8);
        tc::mma_f16(d, ad, bd, IDESC, t > 0 || ks > 0);
      }
    }
    tc::mma_commit(tc::smem_u32(&bar[b]));
  };
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its cells) and channels 16 (w / 4) ..
  auto epilogue = [&](int x0, int y, int z, int b) {
    const int lb = 32 * (warp & 3), hf = warp >> 2, x = x0 + lb + (tid & 31);
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)lb << 16) + 32 * b + 16 * hf, v);
    tc::tmem_wait_ld();
    if (x < X) {
      __half2 hv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) hv[j] = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
      uint4* o = reinterpret_cast<uint4*>(out + (x + (int64_t)X * (y + (int64_t)Y * z)) * NC + 16 * hf);
      o[0] = reinterpret_cast<const uint4*>(hv)[0];
      o[1] = reinterpret_cast<const uint4*>(hv)[1];
    }
  };
  int64_t issued = 0;                        // tiles issued by this CTA
  bool pend = false;                         // a tile whose MMAs may still run
  int px0 = 0, py = 0, pz = 0, pb = 0;
  int64_t pi = 0;
  auto wait_pending = [&]() {
    if (!tc::mbar_wait(tc::smem_u32(&bar[pb]), (uint32_t)((pi >> 1) & 1))) atomicOr(err, 16);
    tc::fence_after_sync();
  };
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int tx = (int)(u % ntx);
    const int64_t r = u / ntx;
    const int z = (int)(r % Z), yr = (int)(r / Z);
    const int x0 = tx * CT_M, y0 = yr * CT_YRUN, y1 = min(Y, y0 + CT_YRUN);
    if (pend) {  // the ring is rewritten below: the last tile's MMAs must be done
      wait_pending();
      epilogue(px0, py, pz, pb);
      pend = false;
    }
    cp_async_wait_all();  // no copy of the previous unit still writes the ring
    tc::fence_before_sync();
    __syncthreads();
    load_slab(x0, y0 - 1, z);
    load_slab(x0, y0, z);
    load_slab(x0, y0 + 1, z);
    cp_async_commit();
    if (y0 + 1 < y1) load_slab(x0, y0 + 2, z);  // for tile y0 + 1
    cp_async_commit();
    cp_async_wait_prev();
    tc::fence_proxy_async_smem();
    __syncthreads();
    for (int y = y0; y < y1; ++y) {
      const int b = (int)(issued & 1);
      if (tid == 0) issue(y, b);
      if (pend) wait_pending();                   // tile y - 1 read the slot of slab y + 3
      if (y + 2 < y1) load_slab(x0, y + 3, z);    // for tile y + 2
      cp_async_commit();                          // (empty at the end of the run)
      if (pend) epilogue(px0, py, pz, pb);
      pend = true;
      px0 = x0; py = y; pz = z; pb = b; pi = issued;
      ++issued;
      cp_async_wait_prev();                       // slab y + 2, for tile y + 1, has arrived
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  if (pend) {
    wait_pending();
    epilogue(px0, py, pz, pb);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// ---- weight gradients (CUDA cores, per-block partials, fixed-order reduce) ----
// G2[co][ci][t] += sum_x P[x][co] Q[x + off_t][ci] for two (P, Q) pairs.
// Tile 4 x 4 x 4 cells, halo 6 x 6 x 6; thread (co = tid / 8, ci = 4 (tid % 8) .. +3).
constexpr int GT = 4, GH = GT + 2, GHC = GH * GH * GH, GTC = GT * GT * GT;

__global__ void __launch_bounds__(256) k_dW2(int X, int Y, int Z, const __half* __restrict__ P1,
                                             const __half* __restrict__ Q1, const __half* __restrict__ P2,
                                             const __half* __restrict__ Q2, float* __restrict__ part) {
  __shared__ __align__(16) __half ps[GTC * NC];
  __shared__ __align__(16) __half qs[GHC * NC];
  const int tid = threadIdx.x, co = tid >> 3, ci = (tid & 7) * 4;
  float acc[NT][4];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[t][j] = 0.f;
  const int ntx = (X + GT - 1) / GT, nty = (Y + GT - 1) / GT, ntz = (Z + GT - 1) / GT;
  const int64_t ntiles = (int64_t)ntx * nty * ntz;
  for (int pass = 0; pass < 2; ++pass) {
    const __half* P = pass ? P2 : P1;
    const __half* Q = pass ? Q2 : Q1;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int x0 = (int)(tile % ntx) * GT, y0 = (int)((tile / ntx) % nty) * GT,
                z0 = (int)(tile / ((int64_t)ntx * nty)) * GT;
      __syncthreads();
      for (int i = tid; i < GTC * 4; i += blockDim.x) {
        int cell = i >> 2, ch = (i & 3) * 8;
        int gx = x0 + cell % GT, gy = y0 + (cell / GT) % GT, gz = z0 + cell / (GT * GT);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gx < X && gy < Y && gz < Z)
          v = *reinterpret_cast<const uint4*>(P + (gx + (int64_t)X * (gy + (int64_t)Y * gz)) * NC + ch);
        *reinterpret_cast<uint4*>(ps + cell * NC + ch) = v;
      }
      for (int i = tid; i < GHC * 4; i += blockDim.x) {
        int cell = i >> 2, ch = (i & 3) * 8;
        int gx = x0 - 1 + cell % GH, gy = y0 - 1 + (cell / GH) % GH, gz = z0 - 1 + cell / (GH * GH);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gx >= 0 && gx < X && gy >= 0 && gy < Y && gz >= 0 && gz < Z)
          v = *reinterpret_cast<const uint4*>(Q + (gx + (int64_t)X * (gy + (int64_t)Y * gz)) * NC + ch);
        *reinterpret_cast<uint4*>(qs + cell * NC + ch) = v;
      }
      __syncthreads();
      for (int cell = 0; cell < GTC; ++cell) {
        const float p = __half2float(ps[cell * NC + co]);
        const int cx = cell % GT, cy = (cell / GT) % GT, cz = cell / (GT * GT);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int hc = (cx + t % 3) + GH * ((cy + (t / 3) % 3) + GH * (cz + t / 9));
          const __half2* q2 = reinterpret_cast<const __half2*>(qs + hc * NC + ci);
          float2 qa = __half22float2(q2[0]), qb = __half22float2(q2[1]);
          acc[t][0] = fmaf(p, qa.x, acc[t][0]);
          acc[t][1] = fmaf(p, qa.y, acc[t][1]);
          acc[t][2] = fmaf(p, qb.x, acc[t][2]);
          acc[t][3] = fmaf(p, qb.y, acc[t][3]);
        }
      }
    }
  }
  float* o = part + (size_t)blockIdx.x * NC * NC * NT;
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) o[(co * NC + ci + j) * NT + t] = acc[t][j];
}

// G1[co][t] += sum_x (P1[x][co] q1(x + off_t) + P2[x][co] q2(x + off_t)); one thread per (co, t)
__global__ void k_dW1(int X, int Y, int Z, const __half* __restrict__ P1, const float* __restrict__ q1,
                      const __half* __restrict__ P2, const float* __restrict__ q2, float* __restrict__ part) {
  const int64_t n = (int64_t)X * Y * Z;
  const int e = threadIdx.x;  // blockDim.x == NC * NT
  const int co = e % NC, t = e / NC;
  const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  float acc = 0.f;
  for (int64_t c = lo; c < hi; ++c) {
    int I, J, K;
    cell_ijk(c, X, Y, I, J, K);
    int i = I + dx, j = J + dy, k = K + dz;
    if (i < 0 || i >= X || j < 0 || j >= Y || k < 0 || k >= Z) continue;
    int64_t nb = i + (int64_t)X * (j + (int64_t)Y * k);
    acc = fmaf(__half2float(P1[c * NC + co]), q1[nb], acc);
    acc = fmaf(__half2float(P2[c * NC + co]), q2[nb], acc);
  }
  part[(size_t)blockIdx.x * NC * NT + co * NT + t] = acc;
}

// out[i] (+)= scale * sum_b part[b][i]  (fixed order)
__global__ void k_reduce_part(int nparts, int len, const float* __restrict__ part, double scale,
                              float* __restrict__ out, int accumulate) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += (double)part[(size_t)b * len + i];
  out[i] = accumulate ? out[i] + (float)(scale * s) : (float)(scale * s);
}

// FP16 compute copies: W1h[t][co] = W1[co][t]; W2h[t][o][i] = W2[o][i][t];
// W2Th[t][o][i] = W2[i][o][26 - t] (adjoint: flipped taps, swapped channels)
__global__ void k_weights_h(const float* __restrict__ W1, const float* __restrict__ W2, __half* __restrict__ W1h,
                            __half* __restrict__ W2h, __half* __restrict__ W2Th) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < NC * NT) {
    int co = e / NT, t = e % NT;
    W1h[t * NC + co] = __float2half(W1[e]);
  }
  if (e < NC * NC * NT) {
    int o = e / (NC * NT), i = (e / NT) % NC, t = e % NT;
    W2h[(t * NC + o) * NC + i] = __float2half(W2[e]);
    W2Th[((NT - 1 - t) * NC + i) * NC + o] = __float2half(W2[e]);
  }
}

// Adam (Kingma & Ba 2015) on FP32 master weights
__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// err = e - y - qr
__global__ void k_err(int64_t n, const double* __restrict__ e, const double* __restrict__ y,
                      const double* __restrict__ qr, double* __restrict__ err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  err[i] = e[i] - y[i] - (qr ? qr[i] : 0.0);
}
// b4 = sigma s (-2 Serr / eSe): dL/dN for the normalised network input
// scal: [0] sumsq, [1] sigma, [2] eSe
__global__ void k_b4(int64_t n, const double* __restrict__ serr, const float* __restrict__ sq,
                     const double* __restrict__ scal, float* __restrict__ b4) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  b4[i] = (float)(-2.0 * serr[i] / scal[2] * scal[1] * (double)sq[i]);
}
// in-place b4 /= tau, tau = sqrt(sumsq / n) at scal[3]; scal[4] <- tau
__global__ void k_norm_b4(int64_t n, float* __restrict__ b4, double* __restrict__ scal) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double tau = sqrt(scal[3] / (double)n);
  if (!(tau > 0.0)) tau = 1.0;
  if (i == 0) scal[4] = tau;
  if (i >= n) return;
  b4[i] = (float)((double)b4[i] / tau);
}

}  // namespace

// ---------------------------------------------------------------------------
struct LearnedNet {
  int X = 0, Y = 0, Z = 0;
  int64_t n = 0;
  double delta = 1e-3;
  float *W1 = nullptr, *W2 = nullptr, *m1 = nullptr, *v1 = nullptr, *m2 = nullptr, *v2 = nullptr;
  float *g1 = nullptr, *g2 = nullptr;
  int adam_t = 0;
  __half *W1h = nullptr, *W2h = nullptr, *W2Th = nullptr;
  float* sq = nullptr;
  double* dinv = nullptr;
  float *u = nullptr, *b4 = nullptr;
  __half *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;
  float* part = nullptr;
  double* red = nullptr;   // RED_BLOCKS partials
  double* scal = nullptr;  // small device scalars
  double *y = nullptr, *err = nullptr, *serr = nullptr;
  double* pcg_q = nullptr;                             // CG work vector
  double *pr = nullptr, *pe = nullptr, *pq = nullptr;  // training pairs
  int npairs = 0;
  int conv_blocks = 0, dw2_blocks = 0, dw1_blocks = 0;
  int conv_engine = 0;  // 32 -> 32 convolutions: 0 = tcgen05 (k_conv2_tc), 1 = mma.sync (k_conv2)
  int sms = 1;
};

namespace {

template <typename T>
hd_status lalloc(hd_op* h, T** p, int64_t n) {
  if (cudaMalloc(p, sizeof(T) * (n > 0 ? n : 1)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "learned net buffers");
  return HD_OK;
}

hd_status net_sumsq_f(hd_op* h, const float* a, int64_t n, double* out) {
  k_sumsq_partial<float><<<RED_BLOCKS, TPB, 0, h->stream>>>(n, a, nullptr, h->net->red);
  k_final_sum<<<1, RED_BLOCKS, 0, h->stream>>>(h->net->red, out);
  HD_LAUNCH_CK(h, "sumsq");
  return HD_OK;
}
hd_status net_dot(hd_op* h, const double* a, const double* b, int64_t n, double* out) {
  k_dot_partial_l<<<RED_BLOCKS, TPB, 0, h->stream>>>(n, a, b, h->net->red);
  k_final_sum<<<1, RED_BLOCKS, 0, h->stream>>>(h->net->red, out);
  HD_LAUNCH_CK(h, "dot");
  return HD_OK;
}

hd_status conv2(hd_op* h, const __half* W, const __half* in, __half* out) {
  LearnedNet* N = h->net;
  if (N->conv_engine == 0) {
    static bool attr_tc[HD_MAX_DEVICES] = {};
    bool* done = device_flag(attr_tc);
    if (!done || !*done) {
      cudaError_t e = cudaFuncSetAttribute(k_conv2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, CT_SMEM);
      if (e != cudaSuccess) return hd_cuda_check(h, e, "cudaFuncSetAttribute(k_conv2_tc)");
      if (done) *done = true;
    }
    prof_mark(h, true);
    k_conv2_tc<<<N->sms, CT_THREADS, CT_SMEM, h->stream>>>(N->X, N->Y, N->Z, W, in, out, h->d_kerr);
    prof_mark(h, false);
    HD_LAUNCH_CK(h, "k_conv2_tc");
    return HD_OK;
  }
  const size_t smem = (size_t)(NT * NC * NC + HCELLS * NC) * sizeof(__half);
  static bool attr[HD_MAX_DEVICES] = {};
  bool* done = device_flag(attr);
  if (!done || !*done) {
    cudaError_t e = cudaFuncSetAttribute(k_conv2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return hd_cuda_check(h, e, "cudaFuncSetAttribute(k_conv2)");
    if (done) *done = true;
  }
  prof_mark(h, true);
  k_conv2<<<N->conv_blocks, 256, smem, h->stream>>>(N->X, N->Y, N->Z, W, in, out);
  prof_mark(h, false);
  HD_LAUNCH_CK(h, "k_conv2");
  return HD_OK;
}

// y = P_L r (net part, FP64 out; accumulate: y += P_L r); leaves u, a1, a2, a3 and sigma
// (scal[1]) for a backward pass
hd_status net_forward(hd_op* h, const double* r, double* y, bool accumulate = false) {
  LearnedNet* N = h->net;
  const int64_t n = N->n;
  hd_status st;
  k_sumsq_partial<double><<<RED_BLOCKS, TPB, 0, h->stream>>>(n, r, N->sq, N->red);
  k_sigma<<<1, RED_BLOCKS, 0, h->stream>>>(N->red, N->scal, n);
  k_make_u<<<nblk(n), TPB, 0, h->stream>>>(n, r, N->sq, N->scal, N->u);
  k_conv1<<<nblk(n), TPB, 0, h->stream>>>(N->X, N->Y, N->Z, N->W1h, N->u, N->a1);
  HD_LAUNCH_CK(h, "conv1");
  if ((st = conv2(h, N->W2h, N->a1, N->a2)) != HD_OK) return st;
  if ((st = conv2(h, N->W2Th, N->a2, N->a3)) != HD_OK) return st;
  k_conv1T<<<nblk(n), TPB, 0, h->stream>>>(N->X, N->Y, N->Z, N->W1h, N->a3, accumulate ? 2 : 0, N->sq, N->scal,
                                            N->delta, r, N->dinv, y, nullptr);
  HD_LAUNCH_CK(h, "conv1T");
  return HD_OK;
}

// Loss of one pair and its weight gradient, accumulated into g1/g2 (accumulate != 0)
hd_status net_pair_grad(hd_op* h, const double* r, const double* e, const double* qr, double* d_loss_out,
                        int accumulate) {
  LearnedNet* N = h->net;
  const int64_t n = N->n;
  hd_status st;
  if ((st = net_forward(h, r, N->y)) != HD_OK) return st;
  k_err<<<nblk(n), TPB, 0, h->stream>>>(n, e, N->y, qr, N->err);
  if ((st = schur_apply(h, N->err, N->serr)) != HD_OK) return st;
  // eSe at scal[2]: e . S e, using y as scratch for S e
  if ((st = schur_apply(h, e, N->y)) != HD_OK) return st;
  if ((st = net_dot(h, e, N->y, n, N->scal + 2)) != HD_OK) return st;
  if ((st = net_dot(h, N->err, N->serr, n, N->scal + 5)) != HD_OK) return st;
  // loss = errSerr / eSe (host reads scal[5] / scal[2])
  k_b4<<<nblk(n), TPB, 0, h->stream>>>(n, N->serr, N->sq, N->scal, N->b4);
  if ((st = net_sumsq_f(h, N->b4, n, N->scal + 3)) != HD_OK) return st;
  k_norm_b4<<<nblk(n), TPB, 0, h->stream>>>(n, N->b4, N->scal);
  k_conv1<<<nblk(n), TPB, 0, h->stream>>>(N->X, N->Y, N->Z, N->W1h, N->b4, N->b3);
  HD_LAUNCH_CK(h, "backward conv1");
  if ((st = conv2(h, N->W2h, N->b3, N->b2)) != HD_OK) return st;
  if ((st = conv2(h, N->W2Th, N->b2, N->b1)) != HD_OK) return st;
  k_dW2<<<N->dw2_blocks, 256, 0, h->stream>>>(N->X, N->Y, N->Z, N->b2, N->a1, N->a2, N->b3, N->part);
  HD_LAUNCH_CK(h, "k_dW2");
  // tau (scal[4]) scales the gradient back; read on the host to pass as a kernel scale
  double tau = 0.0, lossv[6];
  HD_CK(h, cudaMemcpyAsync(lossv, N->scal, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  tau = lossv[4];
  if (d_loss_out) *d_loss_out += lossv[5] / lossv[2];
  k_reduce_part<<<(NC * NC * NT + 255) / 256, 256, 0, h->stream>>>(N->dw2_blocks, NC * NC * NT, N->part, tau, N->g2,
                                                                   accumulate);
  k_dW1<<<N->dw1_blocks, NC * NT, 0, h->stream>>>(N->X, N->Y, N->Z, N->b1, N->u, N->a3, N->b4, N->part);
  k_reduce_part<<<(NC * NT + 255) / 256, 256, 0, h->stream>>>(N->dw1_blocks, NC * NT, N->part, tau, N->g1,
                                                              accumulate);
  HD_LAUNCH_CK(h, "weight gradients");
  return HD_OK;
}

hd_status refresh_half(hd_op* h) {
  LearnedNet* N = h->net;
  k_weights_h<<<(NC * NC * NT + 255) / 256, 256, 0, h->stream>>>(N->W1, N->W2, N->W1h, N->W2h, N->W2Th);
  HD_LAUNCH_CK(h, "weights to FP16");
  return HD_OK;
}

// S~ e = r by conjugate gradients preconditioned with the V-cycle (FP64), to rtol.
hd_status pcg_schur(hd_op* h, const double* r, double* e, double rtol, int maxit, int* its) {
  LearnedNet* N = h->net;
  const int64_t n = N->n;
  double *res = N->y, *z = N->err, *p = N->serr, *q = N->pcg_q;
  hd_status st;
  HD_CK(h, cudaMemsetAsync(e, 0, sizeof(double) * n, h->stream));
  HD_CK(h, cudaMemcpyAsync(res, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  if ((st = vcycle_apply(h, res, z)) != HD_OK) return st;
  if (h->singular && (st = project_mean(h, z)) != HD_OK) return st;
  HD_CK(h, cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  double hv[2];
  if ((st = net_dot(h, res, z, n, N->scal + 6)) != HD_OK) return st;
  if ((st = net_dot(h, res, res, n, N->scal + 7)) != HD_OK) return st;
  HD_CK(h, cudaMemcpyAsync(hv, N->scal + 6, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  double rz = hv[0], r0 = std::sqrt(hv[1]);
  int it = 0;
  for (it = 0; it < maxit && r0 > 0; ++it) {
    if ((st = schur_apply(h, p, q)) != HD_OK) return st;
    if ((st = net_dot(h, p, q, n, N->scal + 6)) != HD_OK) return st;
    HD_CK(h, cudaMemcpyAsync(hv, N->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HD_CK(h, cudaStreamSynchronize(h->stream));
    double alpha = rz / hv[0];
    if ((st = axpy_dev(h, n, alpha, p, e)) != HD_OK) return st;
    if ((st = axpy_dev(h, n, -alpha, q, res)) != HD_OK) return st;
    if ((st = net_dot(h, res, res, n, N->scal + 7)) != HD_OK) return st;
    if ((st = vcycle_apply(h, res, z)) != HD_OK) return st;
    if (h->singular && (st = project_mean(h, z)) != HD_OK) return st;
    if ((st = net_dot(h, res, z, n, N->scal + 6)) != HD_OK) return st;
    HD_CK(h, cudaMemcpyAsync(hv, N->scal + 6, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    HD_CK(h, cudaStreamSynchronize(h->stream));
    if (std::sqrt(hv[1]) <= rtol * r0) { ++it; break; }
    double beta = hv[0] / rz;
    rz = hv[0];
    if ((st = xpay_dev(h, n, z, beta, p)) != HD_OK) return st;  // p = z + beta p
  }
  if (its) *its = it;
  return HD_OK;
}

}  // namespace

void learned_free(hd_op* h) {
  LearnedNet* N = h->net;
  if (!N) return;
  void* ptrs[] = {N->W1, N->W2, N->m1, N->v1, N->m2, N->v2, N->g1, N->g2, N->W1h, N->W2h, N->W2Th, N->sq,
                  N->dinv, N->u, N->b4, N->a1, N->a2, N->a3, N->b1, N->b2, N->b3, N->part, N->red, N->scal,
                  N->y, N->err, N->serr, N->pcg_q, N->pr, N->pe, N->pq};
  for (void* p : ptrs) cudaFree(p);
  delete N;
  h->net = nullptr;
}

// z += P_L r (the network term); FP64 in/out
hd_status learned_net_add(hd_op* h, const double* r, double* z) { return net_forward(h, r, z, true); }

// z = V r + P_L r (learned Schur preconditioner on an L2 vector); FP64 in/out
hd_status learned_schur_apply(hd_op* h, const double* r, double* z) {
  hd_status st = vcycle_apply(h, r, z);
  if (st != HD_OK) return st;
  return net_forward(h, r, z, true);
}

extern "C" {

hd_status hd_learned_init(hd_handle h, int32_t nc, uint64_t seed, double delta) {
  if (!h || nc != NC || !(delta >= 0)) return HD_ERR_INVALID_ARG;
  learned_free(h);
  LearnedNet* N = new (std::nothrow) LearnedNet();
  if (!N) return HD_ERR_OOM;
  h->net = N;
  N->X = h->L.X; N->Y = h->L.Y; N->Z = h->L.Z;
  N->n = h->n_l2;
  N->delta = delta;
  const int64_t n = N->n, nw1 = NC * NT, nw2 = NC * NC * NT;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  N->conv_blocks = 2 * (sms > 0 ? sms : 1);
  N->sms = sms > 0 ? sms : 1;
  N->dw2_blocks = 2 * (sms > 0 ? sms : 1);
  N->dw1_blocks = sms > 0 ? sms : 1;
  hd_status st = HD_OK;
  do {
    if ((st = lalloc(h, &N->W1, nw1)) || (st = lalloc(h, &N->W2, nw2)) || (st = lalloc(h, &N->m1, nw1)) ||
        (st = lalloc(h, &N->v1, nw1)) || (st = lalloc(h, &N->m2, nw2)) || (st = lalloc(h, &N->v2, nw2)) ||
        (st = lalloc(h, &N->g1, nw1)) || (st = lalloc(h, &N->g2, nw2)) || (st = lalloc(h, &N->W1h, nw1)) ||
        (st = lalloc(h, &N->W2h, nw2)) || (st = lalloc(h, &N->W2Th, nw2)) || (st = lalloc(h, &N->sq, n)) ||
        (st = lalloc(h, &N->dinv, n)) || (st = lalloc(h, &N->u, n)) || (st = lalloc(h, &N->b4, n)) ||
        (st = lalloc(h, &N->a1, n * NC)) || (st = lalloc(h, &N->a2, n * NC)) || (st = lalloc(h, &N->a3, n * NC)) ||
        (st = lalloc(h, &N->b1, n * NC)) || (st = lalloc(h, &N->b2, n * NC)) || (st = lalloc(h, &N->b3, n * NC)) ||
        (st = lalloc(h, &N->part, (int64_t)N->dw2_blocks * nw2)) || (st = lalloc(h, &N->red, RED_BLOCKS)) ||
        (st = lalloc(h, &N->scal, 16)) || (st = lalloc(h, &N->y, n)) || (st = lalloc(h, &N->err, n)) ||
        (st = lalloc(h, &N->serr, n)) || (st = lalloc(h, &N->pcg_q, n)))
      break;
    // seeded initial weights (splitmix64 -> Box-Muller), scaled like the reference init
    std::vector<float> w1(nw1), w2(nw2);
    uint64_t s = seed;
    auto next = [&]() {
      s += 0x9E3779B97F4A7C15ull;
      uint64_t z = s;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return ((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    auto gauss = [&]() {
      double u1 = next(), u2 = next();
      if (u1 < 1e-300) u1 = 1e-300;
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    };
    // small: the network term starts four orders of magnitude below its unit-scale size,
    // so the preconditioner starts at the plain cycle
    for (auto& v : w1) v = (float)(0.1 * gauss() / std::sqrt(27.0));
    for (auto& v : w2) v = (float)(0.1 * gauss() / std::sqrt(27.0 * NC));
    HD_CK(h, cudaMemcpyAsync(N->W1, w1.data(), nw1 * 4, cudaMemcpyHostToDevice, h->stream));
    HD_CK(h, cudaMemcpyAsync(N->W2, w2.data(), nw2 * 4, cudaMemcpyHostToDevice, h->stream));
    HD_CK(h, cudaMemsetAsync(N->m1, 0, nw1 * 4, h->stream));
    HD_CK(h, cudaMemsetAsync(N->v1, 0, nw1 * 4, h->stream));
    HD_CK(h, cudaMemsetAsync(N->m2, 0, nw2 * 4, h->stream));
    HD_CK(h, cudaMemsetAsync(N->v2, 0, nw2 * 4, h->stream));
    k_sq<<<nblk(n), TPB, 0, h->stream>>>(n, h->lv[0].diag, N->sq, N->dinv);
    HD_LAUNCH_CK(h, "k_sq");
    if ((st = refresh_half(h)) != HD_OK) break;
    HD_CK(h, cudaStreamSynchronize(h->stream));
  } while (0);
  if (st != HD_OK) learned_free(h);
  return st;
}

hd_status hd_learned_set_weights(hd_handle h, const float* W1, const float* W2) {
  if (!h || !h->net || !W1 || !W2) return HD_ERR_INVALID_ARG;
  LearnedNet* N = h->net;
  HD_CK(h, cudaMemcpyAsync(N->W1, W1, NC * NT * 4, cudaMemcpyHostToDevice, h->stream));
  HD_CK(h, cudaMemcpyAsync(N->W2, W2, NC * NC * NT * 4, cudaMemcpyHostToDevice, h->stream));
  hd_status st = refresh_half(h);
  if (st != HD_OK) return st;
  HD_CK(h, cudaStreamSynchronize(h->stream));
  return HD_OK;
}

hd_status hd_learned_get_weights(hd_handle h, float* W1, float* W2) {
  if (!h || !h->net || !W1 || !W2) return HD_ERR_INVALID_ARG;
  HD_CK(h, cudaMemcpyAsync(W1, h->net->W1, NC * NT * 4, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaMemcpyAsync(W2, h->net->W2, NC * NC * NT * 4, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  return HD_OK;
}

hd_status hd_learned_apply(hd_handle h, const double* r, double* z) {
  if (!h || !h->net || !r || !z || r == z) return HD_ERR_INVALID_ARG;
  return net_forward(h, r, z);
}

hd_status hd_learned_grad(hd_handle h, int32_t npairs, const double* r, const double* e, const double* qr,
                          float* gW1, float* gW2, double* loss) {
  if (!h || !h->net || npairs < 1 || !r || !e || !gW1 || !gW2 || !loss) return HD_ERR_INVALID_ARG;
  LearnedNet* N = h->net;
  double L = 0.0;
  for (int p = 0; p < npairs; ++p) {
    hd_status st = net_pair_grad(h, r + (size_t)p * N->n, e + (size_t)p * N->n, qr ? qr + (size_t)p * N->n : nullptr,
                                 &L, p > 0);
    if (st != HD_OK) return st;
  }
  HD_CK(h, cudaMemcpyAsync(gW1, N->g1, NC * NT * 4, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaMemcpyAsync(gW2, N->g2, NC * NC * NT * 4, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  *loss = L;
  return HD_OK;
}

hd_status hd_coarse_correction(hd_handle h, const double* r, double* z) {
  if (!h || !r || !z || r == z) return HD_ERR_INVALID_ARG;
  HD_CK(h, cudaMemsetAsync(z, 0, sizeof(double) * h->n_l2, h->stream));
  return coarse_correction(h, r, z);
}

hd_status hd_learned_train(hd_handle h, const hd_train_opts* o, hd_train_info* info) {
  if (!h || !h->net || !o || o->npairs < 1 || o->steps < 0 || !(o->lr > 0)) return HD_ERR_INVALID_ARG;
  LearnedNet* N = h->net;
  const int64_t n = N->n, ntot = h->n_rt + h->n_l2;
  hd_status st;
  cudaEvent_t e0, e1;
  HD_CK(h, cudaEventCreate(&e0));
  HD_CK(h, cudaEventCreate(&e1));
  HD_CK(h, cudaEventRecord(e0, h->stream));
  // 1. residuals the plain solver feeds its Schur preconditioner: the q parts of the
  //    Lanczos vectors of a plain MINRES solve with a seeded random right-hand side
  if (N->npairs < o->npairs) {
    cudaFree(N->pr); cudaFree(N->pe); cudaFree(N->pq);
    N->pr = N->pe = N->pq = nullptr;
    if ((st = lalloc(h, &N->pr, n * o->npairs)) || (st = lalloc(h, &N->pe, n * o->npairs)) ||
        (st = lalloc(h, &N->pq, n * o->npairs)))
      return st;
    N->npairs = o->npairs;
  }
  double *b = nullptr, *x = nullptr;
  if ((st = lalloc(h, &b, ntot)) || (st = lalloc(h, &x, ntot))) return st;
  {
    std::vector<double> hb(ntot);
    uint64_t s = o->seed;
    for (auto& v : hb) {
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      v = ((s >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
    }
    HD_CK(h, cudaMemcpyAsync(b, hb.data(), ntot * 8, cudaMemcpyHostToDevice, h->stream));
    // a consistent right-hand side when S~ is singular: zero-mean q part
    if (h->singular && (st = project_mean(h, b + h->n_rt)) != HD_OK) return st;
  }
  const int mode_save = h->schur_mode;
  h->schur_mode = 0;
  h->cap_buf = N->pr;
  h->cap_every = o->capture_every > 0 ? o->capture_every : 1;
  h->cap_max = o->npairs;
  h->cap_count = 0;
  hd_solve_opts so{};
  so.rtol = 1e-12;
  so.maxit = h->cap_every * o->npairs;
  so.check_every = 16;
  hd_solve_info si{};
  minres_run(h, b, x, &so, &si);
  h->cap_buf = nullptr;
  h->schur_mode = mode_save;
  const int np = h->cap_count;
  cudaFree(b);
  cudaFree(x);
  if (np < 1) return hd_fail(h, HD_ERR_NOT_CONVERGED, "no residuals captured");
  // 2. targets e = S~^-1 r by V-cycle-preconditioned CG, and the fixed part V r (the
  //    V/W-cycle the network is added to; zero mean in the singular case, as applied)
  int max_pcg = 0;
  for (int p = 0; p < np; ++p) {
    int its = 0;
    if ((st = pcg_schur(h, N->pr + p * n, N->pe + p * n, 1e-10, 2000, &its)) != HD_OK) return st;
    max_pcg = its > max_pcg ? its : max_pcg;
    if ((st = vcycle_apply(h, N->pr + p * n, N->pq + p * n)) != HD_OK) return st;
    if (h->singular && (st = project_mean(h, N->pq + p * n)) != HD_OK) return st;
  }
  // 3. Adam on the mean energy-norm loss over the pairs
  double L0 = 0.0, L = 0.0;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int step = 0; step <= o->steps; ++step) {
    L = 0.0;
    for (int p = 0; p < np; ++p)
      if ((st = net_pair_grad(h, N->pr + p * n, N->pe + p * n, N->pq + p * n, &L, p > 0)) != HD_OK) return st;
    L /= np;
    if (step == 0) L0 = L;
    if (step == o->steps) break;
    N->adam_t++;
    const float c1 = 1.f - std::pow(b1, (float)N->adam_t), c2 = 1.f - std::pow(b2, (float)N->adam_t);
    const float lr = (float)o->lr;
    // g holds the sum over pairs = np x the gradient of the mean; Adam's step is
    // invariant to that scale except through epsilon, which is scaled with it
    const float eps = 1e-8f * (float)np;
    k_adam<<<(NC * NT + 255) / 256, 256, 0, h->stream>>>(NC * NT, N->W1, N->g1, N->m1, N->v1, lr, b1, b2, eps, c1,
                                                         c2);
    k_adam<<<(NC * NC * NT + 255) / 256, 256, 0, h->stream>>>(NC * NC * NT, N->W2, N->g2, N->m2, N->v2, lr, b1, b2,
                                                              eps, c1, c2);
    HD_LAUNCH_CK(h, "adam");
    if ((st = refresh_half(h)) != HD_OK) return st;
  }
  HD_CK(h, cudaEventRecord(e1, h->stream));
  HD_CK(h, cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->pairs = np;
    info->loss_initial = L0;
    info->loss_final = L;
    info->pcg_max_iterations = max_pcg;
    info->ms_total = ms;
  }
  return HD_OK;
}

hd_status hd_set_schur_prec(hd_handle h, int32_t mode) {
  if (!h || (mode != 0 && mode != 1)) return HD_ERR_INVALID_ARG;
  if (mode == 1 && !h->net) return hd_fail(h, HD_ERR_INVALID_ARG, "learned preconditioner not initialised");
  h->schur_mode = mode;
  return HD_OK;
}

hd_status hd_enable_learned(hd_handle h, int32_t on) {
  if (!h || (on != 0 && on != 1)) return HD_ERR_INVALID_ARG;
  return hd_set_schur_prec(h, on);
}

// Network file: magic, channels, taps, delta, then W1 and W2 (FP32, host byte order).
struct NetFileHeader {
  char magic[8];
  int32_t nc, taps;
  double delta;
};
static const char kNetMagic[8] = {'H', 'D', 'L', 'N', 'E', 'T', '0', '1'};

hd_status hd_learned_save(hd_handle h, const char* path) {
  if (!h || !path) return HD_ERR_INVALID_ARG;
  if (!h->net) return hd_fail(h, HD_ERR_INVALID_ARG, "learned preconditioner not initialised");
  std::vector<float> w1(NC * NT), w2(NC * NC * NT);
  hd_status st = hd_learned_get_weights(h, w1.data(), w2.data());
  if (st != HD_OK) return st;
  NetFileHeader hd{};
  std::memcpy(hd.magic, kNetMagic, sizeof hd.magic);
  hd.nc = NC;
  hd.taps = NT;
  hd.delta = h->net->delta;
  FILE* f = std::fopen(path, "wb");
  if (!f) return hd_fail(h, HD_ERR_INVALID_ARG, std::string("learned save: cannot open ") + path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(w1.data(), 4, w1.size(), f) == w1.size() &&
            std::fwrite(w2.data(), 4, w2.size(), f) == w2.size();
  ok = std::fclose(f) == 0 && ok;
  return ok ? HD_OK : hd_fail(h, HD_ERR_INVALID_ARG, std::string("learned save: write failed: ") + path);
}

hd_status hd_learned_load(hd_handle h, const char* path) {
  if (!h || !path) return HD_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return hd_fail(h, HD_ERR_INVALID_ARG, std::string("learned load: cannot open ") + path);
  NetFileHeader hd{};
  std::vector<float> w1(NC * NT), w2(NC * NC * NT);
  std::string err;
  if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, kNetMagic, sizeof hd.magic) != 0)
    err = "not a learned-preconditioner file";
  else if (hd.nc != NC || hd.taps != NT || !(hd.delta >= 0))
    err = "network of another shape";
  else if (std::fread(w1.data(), 4, w1.size(), f) != w1.size() || std::fread(w2.data(), 4, w2.size(), f) != w2.size())
    err = "truncated file";
  else if (std::fgetc(f) != EOF)
    err = "trailing bytes after the weights";
  std::fclose(f);
  if (!err.empty()) return hd_fail(h, HD_ERR_INVALID_ARG, "learned load: " + err + ": " + path);
  hd_status st = HD_OK;
  if (!h->net || h->net->delta != hd.delta) st = hd_learned_init(h, NC, 0, hd.delta);
  if (st != HD_OK) return st;
  return hd_learned_set_weights(h, w1.data(), w2.data());
}

}  // extern "C"

extern "C" hd_status hd_learned_conv_engine(hd_handle h, int32_t engine) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (!h->net) return hd_fail(h, HD_ERR_INVALID_ARG, "hd_learned_init has not been called");
  if (engine != 0 && engine != 1) return hd_fail(h, HD_ERR_INVALID_ARG, "convolution engine: 0 or 1");
  h->net->conv_engine = engine;
  return HD_OK;
}
