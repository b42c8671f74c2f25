// DG mass inverse of any degree (Sec. 3.1): y = W^-1 x for the block-diagonal L2 mass
// W_e[a][b] = int_e alpha_e psi_a psi_b / det J, k = 2..9, by the approaches the paper
// compares: the explicit inverse (batched gemv), the Cholesky factor (two triangular
// solves), and the fused per-element CG in the Gauss-Legendre nodal basis or in the
// histopolation basis (Sec. 2.5). FP64 throughout; the degree is a run-time value (the
// block operator's kernels are compiled per degree up to k = 5).
//
// Layouts: L2 vectors in lattice order (cell I + X (J + Y Z), X = nx k, ...); element-
// local index a = a1 + k (a2 + k a3); per-element matrices [E][n][n] row-major, n = k^3;
// point values [E][q^3], p = p1 + q (p2 + q p3).
#include <cmath>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "hd_internal.h"
#include "k_l2elem.cuh"

#define MI_MAXK 9
#define MI_MAXQ 12

struct MiTab {
  int k, q;
  double B[MI_MAXQ * MI_MAXK];   // the basis the method works in, at the points: B[p k + a]
  double BH[MI_MAXQ * MI_MAXK];  // histopolation basis at the points (assembly)
  double TT[MI_MAXK * MI_MAXK];  // GL nodal -> histopolation coefficients (GL-basis CG)
  double gx[MI_MAXQ], gw[MI_MAXQ];
};

// the CG's tables in its arithmetic (double or double-float)
template <typename T>
struct MiCgTab {
  int k, q;
  T B[MI_MAXQ * MI_MAXK];
  T TT[MI_MAXK * MI_MAXK];
};

struct hd_massinv {
  int nx = 0, ny = 0, nz = 0, k = 0, q = 0, method = 0;
  int64_t E = 0, n = 0;          // elements, DOFs per element
  cudaStream_t stream = nullptr;
  MiTab tab{};
  MiCgTab<double> cgd{};
  MiCgTab<dfloat> cgx{};
  double* d_wdet = nullptr;      // [E][q^3] w_p alpha / det J
  double* d_diag = nullptr;      // [E][n] Jacobi diagonal (CG methods)
  double* d_mat = nullptr;       // [E][n][n] W_e^-1 (dense) or its Cholesky factor L (lower)
  double* d_aux = nullptr;       // setup scratch: [E][n][n] L^-1 (dense)
  int emul = 0;                  // CG stages in double-float (fp64_emulation = 1)
  dfloat* x_wdet = nullptr;      // [E][q^3] double-float copy of wdet
  dfloat* x_dinv = nullptr;      // [E][n] 1 / Jacobi diagonal, double-float
  int* d_flag = nullptr;         // [0]: det J <= 0; [1]: most CG iterations; [2]: a pivot <= 0
  double setup_ms = 0.0;
};

namespace {

constexpr int MI_THREADS = 256;
constexpr int TILE = 32;

// w_p alpha_e / det J(xi_p) on the trilinear element, one thread per (element, point)
__global__ void k_mi_geom(int64_t E, int nx, int ny, MiTab t, const double* __restrict__ vx,
                          const double* __restrict__ vy, const double* __restrict__ vz,
                          const double* __restrict__ alpha, double* __restrict__ wdet, int* __restrict__ flag) {
  const int q = t.q, nq = q * q * q;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= E * nq) return;
  const int64_t e = g / nq;
  const int p = (int)(g - e * nq), p1 = p % q, p2 = (p / q) % q, p3 = p / (q * q);
  const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
  const double xi[3] = {t.gx[p1], t.gx[p2], t.gx[p3]};
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // J[i][a] = d x_i / d xi_a
  for (int c = 0; c < 8; ++c) {
    const int b[3] = {c & 1, (c >> 1) & 1, c >> 2};
    const int64_t id = (ex + b[0]) + (int64_t)(nx + 1) * ((ey + b[1]) + (int64_t)(ny + 1) * (ez + b[2]));
    const double v[3] = {vx[id], vy[id], vz[id]};
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = b[d] ? xi[d] : 1.0 - xi[d];
      df[d] = b[d] ? 1.0 : -1.0;
    }
    const double dn[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) J[i][a] = fma(v[i], dn[a], J[i][a]);
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det > 0.0)) atomicExch(flag, 1);
  wdet[g] = t.gw[p1] * t.gw[p2] * t.gw[p3] * (alpha ? alpha[e] : 1.0) / det;
}

// Jacobi diagonal of W in the basis B: sum_p wdet_p B(p1,a1)^2 B(p2,a2)^2 B(p3,a3)^2
__global__ void k_mi_diag(int64_t E, MiTab t, const double* __restrict__ wdet, double* __restrict__ diag) {
  const int k = t.k, q = t.q, n = k * k * k;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= E * n) return;
  const int64_t e = g / n;
  const int a = (int)(g - e * n), a1 = a % k, a2 = (a / k) % k, a3 = a / (k * k);
  const double* w = wdet + e * (int64_t)q * q * q;
  double s = 0.0;
  for (int p3 = 0; p3 < q; ++p3) {
    const double b3 = t.B[p3 * k + a3] * t.B[p3 * k + a3];
    double s2 = 0.0;
    for (int p2 = 0; p2 < q; ++p2) {
      const double b2 = t.B[p2 * k + a2] * t.B[p2 * k + a2];
      double s1 = 0.0;
      for (int p1 = 0; p1 < q; ++p1) s1 = fma(t.B[p1 * k + a1] * t.B[p1 * k + a1], w[p1 + q * (p2 + q * p3)], s1);
      s2 = fma(b2, s1, s2);
    }
    s = fma(b3, s2, s);
  }
  diag[g] = s;
}


// ---- fused per-element CG (Sec. 2.5, 3.1) ----------------------------------------------
// The stages run in T: FP64, or double-float (pairs of FP32 numbers on the FP32 pipe, about
// 48 significant bits; the FP64 pipe of this GPU has 1/64 of the FP32 rate). The CG's
// inner products, step lengths and stopping test are FP64 in both.
__device__ __forceinline__ double mi_d(double v) { return v; }
__device__ __forceinline__ double mi_d(dfloat v) { return df_to_double(v); }
template <typename T>
__device__ __forceinline__ T mi_t(double v);
template <>
__device__ __forceinline__ double mi_t<double>(double v) { return v; }
template <>
__device__ __forceinline__ dfloat mi_t<dfloat>(double v) { return df_from_double(v); }



// one CTA per element: y_e = W_e^-1 x_e by Jacobi-preconditioned CG from zero, in the
// GL nodal basis (glb: right-hand side TT^T x, result TT a) or the histopolation basis
// (T = double: diag is the Jacobi diagonal; T = dfloat: its inverse)
template <typename T>
__global__ void __launch_bounds__(MI_THREADS)
k_mi_cg(int64_t E, int nx, int ny, MiCgTab<T> t, int glb, int maxit, double tol2, const T* __restrict__ wdet,
        const T* __restrict__ diag, const double* __restrict__ x, double* __restrict__ y, int* __restrict__ flag) {
  extern __shared__ __align__(16) unsigned char mi_smem[];
  const int k = t.k, q = t.q, n = k * k * k;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  T* B = reinterpret_cast<T*>(mi_smem);
  T* TT = B + q * k;
  T* A = TT + k * k;
  T* R = A + n;
  T* P = R + n;
  T* W = P + n;
  T* T1 = W + n;
  T* T2 = T1 + q * k * k;
  T* T3 = T2 + q * q * k;
  double* red = reinterpret_cast<double*>(T3 + q * q * q);
  for (int i = threadIdx.x; i < q * k; i += blockDim.x) B[i] = t.B[i];
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) TT[i] = t.TT[i];
  for (int a = threadIdx.x; a < n; a += blockDim.x) W[a] = mi_t<T>(x[mi_cell(e, a, k, nx, ny)]);
  __syncthreads();
  if (glb) mi_tt3(k, TT, true, W, T1, T2, R);
  else
    for (int a = threadIdx.x; a < n; a += blockDim.x) R[a] = W[a];
  __syncthreads();
  const T* D = diag + e * n;
  const T* wd = wdet + e * (int64_t)q * q * q;
  auto precond = [&](T r, int a) -> T {  // z = r / diag
    if constexpr (std::is_same<T, double>::value) return r / D[a];
    else return r * D[a];
  };
  double rz = 0.0, bb = 0.0;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const T r = R[a], z = precond(r, a);
    A[a] = T(0);
    P[a] = z;
    rz = fma(mi_d(r), mi_d(z), rz);
    bb = fma(mi_d(r), mi_d(r), bb);
  }
  rz = block_sum(rz, red);
  bb = block_sum(bb, red);
  int it = 0;
  if (bb > 0.0) {
    while (it < maxit) {
      mi_apply_w(k, q, B, wd, P, W, T1, T2, T3);
      double pw = 0.0;
      for (int a = threadIdx.x; a < n; a += blockDim.x) pw = fma(mi_d(P[a]), mi_d(W[a]), pw);
      pw = block_sum(pw, red);
      if (!(pw > 0.0)) {  // breakdown (W_e not positive definite, or a NaN)
        if (threadIdx.x == 0) atomicExch(flag + 2, 1);
        break;
      }
      const double alpha = rz / pw;
      const T at = mi_t<T>(alpha), mat = mi_t<T>(-alpha);
      double rr = 0.0, rzn = 0.0;
      for (int a = threadIdx.x; a < n; a += blockDim.x) {
        A[a] = fma(at, P[a], A[a]);
        const T r = fma(mat, W[a], R[a]);
        R[a] = r;
        const T z = precond(r, a);
        W[a] = z;
        const double rd = mi_d(r);
        rr = fma(rd, rd, rr);
        rzn = fma(rd, mi_d(z), rzn);
      }
      rr = block_sum(rr, red);
      rzn = block_sum(rzn, red);
      ++it;
      if (rr <= tol2 * bb) break;
      const T beta = mi_t<T>(rzn / rz);
      rz = rzn;
      for (int a = threadIdx.x; a < n; a += blockDim.x) P[a] = fma(beta, P[a], W[a]);
      __syncthreads();
    }
  }
  __syncthreads();
  const T* res = A;
  if (glb) {
    mi_tt3(k, TT, false, A, T1, T2, W);
    res = W;
  }
  for (int a = threadIdx.x; a < n; a += blockDim.x) y[mi_cell(e, a, k, nx, ny)] = mi_d(res[a]);
  if (threadIdx.x == 0) atomicMax(flag + 1, it);
}

// ---- direct methods: assembly and tiled factorisations in global memory ----------------
// W_e[a][b] = sum_p wd_p psi_a(p) psi_b(p), one CTA per element: M1[(a1, b1), p2, p3] =
// sum_p1 BH(p1,a1) BH(p1,b1) wd_p in shared memory, then every entry from M1 (q^2 terms)
__global__ void __launch_bounds__(MI_THREADS)
k_mi_assemble(int64_t E, MiTab t, const double* __restrict__ wdet, double* __restrict__ mat) {
  extern __shared__ double sm[];
  const int k = t.k, q = t.q, n = k * k * k, kk = k * k, qq = q * q;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  double* BH = sm;
  double* M1 = BH + q * k;
  for (int i = threadIdx.x; i < q * k; i += blockDim.x) BH[i] = t.BH[i];
  __syncthreads();
  const double* wd = wdet + e * (int64_t)qq * q;
  for (int i = threadIdx.x; i < kk * qq; i += blockDim.x) {
    const int ab = i % kk, r = i / kk, a1 = ab % k, b1 = ab / k;  // r = p2 + q p3
    double s = 0.0;
    for (int p = 0; p < q; ++p) s = fma(BH[p * k + a1] * BH[p * k + b1], wd[p + q * r], s);
    M1[i] = s;
  }
  __syncthreads();
  double* W = mat + e * (int64_t)n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int a = i / n, b = i - a * n;
    const int a1 = a % k, a2 = (a / k) % k, a3 = a / kk, b1 = b % k, b2 = (b / k) % k, b3 = b / kk;
    const double* m = M1 + (a1 + k * b1);
    double s = 0.0;
    for (int p3 = 0; p3 < q; ++p3) {
      double s2 = 0.0;
      for (int p2 = 0; p2 < q; ++p2) s2 = fma(BH[p2 * k + a2] * BH[p2 * k + b2], m[kk * (p2 + q * p3)], s2);
      s = fma(BH[p3 * k + a3] * BH[p3 * k + b3], s2, s);
    }
    W[i] = s;
  }
}

// 32 x 32 tiles of an n x n row-major matrix in shared memory (row stride 33); outside
// the matrix 0, or 1 on the diagonal of a diagonal tile (pad)
__device__ void tile_load(const double* A, int n, int I, int J, double* T, bool pad) {
  for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
    const int r = i / TILE, c = i % TILE, gi = I * TILE + r, gj = J * TILE + c;
    T[r * 33 + c] = (gi < n && gj < n) ? A[(int64_t)gi * n + gj] : ((pad && r == c) ? 1.0 : 0.0);
  }
}
__device__ void tile_store(double* A, int n, int I, int J, const double* T) {
  for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
    const int r = i / TILE, c = i % TILE, gi = I * TILE + r, gj = J * TILE + c;
    if (gi < n && gj < n) A[(int64_t)gi * n + gj] = T[r * 33 + c];
  }
}
// acc[j] += sum_l opA(r, l) opB(l, c0 + j) for this thread's row r = tid / 8 and columns
// c0 = 4 (tid % 8) .. c0 + 3 of a tile (256 threads); ta / tb: the operand transposed
__device__ __forceinline__ void tile_mma(const double* TA, bool ta, const double* TB, bool tb, double acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  for (int l = 0; l < TILE; ++l) {
    const double a = ta ? TA[l * 33 + r] : TA[r * 33 + l];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = fma(a, tb ? TB[(c0 + j) * 33 + l] : TB[l * 33 + c0 + j], acc[j]);
  }
}

// W_e = L L^T in place (lower triangle; the upper one is left undefined), right-looking by
// 32-column panels: factor the diagonal tile (one warp), solve the panel below it, update
// the trailing tiles. flag: a pivot that is not positive.
__global__ void __launch_bounds__(MI_THREADS) k_mi_potrf(int64_t E, int n, double* __restrict__ mat, int* flag) {
  // flag: the pivot flag word
  __shared__ double TD[TILE * 33], TA[TILE * 33], TB[TILE * 33];
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  double* A = mat + e * (int64_t)n * n;
  const int nb = (n + TILE - 1) / TILE, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int J = 0; J < nb; ++J) {
    tile_load(A, n, J, J, TD, true);
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < TILE; ++j) {
        if (lane == 0) {
          const double d = TD[j * 33 + j];
          if (!(d > 0.0)) atomicExch(flag, 1);
          TD[j * 33 + j] = sqrt(d > 0.0 ? d : 1.0);
        }
        __syncwarp();
        const double d = TD[j * 33 + j];
        if (lane > j) TD[lane * 33 + j] /= d;
        __syncwarp();
        if (lane > j)
          for (int l = j + 1; l <= lane; ++l) TD[lane * 33 + l] = fma(-TD[lane * 33 + j], TD[l * 33 + j], TD[lane * 33 + l]);
        __syncwarp();
      }
    }
    __syncthreads();
    tile_store(A, n, J, J, TD);
    // panel: row i below the diagonal tile, x L_JJ^T = a by forward substitution
    const int bc = min(TILE, n - J * TILE);
    for (int i = (J + 1) * TILE + threadIdx.x; i < n; i += blockDim.x) {
      double* row = A + (int64_t)i * n + J * TILE;  // solved in place, entry by entry
      for (int c = 0; c < bc; ++c) {
        double s = row[c];
        for (int l = 0; l < c; ++l) s = fma(-row[l], TD[c * 33 + l], s);
        row[c] = s / TD[c * 33 + c];
      }
    }
    __syncthreads();
    // trailing tiles A_IK -= L_IJ L_KJ^T, J < K <= I
    for (int I = J + 1; I < nb; ++I) {
      tile_load(A, n, I, J, TA, false);
      for (int K = J + 1; K <= I; ++K) {
        tile_load(A, n, K, J, TB, false);
        __syncthreads();
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        tile_mma(TA, false, TB, true, acc);
        const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4, gi = I * TILE + r;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int gj = K * TILE + c0 + j;
          if (gi < n && gj < n) A[(int64_t)gi * n + gj] -= acc[j];
        }
        __syncthreads();
      }
    }
  }
}

// Y = L^-1 (lower, in aux), then W_e^-1 = Y^T Y (full symmetric storage, over L in mat)
__global__ void __launch_bounds__(MI_THREADS) k_mi_potri(int64_t E, int n, double* __restrict__ mat,
                                                         double* __restrict__ aux) {
  __shared__ double TA[TILE * 33], TB[TILE * 33], TC[TILE * 33];
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  double* L = mat + e * (int64_t)n * n;
  double* Y = aux + e * (int64_t)n * n;
  const int nb = (n + TILE - 1) / TILE, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  // diagonal tiles: Y_II = L_II^-1, lane c computes column c
  for (int I = 0; I < nb; ++I) {
    tile_load(L, n, I, I, TA, true);
    __syncthreads();
    if (warp == 0) {
      const int c = lane;
      for (int rr = 0; rr < TILE; ++rr) {
        double s = 0.0;
        if (rr >= c) {
          s = (rr == c) ? 1.0 : 0.0;
          for (int l = c; l < rr; ++l) s = fma(-TA[rr * 33 + l], TB[l * 33 + c], s);
          s /= TA[rr * 33 + rr];
        }
        TB[rr * 33 + c] = s;
      }
    }
    __syncthreads();
    tile_store(Y, n, I, I, TB);
    __syncthreads();
  }
  // below the diagonal: Y_IJ = -Y_II sum_{K=J}^{I-1} L_IK Y_KJ, rows I ascending
  for (int J = 0; J < nb; ++J)
    for (int I = J + 1; I < nb; ++I) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int K = J; K < I; ++K) {
        tile_load(L, n, I, K, TA, false);
        tile_load(Y, n, K, J, TB, K == J);
        __syncthreads();
        tile_mma(TA, false, TB, false, acc);
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) TC[r * 33 + c0 + j] = acc[j];
      tile_load(Y, n, I, I, TA, true);
      __syncthreads();
      double out[4] = {0.0, 0.0, 0.0, 0.0};
      tile_mma(TA, false, TC, false, out);
#pragma unroll
      for (int j = 0; j < 4; ++j) TB[r * 33 + c0 + j] = -out[j];
      __syncthreads();
      tile_store(Y, n, I, J, TB);
      __syncthreads();
    }
  // W^-1_IJ = sum_{K >= I} Y_KI^T Y_KJ for I >= J, stored with its mirror
  for (int I = 0; I < nb; ++I)
    for (int J = 0; J <= I; ++J) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int K = I; K < nb; ++K) {
        tile_load(Y, n, K, I, TA, false);
        tile_load(Y, n, K, J, TB, false);
        if (K == I || K == J) {  // the upper part of a diagonal tile of Y is zero
          __syncthreads();
          for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
            const int rr = i / TILE, cc = i % TILE;
            if (K == I && cc > rr) TA[rr * 33 + cc] = 0.0;
            if (K == J && cc > rr) TB[rr * 33 + cc] = 0.0;
          }
        }
        __syncthreads();
        tile_mma(TA, true, TB, false, acc);
        __syncthreads();
      }
      const int gi0 = I * TILE + r;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gj = J * TILE + c0 + j;
        if (I == J && c0 + j > r) continue;  // a diagonal tile: each entry from its lower copy
        if (gi0 < n && gj < n) {
          L[(int64_t)gi0 * n + gj] = acc[j];
          L[(int64_t)gj * n + gi0] = acc[j];
        }
      }
      __syncthreads();
    }
}

// y_e = W_e^-1 x_e, one CTA per element; the symmetric inverse is read by columns
// (W[b][a] for consecutive a: coalesced)
__global__ void __launch_bounds__(MI_THREADS)
k_mi_gemv(int64_t E, int nx, int ny, int k, const double* __restrict__ mat, const double* __restrict__ x,
          double* __restrict__ y) {
  extern __shared__ double sm[];
  const int n = k * k * k;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  double* xe = sm;
  for (int a = threadIdx.x; a < n; a += blockDim.x) xe[a] = x[mi_cell(e, a, k, nx, ny)];
  __syncthreads();
  const double* W = mat + e * (int64_t)n * n;
  constexpr int R = (MI_MAXK * MI_MAXK * MI_MAXK + MI_THREADS - 1) / MI_THREADS;
  double acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) acc[j] = 0.0;
#pragma unroll 4
  for (int b = 0; b < n; ++b) {  // unrolled: several columns' loads in flight per thread
    const double xb = xe[b];
    const double* col = W + (int64_t)b * n;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int a = threadIdx.x + j * MI_THREADS;
      if (a < n) acc[j] = fma(col[a], xb, acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int a = threadIdx.x + j * MI_THREADS;
    if (a < n) y[mi_cell(e, a, k, nx, ny)] = acc[j];
  }
}

// y_e = L^-T L^-1 x_e, one CTA per element, by 32-row tiles: the part of each row
// outside the diagonal tile by the whole CTA (8 partial sums per row), the diagonal
// tile's triangular solve by one warp
__global__ void __launch_bounds__(MI_THREADS)
k_mi_potrs(int64_t E, int nx, int ny, int k, const double* __restrict__ mat, const double* __restrict__ x,
           double* __restrict__ y) {
  extern __shared__ double sm[];
  const int n = k * k * k;
  const int64_t e = blockIdx.x;
  if (e >= E) return;
  double* z = sm;               // [n] right-hand side, then the solution
  double* part = z + n;         // [8][32] partial sums
  const double* L = mat + e * (int64_t)n * n;
  for (int a = threadIdx.x; a < n; a += blockDim.x) z[a] = x[mi_cell(e, a, k, nx, ny)];
  __syncthreads();
  const int nb = (n + TILE - 1) / TILE, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // forward: L z = x
  for (int J = 0; J < nb; ++J) {
    const int r = threadIdx.x >> 3, g = threadIdx.x & 7, i = J * TILE + r;
    double s = 0.0;
    if (i < n)
      for (int j = g; j < J * TILE; j += 8) s = fma(L[(int64_t)i * n + j], z[j], s);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (g == 0) part[r] = s;
    __syncthreads();
    if (warp == 0) {
      const int ii = J * TILE + lane;
      double v = ii < n ? z[ii] - part[lane] : 0.0;
      for (int c = 0; c < TILE && J * TILE + c < n; ++c) {
        const double lcc = L[(int64_t)(J * TILE + c) * n + J * TILE + c];
        const double zc = __shfl_sync(0xffffffffu, v, c) / lcc;
        if (lane == c) v = zc;
        if (lane > c && ii < n) v = fma(-L[(int64_t)ii * n + J * TILE + c], zc, v);
      }
      if (ii < n) z[ii] = v;
    }
    __syncthreads();
  }
  // backward: L^T y = z
  for (int J = nb - 1; J >= 0; --J) {
    const int rr = threadIdx.x & 31, g = threadIdx.x >> 5, i = J * TILE + rr;
    double s = 0.0;
    if (i < n)
      for (int j = (J + 1) * TILE + g; j < n; j += 8) s = fma(L[(int64_t)j * n + i], z[j], s);
    part[g * 32 + rr] = s;
    __syncthreads();
    if (warp == 0) {
      const int ii = J * TILE + lane;
      double v = 0.0;
      if (ii < n) {
        v = z[ii];
        for (int q8 = 0; q8 < 8; ++q8) v -= part[q8 * 32 + lane];
      }
      for (int c = TILE - 1; c >= 0; --c) {
        const int gc = J * TILE + c;
        if (gc >= n) continue;
        const double lcc = L[(int64_t)gc * n + gc];
        const double yc = __shfl_sync(0xffffffffu, v, c) / lcc;
        if (lane == c) v = yc;
        if (lane < c) v = fma(-L[(int64_t)gc * n + ii], yc, v);
      }
      if (ii < n) z[ii] = v;
    }
    __syncthreads();
  }
  for (int a = threadIdx.x; a < n; a += blockDim.x) y[mi_cell(e, a, k, nx, ny)] = z[a];
}

// double-float copies for the CG stages: v -> df(v), and 1 / d -> df(1 / d)
__global__ void k_mi_to_df(int64_t n, const double* __restrict__ v, dfloat* __restrict__ o, int inv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) o[i] = df_from_double(inv ? 1.0 / v[i] : v[i]);
}

size_t cg_smem(int k, int q) {
  const int n = k * k * k;
  return sizeof(double) * ((size_t)q * k + k * k + 4 * n + q * k * k + q * q * k + q * q * q + 32);
}

}  // namespace

namespace {
inline unsigned mi_blocks(int64_t n) { return (unsigned)((n + MI_THREADS - 1) / MI_THREADS); }

void mi_free(hd_massinv* h) {
  cudaFree(h->d_wdet);
  cudaFree(h->d_diag);
  cudaFree(h->d_mat);
  cudaFree(h->d_aux);
  cudaFree(h->d_flag);
  cudaFree(h->x_wdet);
  cudaFree(h->x_dinv);
  h->x_wdet = h->x_dinv = nullptr;
  h->d_wdet = h->d_diag = h->d_mat = h->d_aux = nullptr;
  h->d_flag = nullptr;
}

hd_status mi_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HD_OK;
  return e == cudaErrorMemoryAllocation ? HD_ERR_OOM : HD_ERR_CUDA;
}

hd_status mi_setup(hd_massinv* h, const hd_massinv_desc* d) {
  const int k = h->k, q = h->q, n = (int)h->n;
  const int64_t E = h->E, nq = (int64_t)q * q * q, nv = (int64_t)(d->nx + 1) * (d->ny + 1) * (d->nz + 1);
  cudaStream_t s = h->stream;
  double *dvx = nullptr, *dvy = nullptr, *dvz = nullptr, *dal = nullptr;
  hd_status st = HD_OK;
  auto ck = [&](cudaError_t e) {
    if (st == HD_OK && e != cudaSuccess) st = mi_cuda(e);
  };
  ck(cudaMalloc(&h->d_flag, 3 * sizeof(int)));
  ck(cudaMalloc(&h->d_wdet, sizeof(double) * E * nq));
  ck(cudaMalloc(&dvx, sizeof(double) * nv));
  ck(cudaMalloc(&dvy, sizeof(double) * nv));
  ck(cudaMalloc(&dvz, sizeof(double) * nv));
  if (d->alpha) ck(cudaMalloc(&dal, sizeof(double) * E));
  const bool cg = h->method == HD_WINV_CG || h->method == HD_WINV_CG_HIST;
  if (cg) ck(cudaMalloc(&h->d_diag, sizeof(double) * E * n));
  if (cg && h->emul) {
    ck(cudaMalloc(&h->x_wdet, sizeof(dfloat) * E * nq));
    ck(cudaMalloc(&h->x_dinv, sizeof(dfloat) * E * n));
  }
  else ck(cudaMalloc(&h->d_mat, sizeof(double) * E * n * n));
  if (h->method == HD_WINV_DENSE) ck(cudaMalloc(&h->d_aux, sizeof(double) * E * n * n));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ck(cudaEventCreate(&ev[0]));
  ck(cudaEventCreate(&ev[1]));
  if (st == HD_OK) {
    ck(cudaMemsetAsync(h->d_flag, 0, 3 * sizeof(int), s));
    ck(cudaMemcpyAsync(dvx, d->vx, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dvy, d->vy, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(dvz, d->vz, sizeof(double) * nv, cudaMemcpyHostToDevice, s));
    if (dal) ck(cudaMemcpyAsync(dal, d->alpha, sizeof(double) * E, cudaMemcpyHostToDevice, s));
    ck(cudaEventRecord(ev[0], s));
    k_mi_geom<<<mi_blocks(E * nq), MI_THREADS, 0, s>>>(E, h->nx, h->ny, h->tab, dvx, dvy, dvz, dal, h->d_wdet,
                                                        h->d_flag);
    if (cg) {
      k_mi_diag<<<mi_blocks(E * n), MI_THREADS, 0, s>>>(E, h->tab, h->d_wdet, h->d_diag);
      if (h->emul) {
        k_mi_to_df<<<mi_blocks(E * nq), MI_THREADS, 0, s>>>(E * nq, h->d_wdet, h->x_wdet, 0);
        k_mi_to_df<<<mi_blocks(E * n), MI_THREADS, 0, s>>>(E * n, h->d_diag, h->x_dinv, 1);
      }
    } else {
      const size_t sm = sizeof(double) * ((size_t)q * k + (size_t)k * k * q * q);
      const size_t sm_max = sizeof(double) * ((size_t)MI_MAXQ * MI_MAXK + (size_t)MI_MAXK * MI_MAXK * MI_MAXQ * MI_MAXQ);
      ck(cudaFuncSetAttribute(k_mi_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_max));
      k_mi_assemble<<<(unsigned)E, MI_THREADS, sm, s>>>(E, h->tab, h->d_wdet, h->d_mat);
      k_mi_potrf<<<(unsigned)E, MI_THREADS, 0, s>>>(E, n, h->d_mat, h->d_flag + 2);
      if (h->method == HD_WINV_DENSE) k_mi_potri<<<(unsigned)E, MI_THREADS, 0, s>>>(E, n, h->d_mat, h->d_aux);
    }
    ck(cudaGetLastError());
    ck(cudaEventRecord(ev[1], s));
  }
  int flag[3] = {0, 0, 0};
  if (st == HD_OK) ck(cudaMemcpyAsync(flag, h->d_flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (st == HD_OK) ck(cudaStreamSynchronize(s));
  if (st == HD_OK) {
    float ms = 0.0f;
    ck(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    h->setup_ms = ms;
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  cudaFree(dvx);
  cudaFree(dvy);
  cudaFree(dvz);
  cudaFree(dal);
  cudaFree(h->d_aux);
  h->d_aux = nullptr;
  if (st == HD_OK && flag[0]) st = HD_ERR_INVALID_ARG;  // det J <= 0 at a point
  if (st == HD_OK && flag[2]) st = HD_ERR_NAN;          // a pivot <= 0: W_e not positive definite
  return st;
}
}  // namespace

extern "C" hd_status hd_massinv_create(const hd_massinv_desc* d, hd_massinv_handle* out) {
  if (!d || !out || !d->vx || !d->vy || !d->vz) return HD_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->k < 2 || d->k > MI_MAXK) return HD_ERR_INVALID_ARG;
  const int q = d->q > 0 ? d->q : d->k + 2;
  if (q < d->k || q > MI_MAXQ) return HD_ERR_INVALID_ARG;
  if (d->method != HD_WINV_DENSE && d->method != HD_WINV_CHOL && d->method != HD_WINV_CG &&
      d->method != HD_WINV_CG_HIST)
    return HD_ERR_INVALID_ARG;
  if (d->fp64_emulation != 0 && d->fp64_emulation != 1) return HD_ERR_INVALID_ARG;
  if (d->fp64_emulation == 1 && d->method != HD_WINV_CG && d->method != HD_WINV_CG_HIST)
    return HD_ERR_NOT_IMPLEMENTED;
  const int64_t E = (int64_t)d->nx * d->ny * d->nz, n = (int64_t)d->k * d->k * d->k;
  if (E * n >= ((int64_t)1 << 31) || E >= ((int64_t)1 << 31)) return HD_ERR_INVALID_ARG;
  if (d->alpha)
    for (int64_t e = 0; e < E; ++e)
      if (!(d->alpha[e] > 0.0)) return HD_ERR_INVALID_ARG;
  hd_massinv* h = new hd_massinv();
  h->nx = d->nx; h->ny = d->ny; h->nz = d->nz; h->k = d->k; h->q = q; h->method = d->method;
  h->E = E; h->n = n;
  MiTab& t = h->tab;
  t.k = d->k; t.q = q;
  double BG[MI_MAXQ * MI_MAXK];
  hd_l2_tables(d->k, q, t.BH, BG, t.TT, t.gx, t.gw);
  std::memcpy(t.B, d->method == HD_WINV_CG ? BG : t.BH, sizeof(t.B));
  h->cgd.k = h->cgx.k = d->k;
  h->cgd.q = h->cgx.q = q;
  for (int i = 0; i < MI_MAXQ * MI_MAXK; ++i) {
    h->cgd.B[i] = t.B[i];
    h->cgx.B[i] = df_split_host(t.B[i]);
  }
  for (int i = 0; i < MI_MAXK * MI_MAXK; ++i) {
    h->cgd.TT[i] = t.TT[i];
    h->cgx.TT[i] = df_split_host(t.TT[i]);
  }
  h->emul = d->fp64_emulation;
  if (h->method == HD_WINV_CG || h->method == HD_WINV_CG_HIST) {
    // the largest degree's size: handles of other degrees launch the same kernels
    const size_t sm = cg_smem(MI_MAXK, MI_MAXQ);
    if (cudaFuncSetAttribute(k_mi_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaFuncSetAttribute(k_mi_cg<dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
      delete h;
      return HD_ERR_CUDA;
    }
  }
  const hd_status st = mi_setup(h, d);
  if (st != HD_OK) {
    mi_free(h);
    delete h;
    return st;
  }
  *out = h;
  return HD_OK;
}

extern "C" hd_status hd_massinv_set_stream(hd_massinv_handle h, void* stream) {
  if (!h) return HD_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return HD_OK;
}

extern "C" hd_status hd_massinv_apply(hd_massinv_handle h, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  const int k = h->k, n = (int)h->n;
  cudaStream_t s = h->stream;
  if (h->method == HD_WINV_CG || h->method == HD_WINV_CG_HIST) {
    const bool glb = h->method == HD_WINV_CG;
    if (cudaMemsetAsync(h->d_flag + 1, 0, sizeof(int), s) != cudaSuccess) return HD_ERR_CUDA;
    const int maxit = glb ? 60 : 400;
    if (h->emul)
      k_mi_cg<dfloat><<<(unsigned)h->E, MI_THREADS, cg_smem(k, h->q), s>>>(
          h->E, h->nx, h->ny, h->cgx, glb ? 1 : 0, maxit, 1e-28, h->x_wdet, h->x_dinv, x, y, h->d_flag);
    else
      k_mi_cg<double><<<(unsigned)h->E, MI_THREADS, cg_smem(k, h->q), s>>>(
          h->E, h->nx, h->ny, h->cgd, glb ? 1 : 0, maxit, 1e-28, h->d_wdet, h->d_diag, x, y, h->d_flag);
  } else if (h->method == HD_WINV_DENSE) {
    k_mi_gemv<<<(unsigned)h->E, MI_THREADS, sizeof(double) * n, s>>>(h->E, h->nx, h->ny, k, h->d_mat, x, y);
  } else {
    k_mi_potrs<<<(unsigned)h->E, MI_THREADS, sizeof(double) * (n + 256), s>>>(h->E, h->nx, h->ny, k, h->d_mat, x,
                                                                               y);
  }
  return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

extern "C" hd_status hd_massinv_setup_ms(hd_massinv_handle h, double* ms) {
  if (!h || !ms) return HD_ERR_INVALID_ARG;
  *ms = h->setup_ms;
  return HD_OK;
}

extern "C" hd_status hd_massinv_iterations(hd_massinv_handle h, int32_t* its) {
  if (!h || !its) return HD_ERR_INVALID_ARG;
  *its = 0;
  if (h->method != HD_WINV_CG && h->method != HD_WINV_CG_HIST) return HD_OK;
  int v = 0;
  if (cudaMemcpyAsync(&v, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return HD_ERR_CUDA;
  *its = v;
  return HD_OK;
}

extern "C" hd_status hd_massinv_destroy(hd_massinv_handle h) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  mi_free(h);
  delete h;
  return HD_OK;
}
