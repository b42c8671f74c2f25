// Smoothed-aggregation hierarchy of the Schur V/W-cycle (smooth_levels = 1).
//
// The paper applies one AMG V-cycle to the approximate Schur complement S~ and
// relies on its mesh-independent convergence (Sec. 3.2, Sec. 4). Here:
//   level 0: S~ itself, the 7-point face-weight lattice (LevelT, shared with the
//            unsmoothed hierarchy);
//   P_0    = (I - omega D_l1^-1 S~) P0 with P0 the piecewise-constant 2x2x2
//            aggregation and omega = 4/3. A fine cell has at most four nonzeros
//            in its row of P_0: its own aggregate and, in each direction, the
//            aggregate across its one face that leaves the aggregate. They are
//            stored as four values per cell;
//   level 1: A_1 = P_0^T S~ P_0, a 33-point stencil (3x3x3 box and the six cells
//            two steps away along an axis), computed per coarse cell from P_0 and
//            the fine stencil;
//   deeper : plain aggregation, A_{l+1} = P0^T A_l P0, 27-point stencils;
//   coarsest: dense inverse (host Cholesky), + s 1 1^T when S~ is singular.
// l1-Jacobi smoothing (D_l1 = sum_j |A_ij|) on every level, nu sweeps before and
// after, V- or W-cycle as for the unsmoothed hierarchy.
#include <cmath>
#include <vector>

#include "hd_internal.h"
#include "k_level7.cuh"

namespace {

constexpr int TPB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }
constexpr double SA_OMEGA = 4.0 / 3.0;
// Above this many cells a stencil level runs its sweeps unfused: the fused forms
// (first two sweeps from zero; prolongation + sweep) recompute D^-1 b or x + P e at
// every neighbour, which doubles the FP64 operations, and the FP64 pipe (about
// 2 FMA per clock per SM) rather than HBM bounds these sweeps. Below it launch
// overhead dominates and fusing wins.
constexpr int64_t FUSE_MAX = 65536;

// offset o of a stencil level: o < 27 the 3x3x3 box (dx fastest), then +-2 along
// x, y, z (o = 27 + 2 d + (negative ? 1 : 0))
__host__ __device__ __forceinline__ void st_off(int o, int& dx, int& dy, int& dz) {
  if (o < 27) {
    dx = o % 3 - 1;
    dy = (o / 3) % 3 - 1;
    dz = o / 9 - 1;
  } else {
    const int a = o - 27, d = a >> 1, v = (a & 1) ? -2 : 2;
    dx = d == 0 ? v : 0;
    dy = d == 1 ? v : 0;
    dz = d == 2 ? v : 0;
  }
}
// stored (half) offset h -> full offset index: h = 0 the centre, 1..13 the box
// offsets after it in lattice order, 14..16 the +2 axis offsets
__host__ __device__ __forceinline__ int half_full_index(int h) { return h < 14 ? 13 + h : 27 + 2 * (h - 14); }
__host__ __device__ constexpr int n_half(int no) { return no == 33 ? 17 : 14; }

// index of an offset in the 33-offset list, -1 if it is not there
__device__ __forceinline__ int st_index(int dx, int dy, int dz) {
  if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
  if (dy == 0 && dz == 0 && (dx == 2 || dx == -2)) return 27 + (dx < 0);
  if (dx == 0 && dz == 0 && (dy == 2 || dy == -2)) return 29 + (dy < 0);
  if (dx == 0 && dy == 0 && (dz == 2 || dz == -2)) return 31 + (dz < 0);
  return -1;
}

// -- level 0: the smoothed prolongator ---------------------------------------------
// For fine coordinate I along a direction with aggregation factor f and extent X:
// the neighbour across the face that leaves the aggregate is I - 1 for even I and
// I + 1 for odd I (none at the lattice boundary or when f == 1).
__device__ __forceinline__ int out_step(int I, int X, int f) {
  if (f == 1) return 0;
  const int s = (I & 1) ? 1 : -1;
  return (I + s >= 0 && I + s < X) ? s : 0;
}
// the neighbour inside the aggregate along the same direction (0: none)
__device__ __forceinline__ int in_step(int I, int X, int f) {
  if (f == 1) return 0;
  const int s = (I & 1) ? -1 : 1;
  return (I + s >= 0 && I + s < X) ? s : 0;
}

template <typename T>
struct Face7 {  // face weights of cell (I,J,Z) of a LevelT towards -x,+x,-y,+y,-z,+z
  T w[6];
};
template <typename T>
__device__ __forceinline__ Face7<T> faces7(const LevelT<T>& L, int I, int J, int Z) {
  const int64_t xl = I + (int64_t)(L.X + 1) * (J + (int64_t)L.Y * Z);
  const int64_t yl = I + (int64_t)L.X * (J + (int64_t)(L.Y + 1) * Z);
  const int64_t zl = I + (int64_t)L.X * (J + (int64_t)L.Y * Z);
  Face7<T> f;
  f.w[0] = L.wx[xl];
  f.w[1] = L.wx[xl + 1];
  f.w[2] = L.wy[yl];
  f.w[3] = L.wy[yl + L.X];
  f.w[4] = L.wz[zl];
  f.w[5] = L.wz[zl + (int64_t)L.X * L.Y];
  return f;
}

// pv[k * n + i], k = 0: P(i, own aggregate); k = 1, 2, 3: P(i, aggregate across
// the x, y, z face leaving the aggregate) (0 when there is none)
__global__ void k_sa_pvals(LevelT<double> L, int fx, int fy, int fz, double* __restrict__ pv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n();
  if (i >= n) return;
  int I, J, Z;
  lat_coords(i, L.X, L.Y, I, J, Z);
  const Face7<double> f = faces7(L, I, J, Z);
  const int so[3] = {out_step(I, L.X, fx), out_step(J, L.Y, fy), out_step(Z, L.Z, fz)};
  const int si[3] = {in_step(I, L.X, fx), in_step(J, L.Y, fy), in_step(Z, L.Z, fz)};
  const double wd = SA_OMEGA * L.dinv[i];
  double inner = 0.0;  // sum of the weights to neighbours inside the aggregate
  for (int d = 0; d < 3; ++d)
    if (si[d]) inner += f.w[2 * d + (si[d] > 0)];
  pv[i] = 1.0 - wd * (L.diag[i] - inner);
  for (int d = 0; d < 3; ++d) pv[(1 + d) * n + i] = so[d] ? wd * f.w[2 * d + (so[d] > 0)] : 0.0;
}

// coarse coordinates
struct CDims {
  int X, Y, Z, fx, fy, fz;
};
// aggregate coordinate of fine coordinate i for an aggregation factor f in {1, 2}
__device__ __forceinline__ int agg(int i, int f) { return i >> (f - 1); }

// Enumerates the fine cells i with P(i, C) != 0 for coarse cell (Cx, Cy, Cz) and
// calls fn(i, I, J, Z, P(i, C)). Support: the aggregate plus, across each face
// that leaves it, the adjacent fine cells.
template <typename T, typename F>
__device__ __forceinline__ void for_support(const LevelT<T>& L, const CDims& c, const T* __restrict__ pv, int Cx,
                                            int Cy, int Cz, F fn) {
  const int64_t n = L.n();
  const int x0 = max(c.fx * Cx - 1, 0), x1 = min(c.fx * Cx + c.fx, L.X - 1);
  const int y0 = max(c.fy * Cy - 1, 0), y1 = min(c.fy * Cy + c.fy, L.Y - 1);
  const int z0 = max(c.fz * Cz - 1, 0), z1 = min(c.fz * Cz + c.fz, L.Z - 1);
  for (int Z = z0; Z <= z1; ++Z)
    for (int J = y0; J <= y1; ++J)
      for (int I = x0; I <= x1; ++I) {
        const int ax = I / c.fx, ay = J / c.fy, az = Z / c.fz;
        const int64_t i = I + (int64_t)L.X * (J + (int64_t)L.Y * Z);
        int slot = -1;
        if (ax == Cx && ay == Cy && az == Cz) {
          slot = 0;
        } else {
          const int so[3] = {out_step(I, L.X, c.fx), out_step(J, L.Y, c.fy), out_step(Z, L.Z, c.fz)};
          if (so[0] && ay == Cy && az == Cz && (I + so[0]) / c.fx == Cx) slot = 1;
          else if (so[1] && ax == Cx && az == Cz && (J + so[1]) / c.fy == Cy) slot = 2;
          else if (so[2] && ax == Cx && ay == Cy && (Z + so[2]) / c.fz == Cz) slot = 3;
        }
        if (slot >= 0) fn(i, I, J, Z, pv[slot * n + i]);
      }
}

// A_1 = P_0^T S~ P_0, one thread per coarse cell C: for every fine i in the support
// of column C and every stencil neighbour j of i, P(i,C) S~(i,j) P(j,D) is added
// to A_1(C, D) for the (at most four) aggregates D of row j of P_0.
__global__ void k_sa_galerkin(LevelT<double> L, CDims c, const double* __restrict__ pv, StLevelT<double> A1,
                              int* __restrict__ bad) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = A1.n();
  if (C >= nc) return;
  int Cx, Cy, Cz;
  lat_coords(C, c.X, c.Y, Cx, Cy, Cz);
  const int64_t n = L.n();
  double acc[33];
  for (int o = 0; o < 33; ++o) acc[o] = 0.0;
  for_support(L, c, pv, Cx, Cy, Cz, [&](int64_t i, int I, int J, int Z, double p) {
    const Face7<double> f = faces7(L, I, J, Z);
    // j = i and its six neighbours
    for (int k = 0; k < 7; ++k) {
      int dI = 0, dJ = 0, dZ = 0;
      double a;
      if (k == 0) {
        a = L.diag[i];
      } else {
        const int d = (k - 1) >> 1, s = ((k - 1) & 1) ? 1 : -1;
        (d == 0 ? dI : d == 1 ? dJ : dZ) = s;
        if (I + dI < 0 || I + dI >= L.X || J + dJ < 0 || J + dJ >= L.Y || Z + dZ < 0 || Z + dZ >= L.Z) continue;
        a = -f.w[k - 1];
      }
      const int jI = I + dI, jJ = J + dJ, jZ = Z + dZ;
      const int64_t j = jI + (int64_t)L.X * (jJ + (int64_t)L.Y * jZ);
      const int so[3] = {out_step(jI, L.X, c.fx), out_step(jJ, L.Y, c.fy), out_step(jZ, L.Z, c.fz)};
      const int Dx = jI / c.fx, Dy = jJ / c.fy, Dz = jZ / c.fz;
      for (int s = 0; s < 4; ++s) {
        int ex = Dx, ey = Dy, ez = Dz;
        if (s == 1) { if (!so[0]) continue; ex = (jI + so[0]) / c.fx; }
        if (s == 2) { if (!so[1]) continue; ey = (jJ + so[1]) / c.fy; }
        if (s == 3) { if (!so[2]) continue; ez = (jZ + so[2]) / c.fz; }
        const int o = st_index(ex - Cx, ey - Cy, ez - Cz);
        if (o < 0) {
          atomicExch(bad, 1);
          continue;
        }
        acc[o] = fma(p * a, pv[s * n + j], acc[o]);
      }
    }
  });
  for (int o = 0; o < 33; ++o) A1.a[o * nc + C] = acc[o];
}

// A_{l+1} = P0^T A_l P0 for plain aggregation of a stencil level (27-point result)
__global__ void k_ua_galerkin(StLevelT<double> F, CDims c, StLevelT<double> A, int* __restrict__ bad) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = A.n(), n = F.n();
  if (C >= nc) return;
  int Cx, Cy, Cz;
  lat_coords(C, c.X, c.Y, Cx, Cy, Cz);
  double acc[27];
  for (int o = 0; o < 27; ++o) acc[o] = 0.0;
  for (int Z = c.fz * Cz; Z < min(c.fz * Cz + c.fz, F.Z); ++Z)
    for (int J = c.fy * Cy; J < min(c.fy * Cy + c.fy, F.Y); ++J)
      for (int I = c.fx * Cx; I < min(c.fx * Cx + c.fx, F.X); ++I) {
        const int64_t i = I + (int64_t)F.X * (J + (int64_t)F.Y * Z);
        for (int o = 0; o < F.no; ++o) {
          const double a = F.a[o * n + i];
          if (a == 0.0) continue;
          int dx, dy, dz;
          st_off(o, dx, dy, dz);
          const int jI = I + dx, jJ = J + dy, jZ = Z + dz;
          if (jI < 0 || jI >= F.X || jJ < 0 || jJ >= F.Y || jZ < 0 || jZ >= F.Z) {
            atomicExch(bad, 1);
            continue;
          }
          const int ox = jI / c.fx - Cx, oy = jJ / c.fy - Cy, oz = jZ / c.fz - Cz;
          if (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1) {
            atomicExch(bad, 1);
            continue;
          }
          acc[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] += a;
        }
      }
  for (int o = 0; o < 27; ++o) A.a[o * nc + C] = acc[o];
}

// keep the centre and the later offsets (setup: full -> half storage)
__global__ void k_st_compress(StLevelT<double> A, double* __restrict__ half) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = A.n();
  if (c >= n) return;
  for (int h = 0; h < n_half(A.no); ++h) half[h * n + c] = A.a[half_full_index(h) * n + c];
}

__global__ void k_st_dinv(StLevelT<double> A) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = A.n();
  if (c >= n) return;
  double s = 0.0;
  for (int o = 0; o < A.no; ++o) s += fabs(A.a[o * n + c]);
  A.dinv[c] = 1.0 / s;
}

// -- solve-time kernels of the stencil levels ---------------------------------------
// (A x)_c from the half-stored symmetric stencil; x_at(I, J, Z, k) supplies the
// vector value at lattice cell (I, J, Z) with linear index k. Which neighbours
// exist is decided once per cell (flags for steps -2..2 per direction), so that
// each unrolled offset costs a few flag tests and one index add: these sweeps
// are otherwise bound by integer address arithmetic rather than by the FP units
// or HBM. Cell indices fit 32 bits (stencil levels are at most 1/8 of the fine
// lattice).
template <typename T, int NO, typename XA>
__device__ __forceinline__ T st_row(const StLevelT<T>& L, int c, int I, int J, int Z, XA x_at) {
  constexpr int NH = n_half(NO);
  const int64_t n = L.n();
  const int X = L.X, XY = L.X * L.Y;
  const bool fx[5] = {I >= 2, I >= 1, true, I + 1 < L.X, I + 2 < L.X};
  const bool fy[5] = {J >= 2, J >= 1, true, J + 1 < L.Y, J + 2 < L.Y};
  const bool fz[5] = {Z >= 2, Z >= 1, true, Z + 1 < L.Z, Z + 2 < L.Z};
  T s = L.a[c] * x_at(I, J, Z, c);
#pragma unroll
  for (int h = 1; h < NH; ++h) {
    int dx, dy, dz;
    st_off(half_full_index(h), dx, dy, dz);
    const int d = dx + X * dy + XY * dz;
    const T* ah = L.a + h * n;
    if (fx[2 + dx] && fy[2 + dy] && fz[2 + dz]) s = fma(ah[c], x_at(I + dx, J + dy, Z + dz, c + d), s);
    if (fx[2 - dx] && fy[2 - dy] && fz[2 - dz]) s = fma(ah[c - d], x_at(I - dx, J - dy, Z - dz, c - d), s);
  }
  return s;
}

template <typename T>
__global__ void k_st_scale(StLevelT<T> L, const T* __restrict__ b, T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  x[c] = L.dinv[c] * b[c];
}

// two l1-Jacobi sweeps from a zero guess in one pass: x1 = D^-1 b is formed on
// the fly at the neighbours, x2 = x1 + D^-1 (b - A x1)
template <typename T, int NO>
__global__ void k_st_scale_jacobi(StLevelT<T> L, const T* __restrict__ b, T* __restrict__ xo) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  auto xa = [&](int, int, int, int k) { return L.dinv[k] * b[k]; };
  const T r = b[c] - st_row<T, NO>(L, (int)c, I, J, Z, xa);
  xo[c] = fma(L.dinv[c], r, xa(I, J, Z, (int)c));
}

template <typename T, int NO>
__global__ void k_st_jacobi(StLevelT<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  auto xa = [&](int, int, int, int k) { return x[k]; };
  const T r = b[c] - st_row<T, NO>(L, (int)c, I, J, Z, xa);
  xo[c] = fma(L.dinv[c], r, x[c]);
}

// r = b - A x on a stencil level (fine-parallel half of the restriction)
template <typename T, int NO>
__global__ void k_st_resid(StLevelT<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  auto xa = [&](int, int, int, int k) { return x[k]; };
  r[c] = b[c] - st_row<T, NO>(L, (int)c, I, J, Z, xa);
}

// b_C = sum of r over the aggregate of C (plain aggregation; fine lattice X x Y x Z)
template <typename T>
__global__ void k_agg_sum(int X, int Y, int Z, CDims cd, const T* __restrict__ r, T* __restrict__ bc) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (C >= (int64_t)cd.X * cd.Y * cd.Z) return;
  int Cx, Cy, Cz;
  lat_coords(C, cd.X, cd.Y, Cx, Cy, Cz);
  T s = (T)0;
  for (int k = cd.fz * Cz; k < min(cd.fz * Cz + cd.fz, Z); ++k)
    for (int j = cd.fy * Cy; j < min(cd.fy * Cy + cd.fy, Y); ++j)
      for (int i = cd.fx * Cx; i < min(cd.fx * Cx + cd.fx, X); ++i) s += r[i + (int64_t)X * (j + (int64_t)Y * k)];
  bc[C] = s;
}

template <typename T>
__global__ void k_st_prolong_add(StLevelT<T> L, CDims cd, const T* __restrict__ e, T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  x[c] += e[agg(I, cd.fx) + (int64_t)cd.X * (agg(J, cd.fy) + (int64_t)cd.Y * agg(Z, cd.fz))];
}

// x' = x + P0 e, then one l1-Jacobi sweep from x' (the first post-smoothing sweep)
template <typename T, int NO>
__global__ void k_st_jacobi_prolong(StLevelT<T> L, CDims cd, const T* __restrict__ b, const T* __restrict__ x,
                                    const T* __restrict__ e, T* __restrict__ xo) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  auto xa = [&](int i, int j, int z, int k) {
    return x[k] + e[agg(i, cd.fx) + cd.X * (agg(j, cd.fy) + cd.Y * agg(z, cd.fz))];
  };
  const T xs = xa(I, J, Z, (int)c);
  const T r = b[c] - st_row<T, NO>(L, (int)c, I, J, Z, xa);
  xo[c] = fma(L.dinv[c], r, xs);
}

// -- level-0 transfers with the smoothed prolongator ------------------------------------
template <typename T>
__global__ void k_sa_res0(LevelT<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  r[c] = stencil_res<T>(L, x, b[c], x[c], I, J, Z, c);
}

// b_C = (P_0^T r)_C. The support of column C is enumerated directly: the
// aggregate's cells (slot 0), then for each direction d with factor 2 the layers
// of fine cells just below and above the aggregate (slot 1 + d), which lie
// across the face that leaves their own aggregate.
template <typename T>
__global__ void k_sa_restrict0(LevelT<T> L, CDims cd, const T* __restrict__ pv, const T* __restrict__ r,
                               T* __restrict__ bc) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (C >= (int64_t)cd.X * cd.Y * cd.Z) return;
  int Cc[3];
  lat_coords(C, cd.X, cd.Y, Cc[0], Cc[1], Cc[2]);
  const int ext[3] = {L.X, L.Y, L.Z}, f[3] = {cd.fx, cd.fy, cd.fz};
  const int64_t str[3] = {1, (int64_t)L.X, (int64_t)L.X * L.Y};
  const int64_t n = L.n();
  int lo[3], hi[3];  // aggregate range [lo, hi] per direction
  for (int d = 0; d < 3; ++d) {
    lo[d] = f[d] * Cc[d];
    hi[d] = min(lo[d] + f[d], ext[d]) - 1;
  }
  T s = (T)0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int64_t i = x + str[1] * y + str[2] * z;
        s = fma(pv[i], r[i], s);
      }
  for (int d = 0; d < 3; ++d) {
    if (f[d] != 2) continue;
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const int layer[2] = {lo[d] - 1, lo[d] + 2};
    for (int t = 0; t < 2; ++t) {
      const int c = layer[t];
      if (c < 0 || c >= ext[d] || (t == 1 && hi[d] != lo[d] + 1)) continue;
      for (int b = lo[e2]; b <= hi[e2]; ++b)
        for (int a = lo[e1]; a <= hi[e1]; ++a) {
          const int64_t i = str[d] * c + str[e1] * a + str[e2] * b;
          s = fma(pv[(1 + d) * n + i], r[i], s);
        }
    }
  }
  bc[C] = s;
}

// x += P_0 e
template <typename T>
__global__ void k_sa_prolong0(LevelT<T> L, CDims cd, const T* __restrict__ pv, const T* __restrict__ e,
                              T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n();
  if (c >= n) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  const int Dx = agg(I, cd.fx), Dy = agg(J, cd.fy), Dz = agg(Z, cd.fz);
  auto ev = [&](int ex, int ey, int ez) { return e[ex + (int64_t)cd.X * (ey + (int64_t)cd.Y * ez)]; };
  T v = pv[c] * ev(Dx, Dy, Dz);
  const int sx = out_step(I, L.X, cd.fx), sy = out_step(J, L.Y, cd.fy), sz = out_step(Z, L.Z, cd.fz);
  if (sx) v = fma(pv[n + c], ev(agg(I + sx, cd.fx), Dy, Dz), v);
  if (sy) v = fma(pv[2 * n + c], ev(Dx, agg(J + sy, cd.fy), Dz), v);
  if (sz) v = fma(pv[3 * n + c], ev(Dx, Dy, agg(Z + sz, cd.fz)), v);
  x[c] += v;
}

template <typename T>
__global__ void k_to_f32_sa(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

template <typename T>
CDims cdims_of(const StLevelT<T>& c) {
  return CDims{c.X, c.Y, c.Z, c.fx, c.fy, c.fz};
}

// -- the cycle ----------------------------------------------------------------------
// levels >= 1: st[l - 1]; the last one is solved densely
template <typename T>
const T* sa_level(hd_op* h, std::vector<StLevelT<T>>& st, int l, const T* b, T* out) {
  StLevelT<T>& L = st[l - 1];
  const int last = (int)st.size();
  if (l == last) {
    T* dst = out ? out : L.x0;
    k_vc_coarse<T><<<nblk(L.n() * 32), TPB, 0, h->stream>>>((int)L.n(), h->d_sa_coarse_inv, b, dst);
    return dst;
  }
  StLevelT<T>& C = st[l];
  const CDims cd = cdims_of(C);
  const int nu = h->nu;
  const bool w33 = L.no == 33;
  auto jacobi = [&](const T* x, T* xo) {
    if (w33) k_st_jacobi<T, 33><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, x, xo);
    else k_st_jacobi<T, 27><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, x, xo);
  };
  T* cur = L.x0;
  int s0 = 1;
  const bool fuse = L.n() <= FUSE_MAX;
  if (nu >= 2 && fuse) {  // the first two sweeps fused
    if (w33) k_st_scale_jacobi<T, 33><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur);
    else k_st_scale_jacobi<T, 27><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur);
    s0 = 2;
  } else {
    k_st_scale<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur);
  }
  for (int s = s0; s < nu; ++s) {
    T* o = (cur == L.x0) ? L.x1 : L.x0;
    jacobi(cur, o);
    cur = o;
  }
  const int repeats = (h->cycle == 2 && l + 1 < last && (h->w_levels == 0 || l < h->w_levels)) ? 2 : 1;
  const T* xc = nullptr;
  for (int rep = 0; rep < repeats; ++rep) {
    if (rep > 0) k_st_prolong_add<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, xc, cur);
    T* rtmp = (cur == L.x0) ? L.x1 : L.x0;  // free until the post-smoothing
    if (w33) k_st_resid<T, 33><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, rtmp);
    else k_st_resid<T, 27><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, rtmp);
    k_agg_sum<T><<<nblk(C.n()), TPB, 0, h->stream>>>(L.X, L.Y, L.Z, cd, rtmp, C.b);
    xc = sa_level<T>(h, st, l + 1, C.b, nullptr);
  }
  T* o = (nu == 1 && out) ? out : ((cur == L.x0) ? L.x1 : L.x0);
  if (fuse) {
    if (w33) k_st_jacobi_prolong<T, 33><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, b, cur, xc, o);
    else k_st_jacobi_prolong<T, 27><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, b, cur, xc, o);
  } else {
    k_st_prolong_add<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, xc, cur);
    jacobi(cur, o);
  }
  cur = o;
  for (int s = 1; s < nu; ++s) {
    T* o2 = (s == nu - 1 && out) ? out : ((cur == L.x0) ? L.x1 : L.x0);
    jacobi(cur, o2);
    cur = o2;
  }
  return cur;
}

// level 0 (7-point lattice) with the smoothed transfers to level 1
template <typename T>
void sa_cycle0(hd_op* h, LevelT<T>& L, const T* pv, std::vector<StLevelT<T>>& st, const T* b, T* out) {
  const CDims cd = cdims_of(st[0]);
  const int nu = h->nu;
  T* cur = L.x0;
  k_vc_scale<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur);
  for (int s = 1; s < nu; ++s) {
    T* o = (cur == L.x0) ? L.x1 : L.x0;
    k_vc_jacobi<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, o);
    cur = o;
  }
  const int last = (int)st.size();
  const int repeats = (h->cycle == 2 && 1 < last) ? 2 : 1;  // level 0 (w_levels >= 1 or 0)
  const T* xc = nullptr;
  for (int rep = 0; rep < repeats; ++rep) {
    if (rep > 0) k_sa_prolong0<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, pv, xc, cur);
    k_sa_res0<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, L.b);
    k_sa_restrict0<T><<<nblk(st[0].n()), TPB, 0, h->stream>>>(L, cd, pv, L.b, st[0].b);
    xc = sa_level<T>(h, st, 1, st[0].b, nullptr);
  }
  k_sa_prolong0<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, pv, xc, cur);
  for (int s = 0; s < nu; ++s) {
    T* o = (s == nu - 1) ? out : ((cur == L.x0) ? L.x1 : L.x0);
    k_vc_jacobi<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, o);
    cur = o;
  }
  if (nu == 0) cudaMemcpyAsync(out, cur, sizeof(T) * L.n(), cudaMemcpyDeviceToDevice, h->stream);
}

template <typename T>
hd_status alloc_st(hd_op* h, StLevelT<T>& L, bool coefs) {
  const int64_t n = L.n();
  // FP64 setup needs all offsets; the FP32 copy is made from the half storage
  const int64_t na = sizeof(T) == 8 ? L.no : n_half(L.no);
  if (coefs && cudaMalloc(&L.a, sizeof(T) * n * na) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "stencil level");
  if (cudaMalloc(&L.dinv, sizeof(T) * n) != cudaSuccess || cudaMalloc(&L.x0, sizeof(T) * n) != cudaSuccess ||
      cudaMalloc(&L.x1, sizeof(T) * n) != cudaSuccess || cudaMalloc(&L.b, sizeof(T) * n) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "stencil level");
  return HD_OK;
}
template <typename T>
void free_st(StLevelT<T>& L) {
  cudaFree(L.a);
  cudaFree(L.dinv);
  cudaFree(L.x0);
  cudaFree(L.x1);
  cudaFree(L.b);
}

}  // namespace

hd_status sa_setup(hd_op* h) {
  if (!h->sa || h->lv.size() < 2) return HD_OK;  // one level: nothing to smooth
  const LevelT<double>& L0 = h->lv[0];
  const int64_t n0 = L0.n();
  if (cudaMalloc(&h->sa_p, sizeof(double) * 4 * n0) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA prolongator");
  const LevelT<double>& l1 = h->lv[1];
  k_sa_pvals<<<nblk(n0), TPB, 0, h->stream>>>(L0, l1.fx, l1.fy, l1.fz, h->sa_p);
  HD_LAUNCH_CK(h, "k_sa_pvals");
  int* d_bad = nullptr;
  if (cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "flag");
  HD_CK(h, cudaMemsetAsync(d_bad, 0, sizeof(int), h->stream));
  hd_status st = HD_OK;
  for (size_t l = 1; l < h->lv.size() && st == HD_OK; ++l) {
    const LevelT<double>& g = h->lv[l];  // same lattice dimensions as the unsmoothed level
    StLevelT<double> s{};
    s.X = g.X; s.Y = g.Y; s.Z = g.Z; s.fx = g.fx; s.fy = g.fy; s.fz = g.fz;
    s.no = (l == 1) ? 33 : 27;
    st = alloc_st<double>(h, s, true);
    h->st.push_back(s);
    if (st != HD_OK) break;
    const StLevelT<double>& S = h->st.back();
    const CDims cd = cdims_of(S);
    if (l == 1) k_sa_galerkin<<<nblk(S.n()), TPB, 0, h->stream>>>(L0, cd, h->sa_p, S, d_bad);
    else k_ua_galerkin<<<nblk(S.n()), TPB, 0, h->stream>>>(h->st[h->st.size() - 2], cd, S, d_bad);
    k_st_dinv<<<nblk(S.n()), TPB, 0, h->stream>>>(S);
    if (cudaGetLastError() != cudaSuccess) st = hd_fail(h, HD_ERR_CUDA, "SA Galerkin");
  }
  int bad = 0;
  if (st == HD_OK && cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    st = hd_fail(h, HD_ERR_CUDA, "SA flag");
  if (st == HD_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = hd_fail(h, HD_ERR_CUDA, "SA setup");
  cudaFree(d_bad);
  if (st != HD_OK) return st;
  if (bad) return hd_fail(h, HD_ERR_BOUNDS, "smoothed-aggregation stencil outside its offset set");
  // coarsest: dense matrix from the stencil, inverse on the host
  const StLevelT<double>& c = h->st.back();
  const int n = (int)c.n();
  std::vector<double> a((size_t)c.no * n);
  HD_CK(h, cudaMemcpy(a.data(), c.a, sizeof(double) * a.size(), cudaMemcpyDeviceToHost));
  std::vector<double> A((size_t)n * n, 0.0), inv;
  for (int Z = 0; Z < c.Z; ++Z)
    for (int J = 0; J < c.Y; ++J)
      for (int I = 0; I < c.X; ++I) {
        const int r = I + c.X * (J + c.Y * Z);
        for (int o = 0; o < c.no; ++o) {
          int dx, dy, dz;
          st_off(o, dx, dy, dz);
          const int i = I + dx, j = J + dy, z = Z + dz;
          if (i < 0 || i >= c.X || j < 0 || j >= c.Y || z < 0 || z >= c.Z) continue;
          A[(size_t)r * n + (i + c.X * (j + c.Y * z))] += a[(size_t)o * n + r];
        }
      }
  if ((st = dense_spd_inverse(h, A, n, h->singular, inv)) != HD_OK) return st;
  if (cudaMalloc(&h->d_sa_coarse_inv, sizeof(double) * inv.size()) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "SA coarse inverse");
  HD_CK(h, cudaMemcpy(h->d_sa_coarse_inv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice));
  // half storage of the (symmetric) stencils for the solve
  for (StLevelT<double>& s : h->st) {
    double* half = nullptr;
    if (cudaMalloc(&half, sizeof(double) * s.n() * n_half(s.no)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "stencil level");
    k_st_compress<<<nblk(s.n()), TPB, 0, h->stream>>>(s, half);
    HD_LAUNCH_CK(h, "k_st_compress");
    HD_CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(s.a);
    s.a = half;
  }
  return HD_OK;
}

hd_status sa_setup_f32(hd_op* h) {
  if (h->st.empty() || !h->stf.empty()) return HD_OK;
  const int64_t n0 = h->lv[0].n();
  if (cudaMalloc(&h->sa_pf, sizeof(float) * 4 * n0) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA f32");
  k_to_f32_sa<float><<<nblk(4 * n0), TPB, 0, h->stream>>>(4 * n0, h->sa_p, h->sa_pf);
  for (const StLevelT<double>& d : h->st) {
    StLevelT<float> f{};
    f.X = d.X; f.Y = d.Y; f.Z = d.Z; f.fx = d.fx; f.fy = d.fy; f.fz = d.fz; f.no = d.no;
    hd_status st = alloc_st<float>(h, f, true);
    h->stf.push_back(f);
    if (st != HD_OK) return st;
    k_to_f32_sa<float><<<nblk(d.n() * n_half(d.no)), TPB, 0, h->stream>>>(d.n() * n_half(d.no), d.a, f.a);
    k_to_f32_sa<float><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.dinv, f.dinv);
  }
  HD_LAUNCH_CK(h, "SA f32");
  return HD_OK;
}

void sa_free(hd_op* h) {
  for (auto& s : h->st) free_st<double>(s);
  for (auto& s : h->stf) free_st<float>(s);
  h->st.clear();
  h->stf.clear();
  cudaFree(h->sa_p);
  cudaFree(h->sa_pf);
  cudaFree(h->d_sa_coarse_inv);
  h->sa_p = nullptr;
  h->sa_pf = nullptr;
  h->d_sa_coarse_inv = nullptr;
}

hd_status sa_vcycle(hd_op* h, const double* b, double* x) {
  return run_graphed(h, b, x, 2, [&]() { sa_cycle0<double>(h, h->lv[0], h->sa_p, h->st, b, x); });
}

hd_status sa_vcycle_f32(hd_op* h, const float* b, float* x) {
  return run_graphed(h, b, x, 3, [&]() { sa_cycle0<float>(h, h->lvf[0], h->sa_pf, h->stf, b, x); });
}
