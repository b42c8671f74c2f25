// Smoothed-aggregation hierarchy of the Schur V/W-cycle (smooth_levels = 1 or 2).
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
//   level 2: with smooth_levels = 2, P_1 = (I - omega D_l1^-1 A_1) P0 on level 1
//            as well (at most 11 nonzeros per row, see below) and A_2 = P_1^T A_1
//            P_1, a 179-point stencil; level 3 its plain aggregation, 81 points;
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

// Offset shapes of the stencil levels, by their number of offsets NO:
//   27 : the 3x3x3 box (plain aggregation of a level whose offsets reach 2 at most
//        along an axis and 1 across it);
//   33 : the box and (+-2, 0, 0) with its permutations (P_0^T S~ P_0);
//   179: the 5x5x5 box and (+-3, a, b), |a|, |b| <= 1, with its permutations
//        (P_1^T A_1 P_1 when the prolongator of level 1 is smoothed as well);
//   81 : the box and (+-2, a, b), |a|, |b| <= 1, with its permutations (plain
//        aggregation of the 179-point level).
// Offset o < B^3 (B = 3, or 5 for 179) runs over the box, dx fastest. The rest are
// axial: for 33, o = B^3 + 2 d + (negative); for 81 and 179, o = B^3 + 18 d +
// 9 (negative) + (a + 1) + 3 (b + 1), with d the axis and (a, b) the offsets
// across it in the order of the two remaining axes.
template <int NO>
struct Shape {
  static_assert(NO == 27 || NO == 33 || NO == 81 || NO == 179, "stencil shape");
  static constexpr int R = NO == 179 ? 2 : 1;  // box radius
  static constexpr int B = 2 * R + 1;
  static constexpr int NB = B * B * B;
  static constexpr int NH = (NO + 1) / 2;                         // stored (half) offsets
};
__host__ __device__ constexpr int n_half(int no) { return (no + 1) / 2; }

template <int NO>
__host__ __device__ __forceinline__ constexpr void st_off(int o, int& dx, int& dy, int& dz) {
  using S = Shape<NO>;
  if (o < S::NB) {
    dx = o % S::B - S::R;
    dy = (o / S::B) % S::B - S::R;
    dz = o / (S::B * S::B) - S::R;
    return;
  }
  const int a = o - S::NB;
  int d = 0, v = 0, u = 0, w = 0;
  if (NO == 33) {
    d = a >> 1;
    v = (a & 1) ? -2 : 2;
  } else {
    d = a / 18;
    const int r = a % 18;
    v = r >= 9 ? -(S::R + 1) : S::R + 1;
    u = (r % 9) % 3 - 1;
    w = (r % 9) / 3 - 1;
  }
  dx = d == 0 ? v : u;
  dy = d == 0 ? u : d == 1 ? v : w;
  dz = d == 2 ? v : w;
}
// run-time shape on the host (setup: the dense coarsest matrix)
inline void st_off_any(int no, int o, int& dx, int& dy, int& dz) {
  switch (no) {
    case 27: st_off<27>(o, dx, dy, dz); break;
    case 33: st_off<33>(o, dx, dy, dz); break;
    case 81: st_off<81>(o, dx, dy, dz); break;
    default: st_off<179>(o, dx, dy, dz); break;
  }
}

// stored (half) offset h -> full offset index: h = 0 the centre, then the box
// offsets after it in lattice order, then the positive axial offsets
template <int NO>
__host__ __device__ __forceinline__ constexpr int half_full_index(int h) {
  using S = Shape<NO>;
  constexpr int cb = (S::NB - 1) / 2;
  if (h <= cb) return cb + h;
  const int j = h - cb - 1;
  return NO == 33 ? S::NB + 2 * j : S::NB + 18 * (j / 9) + j % 9;
}

// index of an offset in the list of shape NO, -1 if it is not there
template <int NO>
__host__ __device__ __forceinline__ int st_index(int dx, int dy, int dz) {
  using S = Shape<NO>;
  if (abs(dx) <= S::R && abs(dy) <= S::R && abs(dz) <= S::R)
    return (dx + S::R) + S::B * (dy + S::R) + S::B * S::B * (dz + S::R);
  if (NO == 27) return -1;
  const int A = S::R + 1;  // the axial step
  int d, v, u, w;
  if (abs(dx) == A) { d = 0; v = dx; u = dy; w = dz; }
  else if (abs(dy) == A) { d = 1; v = dy; u = dx; w = dz; }
  else if (abs(dz) == A) { d = 2; v = dz; u = dx; w = dy; }
  else return -1;
  if (NO == 33) return (u == 0 && w == 0) ? S::NB + 2 * d + (v < 0) : -1;
  if (abs(u) > 1 || abs(w) > 1) return -1;
  return S::NB + 18 * d + (v < 0 ? 9 : 0) + (u + 1) + 3 * (w + 1);
}

// Calls f(std::integral_constant<int, NO>) for a level's run-time shape.
template <typename F>
void with_shape(int no, F f) {
  switch (no) {
    case 27: f(std::integral_constant<int, 27>{}); break;
    case 33: f(std::integral_constant<int, 33>{}); break;
    case 81: f(std::integral_constant<int, 81>{}); break;
    default: f(std::integral_constant<int, 179>{}); break;
  }
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
  int X, Y, Z, fx, fy, fz;  // fx, fy, fz: pair factors (the smoothed transfers need pairs)
  Agg1 ag[3];               // the aggregation per axis (any)
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
        const int o = st_index<33>(ex - Cx, ey - Cy, ez - Cz);
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

// A_{l+1} = P0^T A_l P0 for plain aggregation of a stencil level of shape NI into
// one of shape NOUT
template <int NI, int NOUT>
__global__ void k_ua_galerkin(StLevelT<double> F, CDims c, StLevelT<double> A, int* __restrict__ bad) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = A.n(), n = F.n();
  if (C >= nc) return;
  int Cx, Cy, Cz;
  lat_coords(C, c.X, c.Y, Cx, Cy, Cz);
  double acc[NOUT];
  for (int o = 0; o < NOUT; ++o) acc[o] = 0.0;
  for (int Z = agg_lo(c.ag[2], Cz); Z < agg_hi(c.ag[2], Cz, F.Z); ++Z)
    for (int J = agg_lo(c.ag[1], Cy); J < agg_hi(c.ag[1], Cy, F.Y); ++J)
      for (int I = agg_lo(c.ag[0], Cx); I < agg_hi(c.ag[0], Cx, F.X); ++I) {
        const int64_t i = I + (int64_t)F.X * (J + (int64_t)F.Y * Z);
        for (int o = 0; o < NI; ++o) {
          const double a = F.a[o * n + i];
          if (a == 0.0) continue;
          int dx, dy, dz;
          st_off<NI>(o, dx, dy, dz);
          const int jI = I + dx, jJ = J + dy, jZ = Z + dz;
          if (jI < 0 || jI >= F.X || jJ < 0 || jJ >= F.Y || jZ < 0 || jZ >= F.Z) {
            atomicExch(bad, 1);
            continue;
          }
          const int oc =
              st_index<NOUT>(agg_of(c.ag[0], jI) - Cx, agg_of(c.ag[1], jJ) - Cy, agg_of(c.ag[2], jZ) - Cz);
          if (oc < 0) {
            atomicExch(bad, 1);
            continue;
          }
          acc[oc] += a;
        }
      }
  for (int o = 0; o < NOUT; ++o) A.a[o * nc + C] = acc[o];
}

// keep the centre and the later offsets (setup: full -> half storage)
template <int NO>
__global__ void k_st_compress(StLevelT<double> A, double* __restrict__ half) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = A.n();
  if (c >= n) return;
  for (int h = 0; h < Shape<NO>::NH; ++h) half[h * n + c] = A.a[half_full_index<NO>(h) * n + c];
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
// exist is decided once per cell (flags for steps -3..3 per direction), so that
// each unrolled offset costs a few flag tests and one index add: these sweeps
// are otherwise bound by integer address arithmetic rather than by the FP units
// or HBM. Cell indices fit 32 bits (stencil levels are at most 1/8 of the fine
// lattice).
template <typename T, int NO, typename XA>
__device__ __forceinline__ T st_row(const StLevelT<T>& L, int c, int I, int J, int Z, XA x_at) {
  constexpr int NH = Shape<NO>::NH;
  const int64_t n = L.n();
  const int X = L.X, XY = L.X * L.Y;
  const bool fx[7] = {I >= 3, I >= 2, I >= 1, true, I + 1 < L.X, I + 2 < L.X, I + 3 < L.X};
  const bool fy[7] = {J >= 3, J >= 2, J >= 1, true, J + 1 < L.Y, J + 2 < L.Y, J + 3 < L.Y};
  const bool fz[7] = {Z >= 3, Z >= 2, Z >= 1, true, Z + 1 < L.Z, Z + 2 < L.Z, Z + 3 < L.Z};
  // FP32 levels hold the row sum in the centre slot and act on differences (rowsum_form)
  const T xc = x_at(I, J, Z, c), o = rowsum_form<T>() ? xc : (T)0;
  T s = L.a[c] * xc;
#pragma unroll
  for (int h = 1; h < NH; ++h) {
    int dx, dy, dz;
    st_off<NO>(half_full_index<NO>(h), dx, dy, dz);
    const int d = dx + X * dy + XY * dz;
    const T* ah = L.a + h * n;
    const bool okp = fx[3 + dx] && fy[3 + dy] && fz[3 + dz];
    const bool okm = fx[3 - dx] && fy[3 - dy] && fz[3 - dz];
    // every load is issued unconditionally, at the own cell where the neighbour
    // is missing (a branch per offset would keep the loads from overlapping).
    // The stored coefficient towards a missing +d neighbour is an exact zero;
    // the mirrored one is selected away.
    const T ap = ah[c];
    T am = ah[okm ? c - d : c];
    am = okm ? am : (T)0;
    s = fma(ap, rs_diff(x_at(okp ? I + dx : I, okp ? J + dy : J, okp ? Z + dz : Z, okp ? c + d : c), o), s);
    s = fma(am, rs_diff(x_at(okm ? I - dx : I, okm ? J - dy : J, okm ? Z - dz : Z, okm ? c - d : c), o), s);
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

// The wide shapes (81 and 179 offsets) sit on small levels: one thread per cell
// leaves a few waves of threads that each walk a long serial chain of loads.
// There a block of G warps takes 32 consecutive cells and warp w the stored
// offsets h with h % G == w (the centre with warp 0); the G partial sums meet in
// shared memory in a fixed order and warp 0 finishes the cell.
template <int NO>
struct SplitG {  // 8 and 4 measured best (16 warps per 32 cells: slower)
  static constexpr int G = NO == 179 ? 8 : 4;
};

// Warp W's part of (A x)_c: the stored offsets h = W, W + G, ... (the centre with
// warp 0). The offsets are known at compile time, so all loads are issued first
// and the products added afterwards, in the order +d, -d per offset.
template <typename T, int NO, int W, typename XA>
__device__ __forceinline__ T st_row_part(const StLevelT<T>& L, int c, int I, int J, int Z, XA x_at) {
  constexpr int NH = Shape<NO>::NH, G = SplitG<NO>::G;
  constexpr int H0 = W == 0 ? G : W;
  constexpr int CNT = H0 < NH ? (NH - 1 - H0) / G + 1 : 0;
  constexpr int NV = CNT > 0 ? 2 * CNT : 1;
  const int64_t n = L.n();
  const int X = L.X, XY = L.X * L.Y;
  const bool fx[7] = {I >= 3, I >= 2, I >= 1, true, I + 1 < L.X, I + 2 < L.X, I + 3 < L.X};
  const bool fy[7] = {J >= 3, J >= 2, J >= 1, true, J + 1 < L.Y, J + 2 < L.Y, J + 3 < L.Y};
  const bool fz[7] = {Z >= 3, Z >= 2, Z >= 1, true, Z + 1 < L.Z, Z + 2 < L.Z, Z + 3 < L.Z};
  T av[NV], xv[NV];
#pragma unroll
  for (int j = 0; j < CNT; ++j) {
    const int h = H0 + G * j;
    int dx, dy, dz;
    st_off<NO>(half_full_index<NO>(h), dx, dy, dz);
    const int d = dx + X * dy + XY * dz;
    const T* ah = L.a + h * n;
    const bool okp = fx[3 + dx] && fy[3 + dy] && fz[3 + dz];
    const bool okm = fx[3 - dx] && fy[3 - dy] && fz[3 - dz];
    // missing neighbours: loads at the own cell; the stored +d coefficient is an
    // exact zero there and the mirrored one is selected away
    av[2 * j] = ah[c];
    const T am = ah[okm ? c - d : c];
    av[2 * j + 1] = okm ? am : (T)0;
    xv[2 * j] = x_at(okp ? I + dx : I, okp ? J + dy : J, okp ? Z + dz : Z, okp ? c + d : c);
    xv[2 * j + 1] = x_at(okm ? I - dx : I, okm ? J - dy : J, okm ? Z - dz : Z, okm ? c - d : c);
  }
  // FP32 levels: the row sum in the centre slot, the offsets on differences (rowsum_form)
  const T xc = (W == 0 || rowsum_form<T>()) ? x_at(I, J, Z, c) : (T)0, o = rowsum_form<T>() ? xc : (T)0;
  T s = W == 0 ? L.a[c] * xc : (T)0;
#pragma unroll
  for (int j = 0; j < 2 * CNT; ++j) s = fma(av[j], rs_diff(xv[j], o), s);
  return s;
}

// The stored offsets of the wide shapes as a table in constant memory, packed
// (dx + 3) | (dy + 3) << 4 | (dz + 3) << 8.
template <int NO>
struct HalfOffs {
  int v[Shape<NO>::NH];
};
template <int NO>
constexpr HalfOffs<NO> half_offs() {
  HalfOffs<NO> t{};
  for (int h = 0; h < Shape<NO>::NH; ++h) {
    int dx = 0, dy = 0, dz = 0;
    st_off<NO>(half_full_index<NO>(h), dx, dy, dz);
    t.v[h] = (dx + 3) | (dy + 3) << 4 | (dz + 3) << 8;
  }
  return t;
}
__constant__ HalfOffs<81> c_hoffs81 = half_offs<81>();
__constant__ HalfOffs<179> c_hoffs179 = half_offs<179>();
template <int NO>
__device__ __forceinline__ int half_off_packed(int h) {
  if constexpr (NO == 179) return c_hoffs179.v[h];
  else return c_hoffs81.v[h];
}

// st_row_part for the double-float levels of the wide shapes: one loop body for
// every warp (the warp index only picks the first offset), the offsets from the
// table above, U offsets' loads issued before their products are added. The sum
// runs over the same terms in the same order as st_row_part. The unrolled form
// has G distinct bodies, which in double-float outgrow the instruction cache
// (179 points: 2.3x the FP64 kernel's time).
template <typename T, int NO, typename XA>
__device__ __forceinline__ T st_row_part_loop(const StLevelT<T>& L, int c, int I, int J, int Z, int w, XA x_at) {
  static_assert(!rowsum_form<T>(), "row-sum levels act on differences");
  static_assert(NO == 81 || NO == 179, "wide shapes only");
  constexpr int NH = Shape<NO>::NH, G = SplitG<NO>::G, U = 4;
  const int64_t n = L.n();
  const int X = L.X, XY = L.X * L.Y;
  T s = w == 0 ? L.a[c] * x_at(I, J, Z, c) : (T)0;
  for (int h0 = w == 0 ? G : w; h0 < NH; h0 += G * U) {
    T av[2 * U], xv[2 * U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int h = h0 + G * u;
      const bool in = h < NH;
      const int p = half_off_packed<NO>(in ? h : 0);  // h = 0: the zero offset
      const int dx = (p & 15) - 3, dy = (p >> 4 & 15) - 3, dz = (p >> 8) - 3;
      const int d = dx + X * dy + XY * dz;
      const bool okp = in && (unsigned)(I + dx) < (unsigned)L.X && (unsigned)(J + dy) < (unsigned)L.Y &&
                       (unsigned)(Z + dz) < (unsigned)L.Z;
      const bool okm = in && (unsigned)(I - dx) < (unsigned)L.X && (unsigned)(J - dy) < (unsigned)L.Y &&
                       (unsigned)(Z - dz) < (unsigned)L.Z;
      // as in st_row_part: loads at the own cell where a neighbour is missing, the
      // stored +d coefficient there is an exact zero, the mirrored one selected away
      const T* ah = L.a + (int64_t)(in ? h : 0) * n;
      const T ap = ah[c];
      const T am = ah[okm ? c - d : c];
      av[2 * u] = in ? ap : (T)0;
      av[2 * u + 1] = okm ? am : (T)0;
      xv[2 * u] = x_at(okp ? I + dx : I, okp ? J + dy : J, okp ? Z + dz : Z, okp ? c + d : c);
      xv[2 * u + 1] = x_at(okm ? I - dx : I, okm ? J - dy : J, okm ? Z - dz : Z, okm ? c - d : c);
    }
#pragma unroll
    for (int j = 0; j < 2 * U; ++j) s = fma(av[j], xv[j], s);
  }
  return s;
}

template <typename T, int NO, typename XA>
__device__ __forceinline__ T st_row_part_any(const StLevelT<T>& L, int c, int I, int J, int Z, int w, XA x_at) {
  if constexpr (std::is_same<T, dfloat>::value) {
    return st_row_part_loop<T, NO>(L, c, I, J, Z, w, x_at);
  } else {
    switch (w) {  // uniform per warp
      case 0: return st_row_part<T, NO, 0>(L, c, I, J, Z, x_at);
      case 1: return st_row_part<T, NO, 1>(L, c, I, J, Z, x_at);
      case 2: return st_row_part<T, NO, 2>(L, c, I, J, Z, x_at);
      case 3: return st_row_part<T, NO, 3>(L, c, I, J, Z, x_at);
    }
    if constexpr (SplitG<NO>::G > 4) {
      switch (w) {
        case 4: return st_row_part<T, NO, 4>(L, c, I, J, Z, x_at);
        case 5: return st_row_part<T, NO, 5>(L, c, I, J, Z, x_at);
        case 6: return st_row_part<T, NO, 6>(L, c, I, J, Z, x_at);
        case 7: return st_row_part<T, NO, 7>(L, c, I, J, Z, x_at);
      }
    }
    return (T)0;
  }
}

// (A x)_c for the cell of this lane, complete in warp 0 (other warps: undefined).
// Every thread of the block must call it (it holds a block barrier).
template <typename T, int NO, typename XA>
__device__ __forceinline__ T st_row_split(const StLevelT<T>& L, bool live, int c, int I, int J, int Z, XA x_at) {
  constexpr int G = SplitG<NO>::G;
  __shared__ T part[G][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  part[w][lane] = live ? st_row_part_any<T, NO>(L, c, I, J, Z, w, x_at) : (T)0;
  __syncthreads();
  T t = (T)0;
  if (w == 0)
    for (int g = 0; g < G; ++g) t += part[g][lane];
  return t;
}

#define HD_SPLIT_CELL                                                 \
  const int64_t c64 = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31); \
  const bool live = c64 < L.n();                                      \
  const int c = live ? (int)c64 : 0;                                  \
  int I = 0, J = 0, Z = 0;                                            \
  if (live) lat_coords(c, L.X, L.Y, I, J, Z);                         \
  const bool fin = live && threadIdx.x < 32;

template <typename T, int NO>
__global__ void __launch_bounds__(32 * SplitG<NO>::G)
    k_st_jacobi_split(StLevelT<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo) {
  HD_SPLIT_CELL
  auto xa = [&](int, int, int, int k) { return x[k]; };
  const T ax = st_row_split<T, NO>(L, live, c, I, J, Z, xa);
  if (fin) xo[c] = fma(L.dinv[c], b[c] - ax, x[c]);
}

template <typename T, int NO>
__global__ void __launch_bounds__(32 * SplitG<NO>::G)
    k_st_resid_split(StLevelT<T> L, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  HD_SPLIT_CELL
  auto xa = [&](int, int, int, int k) { return x[k]; };
  const T ax = st_row_split<T, NO>(L, live, c, I, J, Z, xa);
  if (fin) r[c] = b[c] - ax;
}

template <typename T, int NO>
__global__ void __launch_bounds__(32 * SplitG<NO>::G)
    k_st_scale_jacobi_split(StLevelT<T> L, const T* __restrict__ b, T* __restrict__ xo) {
  HD_SPLIT_CELL
  auto xa = [&](int, int, int, int k) { return L.dinv[k] * b[k]; };
  const T ax = st_row_split<T, NO>(L, live, c, I, J, Z, xa);
  if (fin) xo[c] = fma(L.dinv[c], b[c] - ax, xa(I, J, Z, c));
}

template <typename T, int NO>
__global__ void __launch_bounds__(32 * SplitG<NO>::G)
    k_st_jacobi_prolong_split(StLevelT<T> L, CDims cd, const T* __restrict__ b, const T* __restrict__ x,
                              const T* __restrict__ e, T* __restrict__ xo) {
  HD_SPLIT_CELL
  auto xa = [&](int i, int j, int z, int k) {
    return x[k] + e[agg_of(cd.ag[0], i) + cd.X * (agg_of(cd.ag[1], j) + cd.Y * agg_of(cd.ag[2], z))];
  };
  const T ax = st_row_split<T, NO>(L, live, c, I, J, Z, xa);
  if (fin) xo[c] = fma(L.dinv[c], b[c] - ax, xa(I, J, Z, c));
}
#undef HD_SPLIT_CELL

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
  for (int k = agg_lo(cd.ag[2], Cz); k < agg_hi(cd.ag[2], Cz, Z); ++k)
    for (int j = agg_lo(cd.ag[1], Cy); j < agg_hi(cd.ag[1], Cy, Y); ++j)
      for (int i = agg_lo(cd.ag[0], Cx); i < agg_hi(cd.ag[0], Cx, X); ++i) s += r[i + (int64_t)X * (j + (int64_t)Y * k)];
  bc[C] = s;
}

template <typename T>
__global__ void k_st_prolong_add(StLevelT<T> L, CDims cd, const T* __restrict__ e, T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  x[c] += e[agg_of(cd.ag[0], I) + (int64_t)cd.X * (agg_of(cd.ag[1], J) + (int64_t)cd.Y * agg_of(cd.ag[2], Z))];
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
    return x[k] + e[agg_of(cd.ag[0], i) + cd.X * (agg_of(cd.ag[1], j) + cd.Y * agg_of(cd.ag[2], z))];
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
  // no branches: a missing slot (no step out of the aggregate) holds an exact
  // zero and points at the own aggregate
  const int sx = out_step(I, L.X, cd.fx), sy = out_step(J, L.Y, cd.fy), sz = out_step(Z, L.Z, cd.fz);
  const T p0 = pv[c], p1 = pv[n + c], p2 = pv[2 * n + c], p3 = pv[3 * n + c];
  const T e0 = ev(Dx, Dy, Dz), e1 = ev(agg(I + sx, cd.fx), Dy, Dz), e2 = ev(Dx, agg(J + sy, cd.fy), Dz),
          e3 = ev(Dx, Dy, agg(Z + sz, cd.fz));
  T v = p0 * e0;
  v = fma(p1, e1, v);
  v = fma(p2, e2, v);
  v = fma(p3, e3, v);
  x[c] += v;
}

// -- level 0 with element-aligned aggregates (any groups per axis) ---------------------
// A fine cell's row of P_0 = (I - omega D_l1^-1 S~) P0 has its own aggregate and, for
// each face that leaves the aggregate, the aggregate across it: with groups of one
// cell both faces along an axis can leave it. Stored as [7][n]: slot 0 the own
// aggregate, slot 1 + 2 d + t the aggregate across the face of axis d on the low
// (t = 0) or high (t = 1) side (0 when that face stays inside or is on the boundary).
constexpr int PG_SLOTS = 7;

__global__ void k_sa_pvals_g(LevelT<double> L, CDims cd, double* __restrict__ pv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n();
  if (i >= n) return;
  int crd[3];
  lat_coords(i, L.X, L.Y, crd[0], crd[1], crd[2]);
  const int ext[3] = {L.X, L.Y, L.Z};
  const Face7<double> f = faces7(L, crd[0], crd[1], crd[2]);
  const double wd = SA_OMEGA * L.dinv[i];
  double inner = 0.0;
  for (int d = 0; d < 3; ++d) {
    const int a = agg_of(cd.ag[d], crd[d]);
    for (int t = 0; t < 2; ++t) {
      const int nb = crd[d] + (t ? 1 : -1);
      double v = 0.0;
      if (nb >= 0 && nb < ext[d]) {
        if (agg_of(cd.ag[d], nb) == a) inner += f.w[2 * d + t];
        else v = wd * f.w[2 * d + t];
      }
      pv[(1 + 2 * d + t) * n + i] = v;
    }
  }
  pv[i] = 1.0 - wd * (L.diag[i] - inner);
}

// A_1 = P_0^T S~ P_0 (81-point shape), one thread per coarse cell C: over the support
// of column C (the aggregate, and the cells one step outside it along one axis), every
// stencil neighbour j and every nonzero of row j of P_0.
__global__ void k_sa_galerkin_g(LevelT<double> L, CDims c, const double* __restrict__ pv, StLevelT<double> A1,
                                int* __restrict__ bad) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = A1.n();
  if (C >= nc) return;
  int Cc[3];
  lat_coords(C, c.X, c.Y, Cc[0], Cc[1], Cc[2]);
  const int ext[3] = {L.X, L.Y, L.Z};
  const int64_t n = L.n();
  int lo[3], hi[3];  // aggregate [lo, hi)
  for (int d = 0; d < 3; ++d) {
    lo[d] = agg_lo(c.ag[d], Cc[d]);
    hi[d] = agg_hi(c.ag[d], Cc[d], ext[d]);
  }
  double acc[81];
  for (int o = 0; o < 81; ++o) acc[o] = 0.0;
  for (int Z = max(lo[2] - 1, 0); Z <= min(hi[2], ext[2] - 1); ++Z)
    for (int J = max(lo[1] - 1, 0); J <= min(hi[1], ext[1] - 1); ++J)
      for (int I = max(lo[0] - 1, 0); I <= min(hi[0], ext[0] - 1); ++I) {
        const int ic[3] = {I, J, Z};
        int out = -1, nout = 0;
        for (int d = 0; d < 3; ++d)
          if (ic[d] < lo[d] || ic[d] >= hi[d]) {
            out = d;
            ++nout;
          }
        if (nout > 1) continue;
        const int64_t i = I + (int64_t)L.X * (J + (int64_t)L.Y * Z);
        // slot of column C in row i: own, or across the face of axis `out` towards the aggregate
        const int slot = nout == 0 ? 0 : 1 + 2 * out + (ic[out] < lo[out] ? 1 : 0);
        const double p = pv[slot * n + i];
        if (p == 0.0) continue;
        const Face7<double> f = faces7(L, I, J, Z);
        for (int k = 0; k < 7; ++k) {
          int jc[3] = {I, J, Z};
          double a;
          if (k == 0) {
            a = L.diag[i];
          } else {
            const int d = (k - 1) >> 1, t = (k - 1) & 1;
            jc[d] += t ? 1 : -1;
            if (jc[d] < 0 || jc[d] >= ext[d]) continue;
            a = -f.w[k - 1];
          }
          const int64_t j = jc[0] + (int64_t)L.X * (jc[1] + (int64_t)L.Y * jc[2]);
          const int Dj[3] = {agg_of(c.ag[0], jc[0]), agg_of(c.ag[1], jc[1]), agg_of(c.ag[2], jc[2])};
          for (int sl = 0; sl < PG_SLOTS; ++sl) {
            const double q = pv[sl * n + j];
            if (q == 0.0) continue;
            int D[3] = {Dj[0], Dj[1], Dj[2]};
            if (sl > 0) {
              const int d = (sl - 1) >> 1, t = (sl - 1) & 1;
              D[d] = agg_of(c.ag[d], jc[d] + (t ? 1 : -1));  // a nonzero slot has this neighbour
            }
            const int o = st_index<81>(D[0] - Cc[0], D[1] - Cc[1], D[2] - Cc[2]);
            if (o < 0) {
              atomicExch(bad, 1);
              continue;
            }
            acc[o] = fma(p * a, q, acc[o]);
          }
        }
      }
  for (int o = 0; o < 81; ++o) A1.a[o * nc + C] = acc[o];
}

// b_C = (P_0^T r)_C: the aggregate's cells (slot 0), then along each axis the layer
// just below the aggregate (their high-side slot) and just above it (low-side slot)
template <typename T>
__global__ void k_sa_restrict0_g(LevelT<T> L, CDims cd, const T* __restrict__ pv, const T* __restrict__ r,
                                 T* __restrict__ bc) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (C >= (int64_t)cd.X * cd.Y * cd.Z) return;
  int Cc[3];
  lat_coords(C, cd.X, cd.Y, Cc[0], Cc[1], Cc[2]);
  const int ext[3] = {L.X, L.Y, L.Z};
  const int64_t str[3] = {1, (int64_t)L.X, (int64_t)L.X * L.Y};
  const int64_t n = L.n();
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = agg_lo(cd.ag[d], Cc[d]);
    hi[d] = agg_hi(cd.ag[d], Cc[d], ext[d]);
  }
  T s = (T)0;
  for (int z = lo[2]; z < hi[2]; ++z)
    for (int y = lo[1]; y < hi[1]; ++y)
      for (int x = lo[0]; x < hi[0]; ++x) {
        const int64_t i = x + str[1] * y + str[2] * z;
        s = fma(pv[i], r[i], s);
      }
  for (int d = 0; d < 3; ++d) {
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    const int layer[2] = {lo[d] - 1, hi[d]};
    for (int t = 0; t < 2; ++t) {
      const int c = layer[t];
      if (c < 0 || c >= ext[d]) continue;
      const int64_t slot = 1 + 2 * d + (t == 0 ? 1 : 0);
      for (int b = lo[e2]; b < hi[e2]; ++b)
        for (int a = lo[e1]; a < hi[e1]; ++a) {
          const int64_t i = str[d] * c + str[e1] * a + str[e2] * b;
          s = fma(pv[slot * n + i], r[i], s);
        }
    }
  }
  bc[C] = s;
}

// x += P_0 e
template <typename T>
__global__ void k_sa_prolong0_g(LevelT<T> L, CDims cd, const T* __restrict__ pv, const T* __restrict__ e,
                                T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n();
  if (c >= n) return;
  int crd[3];
  lat_coords(c, L.X, L.Y, crd[0], crd[1], crd[2]);
  const int ext[3] = {L.X, L.Y, L.Z};
  const int D[3] = {agg_of(cd.ag[0], crd[0]), agg_of(cd.ag[1], crd[1]), agg_of(cd.ag[2], crd[2])};
  auto ev = [&](int ex, int ey, int ez) { return e[ex + (int64_t)cd.X * (ey + (int64_t)cd.Y * ez)]; };
  T v = pv[c] * ev(D[0], D[1], D[2]);
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 2; ++t) {
      const int nb = crd[d] + (t ? 1 : -1);
      // a slot without a neighbour outside the aggregate holds an exact zero: point it at the own one
      int A[3] = {D[0], D[1], D[2]};
      if (nb >= 0 && nb < ext[d]) A[d] = agg_of(cd.ag[d], nb);
      v = fma(pv[(1 + 2 * d + t) * n + c], ev(A[0], A[1], A[2]), v);
    }
  x[c] += v;
}

// -- level 1 -> 2 with a smoothed prolongator (smooth_levels = 2) --------------------
// P_1 = (I - omega D_l1^-1 A_1) P0 on the 33-point level 1. Along a direction with
// factor 2, let s = +1 for an odd fine coordinate and -1 for an even one (the side
// on which the cell's aggregate has its other cell). A fine cell's row of P_1 then
// has at most 11 nonzeros: slots 0..7, the aggregates agg + (b0 sx, b1 sy, b2 sz)
// for bits b of the slot (slot 0 is the own aggregate), reached through the box
// offsets and the axial steps towards s; slots 8 + d, the aggregate at -s along d
// alone, reached through the axial step of 2 away from s. Stored as [11][n1].
constexpr int P1_SLOTS = 11;

struct AxisPos {  // fine coordinate along one direction: aggregate and side
  int a, s;
};
__device__ __forceinline__ AxisPos axis_pos(int I, int f) { return AxisPos{I >> (f - 1), f == 2 ? ((I & 1) ? 1 : -1) : 0}; }

// slot of the aggregate at offset D from the cell's own, -1 if the row has none
__device__ __forceinline__ int p1_slot(const int D[3], const int s[3]) {
  int bits = 0, far = -1;
  for (int d = 0; d < 3; ++d) {
    if (D[d] == 0) continue;
    if (s[d] != 0 && D[d] == s[d]) {
      bits |= 1 << d;
    } else if (s[d] != 0 && D[d] == -s[d] && far < 0) {
      far = d;
    } else {
      return -1;
    }
  }
  if (far >= 0) return bits ? -1 : 8 + far;
  return bits;
}
// coarse cell t of slot k for a fine cell with aggregate a and sides s; false when
// the slot has no aggregate inside the coarse lattice ce
__device__ __forceinline__ bool p1_target(int k, const int a[3], const int s[3], const int ce[3], int t[3]) {
  for (int d = 0; d < 3; ++d) t[d] = a[d];
  if (k < 8) {
    for (int d = 0; d < 3; ++d)
      if ((k >> d) & 1) {
        if (!s[d]) return false;
        t[d] += s[d];
      }
  } else {
    const int d = k - 8;
    if (!s[d]) return false;
    t[d] -= s[d];
  }
  for (int d = 0; d < 3; ++d)
    if (t[d] < 0 || t[d] >= ce[d]) return false;
  return true;
}

// P_1 from the full-storage 33-point level (its l1 inverse diagonal included)
__global__ void k_sa_pvals1(StLevelT<double> A1, CDims cd, double* __restrict__ p1, int* __restrict__ bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = A1.n();
  if (i >= n) return;
  int I, J, Z;
  lat_coords(i, A1.X, A1.Y, I, J, Z);
  const AxisPos px = axis_pos(I, cd.fx), py = axis_pos(J, cd.fy), pz = axis_pos(Z, cd.fz);
  const int s[3] = {px.s, py.s, pz.s};
  double acc[P1_SLOTS];
  for (int k = 0; k < P1_SLOTS; ++k) acc[k] = 0.0;
  acc[0] = 1.0;
  const double wd = SA_OMEGA * A1.dinv[i];
  for (int o = 0; o < 33; ++o) {
    const double a = A1.a[o * n + i];
    if (a == 0.0) continue;
    int dx, dy, dz;
    st_off<33>(o, dx, dy, dz);
    const int jI = I + dx, jJ = J + dy, jZ = Z + dz;
    if (jI < 0 || jI >= A1.X || jJ < 0 || jJ >= A1.Y || jZ < 0 || jZ >= A1.Z) {
      atomicExch(bad, 1);
      continue;
    }
    const int D[3] = {(jI >> (cd.fx - 1)) - px.a, (jJ >> (cd.fy - 1)) - py.a, (jZ >> (cd.fz - 1)) - pz.a};
    const int k = p1_slot(D, s);
    if (k < 0) {
      atomicExch(bad, 1);
      continue;
    }
    acc[k] -= wd * a;
  }
  for (int k = 0; k < P1_SLOTS; ++k) p1[k * n + i] = acc[k];
}

// Enumerates the fine cells i with a slot for coarse cell C in their row of P_1
// and calls fn(i, I, J, Z, slot). Per direction with factor 2 the candidates are
// 2C-2 .. 2C+3 (the aggregate, one layer on each side through the box slots and a
// second layer through the axial slot); factor 1 leaves C itself.
template <typename F>
__device__ __forceinline__ void for_support1(int X, int Y, int Zn, const CDims& cd, int Cx, int Cy, int Cz, F fn) {
  const int x0 = cd.fx == 2 ? max(2 * Cx - 2, 0) : Cx, x1 = cd.fx == 2 ? min(2 * Cx + 3, X - 1) : Cx;
  const int y0 = cd.fy == 2 ? max(2 * Cy - 2, 0) : Cy, y1 = cd.fy == 2 ? min(2 * Cy + 3, Y - 1) : Cy;
  const int z0 = cd.fz == 2 ? max(2 * Cz - 2, 0) : Cz, z1 = cd.fz == 2 ? min(2 * Cz + 3, Zn - 1) : Cz;
  for (int Z = z0; Z <= z1; ++Z)
    for (int J = y0; J <= y1; ++J)
      for (int I = x0; I <= x1; ++I) {
        const AxisPos px = axis_pos(I, cd.fx), py = axis_pos(J, cd.fy), pz = axis_pos(Z, cd.fz);
        const int s[3] = {px.s, py.s, pz.s};
        const int D[3] = {Cx - px.a, Cy - py.a, Cz - pz.a};
        const int k = p1_slot(D, s);
        if (k >= 0) fn(I + X * (J + Y * Z), I, J, Z, k);
      }
}

// A_2 = P_1^T A_1 P_1 (179-point), one thread per coarse cell C: for every fine i
// in the support of column C, every neighbour j of i and every slot of row j
template <int NOUT>
__global__ void k_sa_galerkin1(StLevelT<double> A1, CDims cd, const double* __restrict__ p1, StLevelT<double> A2,
                               int* __restrict__ bad) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nc = A2.n();
  if (C >= nc) return;
  int Cx, Cy, Cz;
  lat_coords(C, cd.X, cd.Y, Cx, Cy, Cz);
  const int64_t n = A1.n();
  const int ce[3] = {cd.X, cd.Y, cd.Z};
  double acc[NOUT];
  for (int o = 0; o < NOUT; ++o) acc[o] = 0.0;
  for_support1(A1.X, A1.Y, A1.Z, cd, Cx, Cy, Cz, [&](int i, int I, int J, int Z, int k) {
    const double p = p1[k * n + i];
    if (p == 0.0) return;
    for (int o = 0; o < 33; ++o) {
      const double a = A1.a[o * n + i];
      if (a == 0.0) continue;
      int dx, dy, dz;
      st_off<33>(o, dx, dy, dz);
      const int jI = I + dx, jJ = J + dy, jZ = Z + dz;
      if (jI < 0 || jI >= A1.X || jJ < 0 || jJ >= A1.Y || jZ < 0 || jZ >= A1.Z) {
        atomicExch(bad, 1);
        continue;
      }
      const int j = jI + A1.X * (jJ + A1.Y * jZ);
      const AxisPos qx = axis_pos(jI, cd.fx), qy = axis_pos(jJ, cd.fy), qz = axis_pos(jZ, cd.fz);
      const int ja[3] = {qx.a, qy.a, qz.a}, js[3] = {qx.s, qy.s, qz.s};
      for (int t = 0; t < P1_SLOTS; ++t) {
        int e[3];
        if (!p1_target(t, ja, js, ce, e)) continue;
        const double q = p1[t * n + j];
        if (q == 0.0) continue;
        const int oc = st_index<NOUT>(e[0] - Cx, e[1] - Cy, e[2] - Cz);
        if (oc < 0) {
          atomicExch(bad, 1);
          continue;
        }
        acc[oc] = fma(p * a, q, acc[oc]);
      }
    }
  });
  for (int o = 0; o < NOUT; ++o) A2.a[o * nc + C] = acc[o];
}

// b_C = (P_1^T r)_C, one thread per coarse cell (neighbouring threads then read
// neighbouring aggregates). The support is enumerated directly: per direction
// with factor 2 the positions 2C-1 .. 2C+2 through the box slots (bit 1 at the
// two outer ones), then 2C-2 / 2C+3 through the axial slot with the other two
// directions inside the aggregate; 64 + 24 fine cells. Each row of four is
// loaded before it is added; a missing cell reads the aggregate's first cell
// with weight zero.
template <typename T>
__global__ void k_sa_restrict1(StLevelT<T> L, CDims cd, const T* __restrict__ p1, const T* __restrict__ r,
                               T* __restrict__ bc) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (C >= (int64_t)cd.X * cd.Y * cd.Z) return;
  int Cx, Cy, Cz;
  lat_coords(C, cd.X, cd.Y, Cx, Cy, Cz);
  const int64_t n = L.n();
  const int64_t sy = L.X, sz = (int64_t)L.X * L.Y;
  // position q = 0..3 of the box part along a direction: fine coordinate, slot bit
  auto box_pos = [](int f, int ce, int extent, int q, int& x, int& bit) {
    if (f == 2) {
      x = 2 * ce - 1 + q;
      bit = (q == 0 || q == 3);
      return x >= 0 && x < extent;
    }
    x = ce;
    bit = 0;
    return q == 1;
  };
  const int64_t i0 = (cd.fx == 2 ? 2 * Cx : Cx) + sy * (cd.fy == 2 ? 2 * Cy : Cy) + sz * (cd.fz == 2 ? 2 * Cz : Cz);
  T s = (T)0;
  for (int row = 0; row < 16; ++row) {
    int y, z, by, bz;
    const bool okr = box_pos(cd.fy, Cy, L.Y, row & 3, y, by) & box_pos(cd.fz, Cz, L.Z, row >> 2, z, bz);
    T pw[4], rv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int x, bx;
      const bool ok = okr & box_pos(cd.fx, Cx, L.X, q, x, bx);
      const int64_t i = ok ? x + sy * y + sz * z : i0;
      const T p = p1[(ok ? (bx | (by << 1) | (bz << 2)) : 0) * n + i];
      pw[q] = ok ? p : (T)0;
      rv[q] = r[i];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) s = fma(pw[q], rv[q], s);
  }
  // axial cells, direction d: (side, lateral bits u, v) over the other two
  // directions in the order (d + 1) % 3, (d + 2) % 3
  auto axial = [&](int d, int fd, int cdd, int extd, int fa, int ca, int exta, int fb, int cb, int extb, int64_t sdd,
                   int64_t sa, int64_t sb) {
    T pw[8], rv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int side = k >> 2, u = k & 1, v = (k >> 1) & 1;
      const int pd = side ? 2 * cdd + 3 : 2 * cdd - 2;
      const int pa = fa == 2 ? 2 * ca + u : ca, pb = fb == 2 ? 2 * cb + v : cb;
      const bool ok = fd == 2 && pd >= 0 && pd < extd && (fa == 2 || u == 0) && pa < exta && (fb == 2 || v == 0) &&
                      pb < extb;
      const int64_t i = ok ? sdd * pd + sa * pa + sb * pb : i0;
      const T p = p1[(8 + d) * n + i];
      pw[k] = ok ? p : (T)0;
      rv[k] = r[i];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fma(pw[k], rv[k], s);
  };
  axial(0, cd.fx, Cx, L.X, cd.fy, Cy, L.Y, cd.fz, Cz, L.Z, 1, sy, sz);
  axial(1, cd.fy, Cy, L.Y, cd.fz, Cz, L.Z, cd.fx, Cx, L.X, sy, sz, 1);
  axial(2, cd.fz, Cz, L.Z, cd.fx, Cx, L.X, cd.fy, Cy, L.Y, sz, 1, sy);
  bc[C] = s;
}

// x += P_1 e. A slot without an aggregate holds an exact zero, so its target is
// only clamped into the coarse lattice (no branch per slot).
template <typename T>
__global__ void k_sa_prolong1(StLevelT<T> L, CDims cd, const T* __restrict__ p1, const T* __restrict__ e,
                              T* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = L.n();
  if (c >= n) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  const AxisPos px = axis_pos(I, cd.fx), py = axis_pos(J, cd.fy), pz = axis_pos(Z, cd.fz);
  // coarse coordinate a + m s per direction, clamped, for m = -1, 0, 1
  auto cl = [](int v, int hi) { return min(max(v, 0), hi - 1); };
  const int xs[3] = {cl(px.a - px.s, cd.X), px.a, cl(px.a + px.s, cd.X)};
  const int ys[3] = {cl(py.a - py.s, cd.Y), py.a, cl(py.a + py.s, cd.Y)};
  const int zs[3] = {cl(pz.a - pz.s, cd.Z), pz.a, cl(pz.a + pz.s, cd.Z)};
  auto ev = [&](int ix, int iy, int iz) { return e[xs[ix] + cd.X * (ys[iy] + cd.Y * zs[iz])]; };
  T v = (T)0;
#pragma unroll
  for (int k = 0; k < 8; ++k) v = fma(p1[k * n + c], ev(1 + (k & 1), 1 + ((k >> 1) & 1), 1 + (k >> 2)), v);
  v = fma(p1[8 * n + c], ev(0, 1, 1), v);
  v = fma(p1[9 * n + c], ev(1, 0, 1), v);
  v = fma(p1[10 * n + c], ev(1, 1, 0), v);
  x[c] += v;
}

// row sums of a FP64 stencil level (its row applied to the constant 1), the centre
// slot of its FP32 copy (rowsum_form)
template <int NO>
__global__ void k_st_rowsum(StLevelT<double> L, float* __restrict__ centre) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= L.n()) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  auto one = [](int, int, int, int) { return 1.0; };
  centre[c] = (float)st_row<double, NO>(L, (int)c, I, J, Z, one);
}

template <typename T>
__global__ void k_to_f32_sa(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (T)a[i];
}

template <typename Lv>
CDims cdims_of(const Lv& c) {
  return CDims{c.X, c.Y, c.Z, c.fx, c.fy, c.fz, {c.ag[0], c.ag[1], c.ag[2]}};
}

// -- the cycle ----------------------------------------------------------------------
// levels >= 1: st[l - 1]; the last one is solved densely. p1: the smoothed
// prolongator from level 1 to level 2 (nullptr: plain aggregation there too).
template <typename T>
const T* sa_level(hd_op* h, std::vector<StLevelT<T>>& st, const T* p1, int l, const T* b, T* out) {
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
  const bool smoothed = l == 1 && p1 != nullptr;
  const unsigned g = nblk(L.n());
  cudaStream_t sm = h->stream;
  // wide shapes: 32 cells per block of SplitG warps
  const unsigned gs = (unsigned)((L.n() + 31) / 32);
  auto jacobi = [&](const T* x, T* xo) {
    with_shape(L.no, [&](auto t) {
      constexpr int NO = decltype(t)::value;
      if constexpr (NO >= 81) k_st_jacobi_split<T, NO><<<gs, 32 * SplitG<NO>::G, 0, sm>>>(L, b, x, xo);
      else k_st_jacobi<T, NO><<<g, TPB, 0, sm>>>(L, b, x, xo);
    });
  };
  auto prolong = [&](const T* xc, T* x) {
    if (smoothed) k_sa_prolong1<T><<<g, TPB, 0, sm>>>(L, cd, p1, xc, x);
    else k_st_prolong_add<T><<<g, TPB, 0, sm>>>(L, cd, xc, x);
  };
  T* cur = L.x0;
  int s0 = 1;
  const bool fuse = L.n() <= FUSE_MAX;
  if (nu >= 2 && fuse) {  // the first two sweeps fused
    with_shape(L.no, [&](auto t) {
      constexpr int NO = decltype(t)::value;
      if constexpr (NO >= 81) k_st_scale_jacobi_split<T, NO><<<gs, 32 * SplitG<NO>::G, 0, sm>>>(L, b, cur);
      else k_st_scale_jacobi<T, NO><<<g, TPB, 0, sm>>>(L, b, cur);
    });
    s0 = 2;
  } else {
    k_st_scale<T><<<g, TPB, 0, sm>>>(L, b, cur);
  }
  for (int s = s0; s < nu; ++s) {
    T* o = (cur == L.x0) ? L.x1 : L.x0;
    jacobi(cur, o);
    cur = o;
  }
  const int repeats = (h->cycle == 2 && l + 1 < last && (h->w_levels == 0 || l < h->w_levels)) ? 2 : 1;
  const T* xc = nullptr;
  for (int rep = 0; rep < repeats; ++rep) {
    if (rep > 0) prolong(xc, cur);
    T* rtmp = (cur == L.x0) ? L.x1 : L.x0;  // free until the post-smoothing
    with_shape(L.no, [&](auto t) {
      constexpr int NO = decltype(t)::value;
      if constexpr (NO >= 81) k_st_resid_split<T, NO><<<gs, 32 * SplitG<NO>::G, 0, sm>>>(L, b, cur, rtmp);
      else k_st_resid<T, NO><<<g, TPB, 0, sm>>>(L, b, cur, rtmp);
    });
    if (smoothed) k_sa_restrict1<T><<<nblk(C.n()), TPB, 0, sm>>>(L, cd, p1, rtmp, C.b);
    else k_agg_sum<T><<<nblk(C.n()), TPB, 0, sm>>>(L.X, L.Y, L.Z, cd, rtmp, C.b);
    xc = sa_level<T>(h, st, p1, l + 1, C.b, nullptr);
  }
  T* o = (nu == 1 && out) ? out : ((cur == L.x0) ? L.x1 : L.x0);
  if (fuse && !smoothed) {
    with_shape(L.no, [&](auto t) {
      constexpr int NO = decltype(t)::value;
      if constexpr (NO >= 81)
        k_st_jacobi_prolong_split<T, NO><<<gs, 32 * SplitG<NO>::G, 0, sm>>>(L, cd, b, cur, xc, o);
      else k_st_jacobi_prolong<T, NO><<<g, TPB, 0, sm>>>(L, cd, b, cur, xc, o);
    });
  } else {
    prolong(xc, cur);
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
void sa_cycle0(hd_op* h, LevelT<T>& L, const T* pv, std::vector<StLevelT<T>>& st, const T* p1, const T* b,
               T* out) {
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
  auto prolong0 = [&](const T* e, T* x) {
    if (h->sa_gen) k_sa_prolong0_g<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, pv, e, x);
    else k_sa_prolong0<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, cd, pv, e, x);
  };
  for (int rep = 0; rep < repeats; ++rep) {
    if (rep > 0) prolong0(xc, cur);
    k_sa_res0<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, L.b);
    if (h->sa_gen) k_sa_restrict0_g<T><<<nblk(st[0].n()), TPB, 0, h->stream>>>(L, cd, pv, L.b, st[0].b);
    else k_sa_restrict0<T><<<nblk(st[0].n()), TPB, 0, h->stream>>>(L, cd, pv, L.b, st[0].b);
    xc = sa_level<T>(h, st, p1, 1, st[0].b, nullptr);
  }
  prolong0(xc, cur);
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
  const int64_t na = std::is_same<T, double>::value ? L.no : n_half(L.no);
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
  const LevelT<double>& l1 = h->lv[1];
  // element-aligned groups of one cell: the general level-0 transfer (7 slots per cell)
  h->sa_gen = !agg_pairs(l1.ag);
  if (h->sa_gen && h->sa >= 2)
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "smooth_levels = 2 with element-aligned groups of one cell");
  const int slots = h->sa_gen ? PG_SLOTS : 4;
  if (cudaMalloc(&h->sa_p, sizeof(double) * slots * n0) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "SA prolongator");
  if (h->sa_gen) k_sa_pvals_g<<<nblk(n0), TPB, 0, h->stream>>>(L0, cdims_of(l1), h->sa_p);
  else k_sa_pvals<<<nblk(n0), TPB, 0, h->stream>>>(L0, l1.fx, l1.fy, l1.fz, h->sa_p);
  HD_LAUNCH_CK(h, "k_sa_pvals");
  int* d_bad = nullptr;
  if (cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "flag");
  HD_CK(h, cudaMemsetAsync(d_bad, 0, sizeof(int), h->stream));
  hd_status st = HD_OK;
  const bool two = h->sa >= 2;
  for (size_t l = 1; l < h->lv.size() && st == HD_OK; ++l) {
    const LevelT<double>& g = h->lv[l];  // same lattice dimensions as the unsmoothed level
    StLevelT<double> s{};
    s.X = g.X; s.Y = g.Y; s.Z = g.Z;
    set_agg(s, g.ag[0], g.ag[1], g.ag[2]);
    // shapes: 33 on level 1; with the second smoothed level 179 on level 2 and 81
    // on level 3; 27 elsewhere. Element-aligned groups of one cell (general
    // transfers): 81 on level 1 and below every general transfer
    const bool gen = !agg_pairs(g.ag);
    if (h->sa_gen) s.no = (l == 1 || gen) ? 81 : 27;
    else s.no = (l == 1) ? 33 : (two && l == 2) ? 179 : (two && l == 3) ? 81 : 27;
    st = alloc_st<double>(h, s, true);
    h->st.push_back(s);
    if (st != HD_OK) break;
    const StLevelT<double>& S = h->st.back();
    const CDims cd = cdims_of(S);
    const unsigned gc = nblk(S.n());
    if (l == 1) {
      if (h->sa_gen) k_sa_galerkin_g<<<gc, TPB, 0, h->stream>>>(L0, cd, h->sa_p, S, d_bad);
      else k_sa_galerkin<<<gc, TPB, 0, h->stream>>>(L0, cd, h->sa_p, S, d_bad);
    } else if (gen) {
      const StLevelT<double>& F = h->st[h->st.size() - 2];
      if (F.no == 81) k_ua_galerkin<81, 81><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
      else if (F.no == 27) k_ua_galerkin<27, 81><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
      else st = hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "element-aligned groups below this stencil shape");
    } else if (two && l == 2) {
      const StLevelT<double>& A1 = h->st[0];
      if (cudaMalloc(&h->sa_p1, sizeof(double) * P1_SLOTS * A1.n()) != cudaSuccess) {
        st = hd_fail(h, HD_ERR_OOM, "SA prolongator of level 1");
        break;
      }
      k_sa_pvals1<<<nblk(A1.n()), TPB, 0, h->stream>>>(A1, cd, h->sa_p1, d_bad);
      k_sa_galerkin1<179><<<gc, TPB, 0, h->stream>>>(A1, cd, h->sa_p1, S, d_bad);
    } else {
      const StLevelT<double>& F = h->st[h->st.size() - 2];
      if (F.no == 179) k_ua_galerkin<179, 81><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
      else if (F.no == 81) k_ua_galerkin<81, 27><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
      else if (F.no == 33) k_ua_galerkin<33, 27><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
      else k_ua_galerkin<27, 27><<<gc, TPB, 0, h->stream>>>(F, cd, S, d_bad);
    }
    k_st_dinv<<<gc, TPB, 0, h->stream>>>(S);
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
          st_off_any(c.no, o, dx, dy, dz);
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
    with_shape(s.no, [&](auto t) { k_st_compress<decltype(t)::value><<<nblk(s.n()), TPB, 0, h->stream>>>(s, half); });
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
  const int64_t np0 = (h->sa_gen ? PG_SLOTS : 4) * n0;
  if (cudaMalloc(&h->sa_pf, sizeof(float) * np0) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA f32");
  k_to_f32_sa<float><<<nblk(np0), TPB, 0, h->stream>>>(np0, h->sa_p, h->sa_pf);
  if (h->sa_p1) {
    const int64_t np = P1_SLOTS * h->st[0].n();
    if (cudaMalloc(&h->sa_p1f, sizeof(float) * np) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA f32");
    k_to_f32_sa<float><<<nblk(np), TPB, 0, h->stream>>>(np, h->sa_p1, h->sa_p1f);
  }
  for (const StLevelT<double>& d : h->st) {
    StLevelT<float> f{};
    f.X = d.X; f.Y = d.Y; f.Z = d.Z; f.no = d.no;
    set_agg(f, d.ag[0], d.ag[1], d.ag[2]);
    hd_status st = alloc_st<float>(h, f, true);
    h->stf.push_back(f);
    if (st != HD_OK) return st;
    k_to_f32_sa<float><<<nblk(d.n() * n_half(d.no)), TPB, 0, h->stream>>>(d.n() * n_half(d.no), d.a, f.a);
    with_shape(d.no, [&](auto t) {  // centre slot: the FP64 row sum (rowsum_form)
      constexpr int NO = decltype(t)::value;
      k_st_rowsum<NO><<<nblk(d.n()), TPB, 0, h->stream>>>(d, f.a);
    });
    k_to_f32_sa<float><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.dinv, f.dinv);
  }
  HD_LAUNCH_CK(h, "SA f32");
  return HD_OK;
}

void sa_free(hd_op* h) {
  for (auto& s : h->st) free_st<double>(s);
  for (auto& s : h->stf) free_st<float>(s);
  for (auto& s : h->stx) free_st<dfloat>(s);
  h->st.clear();
  h->stf.clear();
  h->stx.clear();
  cudaFree(h->sa_px);
  cudaFree(h->sa_p1x);
  h->sa_px = h->sa_p1x = nullptr;
  cudaFree(h->sa_p);
  cudaFree(h->sa_pf);
  cudaFree(h->sa_p1);
  cudaFree(h->sa_p1f);
  cudaFree(h->d_sa_coarse_inv);
  h->sa_p = nullptr;
  h->sa_pf = nullptr;
  h->sa_p1 = nullptr;
  h->sa_p1f = nullptr;
  h->d_sa_coarse_inv = nullptr;
}

hd_status sa_vcycle(hd_op* h, const double* b, double* x) {
  return run_graphed(h, b, x, 2, [&]() { sa_cycle0<double>(h, h->lv[0], h->sa_p, h->st, h->sa_p1, b, x); });
}

hd_status sa_vcycle_df(hd_op* h, const dfloat* b, dfloat* x) {
  return run_graphed(h, b, x, 4, [&]() { sa_cycle0<dfloat>(h, h->lvx[0], h->sa_px, h->stx, h->sa_p1x, b, x); });
}

// double-float copies of the smoothed hierarchy (the stencil levels in half storage, the
// prolongator values), for the FP64 cycle of fp64_emulation = 2
hd_status sa_setup_df(hd_op* h) {
  if (h->st.empty() || !h->stx.empty()) return HD_OK;
  const int64_t np0 = (h->sa_gen ? PG_SLOTS : 4) * h->lv[0].n();
  if (cudaMalloc(&h->sa_px, sizeof(dfloat) * np0) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA df");
  k_to_f32_sa<dfloat><<<nblk(np0), TPB, 0, h->stream>>>(np0, h->sa_p, h->sa_px);
  if (h->sa_p1) {
    const int64_t np = P1_SLOTS * h->st[0].n();
    if (cudaMalloc(&h->sa_p1x, sizeof(dfloat) * np) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "SA df");
    k_to_f32_sa<dfloat><<<nblk(np), TPB, 0, h->stream>>>(np, h->sa_p1, h->sa_p1x);
  }
  for (const StLevelT<double>& d : h->st) {
    StLevelT<dfloat> f{};
    f.X = d.X; f.Y = d.Y; f.Z = d.Z; f.no = d.no;
    set_agg(f, d.ag[0], d.ag[1], d.ag[2]);
    hd_status st = alloc_st<dfloat>(h, f, true);
    h->stx.push_back(f);
    if (st != HD_OK) return st;
    k_to_f32_sa<dfloat><<<nblk(d.n() * n_half(d.no)), TPB, 0, h->stream>>>(d.n() * n_half(d.no), d.a, f.a);
    k_to_f32_sa<dfloat><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.dinv, f.dinv);
  }
  HD_LAUNCH_CK(h, "SA df");
  return HD_OK;
}

hd_status sa_vcycle_f32(hd_op* h, const float* b, float* x) {
  return run_graphed(h, b, x, 3, [&]() { sa_cycle0<float>(h, h->lvf[0], h->sa_pf, h->stf, h->sa_p1f, b, x); });
}
