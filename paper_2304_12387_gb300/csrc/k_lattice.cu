// Lattice kernels: the divergence D and D^T as stencils on the subcell lattice
// (Sec. 2.1: D is the lowest-order divergence of the refined mesh), the
// approximate Schur complement S~ = C~ + D M~^-1 D^T as a 7-point M-matrix
// stencil (Eq. approx-schur-entries), its Galerkin coarse levels and the
// l1-Jacobi V-cycle that stands in for the paper's AMG V-cycle (Sec. 3.2).
#include <cmath>
#include <cstring>
#include <vector>

#include "hd_internal.h"
#include "k_level7.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

__device__ __forceinline__ bool face_is_ess(const LatticeDims& L, int64_t g) {
  if (g < L.n_xf) {
    int I = (int)(g % (L.X + 1));
    return (I == 0 && (L.ess & 1)) || (I == L.X && (L.ess & 2));
  } else if (g < (int64_t)L.n_xf + L.n_yf) {
    int64_t r = g - L.n_xf;
    int J = (int)((r / L.X) % (L.Y + 1));
    return (J == 0 && (L.ess & 4)) || (J == L.Y && (L.ess & 8));
  } else {
    int64_t r = g - L.n_xf - L.n_yf;
    int Z = (int)(r / ((int64_t)L.X * L.Y));
    return (Z == 0 && (L.ess & 16)) || (Z == L.Z && (L.ess & 32));
  }
}

// (D u)_cell = sum over the 6 faces of (+u_high - u_low), essential faces dropped
__global__ void k_div(const LatticeDims L, const double* __restrict__ u, double* __restrict__ yq) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)L.X * L.Y * L.Z;
  if (c >= n) return;
  int I, J, Z;
  lat_coords(c, L.X, L.Y, I, J, Z);
  int64_t xl = I + (int64_t)(L.X + 1) * (J + (int64_t)L.Y * Z);
  int64_t yl = L.n_xf + I + (int64_t)L.X * (J + (int64_t)(L.Y + 1) * Z);
  int64_t yh = yl + L.X;
  int64_t zl = (int64_t)L.n_xf + L.n_yf + I + (int64_t)L.X * (J + (int64_t)L.Y * Z);
  int64_t zh = zl + (int64_t)L.X * L.Y;
  double uxl = (I == 0 && (L.ess & 1)) ? 0.0 : u[xl];
  double uxh = (I == L.X - 1 && (L.ess & 2)) ? 0.0 : u[xl + 1];
  double uyl = (J == 0 && (L.ess & 4)) ? 0.0 : u[yl];
  double uyh = (J == L.Y - 1 && (L.ess & 8)) ? 0.0 : u[yh];
  double uzl = (Z == 0 && (L.ess & 16)) ? 0.0 : u[zl];
  double uzh = (Z == L.Z - 1 && (L.ess & 32)) ? 0.0 : u[zh];
  yq[c] = (uxh - uxl) + (uyh - uyl) + (uzh - uzl);
}

// (D^T q)_face = q_low - q_high (a missing cell contributes 0); 0 on essential faces
template <typename T>
__global__ void k_divT(const LatticeDims L, const T* __restrict__ q, T* __restrict__ yu) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)L.n_xf + L.n_yf + (int64_t)L.X * L.Y * (L.Z + 1);
  if (g >= n) return;
  T v = (T)0;
  if (!face_is_ess(L, g)) {
    if (g < L.n_xf) {
      int I = (int)(g % (L.X + 1));
      int64_t r = g / (L.X + 1);  // J + Y Z
      if (I > 0) v += q[(I - 1) + (int64_t)L.X * r];
      if (I < L.X) v -= q[I + (int64_t)L.X * r];
    } else if (g < (int64_t)L.n_xf + L.n_yf) {
      int64_t r = g - L.n_xf;
      int I = (int)(r % L.X);
      int J = (int)((r / L.X) % (L.Y + 1));
      int64_t Z = r / ((int64_t)L.X * (L.Y + 1));
      if (J > 0) v += q[I + (int64_t)L.X * ((J - 1) + (int64_t)L.Y * Z)];
      if (J < L.Y) v -= q[I + (int64_t)L.X * (J + (int64_t)L.Y * Z)];
    } else {
      int64_t r = g - L.n_xf - L.n_yf;
      int64_t XY = (int64_t)L.X * L.Y;
      int64_t Z = r / XY, c = r % XY;
      if (Z > 0) v += q[c + XY * (Z - 1)];
      if (Z < L.Z) v -= q[c + XY * Z];
    }
  }
  yu[g] = v;
}

// M~ = diag(M) -> 1 on essential faces; 1/(tau M~) (1 on essential faces);
// level-0 face weights m_f = 1/M~_f (0 on essential faces).
__global__ void k_prec_faces(const LatticeDims L, int64_t n_rt, double tau, double* __restrict__ mt,
                             double* __restrict__ mtinv, double* __restrict__ w) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_rt) return;
  if (face_is_ess(L, g)) {
    mt[g] = 1.0;
    mtinv[g] = 1.0;
    w[g] = 0.0;
  } else {
    double m = mt[g];
    mtinv[g] = 1.0 / (tau * m);
    w[g] = 1.0 / m;
  }
}

// C~ per cell: 1/(alpha_e diag W_e) (grad-div) or gamma_e / diag W_e (Darcy)
__global__ void k_ctilde(const LatticeDims L, int k, int64_t n_elem, const double* __restrict__ wdiag,
                         const double* __restrict__ cscale, double* __restrict__ ct) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int nl2 = k * k * k;
  if (t >= n_elem * nl2) return;
  int64_t e = t / nl2;
  int a = (int)(t % nl2);
  int ex = (int)(e % L.nx), ey = (int)((e / L.nx) % L.ny), ez = (int)(e / ((int64_t)L.nx * L.ny));
  int i = a % k, j = (a / k) % k, l = a / (k * k);
  int64_t c = (ex * k + i) + (int64_t)L.X * ((ey * k + j) + (int64_t)L.Y * (ez * k + l));
  ct[c] = cscale[e] / wdiag[t];
}

template <typename T>
__global__ void k_level_diag(LevelT<T> lv) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  int64_t xl = I + (int64_t)(lv.X + 1) * (J + (int64_t)lv.Y * Z);
  int64_t yl = I + (int64_t)lv.X * (J + (int64_t)(lv.Y + 1) * Z);
  int64_t zl = I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z);
  T wxl = lv.wx[xl], wxh = lv.wx[xl + 1];
  T wyl = lv.wy[yl], wyh = lv.wy[yl + lv.X];
  T wzl = lv.wz[zl], wzh = lv.wz[zl + (int64_t)lv.X * lv.Y];
  T d = lv.mass[c] + ((wxl + wxh) + (wyl + wyh) + (wzl + wzh));
  T off = (I > 0 ? wxl : (T)0) + (I < lv.X - 1 ? wxh : (T)0) + (J > 0 ? wyl : (T)0) +
          (J < lv.Y - 1 ? wyh : (T)0) + (Z > 0 ? wzl : (T)0) + (Z < lv.Z - 1 ? wzh : (T)0);
  lv.diag[c] = d;
  lv.dinv[c] = (T)1 / (d + off);
}

// Galerkin coarse level for piecewise-constant aggregation: coarse face weight =
// sum of the fine face weights on it, coarse mass = sum of the children's mass.
__global__ void k_coarsen_x(LevelT<double> f, LevelT<double> c) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)(c.X + 1) * c.Y * c.Z;
  if (t >= n) return;
  int Ic = (int)(t % (c.X + 1)), Jc = (int)((t / (c.X + 1)) % c.Y), Zc = (int)(t / ((int64_t)(c.X + 1) * c.Y));
  int I = min(agg_lo(c.ag[0], Ic), f.X);
  double s = 0.0;
  for (int Z = agg_lo(c.ag[2], Zc); Z < agg_hi(c.ag[2], Zc, f.Z); ++Z)
    for (int J = agg_lo(c.ag[1], Jc); J < agg_hi(c.ag[1], Jc, f.Y); ++J)
      s += f.wx[I + (int64_t)(f.X + 1) * (J + (int64_t)f.Y * Z)];
  c.wx[t] = s;
}
__global__ void k_coarsen_y(LevelT<double> f, LevelT<double> c) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)c.X * (c.Y + 1) * c.Z;
  if (t >= n) return;
  int Ic = (int)(t % c.X), Jc = (int)((t / c.X) % (c.Y + 1)), Zc = (int)(t / ((int64_t)c.X * (c.Y + 1)));
  int J = min(agg_lo(c.ag[1], Jc), f.Y);
  double s = 0.0;
  for (int Z = agg_lo(c.ag[2], Zc); Z < agg_hi(c.ag[2], Zc, f.Z); ++Z)
    for (int I = agg_lo(c.ag[0], Ic); I < agg_hi(c.ag[0], Ic, f.X); ++I)
      s += f.wy[I + (int64_t)f.X * (J + (int64_t)(f.Y + 1) * Z)];
  c.wy[t] = s;
}
__global__ void k_coarsen_z(LevelT<double> f, LevelT<double> c) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = (int64_t)c.X * c.Y * (c.Z + 1);
  if (t >= n) return;
  int Ic, Jc, Zc;
  lat_coords(t, c.X, c.Y, Ic, Jc, Zc);
  int Z = min(agg_lo(c.ag[2], Zc), f.Z);
  double s = 0.0;
  for (int J = agg_lo(c.ag[1], Jc); J < agg_hi(c.ag[1], Jc, f.Y); ++J)
    for (int I = agg_lo(c.ag[0], Ic); I < agg_hi(c.ag[0], Ic, f.X); ++I)
      s += f.wz[I + (int64_t)f.X * (J + (int64_t)f.Y * Z)];
  c.wz[t] = s;
}
__global__ void k_coarsen_mass(LevelT<double> f, LevelT<double> c) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= c.n()) return;
  int Ic, Jc, Zc;
  lat_coords(t, c.X, c.Y, Ic, Jc, Zc);
  double s = 0.0;
  for (int Z = agg_lo(c.ag[2], Zc); Z < agg_hi(c.ag[2], Zc, f.Z); ++Z)
    for (int J = agg_lo(c.ag[1], Jc); J < agg_hi(c.ag[1], Jc, f.Y); ++J)
      for (int I = agg_lo(c.ag[0], Ic); I < agg_hi(c.ag[0], Ic, f.X); ++I)
        s += f.mass[I + (int64_t)f.X * (J + (int64_t)f.Y * Z)];
  c.mass[t] = s;
}

// same with x replaced by x + P xc (coarse value of each cell's aggregate added)
template <typename T>
__device__ __forceinline__ T stencil_res_prolong(const LevelT<T>& lv, const LevelT<T>& cl, const T* __restrict__ x,
                                                 const T* __restrict__ xcrs, T bc, T xself, int I, int J, int Z,
                                                 int64_t c) {
  auto xv = [&](int i, int j, int z) -> T {
    int64_t cc = i + (int64_t)lv.X * (j + (int64_t)lv.Y * z);
    return x[cc] + xcrs[agg_of(cl.ag[0], i) + (int64_t)cl.X * (agg_of(cl.ag[1], j) + (int64_t)cl.Y * agg_of(cl.ag[2], z))];
  };
  int64_t xl = I + (int64_t)(lv.X + 1) * (J + (int64_t)lv.Y * Z);
  int64_t yl = I + (int64_t)lv.X * (J + (int64_t)(lv.Y + 1) * Z);
  int64_t zl = I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z);
  int64_t XY = (int64_t)lv.X * lv.Y;
  T r = fma(-lv.diag[c], xself, bc);
  const T o = rowsum_form<T>() ? xself : (T)0;  // FP32 levels: differences (see rowsum_form)
  if (I > 0) r = fma(lv.wx[xl], rs_diff(xv(I - 1, J, Z), o), r);
  if (I < lv.X - 1) r = fma(lv.wx[xl + 1], rs_diff(xv(I + 1, J, Z), o), r);
  if (J > 0) r = fma(lv.wy[yl], rs_diff(xv(I, J - 1, Z), o), r);
  if (J < lv.Y - 1) r = fma(lv.wy[yl + lv.X], rs_diff(xv(I, J + 1, Z), o), r);
  if (Z > 0) r = fma(lv.wz[zl], rs_diff(xv(I, J, Z - 1), o), r);
  if (Z < lv.Z - 1) r = fma(lv.wz[zl + XY], rs_diff(xv(I, J, Z + 1), o), r);
  return r;
}

template <typename T>
__global__ void k_schur_apply(LevelT<T> lv, const T* __restrict__ x, T* __restrict__ y) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  y[c] = -stencil_res<T>(lv, x, (T)0, x[c], I, J, Z, c);
}

template <typename T>
__global__ void k_vc_jacobi_prolong(LevelT<T> lv, LevelT<T> cl, const T* __restrict__ b, const T* __restrict__ x,
                                    const T* __restrict__ xcrs, T* __restrict__ xo) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  T xs = x[c] + xcrs[agg_of(cl.ag[0], I) + (int64_t)cl.X * (agg_of(cl.ag[1], J) + (int64_t)cl.Y * agg_of(cl.ag[2], Z))];
  xo[c] = fma(lv.dinv[c], stencil_res_prolong<T>(lv, cl, x, xcrs, b[c], xs, I, J, Z, c), xs);
}

// x += P x_c (piecewise-constant prolongation, in place)
template <typename T>
__global__ void k_vc_prolong_add(LevelT<T> lv, LevelT<T> cl, const T* __restrict__ xcrs, T* __restrict__ x) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  x[c] += xcrs[agg_of(cl.ag[0], I) + (int64_t)cl.X * (agg_of(cl.ag[1], J) + (int64_t)cl.Y * agg_of(cl.ag[2], Z))];
}

// coarse right-hand side: sum over each aggregate of the fine residual b - S x
template <typename T>
__global__ void k_vc_restrict(LevelT<T> lv, LevelT<T> cl, const T* __restrict__ b, const T* __restrict__ x,
                              T* __restrict__ bc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cl.n()) return;
  int Ic, Jc, Zc;
  lat_coords(t, cl.X, cl.Y, Ic, Jc, Zc);
  T s = (T)0;
  for (int Z = agg_lo(cl.ag[2], Zc); Z < agg_hi(cl.ag[2], Zc, lv.Z); ++Z)
    for (int J = agg_lo(cl.ag[1], Jc); J < agg_hi(cl.ag[1], Jc, lv.Y); ++J)
      for (int I = agg_lo(cl.ag[0], Ic); I < agg_hi(cl.ag[0], Ic, lv.X); ++I) {
        int64_t c = I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z);
        s += stencil_res<T>(lv, x, b[c], x[c], I, J, Z, c);
      }
  bc[t] = s;
}

// z -= mean(z): deterministic two-pass reduction (fixed per-block chunks, fixed-order final pass)
constexpr int MEAN_BLOCKS = 512;
template <typename T>
__global__ void k_sum_partial(int64_t n, const T* __restrict__ z, double* __restrict__ part) {
  __shared__ double red[256];
  int64_t chunk = (n + MEAN_BLOCKS - 1) / MEAN_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += (double)z[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_mean_final(int64_t n, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[MEAN_BLOCKS];
  red[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (double)n;
}
template <typename T>
void launch_mean(hd_op* h, int64_t n, const T* z, double* part_and_out) {
  k_sum_partial<T><<<MEAN_BLOCKS, 256, 0, h->stream>>>(n, z, part_and_out + 1);
  k_mean_final<<<1, MEAN_BLOCKS, 0, h->stream>>>(n, part_and_out + 1, part_and_out);
}
template <typename T>
__global__ void k_sub_mean(int64_t n, T* __restrict__ z, const double* __restrict__ mean) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = (T)((double)z[i] - mean[0]);
}

// z_u = r_u * mtinv
template <typename T>
__global__ void k_diag_scale(int64_t n, const T* __restrict__ mtinv, const T* __restrict__ r, T* __restrict__ z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  z[i] = r[i] * mtinv[i];
}

template <typename T>
__global__ void k_to_f32(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = (T)a[i];
}

// -- host side -----------------------------------------------------------------

template <typename T>
const T* vcycle_level(hd_op* h, std::vector<LevelT<T>>& lv, const double* coarse_inv, int l, const T* b, T* out) {
  LevelT<T>& L = lv[l];
  const int last = (int)lv.size() - 1;
  if (l == last) {
    T* dst = out ? out : L.x0;
    k_vc_coarse<T><<<nblk(L.n() * 32), TPB, 0, h->stream>>>((int)L.n(), coarse_inv, b, dst);
    return dst;
  }
  LevelT<T>& C = lv[l + 1];
  const int nu = h->nu;
  T* cur = L.x0;
  k_vc_scale<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur);
  for (int s = 1; s < nu; ++s) {
    T* o = (cur == L.x0) ? L.x1 : L.x0;
    k_vc_jacobi<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, o);
    cur = o;
  }
  // W-cycle: a second coarse correction from the updated residual, except just
  // above the coarsest level, where the first one is already exact
  const int repeats = (h->cycle == 2 && l + 1 < last && (h->w_levels == 0 || l < h->w_levels)) ? 2 : 1;
  const T* xc = nullptr;
  for (int rep = 0; rep < repeats; ++rep) {
    if (rep > 0) k_vc_prolong_add<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, C, xc, cur);
    k_vc_restrict<T><<<nblk(C.n()), TPB, 0, h->stream>>>(L, C, b, cur, C.b);
    xc = vcycle_level<T>(h, lv, coarse_inv, l + 1, C.b, nullptr);
  }
  T* o = (nu == 1 && out) ? out : ((cur == L.x0) ? L.x1 : L.x0);
  k_vc_jacobi_prolong<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, C, b, cur, xc, o);
  cur = o;
  for (int s = 1; s < nu; ++s) {
    T* o2 = (s == nu - 1 && out) ? out : ((cur == L.x0) ? L.x1 : L.x0);
    k_vc_jacobi<T><<<nblk(L.n()), TPB, 0, h->stream>>>(L, b, cur, o2);
    cur = o2;
  }
  return cur;
}

}  // namespace

// Runs launch() (which enqueues on h->stream) as a CUDA graph captured on first
// use for this (b, x, key) and replayed on a private stream ordered after and
// before the handle's stream: a V/W-cycle at 64^3 is ~100-200 small launches,
// most of them on coarse levels where launch overhead, not the kernels, sets
// the time. Falls back to direct launches where capture is unavailable.
hd_status run_graphed(hd_op* h, const void* b, void* x, int key, const std::function<void()>& launch) {
  if (!h->graphs_off && !h->gstream) {
    if (cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->gev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->gev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_off = true;
    }
  }
  if (h->graphs_off) {
    launch();
    HD_LAUNCH_CK(h, "vcycle");
    return HD_OK;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : h->vc_graphs)
    if (g.b == b && g.x == x && g.f32 == key) exec = g.exec;
  if (!exec) {
    cudaStream_t saved = h->stream;
    h->stream = h->gstream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch();
      e = cudaStreamEndCapture(h->gstream, &graph);
    }
    h->stream = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      // capture unavailable here: launch directly from now on
      cudaGetLastError();
      h->graphs_off = true;
      launch();
      HD_LAUNCH_CK(h, "vcycle");
      return HD_OK;
    }
    if (h->vc_graphs.size() >= 8) {
      cudaGraphExecDestroy(h->vc_graphs.front().exec);
      h->vc_graphs.erase(h->vc_graphs.begin());
    }
    h->vc_graphs.push_back({b, x, key, exec});
  }
  HD_CK(h, cudaEventRecord(h->gev[0], h->stream));
  HD_CK(h, cudaStreamWaitEvent(h->gstream, h->gev[0], 0));
  HD_CK(h, cudaGraphLaunch(exec, h->gstream));
  HD_CK(h, cudaEventRecord(h->gev[1], h->gstream));
  HD_CK(h, cudaStreamWaitEvent(h->stream, h->gev[1], 0));
  return HD_OK;
}

namespace {

// One V/W-cycle of the unsmoothed hierarchy on level 0 from b into x (graphed)
template <typename T>
hd_status vcycle_graphed(hd_op* h, std::vector<LevelT<T>>& lv, const T* b, T* x, int f32) {
  return run_graphed(h, b, x, f32, [&]() { vcycle_level<T>(h, lv, h->d_coarse_inv, 0, b, x); });
}

template <typename T>
hd_status alloc_level(hd_op* h, LevelT<T>& L, bool own_w) {
  int64_t n = L.n();
  size_t bytes = sizeof(T);
  if (own_w) {
    if (cudaMalloc(&L.wx, bytes * (L.X + 1) * L.Y * L.Z) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level wx");
    if (cudaMalloc(&L.wy, bytes * L.X * (L.Y + 1) * L.Z) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level wy");
    if (cudaMalloc(&L.wz, bytes * L.X * L.Y * (L.Z + 1)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level wz");
    if (cudaMalloc(&L.mass, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level mass");
  }
  if (cudaMalloc(&L.diag, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level diag");
  if (cudaMalloc(&L.dinv, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level dinv");
  if (cudaMalloc(&L.x0, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level x0");
  if (cudaMalloc(&L.x1, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level x1");
  if (cudaMalloc(&L.b, bytes * n) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "level b");
  return HD_OK;
}

template <typename T>
void free_level(LevelT<T>& L, bool own_w) {
  if (own_w) {
    cudaFree(L.wx);
    cudaFree(L.wy);
    cudaFree(L.wz);
    cudaFree(L.mass);
  }
  cudaFree(L.diag);
  cudaFree(L.dinv);
  cudaFree(L.x0);
  cudaFree(L.x1);
  cudaFree(L.b);
}

}  // namespace

hd_status lattice_apply_B(hd_op* h, const double* u, double* yq) {
  if (h->n_l2 > 0) k_div<<<nblk(h->n_l2), TPB, 0, h->stream>>>(h->L, u, yq);
  HD_LAUNCH_CK(h, "k_div");
  return HD_OK;
}

hd_status lattice_apply_Bt(hd_op* h, const double* q, double* yu) {
  if (h->n_rt > 0) k_divT<double><<<nblk(h->n_rt), TPB, 0, h->stream>>>(h->L, q, yu);
  HD_LAUNCH_CK(h, "k_divT");
  return HD_OK;
}

hd_status lattice_apply_Bt_f32(hd_op* h, const float* q, float* yu) {
  if (h->n_rt > 0) k_divT<float><<<nblk(h->n_rt), TPB, 0, h->stream>>>(h->L, q, yu);
  HD_LAUNCH_CK(h, "k_divT f32");
  return HD_OK;
}

// Builds M~^-1, C~, the level hierarchy and the coarsest inverse. Requires
// d_mt (diag M summed over elements), d_wdiag and d_cscale from the element setup.
// Dense SPD inverse on the host for the coarsest level (n <= 4096): Cholesky
// A = R R^T, then A^-1 = R^-T R^-1 column by column; row-major output. When the
// level is singular (constants in the kernel) it inverts A + s 1 1^T with
// s = mean(diag A) / n.
hd_status dense_spd_inverse(hd_op* h, std::vector<double>& A, int n, bool singular, std::vector<double>& inv) {
  if (singular) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += A[(size_t)i * n + i];
    s = (s / n) / n;
    for (auto& a : A) a += s;
  }
  // Cholesky A = R R^T (lower R in place), then A^-1 = R^-T R^-1 column by column
  std::vector<double> R = A;
  for (int j = 0; j < n; ++j) {
    double d = R[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) d -= R[(size_t)j * n + p] * R[(size_t)j * n + p];
    if (!(d > 0.0)) return hd_fail(h, HD_ERR_PREC_INDEFINITE, "coarsest Schur level is not positive definite");
    d = std::sqrt(d);
    R[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = R[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) s -= R[(size_t)i * n + p] * R[(size_t)j * n + p];
      R[(size_t)i * n + j] = s / d;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) col[i] = (i == c) ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i) {  // forward: R y = e_c
      double s = col[i];
      for (int p = 0; p < i; ++p) s -= R[(size_t)i * n + p] * col[p];
      col[i] = s / R[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // backward: R^T x = y
      double s = col[i];
      for (int p = i + 1; p < n; ++p) s -= R[(size_t)p * n + i] * col[p];
      col[i] = s / R[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + c] = col[i];  // row-major: row i holds (A^-1)_{i,:}
  }
  return HD_OK;
}

// Aggregation of an axis of n fine cells (ne elements along it); sets the coarse length.
// Element-aligned groups (`aligned`) where the axis holds an odd number c > 1 of cells
// per element (even c: the pairs are already aligned with the element boundaries).
static Agg1 make_agg(int n, int ne, bool aligned, int& nc) {
  Agg1 a{};
  const int c = (ne > 0 && n % ne == 0) ? n / ne : 0;
  if (n == 1) {
    a.c = 1; a.m = 1;
  } else if (aligned && c > 1 && (c & 1) && c <= 7) {
    // pairs alternately from the low and the high end, the middle cell alone
    int sizes_lo[4], sizes_hi[4], nlo = 0, nhi = 0, lo = 0, hi = c;
    bool low = true;
    while (hi - lo >= 2) {
      if (low) { sizes_lo[nlo++] = 2; lo += 2; } else { sizes_hi[nhi++] = 2; hi -= 2; }
      low = !low;
    }
    int sizes[8], m = 0;
    for (int i = 0; i < nlo; ++i) sizes[m++] = sizes_lo[i];
    if (hi - lo == 1) sizes[m++] = 1;
    for (int i = nhi - 1; i >= 0; --i) sizes[m++] = sizes_hi[i];
    a.c = c; a.m = m;
    int r = 0;
    for (int j = 0; j < m; ++j) {
      a.s[j] = (int8_t)r;
      for (int t = 0; t < sizes[j]; ++t) a.g[r++] = (int8_t)j;
    }
    a.s[m] = (int8_t)c;
  } else {
    a.c = 2; a.m = 1;
  }
  nc = a.m == 1 ? (n + a.c - 1) / a.c : (n / a.c) * a.m;
  return a;
}

hd_status precond_setup(hd_op* h) {
  const LatticeDims& L = h->L;
  // level 0 lives on the fine lattice: its face weights are an RT-sized vector
  LevelT<double> l0{};
  l0.X = L.X; l0.Y = L.Y; l0.Z = L.Z;
  {
    Agg1 one{};
    one.c = 1; one.m = 1;
    set_agg(l0, one, one, one);
  }
  double* w0 = nullptr;
  if (cudaMalloc(&w0, sizeof(double) * h->n_rt) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "face weights");
  l0.wx = w0;
  l0.wy = w0 + L.n_xf;
  l0.wz = w0 + L.n_xf + L.n_yf;
  l0.mass = h->d_ct;
  hd_status st = alloc_level<double>(h, l0, false);
  h->lv.push_back(l0);
  if (st != HD_OK) return st;
  k_prec_faces<<<nblk(h->n_rt), TPB, 0, h->stream>>>(L, h->n_rt, h->tau, h->d_mt, h->d_mtinv, w0);
  HD_LAUNCH_CK(h, "k_prec_faces");
  int nl2 = h->k * h->k * h->k;
  k_ctilde<<<nblk(h->n_elem * nl2), TPB, 0, h->stream>>>(L, h->k, h->n_elem, h->d_wdiag, h->d_cscale, h->d_ct);
  HD_LAUNCH_CK(h, "k_ctilde");
  k_level_diag<double><<<nblk(l0.n()), TPB, 0, h->stream>>>(h->lv[0]);
  HD_LAUNCH_CK(h, "k_level_diag");
  // coarse levels
  while (h->lv.back().n() > h->coarse_max && (int)h->lv.size() < 24) {
    const LevelT<double>& f = h->lv.back();
    LevelT<double> c{};
    const bool al = h->agg_aligned != 0;
    set_agg(c, make_agg(f.X, L.nx, al, c.X), make_agg(f.Y, L.ny, al, c.Y), make_agg(f.Z, L.nz, al, c.Z));
    if (c.X == f.X && c.Y == f.Y && c.Z == f.Z) break;
    st = alloc_level<double>(h, c, true);
    h->lv.push_back(c);
    if (st != HD_OK) return st;
    const LevelT<double>& ff = h->lv[h->lv.size() - 2];
    const LevelT<double>& cc = h->lv.back();
    k_coarsen_x<<<nblk((int64_t)(cc.X + 1) * cc.Y * cc.Z), TPB, 0, h->stream>>>(ff, cc);
    k_coarsen_y<<<nblk((int64_t)cc.X * (cc.Y + 1) * cc.Z), TPB, 0, h->stream>>>(ff, cc);
    k_coarsen_z<<<nblk((int64_t)cc.X * cc.Y * (cc.Z + 1)), TPB, 0, h->stream>>>(ff, cc);
    k_coarsen_mass<<<nblk(cc.n()), TPB, 0, h->stream>>>(ff, cc);
    k_level_diag<double><<<nblk(cc.n()), TPB, 0, h->stream>>>(cc);
    HD_LAUNCH_CK(h, "coarsen");
  }
  // coarsest: dense matrix on the host, Cholesky, explicit inverse
  const LevelT<double>& cl = h->lv.back();
  int n = (int)cl.n();
  std::vector<double> wx((size_t)(cl.X + 1) * cl.Y * cl.Z), wy((size_t)cl.X * (cl.Y + 1) * cl.Z),
      wz((size_t)cl.X * cl.Y * (cl.Z + 1)), diag(n);
  HD_CK(h, cudaMemcpyAsync(wx.data(), cl.wx, wx.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaMemcpyAsync(wy.data(), cl.wy, wy.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaMemcpyAsync(wz.data(), cl.wz, wz.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaMemcpyAsync(diag.data(), cl.diag, diag.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  std::vector<double> A((size_t)n * n, 0.0);
  auto id = [&](int I, int J, int Z) { return I + cl.X * (J + cl.Y * Z); };
  for (int Z = 0; Z < cl.Z; ++Z)
    for (int J = 0; J < cl.Y; ++J)
      for (int I = 0; I < cl.X; ++I) {
        int c = id(I, J, Z);
        A[(size_t)c * n + c] = diag[c];
        if (I + 1 < cl.X) {
          double w = wx[(I + 1) + (size_t)(cl.X + 1) * (J + (size_t)cl.Y * Z)];
          A[(size_t)c * n + id(I + 1, J, Z)] -= w;
          A[(size_t)id(I + 1, J, Z) * n + c] -= w;
        }
        if (J + 1 < cl.Y) {
          double w = wy[I + (size_t)cl.X * ((J + 1) + (size_t)(cl.Y + 1) * Z)];
          A[(size_t)c * n + id(I, J + 1, Z)] -= w;
          A[(size_t)id(I, J + 1, Z) * n + c] -= w;
        }
        if (Z + 1 < cl.Z) {
          double w = wz[I + (size_t)cl.X * (J + (size_t)cl.Y * (Z + 1))];
          A[(size_t)c * n + id(I, J, Z + 1)] -= w;
          A[(size_t)id(I, J, Z + 1) * n + c] -= w;
        }
      }
  std::vector<double> inv;
  if ((st = dense_spd_inverse(h, A, n, h->singular, inv)) != HD_OK) return st;
  h->coarse_n = n;
  if (cudaMalloc(&h->d_coarse_inv, sizeof(double) * inv.size()) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "coarse inverse");
  HD_CK(h, cudaMemcpyAsync(h->d_coarse_inv, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  return HD_OK;
}

// FP32 copies of the preconditioner and element data for the inner mixed-precision solve
hd_status setup_f32(hd_op* h) {
  if (h->have_f32) return HD_OK;
  auto conv = [&](const double* src, float** dst, int64_t n, const char* what) -> hd_status {
    if (cudaMalloc(dst, sizeof(float) * (n > 0 ? n : 1)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, what);
    if (n > 0) k_to_f32<float><<<nblk(n), TPB, 0, h->stream>>>(n, src, *dst);
    HD_LAUNCH_CK(h, what);
    return HD_OK;
  };
  int nq = h->q * h->q * h->q, nl2 = h->k * h->k * h->k;
  hd_status st;
  if ((st = conv(h->d_G, &h->f_G, h->n_elem * 6 * nq, "f32 G")) != HD_OK) return st;
  // W^-1 for the FP32 operator: the dense inverse in FP32 when there is one, else
  // the local CG (geometric weights and Jacobi diagonal)
  if (h->d_winv && (st = conv(h->d_winv, &h->f_winv, h->n_elem * nl2 * nl2, "f32 winv")) != HD_OK) return st;
  if ((st = conv(h->d_wdet, &h->f_wdet, h->n_elem * nq, "f32 wdet")) != HD_OK) return st;
  if ((st = conv(h->d_wgldiag, &h->f_wgldiag, h->n_elem * nl2, "f32 wgl diag")) != HD_OK) return st;
  if ((st = conv(h->d_cscale, &h->f_cscale, h->n_elem, "f32 cscale")) != HD_OK) return st;
  if ((st = conv(h->d_mtinv, &h->f_mtinv, h->n_rt, "f32 mtinv")) != HD_OK) return st;
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const LevelT<double>& d = h->lv[l];
    LevelT<float> f{};
    f.X = d.X; f.Y = d.Y; f.Z = d.Z;
    set_agg(f, d.ag[0], d.ag[1], d.ag[2]);
    if ((st = alloc_level<float>(h, f, true)) != HD_OK) return st;
    h->lvf.push_back(f);
    k_to_f32<float><<<nblk((int64_t)(d.X + 1) * d.Y * d.Z), TPB, 0, h->stream>>>((int64_t)(d.X + 1) * d.Y * d.Z, d.wx, f.wx);
    k_to_f32<float><<<nblk((int64_t)d.X * (d.Y + 1) * d.Z), TPB, 0, h->stream>>>((int64_t)d.X * (d.Y + 1) * d.Z, d.wy, f.wy);
    k_to_f32<float><<<nblk((int64_t)d.X * d.Y * (d.Z + 1)), TPB, 0, h->stream>>>((int64_t)d.X * d.Y * (d.Z + 1), d.wz, f.wz);
    k_to_f32<float><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.mass, f.mass);
    k_level_rowsum<<<nblk(d.n()), TPB, 0, h->stream>>>(d, f.diag);  // row sums (rowsum_form)
    k_to_f32<float><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.dinv, f.dinv);
    HD_LAUNCH_CK(h, "f32 level");
  }
  if ((st = sa_setup_f32(h)) != HD_OK) return st;
  h->have_f32 = true;
  return HD_OK;
}

void precond_free(hd_op* h) {
  sa_free(h);
  for (auto& g : h->vc_graphs) cudaGraphExecDestroy(g.exec);
  h->vc_graphs.clear();
  if (h->gev[0]) cudaEventDestroy(h->gev[0]);
  if (h->gev[1]) cudaEventDestroy(h->gev[1]);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  for (size_t l = 0; l < h->lv.size(); ++l) {
    if (l == 0) cudaFree(h->lv[0].wx);
    free_level<double>(h->lv[l], l > 0);
  }
  h->lv.clear();
  for (auto& f : h->lvf) free_level<float>(f, true);
  h->lvf.clear();
  for (auto& f : h->lvx) free_level<dfloat>(f, true);
  h->lvx.clear();
  cudaFree(h->cyc_b);
  cudaFree(h->cyc_x);
  h->cyc_b = h->cyc_x = nullptr;
}

// double-float copies of the unsmoothed levels (the smoothed ones: sa_setup_df), made on
// first use by the FP64 cycle of fp64_emulation = 2
hd_status setup_df_cycle(hd_op* h) {
  if (!h->lvx.empty()) return HD_OK;
  hd_status st;
  for (size_t l = 0; l < h->lv.size(); ++l) {
    const LevelT<double>& d = h->lv[l];
    LevelT<dfloat> f{};
    f.X = d.X; f.Y = d.Y; f.Z = d.Z;
    set_agg(f, d.ag[0], d.ag[1], d.ag[2]);
    if ((st = alloc_level<dfloat>(h, f, true)) != HD_OK) return st;
    h->lvx.push_back(f);
    const int64_t nxw = (int64_t)(d.X + 1) * d.Y * d.Z, nyw = (int64_t)d.X * (d.Y + 1) * d.Z,
                  nzw = (int64_t)d.X * d.Y * (d.Z + 1);
    k_to_f32<dfloat><<<nblk(nxw), TPB, 0, h->stream>>>(nxw, d.wx, f.wx);
    k_to_f32<dfloat><<<nblk(nyw), TPB, 0, h->stream>>>(nyw, d.wy, f.wy);
    k_to_f32<dfloat><<<nblk(nzw), TPB, 0, h->stream>>>(nzw, d.wz, f.wz);
    k_to_f32<dfloat><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.mass, f.mass);
    k_to_f32<dfloat><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.diag, f.diag);
    k_to_f32<dfloat><<<nblk(d.n()), TPB, 0, h->stream>>>(d.n(), d.dinv, f.dinv);
    HD_LAUNCH_CK(h, "double-float level");
  }
  if (cudaMalloc(&h->cyc_b, sizeof(dfloat) * (h->n_l2 > 0 ? h->n_l2 : 1)) != cudaSuccess ||
      cudaMalloc(&h->cyc_x, sizeof(dfloat) * (h->n_l2 > 0 ? h->n_l2 : 1)) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "double-float cycle vectors");
  if (!h->st.empty() && (st = sa_setup_df(h)) != HD_OK) return st;
  return HD_OK;
}

__global__ void k_from_df(int64_t n, const dfloat* __restrict__ a, double* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

hd_status schur_apply(hd_op* h, const double* x, double* y) {
  const LevelT<double>& L = h->lv[0];
  if (L.n() > 0) k_schur_apply<double><<<nblk(L.n()), TPB, 0, h->stream>>>(L, x, y);
  HD_LAUNCH_CK(h, "k_schur_apply");
  return HD_OK;
}

hd_status vcycle_apply(hd_op* h, const double* b, double* x) {
  if (h->n_l2 == 0) return HD_OK;
  if (h->cycle_df) {  // the cycle in double-float between FP64 vectors
    hd_status st = setup_df_cycle(h);
    if (st != HD_OK) return st;
    const int64_t n = h->n_l2;
    k_to_f32<dfloat><<<nblk(n), TPB, 0, h->stream>>>(n, b, h->cyc_b);
    st = !h->st.empty() ? sa_vcycle_df(h, h->cyc_b, h->cyc_x) : vcycle_graphed<dfloat>(h, h->lvx, h->cyc_b, h->cyc_x, 5);
    if (st != HD_OK) return st;
    k_from_df<<<nblk(n), TPB, 0, h->stream>>>(n, h->cyc_x, x);
    HD_LAUNCH_CK(h, "double-float cycle");
    return HD_OK;
  }
  if (!h->st.empty()) return sa_vcycle(h, b, x);
  return vcycle_graphed<double>(h, h->lv, b, x, 0);
}

static hd_status vcycle_any(hd_op* h, const double* b, double* x) { return vcycle_apply(h, b, x); }
static hd_status vcycle_any(hd_op* h, const float* b, float* x) { return vcycle_apply_f32(h, b, x); }

template <typename T>
static hd_status precond_apply_t(hd_op* h, const T* r, T* z, const T* mtinv, std::vector<LevelT<T>>& lv,
                                 const double* cinv) {
  if (h->n_rt > 0) k_diag_scale<T><<<nblk(h->n_rt), TPB, 0, h->stream>>>(h->n_rt, mtinv, r, z);
  if (h->n_l2 > 0) {
    hd_status sv = vcycle_any(h, r + h->n_rt, z + h->n_rt);
    if (sv != HD_OK) return sv;
    if (h->singular) {
      launch_mean<T>(h, h->n_l2, z + h->n_rt, h->d_red);
      k_sub_mean<T><<<nblk(h->n_l2), TPB, 0, h->stream>>>(h->n_l2, z + h->n_rt, h->d_red);
    }
  }
  HD_LAUNCH_CK(h, "precond");
  return HD_OK;
}

hd_status precond_apply(hd_op* h, const double* r, double* z) {
  if (h->schur_mode == 1) {
    hd_status st = diag_scale(h, r, z);
    if (st != HD_OK) return st;
    if (h->n_l2 > 0) {
      if ((st = learned_schur_apply(h, r + h->n_rt, z + h->n_rt)) != HD_OK) return st;
      if (h->singular && (st = project_mean(h, z + h->n_rt)) != HD_OK) return st;
    }
    return HD_OK;
  }
  return precond_apply_t<double>(h, r, z, h->d_mtinv, h->lv, h->d_coarse_inv);
}

hd_status precond_apply_f32(hd_op* h, const float* r, float* z) {
  hd_status st = setup_f32(h);
  if (st != HD_OK) return st;
  return precond_apply_t<float>(h, r, z, h->f_mtinv, h->lvf, h->d_coarse_inv);
}

// plain aggregation sum b_c = P^T r and injection z += P x_c between levels 0 and 1
__global__ void k_restrict_plain(LevelT<double> lv, LevelT<double> cl, const double* __restrict__ r,
                                 double* __restrict__ bc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cl.n()) return;
  int Ic, Jc, Zc;
  lat_coords(t, cl.X, cl.Y, Ic, Jc, Zc);
  double s = 0.0;
  for (int Z = agg_lo(cl.ag[2], Zc); Z < agg_hi(cl.ag[2], Zc, lv.Z); ++Z)
    for (int J = agg_lo(cl.ag[1], Jc); J < agg_hi(cl.ag[1], Jc, lv.Y); ++J)
      for (int I = agg_lo(cl.ag[0], Ic); I < agg_hi(cl.ag[0], Ic, lv.X); ++I) s += r[I + (int64_t)lv.X * (J + (int64_t)lv.Y * Z)];
  bc[t] = s;
}
__global__ void k_prolong_add(LevelT<double> lv, LevelT<double> cl, const double* __restrict__ xc,
                              double* __restrict__ z) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n()) return;
  int I, J, Z;
  lat_coords(c, lv.X, lv.Y, I, J, Z);
  z[c] += xc[agg_of(cl.ag[0], I) + (int64_t)cl.X * (agg_of(cl.ag[1], J) + (int64_t)cl.Y * agg_of(cl.ag[2], Z))];
}

hd_status coarse_correction(hd_op* h, const double* r, double* z) {
  if (h->lv.size() < 2) return HD_OK;
  LevelT<double>& f = h->lv[0];
  LevelT<double>& c = h->lv[1];
  k_restrict_plain<<<nblk(c.n()), TPB, 0, h->stream>>>(f, c, r, c.b);
  const double* xc = vcycle_level<double>(h, h->lv, h->d_coarse_inv, 1, c.b, nullptr);
  k_prolong_add<<<nblk(f.n()), TPB, 0, h->stream>>>(f, c, xc, z);
  HD_LAUNCH_CK(h, "coarse correction");
  return HD_OK;
}

// FP32 V-cycle on an L2 vector (coarsest level in FP64)
hd_status vcycle_apply_f32(hd_op* h, const float* b, float* x) {
  if (h->n_l2 == 0) return HD_OK;
  hd_status st = setup_f32(h);
  if (st != HD_OK) return st;
  if (!h->stf.empty()) return sa_vcycle_f32(h, b, x);
  return vcycle_graphed<float>(h, h->lvf, b, x, 1);
}

// z_u = r_u / (tau M~) on the RT part (identity on essential dofs)
hd_status diag_scale(hd_op* h, const double* r, double* z) {
  if (h->n_rt > 0) k_diag_scale<double><<<nblk(h->n_rt), TPB, 0, h->stream>>>(h->n_rt, h->d_mtinv, r, z);
  HD_LAUNCH_CK(h, "diag_scale");
  return HD_OK;
}

// z -= mean(z) on an L2 vector (pure-Neumann Darcy: the Schur complement's
// kernel is the constants; Sec. 4.2 orthogonalises after every V-cycle).
hd_status project_mean(hd_op* h, double* z) {
  launch_mean<double>(h, h->n_l2, z, h->d_red);
  k_sub_mean<double><<<nblk(h->n_l2), TPB, 0, h->stream>>>(h->n_l2, z, h->d_red);
  HD_LAUNCH_CK(h, "project_mean");
  return HD_OK;
}

// FP32 copies of the two above (the FP32 vectors of the mixed-precision GMRES)
hd_status diag_scale_f32(hd_op* h, const float* r, float* z) {
  if (h->n_rt > 0) k_diag_scale<float><<<nblk(h->n_rt), TPB, 0, h->stream>>>(h->n_rt, h->f_mtinv, r, z);
  HD_LAUNCH_CK(h, "diag_scale f32");
  return HD_OK;
}
hd_status project_mean_f32(hd_op* h, float* z) {
  launch_mean<float>(h, h->n_l2, z, h->d_red);
  k_sub_mean<float><<<nblk(h->n_l2), TPB, 0, h->stream>>>(h->n_l2, z, h->d_red);
  HD_LAUNCH_CK(h, "project_mean f32");
  return HD_OK;
}
