// C ABI of the hdivsp library: handle lifetime, host-side setup (1D tables of
// the interpolation-histopolation basis, index maps) and the apply entry points.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hd_internal.h"
#include "k_element.cuh"

hd_status hd_fail(hd_op* h, hd_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

hd_status hd_cuda_check(hd_op* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return hd_fail(h, HD_ERR_OOM, m);
  return hd_fail(h, HD_ERR_CUDA, m);
}

namespace {

// ---- 1D tables (Sec. 2.1) -----------------------------------------------------
// Legendre P_n and its first two derivatives on [-1,1] by the three-term recurrence.
void legendre(int n, double x, double& p, double& dp, double& ddp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0, dd0 = 0.0, dd1 = 0.0;
  if (n == 0) { p = 1.0; dp = 0.0; ddp = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    double d2 = ((2 * m + 1) * (p1 + x * d1) - m * d0) / (m + 1);
    double dd2 = ((2 * m + 1) * (2 * d1 + x * dd1) - m * dd0) / (m + 1);
    p0 = p1; p1 = p2; d0 = d1; d1 = d2; dd0 = dd1; dd1 = dd2;
  }
  p = p1; dp = d1; ddp = dd1;
}

// Gauss-Lobatto nodes on [0,1]: 0, 1 and the roots of P_k' (Newton from
// Chebyshev-Gauss-Lobatto points).
std::vector<double> gll(int k) {
  std::vector<double> t(k + 1);
  for (int i = 0; i <= k; ++i) t[i] = -std::cos(M_PI * i / k);
  for (int i = 1; i < k; ++i) {
    double x = t[i];
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre(k, x, p, dp, ddp);
      double dx = dp / ddp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    t[i] = x;
  }
  t[0] = -1.0; t[k] = 1.0;
  for (auto& v : t) v = 0.5 * (v + 1.0);
  return t;
}

// Gauss-Legendre points/weights on [0,1] (Newton on P_q).
void gauss(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q); w.resize(q);
  for (int i = 0; i < q; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double p, dp, ddp;
    for (int it = 0; it < 100; ++it) {
      legendre(q, z, p, dp, ddp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(q, z, p, dp, ddp);
    x[i] = 0.5 * (z + 1.0);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) scaled by 1/2
  }
}

// Lagrange basis on `nodes`: value and derivative of l_i at x.
double lag(const std::vector<double>& nd, int i, double x) {
  double v = 1.0;
  for (size_t m = 0; m < nd.size(); ++m)
    if ((int)m != i) v *= (x - nd[m]) / (nd[i] - nd[m]);
  return v;
}
double dlag(const std::vector<double>& nd, int i, double x) {
  double s = 0.0;
  for (size_t m = 0; m < nd.size(); ++m) {
    if ((int)m == i) continue;
    double t = 1.0 / (nd[i] - nd[m]);
    for (size_t r = 0; r < nd.size(); ++r)
      if ((int)r != i && r != m) t *= (x - nd[r]) / (nd[i] - nd[r]);
    s += t;
  }
  return s;
}

void build_tables(int k, int q, ElemTables& t) {
  std::memset(&t, 0, sizeof(t));
  std::vector<double> xi = gll(k), gx, gw;
  gauss(q, gx, gw);
  for (int p = 0; p < q; ++p) {
    t.gx[p] = gx[p];
    t.gw[p] = gw[p];
    for (int i = 0; i <= k; ++i) t.BI[p * (k + 1) + i] = lag(xi, i, gx[p]);
    // h_j = sum_{i > j} l_i'  (integral of h_j over subcell m is delta_mj)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int i = j + 1; i <= k; ++i) s += dlag(xi, i, gx[p]);
      t.BH[p * k + j] = s;
    }
  }
  // GL nodal basis of the local CG (k Gauss-Legendre nodes): its values at the q
  // quadrature points, and TT[j][m] = integral of L_m over subcell j (Gauss rule
  // with k+2 points per subcell, exact for these degree-(k-1) polynomials)
  std::vector<double> gk, wk, gs, ws;
  gauss(k, gk, wk);
  gauss(k + 2, gs, ws);
  for (int p = 0; p < q; ++p)
    for (int m = 0; m < k; ++m) t.BG[p * k + m] = lag(gk, m, gx[p]);
  for (int j = 0; j < k; ++j)
    for (int m = 0; m < k; ++m) {
      double a = xi[j], b = xi[j + 1], s = 0.0;
      for (size_t i = 0; i < gs.size(); ++i) s += ws[i] * lag(gk, m, a + (b - a) * gs[i]);
      t.TT[j * k + m] = (b - a) * s;
    }
  // 1D histopolation mass (exact: q >= k points for degree 2k-2) and its inverse by
  // Gauss-Jordan elimination with partial pivoting
  double A[HD_MAXK][2 * HD_MAXK];
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      double s = 0.0;
      for (int p = 0; p < q; ++p) s += gw[p] * t.BH[p * k + a] * t.BH[p * k + b];
      A[a][b] = s;
      A[a][k + b] = a == b ? 1.0 : 0.0;
    }
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
    for (int j = 0; j < 2 * k; ++j) std::swap(A[c][j], A[piv][j]);
    const double d = A[c][c];
    for (int j = 0; j < 2 * k; ++j) A[c][j] /= d;
    for (int r = 0; r < k; ++r)
      if (r != c) {
        const double f = A[r][c];
        for (int j = 0; j < 2 * k; ++j) A[r][j] -= f * A[c][j];
      }
  }
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) t.HI[a * k + b] = A[a][k + b];
  // even-odd tables of BI (q x k+1), BH (q x k) and their transposes
  auto eo = [](int R, int C, auto M, double* P, double* N) {
    const int ec = (C + 1) / 2, hc = C / 2;
    for (int r = 0; r < (R + 1) / 2; ++r)
      for (int c = 0; c < ec; ++c)
        P[r * ec + c] = (2 * c + 1 == C) ? M(r, c) : 0.5 * (M(r, c) + M(r, C - 1 - c));
    for (int r = 0; r < R / 2; ++r)
      for (int c = 0; c < hc; ++c) N[r * hc + c] = 0.5 * (M(r, c) - M(r, C - 1 - c));
  };
  eo(q, k + 1, [&](int r, int c) { return t.BI[r * (k + 1) + c]; }, t.BIp, t.BIn);
  eo(q, k, [&](int r, int c) { return t.BH[r * k + c]; }, t.BHp, t.BHn);
  eo(k + 1, q, [&](int r, int c) { return t.BI[c * (k + 1) + r]; }, t.BITp, t.BITn);
  eo(k, q, [&](int r, int c) { return t.BH[c * k + r]; }, t.BHTp, t.BHTn);
}

// Affine fast path: every element a parallelepiped (its trilinear map has no bilinear or
// trilinear part, to 1e-14 of the element's edge length plus 16 ulps of its largest
// coordinate: the rounding of the vertex differences themselves). Then J is constant, the
// geometric factor at point p is w_p times one symmetric 3x3 matrix, and W_e^-1 =
// det J (H^-1 x H^-1 x H^-1): 8 values per element instead of 6 q^3 + k^6. Fills
// ga[E][8] and returns true, or returns false at the first element that is not affine.
static bool affine_factors(const hd_problem_desc* d, const double* bco, std::vector<double>& ga) {
  const int64_t nx = d->nx, ny = d->ny, nz = d->nz, E = nx * ny * nz;
  ga.assign((size_t)E * 8, 0.0);
  for (int64_t e = 0; e < E; ++e) {
    const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
    double v[8][3];
    for (int c = 0; c < 8; ++c) {
      const int64_t id = (ex + (c & 1)) + (nx + 1) * ((ey + ((c >> 1) & 1)) + (ny + 1) * (ez + (c >> 2)));
      v[c][0] = d->vx[id]; v[c][1] = d->vy[id]; v[c][2] = d->vz[id];
    }
    double J[3][3], h = 0.0, vmax = 0.0;  // J[i][a] = d x_i / d xi_a
    for (int i = 0; i < 3; ++i) {
      J[i][0] = v[1][i] - v[0][i];
      J[i][1] = v[2][i] - v[0][i];
      J[i][2] = v[4][i] - v[0][i];
      for (int a = 0; a < 3; ++a) h = std::max(h, std::fabs(J[i][a]));
      for (int c = 0; c < 8; ++c) vmax = std::max(vmax, std::fabs(v[c][i]));
    }
    const double tol = 1e-14 * h + 16.0 * 2.220446049250313e-16 * vmax;
    for (int i = 0; i < 3; ++i) {
      const double t01 = v[3][i] - v[1][i] - v[2][i] + v[0][i], t02 = v[5][i] - v[1][i] - v[4][i] + v[0][i],
                   t12 = v[6][i] - v[2][i] - v[4][i] + v[0][i],
                   t012 = v[7][i] - v[3][i] - v[5][i] - v[6][i] + v[1][i] + v[2][i] + v[4][i] - v[0][i];
      if (std::fabs(t01) > tol || std::fabs(t02) > tol || std::fabs(t12) > tol || std::fabs(t012) > tol)
        return false;
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) return false;
    auto jtj = [&](int a, int b) { return J[0][a] * J[0][b] + J[1][a] * J[1][b] + J[2][a] * J[2][b]; };
    const double f = bco[e] / det;
    double* g = ga.data() + (size_t)e * 8;
    g[0] = f * jtj(0, 0); g[1] = f * jtj(0, 1); g[2] = f * jtj(0, 2);
    g[3] = f * jtj(1, 1); g[4] = f * jtj(1, 2); g[5] = f * jtj(2, 2);
    g[6] = det;
  }
  return true;
}

hd_status dalloc(hd_op* h, double** p, int64_t n, const char* what) {
  if (cudaMalloc(p, sizeof(double) * (n > 0 ? n : 1)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, what);
  return HD_OK;
}

hd_status elem_op(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq) {
  if (h->emul) {
    switch (h->k) {
      case 2: return elem_op_df_k2(h, mode, u, q, yu, yq);
      case 3: return elem_op_df_k3(h, mode, u, q, yu, yq);
      case 4: return elem_op_df_k4(h, mode, u, q, yu, yq);
      case 5: return elem_op_df_k5(h, mode, u, q, yu, yq);
    }
  }
  switch (h->k) {
    case 2: return elem_op_k2(h, mode, u, q, yu, yq);
    case 3: return elem_op_k3(h, mode, u, q, yu, yq);
    case 4: return elem_op_k4(h, mode, u, q, yu, yq);
    case 5: return elem_op_k5(h, mode, u, q, yu, yq);
  }
  return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "k not supported");
}

hd_status elem_op_f32(hd_op* h, int mode, const float* u, const float* q, float* yu, float* yq) {
  switch (h->k) {
    case 2: return elem_op_f32_k2(h, mode, u, q, yu, yq);
    case 3: return elem_op_f32_k3(h, mode, u, q, yu, yq);
    case 4: return elem_op_f32_k4(h, mode, u, q, yu, yq);
    case 5: return elem_op_f32_k5(h, mode, u, q, yu, yq);
  }
  return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "k not supported");
}

// FP32 arithmetic, FP64 vectors (inner operator of the mixed-precision solve)
hd_status elem_op_f32io64(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq) {
  switch (h->k) {
    case 2: return elem_op_f32io64_k2(h, mode, u, q, yu, yq);
    case 3: return elem_op_f32io64_k3(h, mode, u, q, yu, yq);
    case 4: return elem_op_f32io64_k4(h, mode, u, q, yu, yq);
    case 5: return elem_op_f32io64_k5(h, mode, u, q, yu, yq);
  }
  return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "k not supported");
}

hd_status elem_setup(hd_op* h, const double* bcoef, int* d_bad) {
  switch (h->k) {
    case 2: return elem_setup_k2(h, bcoef, d_bad);
    case 3: return elem_setup_k3(h, bcoef, d_bad);
    case 4: return elem_setup_k4(h, bcoef, d_bad);
    case 5: return elem_setup_k5(h, bcoef, d_bad);
  }
  return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "k not supported");
}

// FP64 -> double-float (round-to-nearest hi, remainder lo): setup only
__global__ void k_split_df(int64_t n, const double* __restrict__ a, dfloat* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = a[i];
  float h = __double2float_rn(v);
  b[i] = dfloat(h, __double2float_rn(v - (double)h));
}

// Range guard of the double-float element data, one warp per element: the largest
// magnitude of the element's geometric factors (6 q^3), of its W_e^-1 (k^6) and of
// c_e W_e^-1 must lie in [2^-60, 2^60] (c_e = 0 allowed), so that the significant
// entries and their products with O(1) vector entries keep both halves of the FP32
// pairs normal; entries far below their element's largest (round-off-level zeros)
// flush harmlessly. flag = 1 otherwise, or on a non-finite value.
__device__ __forceinline__ bool df_scale_ok(double m) { return m >= 0x1p-60 && m <= 0x1p60; }
__global__ void k_df_range(int64_t E, int ng, int nw, const double* __restrict__ G, const double* __restrict__ winv,
                           const double* __restrict__ cs, int* __restrict__ flag) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= E) return;
  double mg = 0.0, mw = 0.0;
  bool finite = true;
  for (int i = lane; i < ng; i += 32) {
    const double v = fabs(G[e * ng + i]);
    finite = finite && isfinite(v);
    mg = fmax(mg, v);
  }
  for (int i = lane; i < nw; i += 32) {
    const double v = fabs(winv[e * nw + i]);
    finite = finite && isfinite(v);
    mw = fmax(mw, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mg = fmax(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    mw = fmax(mw, __shfl_xor_sync(0xffffffffu, mw, o));
  }
  finite = __all_sync(0xffffffffu, finite);
  if (lane != 0) return;
  const double c = fabs(cs[e]);
  bool ok = finite && isfinite(c) && df_scale_ok(mg) && (nw == 0 || df_scale_ok(mw));
  if (c != 0.0 && nw > 0) ok = ok && df_scale_ok(c * mw);
  if (!ok) atomicOr(flag, 1);
}

void destroy_all(hd_op* h) {
  tc_free(h);
  part_free(h);
  cudaFree(h->d_vx); cudaFree(h->d_vy); cudaFree(h->d_vz);
  cudaFree(h->d_G); cudaFree(h->d_wdet); cudaFree(h->d_winv); cudaFree(h->d_wdiag); cudaFree(h->d_wgldiag);
  cudaFree(h->d_wchol);
  cudaFree(h->f_wdet); cudaFree(h->f_wgldiag);
  cudaFree(h->x_G); cudaFree(h->x_winv); cudaFree(h->x_cscale);
  cudaFree(h->d_Ga); cudaFree(h->x_Ga);
  cudaFree(h->d_cscale); cudaFree(h->d_mt); cudaFree(h->d_mtinv); cudaFree(h->d_ct);
  cudaFree(h->d_coarse_inv); cudaFree(h->d_kerr); cudaFree(h->d_red); cudaFree(h->d_tmp); cudaFree(h->d_stage);
  cudaFree(h->f_G); cudaFree(h->f_winv); cudaFree(h->f_cscale); cudaFree(h->f_mtinv); cudaFree(h->f_coarse_inv);
  for (double* p : h->mv) cudaFree(p);
  for (float* p : h->fv) cudaFree(p);
  cudaFree(h->d_ms);
  cudaFree(h->gm_V);
  cudaFree(h->gm_w);
  cudaFree(h->gm_part);
  cudaFree(h->gm_dots);
  cudaFree(h->gm_Vf);
  cudaFree(h->gm_wf);
  if (h->gm_host) cudaFreeHost(h->gm_host);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->xev) cudaEventDestroy(e);
  if (h->xstream[0]) cudaStreamDestroy(h->xstream[0]);
  if (h->xstream[1]) cudaStreamDestroy(h->xstream[1]);
  learned_free(h);
  precond_free(h);
}

}  // namespace

// 1D tables of the L2 space of degree k - 1 for q Gauss-Legendre points (Sec. 2.1), any
// k >= 1: BH[p k + j] = h_j(g_p) (histopolation basis on the GLL subcells), BG[p k + m] =
// L_m(g_p) (Lagrange basis on the k Gauss-Legendre nodes), TT[j k + m] = integral of L_m
// over subcell j, and the Gauss points and weights on [0, 1].
void hd_l2_tables(int k, int q, double* BH, double* BG, double* TT, double* gx, double* gw) {
  std::vector<double> xi = gll(k), qx, qw, gk, wk, gs, ws;
  gauss(q, qx, qw);
  gauss(k, gk, wk);
  gauss(k + 2, gs, ws);
  for (int p = 0; p < q; ++p) {
    gx[p] = qx[p];
    gw[p] = qw[p];
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int i = j + 1; i <= k; ++i) s += dlag(xi, i, qx[p]);
      BH[p * k + j] = s;
    }
    for (int m = 0; m < k; ++m) BG[p * k + m] = lag(gk, m, qx[p]);
  }
  for (int j = 0; j < k; ++j)
    for (int m = 0; m < k; ++m) {
      const double a = xi[j], b = xi[j + 1];
      double s = 0.0;
      for (size_t i = 0; i < gs.size(); ++i) s += ws[i] * lag(gk, m, a + (b - a) * gs[i]);
      TT[j * k + m] = (b - a) * s;
    }
}

hd_status elem_op_handle(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq) {
  return elem_op(h, mode, u, q, yu, yq);
}

constexpr int PROF_MAX = 4096;

void prof_mark(hd_op* h, bool before) {
  if (!h->prof || h->prof_n >= PROF_MAX) return;
  if (h->prof_ev.empty()) {
    h->prof_ev.resize(2 * PROF_MAX);
    for (auto& e : h->prof_ev) cudaEventCreate(&e);
  }
  cudaEventRecord(h->prof_ev[2 * h->prof_n + (before ? 0 : 1)], h->stream);
  if (!before) h->prof_n++;
}

// used by the Krylov layer
hd_status apply_op_internal(hd_op* h, const double* x, double* y) {
  HD_CK(h, cudaMemsetAsync(y, 0, sizeof(double) * h->n_rt, h->stream));
  return elem_op(h, OP_M | OP_DT | OP_D | OP_C, x, x + h->n_rt, y, y + h->n_rt);
}

// y = AA x with the FP32 element kernel reading and writing FP64 vectors
hd_status apply_op_mixed_internal(hd_op* h, const double* x, double* y) {
  if (h->inner_op == 1) return tc_apply(h, x, y);
  HD_CK(h, cudaMemsetAsync(y, 0, sizeof(double) * h->n_rt, h->stream));
  return elem_op_f32io64(h, OP_M | OP_DT | OP_D | OP_C, x, x + h->n_rt, y, y + h->n_rt);
}

hd_status apply_op_f32_internal(hd_op* h, const float* x, float* y) {
  if (h->inner_op == 1) return tc_apply_f32(h, x, y);
  HD_CK(h, cudaMemsetAsync(y, 0, sizeof(float) * h->n_rt, h->stream));
  return elem_op_f32(h, OP_M | OP_DT | OP_D | OP_C, x, x + h->n_rt, y, y + h->n_rt);
}

extern "C" {

hd_status hd_create(const hd_problem_desc* d, hd_handle* out) {
  const auto t_create = std::chrono::steady_clock::now();
  if (!d || !out) return HD_ERR_INVALID_ARG;
  *out = nullptr;
  hd_op* h = new (std::nothrow) hd_op();
  if (!h) return HD_ERR_OOM;
  h->desc = *d;
  if (d->kind != HD_GRAD_DIV && d->kind != HD_DARCY) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->k < 2 || d->k > HD_MAXK) { delete h; return HD_ERR_NOT_IMPLEMENTED; }
  if (!d->vx || !d->vy || !d->vz || !d->coef0 || !d->coef1) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->ess_mask > 63) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->elem_rotation) {
    // codes only renumber element-local dofs: kept for the exported maps
    const int64_t E = (int64_t)d->nx * d->ny * d->nz;
    for (int64_t e = 0; e < E; ++e)
      if (d->elem_rotation[e] < 0 || d->elem_rotation[e] > 23) { delete h; return HD_ERR_INVALID_ARG; }
    h->rot.assign(d->elem_rotation, d->elem_rotation + E);
  }
  h->desc.elem_rotation = nullptr;   // the caller's array is only read here
  h->kind = d->kind;
  h->k = d->k;
  h->q = d->q ? d->q : (d->affine ? d->k + 1 : d->k + 2);
  if (h->q != h->k + 1 && h->q != h->k + 2) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->winv_mode != HD_WINV_DENSE && d->winv_mode != HD_WINV_CG && d->winv_mode != HD_WINV_CG_HIST &&
      d->winv_mode != HD_WINV_CHOL) {
    delete h;
    return HD_ERR_INVALID_ARG;
  }
  if (d->fp64_emulation < 0 || d->fp64_emulation > 2) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->fp64_emulation >= 1 && d->winv_mode != HD_WINV_DENSE) { delete h; return HD_ERR_NOT_IMPLEMENTED; }
  h->emul = d->fp64_emulation >= 1;
  h->cycle_df = d->fp64_emulation == 2;
  h->winv_mode = d->winv_mode;
  h->tau = d->tau > 0 ? d->tau : 1.0;
  h->nu = d->nu > 0 ? d->nu : 2;
  h->coarse_max = d->coarse_max > 0 ? d->coarse_max : 512;
  if (d->cycle < 0 || d->cycle > 2) { delete h; return HD_ERR_INVALID_ARG; }
  h->cycle = d->cycle == 2 ? 2 : 1;
  if (h->coarse_max > 4096) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->smooth_levels < 0) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->smooth_levels > 2) { delete h; return HD_ERR_NOT_IMPLEMENTED; }
  h->sa = d->smooth_levels;
  if (d->w_levels < 0) { delete h; return HD_ERR_INVALID_ARG; }
  h->w_levels = d->w_levels;
  if (d->aggregation != 0 && d->aggregation != 1) { delete h; return HD_ERR_INVALID_ARG; }
  if (d->aggregation == 1 && (h->k % 2) == 1 && h->sa == 2) { delete h; return HD_ERR_NOT_IMPLEMENTED; }
  h->agg_aligned = d->aggregation;
  const int k = h->k;
  LatticeDims& L = h->L;
  L.nx = d->nx; L.ny = d->ny; L.nz = d->nz;
  L.X = d->nx * k; L.Y = d->ny * k; L.Z = d->nz * k;
  int64_t nxf = (int64_t)(L.X + 1) * L.Y * L.Z, nyf = (int64_t)L.X * (L.Y + 1) * L.Z,
          nzf = (int64_t)L.X * L.Y * (L.Z + 1);
  h->n_rt = nxf + nyf + nzf;
  h->n_l2 = (int64_t)L.X * L.Y * L.Z;
  h->n_elem = (int64_t)d->nx * d->ny * d->nz;
  if (h->n_rt + h->n_l2 >= (int64_t)1 << 31) { delete h; return HD_ERR_INVALID_ARG; }
  L.n_xf = (int)nxf; L.n_yf = (int)nyf;
  L.ess = d->ess_mask;
  const int64_t E = h->n_elem, nv = (int64_t)(d->nx + 1) * (d->ny + 1) * (d->nz + 1);
  std::vector<double> bco(E), csc(E);
  bool gamma_zero = true;
  for (int64_t e = 0; e < E; ++e) {
    double c0 = d->coef0[e], c1 = d->coef1[e];
    if (!(c0 > 0.0) || !std::isfinite(c0) || !std::isfinite(c1)) { delete h; return HD_ERR_INVALID_ARG; }
    if (h->kind == HD_GRAD_DIV) {
      if (!(c1 > 0.0)) { delete h; return HD_ERR_INVALID_ARG; }
      bco[e] = c1;          // M_beta
      csc[e] = 1.0 / c0;    // W_alpha^-1 = W^-1 / alpha (alpha constant per element)
      gamma_zero = false;
    } else {
      if (!(c1 >= 0.0)) { delete h; return HD_ERR_INVALID_ARG; }
      bco[e] = 1.0 / c0;    // M_{1/eps}
      csc[e] = c1;          // W^-1 W_gamma W^-1 = gamma W^-1 (gamma constant per element, Sec. 2.4)
      if (c1 != 0.0) gamma_zero = false;
    }
  }
  h->singular = gamma_zero && (d->ess_mask == 63);
  build_tables(k, h->q, h->tab);
  const int nq = h->q * h->q * h->q, nl2 = k * k * k;
  hd_status st = HD_OK;
  double* d_b = nullptr;
  int* d_bad = nullptr;
  do {
    if ((st = dalloc(h, &h->d_vx, nv, "vx")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_vy, nv, "vy")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_vz, nv, "vz")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_G, E * 6 * nq, "geometric factors")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_wdet, E * nq, "wdet")) != HD_OK) break;
    if (h->winv_mode == HD_WINV_DENSE && (st = dalloc(h, &h->d_winv, E * nl2 * nl2, "W inverse")) != HD_OK) break;
    if (h->winv_mode == HD_WINV_CHOL && (st = dalloc(h, &h->d_wchol, E * nl2 * nl2, "W Cholesky")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_wgldiag, E * nl2, "GL-basis W diagonal")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_wdiag, E * nl2, "W diagonal")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_cscale, E, "cscale")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_mt, h->n_rt, "M diagonal")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_mtinv, h->n_rt, "M diagonal inverse")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_ct, h->n_l2, "C~")) != HD_OK) break;
    if ((st = dalloc(h, &h->d_red, 4096, "reduction")) != HD_OK) break;
    if ((st = dalloc(h, &d_b, E, "b coefficient")) != HD_OK) break;
    if (cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) { st = hd_fail(h, HD_ERR_OOM, "flag"); break; }
    if (cudaMalloc(&h->d_kerr, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(h->d_kerr, 0, sizeof(int), h->stream) != cudaSuccess) {
      st = hd_fail(h, HD_ERR_OOM, "kernel error word");
      break;
    }
    if (cudaMallocHost(&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) { st = hd_fail(h, HD_ERR_OOM, "pinned"); break; }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->d_vx, d->vx, nv * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->d_vy, d->vy, nv * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->d_vz, d->vz, nv * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_b, bco.data(), E * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->d_cscale, csc.data(), E * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(h->d_mt, 0, h->n_rt * 8, s) != cudaSuccess || cudaMemsetAsync(d_bad, 0, 4, s) != cudaSuccess) {
      st = hd_fail(h, HD_ERR_CUDA, "upload");
      break;
    }
    if ((st = elem_setup(h, d_b, d_bad)) != HD_OK) break;
    int bad = 0;
    if (cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = hd_fail(h, HD_ERR_CUDA, "setup");
      break;
    }
    if (bad) { st = hd_fail(h, HD_ERR_INVALID_ARG, "inverted element (det J <= 0)"); break; }
    auto t_pre = std::chrono::steady_clock::now();
    if ((st = precond_setup(h)) != HD_OK) break;
    if ((st = sa_setup(h)) != HD_OK) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) { st = hd_fail(h, HD_ERR_CUDA, "setup"); break; }
    auto t_emul = std::chrono::steady_clock::now();
    h->setup_ms[3] = std::chrono::duration<float, std::milli>(t_emul - t_pre).count();
    // the affine fast path of the FP64 and double-float applies (dense W^-1 mode, q = k+1)
    if (h->emul) {
      // the double-float copies hold the FP64 element data to ~48 bits only inside
      // FP32's exponent range: refuse elements whose data leave it (k_df_range)
      const int64_t ng = E * 6 * nq, nw = E * nl2 * nl2;
      if (cudaMemsetAsync(d_bad, 0, 4, s) != cudaSuccess) { st = hd_fail(h, HD_ERR_CUDA, "range check"); break; }
      if (E > 0)
        k_df_range<<<(unsigned)((E * 32 + 255) / 256), 256, 0, s>>>(E, 6 * nq, nw > 0 ? nl2 * nl2 : 0, h->d_G,
                                                                     h->d_winv, h->d_cscale, d_bad);
      int out_of_range = 0;
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(&out_of_range, d_bad, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = hd_fail(h, HD_ERR_CUDA, "range check");
        break;
      }
      if (out_of_range) {
        st = hd_fail(h, HD_ERR_INVALID_ARG,
                     "fp64_emulation = 1: an element's geometric factors, W^-1 or C = c_e W^-1 have their "
                     "largest magnitude outside the double-float range [2^-60, 2^60]; rescale the problem "
                     "or use fp64_emulation = 0");
        break;
      }
    }
    std::vector<double> ga;
    if (d->affine && h->q == k + 1 && h->winv_mode == HD_WINV_DENSE && E > 0 && affine_factors(d, bco.data(), ga)) {
      if ((st = dalloc(h, &h->d_Ga, E * 8, "affine factors")) != HD_OK) break;
      if (cudaMemcpyAsync(h->d_Ga, ga.data(), E * 64, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = hd_fail(h, HD_ERR_CUDA, "upload");
        break;
      }
      if (h->emul) {
        for (int64_t e = 0; e < E && st == HD_OK; ++e) {
          double m = 0.0;
          for (int i = 0; i < 7; ++i) m = std::fmax(m, std::fabs(ga[e * 8 + i]));
          if (!(m >= 0x1p-60 && m <= 0x1p60))
            st = hd_fail(h, HD_ERR_INVALID_ARG,
                         "fp64_emulation = 1: an element's affine factors have their largest magnitude outside "
                         "the double-float range [2^-60, 2^60]; rescale the problem or use fp64_emulation = 0");
        }
        if (st != HD_OK) break;
        if (cudaMalloc(&h->x_Ga, sizeof(dfloat) * E * 8) != cudaSuccess) { st = hd_fail(h, HD_ERR_OOM, "affine factors"); break; }
        k_split_df<<<(unsigned)((E * 8 + 255) / 256), 256, 0, s>>>(E * 8, h->d_Ga, h->x_Ga);
      }
      // ga is read by the copy above: wait before it goes out of scope
      if (cudaStreamSynchronize(s) != cudaSuccess) { st = hd_fail(h, HD_ERR_CUDA, "affine factors"); break; }
    }
    if (h->emul) {
      const int64_t ng = E * 6 * nq, nw = E * nl2 * nl2;
      if (cudaMalloc(&h->x_G, sizeof(dfloat) * (ng > 0 ? ng : 1)) != cudaSuccess ||
          cudaMalloc(&h->x_winv, sizeof(dfloat) * (nw > 0 ? nw : 1)) != cudaSuccess ||
          cudaMalloc(&h->x_cscale, sizeof(dfloat) * (E > 0 ? E : 1)) != cudaSuccess) {
        st = hd_fail(h, HD_ERR_OOM, "double-float copies");
        break;
      }
      if (ng > 0) k_split_df<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(ng, h->d_G, h->x_G);
      if (nw > 0) k_split_df<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(nw, h->d_winv, h->x_winv);
      if (E > 0) k_split_df<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(E, h->d_cscale, h->x_cscale);
      if (cudaGetLastError() != cudaSuccess) { st = hd_fail(h, HD_ERR_CUDA, "double-float split"); break; }
    }
    // the double-float copies of the Schur hierarchy (fp64_emulation = 2), made here so that
    // the allocation-free solve finds them in place
    if (h->cycle_df && (st = setup_df_cycle(h)) != HD_OK) break;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = hd_cuda_check(h, e, "setup"); break; }
    if ((st = noalloc_prepare(h)) != HD_OK) break;
    const auto t_end = std::chrono::steady_clock::now();
    h->setup_ms[4] = std::chrono::duration<float, std::milli>(t_end - t_emul).count();
    h->setup_ms[5] = std::chrono::duration<float, std::milli>(t_end - t_create).count();
  } while (0);
  cudaFree(d_b);
  cudaFree(d_bad);
  if (st != HD_OK) {
    std::fprintf(stderr, "hd_create: %s\n", h->err.c_str());
    destroy_all(h);
    delete h;
    return st;
  }
  *out = h;
  return HD_OK;
}

hd_status hd_destroy(hd_handle h) {
  if (!h) return HD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  destroy_all(h);
  delete h;
  return HD_OK;
}

const char* hd_last_error(hd_handle h) { return h ? h->err.c_str() : "null handle"; }

hd_status hd_set_stream(hd_handle h, void* stream) {
  if (!h) return HD_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return HD_OK;
}

hd_status hd_get_setup_times(hd_handle h, double* ms, int32_t n) {
  if (!h || !ms || n < 0 || n > 6) return HD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) ms[i] = h->setup_ms[i];
  return HD_OK;
}

hd_status hd_get_sizes(hd_handle h, int64_t* n_rt, int64_t* n_l2, int64_t* n_elem) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (n_rt) *n_rt = h->n_rt;
  if (n_l2) *n_l2 = h->n_l2;
  if (n_elem) *n_elem = h->n_elem;
  return HD_OK;
}

// Rotation code r = 4 p + t of a proper cube symmetry: perm = the p-th permutation of
// (0,1,2) in lexicographic order; sgn = the t-th of the sign patterns with
// parity(perm) * sgn0 * sgn1 * sgn2 = +1, counted in increasing order of the bit
// pattern [sgn0 < 0] + 2 [sgn1 < 0] + 4 [sgn2 < 0].
static void cube_rotation(int r, int perm[3], int sgn[3]) {
  static const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const int kParity[6] = {1, -1, -1, 1, 1, -1};
  const int p = r / 4, t = r % 4;
  for (int d = 0; d < 3; ++d) perm[d] = kPerm[p][d];
  int seen = 0;
  for (int bits = 0; bits < 8; ++bits) {
    const int s0 = (bits & 1) ? -1 : 1, s1 = (bits & 2) ? -1 : 1, s2 = (bits & 4) ? -1 : 1;
    if (kParity[p] * s0 * s1 * s2 != 1) continue;
    if (seen++ == t) {
      sgn[0] = s0; sgn[1] = s1; sgn[2] = s2;
      return;
    }
  }
}

static bool lattice_sizes_ok(int32_t nx, int32_t ny, int32_t nz, int32_t k, const int8_t* rot) {
  if (nx < 1 || ny < 1 || nz < 1 || k < 1) return false;
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k, Z = (int64_t)nz * k;
  if ((X + 1) * Y * Z + X * (Y + 1) * Z + X * Y * (Z + 1) >= ((int64_t)1 << 31)) return false;
  if (rot)
    for (int64_t e = 0, E = (int64_t)nx * ny * nz; e < E; ++e)
      if (rot[e] < 0 || rot[e] > 23) return false;
  return true;
}

hd_status hd_lattice_e2d_map_rot(int32_t nx, int32_t ny, int32_t nz, int32_t k, const int8_t* rot,
                                 int32_t* out) {
  if (!out || !lattice_sizes_ok(nx, ny, nz, k, rot)) return HD_ERR_INVALID_ARG;
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k, Z = (int64_t)nz * k;
  const int64_t nxf = (X + 1) * Y * Z, nyf = X * (Y + 1) * Z;
  const int nloc = 3 * (k + 1) * k * k;
  const int64_t E = (int64_t)nx * ny * nz;
  for (int64_t e = 0; e < E; ++e) {
    const int64_t org[3] = {(e % nx) * k, ((e / nx) % ny) * k, (e / ((int64_t)nx * ny)) * k};
    int perm[3], sgn[3];
    cube_rotation(rot ? rot[e] : 0, perm, sgn);
    int32_t* row = out + e * nloc;
    int n = 0;
    for (int d = 0; d < 3; ++d) {          // reference component d: node index along axis d
      int ext[3] = {k, k, k};
      ext[d] = k + 1;
      for (int t2 = 0; t2 < ext[2]; ++t2)
        for (int t1 = 0; t1 < ext[1]; ++t1)
          for (int t0 = 0; t0 < ext[0]; ++t0) {
            const int t[3] = {t0, t1, t2};
            int64_t L[3];
            for (int c = 0; c < 3; ++c) L[perm[c]] = org[perm[c]] + (sgn[c] > 0 ? t[c] : ext[c] - 1 - t[c]);
            int64_t g;
            if (perm[d] == 0) g = L[0] + (X + 1) * (L[1] + Y * L[2]);
            else if (perm[d] == 1) g = nxf + L[0] + X * (L[1] + (Y + 1) * L[2]);
            else g = nxf + nyf + L[0] + X * (L[1] + Y * L[2]);
            row[n++] = (int32_t)(sgn[d] > 0 ? g : -1 - g);
          }
    }
  }
  return HD_OK;
}

hd_status hd_lattice_e2l_map(int32_t nx, int32_t ny, int32_t nz, int32_t k, const int8_t* rot, int32_t* out) {
  if (!out || !lattice_sizes_ok(nx, ny, nz, k, rot)) return HD_ERR_INVALID_ARG;
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k;
  const int64_t E = (int64_t)nx * ny * nz;
  const int nloc = k * k * k;
  for (int64_t e = 0; e < E; ++e) {
    const int64_t org[3] = {(e % nx) * k, ((e / nx) % ny) * k, (e / ((int64_t)nx * ny)) * k};
    int perm[3], sgn[3];
    cube_rotation(rot ? rot[e] : 0, perm, sgn);
    int32_t* row = out + e * nloc;
    int n = 0;
    for (int c2 = 0; c2 < k; ++c2)
      for (int c1 = 0; c1 < k; ++c1)
        for (int c0 = 0; c0 < k; ++c0) {
          const int t[3] = {c0, c1, c2};
          int64_t L[3];
          for (int c = 0; c < 3; ++c) L[perm[c]] = org[perm[c]] + (sgn[c] > 0 ? t[c] : k - 1 - t[c]);
          row[n++] = (int32_t)(L[0] + X * (L[1] + Y * L[2]));
        }
  }
  return HD_OK;
}

hd_status hd_lattice_is_affine(int32_t nx, int32_t ny, int32_t nz, const double* vx, const double* vy,
                               const double* vz, int32_t* affine) {
  if (!vx || !vy || !vz || !affine || nx < 1 || ny < 1 || nz < 1) return HD_ERR_INVALID_ARG;
  hd_problem_desc d{};
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.vx = vx; d.vy = vy; d.vz = vz;
  const std::vector<double> ones((size_t)nx * ny * nz, 1.0);
  std::vector<double> ga;
  *affine = affine_factors(&d, ones.data(), ga) ? 1 : 0;
  return HD_OK;
}

hd_status hd_lattice_e2d_map(int32_t nx, int32_t ny, int32_t nz, int32_t k, int32_t* out) {
  return hd_lattice_e2d_map_rot(nx, ny, nz, k, nullptr, out);
}

hd_status hd_lattice_ess_dofs(int32_t nx, int32_t ny, int32_t nz, int32_t k, uint32_t m, int64_t* out, int64_t* n) {
  if (!n || nx < 1 || ny < 1 || nz < 1 || k < 1 || m > 63) return HD_ERR_INVALID_ARG;
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k, Z = (int64_t)nz * k;
  const int64_t nxf = (X + 1) * Y * Z, nyf = X * (Y + 1) * Z;
  int64_t cnt = 0, cap = *n;
  auto emit = [&](int64_t g) {
    if (out && cnt < cap) out[cnt] = g;
    ++cnt;
  };
  // ascending global id: x-faces, then y-faces, then z-faces, each in id order
  for (int64_t K = 0; K < Z; ++K)
    for (int64_t J = 0; J < Y; ++J)
      for (int64_t I = 0; I <= X; ++I)
        if ((I == 0 && (m & 1)) || (I == X && (m & 2))) emit(I + (X + 1) * (J + Y * K));
  for (int64_t K = 0; K < Z; ++K)
    for (int64_t J = 0; J <= Y; ++J)
      for (int64_t I = 0; I < X; ++I)
        if ((J == 0 && (m & 4)) || (J == Y && (m & 8))) emit(nxf + I + X * (J + (Y + 1) * K));
  for (int64_t K = 0; K <= Z; ++K)
    for (int64_t J = 0; J < Y; ++J)
      for (int64_t I = 0; I < X; ++I)
        if ((K == 0 && (m & 16)) || (K == Z && (m & 32))) emit(nxf + nyf + I + X * (J + Y * K));
  bool overflow = out && cnt > cap;
  *n = cnt;
  return overflow ? HD_ERR_INVALID_ARG : HD_OK;
}

hd_status hd_get_e2d_map(hd_handle h, int32_t* out) {
  if (!h || !out) return HD_ERR_INVALID_ARG;
  return hd_lattice_e2d_map_rot(h->L.nx, h->L.ny, h->L.nz, h->k, h->rot.empty() ? nullptr : h->rot.data(), out);
}

hd_status hd_get_e2l_map(hd_handle h, int32_t* out) {
  if (!h || !out) return HD_ERR_INVALID_ARG;
  return hd_lattice_e2l_map(h->L.nx, h->L.ny, h->L.nz, h->k, h->rot.empty() ? nullptr : h->rot.data(), out);
}

hd_status hd_get_ess_dofs(hd_handle h, int64_t* out, int64_t* n) {
  if (!h || !n) return HD_ERR_INVALID_ARG;
  hd_status s = hd_lattice_ess_dofs(h->L.nx, h->L.ny, h->L.nz, h->k, h->L.ess, out, n);
  if (s != HD_OK) return hd_fail(h, s, "ess dof buffer too small");
  return HD_OK;
}

hd_status hd_apply_A(hd_handle h, const double* u, double* y) {
  if (!h || !u || !y) return HD_ERR_INVALID_ARG;
  HD_CK(h, cudaMemsetAsync(y, 0, sizeof(double) * h->n_rt, h->stream));
  return elem_op(h, OP_M, u, nullptr, y, nullptr);
}

hd_status hd_apply_B(hd_handle h, const double* u, double* yq) {
  if (!h || !u || !yq) return HD_ERR_INVALID_ARG;
  return lattice_apply_B(h, u, yq);
}

hd_status hd_apply_Bt(hd_handle h, const double* q, double* yu) {
  if (!h || !q || !yu) return HD_ERR_INVALID_ARG;
  return lattice_apply_Bt(h, q, yu);
}

hd_status hd_apply_C(hd_handle h, const double* q, double* yq) {
  if (!h || !q || !yq) return HD_ERR_INVALID_ARG;
  return elem_op(h, OP_C | OP_CPOS, nullptr, q, nullptr, yq);
}

hd_status hd_apply_op(hd_handle h, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  return apply_op_internal(h, x, y);
}

// Host-buffer apply, pipelined over slabs of element layers along z: the inputs of
// slab s+1 are copied in (one stream) while slab s is applied (the handle's stream)
// and the outputs of slab s-1 are copied out (a third stream). In lattice order a
// slab's inputs and outputs are four contiguous ranges (x-, y-, z-faces, cells);
// the z-face layer between two slabs receives the two slabs' addends (on zero, so
// in either order the same sum) and is copied out with the upper slab. The slabs
// taper towards both ends (layer weights 1, 2, 5, 8, 8, 5, 2, 1): only the first
// slab's copy in and the last slab's copy out are not overlapped with element work.
hd_status hd_apply_op_host(hd_handle h, const double* xh, double* yh) {
  if (!h || !xh || !yh) return HD_ERR_INVALID_ARG;
  const int64_t n = h->n_rt + h->n_l2;
  if (!h->d_stage) {
    if (cudaMalloc(&h->d_stage, sizeof(double) * 2 * (n > 0 ? n : 1)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "staging buffers");
  }
  double* dx = h->d_stage;
  double* dy = h->d_stage + n;
  const LatticeDims& L = h->L;
  static const int wt[] = {1, 2, 4, 6, 8, 8, 8, 8, 7, 5, 4, 2, 1};
  constexpr int SMAX = (int)(sizeof(wt) / sizeof(wt[0]));
  const int nz = L.nz, S = std::max(1, std::min(nz, SMAX));
  if (!h->xstream[0]) {
    if (cudaStreamCreateWithFlags(&h->xstream[0], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->xstream[1], cudaStreamNonBlocking) != cudaSuccess)
      return hd_cuda_check(h, cudaGetLastError(), "copy streams");
  }
  while ((int)h->xev.size() < 2 * S + 2) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return hd_cuda_check(h, cudaGetLastError(), "copy events");
    h->xev.push_back(e);
  }
  const int K = h->k;
  const int64_t XY = (int64_t)L.X * L.Y, sx = (int64_t)(L.X + 1) * L.Y, sy = (int64_t)L.X * (L.Y + 1);
  const int64_t oy = L.n_xf, oz = (int64_t)L.n_xf + L.n_yf, oq = h->n_rt, E2 = (int64_t)L.nx * L.ny;
  auto copy = [&](double* dst, const double* src, int64_t b, int64_t e, cudaMemcpyKind kind, cudaStream_t s) {
    return e > b ? cudaMemcpyAsync(dst + b, src + b, sizeof(double) * (e - b), kind, s) : cudaSuccess;
  };
  // copies in wait for earlier work on the handle's stream (the staging buffers)
  HD_CK(h, cudaEventRecord(h->xev[2 * S], h->stream));
  HD_CK(h, cudaStreamWaitEvent(h->xstream[0], h->xev[2 * S], 0));
  hd_status st = HD_OK;
  // Slab boundaries: cumulative weights wt (above), at least one layer per slab. The
  // copies in and out are capped near 210 and 193 GB/s on this machine (340 GB/s with both
  // directions at once) and run beside the 3.4 ms kernel. So the first slab is small, for an
  // early kernel start, and the last slabs shrink more slowly, because the copies out are
  // the slower direction. Measured per 64^3 apply (one box, each twice): 8 slabs of weights
  // 1,2,5,8,8,5,2,1: 4.71 ms; 16 equal slabs: 4.76; 2,3,5,7,7,7,7,7,6,5,4,4: 4.50;
  // 1,2,4,6,7,7,7,7,7,6,5,3,2: 4.41; these 13: 4.39.
  int zb[SMAX + 1];
  {
    int wsum = 0, acc = 0;
    for (int i = 0; i < S; ++i) wsum += wt[S == SMAX ? i : 3];
    zb[0] = 0;
    for (int i = 0; i < S; ++i) {
      acc += wt[S == SMAX ? i : 3];
      int z = (int)(((int64_t)nz * acc + wsum / 2) / wsum);
      z = std::max(z, zb[i] + 1);
      z = std::min(z, nz - (S - 1 - i));
      zb[i + 1] = z;
    }
    zb[S] = nz;
  }
  for (int s = 0; s < S && st == HD_OK; ++s) {
    const int z0 = zb[s], z1 = zb[s + 1];
    const int64_t Z0 = (int64_t)z0 * K, Z1 = (int64_t)z1 * K;
    const int64_t zin = Z0 + (s > 0 ? 1 : 0);  // the layer Z0 came with the slab below
    HD_CK(h, copy(dx, xh, sx * Z0, sx * Z1, cudaMemcpyHostToDevice, h->xstream[0]));
    HD_CK(h, copy(dx, xh, oy + sy * Z0, oy + sy * Z1, cudaMemcpyHostToDevice, h->xstream[0]));
    HD_CK(h, copy(dx, xh, oz + XY * zin, oz + XY * (Z1 + 1), cudaMemcpyHostToDevice, h->xstream[0]));
    HD_CK(h, copy(dx, xh, oq + XY * Z0, oq + XY * Z1, cudaMemcpyHostToDevice, h->xstream[0]));
    HD_CK(h, cudaEventRecord(h->xev[s], h->xstream[0]));
    HD_CK(h, cudaStreamWaitEvent(h->stream, h->xev[s], 0));
    HD_CK(h, cudaMemsetAsync(dy + sx * Z0, 0, sizeof(double) * sx * (Z1 - Z0), h->stream));
    HD_CK(h, cudaMemsetAsync(dy + oy + sy * Z0, 0, sizeof(double) * sy * (Z1 - Z0), h->stream));
    HD_CK(h, cudaMemsetAsync(dy + oz + XY * zin, 0, sizeof(double) * XY * (Z1 + 1 - zin), h->stream));
    h->e_first = (int64_t)z0 * E2;
    h->e_end = (int64_t)z1 * E2;
    st = elem_op(h, OP_M | OP_DT | OP_D | OP_C, dx, dx + h->n_rt, dy, dy + h->n_rt);
    h->e_first = 0;
    h->e_end = -1;
    if (st != HD_OK) break;
    HD_CK(h, cudaEventRecord(h->xev[S + s], h->stream));
    HD_CK(h, cudaStreamWaitEvent(h->xstream[1], h->xev[S + s], 0));
    const int64_t zout = (s == S - 1) ? Z1 + 1 : Z1;  // the top layer leaves with the slab above
    HD_CK(h, copy(yh, dy, sx * Z0, sx * Z1, cudaMemcpyDeviceToHost, h->xstream[1]));
    HD_CK(h, copy(yh, dy, oy + sy * Z0, oy + sy * Z1, cudaMemcpyDeviceToHost, h->xstream[1]));
    HD_CK(h, copy(yh, dy, oz + XY * Z0, oz + XY * zout, cudaMemcpyDeviceToHost, h->xstream[1]));
    HD_CK(h, copy(yh, dy, oq + XY * Z0, oq + XY * Z1, cudaMemcpyDeviceToHost, h->xstream[1]));
  }
  if (st != HD_OK) return st;
  HD_CK(h, cudaEventRecord(h->xev[2 * S + 1], h->xstream[1]));
  HD_CK(h, cudaStreamWaitEvent(h->stream, h->xev[2 * S + 1], 0));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  return HD_OK;
}

hd_status hd_apply_prec(hd_handle h, const double* r, double* z) {
  if (!h || !r || !z || r == z) return HD_ERR_INVALID_ARG;
  return precond_apply(h, r, z);
}

hd_status hd_apply_schur(hd_handle h, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  return schur_apply(h, x, y);
}

hd_status hd_vcycle(hd_handle h, const double* b, double* x) {
  if (!h || !b || !x || b == x) return HD_ERR_INVALID_ARG;
  return vcycle_apply(h, b, x);
}

hd_status hd_get_diagonals(hd_handle h, double* mt, double* ct) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (mt) HD_CK(h, cudaMemcpyAsync(mt, h->d_mt, sizeof(double) * h->n_rt, cudaMemcpyDeviceToDevice, h->stream));
  if (ct) HD_CK(h, cudaMemcpyAsync(ct, h->d_ct, sizeof(double) * h->n_l2, cudaMemcpyDeviceToDevice, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  return HD_OK;
}

hd_status hd_get_level(hd_handle h, int32_t l, int32_t* n_levels, int32_t dims[3]) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (n_levels) *n_levels = (int32_t)h->lv.size();
  if (dims) {
    if (l < 0 || l >= (int32_t)h->lv.size()) return hd_fail(h, HD_ERR_INVALID_ARG, "level out of range");
    dims[0] = h->lv[l].X; dims[1] = h->lv[l].Y; dims[2] = h->lv[l].Z;
  }
  return HD_OK;
}

hd_status hd_minres_solve(hd_handle h, const double* b, double* x, const hd_solve_opts* o, hd_solve_info* info) {
  if (!h || !b || !x || !o || b == x || o->maxit < 1 || !(o->rtol > 0)) return HD_ERR_INVALID_ARG;
  if (o->precision != 0 && o->precision != 1) return hd_fail(h, HD_ERR_INVALID_ARG, "precision must be 0 or 1");
  hd_status st = minres_run(h, b, x, o, info);
  if (info) {
    // true residual ||b - AA x|| / ||b|| in FP64
    const int64_t n = h->n_rt + h->n_l2;
    if (!h->d_tmp && cudaMalloc(&h->d_tmp, sizeof(double) * (n > 0 ? n : 1)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "tmp");
    hd_status s2 = apply_op_internal(h, x, h->d_tmp);
    if (s2 != HD_OK) return s2;
    double rn = 0, bn = 0;
    if ((s2 = residual_norms(h, b, h->d_tmp, &rn, &bn)) != HD_OK) return s2;
    info->true_relres = bn > 0 ? rn / bn : rn;
  }
  return st;
}

hd_status hd_profile(hd_handle h, int32_t enable) {
  if (!h) return HD_ERR_INVALID_ARG;
  h->prof = enable != 0;
  return HD_OK;
}

hd_status hd_profile_read(hd_handle h, int32_t* launches, double* ms) {
  if (!h || !launches || !ms) return HD_ERR_INVALID_ARG;
  HD_CK(h, cudaStreamSynchronize(h->stream));
  double tot = 0.0;
  for (int i = 0; i < h->prof_n; ++i) {
    float t = 0.f;
    HD_CK(h, cudaEventElapsedTime(&t, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    tot += t;
  }
  *launches = h->prof_n;
  *ms = tot;
  h->prof_n = 0;
  return HD_OK;
}

hd_status hd_apply_op_f32(hd_handle h, const float* x, float* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  hd_status st = setup_f32(h);
  if (st != HD_OK) return st;
  return apply_op_f32_internal(h, x, y);
}

hd_status hd_apply_prec_f32(hd_handle h, const float* r, float* z) {
  if (!h || !r || !z || r == z) return HD_ERR_INVALID_ARG;
  return precond_apply_f32(h, r, z);
}

}  // extern "C"
