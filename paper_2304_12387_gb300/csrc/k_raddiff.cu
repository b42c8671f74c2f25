// Grey nonlinear radiation diffusion (Sec. 4.3): the SDIRK3 time integrator, the outer
// fixed point of each stage and its element-wise Newton solve, around the Darcy solves of
// the block operator (Eq. transformed-system-darcy).
//
// Unknowns per stage: e (material energy, L2), Eh = W E (radiation energy, carried
// transformed) and F (flux, RT). The stage residual, with beta = 1 / (dt a_ii), is
//   R1 = rho beta W (e - e*) + c sigma (a N(e) - Eh) - Q
//   R2 = beta (Eh - Eh*) + W D F - c sigma (a N(e) - Eh) - S
//   R3 = M_{3 sigma/c} F - D^T Eh
// with N(e)_j = sum_p w_p T_p^4 psi_j(xi_p), where T_p = e(x_p) / Cv, e(x_p) = sum_a
// psi_a(xi_p) e_a / det J_p, and W_ab = sum_p (w_p / det J_p) psi_a psi_b.
//
// Step (1) of a pass: one CTA per element runs Newton on (R1_e, R2_e) with F fixed. The
// Jacobian is [[rho beta W + c sigma a N', -c sigma I], [-c sigma a N', (beta + c sigma) I]]
// with N' = the weighted mass of 4 T^3 / Cv. Eliminating dEh leaves
//   (rho beta W + c sigma a theta N') de = -R1 - (c sigma / (beta + c sigma)) R2,
//   theta = beta / (beta + c sigma),
// an SPD weighted mass. It is solved by Jacobi-preconditioned CG in the Gauss-Legendre
// nodal basis (Sec. 2.5). Then dEh = (-R2 + c sigma a N' de) / (beta + c sigma). The same
// CTA forms the Darcy right-hand side W^-1 (S + c sigma a N(e) + beta Eh*) at the end.
// Step (2) is the handle's MINRES on the Darcy operator, warm-started.
// Everything runs in FP64. The kernel keeps the FP64 pipe busy (70 % at 24^3), but in the
// Gauss-Legendre basis the CG converges in a few iterations, so about half of that work is
// the residual itself; the CG alone in double-float was slower (conversions included).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hd_internal.h"
#include "k_l2elem.cuh"

namespace {

constexpr int RD_THREADS = 256;
constexpr int RD_CG_MAXIT = 100;
constexpr double RD_CG_TOL2 = 1e-28;    // CG: relative residual 1e-14
constexpr double RD_NEWTON_FLOOR = 1e-14;
constexpr double RD_LINEAR_FLOOR = 1e-12;  // mixed-precision Darcy solves: ||b - AA x|| / ||b||
constexpr int RD_LINEAR_MAX_OUTER = 6;     // their FP64 residual corrections per Darcy step

struct RdTab {
  int k, q;
  double BH[HD_MAXQ * HD_MAXK];  // histopolation basis at the points: BH[p k + a]
  double BG[HD_MAXQ * HD_MAXK];  // Gauss-Legendre Lagrange basis (k nodes) at the points
  double TT[HD_MAXK * HD_MAXK];  // GL nodal -> histopolation coefficients
  double gx[HD_MAXQ], gw[HD_MAXQ];
};

// the per-element kernel's arguments; NEWTON = false evaluates (R1, R2) only
struct RdArgs {
  int64_t E;
  int nx, ny;
  RdTab t;
  double rho, cv, a, beta, rtol;
  int maxit;
  const double* wdet;  // [E][q^3] w_p / det J_p
  const double* cs;    // [E] c sigma_e
  const double *es, *Ehs, *Q, *S, *div;  // stage start, loads (NULL = 0), D F
  double *e, *Eh;      // in (and out with NEWTON)
  double* g;           // NEWTON: W^-1 (S + c sigma a N(e) + beta Eh*)
  double* r;           // residual: [R1; R2] (NULL: not written)
  double* part;        // residual: ||(R1_e, R2_e)||^2 per element
  int* flag;           // [1] most Newton steps, [2] a CG breakdown, [3] Newton at maxit unconverged
};

// shared-memory doubles of one element
__host__ __device__ inline int rd_smem_doubles(int k, int q) {
  const int n = k * k * k, nq = q * q * q;
  return 3 * q * k + k * k + 4 * nq + 20 * n + q * k * k + q * q * k + nq + 8;
}

// One CTA per element: (R1, R2) at (e, Eh), and with NEWTON the Newton loop of step (1)
// and the Darcy right-hand side.
// The Newton kernel holds 126 registers unbounded (two CTAs per SM); asked for three CTAs per
// SM it fits 80 with a small spill: 0.73 us per element and pass at 48^3 and 64^3, k = 4,
// against 1.10 and 0.76 us (four or five CTAs per SM: no better).
#ifndef HD_RAD_MINB
#define HD_RAD_MINB 3
#endif
template <bool NEWTON>
__global__ void __launch_bounds__(RD_THREADS, NEWTON ? HD_RAD_MINB : 1) k_rad_elem(RdArgs A) {
  extern __shared__ __align__(16) double rd_smem[];
  const int k = A.t.k, q = A.t.q, n = k * k * k, nq = q * q * q;
  const int64_t el = blockIdx.x;
  if (el >= A.E) return;
  double* BH = rd_smem;
  double* BG = BH + q * k;
  double* BG2 = BG + q * k;  // squares of BG (the CG's Jacobi diagonal)
  double* TT = BG2 + q * k;
  double* WQ = TT + k * k;   // w_p (tensor Gauss weights)
  double* WD = WQ + nq;      // w_p / det J_p
  double* TP = WD + nq;      // T at the points
  double* OM = TP + nq;      // weights of the Newton system
  double* ev = OM + nq;
  double* Eh = ev + n;
  double* es = Eh + n;
  double* Ehs = es + n;
  double* Qv = Ehs + n;
  double* Sv = Qv + n;
  double* WDF = Sv + n;
  double* Wes = WDF + n;
  double* R1 = Wes + n;
  double* R2 = R1 + n;
  double* Nv = R2 + n;
  double* V = Nv + n;
  double* X = V + n;   // CG: iterate, residual, direction, product, Jacobi diagonal,
  double* Rc = X + n;  // right-hand side in the GL basis
  double* Pc = Rc + n;
  double* Wc = Pc + n;
  double* DG = Wc + n;
  double* Bc = DG + n;
  double* DE = Bc + n;
  double* ZZ = DE + n;
  double* T1 = ZZ + n;
  double* T2 = T1 + q * k * k;
  double* T3 = T2 + q * q * k;
  double* red = T3 + nq;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < q * k; i += nt) {
    BH[i] = A.t.BH[i];
    BG[i] = A.t.BG[i];
    BG2[i] = A.t.BG[i] * A.t.BG[i];
  }
  for (int i = tid; i < k * k; i += nt) TT[i] = A.t.TT[i];
  const double* wd = A.wdet + el * nq;
  for (int p = tid; p < nq; p += nt) {
    WQ[p] = A.t.gw[p % q] * A.t.gw[(p / q) % q] * A.t.gw[p / (q * q)];
    WD[p] = wd[p];
  }
  for (int a = tid; a < n; a += nt) {
    const int64_t c = mi_cell(el, a, k, A.nx, A.ny);
    ev[a] = A.e[c];
    Eh[a] = A.Eh[c];
    es[a] = A.es[c];
    Ehs[a] = A.Ehs[c];
    Qv[a] = A.Q ? A.Q[c] : 0.0;
    Sv[a] = A.S ? A.S[c] : 0.0;
    V[a] = A.div[c];
  }
  __syncthreads();
  const double cs = A.cs[el], rb = A.rho * A.beta, ca = cs * A.a;
  mi_apply_w(k, q, BH, WD, V, WDF, T1, T2, T3);  // W D F
  mi_apply_w(k, q, BH, WD, es, Wes, T1, T2, T3); // W e*

  // y = K^-1 b for K = the weighted mass with point weights om (histopolation basis in
  // and out): Jacobi-preconditioned CG on TT^T K TT in the GL nodal basis, from zero
  auto cg = [&](const double* om, const double* b, double* y) {
    mi_tt3(k, TT, true, b, T1, T2, Rc);
    mi_from_points(k, q, BG2, om, T2, T1, DG);
    double rz = 0.0, bb = 0.0;
    for (int a = tid; a < n; a += nt) {
      const double z = Rc[a] / DG[a];
      X[a] = 0.0;
      Pc[a] = z;
      rz = fma(Rc[a], z, rz);
      bb = fma(Rc[a], Rc[a], bb);
    }
    rz = block_sum(rz, red);
    bb = block_sum(bb, red);
    for (int it = 0; bb > 0.0 && it < RD_CG_MAXIT; ++it) {
      mi_apply_w(k, q, BG, om, Pc, Wc, T1, T2, T3);
      double pw = 0.0;
      for (int a = tid; a < n; a += nt) pw = fma(Pc[a], Wc[a], pw);
      pw = block_sum(pw, red);
      if (!(pw > 0.0)) {  // not positive definite (T^3 < 0 at a point), or a NaN
        if (tid == 0) atomicExch(A.flag + 2, 1);
        break;
      }
      const double al = rz / pw;
      double rr = 0.0, rzn = 0.0;
      for (int a = tid; a < n; a += nt) {
        X[a] = fma(al, Pc[a], X[a]);
        const double r = fma(-al, Wc[a], Rc[a]);
        Rc[a] = r;
        rr = fma(r, r, rr);
        rzn = fma(r, r / DG[a], rzn);
      }
      rr = block_sum(rr, red);
      rzn = block_sum(rzn, red);
      if (rr <= RD_CG_TOL2 * bb) break;
      const double be = rzn / rz;
      rz = rzn;
      for (int a = tid; a < n; a += nt) Pc[a] = fma(be, Pc[a], Rc[a] / DG[a]);
      __syncthreads();
    }
    __syncthreads();
    mi_tt3(k, TT, false, X, T1, T2, y);
  };

  // T at the points and the emission N(e) of the current e; then (R1, R2) and the norms
  double rn = 0.0, sc = 0.0;
  auto residual = [&]() {
    mi_to_points(k, q, BH, ev, T1, T2, TP, (const double*)nullptr);
    for (int p = tid; p < nq; p += nt) {
      const double T = TP[p] * WD[p] / (WQ[p] * A.cv);  // 1 / det J_p = WD_p / w_p
      TP[p] = T;
      const double T2p = T * T;
      T3[p] = WQ[p] * T2p * T2p;
    }
    __syncthreads();
    mi_from_points(k, q, BH, T3, T2, T1, Nv);
    mi_apply_w(k, q, BH, WD, ev, V, T1, T2, T3);  // W e
    double s1 = 0.0, s2 = 0.0;
    for (int a = tid; a < n; a += nt) {
      const double cpl = cs * (A.a * Nv[a] - Eh[a]);
      const double r1 = rb * (V[a] - Wes[a]) + cpl - Qv[a];
      const double r2 = A.beta * (Eh[a] - Ehs[a]) + WDF[a] - cpl - Sv[a];
      R1[a] = r1;
      R2[a] = r2;
      s1 = fma(r1, r1, fma(r2, r2, s1));
      const double u = rb * V[a], v = A.beta * Eh[a];
      s2 = fma(u, u, fma(v, v, s2));
    }
    rn = block_sum(s1, red);
    sc = block_sum(s2, red);
  };

  residual();
  if constexpr (!NEWTON) {
    if (A.r)
      for (int a = tid; a < n; a += nt) {
        const int64_t c = mi_cell(el, a, k, A.nx, A.ny);
        A.r[c] = R1[a];
        A.r[A.E * n + c] = R2[a];
      }
    if (tid == 0) A.part[el] = rn;
    return;
  } else {
    const double r0 = rn, bc = A.beta + cs, th = A.beta / bc;
    int it = 0;
    bool done = false;
    for (;;) {
      done = rn <= A.rtol * A.rtol * r0 || rn <= RD_NEWTON_FLOOR * RD_NEWTON_FLOOR * sc;
      if (done || it == A.maxit) break;
      for (int p = tid; p < nq; p += nt) {
        const double T = TP[p];
        OM[p] = WD[p] * (rb + 4.0 * ca * th * T * T * T / A.cv);
      }
      for (int a = tid; a < n; a += nt) Bc[a] = -R1[a] - (cs / bc) * R2[a];
      __syncthreads();
      cg(OM, Bc, DE);
      for (int p = tid; p < nq; p += nt) {  // N' de: weights w_p 4 T^3 / (Cv det J_p)
        const double T = TP[p];
        OM[p] = WD[p] * 4.0 * T * T * T / A.cv;
      }
      __syncthreads();
      mi_apply_w(k, q, BH, OM, DE, ZZ, T1, T2, T3);
      for (int a = tid; a < n; a += nt) {
        ev[a] += DE[a];
        Eh[a] += (-R2[a] + ca * ZZ[a]) / bc;
      }
      __syncthreads();
      ++it;
      residual();
    }
    // the Darcy right-hand side from the final e (N is current)
    for (int a = tid; a < n; a += nt) Bc[a] = Sv[a] + ca * Nv[a] + A.beta * Ehs[a];
    __syncthreads();
    cg(WD, Bc, ZZ);
    for (int a = tid; a < n; a += nt) {
      const int64_t c = mi_cell(el, a, k, A.nx, A.ny);
      A.e[c] = ev[a];
      A.Eh[c] = Eh[a];
      A.g[c] = ZZ[a];
    }
    if (tid == 0) {
      atomicMax(A.flag + 1, it);
      if (!done) atomicExch(A.flag + 3, 1);
    }
  }
}

}  // namespace

namespace {

// w_p / det J(xi_p) on the trilinear element, one thread per (element, point); flag[0]:
// det J <= 0 somewhere
__global__ void k_rad_geom(int64_t E, int nx, int ny, RdTab t, const double* __restrict__ vx,
                           const double* __restrict__ vy, const double* __restrict__ vz, double* __restrict__ wdet,
                           int* __restrict__ flag) {
  const int q = t.q, nq = q * q * q;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= E * nq) return;
  const int64_t e = g / nq;
  const int p = (int)(g - e * nq), p1 = p % q, p2 = (p / q) % q, p3 = p / (q * q);
  const int64_t ex = e % nx, ey = (e / nx) % ny, ez = e / ((int64_t)nx * ny);
  const double xi[3] = {t.gx[p1], t.gx[p2], t.gx[p3]};
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // J[i][d] = d x_i / d xi_d
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
      for (int d = 0; d < 3; ++d) J[i][d] = fma(v[i], dn[d], J[i][d]);
  }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det > 0.0)) atomicExch(flag, 1);
  wdet[g] = t.gw[p1] * t.gw[p2] * t.gw[p3] / det;
}

// load_j = sum_p w_p v_p psi_j(xi_p), one CTA per element
__global__ void __launch_bounds__(RD_THREADS) k_rad_load(int64_t E, int nx, int ny, RdTab t,
                                                         const double* __restrict__ v, double* __restrict__ load) {
  extern __shared__ __align__(16) double rd_smem[];
  const int k = t.k, q = t.q, n = k * k * k, nq = q * q * q;
  const int64_t el = blockIdx.x;
  if (el >= E) return;
  double* BH = rd_smem;
  double* T1 = BH + q * k;
  double* T2 = T1 + q * k * k;
  double* T3 = T2 + q * q * k;
  double* L = T3 + nq;
  for (int i = threadIdx.x; i < q * k; i += blockDim.x) BH[i] = t.BH[i];
  for (int p = threadIdx.x; p < nq; p += blockDim.x)
    T3[p] = t.gw[p % q] * t.gw[(p / q) % q] * t.gw[p / (q * q)] * v[el * nq + p];
  __syncthreads();
  mi_from_points(k, q, BH, T3, T2, T1, L);
  for (int a = threadIdx.x; a < n; a += blockDim.x) load[mi_cell(el, a, k, nx, ny)] = L[a];
}

// y = W^-1 x per element: the CG of k_rad_elem with the weights w_p / det J_p
__global__ void __launch_bounds__(RD_THREADS) k_rad_winv(int64_t E, int nx, int ny, RdTab t,
                                                         const double* __restrict__ wdet,
                                                         const double* __restrict__ x, double* __restrict__ y,
                                                         int* __restrict__ flag) {
  extern __shared__ __align__(16) double rd_smem[];
  const int k = t.k, q = t.q, n = k * k * k, nq = q * q * q;
  const int64_t el = blockIdx.x;
  if (el >= E) return;
  double* BG = rd_smem;
  double* BG2 = BG + q * k;
  double* TT = BG2 + q * k;
  double* WD = TT + k * k;
  double* B = WD + nq;
  double* X = B + n;
  double* Rc = X + n;
  double* Pc = Rc + n;
  double* Wc = Pc + n;
  double* DG = Wc + n;
  double* Yv = DG + n;
  double* T1 = Yv + n;
  double* T2 = T1 + q * k * k;
  double* T3 = T2 + q * q * k;
  double* red = T3 + nq;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < q * k; i += nt) {
    BG[i] = t.BG[i];
    BG2[i] = t.BG[i] * t.BG[i];
  }
  for (int i = tid; i < k * k; i += nt) TT[i] = t.TT[i];
  for (int p = tid; p < nq; p += nt) WD[p] = wdet[el * nq + p];
  for (int a = tid; a < n; a += nt) B[a] = x[mi_cell(el, a, k, nx, ny)];
  __syncthreads();
  mi_tt3(k, TT, true, B, T1, T2, Rc);
  mi_from_points(k, q, BG2, WD, T2, T1, DG);
  double rz = 0.0, bb = 0.0;
  for (int a = tid; a < n; a += nt) {
    const double z = Rc[a] / DG[a];
    X[a] = 0.0;
    Pc[a] = z;
    rz = fma(Rc[a], z, rz);
    bb = fma(Rc[a], Rc[a], bb);
  }
  rz = block_sum(rz, red);
  bb = block_sum(bb, red);
  for (int it = 0; bb > 0.0 && it < RD_CG_MAXIT; ++it) {
    mi_apply_w(k, q, BG, WD, Pc, Wc, T1, T2, T3);
    double pw = 0.0;
    for (int a = tid; a < n; a += nt) pw = fma(Pc[a], Wc[a], pw);
    pw = block_sum(pw, red);
    if (!(pw > 0.0)) {
      if (tid == 0) atomicExch(flag + 2, 1);
      break;
    }
    const double al = rz / pw;
    double rr = 0.0, rzn = 0.0;
    for (int a = tid; a < n; a += nt) {
      X[a] = fma(al, Pc[a], X[a]);
      const double r = fma(-al, Wc[a], Rc[a]);
      Rc[a] = r;
      rr = fma(r, r, rr);
      rzn = fma(r, r / DG[a], rzn);
    }
    rr = block_sum(rr, red);
    rzn = block_sum(rzn, red);
    if (rr <= RD_CG_TOL2 * bb) break;
    const double be = rzn / rz;
    rz = rzn;
    for (int a = tid; a < n; a += nt) Pc[a] = fma(be, Pc[a], Rc[a] / DG[a]);
    __syncthreads();
  }
  __syncthreads();
  mi_tt3(k, TT, false, X, T1, T2, Yv);
  for (int a = tid; a < n; a += nt) y[mi_cell(el, a, k, nx, ny)] = Yv[a];
}
__host__ inline int rd_winv_smem_doubles(int k, int q) {
  const int n = k * k * k, nq = q * q * q;
  return 2 * q * k + k * k + nq + 7 * n + q * k * k + q * q * k + nq + 8;
}
__host__ inline int rd_load_smem_doubles(int k, int q) {
  return q * k + q * k * k + q * q * k + q * q * q + k * k * k;
}

// out[0] = sum_i part[i] + sum_j v[j]^2, in a fixed order (one CTA)
__global__ void k_rad_sumsq(int64_t np, const double* __restrict__ part, int64_t nv, const double* __restrict__ v,
                            double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) s = fma(v[i], v[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = t;
  }
}

// y = s x (s = -1: the sign change between Eh and the Darcy unknown)
__global__ void k_rad_scale(int64_t n, double s, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = s * x[i];
}

// y = x0 + c1 x1 + c2 x2 (x1, x2 may be NULL)
__global__ void k_rad_comb(int64_t n, const double* __restrict__ x0, double c1, const double* __restrict__ x1,
                           double c2, const double* __restrict__ x2, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x0[i];
  if (x1) v = fma(c1, x1[i], v);
  if (x2) v = fma(c2, x2[i], v);
  y[i] = v;
}

// k = (u - u*) / (dt a_ii)
__global__ void k_rad_rate(int64_t n, double inv, const double* __restrict__ u, const double* __restrict__ us,
                           double* __restrict__ kr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) kr[i] = (u[i] - us[i]) * inv;
}

inline unsigned rd_blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

struct hd_rad {
  hd_handle op = nullptr;
  int nx = 0, ny = 0, nz = 0, k = 0, q = 0;
  int64_t E = 0, n_rt = 0, n_l2 = 0;
  double rho = 1, cv = 1, a = 1, c = 1, dt = 0, beta = 0;
  double A[3][3] = {}, cst[3] = {};
  double outer_rtol = 1e-12, newton_rtol = 1e-8, linear_rtol = 1e-8;
  int outer_maxit = 10, newton_maxit = 30, linear_maxit = 20000, linear_precision = 0;
  cudaStream_t stream = nullptr;
  RdTab tab{};
  std::vector<double> hvx, hvy, hvz;
  double* d_wdet = nullptr;  // [E][q^3]
  double* d_cs = nullptr;    // [E] c sigma
  double* d_x = nullptr;     // Darcy unknown [F; -Eh]
  double* d_b = nullptr;     // Darcy right-hand side [0; W^-1 G]
  double* d_y = nullptr;     // AA x (R3)
  double* d_div = nullptr;   // D F
  double* d_part = nullptr;  // [E] element residual norms^2
  double* d_sum = nullptr;
  double* d_en = nullptr;    // step: e_n, Eh_n, stage starts and rates
  double* d_Ehn = nullptr;
  double* d_es = nullptr;
  double* d_Ehs = nullptr;
  double* d_ke = nullptr;    // [3][n_l2]
  double* d_kE = nullptr;
  int* d_flag = nullptr;     // [0] det J <= 0, [1] most Newton steps, [2] CG breakdown, [3] Newton unconverged
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::string err;
};

namespace {

hd_status rd_fail(hd_rad* h, hd_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}
hd_status rd_cuda(hd_rad* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HD_OK;
  return rd_fail(h, e == cudaErrorMemoryAllocation ? HD_ERR_OOM : HD_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
#define RD_CK(h, call)                                       \
  do {                                                       \
    hd_status s_ = rd_cuda((h), (call), #call);              \
    if (s_ != HD_OK) return s_;                              \
  } while (0)
#define RD_ST(h, call)                                       \
  do {                                                       \
    hd_status s_ = (call);                                   \
    if (s_ != HD_OK) return rd_fail((h), s_, std::string(#call) + ": " + hd_last_error((h)->op)); \
  } while (0)

// Alexander's SDIRK3: gamma is the root in (1/6, 1/2) of 6x^3 - 18x^2 + 9x - 1 (Newton from
// 0.44); c = (gamma, (1 + gamma) / 2, 1), a21 = (1 - gamma) / 2, last row b with
// b1 = -(6 gamma^2 - 16 gamma + 1) / 4, b2 = (6 gamma^2 - 20 gamma + 5) / 4, b3 = gamma.
void sdirk3_tableau(double A[3][3], double c[3]) {
  double g = 0.44;
  for (int i = 0; i < 60; ++i) {
    const double f = ((6.0 * g - 18.0) * g + 9.0) * g - 1.0, df = (18.0 * g - 36.0) * g + 9.0;
    const double d = f / df;
    g -= d;
    if (std::fabs(d) < 1e-17) break;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = 0.0;
  A[0][0] = A[1][1] = A[2][2] = g;
  A[1][0] = (1.0 - g) / 2.0;
  A[2][0] = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
  A[2][1] = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
  c[0] = g;
  c[1] = (1.0 + g) / 2.0;
  c[2] = 1.0;
}

void rd_free(hd_rad* h) {
  for (double* p : {h->d_wdet, h->d_cs, h->d_x, h->d_b, h->d_y, h->d_div, h->d_part, h->d_sum, h->d_en, h->d_Ehn,
                    h->d_es, h->d_Ehs, h->d_ke, h->d_kE})
    cudaFree(p);
  cudaFree(h->d_flag);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->op) hd_destroy(h->op);
}

RdArgs rd_args(hd_rad* h) {
  RdArgs A{};
  A.E = h->E;
  A.nx = h->nx;
  A.ny = h->ny;
  A.t = h->tab;
  A.rho = h->rho;
  A.cv = h->cv;
  A.a = h->a;
  A.beta = h->beta;
  A.rtol = h->newton_rtol;
  A.maxit = h->newton_maxit;
  A.wdet = h->d_wdet;
  A.cs = h->d_cs;
  A.flag = h->d_flag;
  return A;
}

size_t rd_elem_smem(hd_rad* h) { return sizeof(double) * rd_smem_doubles(h->k, h->q); }

// ||(R1, R2, R3)||_2 at (e, Eh, F) (host), and r = [R1; R2; R3] when r != NULL
hd_status rd_residual(hd_rad* h, const double* es, const double* Ehs, const double* Q, const double* S,
                      const double* e, const double* Eh, const double* F, double* r, double* norm) {
  cudaStream_t s = h->stream;
  RD_ST(h, hd_apply_B(h->op, F, h->d_div));
  RdArgs A = rd_args(h);
  A.es = es;
  A.Ehs = Ehs;
  A.Q = Q;
  A.S = S;
  A.div = h->d_div;
  A.e = const_cast<double*>(e);
  A.Eh = const_cast<double*>(Eh);
  A.r = r;
  A.part = h->d_part;
  k_rad_elem<false><<<(unsigned)h->E, RD_THREADS, rd_elem_smem(h), s>>>(A);
  RD_CK(h, cudaGetLastError());
  RD_CK(h, cudaMemcpyAsync(h->d_x, F, sizeof(double) * h->n_rt, cudaMemcpyDeviceToDevice, s));
  k_rad_scale<<<rd_blocks(h->n_l2), 256, 0, s>>>(h->n_l2, -1.0, Eh, h->d_x + h->n_rt);
  RD_ST(h, hd_apply_op(h->op, h->d_x, h->d_y));
  if (r) RD_CK(h, cudaMemcpyAsync(r + 2 * h->n_l2, h->d_y, sizeof(double) * h->n_rt, cudaMemcpyDeviceToDevice, s));
  k_rad_sumsq<<<1, 1024, 0, s>>>(h->E, h->d_part, h->n_rt, h->d_y, h->d_sum);
  double v = 0.0;
  RD_CK(h, cudaMemcpyAsync(&v, h->d_sum, sizeof(double), cudaMemcpyDeviceToHost, s));
  RD_CK(h, cudaStreamSynchronize(s));
  if (!std::isfinite(v)) return rd_fail(h, HD_ERR_NAN, "non-finite stage residual");
  *norm = std::sqrt(v);
  return HD_OK;
}

float rd_elapsed(hd_rad* h) {
  float ms = 0.f;
  cudaEventSynchronize(h->ev[1]);
  cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
  return ms;
}

hd_status rd_stage(hd_rad* h, const double* es, const double* Ehs, const double* Q, const double* S, double* e,
                   double* Eh, double* F, hd_rad_info* info) {
  cudaStream_t s = h->stream;
  double r0 = 0.0, r = 0.0;
  RD_CK(h, cudaEventRecord(h->ev[0], s));
  hd_status st = rd_residual(h, es, Ehs, Q, S, e, Eh, F, nullptr, &r0);
  if (st != HD_OK) return st;
  RD_CK(h, cudaEventRecord(h->ev[1], s));
  info->ms_residual += rd_elapsed(h);
  info->stages += 1;
  if (r0 == 0.0) return HD_OK;
  double r_prev = r0;
  int passes = 0;
  bool conv = false;
  for (int m = 0; m < h->outer_maxit; ++m) {
    // (1) F lagged: Newton per element, and the Darcy right-hand side W^-1 G into d_b
    RD_CK(h, cudaEventRecord(h->ev[0], s));
    RD_CK(h, cudaMemsetAsync(h->d_flag + 1, 0, 3 * sizeof(int), s));
    RD_ST(h, hd_apply_B(h->op, F, h->d_div));
    RdArgs A = rd_args(h);
    A.es = es;
    A.Ehs = Ehs;
    A.Q = Q;
    A.S = S;
    A.div = h->d_div;
    A.e = e;
    A.Eh = Eh;
    A.g = h->d_b + h->n_rt;
    k_rad_elem<true><<<(unsigned)h->E, RD_THREADS, rd_elem_smem(h), s>>>(A);
    RD_CK(h, cudaGetLastError());
    int fl[3] = {0, 0, 0};
    RD_CK(h, cudaMemcpyAsync(fl, h->d_flag + 1, sizeof(fl), cudaMemcpyDeviceToHost, s));
    RD_CK(h, cudaEventRecord(h->ev[1], s));
    info->ms_newton += rd_elapsed(h);
    if (fl[1]) return rd_fail(h, HD_ERR_NAN, "a Newton system was not positive definite");
    if (fl[0] > info->newton_max) info->newton_max = fl[0];
    // (2) e fixed: the Darcy solve for x = [F; -Eh], warm-started
    RD_CK(h, cudaEventRecord(h->ev[0], s));
    RD_CK(h, cudaMemsetAsync(h->d_b, 0, sizeof(double) * h->n_rt, s));
    RD_CK(h, cudaMemcpyAsync(h->d_x, F, sizeof(double) * h->n_rt, cudaMemcpyDeviceToDevice, s));
    k_rad_scale<<<rd_blocks(h->n_l2), 256, 0, s>>>(h->n_l2, -1.0, Eh, h->d_x + h->n_rt);
    hd_solve_opts o{};
    o.rtol = h->linear_rtol;
    o.maxit = h->linear_maxit;
    o.use_x0 = 1;
    o.check_every = 4;
    bool solve = true;
    if (h->linear_precision == 1) {  // target: the true residual falls by linear_rtol
      const int64_t n = h->n_rt + h->n_l2;
      RD_ST(h, hd_apply_op(h->op, h->d_x, h->d_y));
      k_rad_comb<<<rd_blocks(n), 256, 0, s>>>(n, h->d_b, -1.0, h->d_y, 0.0, nullptr, h->d_y);
      double nn[2] = {0.0, 0.0};
      k_rad_sumsq<<<1, 1024, 0, s>>>(0, nullptr, n, h->d_y, h->d_sum);
      RD_CK(h, cudaMemcpyAsync(&nn[0], h->d_sum, sizeof(double), cudaMemcpyDeviceToHost, s));
      k_rad_sumsq<<<1, 1024, 0, s>>>(0, nullptr, n, h->d_b, h->d_sum);
      RD_CK(h, cudaMemcpyAsync(&nn[1], h->d_sum, sizeof(double), cudaMemcpyDeviceToHost, s));
      RD_CK(h, cudaStreamSynchronize(s));
      if (!std::isfinite(nn[0]) || !std::isfinite(nn[1])) return rd_fail(h, HD_ERR_NAN, "non-finite Darcy residual");
      // a true residual below ~1e-12 ||b|| is at the FP64 operator's rounding level: there the
      // warm start is kept (a recurrence estimate, as in the FP64 solve, would keep falling)
      const double rel0 = nn[1] > 0.0 ? std::sqrt(nn[0] / nn[1]) : 0.0;
      solve = rel0 > RD_LINEAR_FLOOR;
      o.precision = 1;
      o.rtol = 1e-4;
      o.max_outer = RD_LINEAR_MAX_OUTER;
      o.outer_rtol = std::max(h->linear_rtol * rel0, RD_LINEAR_FLOOR);
    }
    hd_solve_info si{};
    if (solve) {
      const hd_status ls = hd_minres_solve(h->op, h->d_b, h->d_x, &o, &si);
      // The mixed solve's stop uses the true residual, whose rounding (the operator applied to
      // a large x) can lie above the target: after RD_LINEAR_MAX_OUTER corrections its
      // iterate is kept, and the stage residual decides whether the pass converged.
      const bool kept = ls == HD_ERR_NOT_CONVERGED && h->linear_precision == 1 && std::isfinite(si.true_relres);
      if (ls != HD_OK && !kept)
        return rd_fail(h, ls, std::string("Darcy solve: ") + hd_last_error(h->op));
    }
    RD_CK(h, cudaMemcpyAsync(F, h->d_x, sizeof(double) * h->n_rt, cudaMemcpyDeviceToDevice, s));
    k_rad_scale<<<rd_blocks(h->n_l2), 256, 0, s>>>(h->n_l2, -1.0, h->d_x + h->n_rt, Eh);
    RD_CK(h, cudaEventRecord(h->ev[1], s));
    info->ms_linear += rd_elapsed(h);
    info->linear_solves += 1;
    info->linear_iterations += si.iterations;
    // the stage residual
    RD_CK(h, cudaEventRecord(h->ev[0], s));
    st = rd_residual(h, es, Ehs, Q, S, e, Eh, F, nullptr, &r);
    if (st != HD_OK) return st;
    RD_CK(h, cudaEventRecord(h->ev[1], s));
    info->ms_residual += rd_elapsed(h);
    passes = m + 1;
    // converged, or at the rounding floor: no longer halving, already near the target
    if (r <= h->outer_rtol * r0 || (r > 0.5 * r_prev && r <= 1e3 * h->outer_rtol * r0)) {
      conv = true;
      break;
    }
    r_prev = r;
  }
  info->outer += passes;
  if (passes > info->outer_max) info->outer_max = passes;
  if (r / r0 > info->relres) info->relres = r / r0;
  if (!conv) return rd_fail(h, HD_ERR_NOT_CONVERGED, "stage: outer iteration did not reach its tolerance");
  return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_rad_create(const hd_rad_desc* d, hd_rad_handle* out) {
  if (!d || !out) return HD_ERR_INVALID_ARG;
  *out = nullptr;
  const hd_problem_desc& m = d->mesh;
  if (m.nx < 1 || m.ny < 1 || m.nz < 1 || !m.vx || !m.vy || !m.vz || !d->sigma) return HD_ERR_INVALID_ARG;
  if (!(d->rho > 0) || !(d->cv > 0) || !(d->a > 0) || !(d->c > 0) || !(d->dt > 0)) return HD_ERR_INVALID_ARG;
  if (d->outer_rtol < 0 || d->newton_rtol < 0 || d->linear_rtol < 0 || d->outer_maxit < 0 || d->newton_maxit < 0 ||
      d->linear_maxit < 0)
    return HD_ERR_INVALID_ARG;
  const int64_t E = (int64_t)m.nx * m.ny * m.nz;
  for (int64_t e = 0; e < E; ++e)
    if (!(d->sigma[e] > 0) || !std::isfinite(d->sigma[e])) return HD_ERR_INVALID_ARG;
  hd_rad* h = new hd_rad();
  h->nx = m.nx;
  h->ny = m.ny;
  h->nz = m.nz;
  h->k = m.k;
  h->E = E;
  h->rho = d->rho;
  h->cv = d->cv;
  h->a = d->a;
  h->c = d->c;
  h->dt = d->dt;
  sdirk3_tableau(h->A, h->cst);
  h->beta = 1.0 / (h->dt * h->A[0][0]);
  if (d->outer_rtol > 0) h->outer_rtol = d->outer_rtol;
  if (d->newton_rtol > 0) h->newton_rtol = d->newton_rtol;
  if (d->linear_rtol > 0) h->linear_rtol = d->linear_rtol;
  if (d->linear_precision < 0 || d->linear_precision > 1) {
    delete h;
    return HD_ERR_INVALID_ARG;
  }
  h->linear_precision = d->linear_precision;
  if (d->outer_maxit > 0) h->outer_maxit = d->outer_maxit;
  if (d->newton_maxit > 0) h->newton_maxit = d->newton_maxit;
  if (d->linear_maxit > 0) h->linear_maxit = d->linear_maxit;
  // the Darcy operator: eps = c / (3 sigma), gamma = beta + c sigma, reflecting walls
  std::vector<double> eps(E), gam(E), cs(E);
  for (int64_t e = 0; e < E; ++e) {
    cs[e] = h->c * d->sigma[e];
    eps[e] = h->c / (3.0 * d->sigma[e]);
    gam[e] = h->beta + cs[e];
  }
  hd_problem_desc pd = m;
  pd.kind = HD_DARCY;
  pd.coef0 = eps.data();
  pd.coef1 = gam.data();
  pd.ess_mask = 63u;
  pd.affine = 0;
  pd.elem_rotation = nullptr;
  hd_status st = hd_create(&pd, &h->op);
  if (st != HD_OK) {
    delete h;
    return st;
  }
  h->q = h->op->q;
  int64_t ne = 0;
  hd_get_sizes(h->op, &h->n_rt, &h->n_l2, &ne);
  h->tab.k = h->k;
  h->tab.q = h->q;
  hd_l2_tables(h->k, h->q, h->tab.BH, h->tab.BG, h->tab.TT, h->tab.gx, h->tab.gw);
  const int64_t nv = (int64_t)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
  h->hvx.assign(m.vx, m.vx + nv);
  h->hvy.assign(m.vy, m.vy + nv);
  h->hvz.assign(m.vz, m.vz + nv);
  const int64_t nq = (int64_t)h->q * h->q * h->q, nl = h->n_l2;
  auto fail = [&](hd_status s) {
    rd_free(h);
    delete h;
    return s;
  };
  double* dv[3] = {nullptr, nullptr, nullptr};
  cudaError_t ce = cudaSuccess;
  for (double** p : {&h->d_wdet}) ce = ce ? ce : cudaMalloc(p, sizeof(double) * E * nq);
  for (double** p : {&h->d_cs, &h->d_part}) ce = ce ? ce : cudaMalloc(p, sizeof(double) * E);
  for (double** p : {&h->d_x, &h->d_b, &h->d_y}) ce = ce ? ce : cudaMalloc(p, sizeof(double) * (h->n_rt + nl));
  for (double** p : {&h->d_div, &h->d_en, &h->d_Ehn, &h->d_es, &h->d_Ehs})
    ce = ce ? ce : cudaMalloc(p, sizeof(double) * nl);
  for (double** p : {&h->d_ke, &h->d_kE}) ce = ce ? ce : cudaMalloc(p, sizeof(double) * 3 * nl);
  if (!ce) ce = cudaMalloc(&h->d_sum, sizeof(double));
  if (!ce) ce = cudaMalloc(&h->d_flag, 4 * sizeof(int));
  for (int i = 0; i < 3 && !ce; ++i) ce = cudaMalloc(&dv[i], sizeof(double) * nv);
  if (!ce) ce = cudaMemcpy(dv[0], m.vx, sizeof(double) * nv, cudaMemcpyHostToDevice);
  if (!ce) ce = cudaMemcpy(dv[1], m.vy, sizeof(double) * nv, cudaMemcpyHostToDevice);
  if (!ce) ce = cudaMemcpy(dv[2], m.vz, sizeof(double) * nv, cudaMemcpyHostToDevice);
  if (!ce) ce = cudaMemcpy(h->d_cs, cs.data(), sizeof(double) * E, cudaMemcpyHostToDevice);
  if (!ce) ce = cudaMemset(h->d_flag, 0, 4 * sizeof(int));
  if (!ce) {
    k_rad_geom<<<rd_blocks(E * nq), 256>>>(E, m.nx, m.ny, h->tab, dv[0], dv[1], dv[2], h->d_wdet, h->d_flag);
    ce = cudaGetLastError();
  }
  int bad = 0;
  if (!ce) ce = cudaMemcpy(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  for (double* p : dv) cudaFree(p);
  if (!ce) ce = cudaFuncSetAttribute(k_rad_elem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rd_elem_smem(h));
  if (!ce) ce = cudaFuncSetAttribute(k_rad_elem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rd_elem_smem(h));
  if (!ce) ce = cudaEventCreate(&h->ev[0]);
  if (!ce) ce = cudaEventCreate(&h->ev[1]);
  if (ce) return fail(ce == cudaErrorMemoryAllocation ? HD_ERR_OOM : HD_ERR_CUDA);
  if (bad) return fail(HD_ERR_INVALID_ARG);
  *out = h;
  return HD_OK;
}

hd_status hd_rad_destroy(hd_rad_handle h) {
  if (!h) return HD_ERR_INVALID_ARG;
  rd_free(h);
  delete h;
  return HD_OK;
}

hd_status hd_rad_set_stream(hd_rad_handle h, void* stream) {
  if (!h) return HD_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return hd_set_stream(h->op, stream);
}

const char* hd_rad_last_error(hd_rad_handle h) { return h ? h->err.c_str() : ""; }

hd_status hd_rad_get_sizes(hd_rad_handle h, int64_t* n_rt, int64_t* n_l2, int64_t* n_elem, int32_t* q) {
  if (!h) return HD_ERR_INVALID_ARG;
  if (n_rt) *n_rt = h->n_rt;
  if (n_l2) *n_l2 = h->n_l2;
  if (n_elem) *n_elem = h->E;
  if (q) *q = h->q;
  return HD_OK;
}

hd_status hd_rad_get_op(hd_rad_handle h, hd_handle* op) {
  if (!h || !op) return HD_ERR_INVALID_ARG;
  *op = h->op;
  return HD_OK;
}

hd_status hd_rad_points(hd_rad_handle h, double* xyz) {
  if (!h || !xyz) return HD_ERR_INVALID_ARG;
  const int q = h->q, nq = q * q * q;
  for (int64_t e = 0; e < h->E; ++e) {
    const int64_t ex = e % h->nx, ey = (e / h->nx) % h->ny, ez = e / ((int64_t)h->nx * h->ny);
    for (int p = 0; p < nq; ++p) {
      const double xi[3] = {h->tab.gx[p % q], h->tab.gx[(p / q) % q], h->tab.gx[p / (q * q)]};
      double x[3] = {0.0, 0.0, 0.0};
      for (int c = 0; c < 8; ++c) {
        const int b[3] = {c & 1, (c >> 1) & 1, c >> 2};
        const int64_t id = (ex + b[0]) + (int64_t)(h->nx + 1) * ((ey + b[1]) + (int64_t)(h->ny + 1) * (ez + b[2]));
        const double w = (b[0] ? xi[0] : 1.0 - xi[0]) * (b[1] ? xi[1] : 1.0 - xi[1]) * (b[2] ? xi[2] : 1.0 - xi[2]);
        x[0] += w * h->hvx[id];
        x[1] += w * h->hvy[id];
        x[2] += w * h->hvz[id];
      }
      double* o = xyz + 3 * (e * nq + p);
      o[0] = x[0];
      o[1] = x[1];
      o[2] = x[2];
    }
  }
  return HD_OK;
}

hd_status hd_rad_load(hd_rad_handle h, const double* values, double* load) {
  if (!h || !values || !load) return HD_ERR_INVALID_ARG;
  const size_t sm = sizeof(double) * rd_load_smem_doubles(h->k, h->q);
  k_rad_load<<<(unsigned)h->E, RD_THREADS, sm, h->stream>>>(h->E, h->nx, h->ny, h->tab, values, load);
  RD_CK(h, cudaGetLastError());
  return HD_OK;
}

hd_status hd_rad_winv(hd_rad_handle h, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  const size_t sm = sizeof(double) * rd_winv_smem_doubles(h->k, h->q);
  RD_CK(h, cudaMemsetAsync(h->d_flag + 2, 0, sizeof(int), h->stream));
  k_rad_winv<<<(unsigned)h->E, RD_THREADS, sm, h->stream>>>(h->E, h->nx, h->ny, h->tab, h->d_wdet, x, y, h->d_flag);
  RD_CK(h, cudaGetLastError());
  return HD_OK;
}

hd_status hd_rad_residual(hd_rad_handle h, const double* e_star, const double* Eh_star, const double* q_load,
                          const double* s_load, const double* e, const double* Eh, const double* F, double* r,
                          double* norm) {
  if (!h || !e_star || !Eh_star || !e || !Eh || !F) return HD_ERR_INVALID_ARG;
  double v = 0.0;
  hd_status st = rd_residual(h, e_star, Eh_star, q_load, s_load, e, Eh, F, r, &v);
  if (st == HD_OK && norm) *norm = v;
  return st;
}

hd_status hd_rad_stage(hd_rad_handle h, const double* e_star, const double* Eh_star, const double* q_load,
                       const double* s_load, double* e, double* Eh, double* F, hd_rad_info* info) {
  if (!h || !e_star || !Eh_star || !e || !Eh || !F) return HD_ERR_INVALID_ARG;
  if (e == e_star || Eh == Eh_star) return HD_ERR_INVALID_ARG;
  hd_rad_info loc{};
  hd_status st = rd_stage(h, e_star, Eh_star, q_load, s_load, e, Eh, F, &loc);
  loc.status = st;
  if (info) *info = loc;
  return st;
}

hd_status hd_rad_step(hd_rad_handle h, double* e, double* Eh, double* F, const double* q_loads,
                      const double* s_loads, hd_rad_info* info) {
  if (!h || !e || !Eh || !F) return HD_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  const int64_t nl = h->n_l2;
  hd_rad_info loc{};
  hd_status st = HD_OK;
  auto body = [&]() -> hd_status {
    RD_CK(h, cudaMemcpyAsync(h->d_en, e, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
    RD_CK(h, cudaMemcpyAsync(h->d_Ehn, Eh, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < 3; ++i) {
      // stage start u* = u_n + dt sum_{j < i} a_ij k_j
      const double c1 = h->dt * h->A[i][0], c2 = h->dt * h->A[i][1];
      const double* k1e = i > 0 ? h->d_ke : nullptr;
      const double* k2e = i > 1 ? h->d_ke + nl : nullptr;
      const double* k1E = i > 0 ? h->d_kE : nullptr;
      const double* k2E = i > 1 ? h->d_kE + nl : nullptr;
      k_rad_comb<<<rd_blocks(nl), 256, 0, s>>>(nl, h->d_en, c1, k1e, c2, k2e, h->d_es);
      k_rad_comb<<<rd_blocks(nl), 256, 0, s>>>(nl, h->d_Ehn, c1, k1E, c2, k2E, h->d_Ehs);
      RD_CK(h, cudaGetLastError());
      hd_status si = rd_stage(h, h->d_es, h->d_Ehs, q_loads ? q_loads + i * nl : nullptr,
                              s_loads ? s_loads + i * nl : nullptr, e, Eh, F, &loc);
      if (si != HD_OK) return si;
      const double inv = 1.0 / (h->dt * h->A[i][i]);
      k_rad_rate<<<rd_blocks(nl), 256, 0, s>>>(nl, inv, e, h->d_es, h->d_ke + i * nl);
      k_rad_rate<<<rd_blocks(nl), 256, 0, s>>>(nl, inv, Eh, h->d_Ehs, h->d_kE + i * nl);
      RD_CK(h, cudaGetLastError());
    }
    RD_CK(h, cudaStreamSynchronize(s));
    return HD_OK;
  };
  st = body();
  loc.status = st;
  if (info) *info = loc;
  return st;
}

}  // extern "C"
