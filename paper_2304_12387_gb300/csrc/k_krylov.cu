// Krylov layer: deterministic FP64 inner products (warp shuffles -> fixed
// per-block partials -> one fixed-order final pass) and preconditioned MINRES
// (Paige & Saunders 1975) with its Lanczos/Givens scalars kept on the device,
// so an iteration needs no host round trip (Sec. 3: MINRES with the
// block-diagonal preconditioner); restarted GMRES for the block-triangular
// preconditioner of the remark in Sec. 2.3.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "dfloat.cuh"
#include "hd_internal.h"

namespace {
constexpr int TPB = 256;
constexpr int DOT_BLOCKS = 1024;  // fixed: the reduction order does not depend on the data
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (ln < (int)(blockDim.x >> 5)) ? sh[ln] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

// partial[b] = sum over block b's contiguous chunk of a[i]*b[i]
__global__ void k_dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ partial) {
  __shared__ double sh[32];
  int64_t chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_dot_final(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = block_sum(partial[threadIdx.x], sh);  // blockDim.x == DOT_BLOCKS
  if (threadIdx.x == 0) out[0] = s;
}

}  // namespace

struct MinresState {
  double beta, beta_prev, alpha, c, s, d_bar, eps, eps_next, delta, gamma, phi, phi_bar, eta0, rtol;
  double inv_beta, inv_gamma, alpha_over_beta;  // published by the one-thread kernels: the vector
                                                // kernels multiply (an FP64 divide per element is
                                                // several FP64 ops on this GPU)
  double dot;       // scratch result of the last inner product
  int done_at;      // iteration at which the recurrence stopped (-1: running)
  int status;       // HD_OK / HD_ERR_*
};

namespace {

// y -= (beta/beta_prev) r_pp (when it > 1); partial sums of v.y
__global__ void k_mr_lanczos1(int64_t n, int it, const MinresState* __restrict__ st, const double* __restrict__ v,
                              double* __restrict__ y, const double* __restrict__ rpp, double* __restrict__ partial) {
  __shared__ double sh[32];
  const double f = (it > 1) ? st->beta / st->beta_prev : 0.0;
  int64_t chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double yi = y[i];
    if (it > 1) yi = fma(-f, rpp[i], yi);
    y[i] = yi;
    s = fma(v[i], yi, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_mr_alpha(MinresState* st, const double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = block_sum(partial[threadIdx.x], sh);
  if (threadIdx.x == 0) {
    st->alpha = s;
    st->alpha_over_beta = s / st->beta;
  }
}

// y -= (alpha/beta) r_p  (y becomes the new Lanczos vector r);  z_u = r_u * mtinv
__global__ void k_mr_lanczos2(int64_t n, int64_t n_rt, const MinresState* __restrict__ st,
                              double* __restrict__ y, const double* __restrict__ rp,
                              const double* __restrict__ mtinv, double* __restrict__ z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f = st->alpha_over_beta;
  double yi = fma(-f, rp[i], y[i]);
  y[i] = yi;
  if (i < n_rt) z[i] = yi * mtinv[i];
}

// beta_{j+1} from the partials of r.z; then the Givens update and the stopping test
__global__ void k_mr_beta_givens(MinresState* st, const double* __restrict__ partial, int it) {
  __shared__ double sh[32];
  double b2 = block_sum(partial[threadIdx.x], sh);
  if (threadIdx.x != 0 || st->done_at >= 0) return;
  if (!(b2 >= 0.0) || !isfinite(st->alpha)) {
    st->status = isfinite(b2) && isfinite(st->alpha) ? HD_ERR_PREC_INDEFINITE : HD_ERR_NAN;
    st->done_at = it - 1;
    return;
  }
  st->beta_prev = st->beta;
  st->beta = sqrt(b2);
  // previous rotation applied to the new column, then a new rotation
  st->eps = st->eps_next;
  double delta = st->c * st->d_bar + st->s * st->alpha;
  double g_bar = st->s * st->d_bar - st->c * st->alpha;
  st->eps_next = st->s * st->beta;
  st->d_bar = -st->c * st->beta;
  double gamma = hypot(g_bar, st->beta);
  if (!(gamma > 0.0)) {
    st->status = HD_ERR_NAN;
    st->done_at = it - 1;
    return;
  }
  st->c = g_bar / gamma;
  st->s = st->beta / gamma;
  st->delta = delta;
  st->gamma = gamma;
  st->inv_gamma = 1.0 / gamma;
  st->inv_beta = 1.0 / st->beta;
  st->phi = st->c * st->phi_bar;
  st->phi_bar = st->s * st->phi_bar;
  if (fabs(st->phi_bar) <= st->rtol * st->eta0) {
    st->status = HD_OK;
    st->done_at = it;
  }
}

// w_new = (v - eps w_pp - delta w_p)/gamma; x += phi w_new; v_next = z / beta
__global__ void k_mr_update(int64_t n, int it, const MinresState* __restrict__ st, const double* __restrict__ v,
                            const double* __restrict__ wpp, const double* __restrict__ wp, double* __restrict__ wn,
                            double* __restrict__ x, const double* __restrict__ z, double* __restrict__ vnext) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (st->done_at >= 0 && st->done_at < it) return;
  double w = fma(-st->eps, wpp[i], fma(-st->delta, wp[i], v[i])) * st->inv_gamma;
  wn[i] = w;
  x[i] = fma(st->phi, w, x[i]);
  vnext[i] = z[i] * st->inv_beta;
}

__global__ void k_mr_init(MinresState* st, const double* __restrict__ partial, double rtol) {
  __shared__ double sh[32];
  double b2 = block_sum(partial[threadIdx.x], sh);
  if (threadIdx.x != 0) return;
  st->rtol = rtol;
  st->beta_prev = 0.0;
  st->c = -1.0;
  st->s = 0.0;
  st->d_bar = 0.0;
  st->eps = 0.0;
  st->eps_next = 0.0;
  st->done_at = -1;
  st->status = HD_OK;
  if (!(b2 >= 0.0)) {
    st->status = isfinite(b2) ? HD_ERR_PREC_INDEFINITE : HD_ERR_NAN;
    st->done_at = 0;
    st->beta = 1.0;
    st->inv_beta = 1.0;
    return;
  }
  st->beta = sqrt(b2);
  st->eta0 = st->beta;
  st->phi_bar = st->beta;
  if (st->beta == 0.0) {
    st->done_at = 0;
    st->beta = 1.0;
  }
  st->inv_beta = 1.0 / st->beta;
}

__global__ void k_scale_div(int64_t n, const double* __restrict__ z, const MinresState* __restrict__ st,
                            double* __restrict__ v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  v[i] = z[i] * st->inv_beta;
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = a * x[i] + b * y[i];
}

// partial sums of (a - b)^2 and a^2
__global__ void k_resid_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ partial) {
  __shared__ double sh[32];
  int64_t chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double s = 0.0, t = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double d = a[i] - b[i];
    s = fma(d, d, s);
    t = fma(a[i], a[i], t);
  }
  s = block_sum(s, sh);
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    partial[DOT_BLOCKS + blockIdx.x] = t;
  }
}

__global__ void k_resid_final(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = block_sum(partial[threadIdx.x], sh);
  double t = block_sum(partial[DOT_BLOCKS + threadIdx.x], sh);
  if (threadIdx.x == 0) {
    out[0] = s;
    out[1] = t;
  }
}

}  // namespace

// ||b - y||_2 and ||b||_2 (y = AA x computed by the caller)
hd_status residual_norms(hd_op* h, const double* b, const double* y, double* rn, double* bn) {
  const int64_t n = h->n_rt + h->n_l2;
  k_resid_partial<<<DOT_BLOCKS, TPB, 0, h->stream>>>(n, b, y, h->d_red);
  k_resid_final<<<1, DOT_BLOCKS, 0, h->stream>>>(h->d_red, h->d_red + 2 * DOT_BLOCKS);
  HD_LAUNCH_CK(h, "residual norms");
  HD_CK(h, cudaMemcpyAsync(h->h_pinned, h->d_red + 2 * DOT_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  *rn = std::sqrt(h->h_pinned[0]);
  *bn = std::sqrt(h->h_pinned[1]);
  return HD_OK;
}

hd_status dot_device(hd_op* h, const double* a, const double* b, int64_t n, double* d_out) {
  k_dot_partial<<<DOT_BLOCKS, TPB, 0, h->stream>>>(n, a, b, h->d_red);
  k_dot_final<<<1, DOT_BLOCKS, 0, h->stream>>>(h->d_red, d_out);
  HD_LAUNCH_CK(h, "dot");
  return HD_OK;
}

hd_status apply_op_internal(hd_op* h, const double* x, double* y);
hd_status apply_op_f32_internal(hd_op* h, const float* x, float* y);
hd_status apply_op_mixed_internal(hd_op* h, const double* x, double* y);

namespace {

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_f2d(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
// y = b - y
__global__ void k_rsub(int64_t n, const double* __restrict__ b, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = b[i] - y[i];
}
// x += e
__global__ void k_add(int64_t n, const double* __restrict__ e, double* __restrict__ x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += e[i];
}

}  // namespace

static hd_status ensure_minres(hd_op* h) {
  if (!h->mv.empty()) return HD_OK;
  int64_t n = h->n_rt + h->n_l2;
  for (int i = 0; i < 11; ++i) {  // 9 recurrence vectors + outer residual + correction
    double* p = nullptr;
    if (cudaMalloc(&p, sizeof(double) * (n > 0 ? n : 1)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "minres work");
    h->mv.push_back(p);
  }
  if (cudaMalloc(&h->d_ms, sizeof(MinresState)) != cudaSuccess) return hd_fail(h, HD_ERR_OOM, "minres state");
  return HD_OK;
}

static hd_status ensure_f32_work(hd_op* h) {
  if (!h->fv.empty()) return HD_OK;
  hd_status st = setup_f32(h);
  if (st != HD_OK) return st;
  int64_t n = h->n_rt + h->n_l2;
  const int64_t sizes[4] = {n, n, h->n_l2, h->n_l2};
  for (int i = 0; i < 4; ++i) {
    float* p = nullptr;
    if (cudaMalloc(&p, sizeof(float) * (sizes[i] > 0 ? sizes[i] : 1)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "f32 work");
    h->fv.push_back(p);
  }
  return HD_OK;
}

namespace {
__global__ void k_axpy_d(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}
__global__ void k_xpay_d(int64_t n, const double* __restrict__ z, double b, double* __restrict__ p) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = fma(b, p[i], z[i]);
}
}  // namespace

hd_status axpy_dev(hd_op* h, int64_t n, double a, const double* x, double* y) {
  k_axpy_d<<<nblk(n), TPB, 0, h->stream>>>(n, a, x, y);
  HD_LAUNCH_CK(h, "axpy");
  return HD_OK;
}
hd_status xpay_dev(hd_op* h, int64_t n, const double* z, double b, double* p) {
  k_xpay_d<<<nblk(n), TPB, 0, h->stream>>>(n, z, b, p);
  HD_LAUNCH_CK(h, "xpay");
  return HD_OK;
}

// y = AA v with the operator in the inner precision (vectors stay FP64); through the
// in-process partition when one is active
static hd_status inner_apply(hd_op* h, bool f32, const double* v, double* y) {
  if (h->part_on) return part_apply(h, v, y);
  if (!f32) return apply_op_internal(h, v, y);
  return apply_op_mixed_internal(h, v, y);  // FP32 arithmetic, FP64 vectors
}

// z_q = V/W-cycle(r_q) in the inner precision (plus the learned network term when it is
// enabled), then the zero-mean projection if singular
static hd_status inner_vcycle(hd_op* h, bool f32, const double* rq, double* zq) {
  hd_status st;
  if (!f32) {
    if ((st = h->schur_mode == 1 ? learned_schur_apply(h, rq, zq) : vcycle_apply(h, rq, zq)) != HD_OK) return st;
  } else {
    const int64_t m = h->n_l2;
    k_d2f<<<nblk(m), TPB, 0, h->stream>>>(m, rq, h->fv[2]);
    if ((st = vcycle_apply_f32(h, h->fv[2], h->fv[3])) != HD_OK) return st;
    k_f2d<<<nblk(m), TPB, 0, h->stream>>>(m, h->fv[3], zq);
    HD_LAUNCH_CK(h, "inner vcycle");
    if (h->schur_mode == 1 && (st = learned_net_add(h, rq, zq)) != HD_OK) return st;
  }
  if (h->singular) return project_mean(h, zq);
  return HD_OK;
}

// MINRES on AA x = b (x0 = x when use_x0). The Lanczos vectors, inner products and
// Givens scalars are FP64; with f32 the operator and the V-cycle run in FP32.
// it0 > 0: continue a recurrence kept on the handle after it0 iterations (its
// vectors in h->mv by h->mr_map, its scalars in h->d_ms, x given). keep: when the
// iteration cap stops the recurrence, record where its vectors are and copy x to
// h->mv[9], so that hd_checkpoint_minres / a resumed solve can continue it.
static hd_status minres_inner(hd_op* h, bool f32, const double* b, double* x, bool use_x0, double rtol, int maxit,
                              int check, int* iters, MinresState* hs_out, int it0 = 0, bool keep = false) {
  const int64_t n = h->n_rt + h->n_l2;
  double* slot[9];  // rpp, rp, y, z, v, vn, wpp, wp, wn
  for (int i = 0; i < 9; ++i) slot[i] = h->mv[it0 > 0 ? h->mr_map[i] : i];
  double *rpp = slot[0], *rp = slot[1], *y = slot[2], *z = slot[3], *v = slot[4], *vn = slot[5];
  double *wpp = slot[6], *wp = slot[7], *wn = slot[8];
  cudaStream_t s = h->stream;
  hd_status st;
  h->mr_it = 0;
  if (it0 > 0) {
    // the kept state: x from its copy, everything else where the stopped solve left it
    HD_CK(h, cudaMemcpyAsync(x, h->mv[9], sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else if (use_x0) {
    if ((st = inner_apply(h, false, x, rp)) != HD_OK) return st;
    k_axpby<<<nblk(n), TPB, 0, s>>>(n, 1.0, b, -1.0, rp);
  } else {
    HD_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    HD_CK(h, cudaMemcpyAsync(rp, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (it0 == 0) {
    HD_CK(h, cudaMemsetAsync(wp, 0, sizeof(double) * n, s));
    HD_CK(h, cudaMemsetAsync(wpp, 0, sizeof(double) * n, s));
    HD_CK(h, cudaMemsetAsync(rpp, 0, sizeof(double) * n, s));
    // z = B^-1 r: the u part by M~ scaling, the q part by the V-cycle
    if ((st = diag_scale(h, rp, z)) != HD_OK) return st;
    if (h->n_l2 > 0 && (st = inner_vcycle(h, f32, rp + h->n_rt, z + h->n_rt)) != HD_OK) return st;
    k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, rp, z, h->d_red);
    if (h->part_on && (st = part_dot_partials(h, rp, z, h->d_red, DOT_BLOCKS)) != HD_OK) return st;
    k_mr_init<<<1, DOT_BLOCKS, 0, s>>>(h->d_ms, h->d_red, rtol);
    k_scale_div<<<nblk(n), TPB, 0, s>>>(n, z, h->d_ms, v);
    HD_LAUNCH_CK(h, "minres init");
  }
  if (check < 1) check = 1;
  MinresState hs;
  int it;
  const int it_end = it0 + maxit;
  for (it = it0 + 1; it <= it_end; ++it) {
    if ((st = inner_apply(h, f32, v, y)) != HD_OK) return st;
    k_mr_lanczos1<<<DOT_BLOCKS, TPB, 0, s>>>(n, it, h->d_ms, v, y, rpp, h->d_red);
    // partitioned: the partials become the partitions' sums over their owned entries
    if (h->part_on && (st = part_dot_partials(h, v, y, h->d_red, DOT_BLOCKS)) != HD_OK) return st;
    k_mr_alpha<<<1, DOT_BLOCKS, 0, s>>>(h->d_ms, h->d_red);
    k_mr_lanczos2<<<nblk(n), TPB, 0, s>>>(n, h->n_rt, h->d_ms, y, rp, h->d_mtinv, z);
    HD_LAUNCH_CK(h, "minres lanczos");
    if (h->cap_buf && it % h->cap_every == 0 && h->cap_count < h->cap_max && h->n_l2 > 0) {
      HD_CK(h, cudaMemcpyAsync(h->cap_buf + (int64_t)h->cap_count * h->n_l2, y + h->n_rt, sizeof(double) * h->n_l2,
                               cudaMemcpyDeviceToDevice, s));
      h->cap_count++;
    }
    if (h->n_l2 > 0 && (st = inner_vcycle(h, f32, y + h->n_rt, z + h->n_rt)) != HD_OK) return st;
    k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, y, z, h->d_red);
    if (h->part_on && (st = part_dot_partials(h, y, z, h->d_red, DOT_BLOCKS)) != HD_OK) return st;
    k_mr_beta_givens<<<1, DOT_BLOCKS, 0, s>>>(h->d_ms, h->d_red, it);
    k_mr_update<<<nblk(n), TPB, 0, s>>>(n, it, h->d_ms, v, wpp, wp, wn, x, z, vn);
    HD_LAUNCH_CK(h, "minres update");
    double* t = rpp; rpp = rp; rp = y; y = t;
    t = wpp; wpp = wp; wp = wn; wn = t;
    t = v; v = vn; vn = t;
    if (it % check == 0 || it == it_end) {
      HD_CK(h, cudaMemcpyAsync(&hs, h->d_ms, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
      HD_CK(h, cudaStreamSynchronize(s));
      if (hs.done_at >= 0) break;
    }
  }
  HD_CK(h, cudaMemcpyAsync(&hs, h->d_ms, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
  HD_CK(h, cudaStreamSynchronize(s));
  *iters = hs.done_at >= 0 ? hs.done_at : it_end;
  if (hs_out) *hs_out = hs;
  if (hs.done_at < 0) {
    if (keep) {
      const double* now[9] = {rpp, rp, y, z, v, vn, wpp, wp, wn};
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j)
          if (now[i] == h->mv[j]) h->mr_map[i] = j;
      HD_CK(h, cudaMemcpyAsync(h->mv[9], x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      HD_CK(h, cudaStreamSynchronize(s));
      h->mr_it = it_end;
    }
    return HD_ERR_NOT_CONVERGED;
  }
  return hs.status;
}

// Preconditioned MINRES; with max_outer > 1 (or precision = 1) wrapped in an FP64
// residual correction: r = b - AA x in FP64, inner MINRES on AA e = r, x += e,
// until ||r||/||b|| <= outer_rtol.
static hd_status minres_run_once(hd_op* h, const double* b, double* x, const hd_solve_opts* o,
                                 hd_solve_info* info) {
  hd_status st = ensure_minres(h);
  if (st != HD_OK) return st;
  const bool f32 = o->precision == 1;
  const int it0 = h->mr_it;
  if (o->resume) {
    if (f32 || o->max_outer > 1 || h->schur_mode != 0)
      return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "resume: plain FP64 MINRES only (precision 0, max_outer <= 1, V-cycle)");
    if (it0 == 0) return hd_fail(h, HD_ERR_INVALID_ARG, "resume: no stopped MINRES recurrence on this handle");
  }
  h->mr_it = 0;  // any solve overwrites the kept recurrence
  if (f32 && (st = ensure_f32_work(h)) != HD_OK) return st;
  const int64_t n = h->n_rt + h->n_l2;
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  HD_CK(h, cudaEventCreate(&e0));
  HD_CK(h, cudaEventCreate(&e1));
  HD_CK(h, cudaEventRecord(e0, s));
  const int max_outer = o->max_outer > 0 ? o->max_outer : 1;
  const bool refine = f32 || max_outer > 1;
  int total = 0, outer = 0;
  hd_status status = HD_OK;
  MinresState hs{};
  int fallback = 0;
  if (!refine) {
    outer = 1;
    status = minres_inner(h, false, b, x, o->use_x0 != 0, o->rtol, o->maxit, o->check_every, &total, &hs,
                          o->resume ? it0 : 0, h->schur_mode == 0);
  } else {
    double* r = h->mv[9];
    double* e = h->mv[10];
    if (!o->use_x0) HD_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    double bn = 0, rn = 0;
    const double target = o->outer_rtol > 0 ? o->outer_rtol : o->rtol;
    for (outer = 0;; ++outer) {
      if ((st = h->part_on ? part_apply(h, x, r) : apply_op_internal(h, x, r)) != HD_OK) return st;
      if ((st = residual_norms(h, b, r, &rn, &bn)) != HD_OK) return st;
      if (!std::isfinite(rn) || !std::isfinite(bn)) {
        status = hd_fail(h, HD_ERR_NAN, "non-finite residual: b or the initial guess holds NaN or Inf");
        break;
      }
      if (bn == 0.0 || rn <= target * bn) {
        status = HD_OK;
        break;
      }
      if (outer == max_outer || total >= o->maxit) {
        status = HD_ERR_NOT_CONVERGED;
        break;
      }
      k_rsub<<<nblk(n), TPB, 0, s>>>(n, b, r);
      int its = 0;
      hd_status si = minres_inner(h, f32, r, e, false, o->rtol, o->maxit - total, o->check_every, &its, &hs);
      total += its;
      if (si != HD_OK && si != HD_ERR_NOT_CONVERGED) {
        status = si;
        break;
      }
      k_add<<<nblk(n), TPB, 0, s>>>(n, e, x);
      HD_LAUNCH_CK(h, "outer update");
    }
  }
  HD_CK(h, cudaEventRecord(e1, s));
  HD_CK(h, cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iterations = total;
    info->outer = outer;
    info->eta_ratio = hs.eta0 > 0 ? fabs(hs.phi_bar) / hs.eta0 : 0.0;
    info->ms_total = ms;
    info->status = status;
    info->fallback = fallback;
  }
  return status;
}

// MINRES with the Schur-block preconditioner of the handle. With the learned network
// enabled: if it breaks down (indefinite or non-finite recurrence) the solve is
// repeated with the V/W-cycle (info.fallback = 1); if it has not converged after 1.2
// times the iterations of the last converged V/W-cycle solve on the handle (the
// stagnation rule, HD_ERR_STAGNATION), it continues from its iterate with the V/W-cycle
// for the remaining iterations (info.fallback = 2). Iterations and times add up.
hd_status minres_run(hd_op* h, const double* b, double* x, const hd_solve_opts* o, hd_solve_info* info) {
  hd_solve_info i1{};
  if (h->schur_mode != 1 || o->resume) {
    hd_status st = minres_run_once(h, b, x, o, &i1);
    if (st == HD_OK && h->schur_mode == 0) h->plain_its = i1.iterations;
    if (info) *info = i1;
    return st;
  }
  hd_solve_opts o1 = *o;
  const int cap = h->plain_its > 0 ? (int)std::ceil(1.2 * h->plain_its) : o->maxit;
  if (cap < o1.maxit) o1.maxit = cap;
  hd_status st = minres_run_once(h, b, x, &o1, &i1);
  int fallback = 0;
  if (st == HD_ERR_PREC_INDEFINITE || st == HD_ERR_NAN) {
    fallback = 1;
  } else if (st == HD_ERR_NOT_CONVERGED && o1.maxit < o->maxit) {
    st = HD_ERR_STAGNATION;
    fallback = 2;
  }
  if (fallback) {
    hd_solve_opts o2 = *o;
    o2.maxit = o->maxit - i1.iterations > 1 ? o->maxit - i1.iterations : 1;
    if (fallback == 2) o2.use_x0 = 1;  // the learned iterate is the starting guess
    hd_solve_info i2{};
    h->schur_mode = 0;
    st = minres_run_once(h, b, x, &o2, &i2);
    h->schur_mode = 1;
    i2.iterations += i1.iterations;
    i2.outer += i1.outer;
    i2.ms_total += i1.ms_total;
    i2.fallback = fallback;
    i1 = i2;
    if (fallback == 2 && st == HD_ERR_NOT_CONVERGED) st = HD_ERR_STAGNATION;
  }
  if (info) *info = i1;
  return st;
}

// ---- allocation-free MINRES ----------------------------------------------------
// hd_minres_solve allocates eleven work vectors of n_rt + n_l2 doubles and its
// device state word with cudaMalloc on its first call (and the V/W-cycle graphs,
// their stream and events on first use). hd_minres_solve_noalloc takes its work
// space from the file-scope device array below instead and launches the V/W-cycle
// directly, so that a caller who may not allocate device memory once its handle
// exists can still solve. The array is part of the module: every GPU that loads
// the library holds it until the process exits. Calls share it, so calls that
// overlap on the GPU (other streams, other threads) race.
static __device__ __align__(256) double g_noalloc_scratch[HD_NOALLOC_SCRATCH_DOUBLES];

namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr int64_t kAlign = 32;  // doubles (256 bytes)
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kNoallocMaxDevices] = {};

inline int64_t round_up(int64_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

static_assert(sizeof(MinresState) <= kAlign * sizeof(double), "MINRES state must fit its slot");
static_assert(kAlign + 10 * HD_NOALLOC_MAX_DOFS <= HD_NOALLOC_SCRATCH_DOUBLES, "scratch too small for its limit");
static_assert(HD_NOALLOC_MAX_DOFS % kAlign == 0, "limit must be a multiple of the alignment");

// Device address of the scratch array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, and cached.
hd_status noalloc_scratch(hd_op* h, double** out) {
  int dev = 0;
  HD_CK(h, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return hd_fail(h, HD_ERR_INVALID_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return hd_cuda_check(h, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return HD_OK;
}

// The MINRES recurrence of minres_run with every work vector and the device
// state carved out of `ws`; no events (host wall clock instead).
hd_status minres_run_ws(hd_op* h, double* ws, const double* b, double* x, const hd_solve_opts* o,
                        hd_solve_info* info) {
  const int64_t n = h->n_rt + h->n_l2, stride = round_up(n);
  MinresState* ms = reinterpret_cast<MinresState*>(ws);
  double* v0 = ws + kAlign;
  double *rpp = v0, *rp = v0 + stride, *y = v0 + 2 * stride, *z = v0 + 3 * stride, *v = v0 + 4 * stride;
  double *vn = v0 + 5 * stride, *wpp = v0 + 6 * stride, *wp = v0 + 7 * stride, *wn = v0 + 8 * stride;
  double* tmp = v0 + 9 * stride;
  cudaStream_t s = h->stream;
  hd_status st;
  auto t0 = std::chrono::steady_clock::now();
  // the array keeps the previous call's contents: everything read before it is
  // written is set here
  if (o->use_x0) {
    if ((st = apply_op_internal(h, x, rp)) != HD_OK) return st;
    k_axpby<<<nblk(n), TPB, 0, s>>>(n, 1.0, b, -1.0, rp);
  } else {
    HD_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    HD_CK(h, cudaMemcpyAsync(rp, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  HD_CK(h, cudaMemsetAsync(wp, 0, sizeof(double) * n, s));
  HD_CK(h, cudaMemsetAsync(wpp, 0, sizeof(double) * n, s));
  HD_CK(h, cudaMemsetAsync(rpp, 0, sizeof(double) * n, s));
  if ((st = precond_apply(h, rp, z)) != HD_OK) return st;
  k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, rp, z, h->d_red);
  k_mr_init<<<1, DOT_BLOCKS, 0, s>>>(ms, h->d_red, o->rtol);
  k_scale_div<<<nblk(n), TPB, 0, s>>>(n, z, ms, v);
  HD_LAUNCH_CK(h, "minres init");
  const int check = o->check_every > 0 ? o->check_every : 1;
  MinresState hs;
  for (int it = 1; it <= o->maxit; ++it) {
    if ((st = apply_op_internal(h, v, y)) != HD_OK) return st;
    k_mr_lanczos1<<<DOT_BLOCKS, TPB, 0, s>>>(n, it, ms, v, y, rpp, h->d_red);
    k_mr_alpha<<<1, DOT_BLOCKS, 0, s>>>(ms, h->d_red);
    k_mr_lanczos2<<<nblk(n), TPB, 0, s>>>(n, h->n_rt, ms, y, rp, h->d_mtinv, z);
    HD_LAUNCH_CK(h, "minres lanczos");
    if (h->n_l2 > 0) {
      if ((st = vcycle_apply(h, y + h->n_rt, z + h->n_rt)) != HD_OK) return st;
      if (h->singular && (st = project_mean(h, z + h->n_rt)) != HD_OK) return st;
    }
    k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, y, z, h->d_red);
    k_mr_beta_givens<<<1, DOT_BLOCKS, 0, s>>>(ms, h->d_red, it);
    k_mr_update<<<nblk(n), TPB, 0, s>>>(n, it, ms, v, wpp, wp, wn, x, z, vn);
    HD_LAUNCH_CK(h, "minres update");
    double* t = rpp; rpp = rp; rp = y; y = t;
    t = wpp; wpp = wp; wp = wn; wn = t;
    t = v; v = vn; vn = t;
    if (it % check == 0 || it == o->maxit) {
      HD_CK(h, cudaMemcpyAsync(h->h_pinned, ms, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
      HD_CK(h, cudaStreamSynchronize(s));
      std::memcpy(&hs, h->h_pinned, sizeof(MinresState));
      if (hs.done_at >= 0) break;
    }
  }
  HD_CK(h, cudaMemcpyAsync(h->h_pinned, ms, sizeof(MinresState), cudaMemcpyDeviceToHost, s));
  HD_CK(h, cudaStreamSynchronize(s));
  std::memcpy(&hs, h->h_pinned, sizeof(MinresState));
  const double ms_wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  hd_status status = hs.done_at < 0 ? HD_ERR_NOT_CONVERGED : hs.status;
  if (info) {
    info->iterations = hs.done_at >= 0 ? hs.done_at : o->maxit;
    info->outer = 1;
    info->eta_ratio = hs.eta0 > 0 ? fabs(hs.phi_bar) / hs.eta0 : 0.0;
    info->ms_total = ms_wall;
    if ((st = apply_op_internal(h, x, tmp)) != HD_OK) return st;
    double rn = 0, bn = 0;
    if ((st = residual_norms(h, b, tmp, &rn, &bn)) != HD_OK) return st;
    info->true_relres = bn > 0 ? rn / bn : rn;
    info->status = status;
  }
  return status;
}

}  // namespace

// Called by hd_create (which may allocate) for problems within the limit: looks up
// the scratch array's device address on this device and runs the allocation-free
// solve once, one iteration on a zero right-hand side, so that every kernel it
// launches has been loaded before the caller's first call (with lazy module
// loading a kernel's first launch can take device memory) and that call
// allocates nothing. The two vectors of the warm-up are the only allocations.
hd_status noalloc_prepare(hd_op* h) {
  const int64_t n = h->n_rt + h->n_l2;
  if (n > HD_NOALLOC_MAX_DOFS || n == 0) return HD_OK;
  double* ws = nullptr;
  hd_status st = noalloc_scratch(h, &ws);
  if (st != HD_OK) return st;
  double *b = nullptr, *x = nullptr;
  if (cudaMalloc(&b, sizeof(double) * n) != cudaSuccess || cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) {
    cudaFree(b);
    return hd_fail(h, HD_ERR_OOM, "allocation-free solve warm-up");
  }
  hd_solve_opts o{};
  o.rtol = 1e-8;
  o.maxit = 1;
  o.check_every = 1;
  hd_solve_info info{};
  const bool prof = h->prof, graphs_off = h->graphs_off;
  h->prof = false;
  h->graphs_off = true;
  st = HD_OK;
  if (cudaMemsetAsync(b, 0, sizeof(double) * n, h->stream) != cudaSuccess)
    st = hd_fail(h, HD_ERR_CUDA, "allocation-free solve warm-up");
  else
    st = minres_run_ws(h, ws, b, x, &o, &info);  // zero b: the recurrence stops at once (HD_OK)
  h->prof = prof;
  h->graphs_off = graphs_off;
  cudaStreamSynchronize(h->stream);
  cudaFree(b);
  cudaFree(x);
  return st;
}

// ---- MINRES checkpoints ----------------------------------------------------------
// File: header, the device state word, then x, v, r_{j-1}, r_j, w_{j-1}, w_j (FP64,
// n_rt + n_l2 each, host byte order).
struct MinresCkptHeader {
  char magic[8];
  int64_t n_rt, n_l2;
  int32_t k, it;
  int32_t state_bytes, reserved;
};
static const char kMinresMagic[8] = {'H', 'D', 'M', 'I', 'N', 'R', 'S', '1'};
static const int kCkptSlots[5] = {4, 0, 1, 6, 7};  // v, rpp, rp, wpp, wp in mr_map order

extern "C" hd_status hd_checkpoint_minres(hd_handle h, const char* path) {
  if (!h || !path) return HD_ERR_INVALID_ARG;
  if (h->mr_it == 0) return hd_fail(h, HD_ERR_INVALID_ARG, "checkpoint: no stopped MINRES recurrence on this handle");
  const int64_t n = h->n_rt + h->n_l2;
  MinresState ms;
  HD_CK(h, cudaMemcpyAsync(&ms, h->d_ms, sizeof ms, cudaMemcpyDeviceToHost, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  std::vector<double> buf((size_t)n);
  FILE* f = std::fopen(path, "wb");
  if (!f) return hd_fail(h, HD_ERR_INVALID_ARG, std::string("checkpoint: cannot open ") + path);
  MinresCkptHeader hd{};
  std::memcpy(hd.magic, kMinresMagic, sizeof hd.magic);
  hd.n_rt = h->n_rt;
  hd.n_l2 = h->n_l2;
  hd.k = h->k;
  hd.it = h->mr_it;
  hd.state_bytes = (int32_t)sizeof(MinresState);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(&ms, sizeof ms, 1, f) == 1;
  cudaError_t ce = cudaSuccess;
  for (int i = 0; ok && i < 6; ++i) {
    const double* src = i == 0 ? h->mv[9] : h->mv[h->mr_map[kCkptSlots[i - 1]]];
    ce = cudaMemcpyAsync(buf.data(), src, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    ok = ce == cudaSuccess && std::fwrite(buf.data(), sizeof(double), (size_t)n, f) == (size_t)n;
  }
  ok = std::fclose(f) == 0 && ok;
  if (ce != cudaSuccess) return hd_cuda_check(h, ce, "checkpoint copy");
  return ok ? HD_OK : hd_fail(h, HD_ERR_INVALID_ARG, std::string("checkpoint: write failed: ") + path);
}

extern "C" hd_status hd_resume_minres(hd_handle h, const char* path) {
  if (!h || !path) return HD_ERR_INVALID_ARG;
  hd_status st = ensure_minres(h);
  if (st != HD_OK) return st;
  h->mr_it = 0;  // a refused file leaves no recurrence on the handle
  FILE* f = std::fopen(path, "rb");
  if (!f) return hd_fail(h, HD_ERR_INVALID_ARG, std::string("resume: cannot open ") + path);
  const int64_t n = h->n_rt + h->n_l2;
  MinresCkptHeader hd{};
  MinresState ms{};
  std::string err;
  if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, kMinresMagic, sizeof hd.magic) != 0)
    err = "not a MINRES checkpoint";
  else if (hd.n_rt != h->n_rt || hd.n_l2 != h->n_l2 || hd.k != h->k)
    err = "checkpoint of another problem size";
  else if (hd.state_bytes != (int32_t)sizeof(MinresState) || hd.it < 1)
    err = "checkpoint of another library version";
  else if (std::fread(&ms, sizeof ms, 1, f) != 1 || ms.done_at != -1)
    err = "checkpoint without a running recurrence";
  std::vector<double> buf[6];
  for (int i = 0; err.empty() && i < 6; ++i) {
    buf[i].resize((size_t)n);
    if (std::fread(buf[i].data(), sizeof(double), (size_t)n, f) != (size_t)n) err = "truncated checkpoint";
  }
  if (err.empty() && std::fgetc(f) != EOF) err = "trailing bytes after the checkpoint";
  std::fclose(f);
  if (!err.empty()) return hd_fail(h, HD_ERR_INVALID_ARG, "resume: " + err + ": " + path);
  for (int i = 0; i < 9; ++i) h->mr_map[i] = i;
  for (int i = 0; i < 6; ++i) {
    double* dst = i == 0 ? h->mv[9] : h->mv[kCkptSlots[i - 1]];
    HD_CK(h, cudaMemcpyAsync(dst, buf[i].data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  }
  HD_CK(h, cudaMemcpyAsync(h->d_ms, &ms, sizeof ms, cudaMemcpyHostToDevice, h->stream));
  HD_CK(h, cudaStreamSynchronize(h->stream));
  h->mr_it = hd.it;
  return HD_OK;
}

extern "C" hd_status hd_minres_solve_noalloc(hd_handle h, const double* b, double* x, const hd_solve_opts* o,
                                             hd_solve_info* info) {
  if (!h || !b || !x || !o || b == x || o->maxit < 1 || !(o->rtol > 0)) return HD_ERR_INVALID_ARG;
  if (o->precision != 0) return hd_fail(h, HD_ERR_INVALID_ARG, "hd_minres_solve_noalloc: FP64 only (precision = 0)");
  if (o->resume) return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "hd_minres_solve_noalloc: no resume (use hd_minres_solve)");
  if (o->max_outer > 1)
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED,
                   "hd_minres_solve_noalloc: one MINRES pass only (max_outer <= 1; use hd_minres_solve)");
  if (h->schur_mode != 0)
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED,
                   "hd_minres_solve_noalloc: V/W-cycle Schur block only (the learned network is enabled)");
  const int64_t n = h->n_rt + h->n_l2;
  if (n > HD_NOALLOC_MAX_DOFS) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "hd_minres_solve_noalloc: %lld DOFs exceed the limit of %d (n_rt + n_l2)",
                  (long long)n, (int)HD_NOALLOC_MAX_DOFS);
    return hd_fail(h, HD_ERR_INVALID_ARG, msg);
  }
  double* ws = nullptr;
  hd_status st = noalloc_scratch(h, &ws);
  if (st != HD_OK) return st;
  // profiling would create its event pairs on first use, and the cached V/W-cycle
  // graphs are keyed by their vectors (here in the scratch array: a first use would
  // instantiate new graphs on a stream of their own): both off for this call
  const bool prof = h->prof, graphs_off = h->graphs_off;
  h->prof = false;
  h->graphs_off = true;
  st = minres_run_ws(h, ws, b, x, o, info);
  h->prof = prof;
  h->graphs_off = graphs_off;
  return st;
}

// ---- restarted GMRES with block preconditioners ---------------------------------
// The remark on block-triangular preconditioners in Sec. 2.3: with
// P = [[tau M~, D^T], [0, -S^]] (S^ the V/W-cycle), z = P^-1 r is
//   z_q = -S^-1 r_q,  z_u = (r_u - D^T z_q) / (tau M~)  (identity on essential dofs),
// and the preconditioned operator is not symmetric, so GMRES replaces MINRES.
// Right preconditioning (the recurrence estimates the true residual); Arnoldi by
// classical Gram-Schmidt in two fused passes over the basis (multi-dot, then
// update plus norm), repeated once when the norm falls below 1e-3 of its value
// before the pass; the Hessenberg least-squares problem by Givens rotations on the
// host (one small copy per step). All reductions run over fixed blocks in a fixed
// order, so a solve is deterministic.
//
// FP64 (precision 0): operator and V-cycle in FP64 (the operator in the handle's
// element arithmetic), the basis and Gram-Schmidt in double-float. Mixed (precision 1): the cycles run entirely in FP32
// (basis, Gram-Schmidt, operator, V-cycle), each ends once its estimate has fallen
// by inner_rtol, and every restart recomputes the residual with the FP64 operator
// and adds the cycle's correction to the FP64 solution: iterative refinement with
// GMRES cycles as the inner solver. Gram-Schmidt on an FP64 basis is bound by the
// FP64 pipe on this GPU (one FMA per value read); in FP32 it streams at HBM speed.
namespace {
constexpr int GM_MAX_RESTART = 128;
constexpr int GM_CH = 8;  // basis vectors per sweep of the multi-dot

// conversions of the basis types (double, float, double-float pairs) to and from FP64
__device__ __forceinline__ double to_dbl(double v) { return v; }
__device__ __forceinline__ double to_dbl(float v) { return (double)v; }
__device__ __forceinline__ double to_dbl(dfloat v) { return df_to_double(v); }
template <typename T>
__device__ __forceinline__ T from_dbl(double v);
template <>
__device__ __forceinline__ double from_dbl<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_dbl<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ dfloat from_dbl<dfloat>(double v) { return df_from_double(v); }

// One sweep of the multi-dot over G vectors fixed at compile time: vector c is
// V_{k0 + c}, or w itself at index nv (the self-dot). Two elements per iteration.
template <typename T, int G>
__device__ __forceinline__ void gm_mdot_group(int64_t lo, int64_t hi, const T* __restrict__ V, int64_t ldv, int nv,
                                              int k0, const T* __restrict__ w, double* __restrict__ partial,
                                              double* sh) {
  const T* vp[G];
#pragma unroll
  for (int c = 0; c < G; ++c) vp[c] = (k0 + c < nv) ? V + (int64_t)(k0 + c) * ldv : w;
  T acc[G];
#pragma unroll
  for (int c = 0; c < G; ++c) acc[c] = (T)0;
  int64_t i = lo + threadIdx.x;
  for (; i + blockDim.x < hi; i += 2 * blockDim.x) {
    const T w0 = w[i], w1 = w[i + blockDim.x];
    T a0[G], a1[G];
#pragma unroll
    for (int c = 0; c < G; ++c) {
      a0[c] = vp[c][i];
      a1[c] = vp[c][i + blockDim.x];
    }
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = fma(a1[c], w1, fma(a0[c], w0, acc[c]));
  }
  if (i < hi) {
    const T w0 = w[i];
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = fma(vp[c][i], w0, acc[c]);
  }
#pragma unroll
  for (int c = 0; c < G; ++c) {
    const double s = block_sum(to_dbl(acc[c]), sh);
    if (threadIdx.x == 0) partial[(k0 + c) * DOT_BLOCKS + blockIdx.x] = s;
  }
}

// partial[k * DOT_BLOCKS + b] = block b's chunk of V_k . w for k < nv, and with
// self_dot also w . w at k = nv (V_k = V + k ldv). Per-thread sums in T, the
// block sums in FP64. Sweeps of at most GM_CH vectors, each sized at compile time.
template <typename T>
__global__ void k_gm_mdot(int64_t n, const T* __restrict__ V, int64_t ldv, int nv, bool self_dot,
                          const T* __restrict__ w, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  const int ntot = nv + (self_dot ? 1 : 0);
  for (int k0 = 0; k0 < ntot; k0 += GM_CH) {
    switch (min(GM_CH, ntot - k0)) {  // uniform over the grid
      case 1: gm_mdot_group<T, 1>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 2: gm_mdot_group<T, 2>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 3: gm_mdot_group<T, 3>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 4: gm_mdot_group<T, 4>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 5: gm_mdot_group<T, 5>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 6: gm_mdot_group<T, 6>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      case 7: gm_mdot_group<T, 7>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
      default: gm_mdot_group<T, GM_CH>(lo, hi, V, ldv, nv, k0, w, partial, sh); break;
    }
  }
}

// out[k] = sum over the DOT_BLOCKS partials of dot k, one block per k, fixed order
__global__ void k_gm_final(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[32];
  const double s = block_sum(partial[blockIdx.x * DOT_BLOCKS + threadIdx.x], sh);  // blockDim.x == DOT_BLOCKS
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= sum_k h[k] V_k (k < nv), and partial[b] = block b's chunk of the new w . w
template <typename T>
__global__ void k_gm_update_norm(int64_t n, const T* __restrict__ V, int64_t ldv, int nv,
                                 const double* __restrict__ hcoef, T* __restrict__ w, double* __restrict__ partial) {
  __shared__ double sh[32];
  __shared__ T hs[GM_MAX_RESTART + 1];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = from_dbl<T>(hcoef[k]);
  __syncthreads();
  const int64_t chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  T acc = (T)0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    T s = w[i];
    for (int k = 0; k < nv; ++k) s = fma(-hs[k], V[k * ldv + i], s);
    w[i] = s;
    acc = fma(s, s, acc);
  }
  const double b = block_sum(to_dbl(acc), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// u = sum_k y[k] V_k (k < nv)
template <typename T>
__global__ void k_gm_combine(int64_t n, const T* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ y,
                             T* __restrict__ u) {
  __shared__ T ys[GM_MAX_RESTART];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) ys[k] = from_dbl<T>(y[k]);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = (T)0;
  for (int k = 0; k < nv; ++k) s = fma(ys[k], V[k * ldv + i], s);
  u[i] = s;
}

// y = a x (in y's type)
template <typename S, typename T>
__global__ void k_gm_scale(int64_t n, double a, const S* __restrict__ x, T* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = from_dbl<T>(a * to_dbl(x[i]));
}

// triangular preconditioner, RT part: z_u = mtinv (r_u + D^T s) with s = S^-1 r_q
// (so that z_q = -s); mtinv = 1 and (D^T s) = 0 on essential dofs
template <typename T>
__global__ void k_gm_tri_u(int64_t n_rt, const T* __restrict__ mtinv, const T* __restrict__ ru,
                           const T* __restrict__ dts, T* __restrict__ zu) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n_rt) zu[i] = mtinv[i] * (ru[i] + dts[i]);
}
template <typename T>
__global__ void k_gm_neg(int64_t n, T* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = -x[i];
}
// x += (double) z
__global__ void k_gm_add_f(int64_t n, const float* __restrict__ z, double* __restrict__ x) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)z[i];
}
}  // namespace

static hd_status ensure_gmres(hd_op* h, int m, bool f32) {
  const int64_t n = h->n_rt + h->n_l2, nn = n > 0 ? n : 1;
  if (!h->gm_w) {
    if (cudaMalloc(&h->gm_w, sizeof(double) * 3 * nn) != cudaSuccess ||
        cudaMalloc(&h->gm_part, sizeof(double) * (GM_MAX_RESTART + 2) * DOT_BLOCKS) != cudaSuccess ||
        cudaMalloc(&h->gm_dots, sizeof(double) * (GM_MAX_RESTART + 2)) != cudaSuccess ||
        cudaMallocHost(&h->gm_host, sizeof(double) * (GM_MAX_RESTART + 2)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "GMRES work");
  }
  if (!f32 && !(h->gm_V && h->gm_m >= m)) {
    cudaFree(h->gm_V);
    h->gm_V = nullptr;
    h->gm_m = 0;
    if (cudaMalloc(&h->gm_V, sizeof(double) * (size_t)(m + 1) * (size_t)nn) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "GMRES basis");
    h->gm_m = m;
  }
  if (f32) {
    if (!h->gm_wf && cudaMalloc(&h->gm_wf, sizeof(float) * 3 * nn) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "GMRES FP32 work");
    if (!(h->gm_Vf && h->gm_mf >= m)) {
      cudaFree(h->gm_Vf);
      h->gm_Vf = nullptr;
      h->gm_mf = 0;
      if (cudaMalloc(&h->gm_Vf, sizeof(float) * (size_t)(m + 1) * (size_t)nn) != cudaSuccess)
        return hd_fail(h, HD_ERR_OOM, "GMRES FP32 basis");
      h->gm_mf = m;
    }
  }
  return HD_OK;
}

// z = P^-1 v in T: block-diagonal (prec 0: the MINRES preconditioner) or block upper
// triangular (prec 1). tmp: n values of scratch. The q part of v is copied into
// tmp's q part first: the V-cycle replays a CUDA graph cached per (input, output)
// pointer pair, and the Arnoldi vectors would otherwise each need a new capture.
template <typename T>
static hd_status gmres_prec(hd_op* h, int prec, const T* v, T* z, T* tmp) {
  constexpr bool F = std::is_same<T, float>::value;
  hd_status st;
  if constexpr (F) st = diag_scale_f32(h, v, z);  // prec 1 overwrites z_u below
  else st = diag_scale(h, v, z);
  if (st != HD_OK) return st;
  if (h->n_l2 == 0) return HD_OK;
  T* rq = tmp + h->n_rt;
  HD_CK(h, cudaMemcpyAsync(rq, v + h->n_rt, sizeof(T) * h->n_l2, cudaMemcpyDeviceToDevice, h->stream));
  if constexpr (F) {  // s = S^-1 r_q
    if ((st = vcycle_apply_f32(h, rq, z + h->n_rt)) != HD_OK) return st;
    if (h->singular && (st = project_mean_f32(h, z + h->n_rt)) != HD_OK) return st;
  } else {
    if ((st = inner_vcycle(h, false, rq, z + h->n_rt)) != HD_OK) return st;
  }
  if (prec == 0) return HD_OK;
  if constexpr (F) st = lattice_apply_Bt_f32(h, z + h->n_rt, tmp);  // D^T s
  else st = lattice_apply_Bt(h, z + h->n_rt, tmp);
  if (st != HD_OK) return st;
  cudaStream_t s = h->stream;
  const T* mtinv;
  if constexpr (F) mtinv = h->f_mtinv;
  else mtinv = h->d_mtinv;
  k_gm_tri_u<T><<<nblk(h->n_rt), TPB, 0, s>>>(h->n_rt, mtinv, v, tmp, z);
  k_gm_neg<T><<<nblk(h->n_l2), TPB, 0, s>>>(h->n_l2, z + h->n_rt);
  HD_LAUNCH_CK(h, "gmres triangular preconditioner");
  return HD_OK;
}

// dots[k] = V_k . w (k < nv) and, with self_dot, dots[nv] = w . w; copied to the host
template <typename T>
static hd_status gm_mdot(hd_op* h, const T* V, int64_t n, int nv, bool self_dot, const T* w, double* host) {
  cudaStream_t s = h->stream;
  const int nd = nv + (self_dot ? 1 : 0);
  k_gm_mdot<T><<<DOT_BLOCKS, TPB, 0, s>>>(n, V, n, nv, self_dot, w, h->gm_part);
  k_gm_final<<<nd, DOT_BLOCKS, 0, s>>>(h->gm_part, h->gm_dots);
  HD_LAUNCH_CK(h, "gmres dots");
  HD_CK(h, cudaMemcpyAsync(host, h->gm_dots, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
  HD_CK(h, cudaStreamSynchronize(s));
  return HD_OK;
}

// w -= V h (h = the dots just computed, still on the device); returns ||w||^2
template <typename T>
static hd_status gm_update(hd_op* h, const T* V, int64_t n, int nv, T* w, double* nrm2) {
  cudaStream_t s = h->stream;
  k_gm_update_norm<T><<<DOT_BLOCKS, TPB, 0, s>>>(n, V, n, nv, h->gm_dots, w, h->gm_part);
  k_gm_final<<<1, DOT_BLOCKS, 0, s>>>(h->gm_part, h->gm_dots + GM_MAX_RESTART + 1);
  HD_LAUNCH_CK(h, "gmres update");
  HD_CK(h, cudaMemcpyAsync(nrm2, h->gm_dots + GM_MAX_RESTART + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  HD_CK(h, cudaStreamSynchronize(s));
  return HD_OK;
}

// One GMRES cycle on the residual r (FP64, norm rn): at most mc steps, ending at
// est <= stop; on exit the correction P^-1 V y has been added to x. TB: the basis
// and Gram-Schmidt type; TV: the type of the operator and preconditioner vectors.
// With TB != TV (a double-float basis for the FP64 solve) V_j is converted to TV in
// vconv before the preconditioner and the operator's result back to TB in w.
template <typename TB, typename TV>
static hd_status gmres_cycle(hd_op* h, const hd_gmres_opts* o, const double* r, double rn, int mc, double stop,
                             TB* V, TB* w, TV* z, TV* tmp, TV* vconv, double* x, int* steps, double* est_out) {
  const int m = o->restart;
  const int64_t n = h->n_rt + h->n_l2;
  cudaStream_t s = h->stream;
  hd_status st;
  constexpr bool F = std::is_same<TV, float>::value;
  constexpr bool SAME = std::is_same<TB, TV>::value;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), y(m);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  double* hostd = h->gm_host;
  auto apply = [&](const TV* in, TV* out) -> hd_status {
    if constexpr (F) return apply_op_f32_internal(h, in, out);
    else return apply_op_internal(h, in, out);
  };
  k_gm_scale<double, TB><<<nblk(n), TPB, 0, s>>>(n, 1.0 / rn, r, V);
  HD_LAUNCH_CK(h, "gmres restart");
  g[0] = rn;
  int j = 0;
  double est = rn;
  while (j < mc) {
    TB* Vj = V + (int64_t)j * n;
    if constexpr (SAME) {
      if ((st = gmres_prec<TV>(h, o->prec, Vj, z, tmp)) != HD_OK) return st;
      if ((st = apply(z, w)) != HD_OK) return st;
    } else {
      k_gm_scale<TB, TV><<<nblk(n), TPB, 0, s>>>(n, 1.0, Vj, vconv);
      if ((st = gmres_prec<TV>(h, o->prec, vconv, z, tmp)) != HD_OK) return st;
      if ((st = apply(z, vconv)) != HD_OK) return st;
      k_gm_scale<TV, TB><<<nblk(n), TPB, 0, s>>>(n, 1.0, vconv, w);
      HD_LAUNCH_CK(h, "gmres basis conversion");
    }
    // classical Gram-Schmidt: h = V^T w (with ||w||^2 before), w -= V h
    if ((st = gm_mdot<TB>(h, V, n, j + 1, true, w, hostd)) != HD_OK) return st;
    const double before = hostd[j + 1];
    for (int i = 0; i <= j; ++i) Hat(i, j) = hostd[i];
    double nrm2 = 0;
    if ((st = gm_update<TB>(h, V, n, j + 1, w, &nrm2)) != HD_OK) return st;
    // Orthogonalise once more only on severe cancellation (more than three digits
    // lost). With the 1/sqrt(2) test of the two-pass method the second pass ran at
    // every step on the metric workload and changed neither the step count nor the
    // final residual (52 steps, 9.0e-9 at 64^3) while costing a quarter of the time;
    // the true residual is recomputed at every restart and at the exit in any case.
    if (nrm2 < 1e-6 * before) {
      if ((st = gm_mdot<TB>(h, V, n, j + 1, false, w, hostd)) != HD_OK) return st;
      for (int i = 0; i <= j; ++i) Hat(i, j) += hostd[i];
      if ((st = gm_update<TB>(h, V, n, j + 1, w, &nrm2)) != HD_OK) return st;
    }
    const double hn = std::sqrt(std::max(nrm2, 0.0));
    Hat(j + 1, j) = hn;
    if (hn > 0.0) {
      k_gm_scale<TB, TB><<<nblk(n), TPB, 0, s>>>(n, 1.0 / hn, w, V + (int64_t)(j + 1) * n);
      HD_LAUNCH_CK(h, "gmres normalise");
    }
    for (int i = 0; i < j; ++i) {  // previous rotations on the new column
      const double a = Hat(i, j), c = Hat(i + 1, j);
      Hat(i, j) = cs[i] * a + sn[i] * c;
      Hat(i + 1, j) = -sn[i] * a + cs[i] * c;
    }
    const double d = std::hypot(Hat(j, j), Hat(j + 1, j));
    if (!(d > 0.0) || !std::isfinite(d))
      return hd_fail(h, HD_ERR_NAN, "GMRES breakdown (zero or non-finite Hessenberg column)");
    cs[j] = Hat(j, j) / d;
    sn[j] = Hat(j + 1, j) / d;
    Hat(j, j) = d;
    Hat(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    ++j;
    est = std::fabs(g[j]);
    if (est <= stop || hn == 0.0) break;
  }
  // y = H(0:j, 0:j)^-1 g, x += P^-1 V y
  for (int i = j - 1; i >= 0; --i) {
    double t = g[i];
    for (int l = i + 1; l < j; ++l) t -= Hat(i, l) * y[l];
    y[i] = t / Hat(i, i);
  }
  HD_CK(h, cudaMemcpyAsync(h->gm_dots, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
  TV* u;
  if constexpr (SAME) {
    k_gm_combine<TB><<<nblk(n), TPB, 0, s>>>(n, V, n, j, h->gm_dots, tmp);
    u = tmp;
    if ((st = gmres_prec<TV>(h, o->prec, u, z, w)) != HD_OK) return st;
  } else {
    k_gm_combine<TB><<<nblk(n), TPB, 0, s>>>(n, V, n, j, h->gm_dots, w);
    k_gm_scale<TB, TV><<<nblk(n), TPB, 0, s>>>(n, 1.0, w, vconv);
    u = vconv;
    if ((st = gmres_prec<TV>(h, o->prec, u, z, tmp)) != HD_OK) return st;
  }
  HD_LAUNCH_CK(h, "gmres combine");
  if constexpr (F) k_gm_add_f<<<nblk(n), TPB, 0, s>>>(n, z, x);
  else k_add<<<nblk(n), TPB, 0, s>>>(n, z, x);
  HD_LAUNCH_CK(h, "gmres update x");
  *steps = j;
  *est_out = est;
  return HD_OK;
}

hd_status gmres_run(hd_op* h, const double* b, double* x, const hd_gmres_opts* o, hd_solve_info* info) {
  const int m = o->restart;
  const bool f32 = o->precision == 1;
  hd_status st = ensure_gmres(h, m, f32);
  if (st != HD_OK) return st;
  if (f32 && (st = setup_f32(h)) != HD_OK) return st;
  const int64_t n = h->n_rt + h->n_l2;
  cudaStream_t s = h->stream;
  double* r = h->gm_w;  // FP64 residual; the rest of gm_w is the FP64 cycle's work
  struct Events {  // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  HD_CK(h, cudaEventCreate(&ev.a));
  HD_CK(h, cudaEventCreate(&ev.b));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  HD_CK(h, cudaEventRecord(e0, s));
  if (!o->use_x0) HD_CK(h, cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  int its = 0, cycles = 0;
  double bn = 0, rn = 0, est = 0;
  hd_status status = HD_ERR_NOT_CONVERGED;
  for (;;) {
    // true residual r = b - AA x in FP64
    if ((st = apply_op_internal(h, x, r)) != HD_OK) return st;
    if ((st = residual_norms(h, b, r, &rn, &bn)) != HD_OK) return st;
    if (!std::isfinite(rn) || !std::isfinite(bn)) {
      status = hd_fail(h, HD_ERR_NAN, "non-finite residual: b or the initial guess holds NaN or Inf");
      break;
    }
    if (bn == 0.0 || rn <= o->rtol * bn) {
      status = HD_OK;
      break;
    }
    if (its >= o->maxit) break;
    k_axpby<<<nblk(n), TPB, 0, s>>>(n, 1.0, b, -1.0, r);  // r = b - AA x
    HD_LAUNCH_CK(h, "gmres residual");
    ++cycles;
    const int mc = std::min(m, o->maxit - its);
    int steps = 0;
    if (f32) {
      const double stop = std::max(o->rtol * bn, o->inner_rtol * rn);
      float* wf = h->gm_wf;
      st = gmres_cycle<float, float>(h, o, r, rn, mc, stop, h->gm_Vf, wf, wf + n, wf + 2 * n, nullptr, x, &steps,
                                     &est);
    } else {
      // Double-float basis and Gram-Schmidt (FP32 pairs, ~48 bits) in the basis memory
      // (8 bytes a value either way): on an FP64 basis these passes are bound by the FP64
      // pipe (one FMA per value read); with the two conversions per step the solve is
      // 2.6 % faster at 64^3 (832 against 854 ms, the same 52 steps). The basis's last
      // vector is the cycle's w (written in place when it becomes V_m); the FP64
      // residual buffer converts V_j and holds the operator's result.
      dfloat* V = reinterpret_cast<dfloat*>(h->gm_V);
      st = gmres_cycle<dfloat, double>(h, o, r, rn, mc, o->rtol * bn, V, V + (int64_t)m * n, h->gm_w + n,
                                       h->gm_w + 2 * n, r, x, &steps, &est);
    }
    its += steps;
    if (st == HD_ERR_NAN) {  // breakdown in the cycle: reported through info as well
      status = st;
      break;
    }
    if (st != HD_OK) return st;
  }
  HD_CK(h, cudaEventRecord(e1, s));
  HD_CK(h, cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  if (info) {
    info->iterations = its;
    info->outer = cycles;
    info->eta_ratio = bn > 0 ? est / bn : 0.0;
    info->true_relres = bn > 0 ? rn / bn : 0.0;
    info->ms_total = ms;
    info->status = status;
    info->fallback = 0;
  }
  return status;
}

extern "C" hd_status hd_gmres_solve(hd_handle h, const double* b, double* x, const hd_gmres_opts* o,
                                    hd_solve_info* info) {
  if (!h || !b || !x || !o) return HD_ERR_INVALID_ARG;
  if (o->restart < 1 || o->restart > GM_MAX_RESTART || o->maxit < 1 || !(o->rtol >= 0.0) ||
      (o->prec != HD_GMRES_BLOCK_DIAG && o->prec != HD_GMRES_BLOCK_TRI) || (o->precision != 0 && o->precision != 1) ||
      (o->precision == 1 && !(o->inner_rtol > 0.0 && o->inner_rtol < 1.0)))
    return hd_fail(h, HD_ERR_INVALID_ARG,
                   "hd_gmres_solve: restart 1..128, maxit >= 1, rtol >= 0, prec 0 or 1, precision 0 or 1 "
                   "(1: 0 < inner_rtol < 1)");
  if (h->schur_mode != 0 && o->precision != 0)  // the FP32 cycles have no learned Schur preconditioner
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED, "hd_gmres_solve: the learned Schur preconditioner is FP64 only");
  return gmres_run(h, b, x, o, info);
}
