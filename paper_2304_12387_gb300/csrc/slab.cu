// Z-slab partition of the element lattice (the paper runs its solvers on up to 256
// GPUs, Sec. 4.2; every call of this library runs on one).
//
// Partition p of P owns the element layers [ez0, ez1) (balanced: ez0 = floor(p nz / P)),
// hence the contiguous id ranges of the x-faces, y-faces and cells with lattice layer
// K in [k ez0, k ez1) and of the z-faces with K in [k ez0, k ez1) (the last partition
// also owns the top boundary layer K = Z). The z-faces of layer K = k ez1 (the upper
// interface, owned by p + 1) are p's halo: its top element layer reads them and adds
// to them. One apply of the block operator then needs two exchanges per interface,
// each of X Y values: the halo values of x from p + 1 to p before the element loop,
// and p's partial sums on the halo faces from p to p + 1 after it (each interface face
// gets exactly two addends, one per side, so the result does not depend on the
// partition). A MINRES iteration adds one reduction of two scalars per partition.
//
// hd_apply_op_partitioned and hd_minres_solve_partitioned emulate P partitions in one
// process on one GPU: every partition has its own full-length buffers, filled with
// NaN outside its owned and halo entries, so that a read outside them shows in the
// result; the exchanges are device copies and an add kernel; dot products are summed
// per partition over its owned ranges and the P sums then in a fixed order (the
// allreduce). The Schur V/W-cycle acts on the gathered L2 vector (on P GPUs: a gather
// of the L2 residual to one rank and a scatter back, the coarse gather taken at the
// finest level).
#include <cstring>
#include <vector>

#include "hd_internal.h"

namespace {

constexpr int TPB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }
constexpr int PART_BLOCKS = 64;  // partial-sum blocks per partition

void plan(const LatticeDims& L, int k, int P, int p, hd_slab* s) {
  const int64_t X = L.X, Y = L.Y, Z = L.Z, XY = X * Y;
  const int64_t sx = (X + 1) * Y, sy = X * (Y + 1);
  const int64_t oy = (int64_t)L.n_xf, oz = (int64_t)L.n_xf + L.n_yf, oq = oz + XY * (Z + 1);
  s->p = p;
  s->P = P;
  s->ez0 = (int32_t)((int64_t)p * L.nz / P);
  s->ez1 = (int32_t)((int64_t)(p + 1) * L.nz / P);
  const int64_t Z0 = (int64_t)s->ez0 * k, Z1 = (int64_t)s->ez1 * k;
  s->xf[0] = sx * Z0;
  s->xf[1] = sx * Z1;
  s->yf[0] = oy + sy * Z0;
  s->yf[1] = oy + sy * Z1;
  s->zf[0] = oz + XY * Z0;
  s->zf[1] = oz + XY * (p == P - 1 ? Z + 1 : Z1);
  s->cell[0] = oq + XY * Z0;
  s->cell[1] = oq + XY * Z1;
  s->halo[0] = p == P - 1 ? 0 : oz + XY * Z1;
  s->halo[1] = p == P - 1 ? 0 : oz + XY * (Z1 + 1);
}

__global__ void k_add_range(int64_t n, const double* __restrict__ src, double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] += src[i];
}

// partial[p * PART_BLOCKS + j] = sum of a_i b_i over chunk j of partition p's owned ranges
// (ranges: P x 4 half-open id ranges)
__global__ void k_part_partial(int P, const int64_t* __restrict__ ranges, const double* __restrict__ a,
                               const double* __restrict__ b, double* __restrict__ partial) {
  __shared__ double sh[TPB / 32];
  const int p = blockIdx.x / PART_BLOCKS, j = blockIdx.x % PART_BLOCKS;
  const int64_t* r = ranges + (int64_t)p * 8;
  const int64_t len = (r[1] - r[0]) + (r[3] - r[2]) + (r[5] - r[4]) + (r[7] - r[6]);
  const int64_t chunk = (len + PART_BLOCKS - 1) / PART_BLOCKS, lo = j * chunk, hi = min(len, lo + chunk);
  double s = 0.0;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    int64_t u = t, g = 0;
    for (int q = 0; q < 4; ++q) {
      const int64_t l = r[2 * q + 1] - r[2 * q];
      if (u < l) {
        g = r[2 * q] + u;
        break;
      }
      u -= l;
    }
    s = fma(a[g], b[g], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TPB / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// out[p] = sum_j partial[p][j] in order (partition p's sum); out[P..nout) = 0
__global__ void k_part_final(int P, const double* __restrict__ partial, double* __restrict__ out, int nout) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nout) return;
  double s = 0.0;
  if (p < P)
    for (int j = 0; j < PART_BLOCKS; ++j) s += partial[p * PART_BLOCKS + j];
  out[p] = s;
}

}  // namespace

struct PartState {
  int P = 0;
  std::vector<hd_slab> slab;
  int64_t* d_ranges = nullptr;  // P x 8
  double* d_partial = nullptr;  // P x PART_BLOCKS
  std::vector<double*> xb, yb;  // per-partition full-length buffers
};

void part_free(hd_op* h) {
  PartState* s = h->part;
  if (!s) return;
  cudaFree(s->d_ranges);
  cudaFree(s->d_partial);
  for (double* p : s->xb) cudaFree(p);
  for (double* p : s->yb) cudaFree(p);
  delete s;
  h->part = nullptr;
}

static hd_status part_setup(hd_op* h, int P) {
  if (h->part && h->part->P == P) return HD_OK;
  part_free(h);
  if (P < 2 || P > h->L.nz) return hd_fail(h, HD_ERR_INVALID_ARG, "partitions: 2 <= P <= nz");
  PartState* s = new (std::nothrow) PartState();
  if (!s) return hd_fail(h, HD_ERR_OOM, "partition state");
  h->part = s;
  s->P = P;
  s->slab.resize(P);
  std::vector<int64_t> r((size_t)P * 8);
  for (int p = 0; p < P; ++p) {
    plan(h->L, h->k, P, p, &s->slab[p]);
    const hd_slab& q = s->slab[p];
    const int64_t v[8] = {q.xf[0], q.xf[1], q.yf[0], q.yf[1], q.zf[0], q.zf[1], q.cell[0], q.cell[1]};
    std::memcpy(&r[(size_t)p * 8], v, sizeof v);
  }
  const int64_t n = h->n_rt + h->n_l2;
  if (cudaMalloc(&s->d_ranges, sizeof(int64_t) * r.size()) != cudaSuccess ||
      cudaMalloc(&s->d_partial, sizeof(double) * P * PART_BLOCKS) != cudaSuccess)
    return hd_fail(h, HD_ERR_OOM, "partition state");
  HD_CK(h, cudaMemcpy(s->d_ranges, r.data(), sizeof(int64_t) * r.size(), cudaMemcpyHostToDevice));
  s->xb.assign(P, nullptr);
  s->yb.assign(P, nullptr);
  for (int p = 0; p < P; ++p)
    if (cudaMalloc(&s->xb[p], sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&s->yb[p], sizeof(double) * n) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "partition buffers");
  return HD_OK;
}

// y = AA x through P emulated partitions (h->part set up)
hd_status part_apply(hd_op* h, const double* x, double* y) {
  PartState* s = h->part;
  const int P = s->P;
  const int64_t n = h->n_rt + h->n_l2, E2 = (int64_t)h->L.nx * h->L.ny;
  cudaStream_t st = h->stream;
  auto copy = [&](double* dst, const double* src, int64_t b, int64_t e) {
    return e > b ? cudaMemcpyAsync(dst + b, src + b, sizeof(double) * (e - b), cudaMemcpyDeviceToDevice, st)
                 : cudaSuccess;
  };
  auto owned = [&](const hd_slab& q, double* dst, const double* src) -> cudaError_t {
    cudaError_t e;
    if ((e = copy(dst, src, q.xf[0], q.xf[1])) != cudaSuccess) return e;
    if ((e = copy(dst, src, q.yf[0], q.yf[1])) != cudaSuccess) return e;
    if ((e = copy(dst, src, q.zf[0], q.zf[1])) != cudaSuccess) return e;
    return copy(dst, src, q.cell[0], q.cell[1]);
  };
  // local storage: owned entries of x; everything else NaN (0xFF bytes)
  for (int p = 0; p < P; ++p) {
    HD_CK(h, cudaMemsetAsync(s->xb[p], 0xFF, sizeof(double) * n, st));
    HD_CK(h, owned(s->slab[p], s->xb[p], x));
  }
  // exchange 1: the halo layer of p from p + 1's storage
  for (int p = 0; p + 1 < P; ++p) HD_CK(h, copy(s->xb[p], s->xb[p + 1], s->slab[p].halo[0], s->slab[p].halo[1]));
  // local applies: owned and halo entries of y start at zero, the rest NaN
  for (int p = 0; p < P; ++p) {
    const hd_slab& q = s->slab[p];
    double* yp = s->yb[p];
    HD_CK(h, cudaMemsetAsync(yp, 0xFF, sizeof(double) * n, st));
    HD_CK(h, cudaMemsetAsync(yp + q.xf[0], 0, sizeof(double) * (q.xf[1] - q.xf[0]), st));
    HD_CK(h, cudaMemsetAsync(yp + q.yf[0], 0, sizeof(double) * (q.yf[1] - q.yf[0]), st));
    HD_CK(h, cudaMemsetAsync(yp + q.zf[0], 0, sizeof(double) * (q.zf[1] - q.zf[0]), st));
    if (q.halo[1] > q.halo[0]) HD_CK(h, cudaMemsetAsync(yp + q.halo[0], 0, sizeof(double) * (q.halo[1] - q.halo[0]), st));
    h->e_first = (int64_t)q.ez0 * E2;
    h->e_end = (int64_t)q.ez1 * E2;
    hd_status r = elem_op_handle(h, OP_M | OP_DT | OP_D | OP_C, s->xb[p], s->xb[p] + h->n_rt, yp, yp + h->n_rt);
    h->e_first = 0;
    h->e_end = -1;
    if (r != HD_OK) return r;
  }
  // exchange 2: p's partial sums on its halo faces are added to p + 1's own
  for (int p = 0; p + 1 < P; ++p) {
    const hd_slab& q = s->slab[p];
    const int64_t m = q.halo[1] - q.halo[0];
    k_add_range<<<nblk(m), TPB, 0, st>>>(m, s->yb[p] + q.halo[0], s->yb[p + 1] + q.halo[0]);
    HD_LAUNCH_CK(h, "interface sums");
  }
  // gather of the owned parts
  for (int p = 0; p < P; ++p) HD_CK(h, owned(s->slab[p], y, s->yb[p]));
  return HD_OK;
}

// partial[0..P) = per-partition sums of a.b over the owned ranges, partial[P..nout) = 0
hd_status part_dot_partials(hd_op* h, const double* a, const double* b, double* partial, int nout) {
  PartState* s = h->part;
  k_part_partial<<<s->P * PART_BLOCKS, TPB, 0, h->stream>>>(s->P, s->d_ranges, a, b, s->d_partial);
  k_part_final<<<(nout + TPB - 1) / TPB, TPB, 0, h->stream>>>(s->P, s->d_partial, partial, nout);
  HD_LAUNCH_CK(h, "partitioned dot");
  return HD_OK;
}

extern "C" {

hd_status hd_slab_plan(int32_t nx, int32_t ny, int32_t nz, int32_t k, int32_t P, int32_t p, hd_slab* out) {
  if (nx < 1 || ny < 1 || nz < 1 || k < 1 || P < 1 || P > nz || p < 0 || p >= P || !out) return HD_ERR_INVALID_ARG;
  const int64_t X = (int64_t)nx * k, Y = (int64_t)ny * k, Z = (int64_t)nz * k;
  const int64_t nxf = (X + 1) * Y * Z, nyf = X * (Y + 1) * Z;
  if (nxf + nyf + X * Y * (Z + 1) + X * Y * Z >= ((int64_t)1 << 31)) return HD_ERR_INVALID_ARG;
  LatticeDims L{};
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.X = (int)X; L.Y = (int)Y; L.Z = (int)Z;
  L.n_xf = (int)nxf; L.n_yf = (int)nyf;
  plan(L, k, P, p, out);
  return HD_OK;
}

hd_status hd_apply_op_partitioned(hd_handle h, int32_t P, const double* x, double* y) {
  if (!h || !x || !y || x == y) return HD_ERR_INVALID_ARG;
  hd_status st = part_setup(h, P);
  if (st != HD_OK) return st;
  return part_apply(h, x, y);
}

hd_status hd_minres_solve_partitioned(hd_handle h, int32_t P, const double* b, double* x, const hd_solve_opts* o,
                                      hd_solve_info* info) {
  if (!h || !b || !x || !o || b == x || o->maxit < 1 || !(o->rtol > 0)) return HD_ERR_INVALID_ARG;
  if (o->precision != 0 || o->resume || h->schur_mode != 0)
    return hd_fail(h, HD_ERR_NOT_IMPLEMENTED,
                   "partitioned MINRES: FP64 (precision 0), no resume, V/W-cycle Schur block");
  hd_status st = part_setup(h, P);
  if (st != HD_OK) return st;
  h->part_on = true;
  st = minres_run(h, b, x, o, info);
  h->part_on = false;
  if (info) {
    double rn = 0, bn = 0;
    const int64_t n = h->n_rt + h->n_l2;
    if (!h->d_tmp && cudaMalloc(&h->d_tmp, sizeof(double) * (n > 0 ? n : 1)) != cudaSuccess)
      return hd_fail(h, HD_ERR_OOM, "tmp");
    hd_status s2 = part_apply(h, x, h->d_tmp);
    if (s2 != HD_OK) return s2;
    if ((s2 = residual_norms(h, b, h->d_tmp, &rn, &bn)) != HD_OK) return s2;
    info->true_relres = bn > 0 ? rn / bn : rn;
  }
  return st;
}

}  // extern "C"
