// Internal declarations of the hdivsp CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "hdivsp.h"

#define HD_MAXK 5
#define HD_MAXQ 7

// 1D tables of the interpolation-histopolation basis evaluated at the
// Gauss-Legendre points (Sec. 2.1). Passed to the element kernels by value so
// that they live in the kernel-parameter constant bank and unrolled loops use
// them as direct operands.
struct ElemTables {
  double BI[HD_MAXQ * (HD_MAXK + 1)];  // BI[p*(k+1)+i] = l_i(g_p), Lagrange at GLL nodes
  double BH[HD_MAXQ * HD_MAXK];        // BH[p*k+j]     = h_j(g_p), histopolation
  double gw[HD_MAXQ];                  // GL weights on [0,1]
  double gx[HD_MAXQ];                  // GL points on [0,1]
  double BG[HD_MAXQ * HD_MAXK];        // BG[p*k+m] = L_m(g_p): Lagrange basis on the k-point GL
                                       //   nodes (the nodal basis of the local CG) at the q points
  double TT[HD_MAXK * HD_MAXK];        // TT[j*k+m] = integral of L_m over subcell j: GL-nodal
                                       //   coefficients -> histopolation coefficients
  double HI[HD_MAXK * HD_MAXK];        // inverse of the 1D histopolation mass H[a][b] = int h_a h_b
                                       //   (affine elements: W_e^-1 = det J  HI x HI x HI)
  // Even-odd form of the centrosymmetric tables (M[R-1-r][C-1-c] = M[r][c]: the GLL and GL
  // points are symmetric about 1/2, and h_j(1 - x) = h_{k-1-j}(x)): for an R x C matrix M,
  // P[r][c] = (M[r][c] + M[r][C-1-c]) / 2 for c < C/2 and P[r][C/2] = M[r][C/2] for odd C
  // (r < ceil(R/2), row stride ceil(C/2)); N[r][c] = (M[r][c] - M[r][C-1-c]) / 2 (r < R/2,
  // c < C/2, row stride C/2). Then out[r] = E_r + O_r and out[R-1-r] = E_r - O_r with
  // E_r = P[r] . (x_c + x_{C-1-c}, middle x), O_r = N[r] . (x_c - x_{C-1-c}). For BI and BH
  // (points x coefficients) and their transposes (BIT, BHT: coefficients x points).
  double BIp[16], BIn[16], BHp[16], BHn[16], BITp[16], BITn[16], BHTp[16], BHTn[16];
};

// One-time set-up per device (the dynamic shared memory opt-in is a function attribute of
// each device): the entry of the current device in a caller-owned static flag array, or
// null when the device cannot be told (then the set-up simply runs again).
#define HD_MAX_DEVICES 64
inline bool* device_flag(bool* flags) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= HD_MAX_DEVICES) return nullptr;
  return flags + dev;
}

// Mesh/lattice constants passed to kernels.
struct LatticeDims {
  int nx, ny, nz;      // elements
  int X, Y, Z;         // subcells
  int n_xf, n_yf;      // number of x- and y-faces (z-faces follow)
  uint32_t ess;        // essential side mask
};

// Aggregation along one lattice axis from a finer level to the next coarser one:
// fine cell i belongs to coarse cell (i / c) m + g[i % c], and coarse cell C covers
// the fine cells [agg_lo(C), agg_hi(C)). Pairs: c = 2, m = 1 (a trailing odd cell
// alone); an axis that is not coarsened: c = 1, m = 1. Element-aligned aggregation
// with an odd number c of cells per element along the axis: c, and m groups per
// element (pairs from both ends of the element, an odd middle cell alone), so that
// no aggregate straddles an element boundary.
struct Agg1 {
  int c, m;
  int8_t g[8];   // group of fine offset r < c within its element
  int8_t s[9];   // first fine offset of group j < m; s[m] = c
};
__host__ __device__ __forceinline__ int agg_of(const Agg1& a, int i) {
  if (a.m == 1) return a.c == 2 ? (i >> 1) : (a.c == 1 ? i : i / a.c);
  const int p = i / a.c;
  return p * a.m + a.g[i - p * a.c];
}
__host__ __device__ __forceinline__ int agg_lo(const Agg1& a, int C) {
  if (a.m == 1) return C * a.c;
  const int p = C / a.m;
  return p * a.c + a.s[C - p * a.m];
}
__host__ __device__ __forceinline__ int agg_hi(const Agg1& a, int C, int n) {
  int h;
  if (a.m == 1) {
    h = C * a.c + a.c;
  } else {
    const int p = C / a.m;
    h = p * a.c + a.s[C - p * a.m + 1];
  }
  return h < n ? h : n;
}

// 1D tables of the L2 space for any degree (defined in hd_api.cu)
void hd_l2_tables(int k, int q, double* BH, double* BG, double* TT, double* gx, double* gw);

// true when every axis of the aggregation is pairs (or not coarsened)
inline bool agg_pairs(const Agg1* a) { return a[0].m == 1 && a[1].m == 1 && a[2].m == 1; }
template <typename Lv>
void set_agg(Lv& c, const Agg1& ax, const Agg1& ay, const Agg1& az) {
  c.ag[0] = ax; c.ag[1] = ay; c.ag[2] = az;
  c.fx = ax.m == 1 ? ax.c : 0;
  c.fy = ay.m == 1 ? ay.c : 0;
  c.fz = az.m == 1 ? az.c : 0;
}

// One level of the V-cycle hierarchy: a 7-point M-matrix stencil on an
// X x Y x Z cell lattice, stored as face weights (boundary faces included,
// essential faces 0), per-cell mass, diagonal and inverse l1 diagonal.
template <typename T>
struct LevelT {
  int X, Y, Z;
  int fx, fy, fz;      // pair factor (2, or 1: not coarsened) from the finer level; 0: ag[] holds groups
  Agg1 ag[3];          // the aggregation from the previous (finer) level, per axis
  T* wx;               // (X+1) Y Z
  T* wy;               // X (Y+1) Z
  T* wz;               // X Y (Z+1)
  T* mass;             // X Y Z
  T* diag;             // mass + sum of the 6 face weights
  T* dinv;             // 1 / (diag + sum of interior face weights)  (l1-Jacobi)
  T* x0;               // work: iterate (ping)
  T* x1;               // work: iterate (pong)
  T* b;                // work: right-hand side (levels >= 1)
  __host__ __device__ int64_t n() const { return (int64_t)X * Y * Z; }
};

// A coarse level of the smoothed-aggregation hierarchy: a symmetric stencil on
// an X x Y x Z cell lattice with NO offsets (33 on the first coarse level: the
// 3x3x3 box and the six cells two steps away along an axis; 27 below: the box;
// 179 and 81 on levels 2 and 3 when level 1's prolongator is smoothed as well).
// Stored by offset, a[h * n + c] = A(c, c + off_h) for the centre and the
// offsets that come later in lattice order (NH = (NO + 1) / 2 of them); the
// mirrored coefficient A(c, c - off_h) is a[h * n + c - off_h]. 0 where the
// neighbour is outside. During setup a holds all NO offsets.
template <typename T>
struct StLevelT {
  int X, Y, Z;
  int fx, fy, fz;      // as in LevelT
  Agg1 ag[3];
  int no;              // 27, 33, 81 or 179
  T* a;                // [NH][n] (setup: [no][n])
  T* dinv;             // 1 / sum_o |a[o][c]|  (l1-Jacobi)
  T* x0;
  T* x1;
  T* b;
  __host__ __device__ int64_t n() const { return (int64_t)X * Y * Z; }
};

// Lattice coordinates (I, J, Z) of cell c on an X x Y x ... lattice, c = I + X (J + Y Z).
// 32-bit unsigned division whenever c fits (64-bit integer division costs several
// times more instructions, and per-cell kernels are otherwise cheap).
__device__ __forceinline__ void lat_coords(int64_t c, int X, int Y, int& I, int& J, int& Z) {
  if (c < 0x7fffffffLL) {
    const unsigned u = (unsigned)c, ux = (unsigned)X, uy = (unsigned)Y, t = u / ux;
    I = (int)(u - t * ux);
    J = (int)(t % uy);
    Z = (int)(t / uy);
  } else {
    const int64_t t = c / X;
    I = (int)(c - t * X);
    J = (int)(t % Y);
    Z = (int)(t / Y);
  }
}

struct MinresState;  // device-side scalars of the MINRES recurrence
struct TcState;      // data of the tensor-core operator (k_op_tc.cu)
struct PartState;    // in-process z-slab partition (slab.cu)

struct hd_op {
  // problem
  hd_problem_desc desc;
  std::vector<int8_t> rot;   // element rotation codes (empty: all lattice-aligned)
  int kind, k, q;
  LatticeDims L;
  int64_t n_rt, n_l2, n_elem;
  double tau;
  int winv_mode, nu, coarse_max;
  // setup phase times in ms (hd_get_setup_times): geometric factors, W^-1 data,
  // diag(M), Schur preconditioner hierarchies, double-float copies, hd_create total
  float setup_ms[6] = {0, 0, 0, 0, 0, 0};
  int cycle = 1;
  int w_levels = 0;    // W repetition on levels < w_levels only (0: all)
  int agg_aligned = 0; // 1: element-aligned aggregation (Agg1) in the Schur hierarchy
  bool singular;
  cudaStream_t stream = nullptr;
  std::string err;
  ElemTables tab;
  ElemTables tabW;     // tables for the W quadrature (same rule)

  // device data (FP64)
  double* d_vx = nullptr;       // vertices (SoA)
  double* d_vy = nullptr;
  double* d_vz = nullptr;
  double* d_G = nullptr;        // [E][6][Q^3] w_p b_e J^T J / det J
  double* d_wdet = nullptr;     // [E][Q^3] w_p / det J
  double* d_winv = nullptr;     // [E][k^3][k^3] unweighted W_e^-1 (dense mode)
  double* d_wdiag = nullptr;    // [E][k^3] diag(W_e) (unweighted)
  double* d_wgldiag = nullptr;  // [E][k^3] diag of W_e in the GL nodal basis (local CG)
  double* d_wchol = nullptr;    // HD_WINV_CHOL: [E][k^3][k^3] Cholesky factor of W_e (reciprocal diagonal)
  double* d_Ga = nullptr;       // affine meshes: [E][8] b_e (J^T J)_{ab} / det J (00,01,02,11,12,22), det J, 0
  dfloat* x_Ga = nullptr;       //   and its double-float copy (the FP64 apply's affine fast path)
  float* f_wdet = nullptr;      // FP32 copies for the inner solve
  float* f_wgldiag = nullptr;
  double* d_cscale = nullptr;   // [E] c_e: C_e = c_e W_e^-1
  double* d_mt = nullptr;       // [n_rt] diag(M), 1 on essential dofs
  double* d_mtinv = nullptr;    // [n_rt] 1/(tau diag M) on free dofs, 1 on essential
  double* d_ct = nullptr;       // [n_l2] C~
  double* d_coarse_inv = nullptr;  // dense inverse of the coarsest level (or of A + s 11^T)
  int* d_kerr = nullptr;        // error word of the element kernel's bounded waits (bit 2)
  int coarse_n = 0;
  std::vector<LevelT<double>> lv;
  // smoothed-aggregation hierarchy (smooth_levels >= 1): prolongator values of
  // level 0 ([4][n_l2]: own aggregate, then the aggregates across the x, y and
  // z faces), stencil levels 1.., dense inverse of its coarsest level
  int sa = 0;
  bool sa_gen = false;  // level-0 aggregation with groups of one cell: [7][n_l2] prolongator values
  double* sa_p = nullptr;
  float* sa_pf = nullptr;
  double* sa_p1 = nullptr;  // smooth_levels = 2: prolongator of level 1 ([11][n_1])
  float* sa_p1f = nullptr;
  std::vector<StLevelT<double>> st;
  std::vector<StLevelT<float>> stf;
  double* d_sa_coarse_inv = nullptr;

  // double-float copies for the emulated-FP64 element kernel (fp64_emulation = 1)
  bool emul = false;
  dfloat* x_G = nullptr;
  dfloat* x_winv = nullptr;
  dfloat* x_cscale = nullptr;

  // FP32 copies for the mixed-precision inner solve
  float* f_G = nullptr;
  float* f_winv = nullptr;
  float* f_cscale = nullptr;
  float* f_mtinv = nullptr;
  float* f_coarse_inv = nullptr;
  std::vector<LevelT<float>> lvf;
  // double-float copies of the Schur hierarchy for the FP64 cycle (fp64_emulation = 2):
  // levels, stencil levels, prolongator values, cycle input and output
  bool cycle_df = false;
  std::vector<LevelT<dfloat>> lvx;
  std::vector<StLevelT<dfloat>> stx;
  dfloat* sa_px = nullptr;
  dfloat* sa_p1x = nullptr;
  dfloat* cyc_b = nullptr;
  dfloat* cyc_x = nullptr;
  bool have_f32 = false;

  // scratch
  double* d_red = nullptr;      // reduction partials
  double* d_tmp = nullptr;      // n_rt + n_l2
  double* h_pinned = nullptr;   // small pinned host buffer
  double* d_stage = nullptr;    // 2 (n_rt + n_l2) staging for *_host calls
  // MINRES work vectors (allocated on first solve)
  std::vector<double*> mv;
  // GMRES (hd_gmres_solve): basis [gm_m + 1][n], work vectors w, z, t [3][n], dot
  // partials and results, pinned host copy
  double* gm_V = nullptr;
  int gm_m = 0;
  double* gm_w = nullptr;
  double* gm_part = nullptr;
  double* gm_dots = nullptr;
  double* gm_host = nullptr;
  float* gm_Vf = nullptr;  // mixed precision: FP32 basis [gm_mf + 1][n] and work [3][n]
  int gm_mf = 0;
  float* gm_wf = nullptr;
  MinresState* d_ms = nullptr;
  // MINRES recurrence kept after a plain FP64 solve stopped at its iteration cap:
  // mr_it iterations done (0: none kept); mr_map[i] = index in mv of rpp, rp, y, z,
  // v, vn, wpp, wp, wn; x copied to mv[9]
  int mr_it = 0;
  int mr_map[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8};
  std::vector<float*> fv;       // FP32 work vectors for the mixed-precision solve
  // Schur-block preconditioner: 0 = V/W-cycle, 1 = V/W-cycle + learned network
  int schur_mode = 0;
  // MINRES iterations of the last converged solve with the V/W-cycle (0: none yet): a
  // solve with the learned network stops after 1.2 times as many and continues with
  // the V/W-cycle (HD_ERR_STAGNATION, info.fallback = 2)
  int plain_its = 0;
  struct LearnedNet* net = nullptr;
  // capture of the Lanczos vectors' L2 parts during a solve (training data)
  double* cap_buf = nullptr;
  int cap_every = 1, cap_max = 0, cap_count = 0;
  // V/W-cycle replayed as CUDA graphs (captured once per input/output pair) on a
  // private stream ordered after/before the handle's stream with events
  struct VcGraph {
    const void* b;
    void* x;
    int f32;  // key: 0/1 FP64/FP32 unsmoothed, 2/3 FP64/FP32 smoothed aggregation
    cudaGraphExec_t exec;
  };
  std::vector<VcGraph> vc_graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  bool graphs_off = false;
  // element window of the next element-kernel launch ([e_first, e_end); e_end < 0: all)
  int64_t e_first = 0, e_end = -1;
  // streams and events of the pipelined host-buffer apply (copy in, copy out)
  cudaStream_t xstream[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> xev;
  // inner operator of the mixed-precision solves: 0 = FP32 element kernel on the CUDA
  // cores, 1 = the tensor-core operator of affine meshes (k_op_tc.cu)
  int inner_op = 0;
  TcState* tc = nullptr;
  // in-process z-slab partition (hd_apply_op_partitioned, hd_minres_solve_partitioned);
  // part_on: MINRES applies the operator and sums its dot products through it
  PartState* part = nullptr;
  bool part_on = false;
  // profiling of the fused element kernel
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs (start, stop)
  int prof_n = 0;                     // recorded pairs
};

// records the start (before=true) or stop event of an element-kernel launch
void prof_mark(hd_op* h, bool before);

// error helpers
hd_status hd_fail(hd_op* h, hd_status s, const std::string& msg);
hd_status hd_cuda_check(hd_op* h, cudaError_t e, const char* what);
#define HD_CK(h, call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return hd_cuda_check((h), e_, #call);    \
  } while (0)
#define HD_LAUNCH_CK(h, what)                                       \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return hd_cuda_check((h), e_, what);     \
  } while (0)

// element-kernel launchers (one translation unit per k); mode bits below
enum {
  OP_M = 1,      // y_u += M u
  OP_DT = 2,     // y_u += D^T q
  OP_D = 4,      // y_q  = D u
  OP_C = 8,      // y_q -= C q  (or = -C q without OP_D); with OP_CPOS: y_q = +C q
  OP_CPOS = 16,
};
// y_u must be zeroed by the caller when OP_M or OP_DT is set.
hd_status launch_elem_op(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq);
hd_status launch_elem_op_f32(hd_op* h, int mode, const float* u, const float* q, float* yu, float* yq);
hd_status launch_elem_setup(hd_op* h);   // geometric factors, W_e^-1, diag(W), diag(M)

// lattice kernels (k_lattice.cu)
hd_status lattice_apply_B(hd_op* h, const double* u, double* yq);
hd_status lattice_apply_Bt(hd_op* h, const double* q, double* yu);
hd_status lattice_apply_Bt_f32(hd_op* h, const float* q, float* yu);
hd_status lattice_ess_identity(hd_op* h, const double* x, double* y);
hd_status precond_setup(hd_op* h);
hd_status precond_apply(hd_op* h, const double* r, double* z);
hd_status precond_apply_f32(hd_op* h, const float* r, float* z);
hd_status schur_apply(hd_op* h, const double* x, double* y);
hd_status vcycle_apply(hd_op* h, const double* b, double* x);
hd_status setup_f32(hd_op* h);
// smoothed-aggregation hierarchy (k_amg.cu)
hd_status sa_setup(hd_op* h);
hd_status sa_setup_f32(hd_op* h);
void sa_free(hd_op* h);
hd_status sa_vcycle(hd_op* h, const double* b, double* x);
hd_status sa_vcycle_f32(hd_op* h, const float* b, float* x);
hd_status sa_vcycle_df(hd_op* h, const dfloat* b, dfloat* x);
hd_status sa_setup_df(hd_op* h);
hd_status setup_df_cycle(hd_op* h);
// runs launch() as a cached CUDA graph keyed by (b, x, key) (k_lattice.cu)
hd_status run_graphed(hd_op* h, const void* b, void* x, int key, const std::function<void()>& launch);
// dense SPD inverse on the host (row-major; adds s 1 1^T first when singular)
hd_status dense_spd_inverse(hd_op* h, std::vector<double>& A, int n, bool singular, std::vector<double>& inv);
void precond_free(hd_op* h);
hd_status project_mean(hd_op* h, double* z);
hd_status vcycle_apply_f32(hd_op* h, const float* b, float* x);
hd_status diag_scale(hd_op* h, const double* r, double* z);
hd_status diag_scale_f32(hd_op* h, const float* r, float* z);
hd_status project_mean_f32(hd_op* h, float* z);
hd_status apply_op_f32_internal(hd_op* h, const float* x, float* y);
hd_status residual_norms(hd_op* h, const double* b, const double* y, double* rn, double* bn);
// z += P_1 V_1 P_1^T r: the coarse correction of the V-cycle hierarchy (nothing with one level)
hd_status coarse_correction(hd_op* h, const double* r, double* z);
// learned Schur preconditioner (k_learned.cu): z = V r + network(r), and z += network(r)
hd_status learned_schur_apply(hd_op* h, const double* r, double* z);
hd_status learned_net_add(hd_op* h, const double* r, double* z);
void learned_free(hd_op* h);
// y += a x ; p = z + b p
hd_status axpy_dev(hd_op* h, int64_t n, double a, const double* x, double* y);
hd_status xpay_dev(hd_op* h, int64_t n, const double* z, double b, double* p);

// Krylov (k_krylov.cu)
hd_status minres_run(hd_op* h, const double* b, double* x, const hd_solve_opts* o, hd_solve_info* info);
// tensor-core operator of affine meshes (k_op_tc.cu): y = AA x with FP16-pair operands
// and FP32 accumulation; set-up on first use
hd_status tc_setup(hd_op* h);
void tc_free(hd_op* h);
hd_status tc_apply(hd_op* h, const double* x, double* y);
hd_status tc_apply_f32(hd_op* h, const float* x, float* y);
// in-process z-slab partition (slab.cu): the partitioned apply, per-partition dot sums
// (partial[0..P) of an nout-entry partial array, zeros after) and clean-up
hd_status part_apply(hd_op* h, const double* x, double* y);
// the fused element kernel of the handle (FP64 or double-float) on [u; q] into [yu; yq]
// (hd_api.cu; mode: OP_* bits; the element window e_first / e_end applies)
hd_status elem_op_handle(hd_op* h, int mode, const double* u, const double* q, double* yu, double* yq);
hd_status part_dot_partials(hd_op* h, const double* a, const double* b, double* partial, int nout);
void part_free(hd_op* h);
// set-up of hd_minres_solve_noalloc on this handle's device (called by hd_create)
hd_status noalloc_prepare(hd_op* h);
hd_status dot_device(hd_op* h, const double* a, const double* b, int64_t n, double* d_out);
