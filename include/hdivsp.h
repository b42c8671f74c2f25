/*
 * hdivsp.h - C ABI of the GB300 matrix-free H(div) saddle-point library.
 *
 * Method: Pazner, Kolev, Vassilevski, "Matrix-free GPU-accelerated saddle-point
 * solvers for high-order problems in H(div)" (arXiv 2304.12387). The library
 * applies, for Raviart-Thomas (RT_k) x discontinuous L2 (Q_{k-1}) discretisations
 * in the interpolation-histopolation basis (Sec. 2.1) on structured hexahedral
 * meshes, the transformed block operator (Eq. transformed-saddle-point)
 *
 *        AA = [[ M , D^T ],
 *              [ D , -C  ]]
 *
 * with M = M_beta (grad-div) or M_{1/eps} (Darcy), D the lattice divergence
 * (two +-1 per column, Sec. 2.1), C = W_alpha^-1 (grad-div, Eq. transformed-system)
 * or W^-1 W_gamma W^-1 (Darcy, Eq. transformed-system-darcy; 0 when gamma = 0),
 * and the block-diagonal preconditioner diag(tau M~, S^) with M~ = diag(M) and
 * S^-1 one multigrid V-cycle on the approximate Schur complement
 * S~ = C~ + D M~^-1 D^T (Eq. approx-schur, Eq. approx-schur-entries), inside
 * preconditioned MINRES (Sec. 3).
 *
 * Conventions (all functions):
 *  - Every function returns hd_status (HD_OK = 0). No exception crosses the ABI.
 *    hd_last_error(h) gives a message for the last failing call on h.
 *  - Vector arguments of the hd_apply_* / hd_vcycle / hd_minres_solve calls are
 *    raw DEVICE pointers to contiguous FP64 arrays (FP32 for *_f32), owned by
 *    the caller, and must not alias each other unless stated. Vectors on the
 *    full block space are [u (n_rt); q (n_l2)].
 *  - All device work is enqueued on the handle's stream (hd_set_stream; default
 *    the legacy stream) and is asynchronous with respect to the host, except
 *    hd_create, hd_destroy, the hd_get_* calls, the *_host calls and
 *    hd_minres_solve, which return after the device work is complete.
 *  - The handle owns all internal device memory; hd_destroy frees it.
 *  - Size/pointer arguments are checked on entry (HD_ERR_INVALID_ARG). CUDA
 *    launch or runtime failures give HD_ERR_CUDA, allocation failures HD_ERR_OOM.
 *
 * Numbering (structured lattice, all elements unrotated): element
 * e = ex + nx (ey + ny ez); with X = nx k, Y = ny k, Z = nz k subcells,
 * L2 dof (cell) I + X (J + Y K); RT dofs: x-faces I + (X+1)(J + Y K), then
 * y-faces I + X (J + (Y+1) K), then z-faces I + X (J + Y K), global orientation
 * +x, +y, +z. Essential (u.n prescribed) RT dofs are eliminated as a
 * constrained identity: (AA x)_ess = x_ess.
 */
#ifndef HDIVSP_H
#define HDIVSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hd_status;
enum {
  HD_OK = 0,
  HD_ERR_INVALID_ARG = 1,
  HD_ERR_CUDA = 2,
  HD_ERR_OOM = 3,
  HD_ERR_NOT_CONVERGED = 4,
  HD_ERR_PREC_INDEFINITE = 5,
  HD_ERR_NAN = 6,
  HD_ERR_STAGNATION = 7,
  HD_ERR_BOUNDS = 8,
  HD_ERR_NOT_IMPLEMENTED = 9
};

/* problem kinds (Eq. grad-div and Eq. darcy) */
enum { HD_GRAD_DIV = 0, HD_DARCY = 1 };

/* how the L2 mass inverse W^-1 is applied (Sec. 3.1) */
enum {
  HD_WINV_DENSE = 0, /* explicit per-element inverse (the inverse + gemv approach of Sec. 3.1),
                        k^6 doubles per element, computed at setup */
  HD_WINV_CG = 1,    /* fused local CG in the Gauss-Legendre nodal basis (Sec. 2.5, 3.1):
                        Jacobi-preconditioned, per-element relative residual 1e-14 (cap 40
                        iterations), no stored inverse */
  HD_WINV_CG_HIST = 2,/* the same fused CG on W in the histopolation basis itself, without the
                        change of basis (the comparison of Sec. 3.1; cap 100 iterations). The
                        FP64 operator only: the FP32 inner operator keeps the GL-basis CG */
  HD_WINV_CHOL = 3    /* the per-element Cholesky factor W_e = L L^T computed at setup (the
                        factorisation approach of Sec. 3.1), k^6 doubles per element; every
                        apply solves two triangular systems per element. FP64 operator only (the
                        FP32 inner operator keeps the GL-basis CG) */
};

/* essential-boundary side bits */
enum {
  HD_SIDE_X0 = 1, HD_SIDE_X1 = 2, HD_SIDE_Y0 = 4,
  HD_SIDE_Y1 = 8, HD_SIDE_Z0 = 16, HD_SIDE_Z1 = 32
};

typedef struct hd_op* hd_handle;

/* Problem description for hd_create. All pointers are HOST pointers that are
 * only read during hd_create. */
typedef struct {
  int32_t kind;          /* HD_GRAD_DIV or HD_DARCY */
  int32_t nx, ny, nz;    /* elements per direction, >= 1 */
  int32_t k;             /* RT degree = subcells per element direction (the paper's p); 2..5 */
  int32_t q;             /* Gauss-Legendre points per direction; 0 -> k+1 if affine else k+2;
                            must be k+1 or k+2 */
  const double* vx;      /* vertex coordinates, (nx+1)(ny+1)(nz+1) each; vertex (i,j,l) */
  const double* vy;      /*   at i + (nx+1)(j + (ny+1) l); elements must have det J > 0 */
  const double* vz;
  const double* coef0;   /* per element: alpha > 0 (grad-div) or eps > 0 (Darcy) */
  const double* coef1;   /* per element: beta > 0 (grad-div) or gamma >= 0 (Darcy) */
  uint32_t ess_mask;     /* HD_SIDE_* bits: sides where u.n is essential */
  int32_t affine;        /* caller states the mesh is affine (only selects the default q) */
  double tau;            /* (1,1) preconditioner scaling tau M~; 0 -> 1 */
  int32_t winv_mode;     /* HD_WINV_DENSE, HD_WINV_CG, HD_WINV_CG_HIST or HD_WINV_CHOL */
  int32_t nu;            /* l1-Jacobi sweeps before and after the coarse correction; 0 -> 2 */
  int32_t coarse_max;    /* at most this many cells on the coarsest level; 0 -> 512 */
  int32_t cycle;         /* 0 or 1: V-cycle; 2: W-cycle (two coarse corrections per level
                            whose coarse level is not the coarsest) */
  int32_t fp64_emulation;/* 0: the element kernel computes in FP64; 1: in double-float (pairs of
                            FP32 numbers, about 48 significant bits) on the FP32 pipe, with FP64
                            vectors in and out and the same FP64 results to ~1e-13 relative;
                            HD_WINV_DENSE only. Setup, lattice kernels and MINRES stay FP64.
                            2: as 1, and the Schur V/W-cycle of the FP64 preconditioner (hd_vcycle,
                            hd_apply_prec, the FP64 solves) in double-float as well: its levels'
                            sweeps, residuals and transfers, between FP64 vectors; the coarsest
                            dense solve and the Krylov recurrences stay FP64. The cycle then
                            agrees with the FP64 one to ~1e-14 relative and remains a fixed
                            symmetric operator for MINRES. The double-float copies of the
                            hierarchy are made in hd_create (about the hierarchy's size again).
                            FP32's exponent range applies: hd_create refuses (HD_ERR_INVALID_ARG)
                            a problem where an element's geometric factors, W_e^-1 or
                            c_e W_e^-1 have their largest magnitude outside [2^-60, 2^60]
                            (entries far below their element's largest flush to zero
                            harmlessly); vector entries with |x| < 2^-126
                            enter the element kernel as 0 and |x| > 3.4e38 as inf, and entries
                            below about 2^-102 keep fewer than 48 bits (keep vectors near O(1)). */
  int32_t smooth_levels; /* prolongation of the Schur V-cycle: 0: piecewise constant on the 2x2x2
                            aggregates (unsmoothed aggregation); 1: the first level's prolongator
                            smoothed, P = (I - 4/3 D_l1^-1 S~) P0 (smoothed aggregation; the first
                            coarse level is a 33-point stencil, the deeper ones 27-point); 2: the
                            second level's prolongator smoothed in the same way with its own
                            l1 diagonal (level 2 a 179-point stencil, level 3 81-point, the
                            deeper ones 27-point). The paper's AMG (Sec. 3.2) gives
                            mesh-independent iteration counts; smoothing restores them for
                            log-normal coefficients. Other values: HD_ERR_NOT_IMPLEMENTED. The
                            learned Schur preconditioner adds its network to this cycle. */
  int32_t w_levels;      /* with cycle = 2: the two coarse corrections are made on levels
                            0..w_levels-1 only, one below (0: on every level); >= 0 */
  const int8_t* elem_rotation; /* NULL (every element lattice-aligned) or n_elem rotation codes
                            0..23: element e places its reference cube by that proper symmetry
                            of the cube (Algorithm 1's local orientations; code convention at
                            hd_lattice_e2d_map_rot). The global RT and L2 bases, hence every
                            operator, do not depend on the codes: the kernels compute each
                            element in its lattice-aligned frame, and the codes shape only the
                            element-local numbering and signs of hd_get_e2d_map and
                            hd_get_e2l_map. A code outside 0..23: HD_ERR_INVALID_ARG. */
  int32_t aggregation;   /* aggregates of the Schur V/W-cycle. 0: pairs of cells per direction
                            (a trailing odd cell alone). 1: element-aligned: along an axis where a
                            level holds c > 1 cells per element (its length a multiple of the
                            element count), the cells of each element are grouped in pairs taken
                            alternately from its two ends, an odd middle cell alone ([2, 1] for
                            c = 3, [2, 1, 2] for c = 5), so that no aggregate straddles an element
                            boundary; pairs elsewhere. For even k both are the same. For odd k,
                            pairs straddle half the element boundaries and the cycle needs about
                            twice the iterations of the aligned one. With odd k the first coarse
                            level of the smoothed hierarchy is then an 81-point stencil (box and
                            (+-2, a, b), |a|, |b| <= 1, with its permutations), and
                            smooth_levels = 2 is not available (HD_ERR_NOT_IMPLEMENTED). Other
                            values: HD_ERR_INVALID_ARG. */
} hd_problem_desc;

/* MINRES options and report (Sec. 3). */
typedef struct {
  double rtol;           /* stop when eta_j <= rtol * eta_0 (eta: B^-1-norm of the residual) */
  int32_t maxit;         /* iteration cap */
  int32_t use_x0;        /* 1: x holds the initial guess; 0: start from zero */
  int32_t check_every;   /* host polls the device-side convergence word every n iterations (>= 1) */
  int32_t precision;     /* 0: FP64 throughout; 1: FP32 operator/preconditioner inside an
                            FP64 outer residual correction (see hd_minres_solve) */
  double outer_rtol;     /* precision = 1: target true relative residual ||b-AAx||/||b|| */
  int32_t max_outer;     /* precision = 1: at most this many outer corrections */
  int32_t resume;        /* 1: continue the recurrence kept on the handle (see hd_checkpoint_minres)
                            for up to maxit more iterations; rtol, use_x0 are those of the stopped
                            solve, x receives its iterate first; plain FP64 path only */
} hd_solve_opts;

typedef struct {
  int32_t iterations;    /* total inner MINRES iterations */
  int32_t outer;         /* outer corrections (precision = 1), else 1 */
  double eta_ratio;      /* final eta_j / eta_0 of the last inner solve */
  double true_relres;    /* ||b - AA x||_2 / ||b||_2 in FP64 at exit */
  double ms_total;       /* device time of the solve (CUDA events) */
  hd_status status;
  int32_t fallback;      /* learned Schur preconditioner (hd_minres_solve): 1: it broke down and
                            the solve was repeated with the V/W-cycle; 2: it stagnated (no
                            convergence within 1.2 times the iterations of the last converged
                            V/W-cycle solve on the handle) and the solve continued from its
                            iterate with the V/W-cycle; iterations and ms_total add up */
} hd_solve_info;

/* Training options and report of the learned Schur preconditioner. */
typedef struct {
  int32_t npairs;        /* residual/correction pairs taken from the plain solver */
  int32_t capture_every; /* take the L2 part of every n-th Lanczos vector of a plain MINRES solve */
  int32_t steps;         /* Adam steps on the mean loss over all pairs */
  double lr;             /* Adam learning rate */
  uint64_t seed;         /* seed of the random right-hand side of the data-generating solve */
} hd_train_opts;

typedef struct {
  int32_t pairs;             /* pairs actually captured */
  double loss_initial;       /* mean energy-norm loss before training */
  double loss_final;         /* after the last step */
  int32_t pcg_max_iterations;/* CG iterations of the hardest target solve */
  double ms_total;           /* device time of data generation and training */
} hd_train_info;

/* -- lifetime ----------------------------------------------------------- */
/* Builds the operator: 1D tables, geometric factors at quadrature points,
 * the per-element W^-1 (dense mode), diag(M), diag(W), S~ and the V-cycle
 * hierarchy (setup of Sec. 3.1-3.2). Uses the current CUDA device. */
hd_status hd_create(const hd_problem_desc* desc, hd_handle* out);
hd_status hd_destroy(hd_handle h);
const char* hd_last_error(hd_handle h);
/* stream: a cudaStream_t (NULL = legacy default stream). */
hd_status hd_set_stream(hd_handle h, void* stream);

/* -- sizes and index maps ----------------------------------------------- */
hd_status hd_get_sizes(hd_handle h, int64_t* n_rt, int64_t* n_l2, int64_t* n_elem);
/* Setup phase times of hd_create in milliseconds (the setup Sec. 3.1 times apart from
 * the solve): ms[0] geometric factors, ms[1] the W^-1 data (dense per-element
 * inverses, or the Jacobi diagonals of the local CG), ms[2] diag(M), ms[3] the Schur
 * preconditioner hierarchies, ms[4] the double-float copies, ms[5] hd_create in
 * total (host clock). ms[0..2] are CUDA-event times. Writes the first n (0..6)
 * entries to the host array ms; HD_ERR_INVALID_ARG otherwise. */
hd_status hd_get_setup_times(hd_handle h, double* ms, int32_t n);
/* Signed element-to-RT-dof map of Algorithm 1 (element_map, rt_local_to_global
 * and the orientations folded in): host_out has n_elem * 3(k+1)k^2 int32 entries,
 * row e lists the global id g of each local dof, stored as g when local and global
 * orientation agree and as -1-g otherwise. Local order: x-component
 * i + (k+1)(j + k l), then y-component i + k (j + (k+1) l), then z-component
 * i + k (j + k l). */
hd_status hd_get_e2d_map(hd_handle h, int32_t* host_out);
/* Element-to-L2-dof map (Algorithm 1's element_map and l2_global_to_local, inverted):
 * host_out has n_elem * k^3 int32 entries, row e lists the lattice cell id of each
 * local L2 dof a + k (b + k c) of element e in its own (possibly rotated) frame. */
hd_status hd_get_e2l_map(hd_handle h, int32_t* host_out);
/* Essential RT dofs in ascending order; *n in: capacity of host_out, out: count
 * (host_out may be NULL to query the count). */
hd_status hd_get_ess_dofs(hd_handle h, int64_t* host_out, int64_t* n);

/* Host-only builders of the same maps from the mesh sizes (no handle, no GPU):
 * out has nx*ny*nz * 3(k+1)k^2 entries (hd_lattice_e2d_map), or holds up to *n
 * essential dofs (hd_lattice_ess_dofs; *n out: count; out may be NULL).
 * Return HD_ERR_INVALID_ARG on bad sizes or when the id range exceeds int32. */
hd_status hd_lattice_e2d_map(int32_t nx, int32_t ny, int32_t nz, int32_t k, int32_t* out);
/* The same maps for rotated elements (Algorithm 1 with non-trivial sigma_loc * sigma_glob).
 * rot: NULL or nx*ny*nz codes 0..23 (host). Element e with code r maps its reference
 * coordinates xi to the lattice-aligned ones eta = 1/2 + R (xi - 1/2), where R sends
 * reference axis d to lattice axis perm[d] with sign sgn[d]; r = 4 p + t, p the index of
 * perm among the 6 permutations of (0,1,2) in lexicographic order, t the index of sgn
 * among the 4 sign patterns with det R = +1, in increasing order of
 * [sgn0 < 0] + 2 [sgn1 < 0] + 4 [sgn2 < 0] (r = 0: identity). Along reference axis d
 * a node index t in [0,k] becomes t or k - t and an interval index t in [0,k) becomes t
 * or k - 1 - t (sgn[d] = +1 or -1); the RT dofs of reference component d lie on the
 * faces normal to lattice axis perm[d] and carry the orientation sgn[d] (stored as
 * -1-g when it is -1). hd_lattice_e2l_map writes nx*ny*nz * k^3 cell ids, local order
 * a + k (b + k c). A code outside 0..23 or bad sizes: HD_ERR_INVALID_ARG. */
/* Whether hd_create takes the affine fast path for this mesh (given affine = 1, q = k+1 and the
 * dense W^-1): *affine = 1 when every element is a parallelepiped, i.e. for each coordinate the
 * bilinear and trilinear combinations of its 8 vertices (v110 - v100 - v010 + v000 and the like)
 * are at most 1e-14 of its largest edge vector component plus 16 ulps of its largest vertex
 * coordinate, and det J > 0; else 0. Host only (no GPU); vertex layout as in hd_problem_desc.
 * Bad sizes or NULL pointers: HD_ERR_INVALID_ARG. Not in the paper: the fast path's test. */
hd_status hd_lattice_is_affine(int32_t nx, int32_t ny, int32_t nz, const double* vx, const double* vy,
                               const double* vz, int32_t* affine);
hd_status hd_lattice_e2d_map_rot(int32_t nx, int32_t ny, int32_t nz, int32_t k, const int8_t* rot,
                                 int32_t* out);
hd_status hd_lattice_e2l_map(int32_t nx, int32_t ny, int32_t nz, int32_t k, const int8_t* rot,
                             int32_t* out);
hd_status hd_lattice_ess_dofs(int32_t nx, int32_t ny, int32_t nz, int32_t k, uint32_t ess_mask,
                              int64_t* out, int64_t* n);

/* -- operator blocks (Sec. 3: the per-iteration operations) ---------------- */
/* y = M u (RT mass by sum factorisation, Eq. matrices); identity on essential dofs. */
hd_status hd_apply_A(hd_handle h, const double* u, double* y);
/* yq = D u (lattice divergence; essential columns dropped). */
hd_status hd_apply_B(hd_handle h, const double* u, double* yq);
/* yu = D^T q (zero on essential dofs). */
hd_status hd_apply_Bt(hd_handle h, const double* q, double* yu);
/* yq = C q: W_alpha^-1 q (grad-div) or gamma_e W^-1 q (Darcy, piecewise-constant
 * gamma, Sec. 2.4); zero for Darcy with gamma = 0. */
hd_status hd_apply_C(hd_handle h, const double* q, double* yq);
/* y = AA x, x = [u; q~], in one fused element pass (Eq. transformed-saddle-point). */
hd_status hd_apply_op(hd_handle h, const double* x, double* y);
/* Same as hd_apply_op with HOST input and output: copies x in, applies, copies y
 * out on the handle's stream and waits for it. */
hd_status hd_apply_op_host(hd_handle h, const double* x_host, double* y_host);

/* -- preconditioner (Sec. 2.3, 3.2) --------------------------------------- */
/* z = B^-1 r with B = diag(tau M~, S^): z_u = r_u / (tau M~) (z = r on essential
 * dofs), z_q = one V-cycle on S~ (projected to zero mean if S~ is singular). */
hd_status hd_apply_prec(hd_handle h, const double* r, double* z);
/* y = S~ x on the L2 lattice (7-point stencil, Eq. approx-schur-entries). */
hd_status hd_apply_schur(hd_handle h, const double* x, double* y);
/* x = one V-cycle on S~ applied to b (no projection). */
hd_status hd_vcycle(hd_handle h, const double* b, double* x);
/* Device copies of M~ = diag(M) (n_rt; 1 on essential dofs) and C~ (n_l2). */
hd_status hd_get_diagonals(hd_handle h, double* mt, double* ct);
/* Number of V-cycle levels and the lattice dimensions of level l. */
hd_status hd_get_level(hd_handle h, int32_t l, int32_t* n_levels, int32_t dims[3]);

/* -- solver (Sec. 3) ------------------------------------------------------ */
/* Solves AA x = b with block-preconditioned MINRES. b, x: device FP64 vectors of
 * length n_rt + n_l2. Returns HD_OK on convergence, HD_ERR_NOT_CONVERGED when
 * maxit is reached (x holds the last iterate), HD_ERR_PREC_INDEFINITE or
 * HD_ERR_NAN when the recurrence breaks down, HD_ERR_STAGNATION when the learned
 * Schur preconditioner stagnated (info.fallback = 2) and the continuation with the
 * V/W-cycle did not converge within maxit either. */
hd_status hd_minres_solve(hd_handle h, const double* b, double* x,
                          const hd_solve_opts* opts, hd_solve_info* info);

/* -- MINRES checkpoints ------------------------------------------------------ */
/* A plain FP64 solve (precision 0, max_outer <= 1, V-cycle Schur block) that stops at
 * its iteration cap keeps its recurrence on the handle: the iterate x, the Lanczos
 * vectors v_j, r_{j-1}, r_j, the direction vectors w_{j-1}, w_j and the device
 * scalars (Givens rotation, eta, iteration count). Any later solve on the handle
 * replaces it. A solve with opts.resume = 1 continues it exactly where it stopped:
 * with the same kernels, N iterations then a resume of M give the same x, bit for
 * bit, as N + M iterations in one call, and info.iterations counts from the start.
 *
 * hd_checkpoint_minres writes the kept recurrence to `path` (a header, then six
 * FP64 vectors of n_rt + n_l2 entries; host byte order); HD_ERR_INVALID_ARG when
 * the handle keeps none or the file cannot be written. hd_resume_minres reads such
 * a file into a handle of the same problem size (n_rt, n_l2, k), after which a solve
 * with opts.resume = 1 continues it; HD_ERR_INVALID_ARG for a missing, foreign,
 * truncated or differently sized file (the handle keeps no recurrence then). */
hd_status hd_checkpoint_minres(hd_handle h, const char* path);
hd_status hd_resume_minres(hd_handle h, const char* path);

/* -- GMRES with block preconditioners ----------------------------------------- */
/* The remark on block-triangular preconditioners in Sec. 2.3: with exact blocks,
 * P = [[M, D^T], [0, -S]] gives GMRES convergence in two iterations; with the
 * approximations tau M~ and the Schur V/W-cycle S^,
 *   z = P^-1 r:  z_q = -S^-1 r_q,  z_u = (r_u - D^T z_q) / (tau M~)
 * (identity on essential dofs, zero-mean z_q in the singular case). The
 * preconditioned operator is not symmetric, hence GMRES (right-preconditioned,
 * restarted, Saad & Schultz 1986) instead of MINRES. */
enum {
  HD_GMRES_BLOCK_DIAG = 0, /* the block-diagonal preconditioner of hd_minres_solve */
  HD_GMRES_BLOCK_TRI = 1   /* the block upper-triangular one above */
};
typedef struct {
  double rtol;      /* stop when ||b - AA x||_2 <= rtol ||b||_2; the recurrence estimates the
                       true residual (right preconditioning) and every restart and the exit
                       recompute it in FP64 */
  int32_t maxit;    /* Arnoldi steps in total (>= 1) */
  int32_t restart;  /* steps before a restart, 1..128; the basis takes restart + 1 device
                       vectors of n_rt + n_l2 doubles (allocated on the first call and kept) */
  int32_t prec;     /* HD_GMRES_BLOCK_DIAG or HD_GMRES_BLOCK_TRI */
  int32_t use_x0;   /* 1: start from x, else from zero */
  int32_t precision;/* 0: FP64 operator and V-cycle, the basis and Gram-Schmidt in double-float
                       (FP32 pairs, ~48 bits); 1: every cycle in FP32 (basis, Gram-Schmidt,
                       operator, V-cycle), every restart recomputing the residual with the FP64
                       operator and adding the cycle's correction to the FP64 solution (a
                       residual correction with GMRES cycles as the inner solver) */
  double inner_rtol;/* precision 1: a cycle ends once its estimate has fallen below inner_rtol
                       times the cycle's starting residual (0 < inner_rtol < 1) */
} hd_gmres_opts;
/* GMRES on AA x = b (device vectors of n_rt + n_l2 doubles, owned by the caller) with
 * the handle's operator (FP64 or double-float element kernel) and FP64 V/W-cycle.
 * Arnoldi by classical Gram-Schmidt, a second pass when the norm drops below 1e-3 of
 * its value; fixed-order reductions (deterministic). info->iterations = Arnoldi
 * steps, info->outer = restart cycles, info->eta_ratio = the last estimate / ||b||,
 * info->true_relres the FP64 true residual at exit. HD_ERR_NOT_CONVERGED when maxit
 * runs out, HD_ERR_NAN on a breakdown, HD_ERR_OOM when the basis does not fit,
 * HD_ERR_NOT_IMPLEMENTED for precision 1 with the learned Schur preconditioner enabled (it
 * replaces S^-1 in precision 0). */
hd_status hd_gmres_solve(hd_handle h, const double* b, double* x, const hd_gmres_opts* opts,
                         hd_solve_info* info);

/* -- profiling ------------------------------------------------------------- */
/* enable != 0: record a CUDA event pair on the handle's stream around every
 * launch of the fused element kernel (up to 4096 launches, then recording
 * stops). hd_profile_read waits for the stream, returns the number of recorded
 * launches and their summed device time in ms, and clears the record. */
hd_status hd_profile(hd_handle h, int32_t enable);
hd_status hd_profile_read(hd_handle h, int32_t* launches, double* ms);

/* -- z-slab partition (the multi-GPU runs of Sec. 4.2; emulated on one GPU) ------ */
/* Partition p of P (P <= nz) owns the element layers [ez0, ez1) with
 * ez0 = floor(p nz / P), and the global ids in the half-open ranges below: the x-faces,
 * y-faces and cells of lattice layers K in [k ez0, k ez1), the z-faces of layers
 * [k ez0, k ez1) (the last partition: up to and including the top layer K = Z). Its halo
 * is the z-face layer K = k ez1 (owned by p + 1; empty for the last partition): its top
 * element layer reads those faces and adds to them. An apply of the block operator needs
 * per interface two exchanges of X Y values: x on the halo from p + 1 to p before the
 * element loop, p's partial sums on the halo from p to p + 1 after it (two addends per
 * interface face, so the result does not depend on P); a MINRES iteration needs one sum
 * of two scalars over the partitions. */
typedef struct {
  int32_t p, P;
  int32_t ez0, ez1;      /* element layers */
  int64_t xf[2];         /* owned x-face ids [xf[0], xf[1]) */
  int64_t yf[2];         /* owned y-face ids */
  int64_t zf[2];         /* owned z-face ids */
  int64_t cell[2];       /* owned L2 dofs, as ids of the block vector (n_rt + cell) */
  int64_t halo[2];       /* z-face ids of the halo layer */
} hd_slab;
/* Host only (no GPU). HD_ERR_INVALID_ARG for bad sizes, P > nz or p outside [0, P). */
hd_status hd_slab_plan(int32_t nx, int32_t ny, int32_t nz, int32_t k, int32_t P, int32_t p, hd_slab* out);
/* y = AA x (device vectors as hd_apply_op) through P partitions emulated on this GPU:
 * every partition applies its element layers to its own full-length buffers, which
 * hold NaN outside its owned and halo entries (a read outside them shows in y); the
 * halo values and interface sums move by device copies and an add kernel; y gathers
 * the owned parts. Equal to hd_apply_op bit for bit. The first call for a P allocates
 * 2 P vectors of n_rt + n_l2 doubles on the handle. */
hd_status hd_apply_op_partitioned(hd_handle h, int32_t P, const double* x, double* y);
/* hd_minres_solve (precision 0, no resume, V/W-cycle Schur block) with the operator
 * applied as in hd_apply_op_partitioned and every inner product summed per partition
 * over its owned entries, then over the P partitions in order (the allreduce); the
 * Schur V/W-cycle runs on the whole L2 vector (on P GPUs a gather to one rank and a
 * scatter back). Iterates equal the unpartitioned solve's to rounding (the sums
 * associate differently). Other options: HD_ERR_NOT_IMPLEMENTED. */
hd_status hd_minres_solve_partitioned(hd_handle h, int32_t P, const double* b, double* x,
                                      const hd_solve_opts* opts, hd_solve_info* info);

/* -- allocation-free solve (no counterpart in the paper) -------------------- */
/* Same computation and result as hd_minres_solve with precision = 0, max_outer <= 1
 * and the V/W-cycle Schur block, for callers that may not allocate device memory once
 * their handle exists: for instance a time-stepping or embedding host that fixes its
 * device memory budget after initialisation, or code running where another component
 * owns the device allocator. hd_minres_solve allocates, on its first call, eleven work
 * vectors of n_rt + n_l2 doubles and a device state word with cudaMalloc (and, on first
 * use for each pair of vectors, a CUDA graph of the V/W-cycle with its own stream and
 * events); this entry point instead takes ten work vectors and the 256-byte state slot
 * from a fixed device array compiled into the library (HD_NOALLOC_SCRATCH_DOUBLES
 * doubles = 16 MiB, held by every GPU that loads the library until the process exits),
 * launches the V/W-cycle without a graph, and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *  - Limit: n_rt + n_l2 <= HD_NOALLOC_MAX_DOFS; larger problems are rejected
 *    with HD_ERR_INVALID_ARG (message in hd_last_error).
 *  - precision != 0: HD_ERR_INVALID_ARG. max_outer > 1 (the FP64 residual-correction
 *    loop), resume, or the learned Schur preconditioner enabled on the handle:
 *    HD_ERR_NOT_IMPLEMENTED (use hd_minres_solve). The Lanczos-vector capture of
 *    hd_learned_train does not run inside this call.
 *  - hd_create, on a problem within the limit, looks up the array's device address
 *    with the handle's device current and runs this solve once (one iteration on a
 *    zero right-hand side, in two vectors it frees again), so that every kernel the
 *    solve launches is loaded before the caller's first call (with lazy module
 *    loading a kernel's first launch can take device memory). Create the handle
 *    before any stream capture.
 *  - Every call shares the one array and it keeps the last call's contents
 *    (the call initialises what it reads); calls that overlap on the GPU race.
 *  - Profiling (hd_profile) is suspended during the call; ms_total is host
 *    wall-clock time. */
#define HD_NOALLOC_SCRATCH_DOUBLES (2 * 1024 * 1024)
#define HD_NOALLOC_MAX_DOFS 209696
hd_status hd_minres_solve_noalloc(hd_handle h, const double* b, double* x,
                                  const hd_solve_opts* opts, hd_solve_info* info);

/* -- learned Schur-complement preconditioner -------------------------------- */
/* The paper preconditions S~ with one AMG V-cycle (Sec. 3.2). The learned variant
 * adds to the handle's V/W-cycle V a linear, symmetric-by-construction conv net on
 * the L2 cell lattice:
 *   P r = V r + s C1^T C2^T C2 C1 (s r) + delta r/d,  s = d^-1/2, d = diag(S~),
 * C1 a 3x3x3 convolution 1 -> nc, C2 3x3x3 nc -> nc (nc = 32), no bias or
 * activation. The network term is positive semi-definite for any weights, so P is
 * SPD; the initial weights are small (P starts at the plain cycle). Weights
 * W1[co][t] (nc x 27) and W2[co][ci][t] (nc x nc x 27), tap t = dx + 3 (dy + 3 dz)
 * for the neighbour at offset (dx-1, dy-1, dz-1); activations FP16, accumulation
 * FP32, so the network term is symmetric to FP16 rounding only: use it inside the
 * FP64 residual correction of hd_minres_solve (precision = 1 or max_outer > 1),
 * where V runs in FP32 and the outer loop restores the FP64 residual. */
hd_status hd_learned_init(hd_handle h, int32_t nc, uint64_t seed, double delta);
/* host FP32 weight arrays in the layout above */
hd_status hd_learned_set_weights(hd_handle h, const float* W1, const float* W2);
hd_status hd_learned_get_weights(hd_handle h, float* W1, float* W2);
/* z = network part of P (s C1^T C2^T C2 C1 (s r) + delta r/d) applied to an L2 vector r
 * (device FP64) */
hd_status hd_learned_apply(hd_handle h, const double* r, double* z);
/* z = P_1 V_1 P_1^T r (device FP64 L2 vectors; zero with a single level) */
hd_status hd_coarse_correction(hd_handle h, const double* r, double* z);
/* Loss sum_p ||e_p - P r_p||_S~^2 / ||e_p||_S~^2 with P = net + Q, Q r_p = qr_p given
 * (qr may be NULL for Q = 0), and its gradient w.r.t. W1, W2: r, e, qr are device
 * arrays of npairs stacked L2 vectors; gW1, gW2, loss are host outputs. */
hd_status hd_learned_grad(hd_handle h, int32_t npairs, const double* r, const double* e, const double* qr,
                          float* gW1, float* gW2, double* loss);
/* Generates training pairs from a plain solve (Lanczos-vector L2 parts r,
 * e = S~^-1 r by V-cycle-preconditioned CG to 1e-10, and the fixed part V r) and runs
 * Adam on the loss of hd_learned_grad with qr = V r. */
hd_status hd_learned_train(hd_handle h, const hd_train_opts* opts, hd_train_info* info);
/* 0: V/W-cycle (default); 1: V/W-cycle + learned network for the Schur block in
 * hd_apply_prec, hd_minres_solve (fallbacks: info.fallback) and FP64 hd_gmres_solve. */
hd_status hd_set_schur_prec(hd_handle h, int32_t mode);
/* on = 1: hd_set_schur_prec(h, 1); on = 0: back to the V-cycle */
hd_status hd_enable_learned(hd_handle h, int32_t on);
/* The network (nc, delta, W1, W2 in the layout above; FP32, host byte order) to a
 * file and back. hd_learned_load initialises the network when the handle has none
 * (or another delta); HD_ERR_INVALID_ARG for a missing, foreign or truncated file.
 * Training runs as one call, so no optimiser state is kept. */
hd_status hd_learned_save(hd_handle h, const char* path);
hd_status hd_learned_load(hd_handle h, const char* path);
/* The engine of the network's 32 -> 32 convolutions (forward and adjoint, in every apply
 * and in training): 0 (default) the 5th-generation tensor cores (tcgen05.mma kind::f16,
 * FP16 operands in shared memory, FP32 accumulators in tensor memory; 128 cells of an
 * x-line per tile, persistent, one CTA per SM), 1 the warp-level mma.sync m16n8k16 path.
 * Both accumulate in FP32 and round to FP16, so they agree to FP16 rounding. A bounded
 * wait of the tensor-core path that runs out is reported by hd_tc_status. Needs
 * hd_learned_init first; other values: HD_ERR_INVALID_ARG. */
hd_status hd_learned_conv_engine(hd_handle h, int32_t engine);

/* -- FP32 variants (inner operators of the mixed-precision solve) ---------- */
hd_status hd_apply_op_f32(hd_handle h, const float* x, float* y);
hd_status hd_apply_prec_f32(hd_handle h, const float* r, float* z);

/* -- tensor-core operator of affine meshes (inner operator, mixed precision) -- */
/* On parallelepiped elements the Piola-mapped RT mass is M_e = sum_ab G_ab K_ab
 * (Eq. matrices with J constant: G = beta J^T J / det J per element, K_ab the
 * reference-cube blocks between velocity components, the same for every element),
 * so the element loop becomes dense GEMMs with the elements of a tile of 128 as rows,
 * which these calls run on the tensor cores (tcgen05.mma, FP16 operands, FP32
 * accumulators in tensor memory). Each operand is split into an FP16 pair
 * (hi + lo, with power-of-two scaling per element component and per block), three
 * products per block: an FP32-class operator (relative error about 1e-6 of the
 * largest entry, against ~1e-16 for hd_apply_op). D, D^T and C = c_e det J
 * (H^-1 x H^-1 x H^-1) (the affine W_e^-1) run in FP32 on the CUDA cores in the same
 * kernel. Requires a handle on the affine fast path (hd_create with affine = 1,
 * q = k + 1, HD_WINV_DENSE, every element a parallelepiped), k = 2..4 and a GPU of
 * the sm_100 family; else HD_ERR_NOT_IMPLEMENTED. The first call builds the split
 * reference blocks and FP32 element factors on the handle (allocates).
 * x, y: device vectors of n_rt + n_l2 entries (FP64, or FP32 for _f32), not aliased. */
hd_status hd_apply_op_tc(hd_handle h, const double* x, double* y);
hd_status hd_apply_op_tc_f32(hd_handle h, const float* x, float* y);
/* Inner operator of the mixed-precision solves (hd_minres_solve and hd_gmres_solve
 * with precision = 1, and hd_apply_op_f32): 0 = the FP32 element kernel (default),
 * 1 = the tensor-core operator above (same requirements; HD_ERR_NOT_IMPLEMENTED
 * otherwise, the mode is then unchanged). */
hd_status hd_set_inner_operator(hd_handle h, int32_t mode);
/* HD_OK, or HD_ERR_CUDA when a bounded wait ran out since the last call: inside the
 * tensor-core kernel (which then skipped the rest of its work), inside the tensor-core
 * convolution of the learned network, or inside the element kernel of a library built
 * with HD_DF_STAGE=1 (its W_e^-1 rows staged by bulk copies; off by default).
 * Synchronises the handle's stream and clears the record. */
hd_status hd_tc_status(hd_handle h);

/* -- DG mass inverse of any degree (Sec. 3.1, the setup and solve study) ------------ */
/* The block-diagonal L2 mass W = diag(W_e), W_e[a][b] = integral over element e of
 * alpha_e psi_a psi_b / det J (the L2 basis psi_a = h_a1 h_a2 h_a3 of Sec. 2.1, Q_{k-1}:
 * k^3 DOFs per element, integrals by the q^3 Gauss rule on the trilinear element), and
 * y = W^-1 x by one of the approaches compared in Sec. 3.1, for k = 2..9 (the paper's
 * p = k - 1 = 1..8; the block operator's handle covers k <= 5):
 *   HD_WINV_DENSE   setup: W_e assembled and inverted (its Cholesky factor, the factor's
 *                   inverse, W_e^-1 = L^-T L^-1); apply: one batched gemv (k^6 doubles/element)
 *   HD_WINV_CHOL    setup: W_e = L L^T; apply: two triangular solves per element
 *   HD_WINV_CG      setup: w_p alpha / det J at the points and the Jacobi diagonal of W in
 *                   the Gauss-Legendre nodal basis; apply: change of basis, the fused
 *                   per-element Jacobi-preconditioned CG to a relative residual of 1e-14
 *                   (at most 60 iterations), change of basis back (Sec. 2.5)
 *   HD_WINV_CG_HIST the same CG in the histopolation basis itself (at most 400 iterations)
 * All in FP64, or the CG stages in double-float (fp64_emulation). Vectors: device, n_l2 = (nx k)(ny k)(nz k) doubles in the lattice order
 * of the block operator's L2 part (cell I + X (J + Y Z)); x and y not aliased. The
 * handle owns its device data; calls run on its stream. */
typedef struct hd_massinv* hd_massinv_handle;
typedef struct {
  int32_t nx, ny, nz;    /* elements per direction, >= 1 */
  int32_t k;             /* k^3 L2 DOFs per element; 2..9 */
  int32_t q;             /* Gauss-Legendre points per direction; 0 -> k + 2; k..12 */
  const double* vx;      /* host vertex coordinates, layout as in hd_problem_desc */
  const double* vy;
  const double* vz;
  const double* alpha;   /* host, per element, > 0; NULL: 1 */
  int32_t method;        /* HD_WINV_DENSE, HD_WINV_CHOL, HD_WINV_CG or HD_WINV_CG_HIST */
  int32_t fp64_emulation;/* CG methods: 0 stages in FP64; 1 the sum-factorised stages and CG vectors
                            in double-float (FP32 pairs on the FP32 pipe, about 48 significant
                            bits), inner products, step lengths and stopping test in FP64; the
                            point weights w_p alpha / det J must lie in FP32's normal range.
                            Direct methods: 1 is HD_ERR_NOT_IMPLEMENTED. Other values:
                            HD_ERR_INVALID_ARG */
} hd_massinv_desc;
/* Builds the data of `method` on the current device and synchronises. Errors:
 * HD_ERR_INVALID_ARG (sizes, null pointers, method, alpha <= 0, det J <= 0 at a point),
 * HD_ERR_OOM, HD_ERR_CUDA, HD_ERR_NAN (a W_e not positive definite in the factorisation). */
hd_status hd_massinv_create(const hd_massinv_desc* desc, hd_massinv_handle* out);
/* stream: a cudaStream_t (NULL = legacy default stream). */
hd_status hd_massinv_set_stream(hd_massinv_handle h, void* stream);
/* y = W^-1 x (asynchronous on the handle's stream). */
hd_status hd_massinv_apply(hd_massinv_handle h, const double* x, double* y);
/* Device time of the setup in ms (geometric factors, diagonal or assembly and
 * factorisation), measured with events inside hd_massinv_create. */
hd_status hd_massinv_setup_ms(hd_massinv_handle h, double* ms);
/* CG methods: the largest number of iterations any element needed in the last apply
 * (synchronises); 0 for the direct methods. */
hd_status hd_massinv_iterations(hd_massinv_handle h, int32_t* its);
hd_status hd_massinv_destroy(hd_massinv_handle h);

/* -- grey nonlinear radiation diffusion (Sec. 4.3) ----------------------------------- */
/* The time integrator and nonlinear iteration that drive repeated Darcy solves. Model
 * (Eq. rad-diff-e, rad-diff-E, rad-diff-F), with T = e / Cv:
 *   rho de/dt = -c sigma (a T^4 - E) + Q,   dE/dt + div F = c sigma (a T^4 - E) + S,
 *   F = -(c / (3 sigma)) grad E,            F.n = 0 on every side (reflecting walls).
 * e and E lie in the L2 space (k^3 histopolation DOFs per element), and F lies in RT_k.
 * The opacity sigma is constant on each element; rho, Cv, a and c are constants.
 * E is carried as Eh = W E (W the L2 mass), the transformed L2 unknown of Eq.
 * transformed-system-darcy up to its sign.
 * Time stepping: Alexander's three-stage, L-stable, stiffly accurate SDIRK method. A
 * stage with beta = 1 / (dt a_ii), stage-start values (e*, Eh*) and source loads
 * Q_j = (Q, psi_j), S_j = (S, psi_j) solves
 *   R1 = rho beta W (e - e*) + c sigma (a N(e) - Eh) - Q      = 0
 *   R2 = beta (Eh - Eh*) + W D F - c sigma (a N(e) - Eh) - S  = 0
 *   R3 = M_{3 sigma/c} F - D^T Eh                              = 0   (essential rows: F)
 * with N(e)_j = (T(e)^4, psi_j) by the q^3 Gauss rule and D the lattice divergence.
 * The stage iteration follows Sec. 4.3, with two steps per pass:
 *   (1) F lagged: element-wise Newton on (R1, R2) for (e, Eh). Each Newton system is
 *       solved exactly by eliminating Eh (its block is (beta + c sigma) I). That leaves
 *       the SPD weighted mass (rho beta W + c sigma a theta N'(e)), theta = beta /
 *       (beta + c sigma), solved by Jacobi-preconditioned CG in the Gauss-Legendre
 *       nodal basis (Sec. 2.5). The step stops per element once ||(R1_e, R2_e)|| falls to
 *       newton_rtol times its first value, or to 1e-14 times ||(rho beta W e_e,
 *       beta Eh_e)||.
 *   (2) e fixed: the Darcy system of Eq. transformed-system-darcy, with eps = c /
 *       (3 sigma), gamma = beta + c sigma, x = [F; -Eh] and right-hand side
 *       [0; W^-1 (S + c sigma a N(e) + beta Eh*)]. It is solved by the handle's MINRES and
 *       block preconditioner, warm-started, to linear_rtol.
 * Passes repeat until ||(R1, R2, R3)||_2 <= outer_rtol times its value at the stage's
 * initial guess, or until, already below 1e3 outer_rtol times that value, it no longer
 * halves (its rounding floor). Every stage of every
 * step shares one Darcy operator, because a_ii is the same for all three stages.
 * The handle owns the Darcy operator (hd_rad_get_op) and its own device data.
 * Vectors are device FP64, in the lattice order of the block operator: n_l2 for e, Eh
 * and loads, n_rt for F, [E][q^3] for point values. Calls run on the handle's stream;
 * the stage and step calls synchronise it. */
typedef struct hd_rad* hd_rad_handle;
typedef struct {
  hd_problem_desc mesh;  /* nx, ny, nz, k, q, vx, vy, vz and the solver options of the Darcy
                            operator (tau, winv_mode, nu, coarse_max, cycle, fp64_emulation,
                            smooth_levels, w_levels, aggregation). kind, coef0, coef1, ess_mask,
                            affine and elem_rotation are ignored: hd_rad_create sets them */
  const double* sigma;   /* host, per element opacity > 0 */
  double rho, cv, a, c;  /* density, specific heat, radiation constant, speed of light; > 0 */
  double dt;             /* time step > 0 */
  double outer_rtol;     /* stage tolerance; 0 -> 1e-12 */
  int32_t outer_maxit;   /* passes per stage; 0 -> 10 */
  double newton_rtol;    /* 0 -> 1e-8 */
  int32_t newton_maxit;  /* Newton steps per pass; 0 -> 30 */
  double linear_rtol;    /* MINRES tolerance (on eta_j / eta_0); 0 -> 1e-8 */
  int32_t linear_maxit;  /* 0 -> 20000 */
  int32_t linear_precision; /* 0: FP64 MINRES; 1: the mixed-precision solve of hd_minres_solve
                            (FP32 operator and cycle inside an FP64 residual correction, inner
                            tolerance 1e-4), run until the true residual ||b - AA x||_2 has
                            fallen to linear_rtol times its value at the warm start, but not
                            below 1e-12 ||b||_2 (the FP64 operator's rounding level; a warm
                            start already there is kept), with at most 6 FP64 corrections per
                            Darcy step: where the true residual's rounding lies above the target,
                            the iterate is kept and the stage residual decides */
} hd_rad_desc;
typedef struct {
  int32_t stages;            /* stages solved by the call */
  int32_t outer;             /* passes, summed over the stages */
  int32_t outer_max;         /* most passes of one stage */
  int32_t newton_max;        /* most Newton steps of one element in one pass */
  int32_t linear_solves;
  int32_t linear_iterations; /* MINRES iterations, summed */
  double relres;             /* largest final ||R|| / ||R_0|| over the stages */
  double ms_newton;          /* device time of step (1), with the Darcy right-hand side */
  double ms_linear;          /* device time of step (2) */
  double ms_residual;        /* device time of the residual norms */
  hd_status status;
} hd_rad_info;
/* Builds the Darcy operator (hd_create), the point weights and the work vectors, and
 * synchronises. Errors: HD_ERR_INVALID_ARG (mesh as in hd_create, sigma or a constant
 * <= 0, dt <= 0, det J <= 0 at a point), HD_ERR_OOM, HD_ERR_CUDA. */
hd_status hd_rad_create(const hd_rad_desc* desc, hd_rad_handle* out);
hd_status hd_rad_destroy(hd_rad_handle h);
/* stream: a cudaStream_t (NULL = legacy default stream); also set on the Darcy operator. */
hd_status hd_rad_set_stream(hd_rad_handle h, void* stream);
/* The message of the last error on this handle ("" if none). */
const char* hd_rad_last_error(hd_rad_handle h);
/* Sizes: RT and L2 DOFs, elements, Gauss points per direction. */
hd_status hd_rad_get_sizes(hd_rad_handle h, int64_t* n_rt, int64_t* n_l2, int64_t* n_elem, int32_t* q);
/* The Darcy operator of the handle (owned by it; valid until hd_rad_destroy). */
hd_status hd_rad_get_op(hd_rad_handle h, hd_handle* op);
/* Host: physical coordinates of the Gauss points, [E][q^3][3] doubles, point p = p1 +
 * q (p2 + q p3) of element e = ex + nx (ey + ny ez); for sampling sources and fields. */
hd_status hd_rad_points(hd_rad_handle h, double* xyz);
/* load_j = (v, psi_j) = sum_p w_p v_p psi_j(xi_p) from point values v ([E][q^3]). */
hd_status hd_rad_load(hd_rad_handle h, const double* values, double* load);
/* y = W^-1 x (per element CG in the Gauss-Legendre basis to a relative residual of 1e-14);
 * E = W^-1 Eh, or the L2 projection of a field as hd_rad_winv(hd_rad_load(values)). */
hd_status hd_rad_winv(hd_rad_handle h, const double* x, double* y);
/* The stage residual at (e, Eh, F): r = [R1; R2; R3] (2 n_l2 + n_rt, device; may be NULL)
 * and ||r||_2 (host; may be NULL). Loads may be NULL (zero). Synchronises. */
hd_status hd_rad_residual(hd_rad_handle h, const double* e_star, const double* Eh_star, const double* q_load,
                          const double* s_load, const double* e, const double* Eh, const double* F, double* r,
                          double* norm);
/* One stage: (e, Eh, F) hold the initial guess and receive the solution. Loads may be
 * NULL. Errors: HD_ERR_NOT_CONVERGED (outer_maxit passes without reaching outer_rtol or
 * the rounding floor; the last iterate is kept), HD_ERR_NAN (a Newton system not
 * positive definite, or a non-finite residual), and those of hd_minres_solve. */
hd_status hd_rad_stage(hd_rad_handle h, const double* e_star, const double* Eh_star, const double* q_load,
                       const double* s_load, double* e, double* Eh, double* F, hd_rad_info* info);
/* One SDIRK step of size dt from (e, Eh, F), in place. q_loads and s_loads: NULL (no
 * sources), or the loads at the three stage times t + c_i dt, [3][n_l2] each, with
 * c = (gamma, (1 + gamma) / 2, 1). The flux F of each stage starts from the previous one. */
hd_status hd_rad_step(hd_rad_handle h, double* e, double* Eh, double* F, const double* q_loads,
                      const double* s_loads, hd_rad_info* info);

#ifdef __cplusplus
}
#endif
#endif /* HDIVSP_H */
