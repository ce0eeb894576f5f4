/*
 * mto.h - C ABI of the GB300 hot path of dp-adaptive multi-resolution topology optimization
 * (Gupta, van Keulen, Langelaar, "Design and analysis adaptivity in multi-resolution topology
 * optimization", arXiv:1811.09821), for 2D linear-elastic compliance problems.
 *
 * One analysis-plus-sensitivity pass per design iteration:
 *   (a) mto_build_elements  K_e = sum_s E(rho_s) K0_s over each element's d x d constant-density
 *                           subcells, SIMP E(rho) = Emin + rho^q (E0 - Emin)      (Eqs. 2-3, App. B)
 *   (b) mto_solve           K u = f by matrix-free preconditioned CG (multigrid), minimum-rule
 *                           conformity across p-jumps                              (Eq. 1)
 *   (c) mto_sensitivity     C = f^T u and dC/drho_s = -E'(rho_s) u_e^T K0_s u_e   (self-adjoint)
 *   (d) mto_indicator       Kelly Gamma^a (Eq. 9), density Gamma^d (Sec. 3.2.2), QR error
 *                           (Eq. 14) and the dp map update (Sec. 3.3)
 * plus the optimality-criteria design update mto_oc_update (the paper does not name its optimizer).
 *
 * Conventions
 *  - Mesh: nelx x nely structured quadrilaterals of size hx x hy; element e = ey*nelx + ex.
 *  - Element order p_e in 1..MTO_P_MAX; per-axis design count d_e in 1..MTO_D_MAX, the element
 *    carrying d_e^2 constant-density subcells, subcell s = j*d_e + i (i along x).
 *  - Packed design vectors (rho, dc): element e owns d_e^2 consecutive doubles starting at the
 *    exclusive prefix sum of d^2 ("design_len" values in total).
 *  - Global DOF numbering (identical to the oracle's): vertices row-major; interior nodes of
 *    horizontal edges (edge iy*nelx+ix, left to right); of vertical edges (edge iy*(nelx+1)+ix,
 *    bottom to top); cell-interior nodes (elements row-major, local nodes row-major);
 *    DOF = 2*node + component.  An edge carries order min(p_left, p_right) (minimum rule).
 *  - Pointers documented "device" are caller-owned device memory on the handle's device; "host"
 *    pointers are caller-owned host memory.  The handle owns its tables and workspace.
 *  - Device work is ordered on the caller's stream: each call's work starts after the work
 *    already queued there and the caller's stream waits for it (CUDA events; internally the
 *    handle runs on its own non-blocking stream, where the PCG iterations replay as CUDA
 *    graphs).  Calls that return host scalars (iterations, residuals, compliance) synchronise
 *    before returning.
 *  - Every call returns an mto_status.  On failure the outputs are unspecified and
 *    mto_last_error(h) gives a message.  Device-side failures (non-convergence, non-finite
 *    values, bounded waits that expire) are reported through status words read back by the
 *    host; no kernel traps.
 */
#ifndef MTO_H
#define MTO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MTO_P_MAX 6   /* largest shape-function order accepted by mto_setup (QR uses p+1) */
#define MTO_D_MAX 16  /* largest per-axis design count */

typedef struct mto_handle_s* mto_handle;

typedef enum {
  MTO_OK = 0,
  MTO_EINVAL = 1,    /* bad argument (sizes, ranges, null pointers, call order) */
  MTO_ENOMEM = 2,    /* device or host allocation failed */
  MTO_ECUDA = 3,     /* a CUDA runtime call failed */
  MTO_ENOCONV = 4,   /* the solve hit its iteration limit before the tolerance */
  MTO_ENAN = 5,      /* a non-finite value or a non-positive diagonal appeared */
  MTO_ETIMEOUT = 6   /* a bounded device wait expired */
} mto_status;

typedef enum { MTO_FP64 = 0, MTO_MIXED = 1, MTO_MIXED32 = 2 } mto_precision;

/* Material of Eq. 3 and Sec. 4.1 (E0 = 1, nu = 0.3, q = 3, Emin = 1e-9 E0 in the paper).
 * Plane stress. */
typedef struct {
  double E0, Emin, nu, q;
} mto_material;

/* Solver options.
 *  precision   MTO_FP64: FP64 iterative refinement: each step forms r = f - K u, solves K d = r
 *              by an inner PCG on the FP64 element matrices (FP64 pipes) with FP64 vectors to
 *              inner_rtol relative to r (solving for the correction keeps the recursive CG
 *              residual from drifting from the true one over long solves), and sets u += d.
 *              MTO_MIXED (needs the MTO_MIXED build): FP64 iterative refinement.  Each step forms
 *              the residual r = f - K u with the FP64 matrices and FP64 vectors, then solves
 *              K d = r by an inner PCG that applies the split-precision pair on the FP32 pipes
 *              (error-free products and sums, ~48-bit accurate) with FP64 vectors, to inner_rtol
 *              relative to r, and sets u += d.  A step whose FP64 residual falls short of the
 *              asked reduction by more than 10x (the split pair's 48 bits limiting an
 *              ill-conditioned problem) switches the remaining steps to the FP64 matrices.
 *              MTO_MIXED32 (needs the MTO_MIXED build): the same refinement with FP32 vectors in
 *              the inner PCG (converges only on well-conditioned problems; Jacobi or Schwarz).
 *              Dot products are accumulated in FP64 in every mode.
 *  rtol        stop when ||f - K u||_2 <= rtol ||f||_2 (free DOFs, FP64 residual).
 *  inner_rtol  relative residual reduction asked of each inner solve (<= 0: 1e-6); the last
 *              step asks only the remaining factor.
 *  max_iter    limit on the total number of (inner) PCG iterations.
 *  max_outer   limit on refinement steps (<= 0: 50).
 *  warm_start  nonzero: u on entry is the initial guess (else zero).
 *  check_every PCG iterations between host convergence checks (>= 1).
 *  norm        stopping test: MTO_NORM_L2 (||r||_2 / ||f||_2 <= rtol) or MTO_NORM_JACOBI
 *              (sqrt(r^T D^-1 r / f^T D^-1 f) <= rtol, D = diag(K); the scaled norm also weighs the
 *              rows of nearly void regions, stiffness ~ Emin, which the l2 norm ignores), or
 *              MTO_NORM_ENERGY: compliance accuracy, (C* - C(u)) / C <= rtol for the energy form
 *              C(u) = 2 f^T u - u^T K u of Eq. 1's compliance (its error is ||u* - u||_K^2).  One
 *              correction solve from the residual of the start vector; CG from zero gains
 *              alpha_i r_i^T z_i of energy per iteration and the remaining gains are the error;
 *              they are extrapolated from the sums of the last two windows of 32 gains (S_last,
 *              S_prev: error ~ S_last / (1 - S_last / S_prev)) and the stop is taken when that is
 *              below rtol / 4 times the compliance estimate (a margin for uneven decay).  rtol is then a relative compliance
 *              error (not squared); *relres still reports the l2 residual.
 *              Needs FP64 vectors (MTO_FP64 or MTO_MIXED).  At 10^7 DOFs and stiffness contrasts
 *              of 1e9 the l2 residual of an FP64 evaluation floors near 1e-7, so l2 tolerances
 *              below that cannot be met there, while compliance accuracy can.  A correction solve
 *              that does not meet the energy test within its iterations is followed by another one;
 *              at max_iter the solve returns MTO_ENOCONV.
 *  precond     MTO_PREC_JACOBI (point Jacobi), MTO_PREC_SCHWARZ (element-block additive Schwarz:
 *              per element the inverse of K_e plus the neighbours' share of the assembled diagonal,
 *              which captures the near-null modes of solid/void elements) or MTO_PREC_MG (one
 *              V-cycle of element-based Galerkin multigrid: the order p -> bilinear Q1 on the same
 *              mesh, then 2x2 agglomeration of Q1 elements, Chebyshev-Jacobi smoothing, dense
 *              inverse on the coarsest grid; FP64 vectors only (not MTO_MIXED32); mesh sides must
 *              halve down to a coarsest grid of at most 2048 DOFs, else MTO_EINVAL).
 *  inner_max   mixed solves: cap on the iterations of one inner solve (<= 0: none).
 *  mg_degree   MTO_PREC_MG only: Chebyshev degree of each pre- and post-smoothing on the fine
 *              level (<= 0: 4; at most 16); the Q1 levels use degree 4.
 *  mg_smoother MTO_PREC_MG only: the fine level's smoothing.  MTO_SMOOTH_JACOBI: Chebyshev
 *              polynomials of the point-Jacobi-scaled operator.  MTO_SMOOTH_BLOCK: of the
 *              operator scaled by the element-block inverse sum_e P_e^T (K_e + Delta_e)^-1 P_e (the
 *              blocks of MTO_PREC_SCHWARZ, which capture the element's own near-null modes); one
 *              more block apply per smoothing step, and on the 160 x 80 binary beam a third of the
 *              iterations.  The element blocks' output is masked to the free DOFs (a hanging DOF's
 *              row scatters onto the nodes it interpolates, supported ones included).
 *  mg_operator MTO_PREC_MG with the MTO_MIXED build only: the copy of the matrices the cycle applies
 *              (fine level: its smoothing steps, the restriction residual, the element blocks and the
 *              power iteration of the Chebyshev bounds; Q1 levels: their vertex stencils).
 *              MTO_MG_OP_LEAD: the cycle in FP32, i.e. the FP32 leading part of the split pair, the
 *              stencils rounded to FP32, FP32 vectors (half the bytes; a preconditioner needs a
 *              fixed operator, not the operator's accuracy: the outer PCG keeps the split pair and
 *              the FP64 refinement).  MTO_MG_OP_SPLIT: the split pair, FP64 stencils and vectors.
 *              MTO_MG_OP_AUTO (default): LEAD with MTO_SMOOTH_JACOBI, SPLIT with MTO_SMOOTH_BLOCK
 *              (the FP32-rounded inverses of the element blocks can lose definiteness on binary
 *              designs of extreme stiffness contrast; LEAD with block smoothing is then the
 *              caller's choice, as on the graded designs of the bench).
 * CG iterations run in chunks of check_every (rounded up to a multiple of 4), each a CUDA graph;
 * the reported count stops at convergence, but a chunk already launched completes (cheaply). */
typedef struct {
  int32_t precision;
  double rtol;
  double inner_rtol;
  int32_t max_iter;
  int32_t max_outer;
  int32_t warm_start;
  int32_t check_every;
  int32_t norm;
  int32_t precond;
  int32_t inner_max;
  int32_t mg_degree;
  int32_t mg_smoother;
  int32_t mg_operator;
} mto_solve_opts;

#define MTO_SMOOTH_JACOBI 0
#define MTO_SMOOTH_BLOCK 1
#define MTO_MG_OP_AUTO 0
#define MTO_MG_OP_SPLIT 1
#define MTO_MG_OP_LEAD 2

#define MTO_PREC_JACOBI 0
#define MTO_PREC_SCHWARZ 1
#define MTO_PREC_MG 2

#define MTO_NORM_L2 0
#define MTO_NORM_JACOBI 1
#define MTO_NORM_ENERGY 2

/* Indicator / map-update options (Sec. 3.2, 3.3; values of the paper in brackets).
 *  cycle           adaptive cycle index k~, from 1                                    [1, 2, ...]
 *  alpha, beta     density-band tuning parameters of Eqs. 10-13                       [0.2, 0.8]
 *  frac_a_refine   fraction of elements with the largest Gamma^a raised by one order  [0.10]
 *  frac_a_coarsen  fraction with the smallest Gamma^a lowered by one order            [0.05]
 *  alpha_d_refine, alpha_d_coarsen   fractions of the elements with Gamma^d > 0 (resp. < 0)
 *                  refined (coarsened)                                                [1, 1]
 *  alpha_qr        QR-error threshold                                                 [0.9]
 *  p_max, d_max    caps on the order and on the number of design points per element  [5, 64] */
typedef struct {
  int32_t cycle;
  double alpha, beta;
  double frac_a_refine, frac_a_coarsen;
  double alpha_d_refine, alpha_d_coarsen;
  double alpha_qr;
  int32_t p_max, d_max;
} mto_indicator_opts;

/* Create a handle bound to CUDA device `device` and the caller's CUDA stream `stream` (a
 * cudaStream_t; NULL means the legacy default stream).  The handle creates its own non-blocking
 * stream and a few small buffers; meshes allocate their tables in mto_setup. */
mto_status mto_create(mto_handle* h, int device, void* stream);

/* Free the handle and all device memory it owns.  Accepts NULL. */
mto_status mto_destroy(mto_handle h);

/* Message of the last failure on this handle (empty string when none).  Owned by the handle. */
const char* mto_last_error(mto_handle h);

/* Re-bind the handle to another stream of the same device. */
mto_status mto_set_stream(mto_handle h, void* stream);

/* Define the analysis and design meshes (Sec. 2.1, 3.3): nelx x nely elements of size hx x hy with
 * orders p_map[nel] and per-axis design counts d_map[nel] (host int32, row-major elements).
 * Builds the minimum-rule DOF numbering, the element classes and the subcell stiffness tables
 * K0_s (App. B composite integration) on the device.  Any order jump is accepted (the paper's
 * smoothing keeps jumps <= 2).  Returns the number of DOFs (including supported ones) and the
 * packed design length.  May be called again to change the maps; previous tables are freed.
 * Errors: MTO_EINVAL for sizes < 1, p outside 1..MTO_P_MAX, d outside 1..MTO_D_MAX. */
mto_status mto_setup(mto_handle h, int32_t nelx, int32_t nely, double hx, double hy,
                     const int32_t* p_map, const int32_t* d_map, int64_t* ndof, int64_t* design_len);

/* Homogeneous Dirichlet supports (Eq. 1 "Ku = f" on the free DOFs): fixed[n] host int64 global
 * DOF indices, duplicates allowed.  Must follow mto_setup (which clears them).
 * Errors: MTO_EINVAL for an index outside 0..ndof-1. */
mto_status mto_set_supports(mto_handle h, const int64_t* fixed, int64_t n);

/* Linear springs to ground, for the compliant-mechanism problem of Sec. 4.1 (Fig. 6b: k_in at the
 * input DOF, k_out at the output DOF): the operator of every later solve and apply becomes
 * K + sum_i k_i e_{d_i} e_{d_i}^T (also in the Jacobi diagonal and the multigrid fine level).
 * dofs: host int64[n] global DOFs; k: host double[n] > 0 (stiffnesses on one DOF add up).
 * Replaces earlier springs; n = 0 removes them.  mto_setup clears them.  At most 1024.
 * Errors: MTO_EINVAL for a DOF out of range or k <= 0.  Synchronises. */
mto_status mto_set_springs(mto_handle h, const int64_t* dofs, const double* k, int64_t n);

/* Global DOF of component `comp` (0 = x, 1 = y) at mesh vertex (ix, iy), 0 <= ix <= nelx,
 * 0 <= iy <= nely.  Host output. */
mto_status mto_vertex_dof(mto_handle h, int32_t ix, int32_t iy, int32_t comp, int64_t* dof);

/* Global DOFs of component `comp` (0, 1, or -1 for both) of every node on one side of the
 * domain: 0 = left (x = 0), 1 = right, 2 = bottom (y = 0), 3 = top; ascending.  Host output of
 * capacity `cap`; *count receives the number of DOFs (call with cap = 0 to size the buffer). */
mto_status mto_side_dofs(mto_handle h, int32_t side, int32_t comp, int64_t* out, int64_t cap,
                         int64_t* count);

/* Global DOFs of component `comp` (0 = x, 1 = y) of the nodes of one mesh edge, in parameter order
 * (start vertex, the interior nodes of the edge's order, end vertex): dir 0 is the horizontal edge
 * from vertex (ix, iy) to (ix + 1, iy), dir 1 the vertical edge from (ix, iy) to (ix, iy + 1).
 * Node lookup for loads and supports anywhere on the mesh (vertex and edge nodes).  Host output
 * of capacity `cap`; *count receives p_E + 1, p_E the edge's order (minimum rule).
 * Errors: MTO_EINVAL for an edge outside the mesh. */
mto_status mto_edge_dofs(mto_handle h, int32_t dir, int32_t ix, int32_t iy, int32_t comp, int64_t* out,
                         int64_t cap, int64_t* count);

/* Consistent nodal loads of a uniform traction on one side of the domain (the distributed load of
 * Sec. 4.1, Fig. 6a): for every node k of side `side` (0 = left, 1 = right, 2 = bottom, 3 = top)
 * f[2k + comp] += traction * (integral over the side of N_k ds).  On a boundary edge of order p_E
 * a node's trace is a Lagrange polynomial of the edge's Gauss-Lobatto-Legendre nodes, whose
 * integral is the GLL weight times half the edge length.  traction: force per unit length;
 * f: device double[ndof], accumulated into.  Synchronises. */
mto_status mto_side_load(mto_handle h, int32_t side, int32_t comp, double traction, double* f);

/* As mto_side_dofs, restricted to the nodes whose coordinate along the side (x for the bottom and
 * top sides, y for the left and right sides, from the domain corner at the origin) lies in
 * [s0, s1]: partial supports such as the corner clamps of the force inverter (Sec. 4.1, Fig. 6b). */
mto_status mto_side_dofs_in(mto_handle h, int32_t side, int32_t comp, double s0, double s1, int64_t* out,
                            int64_t cap, int64_t* count);

/* Inspection of the numbering (for tests and tools): for element e, fills per local node
 * (row-major, (p_e+1)^2 nodes) up to 8 (global node, weight) pairs: nodes[ln*8 + k],
 * weights[ln*8 + k], counts[ln].  A weight differs from 1 only on an edge whose order is below
 * p_e (minimum rule).  Host outputs sized (MTO_P_MAX+1)^2 * 8 and (MTO_P_MAX+1)^2. */
mto_status mto_element_nodes(mto_handle h, int64_t e, int64_t* nodes, double* weights, int32_t* counts);

/* Step (a): element stiffness matrices K_e = sum_s E(rho_s) K0_s (Eqs. 2-3 with the composite
 * integration of App. B) for every element, plus the Jacobi diagonal of the assembled operator.
 * rho: device double[design_len] (packed).  Both precisions store the FP64 matrices (the plain
 * FP64 path, refinement residuals, indicators); MTO_MIXED also stores each matrix as a
 * split-precision FP32 pair (hi = fl32(K_e), lo = fl32(K_e - hi), ~48 bits), applied on the FP32
 * pipes with error-free products and sums by the inner iterations of the mixed solves.  Matrices
 * stay in the handle, one row of the circulant-diagonal layout per element (D_k[i] = K[i][i+k mod
 * n_e], k = 0 .. n_e/2), element-major per order class.  Asynchronous. */
mto_status mto_build_elements(mto_handle h, const double* rho, const mto_material* mat, int32_t precision);

/* Inspection (tests, tools): the current matrix of element e as its packed upper triangle
 * (row-major, i <= j, local DOF 2*node + component), n_e (n_e + 1) / 2 doubles into host memory,
 * from the FP64 matrices.  Allocates a small device buffer; synchronises. */
mto_status mto_element_matrix(mto_handle h, int64_t e, double* packed);

/* Which kernel forms the element matrices in mto_build_elements:
 * MTO_BUILD_TENSOR (default): classes with d <= 8 run as one sliced GEMM per class on the tensor
 *   cores (tcgen05: both operands cut into 8 BF16 slices of 7 bits with power-of-two scales, the
 *   slice products summed exactly in FP32 TMEM columns by level, the levels combined in FP64:
 *   agrees with the FP64 kernel to ~1e-15 of each element's largest entry); larger d use the FP64
 *   CUDA-core kernel.
 * MTO_BUILD_SIMT: the FP64 CUDA-core kernel for every class. */
#define MTO_BUILD_TENSOR 0
#define MTO_BUILD_SIMT 1
mto_status mto_set_build_path(mto_handle h, int32_t path);

/* Compliance C = f^T u (Eq. 1 with z = f) of a solved displacement, reduced in the handle's own
 * workspace (fixed order: repeated calls give identical results).  f, u: device double[ndof].
 * C_dev: device double (may be NULL) receives C on the stream; C: host double (may be NULL;
 * then no synchronisation).  At least one of the two must be given. */
mto_status mto_compliance(mto_handle h, const double* f, const double* u, double* C_dev, double* C);

/* Compliance of an approximate displacement in its energy form (Eq. 1 with z = f):
 * C(u) = 2 f^T u - u^T K(rho) u, which equals f^T u at the exact solution and differs from the exact
 * compliance by ||u* - u||_K^2 (second order), so it carries the accuracy that the
 * MTO_NORM_ENERGY solve test controls; f^T u alone is only first-order accurate after a
 * warm-started solve.  u^T K u is summed from element energies sum_s E(rho_s) u_e^T K0_s u_e
 * (each after removing the element's rigid motion in FP64; no global cancellation), in a fixed
 * order.  u, f: device double[ndof]; rho: device double[design_len] (the densities of the build);
 * C: host double.  Synchronises. */
mto_status mto_compliance_energy(mto_handle h, const double* u, const double* f, const double* rho,
                                 const mto_material* mat, double* C);

/* Step (b): solve K u = f on the free DOFs (u = 0 on supports) with the options above, using the
 * matrices of the last mto_build_elements.  f: device double[ndof]; u: device double[ndof]
 * (initial guess when opts->warm_start, overwritten with the solution).  *iters receives the
 * total PCG iterations, *relres the final FP64 relative residual (host outputs, may be NULL).
 * Returns MTO_ENOCONV when max_iter or max_outer is reached first (u holds the last iterate),
 * MTO_ENAN on a breakdown.  Synchronises the stream. */
mto_status mto_solve(mto_handle h, const double* f, double* u, const mto_solve_opts* opts,
                     int32_t* iters, double* relres);

/* Batched calls over n independent instances (one handle each, all on one device; the handles may
 * differ in mesh size, orders, design counts and load case).  Every instance keeps its own stream,
 * workspace and captured CG iteration graphs, so the instances run concurrently on the GPU:
 *  - mto_build_elements_batched: the builds of all instances, asynchronous (rho[i]: device,
 *    instance i's packed design).
 *  - mto_solve_batched: the solves of all instances, advanced together.  The refinement loop of
 *    each (FP64 or MTO_MIXED; the options apply to all, see mto_solve_opts) is kept as a
 *    resumable state; each round launches every unfinished instance's next step (its next chunk
 *    of CG iterations as one CUDA graph launch, or its next residual) on its own stream and then
 *    synchronises once for all, so the host waits once per round instead of once per chunk per
 *    instance.  f[i], u[i]: device double[ndof_i].  iters, relres: host [n] (may be NULL);
 *    status: host mto_status[n] (may be NULL) per instance.  Returns MTO_OK when every instance
 *    converged, else the first failing status (the others still ran to completion).  Handles
 *    must be distinct.  Synchronises.
 *  - mto_sensitivity_batched: step (c) of all instances (FP64); C: host double[n] (may be NULL:
 *    then asynchronous). */
mto_status mto_build_elements_batched(mto_handle* hs, int32_t n, const double* const* rho, const mto_material* mat,
                                      int32_t precision);
mto_status mto_solve_batched(mto_handle* hs, int32_t n, const double* const* f, double* const* u,
                             const mto_solve_opts* opts, int32_t* iters, double* relres, mto_status* status);
mto_status mto_sensitivity_batched(mto_handle* hs, int32_t n, const double* const* u, const double* const* f,
                                   const double* const* rho, const mto_material* mat, double* const* dc, double* C);

/* y = K x on all DOFs (the assembled operator including supported rows), FP64, with the FP64
 * matrices of the last build.  x, y: device double[ndof].  Asynchronous. */
mto_status mto_apply(mto_handle h, const double* x, double* y);

/* y = K x with a chosen operator (tests and tools), over all DOFs like mto_apply.  op:
 *   MTO_OP_FP64   the FP64 element matrices on the FP64 pipes (plain FP64 path, refinement residuals);
 *   MTO_OP_SPLIT  the split-precision pair on the FP32 pipes with FP64 vectors: exactly the kernels the
 *                 inner PCG of MTO_MIXED solves launches (needs the MTO_MIXED build);
 *   MTO_OP_LEAD   the pair's FP32 leading part alone (the hi rows, x rounded to FP32, FP32 sums per
 *                 element, FP64 assembly): the copy of the operator the multigrid cycle may apply
 *                 where it only needs a fixed operator (see mg_operator of mto_solve_opts; MTO_MIXED
 *                 build).  Entries differ from K by the FP32 rounding of the matrices.
 * x, y: device double[ndof].  *xKx (host, may be NULL: then asynchronous) receives x^T y as the
 * operator launches reduce it for CG (per order class, summed in class order).  Synchronises when
 * xKx is given. */
#define MTO_OP_FP64 0
#define MTO_OP_SPLIT 1
#define MTO_OP_LEAD 2
mto_status mto_apply_operator(mto_handle h, int32_t op, const double* x, double* y, double* xKx);

/* Kernel of the split-precision operator for orders with n_e <= 32 (p <= 3); orders above always use
 * the generic kernel.  MTO_OPK_AUTO (default): the register-pipelined persistent kernel, or the
 * bulk-copy staged kernel for classes whose split rows exceed 64 MB; MTO_OPK_PIPE / MTO_OPK_STAGED
 * force one of them; MTO_OPK_GENERIC the plain one-pass kernel.  Applies to later solves and
 * mto_apply_operator calls (captured iteration graphs are discarded).  Synchronises the stream. */
#define MTO_OPK_AUTO -1
#define MTO_OPK_PIPE 0
#define MTO_OPK_STAGED 1
#define MTO_OPK_GENERIC 2
mto_status mto_set_operator_kernel(mto_handle h, int32_t kernel);

/* Autotuner (project-written): for every order class with n_e <= 32 times the split operator's three
 * kernels (register pipeline, bulk-copy staging, generic; CUDA events over 5 launches on the
 * class's own rows after 2 warm-up launches) and keeps the fastest for that class in the handle;
 * the choice is also cached process-wide by (device, order, element count), so later handles with
 * a class of the same size reuse it without timing.  Needs an MTO_MIXED build (it overwrites
 * internal work vectors only).  choice: host int32[MTO_P_MAX + 1] (may be NULL) receives per order
 * the chosen MTO_OPK_* (-2 where not tuned); us: host double[3 (MTO_P_MAX + 1)] (may be NULL) the
 * measured microseconds per launch of each kernel.  mto_set_operator_kernel overrides it.
 * Synchronises. */
mto_status mto_autotune(mto_handle h, int32_t* choice, double* us);

/* Inspection (tests, tools): the split-precision pair of element e after an MTO_MIXED build, as two
 * packed upper triangles (row-major, i <= j): hi[c] = fl32(K_e[c]), lo[c] = fl32(K_e[c] - hi[c]).
 * Host outputs of n_e (n_e + 1) / 2 floats each.  Allocates a small device buffer; synchronises. */
mto_status mto_element_matrix_split(mto_handle h, int64_t e, float* hi, float* lo);

/* Step (c): compliance C = f^T u (Eq. 1 with z = f) and the design sensitivities
 * dc[s] = -E'(rho_s) u_e^T K0_s u_e, E'(rho) = q rho^(q-1) (E0 - Emin): the adjoint of the
 * self-adjoint compliance problem is -u.  u, f: device double[ndof]; rho, dc: device
 * double[design_len]; C: host double (may be NULL: then no synchronisation).  precision as for
 * the build: MTO_MIXED evaluates the quadratic forms in FP32 after an FP64 removal of the
 * element's rigid-body motion. */
mto_status mto_sensitivity(mto_handle h, const double* u, const double* f, const double* rho,
                           const mto_material* mat, int32_t precision, double* dc, double* C);

/* Design transfer after a dp map update (Sec. 3.3; the paper does not say how design values move
 * to new design points): with the handle set up on the new maps, rho_new (device, packed for the
 * handle's current d map) receives for every new subcell the area-weighted mean of the old
 * subcells of the same element it overlaps; an element whose count did not change keeps its
 * values.  d_old: host int32[nel] per-axis counts of the old layout; rho_old: device, packed for
 * d_old.  Keeps every element's material volume.  Synchronises. */
mto_status mto_transfer_design(mto_handle h, const int32_t* d_old, const double* rho_old, double* rho_new);

/* The P2 density filter (Sec. 2.1, Eqs. 4-5) evaluated at the subcell centres:
 * rho_f[s] = sum_t H_st rho[t] / sum_t H_st with H_st = radius - dist(c_s, c_t) over every subcell t of
 * the mesh whose centre c_t lies within `radius` of c_s (across element edges; no volume weights,
 * as printed).  The filtered densities are the physical densities that the build takes
 * (K_e = sum_s E(rho_f[s]) K0_s); the paper uses radius = 0.3 h (Sec. 4.1).  rho, rho_f: device
 * double[design_len], distinct.  radius in (0, 4 min(hx, hy)].  Asynchronous. */
mto_status mto_filter(mto_handle h, double radius, const double* rho, double* rho_f);

/* Adjoint of mto_filter (the chain rule of the sensitivities): g[t] = sum_s H_st g_f[s] / W_s with
 * W_s = sum_k H_sk, i.e. dJ/drho from dJ/drho_f.  g_f, g: device double[design_len], distinct.
 * Asynchronous. */
mto_status mto_filter_adjoint(mto_handle h, double radius, const double* g_f, double* g);

/* Step (c) for a general objective J = z^T u (Eq. 1; the force inverter of Sec. 4.1 has z = the
 * unit vector of the output DOF): dJ/drho_s = -E'(rho_s) v_e^T K0_s u_e, where v is the adjoint
 * field solving K v = z (call mto_solve with f = z; the operator, springs included, is
 * symmetric).  For compliance z = f, so v = u and this equals mto_sensitivity.  u, v: device
 * double[ndof]; rho, dc: device double[design_len].  FP64 quadrature after an FP64 removal of
 * each field's element rigid motion.  Asynchronous. */
mto_status mto_sensitivity_adjoint(mto_handle h, const double* u, const double* v, const double* rho,
                                   const mto_material* mat, double* dc);

/* Step (d): composite refinement indicator and dp map update (Sec. 3.2, 3.3).
 * u: device double[ndof] (the solved displacement), rho: device double[design_len].
 * Outputs (device, [nel]): gamma_a (Kelly, Eq. 9, no square root), gamma_d (density indicator),
 * eps_qr (Eq. 14), p_new, d_new (int32, per-axis design count), theta (int8 flag: -2, -1, 0, 1).
 * Any output pointer may be NULL except those the later stages need internally (all are
 * computed).  Asynchronous. */
mto_status mto_indicator(mto_handle h, const double* u, const double* rho, const mto_material* mat,
                         const mto_indicator_opts* opts, double* gamma_a, double* gamma_d,
                         double* eps_qr, int32_t* p_new, int32_t* d_new, int8_t* theta);

/* Map update only (Sec. 3.3 steps 2-4) from given indicator values (device [nel] each) and the
 * handle's current orders.  For testing the integer logic in isolation. */
mto_status mto_map_update(mto_handle h, const double* gamma_a, const double* gamma_d,
                          const double* eps_qr, const mto_indicator_opts* opts, int32_t* p_new,
                          int32_t* d_new, int8_t* theta);

/* Optimality-criteria update (textbook; the paper does not name its optimizer):
 * rho_new = clip(rho (-dc / (lambda dv))^eta, max(0, rho - move), min(1, rho + move)) with
 * dv = hx hy / d_e^2 and lambda bisected on [0, 1e9] until (l2 - l1)/(l1 + l2) <= 1e-10 so that
 * sum(rho_new dv) = volfrac * nelx * nely * hx * hy.  rho (in), dc (in), rho_new (out): device
 * double[design_len]; *lambda (host, may be NULL) receives the multiplier (synchronises). */
mto_status mto_oc_update(mto_handle h, const double* rho, const double* dc, double volfrac,
                         double move, double eta, double* rho_new, double* lambda);

/* Kernel-family timing for benchmarks.  enable = 1: the launches of each family below are
 * bracketed by CUDA events recorded on the handle's stream; enable = 2 (sampled, low overhead):
 * only the first element-operator launch of every captured chunk of PCG iterations is bracketed;
 * 0: off.  mto_timing_read synchronises the stream and returns the number of timed kernel
 * launches and their summed device time (ms) since the last mto_timing_enable (which resets the
 * counters).  Families: */
#define MTO_TIME_APPLY32 0   /* split-precision operator on FP32 vectors (mixed inner PCG) */
#define MTO_TIME_APPLY64 1   /* FP64 element-by-element operator (plain FP64 path) */
#define MTO_TIME_BUILD 2     /* step (a): subcell tables and element matrices */
#define MTO_TIME_SENS 3      /* step (c): sensitivity quadrature and compliance */
#define MTO_TIME_INDICATOR 4 /* step (d): indicators and map update */
#define MTO_TIME_VECTOR 5    /* PCG vector updates, residuals, precision conversions */
#define MTO_TIME_APPLYDF64 6 /* split-precision operator on FP64 vectors (refinement residuals) */
#define MTO_TIME_PRECOND 7   /* preconditioner: multigrid cycle, element blocks, their set-up */
#define MTO_TIME_OC 8        /* optimality-criteria update */
#define MTO_TIME_APPLYLEAD 9 /* the FP32 leading parts inside the multigrid cycle: level 0's operator
                                (smoothing, restriction residual, power iteration) and its element
                                blocks */
mto_status mto_timing_enable(mto_handle h, int32_t enable);
mto_status mto_timing_read(mto_handle h, int32_t family, int64_t* launches, double* total_ms);

/* Device memory held by the handle, in bytes (host output). */
mto_status mto_memory(mto_handle h, int64_t* bytes);

/* Number of kernel launches this handle has issued since creation (host output). */
mto_status mto_launch_count(mto_handle h, int64_t* count);

/* Compliance C = f^T u of n DOFs without any allocation.  The paper has no counterpart: this is
 * an entry point for callers that manage all device memory themselves (for example around
 * externally captured work).  f, u: device double[n]; C: device double (written); stream: the
 * CUDA stream to launch on (NULL: the legacy default stream); device: the CUDA device that owns
 * f, u and C.  The block partial sums live in a fixed 72 KB array in the library's device memory
 * (8192 partials), so n is limited to 8192 x 2048 = 16,777,216 DOFs; larger n (or n < 0, NULL
 * pointers, a device index outside 0..63) returns MTO_EINVAL before any launch.  The array's
 * finished-block counter must be zero when a launch starts: it is zero when the library loads,
 * each call clears it on the stream before its kernel, and the kernel's last block clears it
 * again.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call outside any stream
 * capture.  Calls that overlap in time on the same device (different streams, host threads)
 * share the array and race: order them on one stream or with events.  The address is kept for the
 * life of the process: do not call this across a cudaDeviceReset.  The summation order depends
 * only on n, so repeated calls give bit-identical results.  Asynchronous; returns
 * MTO_ECUDA when a CUDA call fails. */
mto_status mto_compliance_noalloc(int32_t device, const double* f, const double* u, int64_t n, void* stream,
                                  double* C);

#ifdef __cplusplus
}
#endif

#endif /* MTO_H */
