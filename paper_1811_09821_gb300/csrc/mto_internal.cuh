// Internal declarations of the MTO library: handle layout, element classes, device helpers.
// Everything here is private to libmto; the public surface is include/mto.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/mto.h"

namespace mto {

constexpr int kPMaxTab = MTO_P_MAX + 1;   // tables go one order higher for the QR indicator
constexpr int kConsMax = 8;               // (node, weight) pairs per constrained local node
constexpr int kSlots = 4;                 // PCG scalar ring

// Packed upper triangle of an n x n symmetric matrix, row-major: c(i, j) for i <= j.
__host__ __device__ constexpr int packed_size(int n) { return n * (n + 1) / 2; }
__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Constrained local node: value = sum_k w[k] * value(node[k])  (minimum-rule interpolation).
struct Constraint {
  int cnt;
  int node[kConsMax];
  double w[kConsMax];
};

// Circulant-diagonal storage of a symmetric n_e x n_e element matrix: diagonal k (0 <= k <= n_e/2)
// holds D_k[i] = K[i][(i + k) mod n_e] for i = 0..n_e-1, so one element's matrix is a row of
// L = (n_e/2 + 1) n_e values (every packed entry once, the k = n_e/2 diagonal of an even n_e twice).
// A warp owning one element lets lane i read D_k[i] (contiguous), form K[i][i+k] x_{i+k} for its
// own row and hand K[i][i+k] x_i to lane i+k (the symmetric half) by shuffle.
__host__ __device__ constexpr int diag_count(int ne) { return ne / 2 + 1; }
__host__ __device__ constexpr int diag_row_len(int ne) { return diag_count(ne) * ne; }

// All elements of one shape-function order p.  Element matrices are element-major rows of the
// circulant-diagonal layout: FP64 [n][L] (FP64 path) or the split-precision pair hi, lo [n][L].
struct PClass {
  int p = 0;
  int n = 0;          // elements in the class
  int ld = 0;         // allocated element count (n rounded up to 32)
  int P = 0;          // packed size n_e (n_e + 1) / 2
  int L = 0;          // circulant-diagonal row length per element
  int* elem = nullptr;   // [n] element ids, ascending
  int* gmap = nullptr;   // [n][(p+1)^2] global node id, or -(1 + constraint index)
  int2* dpos = nullptr;  // [P] row positions of packed entry c (second one or -1)
  int* posc = nullptr;   // [L] packed entry stored at each row position
  double* K64 = nullptr;   // FP64 matrices (both builds)
  float* K32 = nullptr;    // split-precision pair (mixed build only): hi = fl32(K_e) ...
  float* K32lo = nullptr;  // ... and lo = fl32(K_e - hi), same layout
  double* B64 = nullptr;   // element-block preconditioner (K_e + Delta_e)^-1, same layouts
  float* B32 = nullptr;
  float* B32lo = nullptr;
};

// Elements of one (p, d) pair: the build and sensitivity granularity.
struct BClass {
  int p = 0, d = 0, S = 0, P = 0;
  int n = 0;
  int* elem = nullptr;   // [n] element ids
  int* slot = nullptr;   // [n] slot of each element in its PClass
  double* K0T = nullptr; // [P][S] subcell stiffness tables, transposed (entry c, subcell s)
  double* stab = nullptr; // sensitivity quadrature tables (FP64 and FP32 copies)
  float* stabf = nullptr;
  unsigned short* tcB = nullptr;  // tensor-core build: BF16 slices of K0 per N tile
  float* tcTau = nullptr;         // and the power-of-two column scales
};

// QR-indicator tables for order p -> p + 1.
struct QRTab {
  int p = 0;
  double* R = nullptr;   // [(p+2)^2][(p+1)^2] scalar load transfer M^(p+1,p) M^(p)^-1
};

// Kernel families timed with CUDA events when timing is enabled (see mto_timing_enable).
enum Family { F_APPLY32 = 0, F_APPLY64 = 1, F_BUILD = 2, F_SENS = 3, F_INDICATOR = 4, F_VECTOR = 5,
              F_APPLYDF64 = 6, F_PRECOND = 7, F_OC = 8, F_APPLYLEAD = 9, F_COUNT = 10 };

struct Timing {
  bool on = false;
  bool sampled = false;   // record only the operator launches marked by `sample` (low overhead)
  bool sample = false;
  bool sample_lead = false;   // also the leading-part operator launches (F_APPLYLEAD) while set
  struct Pending { int fam; int launches; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  std::vector<Pending>* capture_list = nullptr;   // event pairs of a graph being captured
  int64_t launches[F_COUNT] = {0};
  double ms[F_COUNT] = {0};
};

// One bilinear (Q1) level of the multigrid hierarchy on an nx x ny grid of elements.  Element
// matrices are FP64 rows of the circulant-diagonal layout (n_e = 8, L = 40), so the element
// operator kernel of order 1 applies them.
struct MGLevel {
  int nx = 0, ny = 0, nel = 0;
  int64_t nv = 0, n = 0;           // vertices, DOFs
  int* gmap = nullptr;             // [nel][4] vertex ids (x fastest)
  double* K = nullptr;             // [nel][40]
  double* S = nullptr;             // [36][nv] the assembled operator as a vertex stencil: entry
                                   // (o * 4 + 2 c + c') of vertex v couples (v, c) with (v + offset o, c')
  float* S32 = nullptr;            // [36][nv] the same rounded to FP32 (the cycle's copy with mg_operator LEAD)
  float *invd32 = nullptr, *mask32 = nullptr;   // [n] FP32 copies for the FP32 cycle (which keeps its
                                                // vectors x, b, q, d in the FP64 buffers)
  double* mask = nullptr;          // [n] 0 on supported DOFs, else 1
  double* invd = nullptr;          // [n] inverse diagonal, 0 on supported DOFs
  double *x = nullptr, *b = nullptr, *q = nullptr, *d = nullptr;   // [n] cycle vectors
  double* xa = nullptr;            // [n] the other x of the fused smoothing steps (ping-pong)
};

// A captured chunk of CG iterations, replayed until convergence.
struct GraphKey {
  size_t tsize;
  const void* x;
  const void* r;
  int pc;                  // preconditioner (MTO_PREC_*)
  int deg;                 // multigrid smoothing degree
  int nrm;
  const double* ref;
  double tol2;
  int chunk;
  int timing;
  int prec;
  bool operator==(const GraphKey& o) const {
    return tsize == o.tsize && x == o.x && r == o.r && pc == o.pc && deg == o.deg && nrm == o.nrm && ref == o.ref &&
           tol2 == o.tol2 && chunk == o.chunk && timing == o.timing && prec == o.prec;
  }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  std::vector<Timing::Pending> events;   // event pairs recorded on every replay
  int64_t launches_per_replay = 0;
  int64_t captured_launches = 0;
};


}  // namespace mto

struct mto_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;        // the handle's own non-blocking stream (all device work)
  cudaStream_t user_stream = nullptr;   // the caller's stream, ordered with `stream` by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::string err;
  int64_t launches = 0;
  int64_t bytes = 0;
  mto::Timing timing;

  // mesh
  int nelx = 0, nely = 0;
  double hx = 1.0, hy = 1.0;
  int64_t nel = 0, n_nodes = 0, ndof = 0, design_len = 0;
  std::vector<int> p_host, d_host;
  std::vector<int64_t> design_off_host;
  std::vector<int> pH, pV;                     // edge orders
  std::vector<int64_t> h_base, v_base, i_base; // first global node of each edge / cell interior
  std::vector<int64_t> fixed_host;
  bool have_setup = false, have_supports = false;
  int built_precision = -1;
  double k0_nu = -2.0;                         // nu of the current subcell tables

  // device tables
  int* p_d = nullptr;
  int* d_d = nullptr;
  int64_t* design_off_d = nullptr;
  mto::Constraint* cons_d = nullptr;
  int n_cons = 0;
  mto::PClass pc[mto::kPMaxTab + 1];
  std::vector<mto::BClass> bc;
  std::vector<mto::BClass> bc_qr;              // (p+1, d) tables for the QR indicator
  mto::QRTab qr[mto::kPMaxTab + 1];
  int* slot_d = nullptr;                       // [nel] slot of each element within its order class
  int64_t* fixed_d = nullptr;                  // [n_fixed] supported DOFs
  int64_t n_fixed = 0;
  double* filt_W = nullptr;                    // [design_len] density-filter weight sums (adjoint)
  double* oc_t = nullptr;                      // [4][design_len] OC: rho_j B_j^eta and the area-scaled T, L, H
  int64_t* spring_dof_d = nullptr;             // [n_springs] DOFs with a spring to ground (K + k e e^T)
  double* spring_k_d = nullptr;                // [n_springs] their stiffness
  int n_springs = 0;
  int64_t base_bytes = 0;                      // device bytes held independently of the mesh

  // solver workspace
  double* diag64 = nullptr;  // assembled diagonal
  double* invd64 = nullptr;  // inverse diagonal, 0 on supported DOFs
  float* invd32 = nullptr;
  double *r64 = nullptr, *p64 = nullptr, *s64 = nullptr, *u64 = nullptr, *w64 = nullptr;
  float *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *s32 = nullptr, *u32 = nullptr, *w32 = nullptr;
  // CG reductions: 8 slots (r^T z, p^T K p, r^T r, r^T D^-1 r, each by iteration parity) of up to
  // 8 launches; launch j of slot k stores block partials at cg_part + k*cg_stride + j*cg_class_stride,
  // its result at cg_res[8k + j], and counts finished blocks in cg_cnt[8k + j] (zero between launches)
  double* cg_part = nullptr;
  int64_t cg_class_stride = 0, cg_stride = 0;
  double* cg_res = nullptr;                    // [64]
  unsigned* cg_cnt = nullptr;                  // [64]
  int* cg_base = nullptr;                      // first iteration of the running chunk
  bool schwarz_valid = false;
  bool inner_split = false;                    // operator applies use the split pair (mixed inner solves)
  int op_kernel_cls[mto::kPMaxTab + 1] = {-2, -2, -2, -2, -2, -2, -2, -2};   // per order class (autotuner);
                                               // -2: the handle-wide choice below
  int op_kernel = -1;                          // split operator, n_e <= 32: 0 register pipeline, 1 bulk-copy
                                               // staging, 2 the generic per-chunk kernel, -1 by the size
                                               // of the class's rows
  // multigrid preconditioner: levels 1.. (Q1), fine-level transfer tables and work vectors
  std::vector<mto::MGLevel> mg;
  bool mg_ok = false, mg_valid = false;
  std::string mg_why;                          // why no hierarchy exists (mesh does not coarsen)
  int* mg_pidx = nullptr;                      // [n_nodes][4] Q1 vertices of each fine node
  double* mg_pw = nullptr;                     // [n_nodes][4] their bilinear weights
  int* mg_rptr = nullptr;                      // [nv + 1] restriction CSR by vertex
  int* mg_rnode = nullptr;
  double* mg_rw = nullptr;
  double* mg_btab = nullptr;                   // bilinear weights at the GLL nodes, per order
  int mg_boff[mto::kPMaxTab + 2] = {0};
  double *mg_v0 = nullptr, *mg_q0 = nullptr, *mg_d0 = nullptr;   // [ndof] fine-level scratch
  double* mg_Ainv = nullptr;                   // coarsest level: two [N][N] buffers of the
  double* mg_Awork = nullptr;                  // Gauss-Jordan steps ...
  double* mg_Acur = nullptr;                   // ... and the one holding the inverse
  double* mg_lmax = nullptr;                   // [levels] Chebyshev upper bounds
  double2* mg_coef = nullptr;                  // [levels][16] Chebyshev step coefficients (c1, c2)
  double* mg_part = nullptr;                   // reduction partials
  unsigned* mg_cnt = nullptr;
  double* mg_res = nullptr;
  int build_path = MTO_BUILD_TENSOR;
  bool use_graphs = true;
  bool solve_log = false;                      // MTO_SOLVE_LOG=1: one stderr line per refinement step
  double mg_ratio = 0.0;                       // MTO_MG_RATIO: Chebyshev interval lmax / ratio .. lmax (0: 100)
  int mg_q1deg = 0;                            // MTO_MG_Q1DEG: smoothing degree on the Q1 levels (0: 4)
  bool mg_lead = true;   // mg_operator: the cycle of a mixed build on FP32 copies with FP32 vectors
  float* mg_f32 = nullptr;   // [6][ndof] the FP32 cycle's level-0 vectors b, x, q, d, v and invd
  int mg_smoother = 0;                         // fine-level smoothing: MTO_SMOOTH_JACOBI or MTO_SMOOTH_BLOCK
  bool mg_block = false;                       // element-block smoothing in use (set by mg_build)
  std::vector<mto::GraphEntry*> graphs;
  double* red = nullptr;                       // misc reduction scratch [64]
  double* eng = nullptr;                       // CG energy log of the compliance-accuracy test [128]
  int* flags = nullptr;                        // [0] iterations when done, [1] error code, [2..] misc
  int* host_flags = nullptr;                   // pinned host mirror of flags[0..1]
  double* host_pinned = nullptr;               // pinned host mirror for small read-backs [64]
  unsigned long long* sel = nullptr;           // selection / small integer scratch [256]
  void* basis_tab = nullptr;                   // GLL / Gauss tables for the indicator kernels
  double* edge_buf = nullptr;                  // [n_edges + nel] Kelly edge terms, then QR scratch
  int64_t n_edges = 0;
  int* ibuf = nullptr;                         // integer scratch [4 * nel]
  double* dbuf = nullptr;                      // double scratch [2 * nel]
};

// ------------------------------------------------------------------------------------------
// Shared helpers
// ------------------------------------------------------------------------------------------
#define MTO_TRY(expr)                                \
  do {                                               \
    mto_status _s = (expr);                          \
    if (_s != MTO_OK) return _s;                     \
  } while (0)

mto_status mto_fail(mto_handle h, mto_status s, const std::string& msg);
mto_status mto_cuda_check(mto_handle h, cudaError_t e, const char* what);
mto_status mto_after_launch(mto_handle h, const char* what);

// Orders an entry point's work after the caller's stream and the caller's stream after it.
struct StreamJoin {
  mto_handle h;
  explicit StreamJoin(mto_handle h_);
  ~StreamJoin();
};

// Event bracket around the launches of one kernel family on h->stream (no-op when timing is off).
struct TimedScope {
  mto_handle h;
  int fam;
  int64_t launches0;
  cudaEvent_t a = nullptr;
  TimedScope(mto_handle h_, int fam_);
  ~TimedScope();
};
void timing_harvest(mto_handle h);   // call after the stream has been synchronised
void graph_timing_harvest(mto_handle h, mto::GraphEntry* g);
mto::GraphEntry* find_graph(mto_handle h, const mto::GraphKey& k);
mto::GraphEntry* new_graph(mto_handle h, const mto::GraphKey& k);
void clear_graphs(mto_handle h);

template <typename T>
mto_status mto_alloc(mto_handle h, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return MTO_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return mto_fail(h, MTO_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  h->bytes += (int64_t)(count * sizeof(T));
  return MTO_OK;
}

inline int grid_for(int64_t n, int block, int cap = 152 * 16) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------------------------------------
// Finite-element basis on the device (one-time table construction; FP64)
// ------------------------------------------------------------------------------------------
namespace mto {

// Legendre P_n and P_{n-1} at x by the three-term recurrence.
__host__ __device__ inline void legendre_pair(int n, double x, double* pn, double* pn1) {
  double a = 1.0, b = x;  // P_0, P_1
  if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  *pn = b;
  *pn1 = a;
}

// The p+1 Gauss-Lobatto-Legendre nodes (end points and roots of P_p'), ascending.  Newton's
// method on (1 - x^2) P_p'(x) written through the identity (1 - x^2) P_p' = p (P_{p-1} - x P_p),
// started from the Chebyshev-Gauss-Lobatto points; then symmetrised.
__host__ __device__ inline void gll_nodes(int p, double* z) {
  for (int k = 0; k <= p; ++k) {
    double x = -cos(3.14159265358979323846 * k / p);
    if (k > 0 && k < p) {
      for (int it = 0; it < 100; ++it) {
        double pn, pn1;
        legendre_pair(p, x, &pn, &pn1);
        // f(x) = P_{p-1} - x P_p  (proportional to (1-x^2) P_p'), f'(x) = -(p+1) P_p
        double f = pn1 - x * pn;
        double df = -(p + 1) * pn;
        double dx = f / df;
        x -= dx;
        if (fabs(dx) < 1e-17) break;
      }
    }
    z[k] = x;
  }
  for (int k = 0; k <= p / 2; ++k) {
    double s = 0.5 * (z[p - k] - z[k]);
    z[k] = -s;
    z[p - k] = s;
  }
  if (p % 2 == 0) z[p / 2] = 0.0;
}

// n-point Gauss-Legendre rule on [-1, 1]: Newton's method on P_n from cos(pi (k + 3/4)/(n + 1/2)),
// weights 2 / ((1 - x^2) P_n'(x)^2).  Ascending nodes.
__host__ __device__ inline void gauss_rule(int n, double* x, double* w) {
  for (int k = 0; k < n; ++k) {
    double t = cos(3.14159265358979323846 * (k + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre_pair(n, t, &pn, &pn1);
      dp = n * (t * pn - pn1) / (t * t - 1.0);
      double dt = pn / dp;
      t -= dt;
      if (fabs(dt) < 1e-17) break;
    }
    double pn, pn1;
    legendre_pair(n, t, &pn, &pn1);
    dp = n * (t * pn - pn1) / (t * t - 1.0);
    x[n - 1 - k] = t;
    w[n - 1 - k] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
  for (int k = 0; k < n / 2; ++k) {
    double s = 0.5 * (x[n - 1 - k] - x[k]);
    double ww = 0.5 * (w[n - 1 - k] + w[k]);
    x[k] = -s; x[n - 1 - k] = s;
    w[k] = ww; w[n - 1 - k] = ww;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Lagrange polynomial l_k on nodes z[0..n1-1] and its derivative, at x.
__host__ __device__ inline double lagrange_val(const double* z, int n1, int k, double x) {
  double v = 1.0;
  for (int j = 0; j < n1; ++j)
    if (j != k) v *= (x - z[j]) / (z[k] - z[j]);
  return v;
}

__host__ __device__ inline double lagrange_der(const double* z, int n1, int k, double x) {
  double s = 0.0;
  for (int i = 0; i < n1; ++i) {
    if (i == k) continue;
    double t = 1.0 / (z[k] - z[i]);
    for (int j = 0; j < n1; ++j)
      if (j != k && j != i) t *= (x - z[j]) / (z[k] - z[j]);
    s += t;
  }
  return s;
}

// Row-major packed index of (i, j), i <= j, in an n x n upper triangle.
__host__ __device__ inline int packed_index(int n, int i, int j) {
  return i * n - i * (i - 1) / 2 + (j - i);
}

// Entry at row position `pos` (see PClass::dpos) of the element matrix in slot `slot`, as a double:
// from the FP64 matrices when present, else from the split-precision pair (hi + lo).
__device__ __forceinline__ double k_entry(const double* __restrict__ K64, const float* __restrict__ Kh,
                                          const float* __restrict__ Kl, int L, int slot, int pos) {
  const size_t o = (size_t)slot * L + pos;
  if (K64) return K64[o];
  return (double)Kh[o] + (double)Kl[o];
}

// Order-preserving map of a double to an unsigned 64-bit key (for radix selection).
__host__ __device__ inline unsigned long long order_key(double v) {
  unsigned long long u;
  memcpy(&u, &v, 8);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}

}  // namespace mto

// ------------------------------------------------------------------------------------------
// Entry points of the kernel translation units (host wrappers that enqueue on h->stream)
// ------------------------------------------------------------------------------------------
namespace mto {
// fe.cu
mto_status build_tables(mto_handle h);                                  // K0 for all classes, QR tables
// sens.cu (tables)
mto_status build_sens_tables(mto_handle h);
mto_status build_elements(mto_handle h, const double* rho, const mto_material* m, int precision);
mto_status build_diagonal(mto_handle h, int precision);
mto_status element_matrix(mto_handle h, int64_t e, double* host_out);
mto_status element_matrix_split(mto_handle h, int64_t e, float* hi, float* lo);
mto_status build_schwarz(mto_handle h);                                 // element-block preconditioner
// mto_api.cu: (node, weight) list of local node (a, b) of element e (minimum-rule constraints)
int local_node_map_public(mto_handle h, int64_t e, int a, int b, int64_t* nodes, double* w);
// mg.cu (multigrid preconditioner)
mto_status mg_setup(mto_handle h);                                      // hierarchy, transfer tables
mto_status mg_set_masks(mto_handle h);                                  // supports on every level
mto_status mg_build(mto_handle h);                                      // Galerkin operators, bounds
mto_status mg_select_smoother(mto_handle h, int smoother);              // MTO_SMOOTH_* for next solves
mto_status mg_vcycle(mto_handle h, const double* r, double* z, int degree, const int* done, double* dot_part,
                     unsigned* dot_cnt, double* dot_res);
void mg_release(mto_handle h);
// tc.cu
mto_status tc_tables(mto_handle h);
mto_status tc_build_class(mto_handle h, const BClass& b, const double* rho, const mto_material* m, int precision);
int ebe_blocks(int p, int n);                                           // grid of one operator launch
// apply.cu
mto_status apply64(mto_handle h, const double* x, double* y);        // y += K x (FP64 vectors)
mto_status apply_operator(mto_handle h, int op, const double* x, double* y, double* xKx);   // mto_apply_operator
mto_status autotune_operator(mto_handle h, int32_t* choice, double* us);                   // mto_autotune
// same, early exit; lead: of the split pair the FP32 leading part alone (MTO_MIXED builds)
mto_status apply_fine(mto_handle h, const double* x, double* y, const int* done, bool lead = false);
mto_status mg_select_operator(mto_handle h, int op);   // mg_operator of mto_solve_opts
mto_status apply_block(mto_handle h, const double* x, double* y, const int* done, bool lead = false);  // element blocks
// the same on FP32 vectors with the leading part (the FP32 multigrid cycle)
mto_status apply_fine32(mto_handle h, const float* x, float* y, const int* done);
mto_status apply_block32(mto_handle h, const float* x, float* y, const int* done);
mto_status apply_q1(mto_handle h, const MGLevel& l, const double* x, double* y, const int* done);
mto_status solve(mto_handle h, const double* f, double* u, const mto_solve_opts* o, int32_t* iters,
                 double* relres);
mto_status solve_batched(mto_handle* hs, int n, const double* const* f, double* const* u, const mto_solve_opts* o,
                         int32_t* iters, double* relres, mto_status* status);
// sens.cu
// filter.cu
mto_status density_filter(mto_handle h, double R, const double* x, double* out, bool adjoint);
mto_status transfer_design(mto_handle h, const int* d_old_host, const double* rho_old, double* rho_new);
mto_status sensitivity_adjoint(mto_handle h, const double* u, const double* v, const double* rho,
                               const mto_material* m, double* dc);
mto_status sensitivity(mto_handle h, const double* u, const double* f, const double* rho,
                       const mto_material* m, int precision, double* dc, double* C);
// ind.cu
mto_status indicators(mto_handle h, const double* u, const double* rho, const mto_material* m,
                      const mto_indicator_opts* o, double* ga, double* gd, double* eqr, int32_t* pn,
                      int32_t* dn, int8_t* th);
mto_status map_update(mto_handle h, const double* ga, const double* gd, const double* eqr,
                      const mto_indicator_opts* o, int32_t* pn, int32_t* dn, int8_t* th);
mto_status oc_update(mto_handle h, const double* rho, const double* dc, double volfrac, double move,
                     double eta, double* rho_new, double* lambda);
// reductions shared by several units
mto_status dot64(mto_handle h, const double* a, const double* b, int64_t n, double* out_dev);
mto_status sum64(mto_handle h, const double* a, int64_t n, double* out_dev);
// sens.cu
mto_status compliance_energy(mto_handle h, const double* u, const double* f, const double* rho,
                             const mto_material* m, double* C);
}  // namespace mto
