// Multigrid preconditioner for the PCG of step (b).  The paper does not name its solver; on the
// binary 0/1 designs of these workloads (stiffness contrast 1e9) one-level preconditioners need
// tens of thousands of iterations, and their count grows with the mesh, so the solve is
// preconditioned by one V-cycle of an element-based Galerkin multigrid:
//
//   level 0   the order-p element operator itself (minimum-rule conforming, any p map);
//   level 1   bilinear Q1 on the same mesh.  Its element matrices are the exact Galerkin products
//             N_e^T K_e N_e, N_e = bilinear interpolation of the four vertex values at the
//             element's GLL nodes: a Q1 field is continuous and lies in every element's space, so
//             the element-wise products assemble to P^T K P for the global prolongation P;
//   level l+1 2x2 agglomeration of level l: K_E = sum_c J_c^T K_c J_c with J_c the bilinear
//             interpolation of the coarse element's vertices at its child's vertices (again the
//             exact Galerkin operator, because bilinear coarse fields are bilinear on the children);
//   coarsest  a dense inverse (at most 2048 DOFs; coarsening stops at the first grid that small,
//             since one dense mat-vec costs less than the launches of two more levels).
//
// Smoothing: Chebyshev polynomials of the Jacobi-scaled operator on [lmax / 100, lmax], lmax from
// a power iteration (x 1.1), the same polynomial before and after the coarse correction, so the
// cycle is a symmetric positive definite preconditioner.  Supported DOFs are masked on every level
// (they coincide with vertices of the coarser grids for the clamped edge and the MBB supports; the
// fine-level mask is applied to every transfer).  With FP64 matrices, or a mixed build with
// mg_operator SPLIT, every level keeps FP64 vectors and level 0 applies the built matrices (FP64
// or the split pair).  A mixed build otherwise runs the cycle on FP32 copies: FP32 vectors on
// every level, the FP32 leading part of the split pair on level 0, FP32 stencils on the Q1 levels,
// FP32 arithmetic in the level kernels; the coarsest inverse and the reductions stay FP64.  A
// preconditioner only has to be a fixed operator; the outer PCG keeps the split pair and FP64
// vectors, and its residuals are refined in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "mto_internal.cuh"

namespace mto {
namespace {

constexpr int kCoarseTarget = 2048;   // stop coarsening at or below this many DOFs
constexpr int kCoarseMax = 2048;      // largest coarsest grid for the dense inverse
constexpr double kChebRatio = 100.0;  // lmin = lmax / ratio (100 cut the iterations of the 1024 x 512
                                      // beam by a third against 30, at the same smoothing cost)
constexpr int kPowerIts = 30;
constexpr int kCoarseDegree = 4;      // Chebyshev degree on the Q1 levels (the fine level: the option)
constexpr int kMaxDegree = 16;        // largest smoothing degree (coefficient table size)
constexpr int kMGBlocks = 152 * 8;    // vector kernels: one full wave of 8 blocks per SM

// the cycle runs on FP32 copies with FP32 vectors (mixed builds, mg_operator LEAD or AUTO)
bool mg_fp32_cycle(mto_handle h) { return h->mg_lead && h->built_precision == MTO_MIXED; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double; valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = l < (int)((blockDim.x + 31) >> 5) ? part[l] : 0.0;
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

// Entry K[i][j] of an element row in the circulant-diagonal layout (n_e = ne).
__device__ __forceinline__ int circ_pos(int i, int j, int ne) {
  int k = j - i;
  if (k < 0) k += ne;
  if (2 * k <= ne) return k * ne + i;
  return (ne - k) * ne + j;
}

// ---------------------------------------------------------------- Galerkin operators
// Level 1 from the order-PO elements: K1 = N^T K_e N per element (one thread per element).
// The component blocks separate: K1[2V1+c1][2V2+c2] = sum_{a,b} B[a][V1] K_e[2a+c1][2b+c2] B[b][V2].
template <int PO>
__global__ void __launch_bounds__(128) mg_galerkin_p_kernel(int n, const int* __restrict__ elem, int L,
                                                            const double* __restrict__ K64,
                                                            const float* __restrict__ Kh,
                                                            const float* __restrict__ Kl,
                                                            const double* __restrict__ B,
                                                            double* __restrict__ K1) {
  constexpr int NN = (PO + 1) * (PO + 1), NE = 2 * NN;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const size_t row = (size_t)k * L;
  double acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  for (int a = 0; a < NN; ++a) {
    double ba[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) ba[v] = B[a * 4 + v];
#pragma unroll
    for (int c1 = 0; c1 < 2; ++c1) {
      const int i = 2 * a + c1;
      double t[2][4];
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int v = 0; v < 4; ++v) t[c2][v] = 0.0;
      for (int b = 0; b < NN; ++b) {
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          const int pos = circ_pos(i, 2 * b + c2, NE);
          const double kij = K64 ? K64[row + pos] : (double)Kh[row + pos] + (double)Kl[row + pos];
#pragma unroll
          for (int v = 0; v < 4; ++v) t[c2][v] = fma(kij, B[b * 4 + v], t[c2][v]);
        }
      }
#pragma unroll
      for (int v1 = 0; v1 < 4; ++v1)
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
          for (int v2 = 0; v2 < 4; ++v2) acc[2 * v1 + c1][2 * v2 + c2] = fma(ba[v1], t[c2][v2], acc[2 * v1 + c1][2 * v2 + c2]);
    }
  }
  const int e = elem[k];
  double* out = K1 + (size_t)e * 40;
#pragma unroll
  for (int kk = 0; kk <= 4; ++kk)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = (i + kk) & 7;
      out[kk * 8 + i] = 0.5 * (acc[i][j] + acc[j][i]);
    }
}

// Level l+1 from level l: K_E = sum over the 2x2 children of J_c^T K_c J_c (one thread per coarse
// element).  Child vertex (vx, vy) of child (cx, cy) sits at ((cx + vx) / 2, (cy + vy) / 2) of the
// coarse element; coarse vertex (X, Y) has weight (X ? s : 1 - s) (Y ? t : 1 - t) there.
__global__ void __launch_bounds__(128) mg_galerkin_h_kernel(int nxc, int nyc, int nxf, const double* __restrict__ Kf,
                                                            double* __restrict__ Kc) {
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= nxc * nyc) return;
  const int EX = E % nxc, EY = E / nxc;
  double acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  for (int cy = 0; cy < 2; ++cy)
    for (int cx = 0; cx < 2; ++cx) {
      const double* kc = Kf + (size_t)((2 * EY + cy) * nxf + 2 * EX + cx) * 40;
      double J[4][4];   // [child vertex][coarse vertex]
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double s = 0.5 * (cx + (v & 1)), t = 0.5 * (cy + (v >> 1));
#pragma unroll
        for (int V = 0; V < 4; ++V) J[v][V] = ((V & 1) ? s : 1.0 - s) * ((V >> 1) ? t : 1.0 - t);
      }
      double K[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) K[i][j] = kc[circ_pos(i, j, 8)];
#pragma unroll
      for (int c1 = 0; c1 < 2; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          double T[4][4];   // [child vertex v1][coarse vertex V2] = sum_v2 K[2v1+c1][2v2+c2] J[v2][V2]
#pragma unroll
          for (int v1 = 0; v1 < 4; ++v1)
#pragma unroll
            for (int V2 = 0; V2 < 4; ++V2) {
              double t = 0.0;
#pragma unroll
              for (int v2 = 0; v2 < 4; ++v2) t = fma(K[2 * v1 + c1][2 * v2 + c2], J[v2][V2], t);
              T[v1][V2] = t;
            }
#pragma unroll
          for (int V1 = 0; V1 < 4; ++V1)
#pragma unroll
            for (int V2 = 0; V2 < 4; ++V2) {
              double t = 0.0;
#pragma unroll
              for (int v1 = 0; v1 < 4; ++v1) t = fma(J[v1][V1], T[v1][V2], t);
              acc[2 * V1 + c1][2 * V2 + c2] += t;
            }
        }
    }
  double* out = Kc + (size_t)E * 40;
#pragma unroll
  for (int kk = 0; kk <= 4; ++kk)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = (i + kk) & 7;
      out[kk * 8 + i] = 0.5 * (acc[i][j] + acc[j][i]);
    }
}

// The assembled operator of a Q1 level as a stencil per vertex, from the element matrices: vertex
// v = (i, j) couples with the vertices (i + di, j + dj), di, dj in {-1, 0, 1} (offset o =
// 3 (dj + 1) + di + 1), through a 2 x 2 block per offset.  One thread per vertex gathers the
// contributions of its (up to four) elements in a fixed order, so no atomics; the stencil is
// stored offset-major ([36][nv]) for coalesced reads in the apply, in FP64 and rounded to FP32.
__global__ void __launch_bounds__(256) mg_stencil_kernel(int nx, int ny, const double* __restrict__ K,
                                                         double* __restrict__ S, float* __restrict__ S32) {
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % (nx + 1)), j = (int)(v / (nx + 1));
    double acc[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) acc[k] = 0.0;
    for (int ey = j - 1; ey <= j; ++ey) {
      if (ey < 0 || ey >= ny) continue;
      for (int ex = i - 1; ex <= i; ++ex) {
        if (ex < 0 || ex >= nx) continue;
        const double* ke = K + (size_t)(ey * nx + ex) * 40;
        const int a = (i - ex) + 2 * (j - ey);   // local vertex of v (x fastest)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int o = 3 * (ey + (b >> 1) - j + 1) + (ex + (b & 1) - i + 1);
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2) acc[o * 4 + 2 * c + c2] += ke[circ_pos(2 * a + c, 2 * b + c2, 8)];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 36; ++k) {
      S[(size_t)k * nv + v] = acc[k];
      S32[(size_t)k * nv + v] = (float)acc[k];
    }
  }
}

// y = A x on a Q1 level by its vertex stencil (gather only; every DOF, supported ones included):
// FP64 stencil and arithmetic, or (TS = float, the cycle's FP32 copy) the stencil rounded to FP32
// with x rounded to FP32 and FP32 products and sums (36 FP64 FMAs per vertex would make the apply
// bound by GB300's FP64 pipes rather than by memory)
template <typename TS, typename V>
__global__ void __launch_bounds__(256) mg_stencil_apply_kernel(int nx, int ny, const TS* __restrict__ S,
                                                               const V* __restrict__ x, V* __restrict__ y,
                                                               const int* __restrict__ done) {
  if (done && *done) return;
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % (nx + 1)), j = (int)(v / (nx + 1));
    TS y0 = 0, y1 = 0;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        const int ii = i + di, jj = j + dj;
        if (ii < 0 || ii > nx || jj < 0 || jj > ny) continue;
        const int o = 3 * (dj + 1) + di + 1;
        const size_t w = 2 * ((size_t)jj * (nx + 1) + ii);
        const TS x0 = (TS)x[w], x1 = (TS)x[w + 1];
        y0 = fma(S[(size_t)(o * 4 + 0) * nv + v], x0, y0);
        y0 = fma(S[(size_t)(o * 4 + 1) * nv + v], x1, y0);
        y1 = fma(S[(size_t)(o * 4 + 2) * nv + v], x0, y1);
        y1 = fma(S[(size_t)(o * 4 + 3) * nv + v], x1, y1);
      }
    }
    y[2 * v] = (V)y0;
    y[2 * v + 1] = (V)y1;
  }
}

// One Chebyshev step on a Q1 level with q = A x formed in place by the vertex stencil (the apply and
// the update of mg_cheb_kernel in one pass): reads x from xin, writes the updated x to xout (the
// level's two x buffers alternate, so no vertex reads a neighbour's new value), d in place.
// xzero: x = 0 before the step (A x = 0, xin not read).  Stencil and arithmetic as in
// mg_stencil_apply_kernel.
template <typename TS, typename V>
__global__ void __launch_bounds__(256) mg_stencil_cheb_kernel(int nx, int ny, const TS* __restrict__ S,
                                                              const V* __restrict__ xin, V* __restrict__ xout,
                                                              const V* __restrict__ b, const V* __restrict__ invd,
                                                              V* __restrict__ d, const double2* __restrict__ coef,
                                                              int step, int xzero, const int* __restrict__ done) {
  if (done && *done) return;
  const double2 cc = coef[step];
  const V c1 = (V)cc.x, c2 = (V)cc.y;
  const int64_t nv = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % (nx + 1)), j = (int)(v / (nx + 1));
    TS y0 = 0, y1 = 0;
    if (!xzero) {
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int ii = i + di, jj = j + dj;
          if (ii < 0 || ii > nx || jj < 0 || jj > ny) continue;
          const int o = 3 * (dj + 1) + di + 1;
          const size_t w = 2 * ((size_t)jj * (nx + 1) + ii);
          const TS x0 = (TS)xin[w], x1 = (TS)xin[w + 1];
          y0 = fma(S[(size_t)(o * 4 + 0) * nv + v], x0, y0);
          y0 = fma(S[(size_t)(o * 4 + 1) * nv + v], x1, y0);
          y1 = fma(S[(size_t)(o * 4 + 2) * nv + v], x0, y1);
          y1 = fma(S[(size_t)(o * 4 + 3) * nv + v], x1, y1);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const size_t k = 2 * (size_t)v + c;
      const V r = invd[k] * (b[k] - (V)(c ? y1 : y0));
      const V dn = step > 0 ? fma(c1, d[k], c2 * r) : c2 * r;
      d[k] = dn;
      xout[k] = (xzero ? V(0) : xin[k]) + dn;
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(256) mg_copy_kernel(int64_t n, const V* __restrict__ a, V* __restrict__ b,
                                                      const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// assembled diagonal of a Q1 level (atomics), then the masked inverse
__global__ void mg_diag_kernel(int nel, const int* __restrict__ gmap, const double* __restrict__ K,
                               double* __restrict__ diag) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) atomicAdd(diag + 2 * (size_t)gmap[4 * e + (i >> 1)] + (i & 1), K[(size_t)e * 40 + i]);
}

__global__ void mg_invd_kernel(int64_t n, const double* __restrict__ mask, double* __restrict__ diag_inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double dg = diag_inv[i];
    diag_inv[i] = (mask[i] != 0.0 && dg > 0.0) ? 1.0 / dg : 0.0;
  }
}

// coarsest level: dense assembly, supported rows/columns replaced by identity, in-place
// Gauss-Jordan inversion (SPD: no pivoting) in one block
__global__ void mg_dense_assemble_kernel(int nel, int N, const int* __restrict__ gmap, const double* __restrict__ K,
                                         double* __restrict__ A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  for (int i = 0; i < 8; ++i) {
    const int gi = 2 * gmap[4 * e + (i >> 1)] + (i & 1);
    for (int j = 0; j < 8; ++j) {
      const int gj = 2 * gmap[4 * e + (j >> 1)] + (j & 1);
      atomicAdd(A + (size_t)gi * N + gj, K[(size_t)e * 40 + circ_pos(i, j, 8)]);
    }
  }
}

__global__ void mg_dense_fix_kernel(int N, const double* __restrict__ mask, double* __restrict__ A) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / N), j = (int)(t % N);
    if (mask[i] == 0.0 || mask[j] == 0.0) A[t] = (i == j) ? 1.0 : 0.0;
  }
}

// One Gauss-Jordan step of the in-place inversion (SPD: no pivoting), from buffer A into B so that
// every entry is computed from the previous step's values; N launches invert the matrix.
__global__ void __launch_bounds__(256) mg_gj_step_kernel(int N, int k, const double* __restrict__ A,
                                                         double* __restrict__ B, int* __restrict__ err) {
  const double piv = A[(size_t)k * N + k];
  if (!(piv > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = MTO_ENAN;
  }
  const double inv = 1.0 / piv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)N * N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / N), j = (int)(t - (int64_t)i * N);
    double v;
    if (i == k) v = (j == k) ? inv : A[(size_t)k * N + j] * inv;
    else if (j == k) v = -A[(size_t)i * N + k] * inv;
    else v = fma(-A[(size_t)i * N + k] * inv, A[(size_t)k * N + j], A[t]);
    B[t] = v;
  }
}

// x = Ainv b (one warp per row; FP64 inverse and sums, vectors of the cycle's type)
template <typename V>
__global__ void __launch_bounds__(256) mg_coarse_solve_kernel(int N, const double* __restrict__ Ainv,
                                                              const V* __restrict__ b, V* __restrict__ x,
                                                              const int* __restrict__ done) {
  if (done && *done) return;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, l = threadIdx.x & 31;
  if (w >= N) return;
  double s = 0.0;
  for (int j = l; j < N; j += 32) s = fma(Ainv[(size_t)w * N + j], (double)b[j], s);
  s = warp_sum(s);
  if (l == 0) x[w] = (V)s;
}

// ---------------------------------------------------------------- smoothing and transfers
// The cycle's vectors are of type V: double, or float for the cycle on FP32 copies (mixed builds,
// mg_operator LEAD), where the level kernels then also compute in FP32.
//
// One Chebyshev step on level vectors: r = D^-1 (b - q) (q = A x, then cleared), step 0:
// d = r / theta, step s > 0: d = rho_s rho_{s-1} d + (2 rho_s / delta) r; x = d (xzero) or x += d.
// With dpart set, also b^T x of the updated x (the PCG's r^T z after the cycle's last step),
// reduced by the last block to finish in index order into *dres.  With zout set (the FP32
// cycle's last step), the updated x goes to the FP64 output zout instead of x and the reduction
// takes its b from bout (FP64).
template <typename V>
__global__ void __launch_bounds__(256) mg_cheb_kernel(int64_t n, const V* __restrict__ b, V* __restrict__ q,
                                                      const V* __restrict__ invd, V* __restrict__ x,
                                                      V* __restrict__ d, const double2* __restrict__ coef,
                                                      int step, int xzero, const int* __restrict__ done,
                                                      double* __restrict__ dpart, unsigned* __restrict__ dcnt,
                                                      double* __restrict__ dres, int given, int zq,
                                                      double* __restrict__ zout, const double* __restrict__ bout) {
  if (done && *done) return;
  const double2 cc = coef[step];   // (c1, c2), precomputed per level
  const V c1 = (V)cc.x, c2 = (V)cc.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const V bi = b[i];
    // given: q already holds the preconditioned residual (element-block smoothing), else the
    // Jacobi-scaled residual is formed here from q = A x
    const V r = given ? (invd[i] != V(0) ? q[i] : V(0)) : invd[i] * (bi - q[i]);
    if (zq) q[i] = V(0);   // else a separate launch clears q (see mg_zero_kernel)
    const V dn = step > 0 ? fma(c1, d[i], c2 * r) : c2 * r;   // c1 = 0 at step 0
    d[i] = dn;
    const V xn = xzero ? dn : x[i] + dn;
    if (zout) {
      zout[i] = (double)xn;
      acc = fma(bout[i], (double)xn, acc);
    } else {
      x[i] = xn;
      acc = fma((double)bi, (double)xn, acc);
    }
  }
  if (!dpart) return;
  __shared__ int last;
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    dpart[blockIdx.x] = acc;
    __threadfence();
    last = (atomicAdd(dcnt, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(dpart + i);
    t = block_sum(t);
    if (threadIdx.x == 0) {
      *dres = t;
      *dcnt = 0u;
    }
  }
}

// element-block smoothing: w = b - q on free DOFs (0 on supports); q is cleared by the next launch
template <typename V>
__global__ void __launch_bounds__(256) mg_block_resid_kernel(int64_t n, const V* __restrict__ b,
                                                             const V* __restrict__ q, const V* __restrict__ invd,
                                                             V* __restrict__ w, const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = invd[i] != V(0) ? (b ? b[i] : V(0)) - q[i] : V(0);
}

// v = 0 as its own launch: on GB300 a kernel that reads an array and stores zeros into it streams
// at about a third of the rate of the same kernel without that store (see zero_kernel in apply.cu),
// so the large accumulators are cleared separately
template <typename V>
__global__ void __launch_bounds__(256) mg_zero_kernel(int64_t n, V* __restrict__ v, const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = V(0);
}

// the FP32 cycle's entry: b32 = r (rounded), its level-0 vectors' FP32 copy of the inverse diagonal
__global__ void __launch_bounds__(256) mg_demote_kernel(int64_t n, const double* __restrict__ r, float* __restrict__ b,
                                                        const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)r[i];
}

__global__ void __launch_bounds__(256) mg_round_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// accumulators of at least this many entries are cleared by mg_zero_kernel (smaller ones, which stay
// in L2, by the consuming kernel itself)
constexpr int64_t kSeparateZero = 1 << 20;

// level 0 -> 1: b1 = P^T r by the vertex-wise transposed table, the residual r = b - q formed on
// the fly on free DOFs (q = A x stays; the prolongation clears it)
template <typename V>
__global__ void __launch_bounds__(256) mg_restrict0_kernel(int64_t nv, const int* __restrict__ ptr,
                                                           const int* __restrict__ node, const double* __restrict__ w,
                                                           const V* __restrict__ b, const V* __restrict__ q,
                                                           const V* __restrict__ invd, const V* __restrict__ mask,
                                                           V* __restrict__ b1, const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    V s0 = V(0), s1 = V(0);
    for (int k = ptr[v]; k < ptr[v + 1]; ++k) {
      const V wk = (V)w[k];
      const size_t g = 2 * (size_t)node[k];
      if (invd[g] != V(0)) s0 = fma(wk, b[g] - q[g], s0);
      if (invd[g + 1] != V(0)) s1 = fma(wk, b[g + 1] - q[g + 1], s1);
    }
    b1[2 * v] = mask[2 * v] * s0;
    b1[2 * v + 1] = mask[2 * v + 1] * s1;
  }
}

// level 1 -> 0: x += P x1 on free DOFs; q (A x of the pre-smoothed x) cleared
template <typename V>
__global__ void __launch_bounds__(256) mg_prolong0_kernel(int64_t nn, const int* __restrict__ idx,
                                                          const double* __restrict__ w, const V* __restrict__ x1,
                                                          const V* __restrict__ invd, V* __restrict__ x,
                                                          V* __restrict__ q, const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nn; g += (int64_t)gridDim.x * blockDim.x) {
    V s0 = V(0), s1 = V(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const V wk = (V)w[4 * g + k];
      const size_t v = 2 * (size_t)idx[4 * g + k];
      s0 = fma(wk, x1[v], s0);
      s1 = fma(wk, x1[v + 1], s1);
    }
    if (invd[2 * g] != V(0)) x[2 * g] += s0;
    if (invd[2 * g + 1] != V(0)) x[2 * g + 1] += s1;
    q[2 * g] = V(0);
    q[2 * g + 1] = V(0);
  }
}

// level l -> l+1 on vertex grids (full weighting: the transpose of bilinear interpolation) of the
// residual r = b - q formed on the fly on free DOFs (q stays; the prolongation clears it)
template <typename V>
__global__ void __launch_bounds__(256) mg_restrict_h_kernel(int nxc, int nyc, int nxf, int nyf,
                                                            const V* __restrict__ b, const V* __restrict__ q,
                                                            const V* __restrict__ invd, const V* __restrict__ mask,
                                                            V* __restrict__ bc, const int* __restrict__ done) {
  if (done && *done) return;
  const int64_t nvc = (int64_t)(nxc + 1) * (nyc + 1);
  for (int64_t Vx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; Vx < nvc; Vx += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(Vx % (nxc + 1)), J = (int)(Vx / (nxc + 1));
    V s0 = V(0), s1 = V(0);
    for (int dy = -1; dy <= 1; ++dy) {
      const int j = 2 * J + dy;
      if (j < 0 || j > nyf) continue;
      const V wy = dy == 0 ? V(1) : V(0.5);
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = 2 * I + dx;
        if (i < 0 || i > nxf) continue;
        const V wgt = wy * (dx == 0 ? V(1) : V(0.5));
        const size_t f = 2 * ((size_t)j * (nxf + 1) + i);
        if (invd[f] != V(0)) s0 = fma(wgt, b[f] - q[f], s0);
        if (invd[f + 1] != V(0)) s1 = fma(wgt, b[f + 1] - q[f + 1], s1);
      }
    }
    bc[2 * Vx] = mask[2 * Vx] * s0;
    bc[2 * Vx + 1] = mask[2 * Vx + 1] * s1;
  }
}

// level l+1 -> l: x += bilinear interpolation of the coarse correction (free DOFs); q cleared
template <typename V>
__global__ void __launch_bounds__(256) mg_prolong_h_kernel(int nxc, int nxf, int nyf, const V* __restrict__ xc,
                                                           const V* __restrict__ mask, V* __restrict__ xf,
                                                           V* __restrict__ q, const int* __restrict__ done) {
  if (done && *done) return;
  const int64_t nvf = (int64_t)(nxf + 1) * (nyf + 1);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvf; v += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % (nxf + 1)), j = (int)(v / (nxf + 1));
    const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
    const V wi = (i & 1) ? V(0.5) : V(1), wj = (j & 1) ? V(0.5) : V(1);
    V s0 = V(0), s1 = V(0);
    const int is[2] = {i0, i1}, js[2] = {j0, j1};
    const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1;
    for (int b = 0; b < nj; ++b)
      for (int a = 0; a < ni; ++a) {
        const size_t c = 2 * ((size_t)js[b] * (nxc + 1) + is[a]);
        s0 = fma(wi * wj, xc[c], s0);
        s1 = fma(wi * wj, xc[c + 1], s1);
      }
    xf[2 * v] += mask[2 * v] * s0;
    xf[2 * v + 1] += mask[2 * v + 1] * s1;
    q[2 * v] = V(0);
    q[2 * v + 1] = V(0);
  }
}

// ---------------------------------------------------------------- power iteration for lmax
__global__ void mg_pow_init_kernel(int64_t n, const double* __restrict__ invd, double* __restrict__ v,
                                   double* __restrict__ q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t hsh = (uint32_t)(i * 2654435761ull);
    v[i] = invd[i] != 0.0 ? 1.0 + (double)(hsh >> 8) * (1.0 / 16777216.0) : 0.0;
    q[i] = 0.0;
  }
}

// w = D^-1 q (q cleared), ||w||^2 reduced by the last block into *res
__global__ void __launch_bounds__(256) mg_pow_step_kernel(int64_t n, double* __restrict__ q,
                                                          const double* __restrict__ invd, double* __restrict__ w,
                                                          double* __restrict__ part, unsigned* __restrict__ cnt,
                                                          double* __restrict__ res, int given) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = given ? (invd[i] != 0.0 ? q[i] : 0.0) : invd[i] * q[i];
    q[i] = 0.0;
    w[i] = wi;
    s += wi * wi;
  }
  __shared__ int last;
  s = block_sum(s);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last = (atomicAdd(cnt, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(part + i);
    t = block_sum(t);
    if (threadIdx.x == 0) {
      *res = t;
      *cnt = 0u;
    }
  }
}

// v = w / ||w||
__global__ void mg_pow_norm_kernel(int64_t n, const double* __restrict__ w, const double* __restrict__ res,
                                   double* __restrict__ v) {
  const double sc = 1.0 / sqrt(__ldcg(res));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * sc;
}

__global__ void mg_pow_final_kernel(const double* __restrict__ res, double* __restrict__ lmax) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *lmax = 1.1 * sqrt(__ldcg(res));
}

// Chebyshev step coefficients of every level from its bound (one thread per level): step 0
// d = r / theta; step s > 0 d = rho_s rho_{s-1} d + (2 rho_s / delta) r, rho_0 = 1 / sigma,
// rho_s = 1 / (2 sigma - rho_{s-1}), theta, delta the centre and half-width of [lmax / ratio, lmax].
__global__ void mg_cheb_coef_kernel(int nlev, const double* __restrict__ lmax, double ratio, double2* __restrict__ coef) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlev) return;
  const double lm = lmax[l], lo = lm / ratio;
  const double th = 0.5 * (lm + lo), de = 0.5 * (lm - lo), sg = th / de;
  double2* c = coef + (size_t)l * kMaxDegree;
  c[0] = make_double2(0.0, 1.0 / th);
  double rp = 1.0 / sg;
  for (int s = 1; s < kMaxDegree; ++s) {
    const double rc = 1.0 / (2.0 * sg - rp);
    c[s] = make_double2(rc * rp, 2.0 * rc / de);
    rp = rc;
  }
}

int vec_grid(int64_t n) { return grid_for(n, 256, kMGBlocks); }

}  // namespace

// ---------------------------------------------------------------- host side
void mg_release(mto_handle h) {
  for (auto& l : h->mg)
    for (void* p : {(void*)l.gmap, (void*)l.K, (void*)l.S, (void*)l.S32, (void*)l.invd32, (void*)l.mask32, (void*)l.xa,
                    (void*)l.mask, (void*)l.invd, (void*)l.x, (void*)l.b,
                    (void*)l.q, (void*)l.d})
      cudaFree(p);
  h->mg.clear();
  for (void* p : {(void*)h->mg_pidx, (void*)h->mg_pw, (void*)h->mg_rptr, (void*)h->mg_rnode, (void*)h->mg_rw,
                  (void*)h->mg_btab, (void*)h->mg_v0, (void*)h->mg_q0, (void*)h->mg_d0, (void*)h->mg_f32,
                  (void*)h->mg_Ainv,
                  (void*)h->mg_Awork,
                  (void*)h->mg_lmax, (void*)h->mg_coef, (void*)h->mg_part, (void*)h->mg_cnt, (void*)h->mg_res})
    cudaFree(p);
  h->mg_pidx = nullptr;
  h->mg_pw = h->mg_rw = h->mg_btab = h->mg_v0 = h->mg_q0 = h->mg_d0 = h->mg_Ainv = h->mg_lmax = nullptr;
  h->mg_f32 = nullptr;
  h->mg_Awork = h->mg_Acur = nullptr;
  h->mg_coef = nullptr;
  h->mg_part = h->mg_res = nullptr;
  h->mg_rptr = h->mg_rnode = nullptr;
  h->mg_cnt = nullptr;
  h->mg_ok = h->mg_valid = false;
}

// Level sizes, vertex maps and the level-0 <-> level-1 transfer tables (host, once per mesh).
mto_status mg_setup(mto_handle h) {
  mg_release(h);
  int nx = h->nelx, ny = h->nely;
  std::vector<std::pair<int, int>> dims{{nx, ny}};
  while (nx % 2 == 0 && ny % 2 == 0 && 2LL * (nx + 1) * (ny + 1) > kCoarseTarget) {
    nx /= 2;
    ny /= 2;
    dims.push_back({nx, ny});
  }
  const int64_t ncoarse = 2LL * (nx + 1) * (ny + 1);
  if (ncoarse > kCoarseMax) {
    h->mg_why = "multigrid needs mesh sides that halve down to a grid of at most 2048 DOFs (" +
                std::to_string(nx) + " x " + std::to_string(ny) + " elements cannot be halved)";
    return MTO_OK;
  }
  h->mg.resize(dims.size());
  for (size_t l = 0; l < dims.size(); ++l) {
    MGLevel& L = h->mg[l];
    L.nx = dims[l].first;
    L.ny = dims[l].second;
    L.nel = L.nx * L.ny;
    L.nv = (int64_t)(L.nx + 1) * (L.ny + 1);
    L.n = 2 * L.nv;
    std::vector<int> gm((size_t)4 * L.nel);
    for (int e = 0; e < L.nel; ++e) {
      const int ex = e % L.nx, ey = e / L.nx;
      const int v0 = ey * (L.nx + 1) + ex;
      gm[4 * e + 0] = v0;
      gm[4 * e + 1] = v0 + 1;
      gm[4 * e + 2] = v0 + L.nx + 1;
      gm[4 * e + 3] = v0 + L.nx + 2;
    }
    MTO_TRY(mto_alloc(h, &L.gmap, gm.size()));
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(L.gmap, gm.data(), gm.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
    MTO_TRY(mto_alloc(h, &L.K, (size_t)40 * L.nel));
    if (l + 1 < dims.size()) {   // smoothed levels
      MTO_TRY(mto_alloc(h, &L.S, (size_t)36 * L.nv));
      MTO_TRY(mto_alloc(h, &L.S32, (size_t)36 * L.nv));
    }
    for (double** v : {&L.mask, &L.invd, &L.x, &L.xa, &L.b, &L.q, &L.d}) MTO_TRY(mto_alloc(h, v, L.n));
    for (float** v : {&L.invd32, &L.mask32}) MTO_TRY(mto_alloc(h, v, L.n));
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(L.q, 0, L.n * sizeof(double), h->stream), "memset"));
  }

  // bilinear weights of the four vertices at the GLL nodes of each order (node (a, b), x fastest)
  std::vector<double> btab;
  for (int p = 1; p <= kPMaxTab; ++p) {
    h->mg_boff[p] = (int)btab.size();
    double z[kPMaxTab + 2];
    gll_nodes(p, z);
    for (int b = 0; b <= p; ++b)
      for (int a = 0; a <= p; ++a) {
        const double s = 0.5 * (1.0 + z[a]), t = 0.5 * (1.0 + z[b]);
        for (int V = 0; V < 4; ++V) btab.push_back(((V & 1) ? s : 1.0 - s) * ((V >> 1) ? t : 1.0 - t));
      }
  }
  MTO_TRY(mto_alloc(h, &h->mg_btab, btab.size()));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_btab, btab.data(), btab.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));

  // prolongation level 1 -> 0: every global node takes the bilinear interpolant of the vertices
  // of an element in which it is a free (unconstrained) local node
  const int64_t nn = h->n_nodes;
  std::vector<int> pidx((size_t)4 * nn, 0);
  std::vector<double> pw((size_t)4 * nn, 0.0);
  std::vector<char> seen(nn, 0);
  for (int64_t e = 0; e < h->nel; ++e) {
    const int p = h->p_host[e];
    const int ex = (int)(e % h->nelx), ey = (int)(e / h->nelx);
    const int v0 = ey * (h->nelx + 1) + ex;
    const int vs[4] = {v0, v0 + 1, v0 + h->nelx + 1, v0 + h->nelx + 2};
    for (int b = 0; b <= p; ++b)
      for (int a = 0; a <= p; ++a) {
        int64_t nodes[kConsMax];
        double w[kConsMax];
        if (local_node_map_public(h, e, a, b, nodes, w) != 1) continue;
        const int64_t g = nodes[0];
        if (seen[g]) continue;
        seen[g] = 1;
        const double* bw = btab.data() + h->mg_boff[p] + 4 * (b * (p + 1) + a);
        for (int V = 0; V < 4; ++V) {
          pidx[4 * g + V] = vs[V];
          pw[4 * g + V] = bw[V];
        }
      }
  }
  for (int64_t g = 0; g < nn; ++g)
    if (!seen[g]) return mto_fail(h, MTO_EINVAL, "mg_setup: a node belongs to no element as a free node");
  // restriction: the transpose, by vertex (exact zero weights dropped)
  const int64_t nv = h->mg[0].nv;
  std::vector<int> rptr(nv + 1, 0);
  for (int64_t g = 0; g < nn; ++g)
    for (int V = 0; V < 4; ++V)
      if (pw[4 * g + V] != 0.0) ++rptr[pidx[4 * g + V] + 1];
  for (int64_t v = 0; v < nv; ++v) rptr[v + 1] += rptr[v];
  std::vector<int> rnode(rptr[nv]);
  std::vector<double> rw(rptr[nv]);
  std::vector<int> fill(rptr.begin(), rptr.end() - 1);
  for (int64_t g = 0; g < nn; ++g)
    for (int V = 0; V < 4; ++V)
      if (pw[4 * g + V] != 0.0) {
        const int v = pidx[4 * g + V];
        rnode[fill[v]] = (int)g;
        rw[fill[v]] = pw[4 * g + V];
        ++fill[v];
      }
  MTO_TRY(mto_alloc(h, &h->mg_pidx, pidx.size()));
  MTO_TRY(mto_alloc(h, &h->mg_pw, pw.size()));
  MTO_TRY(mto_alloc(h, &h->mg_rptr, rptr.size()));
  MTO_TRY(mto_alloc(h, &h->mg_rnode, rnode.size()));
  MTO_TRY(mto_alloc(h, &h->mg_rw, rw.size()));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_pidx, pidx.data(), pidx.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_pw, pw.data(), pw.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_rptr, rptr.data(), rptr.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_rnode, rnode.data(), rnode.size() * sizeof(int), cudaMemcpyHostToDevice), "upload"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(h->mg_rw, rw.data(), rw.size() * sizeof(double), cudaMemcpyHostToDevice), "upload"));

  for (double** v : {&h->mg_v0, &h->mg_q0, &h->mg_d0}) MTO_TRY(mto_alloc(h, v, h->ndof));
  MTO_TRY(mto_alloc(h, &h->mg_f32, (size_t)6 * h->ndof));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_q0, 0, h->ndof * sizeof(double), h->stream), "memset"));
  MTO_TRY(mto_alloc(h, &h->mg_Ainv, (size_t)ncoarse * ncoarse));
  MTO_TRY(mto_alloc(h, &h->mg_Awork, (size_t)ncoarse * ncoarse));
  MTO_TRY(mto_alloc(h, &h->mg_lmax, h->mg.size() + 1));
  MTO_TRY(mto_alloc(h, &h->mg_coef, (h->mg.size() + 1) * kMaxDegree));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_lmax, 0, (h->mg.size() + 1) * sizeof(double), h->stream), "memset"));
  MTO_TRY(mto_alloc(h, &h->mg_part, kMGBlocks));
  MTO_TRY(mto_alloc(h, &h->mg_cnt, 8));
  MTO_TRY(mto_alloc(h, &h->mg_res, 8));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_cnt, 0, 8 * sizeof(unsigned), h->stream), "memset"));
  h->mg_ok = true;
  h->mg_valid = false;
  return MTO_OK;
}

// Supports on every level: level 1 takes the fine mask of the vertex DOFs (vertices come first
// in the global numbering), level l+1 the mask of the coinciding level-l vertex.
mto_status mg_set_masks(mto_handle h) {
  if (!h->mg_ok) return MTO_OK;
  std::vector<char> fixed(h->ndof, 0);
  for (int64_t g : h->fixed_host) fixed[g] = 1;
  std::vector<double> m(h->mg[0].n);
  for (int64_t i = 0; i < h->mg[0].n; ++i) m[i] = fixed[i] ? 0.0 : 1.0;
  for (size_t l = 0; l < h->mg.size(); ++l) {
    const MGLevel& L = h->mg[l];
    if (l > 0) {
      const MGLevel& F = h->mg[l - 1];
      std::vector<double> mc(L.n);
      for (int J = 0; J <= L.ny; ++J)
        for (int I = 0; I <= L.nx; ++I) {
          const int64_t V = (int64_t)J * (L.nx + 1) + I, v = (int64_t)(2 * J) * (F.nx + 1) + 2 * I;
          mc[2 * V] = m[2 * v];
          mc[2 * V + 1] = m[2 * v + 1];
        }
      m.swap(mc);
    }
    MTO_TRY(mto_cuda_check(h, cudaMemcpy(L.mask, m.data(), L.n * sizeof(double), cudaMemcpyHostToDevice), "upload"));
  }
  h->mg_valid = false;
  return MTO_OK;
}

namespace {

// y = A x on Q1 level l (written, not accumulated): the vertex stencil where it exists, in FP32
// when the cycle runs on FP32 copies (FP32 vectors in the cycle, FP64 ones in the power
// iteration), else in FP64; the coarsest level (no stencil) by its element matrices
mto_status mg_level_apply(mto_handle h, const MGLevel& l, const double* x, double* y, const int* done) {
  if (!l.S) return apply_q1(h, l, x, y, done);
  if (mg_fp32_cycle(h))
    mg_stencil_apply_kernel<float, double><<<vec_grid(l.nv), 256, 0, h->stream>>>(l.nx, l.ny, l.S32, x, y, done);
  else
    mg_stencil_apply_kernel<double, double><<<vec_grid(l.nv), 256, 0, h->stream>>>(l.nx, l.ny, l.S, x, y, done);
  return mto_after_launch(h, "mg_stencil_apply_kernel");
}
mto_status mg_level_apply(mto_handle h, const MGLevel& l, const float* x, float* y, const int* done) {
  if (!l.S32) return mto_fail(h, MTO_EINVAL, "mg: no stencil on this level");
  mg_stencil_apply_kernel<float, float><<<vec_grid(l.nv), 256, 0, h->stream>>>(l.nx, l.ny, l.S32, x, y, done);
  return mto_after_launch(h, "mg_stencil_apply_kernel");
}

// one fused Chebyshev step on a smoothed Q1 level (FP64 stencil in the FP64 cycle, FP32 in the FP32 one)
mto_status mg_level_cheb(mto_handle h, const MGLevel& l, const double* xin, double* xout, const double* b,
                         const double* invd, double* d, const double2* cf, int step, bool xzero, const int* done) {
  mg_stencil_cheb_kernel<double, double><<<vec_grid(l.nv), 256, 0, h->stream>>>(l.nx, l.ny, l.S, xin, xout, b, invd,
                                                                                d, cf, step, xzero, done);
  return mto_after_launch(h, "mg_stencil_cheb_kernel");
}
mto_status mg_level_cheb(mto_handle h, const MGLevel& l, const float* xin, float* xout, const float* b,
                         const float* invd, float* d, const double2* cf, int step, bool xzero, const int* done) {
  mg_stencil_cheb_kernel<float, float><<<vec_grid(l.nv), 256, 0, h->stream>>>(l.nx, l.ny, l.S32, xin, xout, b, invd,
                                                                              d, cf, step, xzero, done);
  return mto_after_launch(h, "mg_stencil_cheb_kernel");
}

// lmax of D^-1 A on one level by power iteration (level < 0: the fine operator)
mto_status mg_power(mto_handle h, int level, double* lmax_out) {
  const bool fine = level < 0;
  const int64_t n = fine ? h->ndof : h->mg[level].n;
  const double* invd = fine ? h->invd64 : h->mg[level].invd;
  double* v = fine ? h->mg_v0 : h->mg[level].x;
  double* q = fine ? h->mg_q0 : h->mg[level].q;
  double* w = fine ? h->mg_d0 : h->mg[level].d;
  const int grd = vec_grid(n);
  mg_pow_init_kernel<<<grd, 256, 0, h->stream>>>(n, invd, v, q);
  MTO_TRY(mto_after_launch(h, "mg_pow_init_kernel"));
  const bool block = fine && h->mg_block;   // lmax of M^-1 A, M^-1 the element-block inverse
  for (int it = 0; it < kPowerIts; ++it) {
    if (fine) MTO_TRY(apply_fine(h, v, q, nullptr, h->mg_lead));
    else MTO_TRY(mg_level_apply(h, h->mg[level], v, q, nullptr));
    if (block) {
      mg_block_resid_kernel<double><<<grd, 256, 0, h->stream>>>(n, nullptr, q, invd, w, nullptr);   // w = -A v
      MTO_TRY(mto_after_launch(h, "mg_block_resid_kernel"));
      mg_zero_kernel<double><<<grd, 256, 0, h->stream>>>(n, q, nullptr);
      MTO_TRY(mto_after_launch(h, "mg_zero_kernel"));
      MTO_TRY(apply_block(h, w, q, nullptr, h->mg_lead));
    }
    mg_pow_step_kernel<<<grd, 256, 0, h->stream>>>(n, q, invd, w, h->mg_part, h->mg_cnt, h->mg_res, block);
    MTO_TRY(mto_after_launch(h, "mg_pow_step_kernel"));
    if (it + 1 < kPowerIts) {
      mg_pow_norm_kernel<<<grd, 256, 0, h->stream>>>(n, w, h->mg_res, v);
      MTO_TRY(mto_after_launch(h, "mg_pow_norm_kernel"));
    }
  }
  mg_pow_final_kernel<<<1, 32, 0, h->stream>>>(h->mg_res, lmax_out);
  return mto_after_launch(h, "mg_pow_final_kernel");
}

}  // namespace

// The fine level's smoothing for the next solves: a change rebuilds the Chebyshev bounds (lazily)
// and drops the captured iteration graphs.
mto_status mg_select_smoother(mto_handle h, int smoother) {
  if (smoother != MTO_SMOOTH_JACOBI && smoother != MTO_SMOOTH_BLOCK)
    return mto_fail(h, MTO_EINVAL, "mto_solve: bad mg_smoother");
  if (smoother == h->mg_smoother) return MTO_OK;
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_solve"));
  h->mg_smoother = smoother;
  h->mg_valid = false;
  clear_graphs(h);
  return MTO_OK;
}

// The copy of the matrices the cycle applies with the MTO_MIXED build (FP32 copies and FP32
// vectors, or the split pair and FP64 stencils with FP64 vectors); a change rebuilds the bounds and
// drops the graphs.  AUTO takes the FP32 cycle with point-Jacobi smoothing only: the FP32
// rounding of the element blocks' inverses (K_e + Delta_e)^-1 can make them indefinite on binary
// designs (measured: corrections that did not converge on 6 of 64 binary instances, which the split
// pair and the Jacobi-smoothed FP32 cycle solved), so the element-block smoother keeps the split
// pair unless LEAD is asked for.  The smoother is selected first.
mto_status mg_select_operator(mto_handle h, int op) {
  if (op != MTO_MG_OP_AUTO && op != MTO_MG_OP_SPLIT && op != MTO_MG_OP_LEAD)
    return mto_fail(h, MTO_EINVAL, "mto_solve: bad mg_operator");
  const bool lead = op == MTO_MG_OP_LEAD || (op == MTO_MG_OP_AUTO && h->mg_smoother == MTO_SMOOTH_JACOBI);
  if (lead == h->mg_lead) return MTO_OK;
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mto_solve"));
  h->mg_lead = lead;
  h->mg_valid = false;
  clear_graphs(h);
  return MTO_OK;
}

// Galerkin operators of every level, diagonals, Chebyshev bounds and the coarsest inverse, for the
// element matrices of the last build (lazily, at the first multigrid solve after a build).
mto_status mg_build(mto_handle h) {
  if (!h->mg_ok) return mto_fail(h, MTO_EINVAL, h->mg_why.empty() ? "multigrid unavailable" : h->mg_why);
  {
  TimedScope ts(h, F_PRECOND);
  MGLevel& L1 = h->mg[0];
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    const PClass& c = h->pc[p];
    if (c.n == 0) continue;
    const double* B = h->mg_btab + h->mg_boff[p];
    const double* K64 = c.K64;   // both builds keep the FP64 matrices
    const int grd = (c.n + 127) / 128;
    switch (p) {
      case 1: mg_galerkin_p_kernel<1><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
      case 2: mg_galerkin_p_kernel<2><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
      case 3: mg_galerkin_p_kernel<3><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
      case 4: mg_galerkin_p_kernel<4><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
      case 5: mg_galerkin_p_kernel<5><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
      case 6: mg_galerkin_p_kernel<6><<<grd, 128, 0, h->stream>>>(c.n, c.elem, c.L, K64, c.K32, c.K32lo, B, L1.K); break;
    }
    MTO_TRY(mto_after_launch(h, "mg_galerkin_p_kernel"));
  }
  for (size_t l = 1; l < h->mg.size(); ++l) {
    const MGLevel& F = h->mg[l - 1];
    MGLevel& C = h->mg[l];
    mg_galerkin_h_kernel<<<(C.nel + 127) / 128, 128, 0, h->stream>>>(C.nx, C.ny, F.nx, F.K, C.K);
    MTO_TRY(mto_after_launch(h, "mg_galerkin_h_kernel"));
  }
  for (auto& L : h->mg) {
    if (L.S) {
      mg_stencil_kernel<<<vec_grid(L.nv), 256, 0, h->stream>>>(L.nx, L.ny, L.K, L.S, L.S32);
      MTO_TRY(mto_after_launch(h, "mg_stencil_kernel"));
    }
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(L.invd, 0, L.n * sizeof(double), h->stream), "memset"));
    mg_diag_kernel<<<(L.nel + 127) / 128, 128, 0, h->stream>>>(L.nel, L.gmap, L.K, L.invd);
    MTO_TRY(mto_after_launch(h, "mg_diag_kernel"));
    mg_invd_kernel<<<vec_grid(L.n), 256, 0, h->stream>>>(L.n, L.mask, L.invd);
    MTO_TRY(mto_after_launch(h, "mg_invd_kernel"));
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(L.q, 0, L.n * sizeof(double), h->stream), "memset"));
  }
  // coarsest: dense inverse
  const MGLevel& C = h->mg.back();
  const int N = (int)C.n;
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_Ainv, 0, sizeof(double) * N * N, h->stream), "memset"));
  mg_dense_assemble_kernel<<<(C.nel + 127) / 128, 128, 0, h->stream>>>(C.nel, N, C.gmap, C.K, h->mg_Ainv);
  MTO_TRY(mto_after_launch(h, "mg_dense_assemble_kernel"));
  mg_dense_fix_kernel<<<vec_grid((int64_t)N * N), 256, 0, h->stream>>>(N, C.mask, h->mg_Ainv);
  MTO_TRY(mto_after_launch(h, "mg_dense_fix_kernel"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->flags + 6, 0, sizeof(int), h->stream), "memset"));
  {
    double* bufs[2] = {h->mg_Ainv, h->mg_Awork};
    const int grd = vec_grid((int64_t)N * N);
    for (int k = 0; k < N; ++k) {
      mg_gj_step_kernel<<<grd, 256, 0, h->stream>>>(N, k, bufs[k & 1], bufs[(k + 1) & 1], h->flags + 6);
      MTO_TRY(mto_after_launch(h, "mg_gj_step_kernel"));
    }
    h->mg_Acur = bufs[N & 1];
  }
  }
  // element-block smoothing of the fine level: the blocks (K_e + Delta_e)^-1 of the element-block
  // preconditioner
  h->mg_block = h->mg_smoother == 1;
  if (h->mg_block && !h->schwarz_valid) MTO_TRY(build_schwarz(h));
  // Chebyshev bounds: fine level first, then every smoothed Q1 level
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_q0, 0, h->ndof * sizeof(double), h->stream), "memset"));
  MTO_TRY(mg_power(h, -1, h->mg_lmax));
  for (size_t l = 0; l + 1 < h->mg.size(); ++l) MTO_TRY(mg_power(h, (int)l, h->mg_lmax + 1 + l));
  mg_cheb_coef_kernel<<<1, 32, 0, h->stream>>>((int)h->mg.size(), h->mg_lmax, h->mg_ratio > 1.0 ? h->mg_ratio : kChebRatio,
                                               h->mg_coef);
  MTO_TRY(mto_after_launch(h, "mg_cheb_coef_kernel"));
  for (auto& L : h->mg) MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(L.q, 0, L.n * sizeof(double), h->stream), "memset"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_q0, 0, h->ndof * sizeof(double), h->stream), "memset"));
  // FP32 copies of the masks and inverse diagonals for the FP32 cycle; its level-0 vectors cleared
  for (auto& L : h->mg) {
    mg_round_kernel<<<vec_grid(L.n), 256, 0, h->stream>>>(L.n, L.invd, L.invd32);
    MTO_TRY(mto_after_launch(h, "mg_round_kernel"));
    mg_round_kernel<<<vec_grid(L.n), 256, 0, h->stream>>>(L.n, L.mask, L.mask32);
    MTO_TRY(mto_after_launch(h, "mg_round_kernel"));
  }
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_f32, 0, 5 * h->ndof * sizeof(float), h->stream), "memset"));
  mg_round_kernel<<<vec_grid(h->ndof), 256, 0, h->stream>>>(h->ndof, h->invd64, h->mg_f32 + 5 * h->ndof);
  MTO_TRY(mto_after_launch(h, "mg_round_kernel"));
  int err = 0;
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_flags + 8, h->flags + 6, sizeof(int), cudaMemcpyDeviceToHost,
                                            h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "mg_build"));
  err = h->host_flags[8];
  if (err) return mto_fail(h, MTO_ENAN, "mg_build: coarsest operator not positive definite");
  h->mg_valid = true;
  return MTO_OK;
}

namespace {

// the level vectors in the cycle's type (the FP32 cycle keeps its FP32 vectors in the FP64 buffers)
template <typename V>
struct LevelV {
  V *x, *b, *q, *d, *xa;
  const V *invd, *mask;
};
template <typename V>
LevelV<V> level_vecs(const MGLevel& L);
template <>
LevelV<double> level_vecs<double>(const MGLevel& L) {
  return {L.x, L.b, L.q, L.d, L.xa, L.invd, L.mask};
}
template <>
LevelV<float> level_vecs<float>(const MGLevel& L) {
  return {reinterpret_cast<float*>(L.x), reinterpret_cast<float*>(L.b), reinterpret_cast<float*>(L.q),
          reinterpret_cast<float*>(L.d), reinterpret_cast<float*>(L.xa), L.invd32, L.mask32};
}

// y += A x (block: the element blocks) on level 0 in the cycle's vector type
mto_status fine_apply(mto_handle h, const double* x, double* y, const int* done, bool lead, bool block) {
  return block ? apply_block(h, x, y, done, lead) : apply_fine(h, x, y, done, lead);
}
mto_status fine_apply(mto_handle h, const float* x, float* y, const int* done, bool, bool block) {
  return block ? apply_block32(h, x, y, done) : apply_fine32(h, x, y, done);
}

// One V-cycle in vector type V.  Level-0 vectors: b (the residual), x (the output), q (A x, kept
// zero between uses), d (Chebyshev direction), v (element-block scratch), invd.  With dot_part
// set, the last smoothing step also reduces b^T x into *dot_res; with zout set (the FP32 cycle),
// that step writes x to zout in FP64 and takes the reduction's b from bout.
template <typename V>
mto_status mg_cycle(mto_handle h, const V* b0, V* x0, V* q0, V* d0, V* v0, const V* invd0, int degree,
                    const int* done, double* dot_part, unsigned* dot_cnt, double* dot_res, double* zout,
                    const double* bout) {
  const int nl = (int)h->mg.size();
  const bool lead = h->mg_lead;
  auto smooth = [&](int lev, const V* b, V* x, V* q, V* d, const V* invd, int64_t n, bool pre,
                    bool last) -> mto_status {
    const int k = lev < 0 ? degree : (h->mg_q1deg > 0 ? h->mg_q1deg : kCoarseDegree);
    const double2* cf = h->mg_coef + (size_t)(lev + 1) * kMaxDegree;
    const int grd = vec_grid(n);
    if (lev >= 0) {   // Q1 level: one fused stencil + Chebyshev launch per step, x ping-ponged
      const MGLevel& L = h->mg[lev];
      V* cur = x;
      V* nxt = level_vecs<V>(L).xa;
      TimedScope ts(h, F_PRECOND);
      for (int s = 0; s < k; ++s) {
        MTO_TRY(mg_level_cheb(h, L, cur, nxt, b, invd, d, cf, s, pre && s == 0, done));
        std::swap(cur, nxt);
      }
      if (cur != x) {   // odd degree: the result is in the other buffer
        mg_copy_kernel<V><<<grd, 256, 0, h->stream>>>(n, cur, x, done);
        MTO_TRY(mto_after_launch(h, "mg_copy_kernel"));
      }
      return MTO_OK;
    }
    const bool block = h->mg_block;   // element-block (additive Schwarz) smoothing of level 0
    for (int s = 0; s < k; ++s) {
      const bool skip_apply = pre && s == 0;   // x = 0: A x = 0
      if (!skip_apply) MTO_TRY(fine_apply(h, x, q, done, lead, false));
      if (block) {   // q <- M^-1 (b - A x)
        {
          TimedScope ts(h, F_PRECOND);
          mg_block_resid_kernel<V><<<grd, 256, 0, h->stream>>>(n, b, q, invd, v0, done);
          MTO_TRY(mto_after_launch(h, "mg_block_resid_kernel"));
          mg_zero_kernel<V><<<grd, 256, 0, h->stream>>>(n, q, done);
          MTO_TRY(mto_after_launch(h, "mg_zero_kernel"));
        }
        MTO_TRY(fine_apply(h, v0, q, done, lead, true));
      }
      TimedScope ts(h, F_PRECOND);
      const bool fin = last && s == k - 1;
      const bool sep = n >= kSeparateZero;
      mg_cheb_kernel<V><<<grd, 256, 0, h->stream>>>(n, b, q, invd, x, d, cf, s, pre && s == 0, done,
                                                     fin ? dot_part : nullptr, dot_cnt, dot_res, block, !sep,
                                                     fin ? zout : nullptr, bout);
      MTO_TRY(mto_after_launch(h, "mg_cheb_kernel"));
      if (sep) {
        mg_zero_kernel<V><<<grd, 256, 0, h->stream>>>(n, q, done);
        MTO_TRY(mto_after_launch(h, "mg_zero_kernel"));
      }
    }
    return MTO_OK;
  };
  // level 0 pre-smoothing and residual
  MTO_TRY(smooth(-1, b0, x0, q0, d0, invd0, h->ndof, true, false));
  MTO_TRY(fine_apply(h, x0, q0, done, lead, false));
  {
    TimedScope ts(h, F_PRECOND);
    const LevelV<V> L1 = level_vecs<V>(h->mg[0]);
    mg_restrict0_kernel<V><<<vec_grid(h->mg[0].nv), 256, 0, h->stream>>>(
        h->mg[0].nv, h->mg_rptr, h->mg_rnode, h->mg_rw, b0, q0, invd0, L1.mask, L1.b, done);
    MTO_TRY(mto_after_launch(h, "mg_restrict0_kernel"));
  }
  // Q1 levels down
  for (int l = 0; l < nl - 1; ++l) {
    const MGLevel& L = h->mg[l];
    const MGLevel& C = h->mg[l + 1];
    const LevelV<V> lv = level_vecs<V>(L), cv = level_vecs<V>(C);
    MTO_TRY(smooth(l, lv.b, lv.x, lv.q, lv.d, lv.invd, L.n, true, false));
    TimedScope ts(h, F_PRECOND);
    MTO_TRY(mg_level_apply(h, L, lv.x, lv.q, done));
    mg_restrict_h_kernel<V><<<vec_grid(C.nv), 256, 0, h->stream>>>(C.nx, C.ny, L.nx, L.ny, lv.b, lv.q, lv.invd,
                                                                   cv.mask, cv.b, done);
    MTO_TRY(mto_after_launch(h, "mg_restrict_h_kernel"));
  }
  {
    TimedScope ts(h, F_PRECOND);
    const MGLevel& C = h->mg.back();
    const LevelV<V> cv = level_vecs<V>(C);
    mg_coarse_solve_kernel<V><<<(int)((C.n * 32 + 255) / 256), 256, 0, h->stream>>>((int)C.n, h->mg_Acur, cv.b,
                                                                                      cv.x, done);
    MTO_TRY(mto_after_launch(h, "mg_coarse_solve_kernel"));
  }
  // up
  for (int l = nl - 2; l >= 0; --l) {
    const MGLevel& L = h->mg[l];
    const MGLevel& C = h->mg[l + 1];
    const LevelV<V> lv = level_vecs<V>(L), cv = level_vecs<V>(C);
    {
      TimedScope ts(h, F_PRECOND);
      mg_prolong_h_kernel<V><<<vec_grid(L.nv), 256, 0, h->stream>>>(C.nx, L.nx, L.ny, cv.x, lv.mask, lv.x, lv.q,
                                                                     done);
      MTO_TRY(mto_after_launch(h, "mg_prolong_h_kernel"));
    }
    MTO_TRY(smooth(l, lv.b, lv.x, lv.q, lv.d, lv.invd, L.n, false, false));
  }
  {
    TimedScope ts(h, F_PRECOND);
    const LevelV<V> L1 = level_vecs<V>(h->mg[0]);
    mg_prolong0_kernel<V><<<vec_grid(h->n_nodes), 256, 0, h->stream>>>(h->n_nodes, h->mg_pidx, h->mg_pw, L1.x,
                                                                        invd0, x0, q0, done);
    MTO_TRY(mto_after_launch(h, "mg_prolong0_kernel"));
  }
  return smooth(-1, b0, x0, q0, d0, invd0, h->ndof, false, true);
}

}  // namespace

// z = M^-1 r: one V-cycle, with r^T z into *dot_res when dot_part is set (block partials in
// dot_part, counter dot_cnt).  FP64 cycle: level-0 vectors b = r, x = z, q = mg_q0, d = mg_d0,
// v = mg_v0.  FP32 cycle (the cycle on FP32 copies of a mixed build): r rounded into its own FP32
// level-0 vectors, z and r^T z written in FP64 by the last smoothing step.
mto_status mg_vcycle(mto_handle h, const double* r, double* z, int degree, const int* done, double* dot_part,
                     unsigned* dot_cnt, double* dot_res) {
  if (mg_fp32_cycle(h)) {
    const int64_t n = h->ndof;
    float* F = h->mg_f32;
    float *b = F, *x = F + n, *q = F + 2 * n, *d = F + 3 * n, *v = F + 4 * n;
    const float* invd = F + 5 * n;
    {
      TimedScope ts(h, F_PRECOND);
      mg_demote_kernel<<<vec_grid(n), 256, 0, h->stream>>>(n, r, b, done);
      MTO_TRY(mto_after_launch(h, "mg_demote_kernel"));
    }
    return mg_cycle<float>(h, b, x, q, d, v, invd, degree, done, dot_part, dot_cnt, dot_res, z, r);
  }
  return mg_cycle<double>(h, r, z, h->mg_q0, h->mg_d0, h->mg_v0, h->invd64, degree, done, dot_part, dot_cnt,
                          dot_res, nullptr, r);
}

}  // namespace mto
