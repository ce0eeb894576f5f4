// Step (b): the matrix-free operator y = sum_e P_e^T K_e P_e x and the preconditioned CG solve of
// K u = f (Eq. 1) inside FP64 iterative refinement (Jacobi, element-block Schwarz or the multigrid
// cycle of mg.cu as preconditioner).  The paper does not name its solver; conformity across
// p-jumps uses the minimum-rule prolongations P_e built by mto_setup.
//
// Operator layout: one element per group of W lanes (one warp for Q3), element matrices in the
// circulant-diagonal layout of mto_internal.cuh; see ebe_kernel.
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "mto_internal.cuh"

namespace mto {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double; result valid in thread 0.  blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
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

// Lanes per element (W), elements per warp (G) and rows per lane (M) for n_e DOFs.
template <int NE>
struct WarpShape {
  static constexpr int W = NE <= 8 ? 8 : (NE <= 16 ? 16 : 32);
  static constexpr int G = 32 / W;
  static constexpr int M = (NE + 31) / 32;
};

// Shuffle value v[reg] from lane src (all lanes take part; reg selects among the M registers).
template <int M, typename V>
__device__ __forceinline__ V shfl_sel(const V (&v)[M], int src, int reg) {
  V out = __shfl_sync(0xffffffffu, v[0], src);
#pragma unroll
  for (int m = 1; m < M; ++m) {
    V t = __shfl_sync(0xffffffffu, v[m], src);
    if (reg == m) out = t;
  }
  return out;
}

// Error-free product of the split pairs (ah + al)(xh + xl), returned as an unevaluated pair
// (pp + pe): TwoProduct of the leading terms by FMA plus the cross terms (al*xl ~ 2^-96 dropped).
template <bool kSplitX>
__device__ __forceinline__ void df_prod(float ah, float al, float xh, float xl, float& pp, float& pe) {
  pp = ah * xh;
  pe = fmaf(ah, xh, -pp);
  if (kSplitX) pe = fmaf(ah, xl, pe);
  pe = fmaf(al, xh, pe);
}

// (sh, sl) += (pp + pe), keeping the rounding error of the leading sum (TwoSum).
__device__ __forceinline__ void df_acc(float& sh, float& sl, float pp, float pe) {
  const float s = sh + pp;
  const float bv = s - sh;
  const float err = (sh - (s - bv)) + (pp - bv);
  sh = s;
  sl += err + pe;
}

// The leading (FP32) part alone, for preconditioners, which need a fixed operator but not the
// operator's accuracy: row i of the lane sums K[i][i+k] x_{i+k} and receives K[i-k][i] x_{i-k} from
// lane i-k, in plain FP32 (x rounded to FP32).  row(k) = D_k[i] of this lane (0 beyond n_e).
template <int NE, int ND, typename RowFn>
__device__ __forceinline__ float lead_rows(RowFn row, float x, int li, int gb) {
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    const float a = row(k);
    int j = li + k;
    if (j >= NE) j -= NE;
    s = fmaf(a, __shfl_sync(0xffffffffu, x, gb + j), s);
    if (k > 0 && 2 * k != NE) {
      int s2 = li - k;
      if (s2 < 0) s2 += NE;
      s += __shfl_sync(0xffffffffu, a * x, gb + s2);
    }
  }
  return s;
}

// y += sum_e P_e^T K_e P_e x, one element per lane group (W lanes; G elements per warp).
// Lane li owns rows i = li + 32 m.  Element matrices are rows of the circulant-diagonal layout:
// at step k lane i reads D_k[i] = K[i][i+k], adds K[i][i+k] x_{i+k} to its row (x_{i+k} by
// shuffle) and hands K[i][i+k] x_i to the lane owning row i+k (shuffle from the receiver's side),
// so each stored entry serves both triangles.  kDF = false: FP64 matrices and arithmetic (plain
// FP64 path).  kDF = true: the split-precision pair on the FP32 pipes with error-free products and
// sums (~48-bit accurate), vectors TX = double (refinement residuals) or float (inner iterations);
// with Kl null, the leading part alone (the lo rows taken as zero).
// A reduction output of one launch: every block stores its partial, the last block to finish
// (counted with an atomic) sums the partials in index order (deterministic) into *res and
// re-arms the counter.  Consumers read res[0 .. nres) (one scalar per launch).
struct Red {
  double* part;   // [gridDim.x]
  unsigned* cnt;
  double* res;
};

__device__ __forceinline__ void reduce_out(double v, const Red& rd) {
  __shared__ int last;
  v = block_sum(v);
  if (threadIdx.x == 0) {
    rd.part[blockIdx.x] = v;
    __threadfence();
    const unsigned t = atomicAdd(rd.cnt, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(rd.part + i);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      *rd.res = s;
      *rd.cnt = 0u;
    }
  }
}

// sum of a few launch results, same order in every thread
__device__ __forceinline__ double sum_res(const double* __restrict__ res, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += __ldcg(res + i);
  return s;
}

// Each launch reduces x^T y (= sum_e x_e^T K_e x_e) into one scalar, so CG gets its curvature
// without an extra pass and without same-address atomics on the data.  With a convergence test
// `cv` the whole launch returns once the residual norm of the previous vector update meets it,
// after block 0 records the iteration count in *done.
struct ConvTest {
  const double* res;   // residual norm^2 results (nullptr: no test)
  int n;
  const double* ref;   // reference norm^2
  double tol2;
  const int* base;     // chunk base iteration (device)
  int local;           // iteration within the chunk
  int* done;
  int* err;
  const double* eng;   // energy test (compliance accuracy) instead of the residual test: see EnergyLog
};

// Compliance-accuracy stopping test.  CG on K d = r from d = 0 gains t_i = alpha_i gamma_i of
// energy per iteration (gamma_i = r_i^T z_i), and ||d* - d_k||_K^2 = sum_{i >= k} t_i, which is
// the compliance error C* - (2 f^T u - u^T K u) of u = u_0 + d_k (Hestenes-Stiefel; the error
// estimates of Strakos and Tichy 2002).  On these problems the gains decay slowly and unevenly, so
// the remaining sum is extrapolated from the last two windows of kEnergyWin gains: with S_last,
// S_prev their sums and q = S_last / S_prev < 1, the error is taken as S_last / (1 - q) (the
// window itself plus a geometric tail); the test stops when that falls below a quarter of tol
// times the compliance estimate C(u_0) + sum_i t_i, C(u_0) = 2 f^T u_0 - u_0^T K u_0 =
// f^T u_0 + u_0^T r_0 (the quarter: measured against FP64 re-solves, the extrapolation alone
// stopped up to ~3x short of tol when the decay of the gains changed pace).
// Layout of the device array: [0] running sum, [1] C(u_0), [2 .. 2 + 2 kEnergyWin) the gains of
// the last 2 kEnergyWin iterations by iteration index, [2 + 2 kEnergyWin] the squared l2 residual
// that ends the run regardless (1e-26 ||f||^2).
constexpr int kEnergyWin = 32;
constexpr int kEnergyRing = 2 * kEnergyWin;
constexpr double kEnergySafety = 0.25;   // the gains decay unevenly: the estimate must be 4x below tol

template <int PO, bool kDF, typename TX>
__global__ void __launch_bounds__(256) ebe_kernel(const double* __restrict__ K64, const float* __restrict__ Kh,
                                                  const float* __restrict__ Kl, int L, int n,
                                                  const int* __restrict__ gmap, const Constraint* __restrict__ cons,
                                                  const TX* __restrict__ x, TX* __restrict__ y, Red red,
                                                  const int* __restrict__ done, ConvTest cv) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN, ND = NE / 2 + 1;
  constexpr int W = WarpShape<NE>::W, G = WarpShape<NE>::G, M = WarpShape<NE>::M;
  constexpr bool kSplitX = kDF && sizeof(TX) == 8;
  if (done && *done) return;
  if (cv.res) {
    const double rr = sum_res(cv.res, cv.n);
    if (!(rr > cv.tol2 * *cv.ref)) {   // converged, or a NaN residual
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!(rr == rr)) *cv.err = MTO_ENAN;
        *cv.done = *cv.base + cv.local + 1;
      }
      return;
    }
  }
  const int lane = threadIdx.x & 31;
  const int li = lane % W, gb = lane - li, gid = lane / W;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  double dot = 0.0;
  for (int base = warp * G; base < n; base += nwarps * G) {
    const int e = base + gid;
    const bool act = e < n;
    // ---- gather x_e: row i = li + 32 m is local DOF i = 2 * node + component
    double xd[M];
    int gi[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int i = li + 32 * m;
      double v = 0.0;
      int g = 0;
      if (act && i < NE) {
        g = __ldg(gmap + (size_t)e * NN + (i >> 1));
        if (g >= 0) {
          v = (double)x[2 * (size_t)g + (i & 1)];
        } else {
          const Constraint& c = cons[-g - 1];
          for (int q = 0; q < c.cnt; ++q) v += c.w[q] * (double)x[2 * (size_t)c.node[q] + (i & 1)];
        }
      }
      xd[m] = v;
      gi[m] = g;
    }
    double acc[M];         // FP64 mode
    float xh[M], xl[M], sh[M], sl[M];   // split mode
#pragma unroll
    for (int m = 0; m < M; ++m) {
      acc[m] = 0.0;
      xh[m] = (float)xd[m];
      xl[m] = kSplitX ? (float)(xd[m] - (double)xh[m]) : 0.0f;
      sh[m] = 0.0f;
      sl[m] = 0.0f;
    }
    const size_t rowb = (size_t)(act ? e : 0) * L;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const bool pair = k > 0 && 2 * k != NE;   // the entry also serves row i + k
      double tdv[M];
      float tph[M], tpe[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int i = li + 32 * m;
        const bool vi = act && i < NE;
        int j = i + k;
        if (j >= NE) j -= NE;
        const int src = gb + (j & 31), reg = j >> 5;
        if (!kDF) {
          const double a = vi ? __ldg(K64 + rowb + k * NE + i) : 0.0;
          const double xj = shfl_sel<M>(xd, src, reg);
          acc[m] = fma(a, xj, acc[m]);
          tdv[m] = a * xd[m];
        } else {
          const float ah = vi ? __ldg(Kh + rowb + k * NE + i) : 0.0f;
          const float al = (vi && Kl) ? __ldg(Kl + rowb + k * NE + i) : 0.0f;
          const float xjh = shfl_sel<M>(xh, src, reg);
          const float xjl = kSplitX ? shfl_sel<M>(xl, src, reg) : 0.0f;
          float pp, pe;
          df_prod<kSplitX>(ah, al, xjh, xjl, pp, pe);
          df_acc(sh[m], sl[m], pp, pe);
          df_prod<kSplitX>(ah, al, xh[m], xl[m], tph[m], tpe[m]);
        }
      }
      if (pair) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r = li + 32 * m;
          int s = r - k;
          if (s < 0) s += NE;
          const int src = gb + (s & 31), reg = (s >> 5) < M ? (s >> 5) : 0;
          if (!kDF) {
            acc[m] += shfl_sel<M>(tdv, src, reg);
          } else {
            const float pp = shfl_sel<M>(tph, src, reg);
            const float pe = shfl_sel<M>(tpe, src, reg);
            df_acc(sh[m], sl[m], pp, pe);
          }
        }
      }
    }
    // ---- scatter P_e^T y_e and the curvature term
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int i = li + 32 * m;
      if (!(act && i < NE)) continue;
      const double yv = kDF ? (double)sh[m] + (double)sl[m] : acc[m];
      const int g = gi[m];
      if (g >= 0) {
        atomicAdd(y + 2 * (size_t)g + (i & 1), (TX)yv);
      } else {
        const Constraint& c = cons[-g - 1];
        for (int q = 0; q < c.cnt; ++q) atomicAdd(y + 2 * (size_t)c.node[q] + (i & 1), (TX)(c.w[q] * yv));
      }
      if (red.part) dot += xd[m] * yv;
    }
  }
  if (red.part) reduce_out(dot, red);
}

// The split-precision operator for n_e <= 32 (one row per lane), software-pipelined: a persistent
// grid walks its elements with a stride, and while a warp computes one element's rows it already
// holds the next element's hi/lo rows (2 (n_e/2 + 1) registers each) and node map, so the
// element stream from L2/HBM never waits on the arithmetic.  Same arithmetic as ebe_kernel.
template <int PO, bool kLo, typename TX>
__global__ void __launch_bounds__(256, 2) ebe_df_pipe_kernel(const float* __restrict__ Kh,
                                                             const float* __restrict__ Kl, int L, int n,
                                                             const int* __restrict__ gmap,
                                                             const Constraint* __restrict__ cons,
                                                             const TX* __restrict__ x, TX* __restrict__ y, Red red,
                                                             const int* __restrict__ done) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN, ND = NE / 2 + 1;
  constexpr int W = WarpShape<NE>::W, G = WarpShape<NE>::G;
  static_assert(WarpShape<NE>::M == 1, "one row per lane");
  constexpr bool kSplitX = sizeof(TX) == 8;
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  const int li = lane % W, gb = lane - li, gid = lane / W;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int stride = nwarps * G;
  float ah[ND], al[ND];
  int gn;
  auto fetch = [&](int e, float (&h)[ND], float (&l)[ND], int& g) {
    const bool v = e < n && li < NE;
    const size_t rowb = (size_t)(v ? e : 0) * L;
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      h[k] = v ? __ldg(Kh + rowb + k * NE + li) : 0.0f;
      l[k] = (kLo && v) ? __ldg(Kl + rowb + k * NE + li) : 0.0f;
    }
    g = v ? __ldg(gmap + (size_t)e * NN + (li >> 1)) : 0;
  };
  double dot = 0.0;
  int base = warp * G;
  if (base < n) fetch(base + gid, ah, al, gn);
  for (; base < n; base += stride) {
    const int e = base + gid;
    const bool act = e < n && li < NE;
    const int g = gn;
    // gather x_e
    double xd = 0.0;
    if (act) {
      if (g >= 0) {
        xd = (double)x[2 * (size_t)g + (li & 1)];
      } else {
        const Constraint& c = cons[-g - 1];
        for (int q = 0; q < c.cnt; ++q) xd += c.w[q] * (double)x[2 * (size_t)c.node[q] + (li & 1)];
      }
    }
    // the next element's rows and node map, in flight during this element's arithmetic
    float bh[ND], bl[ND];
    int gnext = 0;
    fetch(base + stride + gid, bh, bl, gnext);
    float sh = 0.0f, sl = 0.0f;
    if constexpr (kLo) {
      const float xh = (float)xd;
      const float xl = kSplitX ? (float)(xd - (double)xh) : 0.0f;
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        int j = li + k;
        if (j >= NE) j -= NE;
        const int src = gb + j;
        const float xjh = __shfl_sync(0xffffffffu, xh, src);
        const float xjl = kSplitX ? __shfl_sync(0xffffffffu, xl, src) : 0.0f;
        float pp, pe;
        df_prod<kSplitX>(ah[k], al[k], xjh, xjl, pp, pe);
        df_acc(sh, sl, pp, pe);
        if (k > 0 && 2 * k != NE) {
          float tp, te;
          df_prod<kSplitX>(ah[k], al[k], xh, xl, tp, te);
          int s = li - k;
          if (s < 0) s += NE;
          const float rp = __shfl_sync(0xffffffffu, tp, gb + s);
          const float re = __shfl_sync(0xffffffffu, te, gb + s);
          df_acc(sh, sl, rp, re);
        }
      }
    } else {
      sh = lead_rows<NE, ND>([&](int k) { return ah[k]; }, (float)xd, li, gb);
    }
    // scatter P_e^T y_e and the curvature term
    if (act) {
      const double yv = (double)sh + (double)sl;
      if (g >= 0) {
        atomicAdd(y + 2 * (size_t)g + (li & 1), (TX)yv);
      } else {
        const Constraint& c = cons[-g - 1];
        for (int q = 0; q < c.cnt; ++q) atomicAdd(y + 2 * (size_t)c.node[q] + (li & 1), (TX)(c.w[q] * yv));
      }
      if (red.part) dot += xd * yv;
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      ah[k] = bh[k];
      al[k] = bl[k];
    }
    gn = gnext;
  }
  if (red.part) reduce_out(dot, red);
}

// ---- bulk-copy staging (TMA 1D) of element rows into shared memory
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// global -> shared bulk copy completing on `bar` (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// element groups in flight per warp (ring stages): chosen per variant in launch_ebe
constexpr int kTmaWarps = 8;      // warps per block
constexpr unsigned kWaitLimit = 1u << 24;

// The split-precision operator for n_e <= 32 with the element rows staged by bulk copies: every
// warp walks its own sequence of element groups (G elements of W lanes, G = 32 / W) and keeps
// kStages groups' hi/lo rows in its shared-memory ring (a group is refilled as soon as its
// arithmetic is done), so the row stream no longer
// depends on how many warps the registers allow.  x values run two groups ahead in registers and
// node maps two groups ahead of x.  Same arithmetic and reduction as ebe_kernel (kLo = false: the hi rows alone, staged
// and summed as in lead_rows).  Every wait is bounded: on expiry the warp records MTO_ETIMEOUT,
// waits (bounded) for its copies still in flight, and stops.
template <int PO, bool kLo, typename TX, int kStages>
__global__ void __launch_bounds__(kTmaWarps * 32) ebe_df_tma_kernel(const float* __restrict__ Kh,
                                                                    const float* __restrict__ Kl, int L, int n,
                                                                    const int* __restrict__ gmap,
                                                                    const Constraint* __restrict__ cons,
                                                                    const TX* __restrict__ x, TX* __restrict__ y,
                                                                    Red red, const int* __restrict__ done,
                                                                    int* __restrict__ err) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN, ND = NE / 2 + 1;
  constexpr int W = WarpShape<NE>::W, G = WarpShape<NE>::G;
  static_assert(WarpShape<NE>::M == 1, "one row per lane");
  constexpr bool kSplitX = sizeof(TX) == 8;
  constexpr int NM = kLo ? 2 : 1;   // matrices staged per group (hi, lo)
  extern __shared__ __align__(128) unsigned char tma_smem[];
  if (done && *done) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int li = lane % W, gb = lane - li, gid = lane / W;
  const int warp = blockIdx.x * kTmaWarps + wib;
  const int nwarps = gridDim.x * kTmaWarps;
  const int stride = nwarps * G;
  const size_t stage_floats = (size_t)G * L;   // one group's rows (hi or lo)
  float* ring = reinterpret_cast<float*>(tma_smem) + (size_t)wib * kStages * NM * stage_floats;
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<float*>(tma_smem) +
                                               (size_t)kTmaWarps * kStages * NM * stage_floats) +
                   wib * kStages;
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init1(bars + s);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int first = warp * G;
  // issue the copies of group it (base = first + it * stride) into stage it % kStages
  auto issue = [&](int it) {
    const int base = first + it * stride;
    if (base >= n) return;
    const int cnt = n - base < G ? n - base : G;
    const uint32_t bytes = (uint32_t)(cnt * L * sizeof(float));
    float* dst = ring + (size_t)(it % kStages) * NM * stage_floats;
    uint64_t* bar = bars + it % kStages;
    mbar_expect_tx(bar, NM * bytes);
    bulk_g2s(dst, Kh + (size_t)base * L, bytes, bar);
    if constexpr (kLo) bulk_g2s(dst + stage_floats, Kl + (size_t)base * L, bytes, bar);
  };
  if (lane == 0)
    for (int it = 0; it < kStages; ++it) issue(it);
  // node map and x of the current group, node map of the next
  auto load_g = [&](int e) -> int { return (e < n && li < NE) ? __ldg(gmap + (size_t)e * NN + (li >> 1)) : 0; };
  auto load_x = [&](int e, int g) -> double {
    if (!(e < n && li < NE)) return 0.0;
    if (g >= 0) return (double)x[2 * (size_t)g + (li & 1)];
    const Constraint& c = cons[-g - 1];
    double v = 0.0;
    for (int q = 0; q < c.cnt; ++q) v += c.w[q] * (double)x[2 * (size_t)c.node[q] + (li & 1)];
    return v;
  };
  // x runs two groups ahead of the arithmetic and the node maps two groups ahead of x, so every
  // gather has two groups of arithmetic to arrive in
  int g0 = load_g(first + gid), g1 = load_g(first + stride + gid);
  int g2 = load_g(first + 2 * stride + gid), g3 = load_g(first + 3 * stride + gid);
  double x0 = load_x(first + gid, g0), x1 = load_x(first + stride + gid, g1);
  double dot = 0.0;
  bool ok = true;
  int it = 0;
  for (int base = first; base < n; base += stride, ++it) {
    const int e = base + gid;
    const bool act = e < n && li < NE;
    const double x2 = load_x(e + 2 * stride, g2);
    const int g4 = load_g(e + 4 * stride);
    const int g_cur = g0;
    // wait for this group's rows
    const int st = it % kStages;
    const uint32_t parity = (uint32_t)((it / kStages) & 1);
    unsigned spins = 0;
    while (!mbar_test(bars + st, parity)) {
      if (++spins > kWaitLimit) {
        ok = false;
        break;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) break;
    const float* rh = ring + (size_t)st * NM * stage_floats + (size_t)gid * L;
    const float* rl = rh + stage_floats;
    const double xd = x0;
    float sh = 0.0f, sl = 0.0f;
    if constexpr (kLo) {
      const float xh = (float)xd;
      const float xl = kSplitX ? (float)(xd - (double)xh) : 0.0f;
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        const float ah = li < NE ? rh[k * NE + li] : 0.0f;
        const float al = li < NE ? rl[k * NE + li] : 0.0f;
        int j = li + k;
        if (j >= NE) j -= NE;
        const int src = gb + j;
        const float xjh = __shfl_sync(0xffffffffu, xh, src);
        const float xjl = kSplitX ? __shfl_sync(0xffffffffu, xl, src) : 0.0f;
        float pp, pe;
        df_prod<kSplitX>(ah, al, xjh, xjl, pp, pe);
        df_acc(sh, sl, pp, pe);
        if (k > 0 && 2 * k != NE) {
          float tp, te;
          df_prod<kSplitX>(ah, al, xh, xl, tp, te);
          int s2 = li - k;
          if (s2 < 0) s2 += NE;
          const float rp = __shfl_sync(0xffffffffu, tp, gb + s2);
          const float re = __shfl_sync(0xffffffffu, te, gb + s2);
          df_acc(sh, sl, rp, re);
        }
      }
    } else {
      sh = lead_rows<NE, ND>([&](int k) { return li < NE ? rh[k * NE + li] : 0.0f; }, (float)xd, li, gb);
    }
    // the stage is free again: refill it with the group kStages ahead
    __syncwarp();
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(it + kStages);
    }
    if (act) {
      const double yv = (double)sh + (double)sl;
      if (g_cur >= 0) {
        atomicAdd(y + 2 * (size_t)g_cur + (li & 1), (TX)yv);
      } else {
        const Constraint& c = cons[-g_cur - 1];
        for (int q = 0; q < c.cnt; ++q) atomicAdd(y + 2 * (size_t)c.node[q] + (li & 1), (TX)(c.w[q] * yv));
      }
      if (red.part) dot += xd * yv;
    }
    g0 = g1;
    g1 = g2;
    g2 = g3;
    g3 = g4;
    x0 = x1;
    x1 = x2;
  }
  if (!__all_sync(0xffffffffu, ok)) {
    // a wait expired: report, then let this warp's outstanding copies land before the block exits
    if (lane == 0) {
      atomicExch(err, MTO_ETIMEOUT);
      for (int k = 0; k < kStages; ++k) {
        const int itk = it + k;
        if (first + itk * stride >= n) break;
        unsigned sp = 0;
        while (!mbar_test(bars + itk % kStages, (uint32_t)((itk / kStages) & 1)) && ++sp < kWaitLimit) {
        }
      }
    }
    __syncwarp();
  }
  if (red.part) reduce_out(dot, red);
}

size_t tma_smem_bytes(int L, int G, int nm, int stages) {
  return (size_t)kTmaWarps * stages * nm * G * L * sizeof(float) + (size_t)kTmaWarps * stages * sizeof(uint64_t);
}

}  // namespace

// Blocks of one element-operator launch for an order class (fixed per class size).
template <int PO>
int ebe_blocks_p(int n) {
  constexpr int NE = 2 * (PO + 1) * (PO + 1);
  constexpr int G = WarpShape<NE>::G;
  const int warps = (n + G - 1) / G;
  return grid_for((int64_t)warps * 32, 256, 152 * 8);
}

int ebe_blocks(int p, int n) {
  switch (p) {
    case 1: return ebe_blocks_p<1>(n);
    case 2: return ebe_blocks_p<2>(n);
    case 3: return ebe_blocks_p<3>(n);
    case 4: return ebe_blocks_p<4>(n);
    case 5: return ebe_blocks_p<5>(n);
    default: return ebe_blocks_p<6>(n);
  }
}

namespace {

// Ring stages of the staged operator: the split pair and the leading part (MTO_TMA_STAGES="s,l"
// overrides, each of 2, 3, 4, 6; read once per process).  Two stages, measured on the 1024 x 512
// beam: the split pair 438 us per launch against 509 us with three stages, 752 with four and 792
// with six; the leading part 247 us against 263, 316 and 411 us.  The smaller ring leaves room for
// more blocks per SM, and both kernels need those warps more than a deeper ring.
int tma_stages(bool split) {
  static int st[2] = {0, 0};
  if (!st[0]) {
    st[0] = 2;   // split pair
    st[1] = 2;   // leading part
    if (const char* e = std::getenv("MTO_TMA_STAGES")) {
      int a = 0, b = 0;
      if (std::sscanf(e, "%d,%d", &a, &b) == 2) {
        st[0] = a;
        st[1] = b;
      }
    }
  }
  return st[split ? 0 : 1];
}

// The staged operator, persistent: as many 8-warp blocks per SM as shared memory and registers allow
// (the occupancy calculator, once per kernel instance; the shared-memory attribute set with it).
template <int PO, bool kLo, typename TX, int NS>
void launch_tma(mto_handle h, const PClass& c, const float* Mh, const float* Ml, const TX* x, TX* y, Red red,
                const int* done) {
  constexpr int NE = 2 * (PO + 1) * (PO + 1);
  const int warps = (c.n + WarpShape<NE>::G - 1) / WarpShape<NE>::G;
  const size_t smem = tma_smem_bytes(c.L, WarpShape<NE>::G, kLo ? 2 : 1, NS);
  static int per_sm = 0;
  if (!per_sm) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(ebe_df_tma_kernel<PO, kLo, TX, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ebe_df_tma_kernel<PO, kLo, TX, NS>, kTmaWarps * 32, smem) !=
            cudaSuccess ||
        nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    per_sm = nb;
  }
  int blocks = (warps + kTmaWarps - 1) / kTmaWarps;
  if (blocks > 152 * per_sm) blocks = 152 * per_sm;
  ebe_df_tma_kernel<PO, kLo, TX, NS><<<blocks, kTmaWarps * 32, smem, h->stream>>>(Mh, Ml, c.L, c.n, c.gmap,
                                                                                   h->cons_d, x, y, red, done,
                                                                                   h->flags + 1);
}

template <int PO, bool kDF, typename TX>
void launch_ebe(mto_handle h, const PClass& c, const double* M64, const float* Mh, const float* Ml, const TX* x,
                TX* y, Red red, const int* done, const ConvTest& cv) {
  constexpr int NE = 2 * (PO + 1) * (PO + 1);
  const int opk = h->op_kernel_cls[PO] >= -1 ? h->op_kernel_cls[PO] : h->op_kernel;   // per-class choice first
  if constexpr (kDF && WarpShape<NE>::M == 1) {
    if (!cv.res && opk != 2) {
      const int warps = (c.n + WarpShape<NE>::G - 1) / WarpShape<NE>::G;
      // bulk-copy staging pays off when the rows stream from HBM (measured: 6.5 % faster on
      // 1 GB of rows, 6 % slower when they sit in L2), so by default it serves classes whose
      // split rows exceed 64 MB
      const bool lo = Ml != nullptr;   // null: the hi rows alone (a preconditioner's copy)
      const bool big = (size_t)c.n * c.L * (lo ? 2 : 1) * sizeof(float) > ((size_t)64 << 20);
      if (opk == 1 || (opk < 0 && big)) {
        const int ns = tma_stages(lo);
        if (lo) {
          switch (ns) {
            case 2: launch_tma<PO, true, TX, 2>(h, c, Mh, Ml, x, y, red, done); break;
            case 4: launch_tma<PO, true, TX, 4>(h, c, Mh, Ml, x, y, red, done); break;
            case 6: launch_tma<PO, true, TX, 6>(h, c, Mh, Ml, x, y, red, done); break;
            default: launch_tma<PO, true, TX, 3>(h, c, Mh, Ml, x, y, red, done); break;
          }
        } else {
          switch (ns) {
            case 2: launch_tma<PO, false, TX, 2>(h, c, Mh, Ml, x, y, red, done); break;
            case 4: launch_tma<PO, false, TX, 4>(h, c, Mh, Ml, x, y, red, done); break;
            case 6: launch_tma<PO, false, TX, 6>(h, c, Mh, Ml, x, y, red, done); break;
            default: launch_tma<PO, false, TX, 3>(h, c, Mh, Ml, x, y, red, done); break;
          }
        }
        return;
      }
      // persistent: two blocks of 8 warps per SM (the register budget of the pipelined rows)
      int blocks = (warps + 7) / 8;
      if (blocks > 152 * 2) blocks = 152 * 2;
      if (lo)
        ebe_df_pipe_kernel<PO, true, TX><<<blocks, 256, 0, h->stream>>>(Mh, Ml, c.L, c.n, c.gmap, h->cons_d, x, y,
                                                                         red, done);
      else
        ebe_df_pipe_kernel<PO, false, TX><<<blocks, 256, 0, h->stream>>>(Mh, Ml, c.L, c.n, c.gmap, h->cons_d, x, y,
                                                                          red, done);
      return;
    }
  }
  ebe_kernel<PO, kDF, TX><<<ebe_blocks_p<PO>(c.n), 256, 0, h->stream>>>(M64, Mh, Ml, c.L, c.n, c.gmap, h->cons_d, x,
                                                                        y, red, done, cv);
}

// y += S x for the springs to ground (distinct DOFs; launched after the element classes on the same
// stream, so plain adds), with x^T S x as one more reduction result
template <typename T>
__global__ void __launch_bounds__(256) spring_kernel(int n, const int64_t* __restrict__ dof,
                                                     const double* __restrict__ k, const T* __restrict__ x,
                                                     T* __restrict__ y, Red red, const int* __restrict__ done) {
  if (done && *done) return;
  double dot = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double xv = (double)x[dof[i]];
    y[dof[i]] += (T)(k[i] * xv);
    dot += k[i] * xv * xv;
  }
  if (red.part) reduce_out(dot, red);
}

// reduction slot k of the CG buffers (launch j writes part + j * kPartStride, res[j], cnt[j])
Red red_slot(mto_handle h, int k, int j) {
  if (k < 0) return Red{nullptr, nullptr, nullptr};
  return Red{h->cg_part + (size_t)k * h->cg_stride + (size_t)j * h->cg_class_stride, h->cg_cnt + 8 * k + j,
             h->cg_res + 8 * k + j};
}

// y += sum_e P_e^T A_e P_e x over all order classes, where A_e is the element stiffness (which = 0)
// or the element-block preconditioner (which = 1).  FP64 matrices on the FP64 pipes (plain FP64
// path, refinement residuals) or the split-precision pair on the FP32 pipes (inner iterations of
// the mixed solves) with FP64 or FP32 vectors; `lead`: of a split pair the FP32 leading part
// alone (inside the preconditioner).  x^T y goes to reduction slot `slot` (one result per class
// launch; -1: not wanted); *nres receives the number of class launches.
template <typename T>
mto_status apply_all(mto_handle h, int which, const T* x, T* y, int slot, const int* done, ConvTest cv,
                     int* nres = nullptr, bool lead = false) {
  const bool mixed_build = h->built_precision == MTO_MIXED;
  const bool df = which == 1 ? mixed_build : (sizeof(T) == 4 || (mixed_build && (h->inner_split || lead)));
  const int fam = lead       ? F_APPLYLEAD
                  : which == 1 ? F_PRECOND
                               : (df ? (sizeof(T) == 8 ? F_APPLYDF64 : F_APPLY32) : F_APPLY64);
  TimedScope ts(h, fam);
  int ci = 0;
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    const PClass& c = h->pc[p];
    if (c.n == 0) continue;
    const double* M64 = which ? c.B64 : c.K64;
    const float* Mh = which ? c.B32 : c.K32;
    const float* Ml = lead ? nullptr : (which ? c.B32lo : c.K32lo);
    const Red pp = red_slot(h, slot, ci);
    if (df) {
      if (!Mh || (!Ml && !lead)) return mto_fail(h, MTO_EINVAL, "split-precision element matrices are not built");
      switch (p) {
        case 1: launch_ebe<1, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        case 2: launch_ebe<2, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        case 3: launch_ebe<3, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        case 4: launch_ebe<4, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        case 5: launch_ebe<5, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        case 6: launch_ebe<6, true, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
      }
    } else {
      if constexpr (sizeof(T) == 8) {
        if (!M64) return mto_fail(h, MTO_EINVAL, "FP64 element matrices are not built");
        switch (p) {
          case 1: launch_ebe<1, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
          case 2: launch_ebe<2, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
          case 3: launch_ebe<3, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
          case 4: launch_ebe<4, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
          case 5: launch_ebe<5, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
          case 6: launch_ebe<6, false, T>(h, c, M64, Mh, Ml, x, y, pp, done, cv); break;
        }
      } else {
        return mto_fail(h, MTO_EINVAL, "FP32 vectors need the split-precision build");
      }
    }
    ++ci;
    MTO_TRY(mto_after_launch(h, "ebe_kernel"));
  }
  if (which == 0 && h->n_springs) {
    spring_kernel<T><<<1, 256, 0, h->stream>>>(h->n_springs, h->spring_dof_d, h->spring_k_d, x, y,
                                                 red_slot(h, slot, ci), done);
    ++ci;
    MTO_TRY(mto_after_launch(h, "spring_kernel"));
  }
  if (nres) *nres = ci;
  return MTO_OK;
}


// ---------------------------------------------------------------------------------- CG
// Preconditioned CG (Hestenes-Stiefel form).  Per iteration: the operator launch q = K p, which
// also yields p^T K p; a fused vector kernel (alpha, x, r, q = 0, Jacobi z and r^T z, r^T r,
// r^T D^-1 r); the element-block preconditioner z = M^-1 r (Schwarz only, also yielding r^T z);
// and the direction kernel (convergence test, beta, p = z + beta p).  The curvature p^T K p is
// accumulated directly (never formed by subtraction), which matters at the 1e9 stiffness contrast
// of these problems.  Every reduction is finished by the last block of its launch in a fixed order
// (deterministic); consumers add the few launch results of a slot in class order.  Slots alternate
// by iteration parity: kGam = r^T z, kDel = p^T K p, kRR = r^T r, kRD = r^T D^-1 r.
constexpr int kGam = 0, kDel = 2, kRR = 4, kRD = 6;

template <typename T, bool kJacobi>
__global__ void __launch_bounds__(256) cg_vector_kernel(
    int64_t n, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, T* __restrict__ q, T* __restrict__ z,
    const T* __restrict__ invd, const double* __restrict__ gin, int ng, const double* __restrict__ pin, int np,
    Red gout, Red rrout, Red rdout, const int* __restrict__ base, int local, int* __restrict__ done,
    int* __restrict__ err, double* __restrict__ eng) {
  if (*done) return;
  // the step length once per block (an FP64 division per thread costs more than the vector pass
  // on GB300's FP64 pipes)
  __shared__ double s_alpha;
  __shared__ int s_stop;
  if (threadIdx.x == 0) {
    const double rz = sum_res(gin, ng);
    const double pq = sum_res(pin, np);
    const double a = rz / pq;
    s_stop = (!(pq > 0.0) || !isfinite(a)) ? (rz != 0.0 ? 2 : 1) : 0;
    s_alpha = a;
    if (eng && blockIdx.x == 0 && !s_stop) {   // energy gained by this step: alpha_i gamma_i
      const int it = *base + local;
      eng[2 + it % kEnergyRing] = a * rz;
      eng[0] += a * rz;
    }
  }
  __syncthreads();
  const double alpha = s_alpha;
  if (s_stop) {
    // rz = 0: the residual vanished (exact solution); otherwise a breakdown
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (s_stop == 2) *err = MTO_ENAN;
      *done = *base + local + 1;
    }
    return;
  }
  const T a = (T)alpha;
  double g = 0.0, rr = 0.0, rd = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const T inv = invd[j];
    const T qj = q[j];   // q is cleared by the next launch (zero_kernel): see there
    if (!kJacobi) z[j] = (T)0;
    if (inv != (T)0) {
      x[j] = fma(a, p[j], x[j]);
      const T rj = fma(-a, qj, r[j]);
      r[j] = rj;
      const double rjd = (double)rj;
      if (kJacobi) g += rjd * rjd * (double)inv;
      rr += rjd * rjd;
      rd += rjd * rjd * (double)inv;
    }
  }
  if (kJacobi) reduce_out(g, gout);
  reduce_out(rr, rrout);
  reduce_out(rd, rdout);
}

// convergence test on the new residual, then beta = (r^T z)_new / (r^T z)_old and p = z + beta p
// (Jacobi: z = D^-1 r on the fly)
template <typename T, bool kJacobi>
__global__ void __launch_bounds__(256) cg_direction_kernel(
    int64_t n, const T* __restrict__ r, const T* __restrict__ z, T* __restrict__ p, const T* __restrict__ invd,
    const double* __restrict__ gnew, const double* __restrict__ gold, int ng, ConvTest cv) {
  if (*cv.done) return;
  __shared__ double s_beta;
  __shared__ int s_stop;
  if (threadIdx.x == 0) {
    const double crit = sum_res(cv.res, cv.n);
    if (cv.eng) {
      // compliance accuracy: the extrapolated remaining energy against tol x the compliance estimate
      const int it = *cv.base + cv.local;
      int conv = 0;
      if (it + 1 >= kEnergyRing) {
        double s_last = 0.0, s_prev = 0.0;
        for (int k = 0; k < kEnergyWin; ++k) {
          s_last += __ldcg(cv.eng + 2 + (it - k) % kEnergyRing);
          s_prev += __ldcg(cv.eng + 2 + (it - kEnergyWin - k) % kEnergyRing);
        }
        const double q = s_last / s_prev;
        const double cref = __ldcg(cv.eng + 1) + __ldcg(cv.eng);
        conv = q < 1.0 && s_last <= (1.0 - q) * kEnergySafety * cv.tol2 * cref;
      }
      // a residual at the floor of FP64 ends the run however few iterations it took (the energy
      // test needs two windows; a well-conditioned correction converges sooner, and iterating on
      // rounding noise would break down)
      conv = conv || crit <= __ldcg(cv.eng + 2 + kEnergyRing);
      s_stop = !(crit == crit) ? 2 : ((conv || crit == 0.0) ? 1 : 0);
    } else {
      s_stop = !(crit > cv.tol2 * *cv.ref) ? (crit == crit ? 1 : 2) : 0;   // converged, or a NaN residual
    }
    s_beta = s_stop ? 0.0 : sum_res(gnew, ng) / sum_res(gold, ng);
  }
  __syncthreads();
  if (s_stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (s_stop == 2) *cv.err = MTO_ENAN;
      *cv.done = *cv.base + cv.local + 1;
    }
    return;
  }
  const double beta = s_beta;
  const T b = (T)beta;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    // the element-block preconditioner scatters its hanging DOFs' rows onto the nodes they
    // interpolate, supported ones included: z is masked to the free DOFs here
    const T zj = kJacobi ? invd[j] * r[j] : (invd[j] != (T)0 ? z[j] : (T)0);
    p[j] = fma(b, p[j], zj);
  }
}

// start of a CG run from the residual r (zero on supports): q = 0 and, for Jacobi, p = D^-1 r with
// r^T z; for Schwarz z = 0 (the preconditioner launch fills it), p set afterwards
template <typename T, bool kJacobi>
__global__ void __launch_bounds__(256) cg_init_kernel(int64_t n, const T* __restrict__ r, T* __restrict__ p,
                                                      T* __restrict__ q, T* __restrict__ z,
                                                      const T* __restrict__ invd, Red gout) {
  double g = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    q[j] = (T)0;
    if (kJacobi) {
      const T pj = invd[j] * r[j];
      p[j] = pj;
      g += (double)r[j] * (double)pj;
    } else {
      z[j] = (T)0;
    }
  }
  if (kJacobi) reduce_out(g, gout);
}

// v = 0.  Measured on GB300: a vector kernel that reads an array and then stores zeros into it
// streams at ~1.6 TB/s (9.4M doubles, 5 reads and 3 writes), the same kernel without that store at
// ~4.9 TB/s and a kernel of plain stores at ~5.9 TB/s, so the accumulators that the next operator
// launch adds into are cleared by this separate launch instead of by the kernel that consumed them.
template <typename T>
__global__ void __launch_bounds__(256) zero_kernel(int64_t n, T* __restrict__ v, const int* __restrict__ done) {
  if (done && *done) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    v[j] = (T)0;
}

// b = a on free DOFs (invd != 0), 0 on supported ones
template <typename T>
__global__ void __launch_bounds__(256) masked_copy_kernel(int64_t n, const T* __restrict__ a, T* __restrict__ b,
                                                          const T* __restrict__ invd) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    b[j] = invd[j] != (T)0 ? a[j] : (T)0;
}

__global__ void add2_kernel(const double* a, const double* b, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = *a + *b;
}

__global__ void advance_kernel(int* base, int by) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *base += by;
}

// r = f - Ku on free DOFs, 0 on supports; per-block partials of r^T r, f^T f, r^T D^-1 r, f^T D^-1 f
__global__ void __launch_bounds__(256) residual_kernel(int64_t n, const double* __restrict__ f,
                                                       const double* __restrict__ Ku, const double* __restrict__ invd,
                                                       double* __restrict__ r, double* __restrict__ part) {
  double rr = 0.0, ff = 0.0, rd = 0.0, fd = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    const double di = invd[i];
    if (di != 0.0) {
      v = f[i] - Ku[i];
      ff += f[i] * f[i];
      fd += f[i] * f[i] * di;
      rd += v * v * di;
    }
    r[i] = v;
    rr += v * v;
  }
  rr = block_sum(rr);
  ff = block_sum(ff);
  rd = block_sum(rd);
  fd = block_sum(fd);
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x + 0] = rr;
    part[4 * blockIdx.x + 1] = ff;
    part[4 * blockIdx.x + 2] = rd;
    part[4 * blockIdx.x + 3] = fd;
  }
}

// one block: out[k] = sum_b part[4 b + k] (fixed order)
__global__ void sum4_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  for (int k = 0; k < 4; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[4 * b + k];
    v = block_sum(v);
    if (threadIdx.x == 0) out[k] = v;
  }
}

// r32 = (float)(r * scale)
__global__ void __launch_bounds__(256) demote_kernel(int64_t n, const double* __restrict__ r, double scale,
                                                     float* __restrict__ r32, float* __restrict__ x32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r32[i] = (float)(r[i] * scale);
    x32[i] = 0.0f;
  }
}

// u += d
__global__ void __launch_bounds__(256) axpy_kernel(int64_t n, const double* __restrict__ d, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] += d[i];
}

// u += x32 / scale
__global__ void __launch_bounds__(256) promote_kernel(int64_t n, const float* __restrict__ x32, double inv_scale,
                                                      double* __restrict__ u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] += (double)x32[i] * inv_scale;
}

__global__ void __launch_bounds__(256) mask_kernel(int64_t n, const double* __restrict__ invd, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (invd[i] == 0.0) u[i] = 0.0;
}

__global__ void __launch_bounds__(256) dot_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                                  double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum1_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
  v = block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

// grid of the vector kernels (fixed: partial counts): one full wave of 8 blocks of 256 threads per
// SM, so that enough loads are in flight to stream the vectors at HBM speed (with 4 blocks per SM
// the grid-stride loops ran latency-bound at about a sixth of it)
constexpr int kVecBlocks = 152 * 8;

template <typename T>
struct CGVecs {
  T *x, *r, *p, *q, *z;
  const T* invd;
};

template <typename T>
CGVecs<T> cg_vecs(mto_handle h, T* x, T* r);
template <>
CGVecs<double> cg_vecs<double>(mto_handle h, double* x, double* r) {
  return {x, r, h->p64, h->w64, h->u64, h->invd64};
}
template <>
CGVecs<float> cg_vecs<float>(mto_handle h, float* x, float* r) {
  return {x, r, h->p32, h->w32, h->u32, h->invd32};
}

// result j of reduction slot k
inline const double* res_slot(mto_handle h, int k) { return h->cg_res + 8 * k; }

// The preconditioner step z = M^-1 r with r^T z into reduction slot `slot` (element-block Schwarz:
// one result per class launch; multigrid: one).
template <typename T>
mto_status precond_step(mto_handle h, const CGVecs<T>& v, int pc, int deg, int slot, const int* done);
template <>
mto_status precond_step<double>(mto_handle h, const CGVecs<double>& v, int pc, int deg, int slot,
                                const int* done) {
  ConvTest none{};
  if (pc == MTO_PREC_SCHWARZ) return apply_all<double>(h, 1, v.r, v.z, slot, done, none);
  const Red rd = red_slot(h, slot, 0);   // r^T z from the cycle's last smoothing step
  return mg_vcycle(h, v.r, v.z, deg, done, rd.part, rd.cnt, rd.res);
}
template <>
mto_status precond_step<float>(mto_handle h, const CGVecs<float>& v, int pc, int deg, int slot, const int* done) {
  ConvTest none{};
  if (pc == MTO_PREC_SCHWARZ) return apply_all<float>(h, 1, v.r, v.z, slot, done, none);
  return mto_fail(h, MTO_EINVAL, "the multigrid preconditioner needs FP64 vectors (precision MTO_FP64)");
}

// The launches of CG iteration `local` of a chunk (nc = number of order classes).
template <typename T>
mto_status cg_iteration(mto_handle h, const CGVecs<T>& v, int pc, int deg, int nrm, const double* ref, double tol2,
                        int local, int nc) {
  double* eng = nrm == 2 ? h->eng : nullptr;
  const int64_t n = h->ndof;
  const int par = local & 1, nxt = par ^ 1;
  const bool jac = pc == MTO_PREC_JACOBI;
  // r^T z comes from one result per class launch of the element-block preconditioner (which has no
  // spring term), else from one launch; p^T K p from every operator launch (classes + springs)
  const int ng = pc == MTO_PREC_SCHWARZ ? nc : 1;
  const int nop = nc + (h->n_springs ? 1 : 0);
  ConvTest none{};
  h->timing.sample = local == 0;   // sampled timing: the first operator launch of every chunk
  const mto_status sa = apply_all<T>(h, 0, v.p, v.q, kDel + par, h->flags, none);
  h->timing.sample = false;
  MTO_TRY(sa);
  {
    TimedScope ts(h, F_VECTOR);
    if (!jac)
      cg_vector_kernel<T, false><<<kVecBlocks, 256, 0, h->stream>>>(
          n, v.x, v.r, v.p, v.q, v.z, v.invd, res_slot(h, kGam + par), ng, res_slot(h, kDel + par), nop,
          red_slot(h, -1, 0), red_slot(h, kRR + nxt, 0), red_slot(h, kRD + nxt, 0), h->cg_base, local, h->flags,
          h->flags + 1, eng);
    else
      cg_vector_kernel<T, true><<<kVecBlocks, 256, 0, h->stream>>>(
          n, v.x, v.r, v.p, v.q, v.z, v.invd, res_slot(h, kGam + par), ng, res_slot(h, kDel + par), nop,
          red_slot(h, kGam + nxt, 0), red_slot(h, kRR + nxt, 0), red_slot(h, kRD + nxt, 0), h->cg_base, local,
          h->flags, h->flags + 1, eng);
    MTO_TRY(mto_after_launch(h, "cg_vector_kernel"));
    zero_kernel<T><<<kVecBlocks, 256, 0, h->stream>>>(n, v.q, h->flags);
    MTO_TRY(mto_after_launch(h, "zero_kernel"));
  }
  if (!jac) {
    h->timing.sample_lead = local == 0;   // sampled timing: the cycle's leading-part launches too
    const mto_status sp = precond_step<T>(h, v, pc, deg, kGam + nxt, h->flags);
    h->timing.sample_lead = false;
    MTO_TRY(sp);
  }
  {
    TimedScope ts(h, F_VECTOR);
    ConvTest cv{res_slot(h, nrm == 1 ? kRD + nxt : kRR + nxt), 1, ref, tol2, h->cg_base, local, h->flags, h->flags + 1,
                eng};
    if (!jac)
      cg_direction_kernel<T, false><<<kVecBlocks, 256, 0, h->stream>>>(
          n, v.r, v.z, v.p, v.invd, res_slot(h, kGam + nxt), res_slot(h, kGam + par), ng, cv);
    else
      cg_direction_kernel<T, true><<<kVecBlocks, 256, 0, h->stream>>>(
          n, v.r, v.z, v.p, v.invd, res_slot(h, kGam + nxt), res_slot(h, kGam + par), ng, cv);
    MTO_TRY(mto_after_launch(h, "cg_direction_kernel"));
  }
  return MTO_OK;
}

// CG on (x, r) of type T: r is the residual of x (free DOFs, zero on supports).  Stops when the
// residual norm^2 (l2 or Jacobi) <= tol2 * (*ref), or by the energy test (nrm = 2), or after max_it
// iterations.  Iterations run in chunks of `chunk` (even), each captured once as a CUDA graph and
// replayed.  The run is split into its preparation (start vectors, first preconditioner step,
// graph capture), the launch of one chunk (with the asynchronous read-back of the done flags) and
// the check of those flags after a synchronisation, so that a batch of handles can advance
// together (solve_batched); run_cg strings them together for one handle.
template <typename T>
struct CGRun {
  CGVecs<T> v;
  int pc, deg, nrm, nc, chunk;
  const double* ref;
  double tol2;
  GraphEntry* ge = nullptr;
  int k = 0;
};

template <typename T>
mto_status cg_prepare(mto_handle h, CGRun<T>& run, T* x, T* r, int pc, int deg, int nrm, const double* ref,
                      double tol2, int chunk) {
  const bool schwarz = pc != MTO_PREC_JACOBI;   // z kept in its own vector
  const int64_t n = h->ndof;
  CGVecs<T> v = cg_vecs<T>(h, x, r);
  run.v = v;
  run.pc = pc;
  run.deg = deg;
  run.nrm = nrm;
  run.ref = ref;
  run.tol2 = tol2;
  run.chunk = chunk;
  run.k = 0;
  run.ge = nullptr;
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(int), h->stream), "memset"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->cg_base, 0, sizeof(int), h->stream), "memset"));
  // a launch that ended the run early may have left a block count behind
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->cg_cnt, 0, 64 * sizeof(unsigned), h->stream), "memset"));
  if (nrm == 2) {   // energy log of this run (its compliance base eng[1] is set by the caller)
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->eng, 0, sizeof(double), h->stream), "memset"));
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->eng + 2, 0, kEnergyRing * sizeof(double), h->stream), "memset"));
  }
  int nc = 0;
  for (int p = 1; p <= MTO_P_MAX; ++p)
    if (h->pc[p].n) ++nc;
  run.nc = nc;
  {
    TimedScope ts(h, F_VECTOR);
    if (schwarz)
      cg_init_kernel<T, false><<<kVecBlocks, 256, 0, h->stream>>>(n, v.r, v.p, v.q, v.z, v.invd, red_slot(h, -1, 0));
    else
      cg_init_kernel<T, true><<<kVecBlocks, 256, 0, h->stream>>>(n, v.r, v.p, v.q, v.z, v.invd,
                                                                 red_slot(h, kGam, 0));
    MTO_TRY(mto_after_launch(h, "cg_init_kernel"));
  }
  if (pc == MTO_PREC_MG) {
    for (auto& l : h->mg) MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(l.q, 0, l.n * sizeof(double), h->stream), "memset"));
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->mg_q0, 0, n * sizeof(double), h->stream), "memset"));
  }
  if (schwarz) {
    MTO_TRY(precond_step<T>(h, v, pc, deg, kGam, nullptr));
    TimedScope ts(h, F_VECTOR);
    masked_copy_kernel<T><<<kVecBlocks, 256, 0, h->stream>>>(n, v.z, v.p, v.invd);
    MTO_TRY(mto_after_launch(h, "masked_copy_kernel"));
  }
  if (!h->use_graphs) return MTO_OK;
  GraphKey key{sizeof(T), (const void*)x, (const void*)r, pc, deg, nrm, ref, tol2, chunk,
               h->timing.on ? (h->timing.sampled ? 2 : 1) : 0, 2 * h->built_precision + (h->inner_split ? 1 : 0)};
  GraphEntry* ge = find_graph(h, key);
  if (!ge) {
    ge = new_graph(h, key);
    const int64_t l0 = h->launches;
    MTO_TRY(mto_cuda_check(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
                           "cudaStreamBeginCapture"));
    h->timing.capture_list = &ge->events;
    mto_status st = MTO_OK;
    for (int l = 0; l < chunk && st == MTO_OK; ++l) st = cg_iteration<T>(h, v, pc, deg, nrm, ref, tol2, l, nc);
    if (st == MTO_OK) {
      advance_kernel<<<1, 32, 0, h->stream>>>(h->cg_base, chunk);
      st = mto_after_launch(h, "advance_kernel");
    }
    h->timing.capture_list = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    ge->launches_per_replay = h->launches - l0;
    h->launches = l0;   // nothing ran during capture
    if (st != MTO_OK) return st;
    MTO_TRY(mto_cuda_check(h, e, "cudaStreamEndCapture"));
    MTO_TRY(mto_cuda_check(h, cudaGraphInstantiate(&ge->exec, g, 0), "cudaGraphInstantiate"));
    cudaGraphDestroy(g);
  }
  run.ge = ge;
  return MTO_OK;
}

// one chunk of iterations, then the done flags to the pinned host mirror (asynchronous)
template <typename T>
mto_status cg_launch_chunk(mto_handle h, CGRun<T>& run) {
  if (run.ge) {
    MTO_TRY(mto_cuda_check(h, cudaGraphLaunch(run.ge->exec, h->stream), "cudaGraphLaunch"));
    h->launches += run.ge->launches_per_replay;
  } else {
    for (int l = 0; l < run.chunk; ++l)
      MTO_TRY(cg_iteration<T>(h, run.v, run.pc, run.deg, run.nrm, run.ref, run.tol2, l, run.nc));
    advance_kernel<<<1, 32, 0, h->stream>>>(h->cg_base, run.chunk);
    MTO_TRY(mto_after_launch(h, "advance_kernel"));
  }
  run.k += run.chunk;
  return mto_cuda_check(h, cudaMemcpyAsync(h->host_flags, h->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream),
                        "copy");
}

// after the stream has been synchronised: 1 when the run has finished (converged or broken down)
template <typename T>
int cg_check(mto_handle h, CGRun<T>& run) {
  if (run.ge) graph_timing_harvest(h, run.ge);
  timing_harvest(h);
  return h->host_flags[0] != 0 || h->host_flags[1] != 0;
}

template <typename T>
mto_status cg_result(mto_handle h, const CGRun<T>& run, int* iters) {
  const int done = h->host_flags[0];
  *iters = done ? done : run.k;
  if (h->host_flags[1]) return mto_fail(h, MTO_ENAN, "CG breakdown: non-finite or non-positive curvature");
  return MTO_OK;
}

template <typename T>
mto_status run_cg(mto_handle h, T* x, T* r, int pc, int deg, int nrm, const double* ref, double tol2, int max_it,
                  int chunk, int* iters) {
  CGRun<T> run;
  MTO_TRY(cg_prepare<T>(h, run, x, r, pc, deg, nrm, ref, tol2, chunk));
  while (run.k < max_it) {
    MTO_TRY(cg_launch_chunk<T>(h, run));
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    if (cg_check<T>(h, run)) break;
  }
  return cg_result<T>(h, run, iters);
}

// FP64 residual r = f - K u (masked) and its squared norms: h->red[0..3] = (r, f l2; r, f Jacobi),
// read back asynchronously into host_pinned[0..3] (residual_enqueue), then taken after a
// synchronisation (residual_take).
mto_status residual_enqueue(mto_handle h, const double* f, const double* u) {
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->s64, 0, sizeof(double) * h->ndof, h->stream), "memset"));
  ConvTest none{};
  MTO_TRY(apply_all<double>(h, 0, u, h->s64, -1, nullptr, none));
  {
    TimedScope ts(h, F_VECTOR);
    residual_kernel<<<kVecBlocks, 256, 0, h->stream>>>(h->ndof, f, h->s64, h->invd64, h->r64, h->cg_part);
    MTO_TRY(mto_after_launch(h, "residual_kernel"));
    sum4_kernel<<<1, 256, 0, h->stream>>>(h->cg_part, kVecBlocks, h->red);
    MTO_TRY(mto_after_launch(h, "sum4_kernel"));
  }
  return mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned, h->red, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                           h->stream), "copy");
}

void residual_take(mto_handle h, int norm, double* rr, double* ff) {
  timing_harvest(h);
  *rr = h->host_pinned[norm ? 2 : 0];
  *ff = h->host_pinned[norm ? 3 : 1];
}

mto_status true_residual(mto_handle h, const double* f, const double* u, int norm, double* rr, double* ff) {
  MTO_TRY(residual_enqueue(h, f, u));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  residual_take(h, norm, rr, ff);
  return MTO_OK;
}

}  // namespace

mto_status apply64(mto_handle h, const double* x, double* y) {
  ConvTest none{};
  return apply_all<double>(h, 0, x, y, -1, nullptr, none);
}

mto_status apply_operator(mto_handle h, int op, const double* x, double* y, double* xKx) {
  ConvTest none{};
  int nres = 0;
  // a launch that ended a CG run early may have left a finished-block count behind
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->cg_cnt, 0, 64 * sizeof(unsigned), h->stream), "memset"));
  h->inner_split = op != MTO_OP_FP64;
  const mto_status st = apply_all<double>(h, 0, x, y, kGam, nullptr, none, &nres, op == MTO_OP_LEAD);
  h->inner_split = false;
  MTO_TRY(st);
  if (!xKx) return MTO_OK;
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned, h->cg_res + 8 * kGam, nres * sizeof(double),
                                            cudaMemcpyDeviceToHost, h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  timing_harvest(h);
  double s = 0.0;
  for (int i = 0; i < nres; ++i) s += h->host_pinned[i];
  *xKx = s;
  return MTO_OK;
}

// Autotuner of the split operator's kernel per order class (n_e <= 32: register pipeline, bulk-copy
// staging or the generic kernel): each candidate is timed with CUDA events over a few launches on
// the class's own rows and the fastest is kept for the class (in the handle, and in a process-wide
// table keyed by device, order and element count, so instances of the same class size reuse it).
namespace {
struct TuneKey {
  int device, p, n;
  bool operator<(const TuneKey& o) const {
    return device != o.device ? device < o.device : (p != o.p ? p < o.p : n < o.n);
  }
};
std::map<TuneKey, std::pair<int, std::array<float, 3>>> g_tune_cache;
std::mutex g_tune_mutex;
}  // namespace

mto_status autotune_operator(mto_handle h, int32_t* choice, double* us) {
  if (h->built_precision != MTO_MIXED)
    return mto_fail(h, MTO_EINVAL, "mto_autotune: needs the split-precision (MTO_MIXED) build");
  // timed on zeroed work vectors (the values do not matter, only well-formed numbers)
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->p64, 0, h->ndof * sizeof(double), h->stream), "memset"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->w64, 0, h->ndof * sizeof(double), h->stream), "memset"));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  mto_status st = MTO_OK;
  for (int p = 1; p <= MTO_P_MAX && st == MTO_OK; ++p) {
    PClass& c = h->pc[p];
    if (choice) choice[p] = -2;
    if (c.n == 0 || 2 * (p + 1) * (p + 1) > 32) continue;
    std::array<float, 3> t{0.f, 0.f, 0.f};
    int best = -1;
    {
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      auto it = g_tune_cache.find(TuneKey{h->device, p, c.n});
      if (it != g_tune_cache.end()) {
        best = it->second.first;
        t = it->second.second;
      }
    }
    if (best < 0) {
      ConvTest none{};
      const Red nored{nullptr, nullptr, nullptr};
      for (int v = 0; v < 3 && st == MTO_OK; ++v) {
        h->op_kernel_cls[p] = v;
        for (int rep = 0; rep < 7 && st == MTO_OK; ++rep) {
          if (rep == 2) cudaEventRecord(a, h->stream);
          switch (p) {
            case 1: launch_ebe<1, true, double>(h, c, c.K64, c.K32, c.K32lo, h->p64, h->w64, nored, nullptr, none); break;
            case 2: launch_ebe<2, true, double>(h, c, c.K64, c.K32, c.K32lo, h->p64, h->w64, nored, nullptr, none); break;
            case 3: launch_ebe<3, true, double>(h, c, c.K64, c.K32, c.K32lo, h->p64, h->w64, nored, nullptr, none); break;
          }
          st = mto_after_launch(h, "ebe operator (autotune)");
        }
        cudaEventRecord(b, h->stream);
        if (st == MTO_OK) st = mto_cuda_check(h, cudaEventSynchronize(b), "autotune");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t[v] = ms / 5.f;
      }
      best = 0;
      for (int v = 1; v < 3; ++v)
        if (t[v] < t[best]) best = v;
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      g_tune_cache[TuneKey{h->device, p, c.n}] = {best, t};
    }
    h->op_kernel_cls[p] = best;
    if (choice) choice[p] = best;
    if (us)
      for (int v = 0; v < 3; ++v) us[3 * p + v] = 1e3 * t[v];
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  clear_graphs(h);   // captured iterations hold the previous kernels
  return st;
}

mto_status apply_fine(mto_handle h, const double* x, double* y, const int* done, bool lead) {
  ConvTest none{};
  return apply_all<double>(h, 0, x, y, -1, done, none, nullptr, lead);
}

mto_status apply_block(mto_handle h, const double* x, double* y, const int* done, bool lead) {
  ConvTest none{};
  return apply_all<double>(h, 1, x, y, -1, done, none, nullptr, lead);
}

mto_status apply_fine32(mto_handle h, const float* x, float* y, const int* done) {
  ConvTest none{};
  return apply_all<float>(h, 0, x, y, -1, done, none, nullptr, true);
}

mto_status apply_block32(mto_handle h, const float* x, float* y, const int* done) {
  ConvTest none{};
  return apply_all<float>(h, 1, x, y, -1, done, none, nullptr, true);
}

mto_status apply_q1(mto_handle h, const MGLevel& l, const double* x, double* y, const int* done) {
  ConvTest none{};
  ebe_kernel<1, false, double><<<ebe_blocks_p<1>(l.nel), 256, 0, h->stream>>>(
      l.K, nullptr, nullptr, 40, l.nel, l.gmap, nullptr, x, y, Red{nullptr, nullptr, nullptr}, done, none);
  return mto_after_launch(h, "ebe_kernel");
}

__global__ void __launch_bounds__(256) vsum_kernel(int64_t n, const double* __restrict__ a, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += a[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

mto_status sum64(mto_handle h, const double* a, int64_t n, double* out_dev) {
  vsum_kernel<<<kVecBlocks, 256, 0, h->stream>>>(n, a, h->cg_part);
  MTO_TRY(mto_after_launch(h, "vsum_kernel"));
  sum1_kernel<<<1, 256, 0, h->stream>>>(h->cg_part, kVecBlocks, out_dev);
  return mto_after_launch(h, "sum1_kernel");
}

mto_status dot64(mto_handle h, const double* a, const double* b, int64_t n, double* out_dev) {
  dot_kernel<<<kVecBlocks, 256, 0, h->stream>>>(n, a, b, h->cg_part);
  MTO_TRY(mto_after_launch(h, "dot_kernel"));
  sum1_kernel<<<1, 256, 0, h->stream>>>(h->cg_part, kVecBlocks, out_dev);
  return mto_after_launch(h, "sum1_kernel");
}

mto_status solve(mto_handle h, const double* f, double* u, const mto_solve_opts* o, int32_t* iters_out,
                 double* relres_out) {
  const int64_t n = h->ndof;
  const int grd = grid_for(n, 256, 152 * 4);
  const int pc = o->precond;
  const int deg = o->mg_degree > 0 ? o->mg_degree : 4;
  if (deg > 16) return mto_fail(h, MTO_EINVAL, "mto_solve: mg_degree above 16");
  if (pc == MTO_PREC_SCHWARZ && !h->schwarz_valid) MTO_TRY(build_schwarz(h));
  if (pc == MTO_PREC_MG) {
    if (o->precision == MTO_MIXED32)
      return mto_fail(h, MTO_EINVAL, "mto_solve: the multigrid preconditioner needs FP64 vectors");
    MTO_TRY(mg_select_smoother(h, o->mg_smoother));
    MTO_TRY(mg_select_operator(h, o->mg_operator));
    if (!h->mg_valid) MTO_TRY(mg_build(h));
  }
  if (!o->warm_start) MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(u, 0, sizeof(double) * n, h->stream), "memset"));
  else {
    mask_kernel<<<grd, 256, 0, h->stream>>>(n, h->invd64, u);
    MTO_TRY(mto_after_launch(h, "mask_kernel"));
  }
  const int chunk = o->check_every < 2 ? 2 : (o->check_every + 1) / 2 * 2;
  int total = 0;
  double rr = 0.0, ff = 0.0;
  const int max_outer = o->max_outer > 0 ? o->max_outer : 50;
  const bool energy = o->norm == MTO_NORM_ENERGY;
  const int nrm = o->norm == MTO_NORM_JACOBI ? 1 : 0;   // norm of the residual reported and tested
  const double itol = o->inner_rtol > 0 ? o->inner_rtol : 1e-6;
  // mixed refinement: a step whose FP64 residual falls short of the asked reduction by more than
  // 10x shows that the split pair's ~48-bit matrices limit it (condition number near 2^48); the
  // remaining steps then apply the FP64 matrices in the inner PCG too
  bool split = true;
  bool step_converged = false;   // the last correction solve met its test (energy mode stops on it)
  double rr_prev = -1.0, asked = 0.0;
  mto_status st = MTO_ENOCONV;
  const auto t_start = std::chrono::steady_clock::now();
  int last_it = 0;
  for (int outer = 0; outer <= max_outer; ++outer) {
    // FP64 residual with the FP64 element matrices
    h->inner_split = false;
    MTO_TRY(true_residual(h, f, u, nrm, &rr, &ff));
    if (h->solve_log)
      std::fprintf(stderr, "mto_solve: step %d inner_iters %d relres %.3e split %d wall_ms %.1f\n", outer, last_it,
                   ff > 0 ? std::sqrt(rr / ff) : 0.0, (int)split,
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count());
    if (o->precision == MTO_MIXED && rr_prev > 0.0 && std::sqrt(rr / rr_prev) > 10.0 * asked) split = false;
    rr_prev = rr;
    if (!std::isfinite(rr)) {
      st = mto_fail(h, MTO_ENAN, "mto_solve: non-finite residual");
      break;
    }
    if (ff == 0.0 || (!energy && rr <= o->rtol * o->rtol * ff) || (energy && outer > 0 && step_converged)) {
      // the compliance-accuracy mode stops after a correction solve whose energy test was met:
      // that test bounds the compliance error of u itself (the FP64 residual above is only
      // reported); a correction solve that ran out of iterations is followed by another one
      // while the budget lasts
      st = MTO_OK;
      break;
    }
    if (total >= o->max_iter || outer == max_outer) break;
    int it = 0;
    const int cap = o->inner_max > 0 ? o->inner_max : 1 << 30;
    const int budget = o->max_iter - total < cap ? o->max_iter - total : cap;
    if (o->precision != MTO_MIXED32) {
      // refinement step: K d = r with FP64 vectors (d in s64, from zero), to the inner tolerance
      // relative to the current residual (h->red[0] / h->red[2]), then u += d.  MTO_MIXED applies
      // the split pair inside (until it stalls), MTO_FP64 the FP64 matrices.  Solving for the
      // correction keeps the recursively updated CG residual from drifting away from the true
      // one over thousands of iterations (which stalled one long FP64 PCG at 5e-8 on the dp
      // cantilever).  The last step asks no more than a third of the remaining reduction.
      const double need = o->rtol * std::sqrt(ff / rr) / 3.0;
      const double tol_i = need > itol ? (need < 0.1 ? need : 0.1) : itol;
      // the stopping threshold goes to the device (h->red[6]) so the captured graphs stay valid
      h->host_pinned[33] = tol_i * tol_i * h->host_pinned[nrm ? 2 : 0];
      MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->red + 6, h->host_pinned + 33, sizeof(double),
                                                cudaMemcpyHostToDevice, h->stream), "copy"));
      asked = tol_i;
      if (energy) {   // compliance base C(u_0) = f^T u_0 + u_0^T r_0, and the residual floor
        h->host_pinned[34] = 1e-26 * h->host_pinned[1];
        MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->eng + 2 + kEnergyRing, h->host_pinned + 34, sizeof(double),
                                                  cudaMemcpyHostToDevice, h->stream), "copy"));
        MTO_TRY(dot64(h, f, u, n, h->red + 12));
        MTO_TRY(dot64(h, u, h->r64, n, h->red + 13));
        add2_kernel<<<1, 32, 0, h->stream>>>(h->red + 12, h->red + 13, h->eng + 1);
        MTO_TRY(mto_after_launch(h, "add2_kernel"));
      }
      h->inner_split = split && o->precision == MTO_MIXED;
      MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->s64, 0, sizeof(double) * n, h->stream), "memset"));
      const mto_status si = energy ? run_cg<double>(h, h->s64, h->r64, pc, deg, 2, h->red + 6, o->rtol, budget, chunk, &it)
                                   : run_cg<double>(h, h->s64, h->r64, pc, deg, nrm, h->red + 6, 1.0, budget, chunk, &it);
      h->inner_split = false;
      MTO_TRY(si);
      step_converged = h->host_flags[0] != 0;
      TimedScope ts(h, F_VECTOR);
      axpy_kernel<<<grd, 256, 0, h->stream>>>(n, h->s64, u);
      MTO_TRY(mto_after_launch(h, "axpy_kernel"));
    } else {
      // refinement step with FP32 vectors: the residual scaled to unit l2 norm
      const double rr2 = h->host_pinned[0];
      const double scale = 1.0 / std::sqrt(rr2);
      {
        TimedScope ts(h, F_VECTOR);
        demote_kernel<<<grd, 256, 0, h->stream>>>(n, h->r64, scale, h->r32, h->x32);
        MTO_TRY(mto_after_launch(h, "demote_kernel"));
      }
      // the inner residual starts at l2 norm 1, Jacobi norm^2 r^T D^-1 r / ||r||^2
      h->host_pinned[32] = nrm ? h->host_pinned[2] / rr2 : 1.0;
      MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->red + 4, h->host_pinned + 32, sizeof(double),
                                                cudaMemcpyHostToDevice, h->stream), "copy"));
      MTO_TRY(run_cg<float>(h, h->x32, h->r32, pc, deg, nrm, h->red + 4, itol * itol, budget, chunk, &it));
      {
        TimedScope ts(h, F_VECTOR);
        promote_kernel<<<grd, 256, 0, h->stream>>>(n, h->x32, 1.0 / scale, u);
        MTO_TRY(mto_after_launch(h, "promote_kernel"));
      }
    }
    total += it;
    last_it = it;
  }
  if (iters_out) *iters_out = total;
  if (relres_out) *relres_out = ff > 0 ? std::sqrt(rr / ff) : 0.0;
  if (st == MTO_ENOCONV) return mto_fail(h, MTO_ENOCONV, "mto_solve: iteration limit reached");
  return st;
}

// ------------------------------------------------------------------------------------------
// Batched solves: the refinement loop of solve() as a resumable state per handle, advanced for all
// handles between shared synchronisations.  Each handle keeps its own stream, workspace and
// captured iteration graphs, so the instances' chunks of CG iterations run concurrently on the GPU
// and the host waits once per round for all of them instead of once per chunk per instance.
// FP64-vector modes only (MTO_FP64, MTO_MIXED).
namespace {
struct BatchJob {
  mto_handle h = nullptr;
  const double* f = nullptr;
  double* u = nullptr;
  const mto_solve_opts* o = nullptr;
  int pc = 0, deg = 4, chunk = 32, max_outer = 50, nrm = 0;
  bool energy = false;
  double itol = 1e-6;
  int phase = 0;   // 0: residual in flight, 1: CG chunk in flight, 2: finished
  int outer = 0, total = 0, budget = 0;
  double rr = 0.0, ff = 0.0, rr_prev = -1.0, asked = 0.0;
  bool split = true;
  bool converged = false;   // the last correction solve met its test
  CGRun<double> run;
  mto_status st = MTO_ENOCONV;
};

void job_finish(BatchJob& j, mto_status st) {
  j.st = st;
  j.phase = 2;
  j.h->inner_split = false;
}

// the top of one refinement step, with the residual of the current u read back
mto_status job_on_residual(BatchJob& j) {
  mto_handle h = j.h;
  const mto_solve_opts* o = j.o;
  residual_take(h, j.nrm, &j.rr, &j.ff);
  if (o->precision == MTO_MIXED && j.rr_prev > 0.0 && std::sqrt(j.rr / j.rr_prev) > 10.0 * j.asked) j.split = false;
  j.rr_prev = j.rr;
  if (!std::isfinite(j.rr)) {
    job_finish(j, mto_fail(h, MTO_ENAN, "mto_solve_batched: non-finite residual"));
    return MTO_OK;
  }
  if (j.ff == 0.0 || (!j.energy && j.rr <= o->rtol * o->rtol * j.ff) || (j.energy && j.outer > 0 && j.converged)) {
    job_finish(j, MTO_OK);
    return MTO_OK;
  }
  if (j.total >= o->max_iter || j.outer == j.max_outer) {
    job_finish(j, mto_fail(h, MTO_ENOCONV, "mto_solve_batched: iteration limit reached"));
    return MTO_OK;
  }
  const int64_t n = h->ndof;
  const int cap = o->inner_max > 0 ? o->inner_max : 1 << 30;
  j.budget = o->max_iter - j.total < cap ? o->max_iter - j.total : cap;
  const double need = o->rtol * std::sqrt(j.ff / j.rr) / 3.0;
  const double tol_i = need > j.itol ? (need < 0.1 ? need : 0.1) : j.itol;
  h->host_pinned[33] = tol_i * tol_i * h->host_pinned[j.nrm ? 2 : 0];
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->red + 6, h->host_pinned + 33, sizeof(double), cudaMemcpyHostToDevice,
                                            h->stream), "copy"));
  j.asked = tol_i;
  if (j.energy) {
    h->host_pinned[34] = 1e-26 * h->host_pinned[1];
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->eng + 2 + kEnergyRing, h->host_pinned + 34, sizeof(double),
                                              cudaMemcpyHostToDevice, h->stream), "copy"));
    MTO_TRY(dot64(h, j.f, j.u, n, h->red + 12));
    MTO_TRY(dot64(h, j.u, h->r64, n, h->red + 13));
    add2_kernel<<<1, 32, 0, h->stream>>>(h->red + 12, h->red + 13, h->eng + 1);
    MTO_TRY(mto_after_launch(h, "add2_kernel"));
  }
  h->inner_split = j.split && o->precision == MTO_MIXED;
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->s64, 0, sizeof(double) * n, h->stream), "memset"));
  if (j.energy) MTO_TRY(cg_prepare<double>(h, j.run, h->s64, h->r64, j.pc, j.deg, 2, h->red + 6, o->rtol, j.chunk));
  else MTO_TRY(cg_prepare<double>(h, j.run, h->s64, h->r64, j.pc, j.deg, j.nrm, h->red + 6, 1.0, j.chunk));
  MTO_TRY(cg_launch_chunk<double>(h, j.run));
  j.phase = 1;
  return MTO_OK;
}

// after a chunk: the next chunk, or the end of the correction solve and the next residual
mto_status job_on_chunk(BatchJob& j) {
  mto_handle h = j.h;
  const bool fin = cg_check<double>(h, j.run);
  if (!fin && j.run.k < j.budget) return cg_launch_chunk<double>(h, j.run);
  int it = 0;
  const mto_status si = cg_result<double>(h, j.run, &it);
  h->inner_split = false;
  j.converged = h->host_flags[0] != 0;
  j.total += it;
  if (si != MTO_OK) {
    job_finish(j, si);
    return MTO_OK;
  }
  {
    TimedScope ts(h, F_VECTOR);
    axpy_kernel<<<grid_for(h->ndof, 256, 152 * 4), 256, 0, h->stream>>>(h->ndof, h->s64, j.u);
    MTO_TRY(mto_after_launch(h, "axpy_kernel"));
  }
  ++j.outer;
  MTO_TRY(residual_enqueue(h, j.f, j.u));
  j.phase = 0;
  return MTO_OK;
}
}  // namespace

mto_status solve_batched(mto_handle* hs, int n, const double* const* f, double* const* u, const mto_solve_opts* o,
                         int32_t* iters, double* relres, mto_status* status) {
  std::vector<BatchJob> jobs(n);
  // start: preconditioner set-up, start vectors, first residuals (in flight on every stream)
  for (int i = 0; i < n; ++i) {
    BatchJob& j = jobs[i];
    mto_handle h = hs[i];
    j.h = h;
    j.f = f[i];
    j.u = u[i];
    j.o = o;
    j.pc = o->precond;
    j.deg = o->mg_degree > 0 ? o->mg_degree : 4;
    j.chunk = o->check_every < 2 ? 2 : (o->check_every + 1) / 2 * 2;
    j.max_outer = o->max_outer > 0 ? o->max_outer : 50;
    j.energy = o->norm == MTO_NORM_ENERGY;
    j.nrm = o->norm == MTO_NORM_JACOBI ? 1 : 0;
    j.itol = o->inner_rtol > 0 ? o->inner_rtol : 1e-6;
    mto_status st = MTO_OK;
    if (j.deg > 16) st = mto_fail(h, MTO_EINVAL, "mto_solve_batched: mg_degree above 16");
    if (st == MTO_OK && j.pc == MTO_PREC_SCHWARZ && !h->schwarz_valid) st = build_schwarz(h);
    if (st == MTO_OK && j.pc == MTO_PREC_MG) st = mg_select_smoother(h, o->mg_smoother);
    if (st == MTO_OK && j.pc == MTO_PREC_MG) st = mg_select_operator(h, o->mg_operator);
    if (st == MTO_OK && j.pc == MTO_PREC_MG && !h->mg_valid) st = mg_build(h);
    if (st == MTO_OK) {
      if (!o->warm_start) st = mto_cuda_check(h, cudaMemsetAsync(j.u, 0, sizeof(double) * h->ndof, h->stream), "memset");
      else {
        mask_kernel<<<grid_for(h->ndof, 256, 152 * 4), 256, 0, h->stream>>>(h->ndof, h->invd64, j.u);
        st = mto_after_launch(h, "mask_kernel");
      }
    }
    if (st == MTO_OK) st = residual_enqueue(h, j.f, j.u);
    if (st != MTO_OK) job_finish(j, st);
  }
  // rounds: one synchronisation of every unfinished stream, then each job's next step
  for (;;) {
    bool any = false;
    for (auto& j : jobs) {
      if (j.phase == 2) continue;
      any = true;
      const mto_status ss = mto_cuda_check(j.h, cudaStreamSynchronize(j.h->stream), "sync");
      if (ss != MTO_OK) job_finish(j, ss);
    }
    if (!any) break;
    for (auto& j : jobs) {
      if (j.phase == 2) continue;
      const mto_status ss = j.phase == 0 ? job_on_residual(j) : job_on_chunk(j);
      if (ss != MTO_OK) job_finish(j, ss);
    }
  }
  mto_status first = MTO_OK;
  for (int i = 0; i < n; ++i) {
    if (iters) iters[i] = jobs[i].total;
    if (relres) relres[i] = jobs[i].ff > 0 ? std::sqrt(jobs[i].rr / jobs[i].ff) : 0.0;
    if (status) status[i] = jobs[i].st;
    if (first == MTO_OK && jobs[i].st != MTO_OK) first = jobs[i].st;
  }
  return first;
}

}  // namespace mto
