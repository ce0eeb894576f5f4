// Step (b): the matrix-free operator y = sum_e P_e^T K_e P_e x and the Jacobi-preconditioned CG
// solve of K u = f (Eq. 1).  The paper does not name its solver; conformity across p-jumps uses
// the minimum-rule prolongations P_e built by mto_setup.
//
// Operator layout: one element per group of W lanes (one warp for Q3), element matrices in the
// circulant-diagonal layout of mto_internal.cuh; see ebe_kernel.
#include <cmath>
#include <cstdio>
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

// y += sum_e P_e^T K_e P_e x, one element per lane group (W lanes; G elements per warp).
// Lane li owns rows i = li + 32 m.  Element matrices are rows of the circulant-diagonal layout:
// at step k lane i reads D_k[i] = K[i][i+k], adds K[i][i+k] x_{i+k} to its row (x_{i+k} by
// shuffle) and hands K[i][i+k] x_i to the lane owning row i+k (shuffle from the receiver's side),
// so each stored entry serves both triangles.  kDF = false: FP64 matrices and arithmetic (plain
// FP64 path).  kDF = true: the split-precision pair on the FP32 pipes with error-free products and
// sums (~48-bit accurate), vectors TX = double (refinement residuals) or float (inner iterations).
// Also returns x^T y (= sum_e x_e^T K_e x_e) into *pq so the CG curvature needs no extra pass.
template <int PO, bool kDF, typename TX>
__global__ void __launch_bounds__(256) ebe_kernel(const double* __restrict__ K64, const float* __restrict__ Kh,
                                                  const float* __restrict__ Kl, int L, int n,
                                                  const int* __restrict__ gmap, const Constraint* __restrict__ cons,
                                                  const TX* __restrict__ x, TX* __restrict__ y,
                                                  double* __restrict__ pq, const int* __restrict__ done) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN, ND = NE / 2 + 1;
  constexpr int W = WarpShape<NE>::W, G = WarpShape<NE>::G, M = WarpShape<NE>::M;
  constexpr bool kSplitX = kDF && sizeof(TX) == 8;
  if (done && *done) return;
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
          const float al = vi ? __ldg(Kl + rowb + k * NE + i) : 0.0f;
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
      if (pq) dot += xd[m] * yv;
    }
  }
  if (pq) {
    double s = block_sum(dot);
    if (threadIdx.x == 0) atomicAdd(pq, s);
  }
}

template <int PO, bool kDF, typename TX>
void launch_ebe(mto_handle h, const PClass& c, const TX* x, TX* y, double* pq, const int* done) {
  constexpr int NE = 2 * (PO + 1) * (PO + 1);
  constexpr int G = WarpShape<NE>::G;
  const int warps = (c.n + G - 1) / G;
  const int blocks = grid_for((int64_t)warps * 32, 256, 152 * 8);
  ebe_kernel<PO, kDF, TX><<<blocks, 256, 0, h->stream>>>(kDF ? nullptr : c.K64, c.K32, c.K32lo, c.L, c.n, c.gmap,
                                                          h->cons_d, x, y, pq, done);
}

// The assembled operator: FP64 element matrices on the FP64 pipes (plain FP64 path), or the
// split-precision pair on the FP32 pipes (mixed path) with FP64 (residual) or FP32 (inner) vectors.
template <typename T>
mto_status apply_all(mto_handle h, const T* x, T* y, double* pq, const int* done) {
  const bool df = h->built_precision == MTO_MIXED;
  TimedScope ts(h, df ? (sizeof(T) == 8 ? F_APPLYDF64 : F_APPLY32) : F_APPLY64);
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    const PClass& c = h->pc[p];
    if (c.n == 0) continue;
    if (df) {
      if (!c.K32 || !c.K32lo) return mto_fail(h, MTO_EINVAL, "split-precision element matrices are not built");
      switch (p) {
        case 1: launch_ebe<1, true, T>(h, c, x, y, pq, done); break;
        case 2: launch_ebe<2, true, T>(h, c, x, y, pq, done); break;
        case 3: launch_ebe<3, true, T>(h, c, x, y, pq, done); break;
        case 4: launch_ebe<4, true, T>(h, c, x, y, pq, done); break;
        case 5: launch_ebe<5, true, T>(h, c, x, y, pq, done); break;
        case 6: launch_ebe<6, true, T>(h, c, x, y, pq, done); break;
      }
    } else {
      if constexpr (sizeof(T) == 8) {
        if (!c.K64) return mto_fail(h, MTO_EINVAL, "FP64 element matrices are not built");
        switch (p) {
          case 1: launch_ebe<1, false, T>(h, c, x, y, pq, done); break;
          case 2: launch_ebe<2, false, T>(h, c, x, y, pq, done); break;
          case 3: launch_ebe<3, false, T>(h, c, x, y, pq, done); break;
          case 4: launch_ebe<4, false, T>(h, c, x, y, pq, done); break;
          case 5: launch_ebe<5, false, T>(h, c, x, y, pq, done); break;
          case 6: launch_ebe<6, false, T>(h, c, x, y, pq, done); break;
        }
      } else {
        return mto_fail(h, MTO_EINVAL, "FP32 vectors need the split-precision build");
      }
    }
    MTO_TRY(mto_after_launch(h, "ebe_kernel"));
  }
  return MTO_OK;
}

// ---------------------------------------------------------------------------------- PCG kernels
// Iteration k uses scalar slot k & 3 for its reductions; the previous iteration's r^T z is in
// slot (k + 3) & 3.  Slot (k + 2) & 3 is cleared here for iteration k + 2 (no kernel of
// iterations k and k + 1 reads it).

// x += alpha p; r -= alpha q (free DOFs, invd != 0), q = 0; accumulate r^T D^-1 r and r^T r.
template <typename T>
__global__ void __launch_bounds__(256) cg_update_kernel(int64_t n, T* __restrict__ x, T* __restrict__ r,
                                                        const T* __restrict__ p, T* __restrict__ q,
                                                        const T* __restrict__ invd, Scalars* __restrict__ S,
                                                        int k, const int* __restrict__ done) {
  if (*done) return;
  const double alpha = S[(k + 3) & 3].rz / S[k & 3].pq;
  const T a = (T)alpha;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T inv = invd[i];
    T qi = q[i];
    q[i] = 0;
    if (inv != (T)0) {
      x[i] = fma(a, p[i], x[i]);
      T ri = fma(-a, qi, r[i]);
      r[i] = ri;
      double rd = (double)ri;
      rz += rd * rd * (double)inv;
      rr += rd * rd;
    }
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) atomicAdd(&S[k & 3].rz, rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) atomicAdd(&S[k & 3].rr, rr);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Scalars z = {0.0, 0.0, 0.0, 0.0};
    S[(k + 2) & 3] = z;
  }
}

// p = D^-1 r + beta p; convergence / breakdown test on slot k (block 0): r^T r (use_rz = 0) or
// r^T D^-1 r (use_rz = 1) against tol2 * (*ref).
template <typename T>
__global__ void __launch_bounds__(256) cg_direction_kernel(int64_t n, const T* __restrict__ r, T* __restrict__ p,
                                                           const T* __restrict__ invd, Scalars* __restrict__ S,
                                                           int k, const double* __restrict__ ref, double tol2,
                                                           int use_rz, int* __restrict__ done, int* __restrict__ err) {
  if (*done) return;
  const double beta = S[k & 3].rz / S[(k + 3) & 3].rz;
  const T b = (T)beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], invd[i] * r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double rr = S[k & 3].rr;
    double pq = S[k & 3].pq;
    double crit = use_rz ? S[k & 3].rz : rr;
    if (!isfinite(rr) || !isfinite(S[k & 3].rz) || !(pq > 0.0)) {
      if (!(rr == 0.0)) *err = MTO_ENAN;
      *done = k + 1;
    } else if (crit <= tol2 * (*ref)) {
      *done = k + 1;
    }
  }
}

// p = D^-1 r; slot 3 <- (r^T D^-1 r, r^T r) (the "iteration -1" values); clears slots 0 and 1.
template <typename T>
__global__ void __launch_bounds__(256) cg_init_kernel(int64_t n, const T* __restrict__ r, T* __restrict__ p,
                                                      const T* __restrict__ invd, Scalars* __restrict__ S) {
  double rz = 0.0, rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ri = r[i];
    p[i] = invd[i] * ri;
    double rd = (double)ri;
    rz += rd * rd * (double)invd[i];
    rr += rd * rd;
  }
  rz = block_sum(rz);
  if (threadIdx.x == 0) atomicAdd(&S[3].rz, rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) atomicAdd(&S[3].rr, rr);
}

// r = f - Ku on free DOFs, 0 on supports; out[0] += r^T r, out[1] += f^T f, out[2] += r^T D^-1 r,
// out[3] += f^T D^-1 f (free DOFs)
__global__ void __launch_bounds__(256) residual_kernel(int64_t n, const double* __restrict__ f,
                                                       const double* __restrict__ Ku, const double* __restrict__ invd,
                                                       double* __restrict__ r, double* __restrict__ out) {
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
  if (threadIdx.x == 0) atomicAdd(&out[0], rr);
  ff = block_sum(ff);
  if (threadIdx.x == 0) atomicAdd(&out[1], ff);
  rd = block_sum(rd);
  if (threadIdx.x == 0) atomicAdd(&out[2], rd);
  fd = block_sum(fd);
  if (threadIdx.x == 0) atomicAdd(&out[3], fd);
}

// r32 = (float)(r * scale), x32 = 0, q32 = 0
__global__ void __launch_bounds__(256) demote_kernel(int64_t n, const double* __restrict__ r, double scale,
                                                     float* __restrict__ r32, float* __restrict__ x32,
                                                     float* __restrict__ q32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r32[i] = (float)(r[i] * scale);
    x32[i] = 0.0f;
    q32[i] = 0.0f;
  }
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
                                                  double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// FP64 residual r = f - K u (masked) and its squared norms into h->red[0..3] (l2: r, f; Jacobi:
// r, f); returns host copies of the pair selected by `norm`.
mto_status true_residual(mto_handle h, const double* f, const double* u, int norm, double* rr, double* ff) {
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->q64, 0, sizeof(double) * h->ndof, h->stream), "memset"));
  MTO_TRY(apply_all<double>(h, u, h->q64, nullptr, nullptr));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->red, 0, 4 * sizeof(double), h->stream), "memset"));
  TimedScope ts(h, F_VECTOR);
  residual_kernel<<<grid_for(h->ndof, 256, 152 * 4), 256, 0, h->stream>>>(h->ndof, f, h->q64, h->invd64, h->r64, h->red);
  MTO_TRY(mto_after_launch(h, "residual_kernel"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned, h->red, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  timing_harvest(h);
  *rr = h->host_pinned[norm ? 2 : 0];
  *ff = h->host_pinned[norm ? 3 : 1];
  return MTO_OK;
}

// Preconditioned CG on (x, r, p, q) of type T: r is the current residual of x (free DOFs,
// zero on supports), q is zero.  Stops when r^T r <= tol2 * (*ref) or after max_it iterations.
template <typename T>
mto_status run_pcg(mto_handle h, T* x, T* r, T* p, T* q, const T* invd, const double* ref, double tol2,
                   int use_rz, int max_it, int check_every, int* iters) {
  const int64_t n = h->ndof;
  const int blk = 256, grd = grid_for(n, blk, 152 * 4);
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->scal, 0, sizeof(Scalars) * kSlots, h->stream), "memset"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(int), h->stream), "memset"));
  cg_init_kernel<T><<<grd, blk, 0, h->stream>>>(n, r, p, invd, h->scal);
  MTO_TRY(mto_after_launch(h, "cg_init_kernel"));
  int k = 0;
  int done = 0, err = 0;
  while (k < max_it) {
    int chunk = check_every < max_it - k ? check_every : max_it - k;
    for (int j = 0; j < chunk; ++j, ++k) {
      MTO_TRY(apply_all<T>(h, p, q, &h->scal[k & 3].pq, h->flags));
      TimedScope ts(h, F_VECTOR);
      cg_update_kernel<T><<<grd, blk, 0, h->stream>>>(n, x, r, p, q, invd, h->scal, k, h->flags);
      MTO_TRY(mto_after_launch(h, "cg_update_kernel"));
      cg_direction_kernel<T><<<grd, blk, 0, h->stream>>>(n, r, p, invd, h->scal, k, ref, tol2, use_rz,
                                                         h->flags, h->flags + 1);
      MTO_TRY(mto_after_launch(h, "cg_direction_kernel"));
    }
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned, h->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copy"));
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    timing_harvest(h);
    const int* fl = reinterpret_cast<const int*>(h->host_pinned);
    done = fl[0];
    err = fl[1];
    if (done) break;
  }
  *iters = done ? done : k;
  if (err) return mto_fail(h, MTO_ENAN, "PCG breakdown: non-finite or non-positive curvature");
  // leave q zero for the next use (the update kernel clears it; an early exit may not have)
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(q, 0, sizeof(T) * n, h->stream), "memset"));
  return MTO_OK;
}

// squared l2 norm of the last true residual (host copy)
double rr0_l2(mto_handle h) { return h->host_pinned[0]; }

}  // namespace

mto_status apply64(mto_handle h, const double* x, double* y, double* pq) {
  return apply_all<double>(h, x, y, pq, nullptr);
}

mto_status apply32(mto_handle h, const float* x, float* y, double* pq) {
  return apply_all<float>(h, x, y, pq, nullptr);
}

mto_status dot64(mto_handle h, const double* a, const double* b, int64_t n, double* out_dev) {
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(out_dev, 0, sizeof(double), h->stream), "memset"));
  dot_kernel<<<grid_for(n, 256, 152 * 4), 256, 0, h->stream>>>(n, a, b, out_dev);
  return mto_after_launch(h, "dot_kernel");
}

mto_status solve(mto_handle h, const double* f, double* u, const mto_solve_opts* o, int32_t* iters_out,
                 double* relres_out) {
  const int64_t n = h->ndof;
  const int grd = grid_for(n, 256, 152 * 4);
  if (!o->warm_start) MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(u, 0, sizeof(double) * n, h->stream), "memset"));
  else {
    mask_kernel<<<grd, 256, 0, h->stream>>>(n, h->invd64, u);
    MTO_TRY(mto_after_launch(h, "mask_kernel"));
  }
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->q32, 0, sizeof(float) * n, h->stream), "memset"));
  int total = 0;
  double rr = 0.0, ff = 0.0;
  const int max_outer = o->precision == MTO_MIXED ? (o->max_outer > 0 ? o->max_outer : 50) : 20;
  mto_status st = MTO_ENOCONV;
  const int nrm = o->norm == MTO_NORM_JACOBI ? 1 : 0;
  for (int outer = 0; outer <= max_outer; ++outer) {
    MTO_TRY(true_residual(h, f, u, nrm, &rr, &ff));
    if (!std::isfinite(rr)) {
      st = mto_fail(h, MTO_ENAN, "mto_solve: non-finite residual");
      break;
    }
    if (ff == 0.0 || rr <= o->rtol * o->rtol * ff) {
      st = MTO_OK;
      break;
    }
    if (total >= o->max_iter || outer == max_outer) break;
    int it = 0;
    if (o->precision == MTO_FP64) {
      // h->red[1] (h->red[3]) holds f^T f (f^T D^-1 f): CG runs until the residual norm meets rtol
      MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->q64, 0, sizeof(double) * n, h->stream), "memset"));
      MTO_TRY(run_pcg<double>(h, u, h->r64, h->p64, h->q64, h->invd64, h->red + (nrm ? 3 : 1), o->rtol * o->rtol,
                              nrm, o->max_iter - total, o->check_every, &it));
    } else {
      const double scale = 1.0 / std::sqrt(rr0_l2(h));
      TimedScope ts(h, F_VECTOR);
      demote_kernel<<<grd, 256, 0, h->stream>>>(n, h->r64, scale, h->r32, h->x32, h->q32);
      MTO_TRY(mto_after_launch(h, "demote_kernel"));
      // the inner residual starts at (scaled) norm 1 in l2, and at r^T D^-1 r / ||r||^2 in the
      // Jacobi norm: h->red[4] = the reference of the inner test
      const double ref = nrm ? h->host_pinned[2] / rr0_l2(h) : 1.0;
      h->host_pinned[32] = ref;
      MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->red + 4, h->host_pinned + 32, sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy"));
      double itol = o->inner_rtol > 0 ? o->inner_rtol : 1e-4;
      MTO_TRY(run_pcg<float>(h, h->x32, h->r32, h->p32, h->q32, h->invd32, h->red + 4, itol * itol,
                             nrm, o->max_iter - total, o->check_every, &it));
      TimedScope ts2(h, F_VECTOR);
      promote_kernel<<<grd, 256, 0, h->stream>>>(n, h->x32, 1.0 / scale, u);
      MTO_TRY(mto_after_launch(h, "promote_kernel"));
    }
    total += it;
  }
  if (iters_out) *iters_out = total;
  if (relres_out) *relres_out = ff > 0 ? std::sqrt(rr / ff) : 0.0;
  if (st == MTO_ENOCONV) return mto_fail(h, MTO_ENOCONV, "mto_solve: iteration limit reached");
  return st;
}

}  // namespace mto
