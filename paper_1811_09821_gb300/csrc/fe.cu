// Step (a) and its tables: subcell stiffness tables K0_s (App. B composite integration), the QR
// load-transfer tables, the element build K_e = sum_s E(rho_s) K0_s (Eqs. 2-3), and the Jacobi
// diagonal of the assembled operator.
#include <cmath>
#include <vector>

#include "mto_internal.cuh"

namespace mto {
namespace {

// K0T[c][s] = integral over subcell s of (B^T D0 B)_{ij}, c = packed (i, j), unit modulus.
// The (p+1) x (p+1) Gauss rule mapped to the subcell is exact (the integrand has degree <= 2p per
// axis on an affine square).  One thread per (c, s).
__global__ void k0_kernel(int p, int d, double nu, double hx, double hy, double* __restrict__ K0T) {
  const int S = d * d, n1 = p + 1, ne = 2 * n1 * n1, P = packed_size(ne);
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P * S) return;
  int c = idx / S, s = idx - c * S;
  int i = 0, rem = c;
  while (rem >= ne - i) {
    rem -= ne - i;
    ++i;
  }
  int j = i + rem;
  double z[kPMaxTab + 1], gx[kPMaxTab + 1], gw[kPMaxTab + 1];
  gll_nodes(p, z);
  gauss_rule(n1, gx, gw);
  const double f = 1.0 / (1.0 - nu * nu);
  const double D11 = f, D12 = f * nu, D33 = f * 0.5 * (1.0 - nu);
  const int si = s % d, sj = s / d;
  const int ni = i >> 1, ci = i & 1, nj = j >> 1, cj = j & 1;
  const int ai = ni % n1, bi = ni / n1, aj = nj % n1, bj = nj / n1;
  double sum = 0.0;
  for (int qy = 0; qy < n1; ++qy) {
    double eta = -1.0 + (2.0 * sj + 1.0 + gx[qy]) / d;
    for (int qx = 0; qx < n1; ++qx) {
      double xi = -1.0 + (2.0 * si + 1.0 + gx[qx]) / d;
      double wq = gw[qx] * gw[qy] * (hx / (2.0 * d)) * (hy / (2.0 * d));
      double Nxi = lagrange_der(z, n1, ai, xi) * lagrange_val(z, n1, bi, eta) * (2.0 / hx);
      double Nyi = lagrange_val(z, n1, ai, xi) * lagrange_der(z, n1, bi, eta) * (2.0 / hy);
      double Nxj = lagrange_der(z, n1, aj, xi) * lagrange_val(z, n1, bj, eta) * (2.0 / hx);
      double Nyj = lagrange_val(z, n1, aj, xi) * lagrange_der(z, n1, bj, eta) * (2.0 / hy);
      // B columns: u_x -> (Nx, 0, Ny), u_y -> (0, Ny, Nx)
      double bi0 = ci == 0 ? Nxi : 0.0, bi1 = ci == 0 ? 0.0 : Nyi, bi2 = ci == 0 ? Nyi : Nxi;
      double bj0 = cj == 0 ? Nxj : 0.0, bj1 = cj == 0 ? 0.0 : Nyj, bj2 = cj == 0 ? Nyj : Nxj;
      double e = bi0 * (D11 * bj0 + D12 * bj1) + bi1 * (D12 * bj0 + D11 * bj1) + bi2 * D33 * bj2;
      sum += wq * e;
    }
  }
  K0T[idx] = sum;
}

// Scalar load-transfer table of the QR indicator for order p -> p + 1:
// R = M^(p+1,p) M^(p)^-1, M^(p)_{kl} = int N_k^p N_l^p, M^(p+1,p)_{jk} = int N_j^(p+1) N_k^p,
// integrated exactly by a (p+2)-point Gauss rule per axis.  Thread 0 forms and factors M^(p)
// (Cholesky) in shared memory; thread t solves for row t of R.
__global__ void qr_table_kernel(int p, double hx, double hy, double* __restrict__ R) {
  constexpr int NA = (kPMaxTab) * (kPMaxTab);        // max (p+1)^2 for p <= MTO_P_MAX
  constexpr int NB = (kPMaxTab + 1) * (kPMaxTab + 1);
  __shared__ double M[NA * NA];
  __shared__ double Mb[NB * NA];
  const int n1 = p + 1, n2 = p + 2, na = n1 * n1, nb = n2 * n2;
  if (threadIdx.x == 0) {
    double z1[kPMaxTab + 1], z2[kPMaxTab + 1], gx[kPMaxTab + 2], gw[kPMaxTab + 2];
    gll_nodes(p, z1);
    gll_nodes(p + 1, z2);
    int nq = p + 2;
    gauss_rule(nq, gx, gw);
    for (int k = 0; k < na * na; ++k) M[k] = 0.0;
    for (int k = 0; k < nb * na; ++k) Mb[k] = 0.0;
    const double jac = 0.25 * hx * hy;
    for (int qy = 0; qy < nq; ++qy)
      for (int qx = 0; qx < nq; ++qx) {
        double w = gw[qx] * gw[qy] * jac;
        double N1[NA], N2[NB];
        for (int b = 0; b < n1; ++b)
          for (int a = 0; a < n1; ++a)
            N1[b * n1 + a] = lagrange_val(z1, n1, a, gx[qx]) * lagrange_val(z1, n1, b, gx[qy]);
        for (int b = 0; b < n2; ++b)
          for (int a = 0; a < n2; ++a)
            N2[b * n2 + a] = lagrange_val(z2, n2, a, gx[qx]) * lagrange_val(z2, n2, b, gx[qy]);
        for (int k = 0; k < na; ++k)
          for (int l = 0; l < na; ++l) M[k * na + l] += w * N1[k] * N1[l];
        for (int j = 0; j < nb; ++j)
          for (int k = 0; k < na; ++k) Mb[j * na + k] += w * N2[j] * N1[k];
      }
    // Cholesky M = L L^T in place (lower triangle)
    for (int k = 0; k < na; ++k) {
      double s = M[k * na + k];
      for (int m = 0; m < k; ++m) s -= M[k * na + m] * M[k * na + m];
      s = sqrt(s);
      M[k * na + k] = s;
      for (int i = k + 1; i < na; ++i) {
        double t = M[i * na + k];
        for (int m = 0; m < k; ++m) t -= M[i * na + m] * M[k * na + m];
        M[i * na + k] = t / s;
      }
    }
  }
  __syncthreads();
  // row j of R solves M r = (row j of Mb)^T  (M symmetric)
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    double y[NA];
    for (int k = 0; k < na; ++k) {
      double t = Mb[j * na + k];
      for (int m = 0; m < k; ++m) t -= M[k * na + m] * y[m];
      y[k] = t / M[k * na + k];
    }
    for (int k = na - 1; k >= 0; --k) {
      double t = y[k];
      for (int m = k + 1; m < na; ++m) t -= M[m * na + k] * y[m];
      y[k] = t / M[k * na + k];
    }
    for (int k = 0; k < na; ++k) R[j * na + k] = y[k];
  }
}

// K_e = sum_s E(rho_s) K0_s for the elements of one (p, d) class, FP64 FMAs; writes the FP64
// matrices (FP64 path) or the split-precision pair hi = fl32(K_e), lo = fl32(K_e - hi) (mixed
// path) into the order class's interleaved layout.
// Block: 32 elements x 8 column groups; the 32 elements' moduli are staged in shared memory.
__global__ void __launch_bounds__(256) build_simt_kernel(
    int n, int S, int P, const int* __restrict__ elem, const int* __restrict__ slot,
    const int64_t* __restrict__ design_off, const double* __restrict__ rho, double E0, double Emin, double q,
    const double* __restrict__ K0T, int L, const int2* __restrict__ dpos, double* __restrict__ K64,
    float* __restrict__ K32, float* __restrict__ K32lo) {
  extern __shared__ double Es[];  // [32][Sp], Sp odd so that the 32 rows fall in distinct banks
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int base = blockIdx.x * 32;
  const int Sp = S | 1;
  for (int k = threadIdx.x; k < 32 * S; k += blockDim.x) {
    int el = k / S, s = k - el * S;
    double v = 0.0;
    if (base + el < n) {
      double r = rho[design_off[elem[base + el]] + s];
      v = Emin + pow(r, q) * (E0 - Emin);
    }
    Es[el * Sp + s] = v;
  }
  __syncthreads();
  const int k = base + lane;
  if (k >= n) return;
  const int sl = slot[k];
  const double* Ek = Es + lane * Sp;
  for (int c = grp; c < P; c += 8) {
    const double* kc = K0T + (size_t)c * S;
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc = fma(Ek[s], kc[s], acc);
    const int2 ps = dpos[c];
    const size_t o1 = (size_t)sl * L + ps.x, o2 = (size_t)sl * L + ps.y;
    if (K64) {
      K64[o1] = acc;
      if (ps.y >= 0) K64[o2] = acc;
    }
    if (K32) {
      const float hi = (float)acc, lo = (float)(acc - (double)hi);
      K32[o1] = hi;
      K32lo[o1] = lo;
      if (ps.y >= 0) {
        K32[o2] = hi;
        K32lo[o2] = lo;
      }
    }
  }
}

// Diagonal of sum_e P_e^T K_e P_e.  One thread per element of an order class.  Unconstrained
// local nodes add K_ii to their node; elements with constrained nodes add sum_{i,j} w_i w_j K_ij
// over all local pairs that reach the same global node.
template <int PO>
__global__ void diag_kernel(int n, int L, const int2* __restrict__ dpos, const int* __restrict__ gmap,
                            const Constraint* __restrict__ cons, const double* __restrict__ K64,
                            const float* __restrict__ Kh, const float* __restrict__ Kl,
                            double* __restrict__ diag) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  auto Kij = [&](int i, int j) {
    if (i > j) { int tmp = i; i = j; j = tmp; }
    return k_entry(K64, Kh, Kl, L, t, dpos[packed_index(NE, i, j)].x);
  };
  const int* gm = gmap + (size_t)t * NN;
  bool constrained = false;
  for (int ln = 0; ln < NN; ++ln) constrained |= gm[ln] < 0;
  if (!constrained) {
    for (int ln = 0; ln < NN; ++ln) {
      int g = gm[ln];
      atomicAdd(&diag[2 * (size_t)g], Kij(2 * ln, 2 * ln));
      atomicAdd(&diag[2 * (size_t)g + 1], Kij(2 * ln + 1, 2 * ln + 1));
    }
    return;
  }
  for (int l1 = 0; l1 < NN; ++l1) {
    int g1 = gm[l1];
    int c1 = g1 >= 0 ? 1 : cons[-g1 - 1].cnt;
    for (int k1 = 0; k1 < c1; ++k1) {
      int node = g1 >= 0 ? g1 : cons[-g1 - 1].node[k1];
      double w1 = g1 >= 0 ? 1.0 : cons[-g1 - 1].w[k1];
      if (w1 == 0.0) continue;
      double sx = 0.0, sy = 0.0;
      for (int l2 = 0; l2 < NN; ++l2) {
        int g2 = gm[l2];
        int c2 = g2 >= 0 ? 1 : cons[-g2 - 1].cnt;
        for (int k2 = 0; k2 < c2; ++k2) {
          int node2 = g2 >= 0 ? g2 : cons[-g2 - 1].node[k2];
          if (node2 != node) continue;
          double w2 = g2 >= 0 ? 1.0 : cons[-g2 - 1].w[k2];
          sx += w2 * Kij(2 * l1, 2 * l2);
          sy += w2 * Kij(2 * l1 + 1, 2 * l2 + 1);
        }
      }
      atomicAdd(&diag[2 * (size_t)node], w1 * sx);
      atomicAdd(&diag[2 * (size_t)node + 1], w1 * sy);
    }
  }
}

__global__ void invdiag_kernel(int64_t n, const double* __restrict__ diag, double* __restrict__ invd64,
                               float* __restrict__ invd32, int* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double dv = diag[i];
    double v = 1.0 / dv;
    if (!(dv > 0.0) || !isfinite(v)) {
      flags[2] = 1;
      v = 0.0;
    }
    invd64[i] = v;
    invd32[i] = (float)v;
  }
}

__global__ void zero_fixed_kernel(int64_t n, const int64_t* __restrict__ fixed, double* __restrict__ invd64,
                                  float* __restrict__ invd32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    invd64[fixed[i]] = 0.0;
    invd32[fixed[i]] = 0.0f;
  }
}

__global__ void gather_element_matrix_kernel(int P, int L, const int2* __restrict__ dpos, int slot,
                                             const double* __restrict__ K64, const float* __restrict__ Kh,
                                             const float* __restrict__ Kl, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P; c += gridDim.x * blockDim.x)
    out[c] = k_entry(K64, Kh, Kl, L, slot, dpos[c].x);
}

template <int PO>
void launch_diag(mto_handle h, const PClass& c, double* diag) {
  diag_kernel<PO><<<grid_for(c.n, 128, 1 << 30), 128, 0, h->stream>>>(c.n, c.L, c.dpos, c.gmap, h->cons_d,
                                                                      c.K64, c.K32, c.K32lo, diag);
}

// Element-block (additive Schwarz) preconditioner M^-1 = sum_e P_e^T B_e P_e with
// B_e = (K_e + Delta_e)^-1 on the element's local DOFs.  Delta_e adds, at each unconstrained local
// DOF, the rest of the assembled diagonal (the neighbours' share; a hanging DOF of a p-jump edge
// takes the weighted diagonal sum_k w_k^2 D(g_k) of the global DOFs it interpolates), so
// K_e + Delta_e is SPD and
// holds the element's near-null modes exactly (those of solid/void elements, whose stiffness can
// be 1e-10 of the element's largest, which point Jacobi cannot see).  Supported DOFs are
// decoupled (unit row and column): B_e maps their zero residual to zero.  One warp per element:
// FP64 in-place Gauss-Jordan inversion of the SPD block in shared memory, symmetrised, written in
// the circulant-diagonal layout (FP64, or the split-precision pair).
template <int PO>
__global__ void schwarz_kernel(int n, int L, const int2* __restrict__ dpos, const int* __restrict__ gmap,
                               const Constraint* __restrict__ cons,
                               const double* __restrict__ K64, const float* __restrict__ Kh,
                               const float* __restrict__ Kl, const double* __restrict__ diag,
                               const double* __restrict__ invd, double* __restrict__ B64, float* __restrict__ Bh,
                               float* __restrict__ Bl) {
  constexpr int N1 = PO + 1, NN = N1 * N1, NE = 2 * NN, LDA = NE + 1, P = NE * (NE + 1) / 2;
  extern __shared__ double sm[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* A = sm + (size_t)warp * NE * LDA;
  int* fx = reinterpret_cast<int*>(sm + (size_t)wpb * NE * LDA) + warp * NE;
  for (int e = blockIdx.x * wpb + warp; e < n; e += gridDim.x * wpb) {
    for (int idx = lane; idx < NE * NE; idx += 32) {
      const int i = idx / NE, j = idx - (idx / NE) * NE;
      const int a = i < j ? i : j, b = i < j ? j : i;
      A[i * LDA + j] = k_entry(K64, Kh, Kl, L, e, dpos[packed_index(NE, a, b)].x);
    }
    __syncwarp();
    for (int i = lane; i < NE; i += 32) {
      const int g = gmap[(size_t)e * NN + (i >> 1)];
      int fixed = 0;
      if (g >= 0) {
        const size_t gd = 2 * (size_t)g + (i & 1);
        if (invd[gd] == 0.0) fixed = 1;
        else A[i * LDA + i] += fmax(diag[gd] - A[i * LDA + i], 0.0);
      } else {
        // a hanging local DOF interpolates free global DOFs: it takes their weighted diagonal
        const Constraint& c = cons[-g - 1];
        double dh = 0.0;
        for (int k = 0; k < c.cnt; ++k) {
          const size_t gd = 2 * (size_t)c.node[k] + (i & 1);
          if (invd[gd] != 0.0) dh += c.w[k] * c.w[k] * diag[gd];
        }
        A[i * LDA + i] += fmax(dh - A[i * LDA + i], 0.0);
      }
      fx[i] = fixed;
    }
    __syncwarp();
    for (int i = lane; i < NE; i += 32)
      for (int j = 0; j < NE; ++j)
        if (fx[i] || fx[j]) A[i * LDA + j] = (i == j) ? 1.0 : 0.0;
    __syncwarp();
    // in-place Gauss-Jordan inversion (SPD: no pivoting)
    for (int k = 0; k < NE; ++k) {
      const double pinv = 1.0 / A[k * LDA + k];
      __syncwarp();
      for (int j = lane; j < NE; j += 32)
        if (j != k) A[k * LDA + j] *= pinv;
      __syncwarp();
      for (int i = lane; i < NE; i += 32) {
        if (i == k) continue;
        const double f = A[i * LDA + k];
        for (int j = 0; j < NE; ++j)
          if (j != k) A[i * LDA + j] -= f * A[k * LDA + j];
        A[i * LDA + k] = -f * pinv;
      }
      __syncwarp();
      if (lane == 0) A[k * LDA + k] = pinv;
      __syncwarp();
    }
    for (int c = lane; c < P; c += 32) {
      int i = 0, rem = c;
      while (rem >= NE - i) {
        rem -= NE - i;
        ++i;
      }
      const int j = i + rem;
      const double v = 0.5 * (A[i * LDA + j] + A[j * LDA + i]);
      const int2 ps = dpos[c];
      const size_t o1 = (size_t)e * L + ps.x, o2 = (size_t)e * L + ps.y;
      if (B64) {
        B64[o1] = v;
        if (ps.y >= 0) B64[o2] = v;
      } else {
        const float hi = (float)v, lo = (float)(v - (double)hi);
        Bh[o1] = hi;
        Bl[o1] = lo;
        if (ps.y >= 0) {
          Bh[o2] = hi;
          Bl[o2] = lo;
        }
      }
    }
    __syncwarp();
  }
}

template <int PO>
mto_status launch_schwarz(mto_handle h, PClass& c) {
  constexpr int NE = 2 * (PO + 1) * (PO + 1);
  const int wpb = NE <= 32 ? 8 : (NE <= 50 ? 4 : 2);
  const size_t smem = (size_t)wpb * NE * (NE + 1) * sizeof(double) + (size_t)wpb * NE * sizeof(int);
  if (smem > 48 * 1024)
    MTO_TRY(mto_cuda_check(h, cudaFuncSetAttribute(schwarz_kernel<PO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem), "cudaFuncSetAttribute"));
  const bool df = h->built_precision == MTO_MIXED;
  const int blocks = grid_for(c.n, wpb, 152 * 8);
  schwarz_kernel<PO><<<blocks, 32 * wpb, smem, h->stream>>>(c.n, c.L, c.dpos, c.gmap, h->cons_d, c.K64, c.K32,
                                                            c.K32lo, h->diag64, h->invd64, df ? nullptr : c.B64,
                                                            c.B32, c.B32lo);
  return mto_after_launch(h, "schwarz_kernel");
}

}  // namespace

mto_status build_schwarz(mto_handle h) {
  TimedScope ts(h, F_PRECOND);
  const bool df = h->built_precision == MTO_MIXED;
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    PClass& c = h->pc[p];
    if (c.n == 0) continue;
    if (!df && !c.B64) MTO_TRY(mto_alloc(h, &c.B64, (size_t)c.L * c.n));
    if (df && !c.B32) {
      MTO_TRY(mto_alloc(h, &c.B32, (size_t)c.L * c.n));
      MTO_TRY(mto_alloc(h, &c.B32lo, (size_t)c.L * c.n));
    }
    switch (p) {
      case 1: MTO_TRY(launch_schwarz<1>(h, c)); break;
      case 2: MTO_TRY(launch_schwarz<2>(h, c)); break;
      case 3: MTO_TRY(launch_schwarz<3>(h, c)); break;
      case 4: MTO_TRY(launch_schwarz<4>(h, c)); break;
      case 5: MTO_TRY(launch_schwarz<5>(h, c)); break;
      case 6: MTO_TRY(launch_schwarz<6>(h, c)); break;
    }
  }
  h->schwarz_valid = true;
  return MTO_OK;
}

mto_status element_matrix(mto_handle h, int64_t e, double* host_out) {
  const int p = h->p_host[e];
  const PClass& c = h->pc[p];
  int slot = 0;
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(&slot, h->slot_d + e, sizeof(int), cudaMemcpyDeviceToHost), "copy"));
  double* tmp = nullptr;
  MTO_TRY(mto_cuda_check(h, cudaMalloc(&tmp, sizeof(double) * c.P), "cudaMalloc"));
  gather_element_matrix_kernel<<<(c.P + 255) / 256, 256, 0, h->stream>>>(c.P, c.L, c.dpos, slot, c.K64, c.K32,
                                                                         c.K32lo, tmp);
  mto_status st = mto_after_launch(h, "gather_element_matrix_kernel");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(host_out, tmp, sizeof(double) * c.P, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (st == MTO_OK) st = mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  cudaFree(tmp);
  return st;
}

__global__ void gather_element_split_kernel(int P, int L, const int2* __restrict__ dpos, int slot,
                                           const float* __restrict__ Kh, const float* __restrict__ Kl,
                                           float* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P; c += gridDim.x * blockDim.x) {
    const size_t o = (size_t)slot * L + dpos[c].x;
    out[c] = Kh[o];
    out[P + c] = Kl[o];
  }
}

mto_status element_matrix_split(mto_handle h, int64_t e, float* hi, float* lo) {
  const int p = h->p_host[e];
  const PClass& c = h->pc[p];
  if (!c.K32 || !c.K32lo) return mto_fail(h, MTO_EINVAL, "mto_element_matrix_split: no split-precision build");
  int slot = 0;
  MTO_TRY(mto_cuda_check(h, cudaMemcpy(&slot, h->slot_d + e, sizeof(int), cudaMemcpyDeviceToHost), "copy"));
  float* tmp = nullptr;
  MTO_TRY(mto_cuda_check(h, cudaMalloc(&tmp, sizeof(float) * 2 * c.P), "cudaMalloc"));
  gather_element_split_kernel<<<(c.P + 255) / 256, 256, 0, h->stream>>>(c.P, c.L, c.dpos, slot, c.K32, c.K32lo,
                                                                        tmp);
  mto_status st = mto_after_launch(h, "gather_element_split_kernel");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(hi, tmp, sizeof(float) * c.P, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(lo, tmp + c.P, sizeof(float) * c.P, cudaMemcpyDeviceToHost, h->stream),
                        "copy");
  if (st == MTO_OK) st = mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  cudaFree(tmp);
  return st;
}

mto_status build_tables(mto_handle h) {
  for (auto* v : {&h->bc, &h->bc_qr}) {
    for (auto& b : *v) {
      int n = b.P * b.S;
      MTO_TRY(mto_alloc(h, &b.K0T, (size_t)n));
    }
  }
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    if (h->pc[p].n == 0) continue;
    QRTab& q = h->qr[p];
    q.p = p;
    MTO_TRY(mto_alloc(h, &q.R, (size_t)(p + 2) * (p + 2) * (p + 1) * (p + 1)));
    qr_table_kernel<<<1, 64, 0, h->stream>>>(p, h->hx, h->hy, q.R);
    MTO_TRY(mto_after_launch(h, "qr_table_kernel"));
  }
  return MTO_OK;
}

mto_status build_elements(mto_handle h, const double* rho, const mto_material* m, int precision) {
  TimedScope ts(h, F_BUILD);
  // the subcell tables depend only on nu (and the mesh): computed on the first build and again
  // whenever nu changes
  if (!(h->k0_nu == m->nu)) {
    for (auto* v : {&h->bc, &h->bc_qr})
      for (auto& b : *v) {
        int n = b.P * b.S;
        k0_kernel<<<(n + 127) / 128, 128, 0, h->stream>>>(b.p, b.d, m->nu, h->hx, h->hy, b.K0T);
        MTO_TRY(mto_after_launch(h, "k0_kernel"));
      }
    MTO_TRY(tc_tables(h));
    h->k0_nu = m->nu;
  }
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    PClass& c = h->pc[p];
    if (c.n == 0) continue;
    if (!c.K64) MTO_TRY(mto_alloc(h, &c.K64, (size_t)c.L * c.n));
    if (precision == MTO_MIXED && !c.K32) {
      MTO_TRY(mto_alloc(h, &c.K32, (size_t)c.L * c.n));
      MTO_TRY(mto_alloc(h, &c.K32lo, (size_t)c.L * c.n));
    }
  }
  for (auto& b : h->bc) {
    PClass& c = h->pc[b.p];
    if (h->build_path == MTO_BUILD_TENSOR && b.S <= 64) {
      MTO_TRY(tc_build_class(h, b, rho, m, precision));
      continue;
    }
    size_t smem = sizeof(double) * 32 * (b.S | 1);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(build_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    build_simt_kernel<<<(b.n + 31) / 32, 256, smem, h->stream>>>(
        b.n, b.S, b.P, b.elem, b.slot, h->design_off_d, rho, m->E0, m->Emin, m->q, b.K0T, c.L, c.dpos,
        c.K64, precision == MTO_MIXED ? c.K32 : nullptr, precision == MTO_MIXED ? c.K32lo : nullptr);
    MTO_TRY(mto_after_launch(h, "build_simt_kernel"));
  }
  return MTO_OK;
}

// springs to ground add their stiffness to the assembled diagonal (distinct DOFs, one thread each)
__global__ void spring_diag_kernel(int n, const int64_t* __restrict__ dof, const double* __restrict__ k,
                                   double* __restrict__ diag) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) diag[dof[i]] += k[i];
}

mto_status build_diagonal(mto_handle h, int precision) {
  (void)precision;
  TimedScope ts(h, F_BUILD);
  double* diag = h->diag64;
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(diag, 0, sizeof(double) * h->ndof, h->stream), "memset"));
  for (int p = 1; p <= MTO_P_MAX; ++p) {
    const PClass& c = h->pc[p];
    if (c.n == 0) continue;
    switch (p) {
      case 1: launch_diag<1>(h, c, diag); break;
      case 2: launch_diag<2>(h, c, diag); break;
      case 3: launch_diag<3>(h, c, diag); break;
      case 4: launch_diag<4>(h, c, diag); break;
      case 5: launch_diag<5>(h, c, diag); break;
      case 6: launch_diag<6>(h, c, diag); break;
    }
    MTO_TRY(mto_after_launch(h, "diag_kernel"));
  }
  if (h->n_springs) {
    spring_diag_kernel<<<1, 32, 0, h->stream>>>(h->n_springs, h->spring_dof_d, h->spring_k_d, diag);
    MTO_TRY(mto_after_launch(h, "spring_diag_kernel"));
  }
  invdiag_kernel<<<grid_for(h->ndof, 256), 256, 0, h->stream>>>(h->ndof, diag, h->invd64, h->invd32, h->flags);
  MTO_TRY(mto_after_launch(h, "invdiag_kernel"));
  if (h->n_fixed) {
    zero_fixed_kernel<<<grid_for(h->n_fixed, 256), 256, 0, h->stream>>>(h->n_fixed, h->fixed_d, h->invd64, h->invd32);
    MTO_TRY(mto_after_launch(h, "zero_fixed_kernel"));
  }
  return MTO_OK;
}

}  // namespace mto
