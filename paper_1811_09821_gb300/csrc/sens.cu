// Step (c): compliance C = f^T u (Eq. 1 with z = f) and the design sensitivities
// dC/drho_s = -E'(rho_s) w_s,  w_s = u_e^T K0_s u_e = integral over subcell s of eps^T D0 eps,
// E'(rho) = q rho^(q-1) (E0 - Emin).  The compliance problem is self-adjoint (adjoint = -u), so u
// is the only field needed; it is re-gathered per element from the stored global vector.
//
// Kernel: one warp per element.  The element's displacement is gathered in FP64 and its best-fit
// rigid motion (translation and rotation, which K0_s annihilates) is removed in FP64.  Strains at
// the (p+1) x (p+1) Gauss points of every subcell come from a sum-factorised tensor evaluation on
// the element's d(p+1) x d(p+1) point grid; each point adds eps^T D0 eps (a sum of non-negative
// terms) to its subcell.  Compute type T is double (MTO_FP64) or float (MTO_MIXED).
#include <cmath>

#include "mto_internal.cuh"

namespace mto {

// 1D tables of a (p, d) class: [L: N1 x G][D: N1 x G][W: G][Z: N1] with G = d (p+1) points
// xi_g = -1 + (2 i + 1 + x_k)/d (subcell i, Gauss node x_k), L = l_a(xi_g), D = l_a'(xi_g) and
// W = w_k / d (the 1D subcell Jacobian).
__global__ void sens_table_kernel(int p, int d, double* __restrict__ tab, float* __restrict__ tabf) {
  const int n1 = p + 1, G = d * n1;
  double z[kPMaxTab + 1], gx[kPMaxTab + 1], gw[kPMaxTab + 1];
  gll_nodes(p, z);
  gauss_rule(n1, gx, gw);
  const int tot = 2 * n1 * G + G + n1;
  for (int k = threadIdx.x; k < tot; k += blockDim.x) {
    double v;
    if (k < 2 * n1 * G) {
      int which = k / (n1 * G), r = k % (n1 * G), a = r / G, g = r % G;
      int i = g / n1, kk = g % n1;
      double xi = -1.0 + (2.0 * i + 1.0 + gx[kk]) / d;
      v = which == 0 ? lagrange_val(z, n1, a, xi) : lagrange_der(z, n1, a, xi);
    } else if (k < 2 * n1 * G + G) {
      int g = k - 2 * n1 * G;
      v = gw[g % n1] / d;
    } else {
      v = z[k - 2 * n1 * G - G];
    }
    tab[k] = v;
    tabf[k] = (float)v;
  }
}

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// NF = 1: w_s = u_e^T K0_s u_e (compliance, self-adjoint).  NF = 2: w_s = v_e^T K0_s u_e with the
// adjoint field v (a general objective z^T u, Eq. 1): both fields' strains at every point, the
// bilinear energy density eps(v)^T D0 eps(u).
template <int PO, int NF, typename T>
__global__ void __launch_bounds__(128) sens_kernel(
    int n, int d, const int* __restrict__ elem, const int* __restrict__ slot, int ld, const int* __restrict__ gmap,
    const Constraint* __restrict__ cons, const double* __restrict__ u, const double* __restrict__ v,
    const double* __restrict__ rho, const int64_t* __restrict__ design_off, double E0, double Emin, double q,
    double nu, double hx, double hy, const T* __restrict__ tab, const double* __restrict__ Z, double* __restrict__ dc,
    double* __restrict__ eout) {
  constexpr int N1 = PO + 1, NN = N1 * N1;
  static_assert(NN <= 64, "two nodes per lane at most");
  const int G = d * N1;
  extern __shared__ unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per-warp shared layout: A[NF][4][N1][G] (T), part[G] (T), U[NF][2][NN] (T)
  const size_t per_warp = (size_t)(4 * NF * N1 * G + G + 2 * NF * NN) * sizeof(T);
  T* A = reinterpret_cast<T*>(smem_raw + warp * per_warp);
  T* part = A + 4 * NF * N1 * G;
  T* U = part + G;
  const int k = blockIdx.x * (blockDim.x >> 5) + warp;
  if (k >= n) return;
  const int e = elem[k], sl = slot[k];
  const T* L = tab;
  const T* Dd = tab + N1 * G;
  const T* W = tab + 2 * N1 * G;

  // gather each field (FP64) and remove its best-fit rigid motion in FP64 (lanes stride over nodes)
#pragma unroll
  for (int fld = 0; fld < NF; ++fld) {
    const double* x = fld == 0 ? u : v;
    double sux = 0.0, suy = 0.0, snum = 0.0, sden = 0.0;
    double ux[2], uy[2], xl[2], yl[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int ln = lane + 32 * r;
      ux[r] = uy[r] = xl[r] = yl[r] = 0.0;
      if (ln < NN) {
        int g = gmap[(size_t)sl * NN + ln];
        if (g >= 0) {
          ux[r] = x[2 * (size_t)g];
          uy[r] = x[2 * (size_t)g + 1];
        } else {
          const Constraint& c = cons[-g - 1];
          for (int j = 0; j < c.cnt; ++j) {
            ux[r] += c.w[j] * x[2 * (size_t)c.node[j]];
            uy[r] += c.w[j] * x[2 * (size_t)c.node[j] + 1];
          }
        }
        xl[r] = 0.5 * Z[ln % N1] * hx;   // node coordinates about the element centre (FP64 GLL nodes)
        yl[r] = 0.5 * Z[ln / N1] * hy;
        sux += ux[r];
        suy += uy[r];
        snum += xl[r] * uy[r] - yl[r] * ux[r];
        sden += xl[r] * xl[r] + yl[r] * yl[r];
      }
    }
    const double tx = wsum(sux) / NN, ty = wsum(suy) / NN;
    const double om = wsum(snum) / wsum(sden);
    T* Uf = U + 2 * NN * fld;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int ln = lane + 32 * r;
      if (ln < NN) {
        Uf[ln] = (T)(ux[r] - tx + om * yl[r]);
        Uf[NN + ln] = (T)(uy[r] - ty - om * xl[r]);
      }
    }
  }
  __syncwarp();

  // stage 1 (x direction): A_c[b][g] = sum_a U_c[b][a] L[a][g],  Ad_c[b][g] = sum_a U_c[b][a] D[a][g]
  for (int g = lane; g < G; g += 32) {
#pragma unroll
    for (int fld = 0; fld < NF; ++fld) {
      const T* Uf = U + 2 * NN * fld;
      T* Af = A + 4 * N1 * G * fld;
#pragma unroll
      for (int b = 0; b < N1; ++b) {
        T a0 = 0, a1 = 0, d0 = 0, d1 = 0;
#pragma unroll
        for (int a = 0; a < N1; ++a) {
          T l = L[a * G + g], dl = Dd[a * G + g];
          T v0 = Uf[b * N1 + a], v1 = Uf[NN + b * N1 + a];
          a0 = fma(v0, l, a0);
          d0 = fma(v0, dl, d0);
          a1 = fma(v1, l, a1);
          d1 = fma(v1, dl, d1);
        }
        Af[(0 * N1 + b) * G + g] = a0;
        Af[(1 * N1 + b) * G + g] = d0;
        Af[(2 * N1 + b) * G + g] = a1;
        Af[(3 * N1 + b) * G + g] = d1;
      }
    }
  }
  __syncwarp();

  // stage 2 (y direction) and the energy density at every point
  const T sx = (T)(2.0 / hx), sy = (T)(2.0 / hy), jac = (T)(0.25 * hx * hy);
  const double f = 1.0 / (1.0 - nu * nu);
  const T D11 = (T)f, D12 = (T)(f * nu), D33 = (T)(f * 0.5 * (1.0 - nu));
  const double dE = E0 - Emin;
  const int64_t off = design_off[e];
  double energy = 0.0;   // sum_s E(rho_s) w_s of this element (eout)
  for (int j = 0; j < d; ++j) {
    for (int g = lane; g < G; g += 32) {
      T acc = 0;
      for (int kk = 0; kk < N1; ++kk) {
        const int gy = j * N1 + kk;
        T exx[NF], eyy[NF], gam[NF];
#pragma unroll
        for (int fld = 0; fld < NF; ++fld) {
          const T* Af = A + 4 * N1 * G * fld;
          T ex = 0, ey = 0, g0 = 0, g1 = 0;
#pragma unroll
          for (int b = 0; b < N1; ++b) {
            T lb = L[b * G + gy], db = Dd[b * G + gy];
            ex = fma(Af[(1 * N1 + b) * G + g], lb, ex);   // d ux / d xi
            g0 = fma(Af[(0 * N1 + b) * G + g], db, g0);   // d ux / d eta
            g1 = fma(Af[(3 * N1 + b) * G + g], lb, g1);   // d uy / d xi
            ey = fma(Af[(2 * N1 + b) * G + g], db, ey);   // d uy / d eta
          }
          exx[fld] = ex * sx;
          eyy[fld] = ey * sy;
          gam[fld] = g0 * sy + g1 * sx;
        }
        constexpr int o = NF - 1;   // the second field of the bilinear form (the first for NF = 1)
        T en = D11 * (exx[0] * exx[o] + eyy[0] * eyy[o]) + D12 * (exx[0] * eyy[o] + eyy[0] * exx[o]) +
               D33 * gam[0] * gam[o];
        acc = fma(W[gy], en, acc);
      }
      part[g] = acc * W[g] * jac;
    }
    __syncwarp();
    for (int i = lane; i < d; i += 32) {
      T w = 0;
      for (int kk = 0; kk < N1; ++kk) w += part[i * N1 + kk];
      const int s = j * d + i;
      const double r = rho[off + s];
      if (dc) dc[off + s] = -q * pow(r, q - 1.0) * dE * (double)w;
      if (eout) energy += (Emin + pow(r, q) * dE) * (double)w;
    }
    __syncwarp();
  }
  if (eout) {
    energy = wsum(energy);
    if (lane == 0) eout[e] = energy;
  }
}

template <int PO, int NF, typename T>
mto_status launch_sens(mto_handle h, const BClass& b, const double* u, const double* v, const double* rho,
                       const mto_material* m, const T* tab, double* dc, double* eout) {
  const int N1 = PO + 1, G = b.d * N1;
  const size_t per_warp = (size_t)(4 * NF * N1 * G + G + 2 * NF * N1 * N1) * sizeof(T);
  const int warps = 4;
  const size_t smem = per_warp * warps;
  if (smem > 227 * 1024) return mto_fail(h, MTO_EINVAL, "sensitivity: element class too large for shared memory");
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(sens_kernel<PO, NF, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const PClass& c = h->pc[b.p];
  sens_kernel<PO, NF, T><<<(b.n + warps - 1) / warps, 32 * warps, smem, h->stream>>>(
      b.n, b.d, b.elem, b.slot, c.ld, c.gmap, h->cons_d, u, v, rho, h->design_off_d, m->E0, m->Emin, m->q, m->nu,
      h->hx, h->hy, tab, b.stab + 2 * N1 * G + G, dc, eout);
  return mto_after_launch(h, "sens_kernel");
}

template <int NF, typename T>
mto_status sens_all(mto_handle h, const double* u, const double* v, const double* rho, const mto_material* m,
                    double* dc, double* eout = nullptr) {
  for (auto& b : h->bc) {
    const T* tab;
    if constexpr (sizeof(T) == 8) tab = (const T*)b.stab; else tab = (const T*)b.stabf;
    switch (b.p) {
      case 1: MTO_TRY((launch_sens<1, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
      case 2: MTO_TRY((launch_sens<2, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
      case 3: MTO_TRY((launch_sens<3, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
      case 4: MTO_TRY((launch_sens<4, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
      case 5: MTO_TRY((launch_sens<5, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
      case 6: MTO_TRY((launch_sens<6, NF, T>(h, b, u, v, rho, m, tab, dc, eout))); break;
    }
  }
  return MTO_OK;
}

}  // namespace

mto_status build_sens_tables(mto_handle h) {
  for (auto& b : h->bc) {
    const int n1 = b.p + 1, G = b.d * n1, tot = 2 * n1 * G + G + n1;
    MTO_TRY(mto_alloc(h, &b.stab, (size_t)tot));
    MTO_TRY(mto_alloc(h, &b.stabf, (size_t)tot));
    sens_table_kernel<<<1, 256, 0, h->stream>>>(b.p, b.d, b.stab, b.stabf);
    MTO_TRY(mto_after_launch(h, "sens_table_kernel"));
  }
  return MTO_OK;
}

mto_status sensitivity(mto_handle h, const double* u, const double* f, const double* rho, const mto_material* m,
                       int precision, double* dc, double* C) {
  {
  TimedScope ts(h, F_SENS);
  if (precision == MTO_FP64) MTO_TRY((sens_all<1, double>(h, u, nullptr, rho, m, dc)));
  else MTO_TRY((sens_all<1, float>(h, u, nullptr, rho, m, dc)));
  MTO_TRY(dot64(h, f, u, h->ndof, h->red + 8));
  }
  if (C) {
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned + 8, h->red + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy"));
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    *C = h->host_pinned[8];
  }
  return MTO_OK;
}

// dJ/drho_s = -E'(rho_s) v_e^T K0_s u_e for an objective J = z^T u with the adjoint field v
// solving K v = z (Eq. 1; v = u for compliance).  FP64 quadrature.
mto_status sensitivity_adjoint(mto_handle h, const double* u, const double* v, const double* rho,
                               const mto_material* m, double* dc) {
  TimedScope ts(h, F_SENS);
  return sens_all<2, double>(h, u, v, rho, m, dc);
}

// Compliance of an approximate displacement in its energy form, C(u) = 2 f^T u - u^T K u
// (= C* - ||u* - u||_K^2 for the exact u*, so its error is second order in the displacement's):
// u^T K u as the sum of the element energies sum_s E(rho_s) u_e^T K0_s u_e, each after the FP64
// removal of the element's rigid motion (free of the cancellation of a global u^T (K u)), summed
// over the elements in a fixed order.
mto_status compliance_energy(mto_handle h, const double* u, const double* f, const double* rho,
                             const mto_material* m, double* C) {
  {
    TimedScope ts(h, F_SENS);
    MTO_TRY((sens_all<1, double>(h, u, nullptr, rho, m, nullptr, h->dbuf)));
    MTO_TRY(sum64(h, h->dbuf, h->nel, h->red + 10));
    MTO_TRY(dot64(h, f, u, h->ndof, h->red + 11));
  }
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned + 10, h->red + 10, 2 * sizeof(double),
                                            cudaMemcpyDeviceToHost, h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  *C = 2.0 * h->host_pinned[11] - h->host_pinned[10];
  return MTO_OK;
}

}  // namespace mto
