// The P2 density filter of Sec. 2.1 (Eqs. 4-5) at the subcell centres and its adjoint:
//   rho~_s = sum_t H_st rho_t / W_s,   H_st = R - dist(c_s, c_t) for |c_s - c_t| < R,   W_s = sum_t H_st
//   g_t    = sum_s H_st g~_s / W_s     (the chain rule of the sensitivities)
// over all subcells of the mesh (across element edges).  One warp per element, its lanes over the
// element's subcells; each lane walks the neighbouring elements within R (a bounding-box test
// skips those out of reach) and their subcells in a fixed order, so results are deterministic.
// HBM-bound: the stencil reads the design values of at most (2r+1)^2 elements per element.
#include <cmath>
#include <vector>

#include "mto_internal.cuh"

namespace mto {
namespace {

// mode 0: W_s; mode 1: rho~_s = sum_t H_st x_t / W_s (W computed on the fly); mode 2: adjoint
// g_t = sum_s H_st x_s / W_s with W read from `Wbuf`
template <int MODE>
__global__ void __launch_bounds__(128) filter_kernel(int nelx, int nely, double hx, double hy, double R, int reach,
                                                     const int* __restrict__ dmap,
                                                     const int64_t* __restrict__ off,
                                                     const double* __restrict__ x, const double* __restrict__ Wbuf,
                                                     double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nelx * nely) return;
  const int e = warp, ex = e % nelx, ey = e / nelx, d = dmap[e];
  const int64_t o = off[e];
  for (int s = lane; s < d * d; s += 32) {
    const int i = s % d, j = s / d;
    const double cx = (ex + (i + 0.5) / d) * hx, cy = (ey + (j + 0.5) / d) * hy;
    double wsum = 0.0, acc = 0.0;
    for (int ny = ey - reach; ny <= ey + reach; ++ny) {
      if (ny < 0 || ny >= nely) continue;
      // distance from the centre to the neighbour row's y-range
      const double dy0 = fmax(fmax(ny * hy - cy, cy - (ny + 1) * hy), 0.0);
      if (dy0 >= R) continue;
      for (int nx = ex - reach; nx <= ex + reach; ++nx) {
        if (nx < 0 || nx >= nelx) continue;
        const double dx0 = fmax(fmax(nx * hx - cx, cx - (nx + 1) * hx), 0.0);
        if (dx0 * dx0 + dy0 * dy0 >= R * R) continue;
        const int n = ny * nelx + nx, dn = dmap[n];
        const int64_t on = off[n];
        for (int jj = 0; jj < dn; ++jj) {
          const double ty = (ny + (jj + 0.5) / dn) * hy - cy;
          for (int ii = 0; ii < dn; ++ii) {
            const double tx = (nx + (ii + 0.5) / dn) * hx - cx;
            const double dist = sqrt(tx * tx + ty * ty);
            if (!(dist < R)) continue;
            const double w = R - dist;
            const int64_t t = on + jj * dn + ii;
            if (MODE == 0) wsum += w;
            else if (MODE == 1) {
              wsum += w;
              acc = fma(w, x[t], acc);
            } else {
              acc = fma(w, x[t] / Wbuf[t], acc);
            }
          }
        }
      }
    }
    if (MODE == 0) out[o + s] = wsum;
    else if (MODE == 1) out[o + s] = acc / wsum;
    else out[o + s] = acc;
  }
}

// Design transfer between per-element design counts: new subcell (i, j) of element e takes the
// area-weighted mean of the old subcells it overlaps (overlap lengths per axis, both layouts
// uniform over the element); an unchanged count copies the values.  One warp per element, lanes
// over its new subcells.
__global__ void __launch_bounds__(128) transfer_kernel(int nel, const int* __restrict__ d_old,
                                                       const int64_t* __restrict__ off_old,
                                                       const int* __restrict__ d_new,
                                                       const int64_t* __restrict__ off_new,
                                                       const double* __restrict__ rho_old,
                                                       double* __restrict__ rho_new) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (e >= nel) return;
  const int dn = d_new[e], dO = d_old[e];
  const double* src = rho_old + off_old[e];
  double* dst = rho_new + off_new[e];
  for (int s = lane; s < dn * dn; s += 32) {
    if (dn == dO) {
      dst[s] = src[s];
      continue;
    }
    const int i = s % dn, j = s / dn;
    const double ax0 = (double)i / dn, ax1 = (double)(i + 1) / dn;
    const double ay0 = (double)j / dn, ay1 = (double)(j + 1) / dn;
    double acc = 0.0;
    for (int l = 0; l < dO; ++l) {
      const double oy = fmax(0.0, fmin(ay1, (double)(l + 1) / dO) - fmax(ay0, (double)l / dO));
      if (oy == 0.0) continue;
      for (int k = 0; k < dO; ++k) {
        const double ox = fmax(0.0, fmin(ax1, (double)(k + 1) / dO) - fmax(ax0, (double)k / dO));
        acc += ox * oy * src[l * dO + k];
      }
    }
    dst[s] = acc * dn * dn;
  }
}

}  // namespace

mto_status transfer_design(mto_handle h, const int* d_old_host, const double* rho_old, double* rho_new) {
  const int64_t nel = h->nel;
  std::vector<int64_t> off(nel + 1, 0);
  for (int64_t e = 0; e < nel; ++e) {
    if (d_old_host[e] < 1 || d_old_host[e] > MTO_D_MAX)
      return mto_fail(h, MTO_EINVAL, "mto_transfer_design: old design count outside 1..MTO_D_MAX");
    off[e + 1] = off[e] + (int64_t)d_old_host[e] * d_old_host[e];
  }
  int* dd = nullptr;
  int64_t* od = nullptr;
  MTO_TRY(mto_cuda_check(h, cudaMalloc(&dd, nel * sizeof(int)), "cudaMalloc"));
  mto_status st = mto_cuda_check(h, cudaMalloc(&od, (nel + 1) * sizeof(int64_t)), "cudaMalloc");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(dd, d_old_host, nel * sizeof(int), cudaMemcpyHostToDevice, h->stream), "copy");
  if (st == MTO_OK)
    st = mto_cuda_check(h, cudaMemcpyAsync(od, off.data(), (nel + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream),
                        "copy");
  if (st == MTO_OK) {
    transfer_kernel<<<(int)((nel * 32 + 127) / 128), 128, 0, h->stream>>>((int)nel, dd, od, h->d_d, h->design_off_d,
                                                                        rho_old, rho_new);
    st = mto_after_launch(h, "transfer_kernel");
  }
  if (st == MTO_OK) st = mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  cudaFree(dd);
  cudaFree(od);
  return st;
}

mto_status density_filter(mto_handle h, double R, const double* x, double* out, bool adjoint) {
  TimedScope ts(h, F_BUILD);
  const int nel = (int)h->nel;
  const int blocks = (nel * 32 + 127) / 128;
  const double hmin = h->hx < h->hy ? h->hx : h->hy;
  const int reach = (int)std::ceil(R / hmin);
  if (!adjoint) {
    filter_kernel<1><<<blocks, 128, 0, h->stream>>>(h->nelx, h->nely, h->hx, h->hy, R, reach, h->d_d, h->design_off_d,
                                                    x, nullptr, out);
    return mto_after_launch(h, "filter_kernel");
  }
  if (!h->filt_W) MTO_TRY(mto_alloc(h, &h->filt_W, (size_t)h->design_len));
  filter_kernel<0><<<blocks, 128, 0, h->stream>>>(h->nelx, h->nely, h->hx, h->hy, R, reach, h->d_d, h->design_off_d,
                                                  nullptr, nullptr, h->filt_W);
  MTO_TRY(mto_after_launch(h, "filter_kernel"));
  filter_kernel<2><<<blocks, 128, 0, h->stream>>>(h->nelx, h->nely, h->hx, h->hy, R, reach, h->d_d, h->design_off_d,
                                                  x, h->filt_W, out);
  return mto_after_launch(h, "filter_kernel");
}

}  // namespace mto
