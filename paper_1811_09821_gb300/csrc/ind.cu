// Step (d): the composite refinement indicator and the dp map update (Sec. 3.2, 3.3), and the
// optimality-criteria design update.  All FP64: the integer maps must match the oracle exactly,
// so every floating-point decision is taken in double with a fixed reduction order.
#include <cmath>
#include <vector>

#include "mto_internal.cuh"

namespace mto {
namespace {

// Basis constants shared by the indicator kernels: GLL nodes of orders 1..kPMaxTab and Gauss
// rules of 1..kPMaxTab+2 points, filled once per handle by basis_table_kernel.
struct BasisTab {
  double gll[kPMaxTab + 1][kPMaxTab + 1];
  double gx[kPMaxTab + 3][kPMaxTab + 3];
  double gw[kPMaxTab + 3][kPMaxTab + 3];
};

__global__ void basis_table_kernel(BasisTab* t) {
  int p = threadIdx.x;
  if (p >= 1 && p <= kPMaxTab) gll_nodes(p, t->gll[p]);
  if (p >= 1 && p <= kPMaxTab + 2) gauss_rule(p, t->gx[p], t->gw[p]);
}

// Local displacement of element e (order p): 2 (p+1)^2 values, minimum-rule constraints applied.
// both components of local node ln of the element in slot `slot` (through its constraint if hanging)
__device__ __forceinline__ void gather_node(int nn, int slot, int ln, const int* __restrict__ gmap,
                                            const Constraint* __restrict__ cons, const double* __restrict__ u,
                                            double* ue) {
  int g = gmap[(size_t)slot * nn + ln];
  double a = 0.0, b = 0.0;
  if (g >= 0) {
    a = u[2 * (size_t)g];
    b = u[2 * (size_t)g + 1];
  } else {
    const Constraint& c = cons[-g - 1];
    for (int k = 0; k < c.cnt; ++k) {
      a += c.w[k] * u[2 * (size_t)c.node[k]];
      b += c.w[k] * u[2 * (size_t)c.node[k] + 1];
    }
  }
  ue[2 * ln] = a;
  ue[2 * ln + 1] = b;
}

__device__ void gather_element(int p, int slot, const int* __restrict__ gmap, const Constraint* __restrict__ cons,
                               const double* __restrict__ u, double* ue) {
  const int nn = (p + 1) * (p + 1);
  for (int ln = 0; ln < nn; ++ln) gather_node(nn, slot, ln, gmap, cons, u, ue);
}

__device__ __forceinline__ double warp_sum_all(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct ClassPtrs {
  const int* gmap[kPMaxTab + 1];
};

// ------------------------------------------------------------------------------------ Kelly
// Normal derivative (along +x for sides 0/1, +y for sides 2/3) of both components of an order-p
// field at edge parameter t: side 0 x = 0, 1 x = hx, 2 y = 0, 3 y = hy.
__device__ void edge_normal_derivative(const BasisTab* B, int p, int side, const double* ue, double t, double hx,
                                       double hy, double* dx, double* dy) {
  const double* z = B->gll[p];
  const int n1 = p + 1;
  double sx = 0.0, sy = 0.0;
  const double xi = side == 0 ? -1.0 : side == 1 ? 1.0 : t;
  const double eta = side == 2 ? -1.0 : side == 3 ? 1.0 : t;
  for (int b = 0; b < n1; ++b)
    for (int a = 0; a < n1; ++a) {
      double w = side <= 1 ? lagrange_der(z, n1, a, xi) * lagrange_val(z, n1, b, eta) * (2.0 / hx)
                           : lagrange_val(z, n1, a, xi) * lagrange_der(z, n1, b, eta) * (2.0 / hy);
      sx += w * ue[2 * (b * n1 + a)];
      sy += w * ue[2 * (b * n1 + a) + 1];
    }
  *dx = sx;
  *dy = sy;
}

// Edge term c_F * integral_F [du/dn]^2 ds (Eq. 9) for every interior edge: horizontal edges
// first (id iy*nelx + ix, between elements below and above), then vertical edges.
__global__ void kelly_edge_kernel(int nelx, int nely, const int* __restrict__ p_of, const int* __restrict__ slot_of,
                                  ClassPtrs cp, const Constraint* __restrict__ cons, const double* __restrict__ u,
                                  const BasisTab* __restrict__ B, double hx, double hy, double* __restrict__ edge_val) {
  const int64_t nH = (int64_t)(nely + 1) * nelx, nV = (int64_t)nely * (nelx + 1);
  const double hF = sqrt(hx * hx + hy * hy);
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < nH + nV; id += (int64_t)gridDim.x * blockDim.x) {
    int eA, eB, sideA, sideB;
    double len;
    if (id < nH) {
      int iy = (int)(id / nelx), ix = (int)(id % nelx);
      if (iy == 0 || iy == nely) { edge_val[id] = 0.0; continue; }
      eA = (iy - 1) * nelx + ix; eB = iy * nelx + ix; sideA = 3; sideB = 2; len = hx;
    } else {
      int64_t v = id - nH;
      int iy = (int)(v / (nelx + 1)), ix = (int)(v % (nelx + 1));
      if (ix == 0 || ix == nelx) { edge_val[id] = 0.0; continue; }
      eA = iy * nelx + ix - 1; eB = iy * nelx + ix; sideA = 1; sideB = 0; len = hy;
    }
    const int pA = p_of[eA], pB = p_of[eB];
    double uA[2 * (kPMaxTab) * (kPMaxTab)], uB[2 * (kPMaxTab) * (kPMaxTab)];
    gather_element(pA, slot_of[eA], cp.gmap[pA], cons, u, uA);
    gather_element(pB, slot_of[eB], cp.gmap[pB], cons, u, uB);
    const int pF = pA > pB ? pA : pB;
    const int nq = pF + 1;
    double val = 0.0;
    for (int g = 0; g < nq; ++g) {
      double ax, ay, bx, by;
      edge_normal_derivative(B, pA, sideA, uA, B->gx[nq][g], hx, hy, &ax, &ay);
      edge_normal_derivative(B, pB, sideB, uB, B->gx[nq][g], hx, hy, &bx, &by);
      double jx = ax - bx, jy = ay - by;
      val += B->gw[nq][g] * (jx * jx + jy * jy) * 0.5 * len;
    }
    edge_val[id] = hF / (2.0 * pF) * val;
  }
}

// Gamma^a_e = sum of its four edge terms in the fixed order left, right, bottom, top.
__global__ void kelly_sum_kernel(int nelx, int nely, const double* __restrict__ edge_val, double* __restrict__ ga) {
  const int64_t nH = (int64_t)(nely + 1) * nelx, nel = (int64_t)nelx * nely;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    int ix = (int)(e % nelx), iy = (int)(e / nelx);
    double s = edge_val[nH + (int64_t)iy * (nelx + 1) + ix];
    s += edge_val[nH + (int64_t)iy * (nelx + 1) + ix + 1];
    s += edge_val[(int64_t)iy * nelx + ix];
    s += edge_val[(int64_t)(iy + 1) * nelx + ix];
    ga[e] = s;
  }
}

// ------------------------------------------------------------------------------------ Gamma^d
__global__ void minmax_kernel(int64_t n, const double* __restrict__ rho, unsigned long long* __restrict__ mm) {
  unsigned long long lo = ~0ULL, hi = 0ULL;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long k = order_key(rho[i]);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  atomicMin(&mm[0], lo);
  atomicMax(&mm[1], hi);
}

__device__ double key_to_double(unsigned long long k) {
  unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
  double v;
  memcpy(&v, &u, 8);
  return v;
}

// Density indicator (Sec. 3.2.2): per element, the cells' band contributions in cell order.
__global__ void gamma_d_kernel(int64_t nel, const int64_t* __restrict__ off, const double* __restrict__ rho,
                               const unsigned long long* __restrict__ mm, int cycle, double alpha, double beta,
                               double* __restrict__ gd) {
  const double rmin = key_to_double(mm[0]), rmax = key_to_double(mm[1]);
  const double ravg = 0.5 * (rmax + rmin);
  const double fac = ravg * exp(-beta * (cycle - 1));
  const double rl = rmin + (1.0 - alpha) * fac, ru = rmax - (1.0 - alpha) * fac;
  const double cl = rmin + alpha * fac, cu = rmax - alpha * fac;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = off[e], b = off[e + 1];
    const double n = (double)(b - a);
    double g = 0.0;
    for (int64_t j = a; j < b; ++j) {
      const double r = rho[j];
      if (rl <= r && r <= ravg) g += (r - rl) / n;
      else if (ravg < r && r <= ru) g += (ru - r) / n;
      else if (r <= cl) g -= (cl - r) / n;
      else if (r >= cu) g -= (r - cu) / n;
    }
    gd[e] = g;
  }
}

// ------------------------------------------------------------------------------------ QR error
// One warp per element of a (p, d) class (Eq. 14).  Shared layout (doubles): A[P1] (the order p+1
// matrix, lower triangle packed by rows, A_ij at i (i + 1) / 2 + j, factorised in place as
// L D L^T), f[n0], f1[n1], u1[n1], E[S], ue[n0], rd[n1] (reciprocal pivots), cl[n1] (the pivot
// column before scaling), pr[3 n1] (the pinned rows of the unmodified matrix), with
// n0 = 2 (p+1)^2, n1 = 2 (p+2)^2, P1 = n1 (n1 + 1) / 2.  The footprint sets how many elements an
// SM works on at once, and the kernel is bound by GB300's FP64 pipes, so it keeps one triangle.
// eps is invariant to rigid motions of u^(p), which are removed first (FP64) so that the element
// energies carry no cancellation.
__global__ void __launch_bounds__(32) qr_kernel(int p, int d, int n, const int* __restrict__ elem,
                                                const int* __restrict__ slot, int L, const int2* __restrict__ dpos,
                                                const int* __restrict__ gmap,
                                                const Constraint* __restrict__ cons, const double* __restrict__ K64,
                                                const float* __restrict__ Kh, const float* __restrict__ Kl,
                                                const double* __restrict__ K0T1, const double* __restrict__ R,
                                                const double* __restrict__ u, const double* __restrict__ rho,
                                                const int64_t* __restrict__ off, double E0, double Emin, double q,
                                                const BasisTab* __restrict__ B, double hx, double hy,
                                                double* __restrict__ eps) {
  extern __shared__ double sh[];
  const int lane = threadIdx.x;
  const int k = blockIdx.x;
  if (k >= n) return;
  const int e = elem[k], sl = slot[k];
  const int n1d = p + 1;
  const int na = (p + 1) * (p + 1), nb = (p + 2) * (p + 2);
  const int n0 = 2 * na, n1 = 2 * nb, S = d * d;
  const int P1 = packed_size(n1);
  double* A = sh;
  double* f = A + P1;
  double* f1 = f + n0;
  double* u1 = f1 + n1;
  double* E = u1 + n1;
  double* ue = E + S;
  double* rd = ue + n0;
  double* cl = rd + n1;
  double* pr = cl + n1;
  // gather u_e (lanes over nodes), then remove its least-squares rigid motion about the element
  // centre (translations and rotation; node sums over the warp)
  for (int ln = lane; ln < na; ln += 32) gather_node(na, sl, ln, gmap, cons, u, ue);
  __syncwarp();
  {
    const double* z = B->gll[p];
    double tx = 0.0, ty = 0.0, num = 0.0, den = 0.0;
    for (int ln = lane; ln < na; ln += 32) {
      const double x = 0.5 * hx * z[ln % n1d], y = 0.5 * hy * z[ln / n1d];
      tx += ue[2 * ln];
      ty += ue[2 * ln + 1];
      num += x * ue[2 * ln + 1] - y * ue[2 * ln];
      den += x * x + y * y;
    }
    tx = warp_sum_all(tx) / na;
    ty = warp_sum_all(ty) / na;
    const double om = warp_sum_all(num) / warp_sum_all(den);
    for (int ln = lane; ln < na; ln += 32) {
      const double x = 0.5 * hx * z[ln % n1d], y = 0.5 * hy * z[ln / n1d];
      ue[2 * ln] = ue[2 * ln] - tx + om * y;
      ue[2 * ln + 1] = ue[2 * ln + 1] - ty - om * x;
    }
  }
  for (int s = lane; s < S; s += 32) {
    double r = rho[off[e] + s];
    E[s] = Emin + pow(r, q) * (E0 - Emin);
  }
  __syncwarp();
  // f = K_e u_e (order p, FP64 element matrix of the build) and J^(p) = u^T f / 2
  double jp = 0.0;
  for (int i = lane; i < n0; i += 32) {
    double s = 0.0;
    for (int j = 0; j < n0; ++j) {
      int a = i < j ? i : j, b = i < j ? j : i;
      s += k_entry(K64, Kh, Kl, L, sl, dpos[packed_index(n0, a, b)].x) * ue[j];
    }
    f[i] = s;
    jp += ue[i] * s;
  }
  for (int o = 16; o > 0; o >>= 1) jp += __shfl_xor_sync(0xffffffffu, jp, o);
  jp *= 0.5;
  __syncwarp();
  // f1 = R f per component
  for (int i = lane; i < n1; i += 32) {
    const int jn = i >> 1, c = i & 1;
    double s = 0.0;
    for (int kk = 0; kk < na; ++kk) s += R[jn * na + kk] * f[2 * kk + c];
    f1[i] = s;
  }
  // K^(p+1) = sum_s E_s K0_s^(p+1) (table rows by upper packed index (i <= j)) into the lower triangle
  for (int c = lane; c < P1; c += 32) {
    double s = 0.0;
    const double* kc = K0T1 + (size_t)c * S;
    for (int t = 0; t < S; ++t) s = fma(E[t], kc[t], s);
    int i = 0, rem = c;
    while (rem >= n1 - i) { rem -= n1 - i; ++i; }
    const int j = i + rem;
    A[j * (j + 1) / 2 + i] = s;
  }
  __syncwarp();
  // pinned DOFs of the (p+1) element: u_x, u_y at the bottom-left vertex, u_y at the bottom-right
  // vertex; their values are those of u^(p) at the same vertices
  const int fx[3] = {0, 1, 2 * (p + 1) + 1};
  const double v[3] = {ue[0], ue[1], ue[2 * p + 1]};
  auto at = [&](int a, int b) -> double { return a >= b ? A[a * (a + 1) / 2 + b] : A[b * (b + 1) / 2 + a]; };
  // the pinned rows before the modification (for J^(p+1)), and the right-hand side on free DOFs
  for (int i = lane; i < n1; i += 32) {
    const double k0 = at(i, fx[0]), k1 = at(i, fx[1]), k2 = at(i, fx[2]);
    pr[i] = k0;
    pr[n1 + i] = k1;
    pr[2 * n1 + i] = k2;
    double r = f1[i] - k0 * v[0] - k1 * v[1] - k2 * v[2];
    for (int k = 0; k < 3; ++k)
      if (i == fx[k]) r = v[k];
    u1[i] = r;
  }
  __syncwarp();
  // identity rows and columns on the pinned DOFs
  for (int c = lane; c < P1; c += 32) {
    int i = (int)((sqrtf(8.0f * (float)c + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > c) --i;
    while ((i + 1) * (i + 2) / 2 <= c) ++i;
    const int j = c - i * (i + 1) / 2;
    const bool pin = i == fx[0] || i == fx[1] || i == fx[2] || j == fx[0] || j == fx[1] || j == fx[2];
    if (pin) A[c] = (i == j) ? 1.0 : 0.0;
  }
  __syncwarp();
  // A = L D L^T (right-looking).  Column c: the pivot's reciprocal into rd[c], the column kept
  // unscaled in cl and scaled into L; the trailing update A_ij -= L_ic cl_j (c < j <= i) runs over
  // the m (m + 1) / 2 pairs of the trailing block spread evenly over the lanes: pair
  // t = s (s + 1) / 2 + r (0 <= r <= s < m) is row n1 - 1 - r, column n1 - 1 - s.
  for (int c = 0; c < n1; ++c) {
    const double inv = 1.0 / A[c * (c + 1) / 2 + c];
    for (int i = c + 1 + lane; i < n1; i += 32) {
      const double a = A[i * (i + 1) / 2 + c];
      cl[i] = a;
      A[i * (i + 1) / 2 + c] = a * inv;
    }
    if (lane == 0) rd[c] = inv;
    __syncwarp();
    const int m = n1 - 1 - c;
    const int T = m * (m + 1) / 2;
    for (int t = lane; t < T; t += 32) {
      int s = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while (s * (s + 1) / 2 > t) --s;
      while ((s + 1) * (s + 2) / 2 <= t) ++s;
      const int r = t - s * (s + 1) / 2;
      const int i = n1 - 1 - r, j = n1 - 1 - s;
      A[i * (i + 1) / 2 + j] -= A[i * (i + 1) / 2 + c] * cl[j];
    }
    __syncwarp();
  }
  // L y = b, y <- D^-1 y, L^T x = y, column by column (each solved entry updates the rest over the
  // lanes)
  for (int j = 0; j < n1; ++j) {
    const double yj = u1[j];
    for (int i = j + 1 + lane; i < n1; i += 32) u1[i] -= A[i * (i + 1) / 2 + j] * yj;
    __syncwarp();
  }
  for (int i = lane; i < n1; i += 32) u1[i] *= rd[i];
  __syncwarp();
  for (int j = n1 - 1; j >= 0; --j) {
    const double xj = u1[j];
    for (int i = lane; i < j; i += 32) u1[i] -= A[j * (j + 1) / 2 + i] * xj;
    __syncwarp();
  }
  // J^(p+1) = u1^T K u1 / 2 = (u1_f^T f1_f + v^T (K u1)_pinned) / 2: on the free rows K u1 is the
  // right-hand side f1, on the pinned rows the saved rows of the unmodified matrix give it
  double j1 = 0.0;
  for (int i = lane; i < n1; i += 32) {
    const bool pin = i == fx[0] || i == fx[1] || i == fx[2];
    if (!pin) j1 += u1[i] * f1[i];
    j1 += u1[i] * (v[0] * pr[i] + v[1] * pr[n1 + i] + v[2] * pr[2 * n1 + i]);
  }
  for (int o = 16; o > 0; o >>= 1) j1 += __shfl_xor_sync(0xffffffffu, j1, o);
  j1 *= 0.5;
  if (lane == 0) eps[e] = j1 == 0.0 ? 0.0 : 1.0 - jp / j1;
}

// ------------------------------------------------------------------------------------ selection
// k-th smallest (0-based) composite key (order_key(v_i), i) among the items with part(i), found
// by radix selection over the 64-bit key (8 passes of 8 bits) and then the index among equal keys.
// State in sel[]: [0] prefix, [1] rank remaining, [2] result key, [3] result index, [4] valid.
__device__ __forceinline__ bool participates(int mode, double v) {
  return mode == 0 ? true : mode == 1 ? (v < 0.0) : (v > 0.0);
}

__global__ void sel_init_kernel(unsigned long long* sel, const long long* krank) {
  sel[0] = 0ULL;
  sel[1] = (unsigned long long)(*krank);
  sel[4] = 0ULL;
}

__global__ void sel_hist_kernel(int64_t n, const double* __restrict__ v, int mode, int shift,
                                const unsigned long long* __restrict__ sel, unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const unsigned long long prefix = sel[0];
  const unsigned long long himask = shift >= 56 ? 0ULL : (~0ULL << (shift + 8));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = v[i];
    if (!participates(mode, x)) continue;
    unsigned long long key = order_key(x);
    if ((key & himask) != (prefix & himask)) continue;
    atomicAdd(&h[(key >> shift) & 255ULL], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void sel_pick_kernel(int shift, unsigned long long* sel, unsigned int* hist) {
  if (threadIdx.x != 0) return;
  unsigned long long r = sel[1];
  unsigned long long acc = 0;
  int b = 0;
  for (; b < 256; ++b) {
    if (r < acc + hist[b]) break;
    acc += hist[b];
  }
  if (b == 256) b = 255;  // rank beyond the count: cannot happen for a valid rank
  sel[1] = r - acc;
  sel[0] |= (unsigned long long)b << shift;
  for (int i = 0; i < 256; ++i) hist[i] = 0;
}

// count of matching items (key == sel[0]) per chunk of 1024 consecutive indices
__global__ void sel_count_kernel(int64_t n, const double* __restrict__ v, int mode,
                                 const unsigned long long* __restrict__ sel, unsigned int* __restrict__ cnt) {
  const unsigned long long key = sel[0];
  const int64_t chunk = blockIdx.x;
  unsigned int c = 0;
  for (int64_t i = chunk * 1024 + threadIdx.x; i < n && i < (chunk + 1) * 1024; i += blockDim.x) {
    double x = v[i];
    if (participates(mode, x) && order_key(x) == key) ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    cnt[chunk] = s;
  }
}

__global__ void sel_index_kernel(int64_t n, const double* __restrict__ v, int mode, unsigned long long* sel,
                                 const unsigned int* __restrict__ cnt, int64_t nchunks) {
  if (threadIdx.x != 0) return;
  unsigned long long r = sel[1];
  const unsigned long long key = sel[0];
  int64_t c = 0;
  for (; c < nchunks; ++c) {
    if (r < cnt[c]) break;
    r -= cnt[c];
  }
  int64_t idx = -1;
  if (c < nchunks) {
    for (int64_t i = c * 1024; i < n && i < (c + 1) * 1024; ++i) {
      double x = v[i];
      if (participates(mode, x) && order_key(x) == key) {
        if (r == 0) { idx = i; break; }
        --r;
      }
    }
  }
  sel[2] = key;
  sel[3] = (unsigned long long)idx;
  sel[4] = idx >= 0 ? 1ULL : 0ULL;
}

__device__ __forceinline__ bool comp_less(double v, int64_t i, unsigned long long key, unsigned long long idx) {
  unsigned long long k = order_key(v);
  return k < key || (k == key && (unsigned long long)i < idx);
}

__global__ void count_sign_kernel(int64_t n, const double* __restrict__ v, unsigned long long* __restrict__ out) {
  unsigned long long neg = 0, pos = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    neg += v[i] < 0.0;
    pos += v[i] > 0.0;
  }
  atomicAdd(&out[0], neg);
  atomicAdd(&out[1], pos);
}

// Analysis (step 2), density (step 3c) and the flags.  thr: [0..3] analysis coarsen threshold
// (key, idx) and whether it applies, analysis refine threshold; [..] density thresholds.
struct Thresholds {
  unsigned long long ac_key, ac_idx, ar_key, ar_idx, dc_key, dc_idx, dr_key, dr_idx;
  int ac_mode, ar_mode, dc_mode, dr_mode;   // 0 none, 1 all, 2 threshold
};

__device__ __forceinline__ bool in_low(int mode, double v, int64_t i, unsigned long long k, unsigned long long x) {
  return mode == 1 || (mode == 2 && comp_less(v, i, k, x));
}
__device__ __forceinline__ bool in_high(int mode, double v, int64_t i, unsigned long long k, unsigned long long x) {
  return mode == 1 || (mode == 2 && !comp_less(v, i, k, x));
}

__global__ void flags_kernel(int64_t nel, const int* __restrict__ p_in, const double* __restrict__ ga,
                             const double* __restrict__ gd, const unsigned long long* __restrict__ selbuf,
                             Thresholds th, int p_max, int* __restrict__ p_out, int* __restrict__ theta_out) {
  // thresholds computed on the device live in selbuf: [0..1] analysis coarsen, [2..3] analysis
  // refine, [4..5] density coarsen, [6..7] density refine (key, index)
  if (th.ac_mode == 2) { th.ac_key = selbuf[0]; th.ac_idx = selbuf[1]; }
  if (th.ar_mode == 2) { th.ar_key = selbuf[2]; th.ar_idx = selbuf[3]; }
  if (th.dc_mode == 2) { th.dc_key = selbuf[4]; th.dc_idx = selbuf[5]; }
  if (th.dr_mode == 2) { th.dr_key = selbuf[6]; th.dr_idx = selbuf[7]; }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    int p = p_in[e], t = 0;
    if (in_low(th.ac_mode, ga[e], e, th.ac_key, th.ac_idx)) { t = -1; p = p > 1 ? p - 1 : 1; }
    if (in_high(th.ar_mode, ga[e], e, th.ar_key, th.ar_idx)) { t = 1; p = p + 1 < p_max ? p + 1 : p_max; }
    const double g = gd[e];
    if (g < 0.0 && in_low(th.dc_mode, g, e, th.dc_key, th.dc_idx)) {
      if (p == 1) t = -2;
      else if (t == 0) p -= 1;
    }
    if (g > 0.0 && in_high(th.dr_mode, g, e, th.dr_key, th.dr_idx) && (t == 0 || t == -1))
      p = p + 1 < p_max ? p + 1 : p_max;
    p_out[e] = p;
    theta_out[e] = t;
  }
}

// one Jacobi sweep of p_k <- max(p_k, max_{edge neighbours} p_j - 2)
__global__ void smooth_kernel(int nelx, int nely, const int* __restrict__ a, int* __restrict__ b) {
  const int64_t nel = (int64_t)nelx * nely;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    int ix = (int)(e % nelx), iy = (int)(e / nelx);
    int m = a[e];
    int nb = -1000;
    if (ix > 0) nb = max(nb, a[e - 1]);
    if (ix + 1 < nelx) nb = max(nb, a[e + 1]);
    if (iy > 0) nb = max(nb, a[e - nelx]);
    if (iy + 1 < nely) nb = max(nb, a[e + nelx]);
    b[e] = max(m, nb - 2);
  }
}

__device__ int isqrt_dev(int v) {
  int r = 0;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

__global__ void final_kernel(int64_t nel, const int* __restrict__ p_s, const int* __restrict__ theta,
                             const double* __restrict__ eqr, double alpha_qr, int p_max, int d_max,
                             int32_t* __restrict__ p_new, int32_t* __restrict__ d_new, int8_t* __restrict__ th_out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    int p = p_s[e], t = theta[e];
    int nd = 2 * (p + 1) * (p + 1) - 3;
    if (nd > d_max) nd = d_max;
    int d = t == -2 ? 1 : isqrt_dev(nd);
    if (eqr[e] > alpha_qr) p = p + 1 < p_max ? p + 1 : p_max;
    p_new[e] = p;
    d_new[e] = d;
    th_out[e] = (int8_t)t;
  }
}

// ------------------------------------------------------------------------------------ OC
// rho_new_j = clip(rho_j (B_j / lambda)^eta, max(0, rho_j - m), min(1, rho_j + m)), B_j = -dc_j / dv_j,
// written as t_j lambda^-eta with t_j = rho_j B_j^eta formed once.  The volume of a trial lambda is
// sum_j dv_j clip(t_j c, lo_j, hi_j) = sum_j clip(T_j c, L_j, H_j) with T, L, H the values scaled by
// their subcell's area (dv > 0 commutes with the clip), so a bisection pass is a flat stream of
// three arrays with one multiply and one add per value on the FP64 pipes; the clip is taken on the
// integer pipes (non-negative doubles order like their bit patterns).  The volume sum is reduced
// in a fixed order and its last block takes the bisection step itself, so the whole bisection is a
// chain of identical launches with no host round trip.
constexpr int kOCBlock = 256;

__device__ __forceinline__ double oc_pow(double x, double eta) { return eta == 0.5 ? sqrt(x) : pow(x, eta); }

// clip(x, lo, hi) for non-negative lo <= hi (x >= 0 or -0) by signed 64-bit compares of the bits
__device__ __forceinline__ double clip_nonneg(double x, double lo, double hi) {
  long long xi = __double_as_longlong(x);
  const long long li = __double_as_longlong(lo), hi_ = __double_as_longlong(hi);
  xi = xi > li ? xi : li;
  xi = xi < hi_ ? xi : hi_;
  return __longlong_as_double(xi);
}

// t_j, and the area-scaled T_j = dv t_j, L_j = dv max(0, rho_j - m), H_j = dv min(1, rho_j + m)
__global__ void __launch_bounds__(kOCBlock) oc_prep_kernel(int64_t nel, const int64_t* __restrict__ off,
                                                           const int* __restrict__ dmap, double hx, double hy,
                                                           const double* __restrict__ rho,
                                                           const double* __restrict__ dc, double move, double eta,
                                                           double* __restrict__ t, double* __restrict__ T,
                                                           double* __restrict__ Lo, double* __restrict__ Hi) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = w0; e < nel; e += nw) {
    const int d = dmap[e];
    const double dv = hx * hy / ((double)d * d);
    for (int64_t j = off[e] + lane; j < off[e + 1]; j += 32) {
      const double r = rho[j];
      const double tj = r * oc_pow(fmax(-dc[j], 0.0) / dv, eta);
      t[j] = tj;
      T[j] = dv * tj;
      Lo[j] = dv * fmax(0.0, r - move);
      Hi[j] = dv * fmin(1.0, r + move);
    }
  }
}

__global__ void __launch_bounds__(kOCBlock) oc_sum_kernel(int64_t n, const double* __restrict__ T,
                                                          const double* __restrict__ Lo,
                                                          const double* __restrict__ Hi, double eta,
                                                          double* __restrict__ lam, double target, double tol,
                                                          int* __restrict__ done, double* __restrict__ part,
                                                          unsigned* __restrict__ cnt) {
  if (*done) return;
  __shared__ double ws[kOCBlock / 32];
  __shared__ int last;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const double lmid = 0.5 * (lam[0] + lam[1]);
  const double c = eta == 0.5 ? 1.0 / sqrt(lmid) : pow(lmid, -eta);
  double s = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    s += clip_nonneg(T[j] * c, Lo[j], Hi[j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ws[wib] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kOCBlock / 32; ++w) b += ws[w];
    part[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  for (int i = 0; i < (int)gridDim.x; ++i) tot += __ldcg(part + i);
  if (tot > target) lam[0] = lmid; else lam[1] = lmid;
  if ((lam[1] - lam[0]) / (lam[0] + lam[1]) <= tol) *done = 1;
  *cnt = 0u;
}

__global__ void __launch_bounds__(kOCBlock) oc_write_kernel(int64_t n, const double* __restrict__ rho,
                                                            const double* __restrict__ t, double move, double eta,
                                                            const double* __restrict__ lam, double* __restrict__ out) {
  const double lmid = 0.5 * (lam[0] + lam[1]);
  const double c = eta == 0.5 ? 1.0 / sqrt(lmid) : pow(lmid, -eta);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double r = rho[j];
    out[j] = fmin(fmax(t[j] * c, fmax(0.0, r - move)), fmin(1.0, r + move));
  }
}

// ------------------------------------------------------------------------------------ host side
mto_status ensure_basis(mto_handle h, BasisTab** out) {
  if (!h->basis_tab) {
    MTO_TRY(mto_alloc(h, reinterpret_cast<unsigned char**>(&h->basis_tab), sizeof(BasisTab)));
    basis_table_kernel<<<1, 32, 0, h->stream>>>(reinterpret_cast<BasisTab*>(h->basis_tab));
    MTO_TRY(mto_after_launch(h, "basis_table_kernel"));
  }
  *out = reinterpret_cast<BasisTab*>(h->basis_tab);
  return MTO_OK;
}

// Selection of the k-th composite key among participating values; the (key, index) pair is
// copied to out[0..1] (device).  k is read from a device value.
mto_status select_kth(mto_handle h, const double* v, int64_t n, int mode, const long long* k_dev,
                      unsigned long long* out) {
  unsigned int* hist = reinterpret_cast<unsigned int*>(h->sel + 64);   // 256 counters
  unsigned long long* st = h->sel;
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), h->stream), "memset"));
  sel_init_kernel<<<1, 1, 0, h->stream>>>(st, k_dev);
  MTO_TRY(mto_after_launch(h, "sel_init_kernel"));
  const int grd = grid_for(n, 256, 152 * 4);
  for (int shift = 56; shift >= 0; shift -= 8) {
    sel_hist_kernel<<<grd, 256, 0, h->stream>>>(n, v, mode, shift, st, hist);
    MTO_TRY(mto_after_launch(h, "sel_hist_kernel"));
    sel_pick_kernel<<<1, 32, 0, h->stream>>>(shift, st, hist);
    MTO_TRY(mto_after_launch(h, "sel_pick_kernel"));
  }
  const int64_t nch = (n + 1023) / 1024;
  unsigned int* cnt = reinterpret_cast<unsigned int*>(h->ibuf + 3 * h->nel);
  sel_count_kernel<<<(unsigned)nch, 256, 0, h->stream>>>(n, v, mode, st, cnt);
  MTO_TRY(mto_after_launch(h, "sel_count_kernel"));
  sel_index_kernel<<<1, 32, 0, h->stream>>>(n, v, mode, st, cnt, nch);
  MTO_TRY(mto_after_launch(h, "sel_index_kernel"));
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(out, st + 2, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream), "copy"));
  return MTO_OK;
}

}  // namespace

mto_status map_update(mto_handle h, const double* ga, const double* gd, const double* eqr,
                      const mto_indicator_opts* o, int32_t* pn, int32_t* dn, int8_t* th) {
  const int64_t nel = h->nel;
  const int grd = grid_for(nel, 256, 152 * 4);
  unsigned long long* selbuf = h->sel + 8;         // 8 values: the four (key, index) thresholds
  long long* kdev = reinterpret_cast<long long*>(h->sel + 24);
  Thresholds T;
  memset(&T, 0, sizeof(T));
  // analysis step: floor(frac * nel) lowest / highest Gamma^a
  const int64_t nc = (int64_t)std::floor(o->frac_a_coarsen * (double)nel);
  const int64_t nr = (int64_t)std::floor(o->frac_a_refine * (double)nel);
  long long kh[4];
  if (nc >= nel) T.ac_mode = 1;
  else if (nc > 0) {
    T.ac_mode = 2;
    kh[0] = nc;
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(kdev, &kh[0], sizeof(long long), cudaMemcpyHostToDevice, h->stream), "copy"));
    MTO_TRY(select_kth(h, ga, nel, 0, kdev, selbuf + 0));
  }
  if (nr >= nel) T.ar_mode = 1;
  else if (nr > 0) {
    T.ar_mode = 2;
    kh[1] = nel - nr;
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(kdev + 1, &kh[1], sizeof(long long), cudaMemcpyHostToDevice, h->stream), "copy"));
    MTO_TRY(select_kth(h, ga, nel, 0, kdev + 1, selbuf + 2));
  }
  // density step: fractions of the negative / positive Gamma^d elements
  if (o->alpha_d_coarsen >= 1.0) T.dc_mode = 1;
  if (o->alpha_d_refine >= 1.0) T.dr_mode = 1;
  if (T.dc_mode == 0 || T.dr_mode == 0) {
    unsigned long long* cnt = h->sel + 18;
    MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), h->stream), "memset"));
    count_sign_kernel<<<grd, 256, 0, h->stream>>>(nel, gd, cnt);
    MTO_TRY(mto_after_launch(h, "count_sign_kernel"));
    unsigned long long hc[2];
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, h->stream), "copy"));
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    const int64_t nneg = (int64_t)hc[0], npos = (int64_t)hc[1];
    if (T.dc_mode == 0) {
      const int64_t kc = (int64_t)std::floor(o->alpha_d_coarsen * (double)nneg);
      if (kc >= nneg) T.dc_mode = 1;
      else if (kc > 0) {
        T.dc_mode = 2;
        kh[2] = kc;
        MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(kdev + 2, &kh[2], sizeof(long long), cudaMemcpyHostToDevice, h->stream), "copy"));
        MTO_TRY(select_kth(h, gd, nel, 1, kdev + 2, selbuf + 4));
      }
    }
    if (T.dr_mode == 0) {
      const int64_t kr = (int64_t)std::floor(o->alpha_d_refine * (double)npos);
      if (kr >= npos) T.dr_mode = 1;
      else if (kr > 0) {
        T.dr_mode = 2;
        kh[3] = npos - kr;
        MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(kdev + 3, &kh[3], sizeof(long long), cudaMemcpyHostToDevice, h->stream), "copy"));
        MTO_TRY(select_kth(h, gd, nel, 2, kdev + 3, selbuf + 6));
      }
    }
  }
  int* pa = h->ibuf;
  int* pb = h->ibuf + nel;
  int* tt = h->ibuf + 2 * nel;
  flags_kernel<<<grd, 256, 0, h->stream>>>(nel, h->p_d, ga, gd, selbuf, T, o->p_max, pa, tt);
  MTO_TRY(mto_after_launch(h, "flags_kernel"));
  for (int s = 0; s < MTO_P_MAX; ++s) {
    smooth_kernel<<<grd, 256, 0, h->stream>>>(h->nelx, h->nely, pa, pb);
    MTO_TRY(mto_after_launch(h, "smooth_kernel"));
    int* tmp = pa; pa = pb; pb = tmp;
  }
  final_kernel<<<grd, 256, 0, h->stream>>>(nel, pa, tt, eqr, o->alpha_qr, o->p_max, o->d_max, pn, dn, th);
  return mto_after_launch(h, "final_kernel");
}

mto_status indicators(mto_handle h, const double* u, const double* rho, const mto_material* m,
                      const mto_indicator_opts* o, double* ga, double* gd, double* eqr, int32_t* pn, int32_t* dn,
                      int8_t* th) {
  TimedScope ts(h, F_INDICATOR);
  const int64_t nel = h->nel;
  BasisTab* B;
  MTO_TRY(ensure_basis(h, &B));
  // outputs the caller did not ask for go to scratch
  double* ga_ = ga ? ga : h->dbuf;
  double* gd_ = gd ? gd : h->dbuf + nel;
  double* eq_ = eqr ? eqr : h->edge_buf + (h->n_edges);     // after the edge values
  ClassPtrs cp;
  for (int p = 0; p <= kPMaxTab; ++p) {
    cp.gmap[p] = p <= MTO_P_MAX ? h->pc[p].gmap : nullptr;
  }
  // Kelly
  kelly_edge_kernel<<<grid_for(h->n_edges, 128, 152 * 8), 128, 0, h->stream>>>(
      h->nelx, h->nely, h->p_d, h->slot_d, cp, h->cons_d, u, B, h->hx, h->hy, h->edge_buf);
  MTO_TRY(mto_after_launch(h, "kelly_edge_kernel"));
  kelly_sum_kernel<<<grid_for(nel, 256), 256, 0, h->stream>>>(h->nelx, h->nely, h->edge_buf, ga_);
  MTO_TRY(mto_after_launch(h, "kelly_sum_kernel"));
  // density indicator
  unsigned long long* mm = h->sel + 16;
  unsigned long long init[2] = {~0ULL, 0ULL};
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, h->stream), "copy"));
  minmax_kernel<<<grid_for(h->design_len, 256, 152 * 4), 256, 0, h->stream>>>(h->design_len, rho, mm);
  MTO_TRY(mto_after_launch(h, "minmax_kernel"));
  gamma_d_kernel<<<grid_for(nel, 128), 128, 0, h->stream>>>(nel, h->design_off_d, rho, mm, o->cycle, o->alpha,
                                                           o->beta, gd_);
  MTO_TRY(mto_after_launch(h, "gamma_d_kernel"));
  // QR error per (p, d) class
  for (size_t ci = 0; ci < h->bc.size(); ++ci) {
    const BClass& b = h->bc[ci];
    const BClass& b1 = h->bc_qr[ci];
    const PClass& c = h->pc[b.p];
    const int n0 = 2 * (b.p + 1) * (b.p + 1), n1 = 2 * (b.p + 2) * (b.p + 2);
    size_t smem = sizeof(double) * ((size_t)packed_size(n1) + n0 + n1 + n1 + b.S + n0 + n1 + n1 + 3 * n1);
    if (smem > 48 * 1024) cudaFuncSetAttribute(qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_kernel<<<b.n, 32, smem, h->stream>>>(b.p, b.d, b.n, b.elem, b.slot, c.L, c.dpos, c.gmap, h->cons_d,
                                            c.K64, c.K32, c.K32lo, b1.K0T,
                                            h->qr[b.p].R, u, rho, h->design_off_d, m->E0, m->Emin, m->q, B, h->hx,
                                            h->hy, eq_);
    MTO_TRY(mto_after_launch(h, "qr_kernel"));
  }
  if (!pn && !dn && !th) return MTO_OK;
  if (!pn || !dn || !th) return mto_fail(h, MTO_EINVAL, "mto_indicator: p_new, d_new and theta go together");
  return map_update(h, ga_, gd_, eq_, o, pn, dn, th);
}

mto_status oc_update(mto_handle h, const double* rho, const double* dc, double volfrac, double move, double eta,
                     double* rho_new, double* lambda) {
  TimedScope ts(h, F_OC);
  const int64_t nel = h->nel;
  double* lam = h->red + 16;       // [l1, l2]
  int* done = h->flags + 8;
  unsigned* cnt = reinterpret_cast<unsigned*>(h->flags + 9);
  if (!h->oc_t) MTO_TRY(mto_alloc(h, &h->oc_t, (size_t)4 * h->design_len));   // t, T, L, H
  const int64_t n = h->design_len;
  double* T = h->oc_t + n;
  double* Lo = T + n;
  double* Hi = Lo + n;
  const double init[2] = {0.0, 1e9};
  h->host_pinned[48] = init[0];
  h->host_pinned[49] = init[1];
  MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(lam, h->host_pinned + 48, 2 * sizeof(double), cudaMemcpyHostToDevice,
                                            h->stream), "copy"));
  MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(h->flags + 8, 0, 2 * sizeof(int), h->stream), "memset"));
  const double target = volfrac * (double)h->nelx * h->nely * h->hx * h->hy;
  const int grd = grid_for(nel * 32, kOCBlock, 152 * 8);
  const int gsum = grid_for(n, kOCBlock, 152 * 8);
  oc_prep_kernel<<<grd, kOCBlock, 0, h->stream>>>(nel, h->design_off_d, h->d_d, h->hx, h->hy, rho, dc, move, eta,
                                                  h->oc_t, T, Lo, Hi);
  MTO_TRY(mto_after_launch(h, "oc_prep_kernel"));
  // bisection on [0, 1e9] to a relative width of 1e-10 takes at most ~100 halvings; the launches
  // after convergence return at once
  for (int it = 0; it < 128; ++it) {
    oc_sum_kernel<<<gsum, kOCBlock, 0, h->stream>>>(n, T, Lo, Hi, eta, lam, target, 1e-10, done, h->cg_part, cnt);
    MTO_TRY(mto_after_launch(h, "oc_sum_kernel"));
  }
  oc_write_kernel<<<gsum, kOCBlock, 0, h->stream>>>(n, rho, h->oc_t, move, eta, lam, rho_new);
  MTO_TRY(mto_after_launch(h, "oc_write_kernel"));
  if (lambda) {
    MTO_TRY(mto_cuda_check(h, cudaMemcpyAsync(h->host_pinned + 16, lam, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy"));
    MTO_TRY(mto_cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    *lambda = 0.5 * (h->host_pinned[16] + h->host_pinned[17]);
  }
  return MTO_OK;
}

}  // namespace mto
