// Step (a) on the 5th-generation tensor cores: K_e = sum_s E(rho_s) K0_s (Eqs. 2-3, App. B
// composite rule) for every element of a (p, d) class as one GEMM per class,
//   C[e][pos] = sum_s E[e][s] * K0[c(pos)][s],
// M = elements, N = positions of the circulant-diagonal element row, K = subcells.
//
// The element matrices need FP64 accuracy (on the binary designs a relative error of 1e-13 in K_e
// moves the compliance by ~1e-6), so the products cannot be plain BF16 products.  The GEMM is made
// exact by slicing (an Ozaki-type error-free splitting): each element's moduli row is scaled by a
// power of two sigma_e (max E <= sigma_e) and each K0 column by a power of two tau_pos, and both
// are cut into 8 slices of 7 bits (56 bits), E/sigma = sum_i a_i 2^-7i and K0/tau = sum_j b_j 2^-7j
// with integer a_i in [0, 127], b_j in [-127, 127] (exact in BF16).  Every slice product a_i . b_j
// over K <= 64 subcells is an integer below 2^20, and all pairs of one level g = i + j share the
// weight 2^-7g: each level accumulates its (at most 8) slice GEMMs in one FP32 TMEM accumulator
// exactly (sums below 2^23).  Levels g = 2..10 are kept (the dropped levels weigh below 2^-51 of
// the row/column scale, the operands' truncation 2^-56); the epilogue adds the levels in FP64,
// rescales by sigma_e tau_pos (powers of two, exact) and stores the FP64 matrix and, for the mixed
// build, its split pair.
//
// One CTA (4 warps) per 128 elements: the A slices (8 x 128 x K) are formed in shared memory from
// rho once; the CTA then walks the N tiles of 32 positions: B slices copied to shared memory, one
// thread issues the 43 x (K/16) tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 32)
// into 9 level accumulators (288 TMEM columns), commits to an mbarrier, and all threads read
// their row back with tcgen05.ld and store 32 consecutive entries of their element's row.
// Operands use the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix).
// Every wait is bounded: on expiry the kernel records an error word and skips the tile.
#include <cstdio>
#include <vector>

#include "mto_internal.cuh"

namespace mto {
namespace {

constexpr int kTM = 128;        // elements per CTA (MMA M)
constexpr int kTN = 32;         // positions per N tile (MMA N)
constexpr int kSlices = 8;      // slices per operand (8 x 7 = 56 bits)
constexpr int kSliceBits = 7;
constexpr int kOpBits = kSlices * kSliceBits;
constexpr int kLevels = 9;      // levels g = i + j = 2..10
constexpr int kTmemCols = 512;  // 9 x 32 = 288 used (allocations are powers of two)
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle.  lbo = byte stride between core matrices
// along K, sbo = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;                // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in the no-swizzle K-major core-matrix layout of a rows x kpad
// BF16 tile
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int kpad) {
  return (uint32_t)(((row >> 3) * (kpad >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// B operand tables of a class: per N tile, 7 slices of kTN x kpad BF16 in the core layout, and
// the column scales tau (power of two) per position.  One thread per (position, subcell).
__global__ void tc_btable_kernel(int S, int kpad, int L, int ntile, const double* __restrict__ K0T,
                                 const int* __restrict__ posc, unsigned short* __restrict__ Bt,
                                 float* __restrict__ tau) {
  const int pos = blockIdx.x;
  if (pos >= ntile * kTN) return;
  __shared__ double colmax;
  const int c = pos < L ? posc[pos] : -1;
  if (threadIdx.x == 0) {
    double m = 0.0;
    if (c >= 0)
      for (int s = 0; s < S; ++s) m = fmax(m, fabs(K0T[(size_t)c * S + s]));
    colmax = m;
  }
  __syncthreads();
  int ex = 0;
  if (colmax > 0.0) frexp(colmax, &ex);   // colmax < 2^ex
  const double sc = ldexp(1.0, -ex);
  if (threadIdx.x == 0) tau[pos] = colmax > 0.0 ? ldexpf(1.0f, ex) : 0.0f;
  const int tile = pos / kTN, row = pos % kTN;
  for (int s = threadIdx.x; s < kpad; s += blockDim.x) {
    const double w = (c >= 0 && s < S) ? K0T[(size_t)c * S + s] * sc : 0.0;   // |w| < 1
    const double aw = fabs(w);
    const unsigned long long W = (unsigned long long)ldexp(aw, kOpBits);   // floor(|w| 2^56)
    for (int j = 0; j < kSlices; ++j) {
      const int bits = (int)((W >> (kOpBits - kSliceBits * (j + 1))) & 127ull);
      const float v = (w < 0.0 ? -1.0f : 1.0f) * (float)bits;
      const unsigned short b = (unsigned short)(__float_as_uint(v) >> 16);   // exact: |v| <= 127
      unsigned char* base = reinterpret_cast<unsigned char*>(Bt) +
                            ((size_t)tile * kSlices + j) * (size_t)kTN * kpad * 2;
      *reinterpret_cast<unsigned short*>(base + core_off(row, s, kpad)) = b;
    }
  }
}

__global__ void __launch_bounds__(128, 1) tc_build_kernel(
    int n, int S, int kpad, int L, int ntile, const int* __restrict__ elem, const int* __restrict__ slot,
    const int64_t* __restrict__ design_off, const double* __restrict__ rho, double E0, double Emin, double q,
    const unsigned short* __restrict__ Bt, const float* __restrict__ tau, double* __restrict__ K64,
    float* __restrict__ Kh, float* __restrict__ Kl, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const size_t a_bytes = (size_t)kSlices * kTM * kpad * 2;
  const size_t b_bytes = (size_t)kSlices * kTN * kpad * 2;
  unsigned char* As = smem;
  unsigned char* Bs = smem + a_bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + a_bytes + b_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  float* sigma_s = reinterpret_cast<float*>(bar + 2);   // [kTM]
  const int t = threadIdx.x, warp = t >> 5;
  const int base = blockIdx.x * kTM;

  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  if (t == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // A slices: this thread's element row, moduli E_s scaled by sigma_e and cut into 7 x 7 bits.
  // E is monotone in rho, so sigma_e comes from the largest density (one E per element); q = 3
  // takes products instead of pow (GB300's FP64 pipes made the per-subcell pow the bottleneck).
  {
    const int k = base + t;
    const bool act = k < n;
    const bool cube = q == 3.0;
    auto modulus = [&](double r) { return Emin + (cube ? r * r * r : pow(r, q)) * (E0 - Emin); };
    int64_t off = 0;
    double rmax = 0.0;
    if (act) {
      off = design_off[elem[k]];
      for (int s = 0; s < S; ++s) rmax = fmax(rmax, rho[off + s]);
    }
    const double m = act ? modulus(rmax) : 0.0;
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);
    const double sc = ldexp(1.0, -ex);
    sigma_s[t] = m > 0.0 ? ldexpf(1.0f, ex) : 0.0f;
    for (int s = 0; s < kpad; ++s) {
      double v = 0.0;
      if (act && s < S) v = modulus(rho[off + s]) * sc;   // [0, 1)
      const unsigned long long V = (unsigned long long)ldexp(v, kOpBits);   // floor(v 2^56)
      for (int i = 0; i < kSlices; ++i) {
        const float a = (float)((V >> (kOpBits - kSliceBits * (i + 1))) & 127ull);
        const unsigned short b = (unsigned short)(__float_as_uint(a) >> 16);
        *reinterpret_cast<unsigned short*>(As + (size_t)i * kTM * kpad * 2 + core_off(t, s, kpad)) = b;
      }
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16(kTM, kTN);
  const uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
  const int kst = kpad / 16;
  const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
  const int row = base + t;
  const bool act = row < n;
  const int sl = act ? slot[row] : 0;
  const float sig = sigma_s[t];
  uint32_t phase = 0;

  for (int tile = 0; tile < ntile; ++tile) {
    // B slices of this tile into shared memory
    const uint4* src = reinterpret_cast<const uint4*>(Bt + (size_t)tile * kSlices * kTN * kpad);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (size_t i = t; i < b_bytes / 16; i += blockDim.x) dst[i] = src[i];
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) {
      for (int g = 0; g < kLevels; ++g) {
        uint32_t acc = 0;
        const int lev = g + 2;
        for (int i = 1; i <= kSlices; ++i) {
          const int j = lev - i;
          if (j < 1 || j > kSlices) continue;
          for (int ks = 0; ks < kst; ++ks) {
            const uint64_t ad = smem_desc(a0 + (uint32_t)((size_t)(i - 1) * kTM * kpad * 2) + ks * 256u, 128u, sbo);
            const uint64_t bd = smem_desc(b0 + (uint32_t)((size_t)(j - 1) * kTN * kpad * 2) + ks * 256u, 128u, sbo);
            umma_bf16(tmem + (uint32_t)(g * kTN), ad, bd, idesc, acc);
            acc = 1;
          }
        }
      }
      umma_commit(bar);
    }
    // bounded wait for the MMAs; the whole CTA agrees before leaving on expiry
    unsigned spins = 0;
    bool ok = true;
    while (!mbar_try_wait(bar, phase)) {
      if (++spins > kSpinLimit) {
        ok = false;
        break;
      }
    }
    phase ^= 1u;
    tc_fence_after();
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicExch(err, 1);
      break;   // the accumulators are not trustworthy: stop this CTA (the caller reports the error)
    }
    // epilogue: this thread's TMEM lane = its row; chunks of 16 positions.  Every level sum is an
    // integer below 2^23 (exact in FP32); the levels are added from the smallest in FP64 (9 terms
    // per entry), then scaled by sigma_e tau_pos (a power of two: exact)
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int ch = 0; ch < kTN / 16; ++ch) {
      double acc[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] = 0.0;
#pragma unroll 1
      for (int g = kLevels - 1; g >= 0; --g) {
        uint32_t v[16];
        tmem_ld16(lane_addr + (uint32_t)(g * kTN + ch * 16), v);
        tmem_wait_ld();
        const double wgt = ldexp(1.0, -kSliceBits * (g + 2));
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = fma((double)__uint_as_float(v[c]), wgt, acc[c]);
      }
      if (act) {
        const int pos0 = tile * kTN + ch * 16;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int pos = pos0 + c;
          if (pos >= L) break;
          const double kv = acc[c] * ((double)sig * (double)__ldg(tau + pos));
          const size_t o = (size_t)sl * L + pos;
          K64[o] = kv;
          if (Kh) {
            const float hi = (float)kv;
            Kh[o] = hi;
            Kl[o] = (float)(kv - (double)hi);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // TMEM and B reused by the next tile
    tc_fence_after();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(*tmem_slot, kTmemCols);
}

}  // namespace

// Per (p, d) class with d <= 8: B slice tables (once per nu) for the tensor-core build.
mto_status tc_tables(mto_handle h) {
  for (auto& b : h->bc) {
    if (b.S > 64) continue;
    const PClass& c = h->pc[b.p];
    const int kpad = (b.S + 15) / 16 * 16;
    const int ntile = (c.L + kTN - 1) / kTN;
    if (!b.tcB) {
      MTO_TRY(mto_alloc(h, &b.tcB, (size_t)ntile * kSlices * kTN * kpad));
      MTO_TRY(mto_alloc(h, &b.tcTau, (size_t)ntile * kTN));
      MTO_TRY(mto_cuda_check(h, cudaMemsetAsync(b.tcB, 0, sizeof(unsigned short) * ntile * kSlices * kTN * kpad,
                                                h->stream), "memset"));
    }
    tc_btable_kernel<<<ntile * kTN, 64, 0, h->stream>>>(b.S, kpad, c.L, ntile, b.K0T, c.posc, b.tcB, b.tcTau);
    MTO_TRY(mto_after_launch(h, "tc_btable_kernel"));
  }
  return MTO_OK;
}

// Dynamic shared memory of the build kernel, at least 120 KB so that one CTA (and one 512-column
// TMEM allocation) is resident per SM.
size_t tc_smem_bytes(int kpad) {
  const size_t need = (size_t)kSlices * (kTM + kTN) * kpad * 2 + 16 + 4 * kTM + 64;
  return need < 120 * 1024 ? 120 * 1024 : need;
}

// The tensor-core build of one (p, d) class (d <= 8).
mto_status tc_build_class(mto_handle h, const BClass& b, const double* rho, const mto_material* m, int precision) {
  const PClass& c = h->pc[b.p];
  const int kpad = (b.S + 15) / 16 * 16;
  const int ntile = (c.L + kTN - 1) / kTN;
  const size_t smem = tc_smem_bytes(kpad);
  MTO_TRY(mto_cuda_check(h, cudaFuncSetAttribute(tc_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem), "cudaFuncSetAttribute"));
  const int grid = (b.n + kTM - 1) / kTM;
  tc_build_kernel<<<grid, 128, smem, h->stream>>>(
      b.n, b.S, kpad, c.L, ntile, b.elem, b.slot, h->design_off_d, rho, m->E0, m->Emin, m->q, b.tcB, b.tcTau,
      c.K64, precision == MTO_MIXED ? c.K32 : nullptr, precision == MTO_MIXED ? c.K32lo : nullptr, h->flags + 4);
  return mto_after_launch(h, "tc_build_kernel");
}

}  // namespace mto
