// mto_compliance_noalloc: the compliance dot product C = f^T u of step (c) with no device or host
// allocation, for callers that manage all memory themselves.  Its block partial sums live in a
// fixed file-scope device array instead of handle workspace.
#include <mutex>

#include "mto_internal.cuh"

namespace {

constexpr int kBlocks = 8192;                         // partial sums held by the scratch
constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int64_t kPerBlock = (int64_t)kThreads * kPerThread;   // 2048 entries per block
constexpr int64_t kMaxN = (int64_t)kBlocks * kPerBlock;        // 16,777,216 entries

// Scratch: [0, kBlocks) block partials; element kBlocks holds the finished-block counter (as an
// unsigned int), which must be zero when a launch starts.  Zero at module load; every call also
// clears it before its launch, and the last block of a launch clears it again.  72 KB.
static __device__ __align__(256) double g_scratch[kBlocks + 32];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per 2048 consecutive entries; the last block to finish sums the partials in a fixed
// order that depends only on n (strided per thread, then a shuffle tree), not on scheduling, and
// writes *C.
__global__ void __launch_bounds__(kThreads) dot_noalloc_kernel(int64_t n, const double* __restrict__ f,
                                                                const double* __restrict__ u,
                                                                double* __restrict__ scratch,
                                                                double* __restrict__ C) {
  __shared__ double ws[kThreads / 32];
  __shared__ int last;
  unsigned* count = reinterpret_cast<unsigned*>(scratch + kBlocks);
  const int64_t base = (int64_t)blockIdx.x * kPerBlock;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
    if (i < n) s = fma(f[i], u[i], s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b += ws[w];
    scratch[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(count, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) t += __ldcg(scratch + i);
  t = warp_sum(t);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) r += ws[w];
    *C = r;
    *count = 0u;
  }
}

}  // namespace

extern "C" mto_status mto_compliance_noalloc(int32_t device, const double* f, const double* u, int64_t n,
                                             void* stream, double* C) {
  if (!f || !u || !C || n < 0 || n > kMaxN || device < 0 || device >= kMaxDevices) return MTO_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return MTO_ECUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return MTO_ECUDA;
  mto_status st = MTO_OK;
  double* scratch = nullptr;
  {
    // once per device, with that device current: the scratch array's device address (kept for
    // the life of the process, so the library must not be used across a cudaDeviceReset)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) st = MTO_ECUDA;
      else g_scratch_ptr[device] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[device];
  }
  if (st == MTO_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = n == 0 ? 1 : (int)((n + kPerBlock - 1) / kPerBlock);
    if (cudaMemsetAsync(scratch + kBlocks, 0, sizeof(unsigned), s) != cudaSuccess) st = MTO_ECUDA;
    if (st == MTO_OK) {
      dot_noalloc_kernel<<<blocks, kThreads, 0, s>>>(n, f, u, scratch, C);
      if (cudaGetLastError() != cudaSuccess) st = MTO_ECUDA;
    }
  }
  if (prev != device) cudaSetDevice(prev);
  return st;
}
