// Allocation-free variant of s = V^T w (dmrg_gemv_trans_noalloc).
//
// Some callers cannot let a library allocate device memory: an application whose own
// allocator owns all device memory (a framework's caching allocator, or a memory pool
// reserved at start-up), or a latency-critical loop in which cudaMalloc / cudaFree would
// synchronise the device.  This entry point computes the same product as dmrg_gemv_trans
// but keeps its cross-block partial sums in a fixed scratch array that lives in the
// library's own device image instead of a per-call allocation.
//
// The scratch is one file-scope __device__ array of kScratchDoubles doubles (196,864
// bytes); every GPU that loads the library holds it until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress, during the first call
// made on that device (with that device current).  All calls on a device share the array,
// which keeps the previous call's contents; the ticket counter that must start at zero is
// cleared at the start of every call.  Calls that overlap on the GPU (different streams,
// or different host threads, without ordering between them) race on the array.
#include <mutex>

#include "internal.h"

namespace dmrg {
namespace {

constexpr int kNoAllocMaxBlocks = 1024;                 // largest grid the variant launches
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxK = DMRG_MAX_SUBSPACE;         // columns of V (24)
constexpr int kCounterDoubles = 32;                     // 256-byte slot for the ticket
constexpr int kScratchDoubles = kNoAllocMaxBlocks * kNoAllocMaxK + kCounterDoubles;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

double* g_scratch_ptr[kMaxDevices];
cudaError_t g_setup_status[kMaxDevices];
std::once_flag g_setup_once[kMaxDevices];

// Each block sums its rows of V^T w for the k columns, writes the k block sums to the
// scratch rows of its block index, and the last block to finish adds the rows in block
// order (fixed order: the result does not depend on block scheduling).
__global__ void __launch_bounds__(kNoAllocThreads)
gemv_trans_noalloc_kernel(const double* __restrict__ V, int64_t ldv, int64_t n, int k,
                          const double* __restrict__ w, double* __restrict__ s_out,
                          double* scratch) {
  double* partials = scratch;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNoAllocMaxBlocks * kNoAllocMaxK);
  double acc[kNoAllocMaxK];
#pragma unroll
  for (int j = 0; j < kNoAllocMaxK; ++j) acc[j] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double wv = __ldg(w + e);
#pragma unroll
    for (int j = 0; j < kNoAllocMaxK; ++j)
      if (j < k) acc[j] = fma(__ldg(V + j * ldv + e), wv, acc[j]);
  }
  __shared__ double red[kNoAllocThreads / 32][kNoAllocMaxK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kNoAllocMaxK; ++j) {
    if (j < k) {
      double v = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][j] = v;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double v = 0.0;
    for (int wi = 0; wi < kNoAllocThreads / 32; ++wi) v += red[wi][j];
    partials[blockIdx.x * kNoAllocMaxK + j] = v;
  }
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(&partials[b * kNoAllocMaxK + j]);
    s_out[j] = v;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace
}  // namespace dmrg

extern "C" dmrg_status dmrg_gemv_trans_noalloc(const double* V, int64_t ldv, int64_t n,
                                               int32_t k, const double* w, double* s,
                                               void* stream) {
  using namespace dmrg;
  if (k < 1 || k > kNoAllocMaxK) {
    set_error("dmrg_gemv_trans_noalloc: k = %d is outside [1, %d], the column count its "
              "fixed scratch array holds", (int)k, kNoAllocMaxK);
    return DMRG_ERR_INVALID_ARG;
  }
  if (n < 0 || ldv < n || !s || (n > 0 && (!V || !w))) {
    set_error("dmrg_gemv_trans_noalloc: bad argument (need n >= 0, ldv >= n, non-NULL "
              "V, w, s)");
    return DMRG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  DMRG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("dmrg_gemv_trans_noalloc: device index %d beyond %d", dev, kMaxDevices);
    return DMRG_ERR_INVALID_ARG;
  }
  // set-up, once per device, with that device current: the device address of the scratch
  std::call_once(g_setup_once[dev], [dev]() {
    g_setup_status[dev] = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_noalloc_scratch);
  });
  if (g_setup_status[dev] != cudaSuccess) {
    set_error("dmrg_gemv_trans_noalloc: cudaGetSymbolAddress failed: %s",
              cudaGetErrorString(g_setup_status[dev]));
    return DMRG_ERR_CUDA;
  }
  if (n == 0) {
    DMRG_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(double) * k, st));
    return DMRG_OK;
  }
  double* scratch = g_scratch_ptr[dev];
  // the ticket must start at zero: clear it on the stream before the kernel
  DMRG_CUDA_TRY(cudaMemsetAsync(scratch + kNoAllocMaxBlocks * kNoAllocMaxK, 0,
                                sizeof(double) * kCounterDoubles, st));
  int sms = 0;
  DMRG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = sms * 4;
  if (grid > kNoAllocMaxBlocks) grid = kNoAllocMaxBlocks;
  if (grid < 1) grid = 1;
  gemv_trans_noalloc_kernel<<<grid, kNoAllocThreads, 0, st>>>(V, ldv, n, k, w, s, scratch);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}
