// Building blocks shared by the Davidson vector kernels (vec.cu, vec_split.cu): the
// deterministic one-pass cross-block reduction and 16-byte vector loads.  Included inside
// an anonymous namespace of each translation unit.
#pragma once

constexpr int kGridPerSM = 4;
constexpr int kSlots = KMAX + 4;

struct Ticket {
  // returns true in every thread of the last block to arrive
  __device__ static bool last_block(unsigned int* counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int t = atomicAdd(counter, 1u);
      is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return is_last;
  }
};

// Block-reduce the per-thread values acc[0..NDOT+NEXTRA): the first NDOT are dot
// products of which only kdots < NDOT are live (slots 0..kdots), the last NEXTRA are
// always live and go to slots kdots..kdots+NEXTRA.  Every index into acc is a
// compile-time constant, so acc stays in registers.  Stores this block's partial sums at
// partials[blockIdx.x * kSlots + slot].
template <int NDOT, int NEXTRA>
__device__ void block_partials(double (&acc)[NDOT + NEXTRA], int kdots, double* partials) {
  __shared__ double red[kVecThreads / 32][kSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NDOT + NEXTRA; ++j) {
    const bool live = j < NDOT ? (j < kdots) : true;
    const int slot = j < NDOT ? j : kdots + (j - NDOT);
    if (live) {
      double v = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][slot] = v;
    }
  }
  __syncthreads();
  const int nv = kdots + NEXTRA;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) v += red[w][j];
    partials[(int64_t)blockIdx.x * kSlots + j] = v;
  }
}

// In the last block: total[j] = sum over blocks of partials, j < nv.  One warp per slot:
// the lanes add block-strided partials (independent loads, one round trip), then a
// shuffle tree; the order is fixed, so the result is deterministic.
__device__ void final_sums(const double* partials, int nv, double* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < nv; j += nw) {
    double v = 0.0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(&partials[(int64_t)b * kSlots + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) total[j] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ double2 ld2(const double* p) {
  return __ldg(reinterpret_cast<const double2*>(p));
}
__device__ __forceinline__ double2 ld2cg(const double* p) {
  return __ldcg(reinterpret_cast<const double2*>(p));
}


// Split-precision block reduction: each warp reduces its FP32 values with FP32 shuffles
// and its FP64 values with FP64 shuffles (FP64 adds run at about 1/64 of the FP32 rate on
// this part, so a full FP64 warp reduction of ~20 values per thread would cost more than
// the streaming pass itself); the per-warp results are combined in FP64 and stored as
// this block's partial sums, in the slot layout of block_partials.
struct SplitReduce {
  double (*red)[kSlots];
  int lane, warp;
  __device__ void f32(float v, int slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][slot] = (double)v;
  }
  __device__ void f64(double v, int slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][slot] = v;
  }
  __device__ void store(int nv, double* partials) {
    __syncthreads();
    for (int j = threadIdx.x; j < nv; j += blockDim.x) {
      double v = 0.0;
      for (int w = 0; w < kVecThreads / 32; ++w) v += red[w][j];
      partials[(int64_t)blockIdx.x * kSlots + j] = v;
    }
  }
};

#include "cvt.cuh"
