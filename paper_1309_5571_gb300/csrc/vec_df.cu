// Davidson vector kernels in double-float arithmetic (pairs of FP32, ~48 bits).
//
// The vectors stay float64 in memory, but GB300 executes about 0.55 T FP64 FMA/s
// against 6.8 TB/s of HBM, so the FP64 versions of these passes (vec.cu) are bound by the
// FP64 units.  Here every loaded float64 is split exactly into hi + lo with integer
// operations only (hi: the value truncated to 24 significant bits; lo: the remaining
// bits, rounded to 24), the arithmetic runs on the FP32 units with error-free
// transformations (two-sum, fma-based two-product), and results are written back as
// float64 (hi and lo converted exactly by bit manipulation, one FP64 add).  ~48-bit
// arithmetic keeps the Davidson quantities accurate far below the 1e-10 residual
// tolerance (2^-48 = 3.6e-15 relative).  Measured on GB300 these passes are issue-bound and
// not faster than the FP64 ones at the sizes tested, so they are an option
// (dmrg_options.vector_arith = DMRG_VEC_DOUBLE_FLOAT), not the default.
//
//   residual:  x = V y, W y, r = W y - lambda x, ||r||^2, t = r / (lambda - D) (the
//              reciprocal rounded to FP32, the product in double-float), V^T t, ||t||^2
//   cgs:       t -= V s; V^T t (first pass) and ||t||^2
//   overlap:   V^T w and the anchor coupling v_k . W(:,0)
// Cross-block sums: per-warp double-float shuffle reduction, block and grid reductions in
// FP64 over a few values (the one-pass "last block" scheme of vec.cu, fixed order).
#include <math.h>

#include "internal.h"

namespace dmrg {
namespace {

constexpr int kSlotsDF = KMAX + 4;

struct df {
  float h, l;
};

// exact split of a float64 into hi + lo using integer operations only; magnitudes below
// 2^-74 lose their low part, below 2^-126 they are flushed to zero
__device__ __forceinline__ df split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int top = (unsigned int)(b >> 32);
  const int e = (int)((top >> 20) & 0x7ff);
  const unsigned int sign = top & 0x80000000u;
  df r;
  if (e <= 896) {
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  if (e >= 1151) {  // beyond the FP32 range: let the hardware conversion saturate
    r.h = (float)x;
    r.l = 0.0f;
    return r;
  }
  const unsigned int mhi = (unsigned int)((b >> 29) & 0x7FFFFFu);
  r.h = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | mhi);
  const unsigned int mlo = (unsigned int)(b & 0x1FFFFFFFull);  // 29 low bits
  float lo = 0.0f;
  if (mlo != 0u && e >= 949) lo = __uint2float_rn(mlo) * __int_as_float((e - 948) << 23);
  r.l = sign ? -lo : lo;
  return r;
}

// exact conversion of an FP32 value to float64 bits (normal numbers and zero)
__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;  // zero, subnormal, inf, nan: rare path
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double to_d(df a) { return f2d(a.h) + f2d(a.l); }

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  df r;
  r.h = a + b;
  r.l = b - (r.h - a);
  return r;
}

__device__ __forceinline__ df add(df a, df b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  const float e = (a.h - (s - bp)) + (b.h - bp);
  return fast_two_sum(s, e + a.l + b.l);
}

// acc + a * b
__device__ __forceinline__ df fma_df(df a, df b, df acc) {
  const float p = a.h * b.h;
  float pe = fmaf(a.h, b.h, -p);
  pe = fmaf(a.h, b.l, pe);
  pe = fmaf(a.l, b.h, pe);
  const float s = acc.h + p;
  const float bp = s - acc.h;
  const float e = (acc.h - (s - bp)) + (p - bp);
  return fast_two_sum(s, e + pe + acc.l);
}

__device__ __forceinline__ df neg(df a) {
  a.h = -a.h;
  a.l = -a.l;
  return a;
}

__device__ __forceinline__ df shfl_xor(df a, int o) {
  df r;
  r.h = __shfl_xor_sync(0xffffffffu, a.h, o);
  r.l = __shfl_xor_sync(0xffffffffu, a.l, o);
  return r;
}

// block partial sums of NV double-float values (first kdots of NDOT live), written as
// FP64 to partials[blockIdx.x * kSlotsDF + slot] like vec.cu's block_partials
template <int NDOT, int NEXTRA>
__device__ void block_partials_df(df (&acc)[NDOT + NEXTRA], int kdots, double* partials) {
  __shared__ double red[kVecThreads / 32][kSlotsDF];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NDOT + NEXTRA; ++j) {
    const bool live = j < NDOT ? (j < kdots) : true;
    const int slot = j < NDOT ? j : kdots + (j - NDOT);
    if (live) {
      df v = acc[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = add(v, shfl_xor(v, o));
      if (lane == 0) red[warp][slot] = to_d(v);
    }
  }
  __syncthreads();
  const int nv = kdots + NEXTRA;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) v += red[w][j];
    partials[(int64_t)blockIdx.x * kSlotsDF + j] = v;
  }
}

__device__ bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  return is_last;
}

__device__ void final_sums(const double* partials, int nv, double* total) {
  __shared__ double tmp[kVecThreads];
  for (int j = 0; j < nv; ++j) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      v += __ldcg(&partials[(int64_t)b * kSlotsDF + j]);
    tmp[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) tmp[threadIdx.x] += tmp[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) total[j] = tmp[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- overlap
template <int K>
__global__ void __launch_bounds__(kVecThreads, 2)
overlap_df_kernel(const double* __restrict__ V, int64_t ldv, int64_t n,
                  const double* __restrict__ w, const double* __restrict__ w0,
                  double* __restrict__ partials, unsigned int* counter, double* s_out,
                  DevSmall* small, int Bcol) {
  df acc[K + 1];
#pragma unroll
  for (int j = 0; j < K + 1; ++j) acc[j] = df{0.0f, 0.0f};
  const bool anchored = w0 != nullptr && Bcol > 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double vd[K];
#pragma unroll
    for (int j = 0; j < K; ++j) vd[j] = __ldg(V + j * ldv + e);
    const df wv = split(__ldcg(w + e));
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fma_df(split(vd[j]), wv, acc[j]);
    if (anchored) acc[K] = fma_df(split(vd[K - 1]), split(__ldg(w0 + e)), acc[K]);
  }
  block_partials_df<K, 1>(acc, K, partials);
  if (last_block(counter)) {
    __shared__ double tot[K + 1];
    final_sums(partials, K + 1, tot);
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      if (s_out) s_out[j] = tot[j];
      if (Bcol >= 0) {
        double v = tot[j];
        if (anchored && j == 0) v = tot[K];
        small->B[j * KMAX + Bcol] = v;
        small->B[Bcol * KMAX + j] = v;
      }
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// ---------------------------------------------------------------- residual + correction
template <int K>
__global__ void __launch_bounds__(kVecThreads, 2)
residual_df_kernel(const double* __restrict__ V, const double* __restrict__ W,
                   const double* __restrict__ D, int64_t ldv, int64_t n,
                   double* __restrict__ tcol, double* __restrict__ partials,
                   unsigned int* counter, DevSmall* small, int mode) {
  __shared__ df ys[K];
  __shared__ df lam_sh;
  if (threadIdx.x < K) ys[threadIdx.x] = split(small->y[threadIdx.x]);
  if (threadIdx.x == 0) lam_sh = split(small->lambda);
  __syncthreads();
  const df lam_s = lam_sh;
  const df nlam = neg(lam_s);
  df acc[K + 2];  // [0..K): V^T t, [K]: ||r||^2, [K+1]: ||t||^2
#pragma unroll
  for (int j = 0; j < K + 2; ++j) acc[j] = df{0.0f, 0.0f};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    df vs[K];
    df x = {0.0f, 0.0f}, wy = {0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < K; ++j) {
      vs[j] = split(__ldg(V + j * ldv + e));
      x = fma_df(ys[j], vs[j], x);
      wy = fma_df(ys[j], split(__ldg(W + j * ldv + e)), wy);
    }
    const df r = fma_df(nlam, x, wy);  // W y - lambda V y
    // t = r * (1 / (lambda - D)) with the reciprocal rounded to FP32 (the preconditioner is
    // diag of FP32 values) and the product kept in double-float: the part of t left after
    // orthogonalisation against V can be far smaller than t itself, so t needs the full
    // precision of r
    float inv = 1.0f;
    if (mode == 0) {
      const df dd = split(__ldg(D + e));
      float q = (lam_s.h - dd.h) + (lam_s.l - dd.l);
      if (fabsf(q) < 1e-8f) q = q >= 0.0f ? 1e-8f : -1e-8f;
      inv = 1.0f / q;
    }
    const float tp = r.h * inv;
    const df t = fast_two_sum(tp, fmaf(r.h, inv, -tp) + r.l * inv);
    tcol[e] = to_d(t);
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fma_df(vs[j], t, acc[j]);
    acc[K] = fma_df(r, r, acc[K]);
    acc[K + 1] = fma_df(t, t, acc[K + 1]);
  }
  block_partials_df<K, 2>(acc, K, partials);
  if (last_block(counter)) {
    __shared__ double tot[K + 2];
    final_sums(partials, K + 2, tot);
    for (int j = threadIdx.x; j < K; j += blockDim.x) small->s[0][j] = tot[j];
    if (threadIdx.x == 0) {
      small->rnorm2 = tot[K];
      small->tnorm2_before = tot[K + 1];
      small->tnorm2 = tot[K + 1];
      if (!isfinite(tot[K]) || !isfinite(tot[K + 1])) small->flags |= 2;
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- Gram-Schmidt pass
template <int K, bool DOT>
__global__ void __launch_bounds__(kVecThreads, 2)
cgs_df_kernel(const double* __restrict__ V, int64_t ldv, int64_t n, double* tcol,
              double* __restrict__ partials, unsigned int* counter, DevSmall* small, int sin,
              int sout, int second) {
  if (second && small->tnorm2 >= 0.5 * small->tnorm2_before) return;
  __shared__ df ss[K];
  if (threadIdx.x < K) ss[threadIdx.x] = neg(split(small->s[sin][threadIdx.x]));
  __syncthreads();
  df acc[K + 1];
#pragma unroll
  for (int j = 0; j < K + 1; ++j) acc[j] = df{0.0f, 0.0f};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    df vs[K];
#pragma unroll
    for (int j = 0; j < K; ++j) vs[j] = split(__ldg(V + j * ldv + e));
    df t = split(tcol[e]);
#pragma unroll
    for (int j = 0; j < K; ++j) t = fma_df(ss[j], vs[j], t);
    tcol[e] = to_d(t);
    if (DOT) {
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] = fma_df(vs[j], t, acc[j]);
    }
    acc[K] = fma_df(t, t, acc[K]);
  }
  if (DOT) {
    block_partials_df<K, 1>(acc, K, partials);
  } else {
    df a1[1] = {acc[K]};
    block_partials_df<0, 1>(a1, 0, partials);
  }
  if (last_block(counter)) {
    __shared__ double tot[K + 1];
    const int nv = DOT ? K + 1 : 1;
    final_sums(partials, nv, tot);
    if (DOT)
      for (int j = threadIdx.x; j < K; j += blockDim.x) small->s[sout][j] = tot[j];
    if (threadIdx.x == 0) {
      const double nrm = tot[nv - 1];
      small->tnorm2 = nrm;
      if (!isfinite(nrm)) small->flags |= 2;
      *counter = 0u;
    }
  }
}

template <template <int> class F, int K = 1>
struct KDispatchDF {
  template <typename... A>
  static void run(int k, A... a) {
    if (k == K) F<K>::go(a...);
    else KDispatchDF<F, K + 1>::run(k, a...);
  }
};
template <template <int> class F>
struct KDispatchDF<F, KMAX + 1> {
  template <typename... A>
  static void run(int, A...) {}
};

template <int K>
struct OverlapDF {
  static void go(int grid, cudaStream_t st, const double* V, int64_t ldv, int64_t n,
                 const double* w, const double* w0, double* part, unsigned int* cnt,
                 double* s_out, DevSmall* small, int Bcol) {
    overlap_df_kernel<K><<<grid, kVecThreads, 0, st>>>(V, ldv, n, w, w0, part, cnt, s_out, small, Bcol);
  }
};
template <int K>
struct ResidualDF {
  static void go(int grid, cudaStream_t st, const double* V, const double* W, const double* D,
                 int64_t ldv, int64_t n, double* tcol, double* part, unsigned int* cnt,
                 DevSmall* small, int mode) {
    residual_df_kernel<K><<<grid, kVecThreads, 0, st>>>(V, W, D, ldv, n, tcol, part, cnt, small, mode);
  }
};
template <int K>
struct CgsDF {
  static void go(int grid, cudaStream_t st, const double* V, int64_t ldv, int64_t n, double* tcol,
                 double* part, unsigned int* cnt, DevSmall* small, int sin, int sout, int second) {
    if (second)
      cgs_df_kernel<K, false><<<grid, kVecThreads, 0, st>>>(V, ldv, n, tcol, part, cnt, small, sin, sout, 1);
    else
      cgs_df_kernel<K, true><<<grid, kVecThreads, 0, st>>>(V, ldv, n, tcol, part, cnt, small, sin, sout, 0);
  }
};

}  // namespace

// The padded tail (n rounded up to 2 by the FP64 kernels) is handled here element-wise;
// the zero padding of V, W and t stays zero.
dmrg_status launch_overlap_df(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                              const double* vec, double* s_out, DevSmall* small, int Bcol,
                              cudaStream_t st, const double* w0) {
  KDispatchDF<OverlapDF>::run(k, w.grid, st, V, ldv, n, vec, w0, w.partials, w.counter, s_out,
                              small, Bcol);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_residual_df(const VecWork& w, const double* V, const double* W,
                               const double* D, int64_t ldv, int64_t n, int k, double* tcol,
                               DevSmall* small, int mode, cudaStream_t st) {
  KDispatchDF<ResidualDF>::run(k, w.grid, st, V, W, D, ldv, n, tcol, w.partials, w.counter,
                               small, mode);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_cgs_df(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                          double* tcol, DevSmall* small, int sin, int sout, cudaStream_t st,
                          int second) {
  KDispatchDF<CgsDF>::run(k, w.grid, st, V, ldv, n, tcol, w.partials, w.counter, small, sin,
                          sout, second);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg
