// Davidson vector kernels for the mixed-precision solve with split arithmetic: basis
// column 0 in FP64, columns 1..k-1 in FP32.
//
// In the mixed modes column 0 of the basis is the FP64 anchor (the collapsed Ritz vector
// x with its FP64-accurate projection W(:,0)); the other columns were projected in TF32 or
// BF16x3 and carry a relative error of 5e-6 or more.  Near convergence the iterate is
// x + sum_{j>=1} y_j v_j with |y_j| small, so only the terms of column 0 need float64:
//   * the residual W(:,0) - lambda x cancels to |r| << |W(:,0)|;
//   * the orthogonality of new columns to x enters the Rayleigh quotient multiplied by
//     lambda, and the coupling v_j . W(:,0) is small exactly because v_j is orthogonal
//     to x;
// while every term of a column j >= 1 is multiplied by y_j or by an already small
// correction, so the FP32 rounding (2^-24 relative) stays far below the error the
// low-precision projection itself leaves in that column.  The column-0 terms therefore
// run on the FP64 units (a few operations per element), the columns j >= 1 on the FP32
// units (loaded as float64, converted with integer operations, accumulated in FP32 per
// thread and warp, in FP64 across warps and blocks).  The passes are then bound by HBM
// rather than by the FP64 units (about 0.55 T FMA/s on this part); hardware FP64<->FP32
// conversions would run on the FP64 units too.  The anchor iteration itself (k = 1)
// and the final convergence test are entirely float64: with one column (k = 1) the FP64
// kernels of vec.cu run.
//
//   overlap:   B(j, c) = v_j . W(:,c); column 0 and the anchor coupling v_c . W(:,0) in FP64
//   residual:  r = y_0 (W(:,0) - lambda v_0) + sum_{j>=1} y_j (W(:,j) - lambda v_j);
//              t = r / (lambda - D) (mode 0) or r (mode 1); V^T t; ||r||^2, ||t||^2
//   cgs:       t -= s_0 v_0 + sum_{j>=1} s_j v_j; V^T t (first pass); ||t||^2
//   finish:    t -= (v_0 . t) v_0 in FP64 (see finish_split_kernel), t /= ||t||
#include <math.h>

#include <type_traits>

#include "internal.h"

namespace dmrg {
namespace {

#include "vec_common.cuh"

__device__ __forceinline__ float2 cvt2(double2 v) {
  return make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
}

// ---------------------------------------------------------------- overlap
template <int K>
__global__ void __launch_bounds__(kVecThreads, 2)
overlap_split_kernel(const double* __restrict__ V, int64_t ldv, int64_t n2,
                     const double* __restrict__ w, const double* __restrict__ w0,
                     double* __restrict__ partials, unsigned int* counter, double* s_out,
                     DevSmall* small, int Bcol) {
  const bool anchored = w0 != nullptr && Bcol > 0;
  double a0 = 0.0, ac = 0.0;  // v_0 . w, v_{K-1} . W(:,0)
  float acc32[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 0; j < K - 1; ++j) acc32[j] = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 wv = ld2cg(w + 2 * e);
    const double2 v0 = ld2(V + 2 * e);
    double2 vl = v0;
    a0 = fma(v0.x, wv.x, fma(v0.y, wv.y, a0));
    if constexpr (K > 1) {
      double2 v[K - 1];
#pragma unroll
      for (int j = 1; j < K; ++j) v[j - 1] = ld2(V + j * ldv + 2 * e);
      const float2 wf = cvt2(wv);
#pragma unroll
      for (int j = 1; j < K; ++j) {
        const float2 vf = cvt2(v[j - 1]);
        acc32[j - 1] = fmaf(vf.x, wf.x, fmaf(vf.y, wf.y, acc32[j - 1]));
      }
      vl = v[K - 2];
    }
    if (anchored) {
      const double2 a = ld2(w0 + 2 * e);
      ac = fma(vl.x, a.x, fma(vl.y, a.y, ac));
    }
  }
  __shared__ double red[kVecThreads / 32][kSlots];
  SplitReduce sr{red, (int)(threadIdx.x & 31), (int)(threadIdx.x >> 5)};
  sr.f64(a0, 0);
#pragma unroll
  for (int j = 1; j < K; ++j) sr.f32(acc32[j - 1], j);
  sr.f64(ac, K);
  sr.store(K + 1, partials);
  if (Ticket::last_block(counter)) {
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
residual_split_kernel(const double* __restrict__ V, const double* __restrict__ W,
                      const double* __restrict__ D, int64_t ldv, int64_t n2,
                      double* __restrict__ tcol, double* __restrict__ partials,
                      unsigned int* counter, DevSmall* small, int mode) {
  __shared__ double ys[K];
  __shared__ double lam_s;
  if (threadIdx.x < K) ys[threadIdx.x] = small->y[threadIdx.x];
  if (threadIdx.x == 0) lam_s = small->lambda;
  __syncthreads();
  const double lam = lam_s, y0 = ys[0];
  const float lamf = f64_to_f32(lam);
  float yf[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 1; j < K; ++j) yf[j - 1] = f64_to_f32(ys[j]);
  double d0 = 0.0;              // v_0 . t
  float acc32[K > 1 ? K - 1 : 1];  // v_j . t, j >= 1
  float rr = 0.0f, tt = 0.0f;   // ||r||^2, ||t||^2
#pragma unroll
  for (int j = 0; j < K - 1; ++j) acc32[j] = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v0 = ld2(V + 2 * e);
    const double2 w0 = ld2(W + 2 * e);
    float2 vf[K > 1 ? K - 1 : 1];
    float l0 = 0.0f, l1 = 0.0f;
    if constexpr (K > 1) {
      double2 v[K - 1], wv[K - 1];
#pragma unroll
      for (int j = 1; j < K; ++j) v[j - 1] = ld2(V + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) wv[j - 1] = ld2(W + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) {
        vf[j - 1] = cvt2(v[j - 1]);
        const float2 wf = cvt2(wv[j - 1]);
        l0 = fmaf(yf[j - 1], fmaf(-lamf, vf[j - 1].x, wf.x), l0);
        l1 = fmaf(yf[j - 1], fmaf(-lamf, vf[j - 1].y, wf.y), l1);
      }
    }
    const double r0 = fma(y0, fma(-lam, v0.x, w0.x), f32_to_f64(l0));
    const double r1 = fma(y0, fma(-lam, v0.y, w0.y), f32_to_f64(l1));
    double t0 = r0, t1 = r1;
    if (mode == 0) {
      const double2 d = ld2(D + 2 * e);
      float q0 = f64_to_f32(lam - d.x), q1 = f64_to_f32(lam - d.y);
      if (fabsf(q0) < 1e-8f) q0 = q0 >= 0.0f ? 1e-8f : -1e-8f;
      if (fabsf(q1) < 1e-8f) q1 = q1 >= 0.0f ? 1e-8f : -1e-8f;
      t0 = r0 * f32_to_f64(1.0f / q0);
      t1 = r1 * f32_to_f64(1.0f / q1);
    }
    reinterpret_cast<double2*>(tcol)[e] = make_double2(t0, t1);
    d0 = fma(v0.x, t0, fma(v0.y, t1, d0));
    const float rf0 = f64_to_f32(r0), rf1 = f64_to_f32(r1);
    const float tf0 = f64_to_f32(t0), tf1 = f64_to_f32(t1);
    rr = fmaf(rf0, rf0, fmaf(rf1, rf1, rr));
    tt = fmaf(tf0, tf0, fmaf(tf1, tf1, tt));
#pragma unroll
    for (int j = 0; j < K - 1; ++j) acc32[j] = fmaf(vf[j].x, tf0, fmaf(vf[j].y, tf1, acc32[j]));
  }
  // slots [0..K): V^T t, [K]: ||r||^2, [K+1]: ||t||^2
  __shared__ double red[kVecThreads / 32][kSlots];
  SplitReduce sr{red, (int)(threadIdx.x & 31), (int)(threadIdx.x >> 5)};
  sr.f64(d0, 0);
#pragma unroll
  for (int j = 1; j < K; ++j) sr.f32(acc32[j - 1], j);
  sr.f32(rr, K);
  sr.f32(tt, K + 1);
  sr.store(K + 2, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[K + 2];
    final_sums(partials, K + 2, tot);
    for (int j = threadIdx.x; j < K; j += blockDim.x) small->s[0][j] = tot[j];
    if (threadIdx.x == 0) {
      small->rnorm2 = tot[K];
      small->tnorm2_before = tot[K + 1];
      small->tnorm2 = tot[K + 1];
      if (!isfinite(tot[K]) || !isfinite(tot[K + 1])) atomicOr(&small->flags, 2);
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- Gram-Schmidt pass
// Same protocol as the FP64 pass: the second pass (second = 1) runs only when the first
// removed more than half of ||t||^2.
template <int K, bool DOT>
__global__ void __launch_bounds__(kVecThreads, 2)
cgs_split_kernel(const double* __restrict__ V, int64_t ldv, int64_t n2, double* tcol,
                 double* __restrict__ partials, unsigned int* counter, DevSmall* small,
                 int sin, int sout, int second) {
  if (second && small->tnorm2 >= 0.5 * small->tnorm2_before) return;
  if (second && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&small->flags, 4);
  __shared__ double ss[K];
  if (threadIdx.x < K) ss[threadIdx.x] = small->s[sin][threadIdx.x];
  __syncthreads();
  const double s0 = ss[0];
  float sf[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 1; j < K; ++j) sf[j - 1] = f64_to_f32(ss[j]);
  double d0 = 0.0;
  float acc32[K > 1 ? K - 1 : 1];
  float tt = 0.0f;
#pragma unroll
  for (int j = 0; j < K - 1; ++j) acc32[j] = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v0 = ld2(V + 2 * e);
    double2 t = reinterpret_cast<const double2*>(tcol)[e];
    float2 vf[K > 1 ? K - 1 : 1];
    float l0 = 0.0f, l1 = 0.0f;
    if constexpr (K > 1) {
      double2 v[K - 1];
#pragma unroll
      for (int j = 1; j < K; ++j) v[j - 1] = ld2(V + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) {
        vf[j - 1] = cvt2(v[j - 1]);
        l0 = fmaf(sf[j - 1], vf[j - 1].x, l0);
        l1 = fmaf(sf[j - 1], vf[j - 1].y, l1);
      }
    }
    t.x = fma(-s0, v0.x, t.x) - f32_to_f64(l0);
    t.y = fma(-s0, v0.y, t.y) - f32_to_f64(l1);
    reinterpret_cast<double2*>(tcol)[e] = t;
    const float tf0 = f64_to_f32(t.x), tf1 = f64_to_f32(t.y);
    tt = fmaf(tf0, tf0, fmaf(tf1, tf1, tt));
    if (DOT) {
      d0 = fma(v0.x, t.x, fma(v0.y, t.y, d0));
#pragma unroll
      for (int j = 0; j < K - 1; ++j) acc32[j] = fmaf(vf[j].x, tf0, fmaf(vf[j].y, tf1, acc32[j]));
    }
  }
  __shared__ double red[kVecThreads / 32][kSlots];
  SplitReduce sr{red, (int)(threadIdx.x & 31), (int)(threadIdx.x >> 5)};
  if (DOT) {
    sr.f64(d0, 0);
#pragma unroll
    for (int j = 1; j < K; ++j) sr.f32(acc32[j - 1], j);
    sr.f32(tt, K);
    sr.store(K + 1, partials);
  } else {
    sr.f32(tt, 0);
    sr.store(1, partials);
  }
  if (Ticket::last_block(counter)) {
    __shared__ double tot[K + 1];
    const int nv = DOT ? K + 1 : 1;
    final_sums(partials, nv, tot);
    if (DOT)
      for (int j = threadIdx.x; j < K; j += blockDim.x) small->s[sout][j] = tot[j];
    if (threadIdx.x == 0) {
      const double nrm = tot[nv - 1];
      small->tnorm2 = nrm;
      if (!isfinite(nrm)) atomicOr(&small->flags, 2);
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- normalise new column
// The FP32 rounding of the low-precision part of t -= V s leaves a component of t along
// the anchor v_0 of about 1e-9 relative, far above FP64 orthogonality; it would enter the
// anchor coupling v_j . W(:,0) multiplied by lambda.  The first Gram-Schmidt pass measured
// it in FP64 (s[1][0] = v_0 . t); unless the second pass already removed it (flag bit 2),
// it is removed here, in FP64, together with the normalisation:
//   t <- (t - s[1][0] v_0) / sqrt(||t||^2 - s[1][0]^2).
__global__ void finish_split_kernel(const double* __restrict__ v0, double* tcol, int64_t n2,
                                    DevSmall* small) {
  const double before = small->tnorm2_before;
  const double c0 = (small->flags & 4) ? 0.0 : small->s[1][0];
  const double after = small->tnorm2 - c0 * c0;
  const bool breakdown = !(after > 1e-20 * before) || !(after > 0.0);
  if (breakdown) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&small->flags, 1);
    return;
  }
  const double inv = 1.0 / sqrt(after);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 t = reinterpret_cast<double2*>(tcol)[e];
    const double2 v = ld2(v0 + 2 * e);
    t.x = fma(-c0, v.x, t.x) * inv;
    t.y = fma(-c0, v.y, t.y) * inv;
    reinterpret_cast<double2*>(tcol)[e] = t;
  }
}

template <int K>
struct Dispatch {
  template <typename F>
  static void run(int k, F&& f) {
    if (k == K) f(std::integral_constant<int, K>{});
    else Dispatch<K + 1>::run(k, f);
  }
};
template <>
struct Dispatch<KMAX + 1> {
  template <typename F>
  static void run(int, F&&) {}
};

// one wave: two resident blocks per SM (the kernels are limited to 128 registers)
int split_grid(const VecWork& w) { return w.grid / kGridPerSM * 2; }

}  // namespace

dmrg_status launch_overlap_split(const VecWork& w, const double* V, int64_t ldv, int64_t n,
                                 int k, const double* vec, double* s_out, DevSmall* small,
                                 int Bcol, cudaStream_t st, const double* w0) {
  if (k == 1) return launch_overlap(w, V, ldv, n, k, vec, s_out, small, Bcol, st, w0);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<2>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    overlap_split_kernel<K><<<split_grid(w), kVecThreads, 0, st>>>(V, ldv, n2, vec, w0, w.partials,
                                                            w.counter, s_out, small, Bcol);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_residual_split(const VecWork& w, const double* V, const double* W,
                                  const double* D, int64_t ldv, int64_t n, int k, double* tcol,
                                  DevSmall* small, int mode, cudaStream_t st) {
  if (k == 1) return launch_residual(w, V, W, D, ldv, n, k, tcol, small, mode, st);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<2>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    residual_split_kernel<K><<<split_grid(w), kVecThreads, 0, st>>>(V, W, D, ldv, n2, tcol, w.partials,
                                                             w.counter, small, mode);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_cgs_split(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                             double* tcol, DevSmall* small, int sin, int sout, cudaStream_t st,
                             int second) {
  if (k == 1) return launch_cgs(w, V, ldv, n, k, tcol, small, sin, sout, st, second);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<2>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    if (second)
      cgs_split_kernel<K, false><<<split_grid(w), kVecThreads, 0, st>>>(V, ldv, n2, tcol, w.partials,
                                                                 w.counter, small, sin, sout, 1);
    else
      cgs_split_kernel<K, true><<<split_grid(w), kVecThreads, 0, st>>>(V, ldv, n2, tcol, w.partials,
                                                                w.counter, small, sin, sout, 0);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_finish_split(const VecWork& w, const double* V, double* tcol, int64_t n,
                                int k, DevSmall* small, cudaStream_t st) {
  if (k == 1) return launch_finish(tcol, n, small, st);
  finish_split_kernel<<<split_grid(w), kVecThreads, 0, st>>>(V, tcol, (n + 1) / 2, small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg
