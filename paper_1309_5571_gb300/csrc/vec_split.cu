// Davidson vector kernels for the mixed-precision solve with split arithmetic: basis
// column 0 in FP64, columns 1..k-1 stored and computed in FP32.
//
// In the mixed modes column 0 of the basis is the FP64 anchor (the collapsed Ritz vector
// x with its FP64-accurate projection W(:,0)); the other columns were projected in TF32 or
// BF16x3/BF16x2 and carry a relative error of 5e-6 or more.  Near convergence the iterate
// is x + sum_{j>=1} y_j v_j with |y_j| small, so only the terms of column 0 need float64:
//   * the residual W(:,0) - lambda x cancels to |r| << |W(:,0)|;
//   * the orthogonality of new columns to x enters the Rayleigh quotient multiplied by
//     lambda, and the coupling v_j . W(:,0) is small exactly because v_j is orthogonal
//     to x;
// while every term of a column j >= 1 is multiplied by y_j or by an already small
// correction, so FP32 rounding (2^-24 relative) stays far below the error the
// low-precision projection itself leaves in that column.  Columns j >= 1 of V and W are
// therefore also STORED in FP32 (rounded to nearest): the passes read 4 bytes per element
// of them instead of 8, and the projections of those columns read and write FP32 vectors.
// The column-0 terms run on the FP64 units (a few operations per element), the columns
// j >= 1 on the FP32 units (accumulated in FP32 per thread and warp, in FP64 across warps
// and blocks), so the passes are bound by HBM rather than by the FP64 units (about
// 0.55 T FMA/s on this part).  The new direction t is kept in an FP64 work vector through
// the residual, Gram-Schmidt and normalisation passes (its component along the anchor is
// removed in FP64) and rounded to FP32 when it is appended.  The anchor iteration itself
// (k = 1) and the final convergence test are entirely float64: with one column the FP64
// kernels of vec.cu run.
//
//   overlap:   B(j, c) = v_j . w; column 0 and the anchor coupling v_c . W(:,0) in FP64
//   residual:  r = y_0 (W(:,0) - lambda v_0) + sum_{j>=1} y_j (W(:,j) - lambda v_j);
//              t = r / (lambda - D) (mode 0) or r (mode 1); V^T t; ||r||^2, ||t||^2
//   cgs:       t -= s_0 v_0 + sum_{j>=1} s_j v_j; V^T t (first pass); ||t||^2
//   finish:    t -= (v_0 . t) v_0 in FP64 (see finish_split_kernel), t /= ||t||, and the
//              FP32 copy appended to the basis
//   ritz:      x = y_0 v_0 + sum_{j>=1} y_j v_j (the tail in FP32), optionally W y
#include <math.h>

#include <type_traits>

#include "internal.h"

namespace dmrg {
namespace {

#include "vec_common.cuh"

__device__ __forceinline__ float2 cvt2(double2 v) {
  return make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
}
__device__ __forceinline__ float2 ld2f(const float* p) {
  return __ldg(reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ float2 ld2fcg(const float* p) {
  return __ldcg(reinterpret_cast<const float2*>(p));
}

// ---------------------------------------------------------------- overlap
// w is an FP32 basis column (VEC32) or an FP64 vector (the work vector t, or W(:,0)).
// Anchored coupling (column Bcol = K-1 >= 1 against the FP64 anchor): the stored column
// v = v_{K-1} is the FP32 rounding of a direction made orthogonal to v_0 in FP64, so it
// keeps a component alpha = v_0 . v of about 2^-25 / sqrt(n) along v_0, random in sign.
// Entering the coupling as alpha * lambda, it would leave an error floor of that order in
// the Ritz vector; the coupling is therefore that of v - alpha v_0, orthogonal to first
// order:  B(0, K-1) = v . W(:,0) - alpha B(0,0)  (alpha and v . W(:,0) in FP64; the
// remaining terms are products of alpha with quantities that vanish at convergence).
template <int K, bool VEC32>
__global__ void __launch_bounds__(kVecThreads, 2)
overlap_split_kernel(const double* __restrict__ V0, const float* __restrict__ V32, int64_t ldv,
                     int64_t n2, const double* __restrict__ w64, const float* __restrict__ w32,
                     const double* __restrict__ w0, double* __restrict__ partials,
                     unsigned int* counter, double* s_out, DevSmall* small, int Bcol) {
  const bool anchored = w0 != nullptr && Bcol > 0;
  double a0 = 0.0, ac = 0.0, al = 0.0;  // v_0 . w, v_{K-1} . W(:,0), v_0 . v_{K-1}
  float acc32[K > 1 ? K - 1 : 1];
#pragma unroll
  for (int j = 0; j < K - 1; ++j) acc32[j] = 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v0 = ld2(V0 + 2 * e);
    float2 wf;
    double2 wv;
    if constexpr (VEC32) {
      wf = ld2fcg(w32 + 2 * e);
      wv = make_double2(f32_to_f64(wf.x), f32_to_f64(wf.y));
    } else {
      wv = ld2cg(w64 + 2 * e);
      wf = cvt2(wv);
    }
    a0 = fma(v0.x, wv.x, fma(v0.y, wv.y, a0));
    float2 vl = make_float2(0.0f, 0.0f);
    if constexpr (K > 1) {
      float2 v[K - 1];
#pragma unroll
      for (int j = 1; j < K; ++j) v[j - 1] = ld2f(V32 + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j)
        acc32[j - 1] = fmaf(v[j - 1].x, wf.x, fmaf(v[j - 1].y, wf.y, acc32[j - 1]));
      vl = v[K - 2];
    }
    if (anchored) {
      const double2 a = ld2(w0 + 2 * e);
      const double lx = f32_to_f64(vl.x), ly = f32_to_f64(vl.y);
      ac = fma(lx, a.x, fma(ly, a.y, ac));
      al = fma(lx, v0.x, fma(ly, v0.y, al));
    }
  }
  __shared__ double red[kVecThreads / 32][kSlots];
  SplitReduce sr{red, (int)(threadIdx.x & 31), (int)(threadIdx.x >> 5)};
  sr.f64(a0, 0);
#pragma unroll
  for (int j = 1; j < K; ++j) sr.f32(acc32[j - 1], j);
  sr.f64(ac, K);
  sr.f64(al, K + 1);
  sr.store(K + 2, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[K + 2];
    final_sums(partials, K + 2, tot);
    const double b00 = small->B[0];
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      if (s_out) s_out[j] = tot[j];
      if (Bcol >= 0) {
        double v = tot[j];
        if (anchored && j == 0) v = fma(-tot[K + 1], b00, tot[K]);
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
residual_split_kernel(const double* __restrict__ V0, const double* __restrict__ W0,
                      const float* __restrict__ V32, const float* __restrict__ W32,
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
    const double2 v0 = ld2(V0 + 2 * e);
    const double2 w0 = ld2(W0 + 2 * e);
    float2 vf[K > 1 ? K - 1 : 1];
    float l0 = 0.0f, l1 = 0.0f;
    if constexpr (K > 1) {
      float2 wf[K - 1];
#pragma unroll
      for (int j = 1; j < K; ++j) vf[j - 1] = ld2f(V32 + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) wf[j - 1] = ld2f(W32 + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) {
        l0 = fmaf(yf[j - 1], fmaf(-lamf, vf[j - 1].x, wf[j - 1].x), l0);
        l1 = fmaf(yf[j - 1], fmaf(-lamf, vf[j - 1].y, wf[j - 1].y), l1);
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
cgs_split_kernel(const double* __restrict__ V0, const float* __restrict__ V32, int64_t ldv,
                 int64_t n2, double* tcol, double* __restrict__ partials, unsigned int* counter,
                 DevSmall* small, int sin, int sout, int second) {
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
    const double2 v0 = ld2(V0 + 2 * e);
    double2 t = reinterpret_cast<const double2*>(tcol)[e];
    float2 vf[K > 1 ? K - 1 : 1];
    float l0 = 0.0f, l1 = 0.0f;
    if constexpr (K > 1) {
#pragma unroll
      for (int j = 1; j < K; ++j) vf[j - 1] = ld2f(V32 + j * ldv + 2 * e);
#pragma unroll
      for (int j = 1; j < K; ++j) {
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
//   t <- (t - s[1][0] v_0) / sqrt(||t||^2 - s[1][0]^2),
// and t, rounded to nearest FP32, is appended to the basis (out32).  (The rounding leaves
// a component along v_0 of about 2^-25 / sqrt(n) relative, random in sign.)
__global__ void finish_split_kernel(const double* __restrict__ v0, double* tcol, int64_t n2,
                                    DevSmall* small, float* __restrict__ out32) {
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
    reinterpret_cast<float2*>(out32)[e] = make_float2(f64_to_f32_rn(t.x), f64_to_f32_rn(t.y));
  }
}

// FP32 copy (rounded to nearest) of an FP64 vector of n2 pairs, unless a breakdown was
// flagged (the k = 1 passes of vec.cu normalise the work vector in FP64)
__global__ void store32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                               int64_t n2, const DevSmall* small) {
  if (small->flags & 1) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 t = reinterpret_cast<const double2*>(src)[e];
    reinterpret_cast<float2*>(dst)[e] = make_float2(f64_to_f32_rn(t.x), f64_to_f32_rn(t.y));
  }
}

// FP64 vector rounded to nearest FP32 (no flag test)
__global__ void convert32_kernel(const double* __restrict__ src, float* __restrict__ dst,
                                 int64_t n2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 t = reinterpret_cast<const double2*>(src)[e];
    reinterpret_cast<float2*>(dst)[e] = make_float2(f64_to_f32_rn(t.x), f64_to_f32_rn(t.y));
  }
}

// ---------------------------------------------------------------- Ritz vectors
// x = c0_0 v_0 + sum_{j>=1} c0_j v_j (and the same with the second coefficient vector c1 into
// p, and with W into wx, wp): column 0 in FP64, the tail summed in FP32 and added in FP64.
// Coefficients: small->y (x only, NC = 1 with y) or small->C[0], C[1] (two-vector restart).
template <int NC>
__global__ void __launch_bounds__(kVecThreads)
ritz_split_kernel(const double* __restrict__ V0, const double* __restrict__ W0,
                  const float* __restrict__ V32, const float* __restrict__ W32, int64_t ldv,
                  int64_t n2, int k, const DevSmall* small, int use_c, double* __restrict__ x,
                  double* __restrict__ wx, double* __restrict__ p, double* __restrict__ wp) {
  __shared__ double cs[NC][KMAX];
  for (int e = threadIdx.x; e < NC * KMAX; e += blockDim.x) {
    const int c = e / KMAX, j = e - (e / KMAX) * KMAX;
    cs[c][j] = j < k ? (use_c ? small->C[c][j] : small->y[j]) : 0.0;
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v0 = ld2(V0 + 2 * e);
    const double2 w0 = wx ? ld2(W0 + 2 * e) : make_double2(0.0, 0.0);
    float vx[NC], vy[NC], wxx[NC], wxy[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) vx[c] = vy[c] = wxx[c] = wxy[c] = 0.0f;
    for (int j = 1; j < k; ++j) {
      const float2 v = ld2f(V32 + j * ldv + 2 * e);
      const float2 w = wx ? ld2f(W32 + j * ldv + 2 * e) : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float cf = (float)cs[c][j];
        vx[c] = fmaf(cf, v.x, vx[c]);
        vy[c] = fmaf(cf, v.y, vy[c]);
        wxx[c] = fmaf(cf, w.x, wxx[c]);
        wxy[c] = fmaf(cf, w.y, wxy[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double* xo = c == 0 ? x : p;
      double* wo = c == 0 ? wx : wp;
      const double a = cs[c][0];
      reinterpret_cast<double2*>(xo)[e] =
          make_double2(fma(a, v0.x, f32_to_f64(vx[c])), fma(a, v0.y, f32_to_f64(vy[c])));
      if (wx)
        reinterpret_cast<double2*>(wo)[e] =
            make_double2(fma(a, w0.x, f32_to_f64(wxx[c])), fma(a, w0.y, f32_to_f64(wxy[c])));
    }
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

dmrg_status launch_overlap_split(const VecWork& w, const double* V0, const float* V32, int64_t ldv,
                                 int64_t n, int k, const double* vec64, const float* vec32,
                                 double* s_out, DevSmall* small, int Bcol, cudaStream_t st,
                                 const double* w0) {
  if (k == 1 && !vec32) return launch_overlap(w, V0, ldv, n, k, vec64, s_out, small, Bcol, st, w0);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<1>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    if (vec32)
      overlap_split_kernel<K, true><<<split_grid(w), kVecThreads, 0, st>>>(
          V0, V32, ldv, n2, nullptr, vec32, w0, w.partials, w.counter, s_out, small, Bcol);
    else
      overlap_split_kernel<K, false><<<split_grid(w), kVecThreads, 0, st>>>(
          V0, V32, ldv, n2, vec64, nullptr, w0, w.partials, w.counter, s_out, small, Bcol);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_residual_split(const VecWork& w, const double* V0, const double* W0,
                                  const float* V32, const float* W32, const double* D,
                                  int64_t ldv, int64_t n, int k, double* tcol, DevSmall* small,
                                  int mode, cudaStream_t st) {
  if (k == 1) return launch_residual(w, V0, W0, D, ldv, n, k, tcol, small, mode, st);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<2>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    residual_split_kernel<K><<<split_grid(w), kVecThreads, 0, st>>>(V0, W0, V32, W32, D, ldv, n2, tcol,
                                                                   w.partials, w.counter, small, mode);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_cgs_split(const VecWork& w, const double* V0, const float* V32, int64_t ldv,
                             int64_t n, int k, double* tcol, DevSmall* small, int sin, int sout,
                             cudaStream_t st, int second) {
  if (k == 1) return launch_cgs(w, V0, ldv, n, k, tcol, small, sin, sout, st, second);
  const int64_t n2 = (n + 1) / 2;
  Dispatch<2>::run(k, [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    if (second)
      cgs_split_kernel<K, false><<<split_grid(w), kVecThreads, 0, st>>>(V0, V32, ldv, n2, tcol, w.partials,
                                                                       w.counter, small, sin, sout, 1);
    else
      cgs_split_kernel<K, true><<<split_grid(w), kVecThreads, 0, st>>>(V0, V32, ldv, n2, tcol, w.partials,
                                                                      w.counter, small, sin, sout, 0);
  });
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_finish_split(const VecWork& w, const double* V0, double* tcol, int64_t n,
                                int k, DevSmall* small, float* out32, cudaStream_t st) {
  const int64_t n2 = (n + 1) / 2;
  if (k == 1) {
    DMRG_TRY(launch_finish(tcol, n, small, st));
    store32_kernel<<<split_grid(w), kVecThreads, 0, st>>>(tcol, out32, n2, small);
  } else {
    finish_split_kernel<<<split_grid(w), kVecThreads, 0, st>>>(V0, tcol, n2, small, out32);
  }
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_convert32(const VecWork& w, const double* src, float* dst, int64_t n,
                             cudaStream_t st) {
  convert32_kernel<<<split_grid(w), kVecThreads, 0, st>>>(src, dst, (n + 1) / 2);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_ritz_split(const VecWork& w, const double* V0, const double* W0,
                              const float* V32, const float* W32, int64_t ldv, int64_t n, int k,
                              const DevSmall* small, double* x, double* wx, cudaStream_t st) {
  ritz_split_kernel<1><<<split_grid(w), kVecThreads, 0, st>>>(V0, W0, V32, W32, ldv, (n + 1) / 2, k,
                                                             small, 0, x, wx, nullptr, nullptr);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_ritz2_split(const VecWork& w, const double* V0, const double* W0,
                               const float* V32, const float* W32, int64_t ldv, int64_t n, int k,
                               const DevSmall* small, double* x, double* p, double* wx,
                               double* wp, cudaStream_t st) {
  ritz_split_kernel<2><<<split_grid(w), kVecThreads, 0, st>>>(V0, W0, V32, W32, ldv, (n + 1) / 2, k,
                                                             small, 1, x, wx, p, wp);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg
