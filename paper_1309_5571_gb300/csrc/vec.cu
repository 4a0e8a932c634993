// Davidson vector kernels (Algorithm 3, all lines except the projection) and the small
// projected eigenproblem.
//
// Every kernel streams the tall-skinny basis V (and W) once, column-major with columns
// contiguous (leading dimension ldv, a multiple of 32 elements, zero padding beyond n),
// reading 16-byte double2 pairs so a warp touches 512 contiguous bytes per column.  The
// paper's gemv_trans kernel (Sec. 6.1, Algorithm 4) gives each thread a row and keeps
// a belt of column sums in registers, then reduces across the block; here a thread also
// keeps all k <= 24 column sums in registers, the block reduces with warp shuffles, and
// the cross-block reduction is a deterministic one-pass scheme: every block writes its
// partial sums, and the last block to finish (atomic ticket) adds them in block order.
// Several Algorithm 3 lines are fused so each pass over V does as much as possible:
//   residual:  x = V y, W y, r = W y - lambda x, t = r / (lambda - D),  ||r||^2,
//              V^T t and ||t||^2                                 (lines 5, 6, 9, 11)
//   cgs:       t -= V s, then V^T t and ||t||^2                     (lines 12, 11)
//   finish:    normalise t                                           (line 13)
#include <math.h>

#include "internal.h"

namespace dmrg {
namespace {

#include "vec_common.cuh"

// ---------------------------------------------------------------- overlap  s = V^T w
// With w0 != NULL (mixed precision with an FP64 anchor in column 0) the coupling between
// the anchor and column Bcol is taken from the exact anchor projection, v_Bcol . W(:,0),
// instead of v_0 . W(:,Bcol), whose low-precision error would not shrink with the
// correction.  K (the number of basis columns) is a compile-time constant in all the
// kernels below, so loads are issued back to back and accumulators stay in registers.
template <int K>
__global__ void __launch_bounds__(kVecThreads)
overlap_kernel(const double* __restrict__ V, int64_t ldv, int64_t n2,
               const double* __restrict__ w, const double* __restrict__ w0,
               double* __restrict__ partials, unsigned int* counter, double* s_out,
               DevSmall* small, int Bcol) {
  double acc[K + 1];
#pragma unroll
  for (int j = 0; j < K + 1; ++j) acc[j] = 0.0;
  const bool anchored = w0 != nullptr && Bcol > 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = ld2(V + j * ldv + 2 * e);
    const double2 wv = ld2cg(w + 2 * e);
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fma(v[j].x, wv.x, fma(v[j].y, wv.y, acc[j]));
    if (anchored) {
      const double2 a = ld2(w0 + 2 * e);
      acc[K] = fma(v[K - 1].x, a.x, fma(v[K - 1].y, a.y, acc[K]));
    }
  }
  block_partials<K, 1>(acc, K, partials);
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

// Public variant of the overlap for caller-owned V (any ldv, any alignment): scalar loads.
__global__ void __launch_bounds__(kVecThreads)
gemv_trans_kernel(const double* __restrict__ V, int64_t ldv, int64_t n, int k,
                  const double* __restrict__ w, double* __restrict__ partials,
                  unsigned int* counter, double* s_out) {
  double acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) acc[j] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double wv = __ldg(w + e);
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) acc[j] = fma(__ldg(V + j * ldv + e), wv, acc[j]);
  }
  block_partials<KMAX, 0>(acc, k, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[KMAX];
    final_sums(partials, k, tot);
    for (int j = threadIdx.x; j < k; j += blockDim.x) s_out[j] = tot[j];
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// ---------------------------------------------------------------- residual + correction
// r = W y - lambda V y and its norm; t = r / (lambda - D) (mode 0, the diagonal
// correction) or t = r (mode 1); V^T t and ||t||^2.  The preconditioner is a direction,
// not a value that must be exact: its reciprocal is formed in FP32 (an FP64 division costs
// as much as a dozen FP64 operations on this part), the product r * (1/(lambda - D)) in
// FP64.
template <int K>
__global__ void __launch_bounds__(kVecThreads)
residual_kernel(const double* __restrict__ V, const double* __restrict__ W,
                const double* __restrict__ D, int64_t ldv, int64_t n2,
                double* __restrict__ tcol, double* __restrict__ partials,
                unsigned int* counter, DevSmall* small, int mode) {
  __shared__ double ys[K];
  __shared__ double lam_s;
  if (threadIdx.x < K) ys[threadIdx.x] = small->y[threadIdx.x];
  if (threadIdx.x == 0) lam_s = small->lambda;
  __syncthreads();
  const double lam = lam_s;
  double y[K];
#pragma unroll
  for (int j = 0; j < K; ++j) y[j] = ys[j];
  double acc[K + 2];  // [0..K): V^T t, [K]: ||r||^2, [K+1]: ||t||^2
#pragma unroll
  for (int j = 0; j < K + 2; ++j) acc[j] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 v[K];
    double x0 = 0.0, x1 = 0.0, w0 = 0.0, w1 = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = ld2(V + j * ldv + 2 * e);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double2 wv = ld2(W + j * ldv + 2 * e);
      x0 = fma(y[j], v[j].x, x0);
      x1 = fma(y[j], v[j].y, x1);
      w0 = fma(y[j], wv.x, w0);
      w1 = fma(y[j], wv.y, w1);
    }
    const double r0 = fma(-lam, x0, w0), r1 = fma(-lam, x1, w1);
    double t0 = r0, t1 = r1;
    if (mode == 0) {
      const double2 d = ld2(D + 2 * e);
      float q0 = (float)(lam - d.x), q1 = (float)(lam - d.y);
      if (fabsf(q0) < 1e-8f) q0 = q0 >= 0.0f ? 1e-8f : -1e-8f;
      if (fabsf(q1) < 1e-8f) q1 = q1 >= 0.0f ? 1e-8f : -1e-8f;
      t0 = r0 * (double)(1.0f / q0);
      t1 = r1 * (double)(1.0f / q1);
    }
    reinterpret_cast<double2*>(tcol)[e] = make_double2(t0, t1);
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fma(v[j].x, t0, fma(v[j].y, t1, acc[j]));
    acc[K] = fma(r0, r0, fma(r1, r1, acc[K]));
    acc[K + 1] = fma(t0, t0, fma(t1, t1, acc[K + 1]));
  }
  block_partials<K, 2>(acc, K, partials);
  if (Ticket::last_block(counter)) {
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
// t -= V s[sin]; with DOT also s[sout] = V^T t; always ||t||^2.  A second pass
// (second = 1) runs only when the first removed more than half of ||t||^2 -- the
// "twice is enough" test -- and otherwise returns at once; the decision is read from the
// device, so the host launches both passes without waiting.
template <int K, bool DOT>
__global__ void __launch_bounds__(kVecThreads)
cgs_kernel(const double* __restrict__ V, int64_t ldv, int64_t n2, double* tcol,
           double* __restrict__ partials, unsigned int* counter, DevSmall* small, int sin,
           int sout, int second) {
  if (second && small->tnorm2 >= 0.5 * small->tnorm2_before) return;
  if (second && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&small->flags, 4);  // pass 2 ran
  __shared__ double ss[K];
  if (threadIdx.x < K) ss[threadIdx.x] = small->s[sin][threadIdx.x];
  __syncthreads();
  double s[K];
#pragma unroll
  for (int j = 0; j < K; ++j) s[j] = ss[j];
  double acc[K + 1];
#pragma unroll
  for (int j = 0; j < K + 1; ++j) acc[j] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = ld2(V + j * ldv + 2 * e);
    double2 t = reinterpret_cast<const double2*>(tcol)[e];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      t.x = fma(-s[j], v[j].x, t.x);
      t.y = fma(-s[j], v[j].y, t.y);
    }
    reinterpret_cast<double2*>(tcol)[e] = t;
    if (DOT) {
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] = fma(v[j].x, t.x, fma(v[j].y, t.y, acc[j]));
    }
    acc[K] = fma(t.x, t.x, fma(t.y, t.y, acc[K]));
  }
  if (DOT) {
    block_partials<K, 1>(acc, K, partials);
  } else {
    double a1[1] = {acc[K]};
    block_partials<0, 1>(a1, 0, partials);
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

// compile-time dispatch over K = 1 .. KMAX
template <template <int> class F, int K = 1>
struct KDispatch {
  template <typename... A>
  static void run(int k, A... a) {
    if (k == K) F<K>::go(a...);
    else KDispatch<F, K + 1>::run(k, a...);
  }
};
template <template <int> class F>
struct KDispatch<F, KMAX + 1> {
  template <typename... A>
  static void run(int, A...) {}
};

template <int K>
struct OverlapL {
  static void go(int grid, cudaStream_t st, const double* V, int64_t ldv, int64_t n2,
                 const double* w, const double* w0, double* part, unsigned int* cnt,
                 double* s_out, DevSmall* small, int Bcol) {
    overlap_kernel<K><<<grid, kVecThreads, 0, st>>>(V, ldv, n2, w, w0, part, cnt, s_out, small, Bcol);
  }
};
template <int K>
struct ResidualL {
  static void go(int grid, cudaStream_t st, const double* V, const double* W, const double* D,
                 int64_t ldv, int64_t n2, double* tcol, double* part, unsigned int* cnt,
                 DevSmall* small, int mode) {
    residual_kernel<K><<<grid, kVecThreads, 0, st>>>(V, W, D, ldv, n2, tcol, part, cnt, small, mode);
  }
};
template <int K>
struct CgsL {
  static void go(int grid, cudaStream_t st, const double* V, int64_t ldv, int64_t n2,
                 double* tcol, double* part, unsigned int* cnt, DevSmall* small, int sin,
                 int sout, int second) {
    if (second)
      cgs_kernel<K, false><<<grid, kVecThreads, 0, st>>>(V, ldv, n2, tcol, part, cnt, small, sin, sout, 1);
    else
      cgs_kernel<K, true><<<grid, kVecThreads, 0, st>>>(V, ldv, n2, tcol, part, cnt, small, sin, sout, 0);
  }
};

// ---------------------------------------------------------------- normalise new column
__global__ void finish_kernel(double* tcol, int64_t n2, DevSmall* small) {
  const double before = small->tnorm2_before, after = small->tnorm2;
  const bool breakdown = !(after > 1e-20 * before) || !(after > 0.0);
  if (breakdown) {
    if (blockIdx.x == 0 && threadIdx.x == 0) small->flags |= 1;
    return;
  }
  const double inv = 1.0 / sqrt(after);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 t = reinterpret_cast<double2*>(tcol)[e];
    t.x *= inv;
    t.y *= inv;
    reinterpret_cast<double2*>(tcol)[e] = t;
  }
}

// ---------------------------------------------------------------- Ritz vector
__global__ void ritz_kernel(const double* __restrict__ V, const double* __restrict__ W,
                            int64_t ldv, int64_t n, int k, const DevSmall* small,
                            double* __restrict__ x_out, double* __restrict__ wy_out) {
  __shared__ double ys[KMAX];
  if (threadIdx.x < KMAX) ys[threadIdx.x] = threadIdx.x < k ? small->y[threadIdx.x] : 0.0;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double x = 0.0, wy = 0.0;
    for (int j = 0; j < k; ++j) {
      x = fma(ys[j], V[j * ldv + e], x);
      if (wy_out) wy = fma(ys[j], W[j * ldv + e], wy);
    }
    x_out[e] = x;
    if (wy_out) wy_out[e] = wy;
  }
}

// ---------------------------------------------------------------- two-vector restart
__global__ void ritz2_kernel(const double* __restrict__ V, const double* __restrict__ W,
                             int64_t ldv, int64_t n, int k, const DevSmall* small,
                             double* __restrict__ x, double* __restrict__ p,
                             double* __restrict__ wx, double* __restrict__ wp) {
  __shared__ double c0[KMAX], c1[KMAX];
  if (threadIdx.x < KMAX) {
    c0[threadIdx.x] = threadIdx.x < k ? small->C[0][threadIdx.x] : 0.0;
    c1[threadIdx.x] = threadIdx.x < k ? small->C[1][threadIdx.x] : 0.0;
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int j = 0; j < k; ++j) {
      const double v = V[j * ldv + e], w = W[j * ldv + e];
      a = fma(c0[j], v, a);
      b = fma(c1[j], v, b);
      c = fma(c0[j], w, c);
      d = fma(c1[j], w, d);
    }
    x[e] = a;
    p[e] = b;
    wx[e] = c;
    wp[e] = d;
  }
}

__global__ void axpy_pair_kernel(double* __restrict__ p, double* __restrict__ wp,
                                 const double* __restrict__ x, const double* __restrict__ wx,
                                 int64_t n, const DevSmall* small) {
  const double a = small->s[2][0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    p[e] = fma(-a, x[e], p[e]);
    wp[e] = fma(-a, wx[e], wp[e]);
  }
}

__global__ void scale_pair_kernel(double* __restrict__ p, double* __restrict__ wp, int64_t n,
                                  const DevSmall* small) {
  const double inv = 1.0 / sqrt(small->nrm2);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    p[e] *= inv;
    wp[e] *= inv;
  }
}

// ---------------------------------------------------------------- normalise a vector
__global__ void __launch_bounds__(kVecThreads)
sumsq_kernel(const double* __restrict__ src, int64_t n, double* __restrict__ partials,
             unsigned int* counter, DevSmall* small) {
  double acc[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(src[e], src[e], acc[0]);
  block_partials<0, 1>(acc, 0, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      small->nrm2 = tot[0];
      *counter = 0u;
    }
  }
}

__global__ void scale_copy_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                  int64_t n, const DevSmall* small) {
  const double inv = 1.0 / sqrt(small->nrm2);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * inv;
}

__global__ void axpby_kernel(const double* __restrict__ a, double c, const double* __restrict__ b,
                             double* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = fma(c, b[e], a[e]);
}

__global__ void set_B00_kernel(DevSmall* small) {
  // after a restart the basis is the single Ritz vector x with B = [lambda] = 1 x 1
  for (int j = threadIdx.x; j < KMAX * KMAX; j += blockDim.x) small->B[j] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    small->B[0] = small->lambda;
    small->Q[0] = 1.0;
    small->theta[0] = small->lambda;
    small->qk = 1;
  }
}

}  // namespace

static int vec_grid() {
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = std::max(1, sms) * kGridPerSM;
  }
  return grid;
}

dmrg_status vec_work_create(VecWork* w) {
  w->grid = vec_grid();
  DMRG_CUDA_TRY(cudaMalloc((void**)&w->partials, sizeof(double) * (size_t)w->grid * kSlots));
  DMRG_CUDA_TRY(cudaMalloc((void**)&w->counter, sizeof(unsigned int) * 16));
  DMRG_CUDA_TRY(cudaMemset(w->counter, 0, sizeof(unsigned int) * 16));
  return DMRG_OK;
}

void vec_work_destroy(VecWork* w) {
  cudaFree(w->partials);
  cudaFree(w->counter);
  w->partials = nullptr;
  w->counter = nullptr;
}

dmrg_status launch_overlap(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                           const double* vec, double* s_out, DevSmall* small, int Bcol,
                           cudaStream_t st, const double* w0) {
  KDispatch<OverlapL>::run(k, w.grid, st, V, ldv, (int64_t)((n + 1) / 2), vec, w0, w.partials,
                           w.counter, s_out, small, Bcol);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_residual(const VecWork& w, const double* V, const double* W,
                            const double* D, int64_t ldv, int64_t n, int k, double* tcol,
                            DevSmall* small, int mode, cudaStream_t st) {
  KDispatch<ResidualL>::run(k, w.grid, st, V, W, D, ldv, (int64_t)((n + 1) / 2), tcol,
                            w.partials, w.counter, small, mode);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_cgs(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                       double* tcol, DevSmall* small, int sin, int sout, cudaStream_t st,
                       int second) {
  KDispatch<CgsL>::run(k, w.grid, st, V, ldv, (int64_t)((n + 1) / 2), tcol, w.partials,
                       w.counter, small, sin, sout, second);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_finish(double* tcol, int64_t n, DevSmall* small, cudaStream_t st) {
  finish_kernel<<<vec_grid(), kVecThreads, 0, st>>>(tcol, (n + 1) / 2, small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_ritz(const double* V, const double* W, int64_t ldv, int64_t n, int k,
                        const DevSmall* small, double* x_out, double* wy_out, cudaStream_t st) {
  ritz_kernel<<<vec_grid(), kVecThreads, 0, st>>>(V, W, ldv, n, k, small, x_out, wy_out);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_normalize(const VecWork& w, const double* src, double* dst, int64_t n,
                             DevSmall* small, cudaStream_t st) {
  sumsq_kernel<<<w.grid, kVecThreads, 0, st>>>(src, n, w.partials, w.counter, small);
  DMRG_LAUNCH_CHECK();
  scale_copy_kernel<<<w.grid, kVecThreads, 0, st>>>(src, dst, n, small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_axpby(const VecWork& w, const double* a, double c, const double* b, double* out,
                         int64_t n, cudaStream_t st) {
  axpby_kernel<<<w.grid, kVecThreads, 0, st>>>(a, c, b, out, n);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_scale_copy(const VecWork& w, const double* src, double* dst, int64_t n,
                              const DevSmall* small, cudaStream_t st) {
  scale_copy_kernel<<<w.grid, kVecThreads, 0, st>>>(src, dst, n, small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_ritz2(const double* V, const double* W, int64_t ldv, int64_t n, int k,
                         const DevSmall* small, double* x, double* p, double* wx, double* wp,
                         cudaStream_t st) {
  ritz2_kernel<<<vec_grid(), kVecThreads, 0, st>>>(V, W, ldv, n, k, small, x, p, wx, wp);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_orth_pair(const VecWork& w, double* p, double* wp, const double* x,
                             const double* wx, int64_t n, DevSmall* small, cudaStream_t st) {
  // a = x . p (one-column overlap, FP64), p -= a x, ||p||, scale
  DMRG_TRY(launch_overlap(w, x, n, n, 1, p, small->s[2], small, -1, st));
  axpy_pair_kernel<<<vec_grid(), kVecThreads, 0, st>>>(p, wp, x, wx, n, small);
  DMRG_LAUNCH_CHECK();
  sumsq_kernel<<<w.grid, kVecThreads, 0, st>>>(p, n, w.partials, w.counter, small);
  DMRG_LAUNCH_CHECK();
  scale_pair_kernel<<<vec_grid(), kVecThreads, 0, st>>>(p, wp, n, small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_set_B00(DevSmall* small, cudaStream_t st) {
  set_B00_kernel<<<1, 256, 0, st>>>(small);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg

namespace dmrg {

// Public s = V^T w.  The cross-block partial sums live in a stream-ordered scratch
// allocation made for this call.
dmrg_status launch_gemv_trans_public(const double* V, int64_t ldv, int64_t n, int k,
                                     const double* w, double* s, cudaStream_t st) {
  if (n == 0) {
    DMRG_CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(double) * k, st));
    return DMRG_OK;
  }
  VecWork vw;
  vw.grid = vec_grid();
  DMRG_CUDA_TRY(cudaMallocAsync((void**)&vw.partials, sizeof(double) * (size_t)vw.grid * kSlots, st));
  DMRG_CUDA_TRY(cudaMallocAsync((void**)&vw.counter, sizeof(unsigned int), st));
  DMRG_CUDA_TRY(cudaMemsetAsync(vw.counter, 0, sizeof(unsigned int), st));
  gemv_trans_kernel<<<vw.grid, kVecThreads, 0, st>>>(V, ldv, n, k, w, vw.partials, vw.counter, s);
  note_launch();
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(vw.partials, st);
  cudaFreeAsync(vw.counter, st);
  if (e != cudaSuccess) {
    set_error("gemv_trans_kernel: %s", cudaGetErrorString(e));
    return DMRG_ERR_CUDA;
  }
  return DMRG_OK;
}

}  // namespace dmrg
