// FP64 projection: the two launches that evaluate Eq. 11 in float64.
//
// Stage 1 computes, for every record whose two factors are proper operators, the
// intermediate T = A_{i->j} X_{ik} or U = X_{ik} B_{k->l}^T (whichever order costs fewer
// FLOPs).  Stage 2 computes every output segment Y_{jl} as one GEMM whose K dimension is
// the concatenation of all records writing that segment:
//   Y_{jl} = sum_r coef_r P_r Q_r,  P_r Q_r in {T B^T, A U, A X, X B^T},
// so each output element is produced by exactly one CTA, without atomics and with a
// fixed summation order.  GB300 runs float64 at about 1.1 TFLOP/s (measured dgemm), a
// rate a shared-memory-tiled DFMA kernel reaches, so this path uses CUDA-core FP64.
#include "internal.h"

namespace dmrg {
namespace {

constexpr int kThreads = 256;  // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ const double* base_of(const Bases& b, int space) {
  return b.p[space];
}

__global__ void __launch_bounds__(kThreads)
gemm64_kernel(const Tile64* __restrict__ tiles, const Job64* __restrict__ jobs,
              const Seg64* __restrict__ segs, Bases bases, double* __restrict__ c_base_T,
              double* __restrict__ c_base_Y) {
  __shared__ double Ps[kTileK][kTileM + 1];
  __shared__ double Qs[kTileK][kTileN + 1];
  const Tile64 tile = tiles[blockIdx.x];
  const Job64 job = jobs[tile.job];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int mrem = job.M - tile.m0, nrem = job.N - tile.n0;
  for (int si = job.seg_begin; si < job.seg_end; ++si) {
    const Seg64 sg = segs[si];
    const double* P = base_of(bases, sg.P.space) + sg.P.off + (int64_t)tile.m0 * sg.P.rs;
    const double* Q = base_of(bases, sg.Q.space) + sg.Q.off + (int64_t)tile.n0 * sg.Q.cs;
    const bool p_kfast = sg.P.cs == 1;   // K contiguous in P: vary k across threads
    const bool q_nfast = sg.Q.cs == 1;   // N contiguous in Q: vary n across threads
    for (int k0 = 0; k0 < sg.K; k0 += kTileK) {
      const int krem = sg.K - k0;
#pragma unroll
      for (int e = 0; e < (kTileM * kTileK) / kThreads; ++e) {
        const int idx = threadIdx.x + e * kThreads;
        int r, kk;
        if (p_kfast) { kk = idx & (kTileK - 1); r = idx >> 4; }
        else { r = idx & (kTileM - 1); kk = idx >> 6; }
        double v = 0.0;
        if (r < mrem && kk < krem) v = P[(int64_t)r * sg.P.rs + (int64_t)(k0 + kk) * sg.P.cs];
        Ps[kk][r] = sg.alpha * v;
      }
#pragma unroll
      for (int e = 0; e < (kTileN * kTileK) / kThreads; ++e) {
        const int idx = threadIdx.x + e * kThreads;
        int c, kk;
        if (q_nfast) { c = idx & (kTileN - 1); kk = idx >> 6; }
        else { kk = idx & (kTileK - 1); c = idx >> 4; }
        double v = 0.0;
        if (c < nrem && kk < krem) v = Q[(int64_t)(k0 + kk) * sg.Q.rs + (int64_t)c * sg.Q.cs];
        Qs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kTileK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ps[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Qs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  double* C = (job.C.space == SP_T ? c_base_T : c_base_Y) + job.C.off;
  const double* X = bases.p[SP_X] + job.Xaxpy.off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ty + 16 * i;
    if (r >= mrem) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx + 16 * j;
      if (c >= nrem) continue;
      const int64_t rr = tile.m0 + r, cc = tile.n0 + c;
      double v = acc[i][j];
      if (job.axpy != 0.0) v = fma(job.axpy, X[rr * job.Xaxpy.rs + cc], v);
      C[rr * job.C.rs + cc * job.C.cs] = v;
    }
  }
}

}  // namespace

dmrg_status launch_project_fp64(dmrg_plan* p, const double* x, double* y, cudaStream_t st) {
  Bases b;
  b.p[SP_ARENA] = p->arena;
  b.p[SP_X] = x;
  b.p[SP_T] = p->T;
  b.p[SP_Y] = y;
  if (p->ntiles1 > 0) {
    gemm64_kernel<<<(unsigned)p->ntiles1, kThreads, 0, st>>>(p->d_tiles1, p->d_jobs,
                                                             p->d_segs, b, p->T, y);
    DMRG_LAUNCH_CHECK();
  }
  if (p->ntiles2 > 0) {
    gemm64_kernel<<<(unsigned)p->ntiles2, kThreads, 0, st>>>(p->d_tiles2, p->d_jobs,
                                                             p->d_segs, b, p->T, y);
    DMRG_LAUNCH_CHECK();
  }
  return launch_seg_axpy(p, x, y, nullptr, nullptr, st);
}

}  // namespace dmrg
