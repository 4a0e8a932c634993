// Block Davidson-Liu iteration for the lowest few eigenpairs (dmrg_davidson_solve_block).
//
// Sec. 6 names the block extension of the Davidson method (Liu): several candidate vectors
// are added per iteration and a few of the lowest eigenpairs are found, where the paper's
// own solver (Algorithm 3) finds the lowest pair alone.  Per iteration, with k basis
// columns of which those since `done` are new:
//   projection     W(:, c) = H V(:, c) for the new columns        (Eq. 11, FP64-accurate)
//   overlap        B(:, c) = V^T W(:, c), mirrored into row c
//   eigenproblem   all eigenpairs of B in FP64, ascending (all_eig_kernel)
//   residual       for the b lowest: x_c = V y_c, r_c = W y_c - theta_c x_c,
//                  t_c = r_c / (theta_c - D), ||r_c||^2, ||t_c||^2    (one pass, fused)
//   [host]         convergence of the nev lowest; restart when the corrections do not fit
//   per correction CGS2 against the basis (including the corrections accepted before it),
//                  normalise, append; a collapsed one falls back to its raw residual
// The readings are those of the block oracle: corrections for the unconverged pairs among
// the b lowest in ascending order, and a restart to the current Ritz block plus as many of
// the previous iteration's Ritz vectors as leave room for the corrections.
//
// Projections are FP64-accurate (FP64 units or digit products on the tensor cores); the
// vector passes run in FP64.  On this part the FP64 units execute about 0.55 T FMA/s
// against 6.8 TB/s of HBM, so even the single-vector FP64 passes are bound by the FP64
// units, not by bandwidth: a fused multi-vector (BLAS-3 shaped) pass needs the same FP64
// operations per element as the separate ones, and the block form brings no bandwidth
// saving in FP64 arithmetic.  The passes therefore reuse the single-vector kernels, one
// column at a time, except the fused residual above.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace dmrg {
namespace {

#include "vec_common.cuh"

constexpr int kBlockMax = 8;  // largest block size b

// Device side of the block state that DevSmall does not hold.
struct BlockSmall {
  double C[KMAX * KMAX];     // combination coefficients (row-major, column j = output j)
  double rn2[kBlockMax];     // ||r_c||^2 of the b lowest Ritz pairs
  double tn2[kBlockMax];     // ||t_c||^2 of their corrections
};

// For c in [c0, c0 + NB): x_c = V y_c, r_c = W y_c - theta_c x_c, t_c = r_c / (theta_c - D)
// (diagonal correction with the 1e-8 guard) written to T + (c - c0) * ldt and r_c to
// R + (c - c0) * ldt (the fallback of a correction that collapses in Gram-Schmidt);
// ||r_c||^2 and ||t_c||^2 to bs->rn2 / tn2[c].  y_c is column c of small->Q (row-major,
// KMAX columns), theta_c = small->theta[c].
template <int NB>
__global__ void __launch_bounds__(kVecThreads)
block_residual_kernel(const double* __restrict__ V, const double* __restrict__ W,
                      const double* __restrict__ D, int64_t ldv, int64_t n, int k, int c0,
                      double* __restrict__ T, double* __restrict__ R, int64_t ldt,
                      const DevSmall* small, BlockSmall* bs, double* __restrict__ partials,
                      unsigned int* counter) {
  __shared__ double ys[KMAX][NB];
  __shared__ double th[NB];
  for (int e = threadIdx.x; e < KMAX * NB; e += blockDim.x) {
    const int j = e / NB, c = e - (e / NB) * NB;
    ys[j][c] = j < k ? small->Q[j * KMAX + c0 + c] : 0.0;
  }
  if (threadIdx.x < NB) th[threadIdx.x] = small->theta[c0 + threadIdx.x];
  __syncthreads();
  double acc[2 * NB];  // [0, NB): ||r_c||^2, [NB, 2 NB): ||t_c||^2
#pragma unroll
  for (int c = 0; c < 2 * NB; ++c) acc[c] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double x[NB], w[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = w[c] = 0.0;
    for (int j = 0; j < k; ++j) {
      const double v = V[j * ldv + e], wv = W[j * ldv + e];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        x[c] = fma(ys[j][c], v, x[c]);
        w[c] = fma(ys[j][c], wv, w[c]);
      }
    }
    const double d = D[e];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const double r = fma(-th[c], x[c], w[c]);
      double den = th[c] - d;
      if (fabs(den) < 1e-8) den = den >= 0.0 ? 1e-8 : -1e-8;
      const double t = r / den;
      T[c * ldt + e] = t;
      R[c * ldt + e] = r;
      acc[c] = fma(r, r, acc[c]);
      acc[NB + c] = fma(t, t, acc[NB + c]);
    }
  }
  block_partials<0, 2 * NB>(acc, 0, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[2 * NB];
    final_sums(partials, 2 * NB, tot);
    for (int c = threadIdx.x; c < NB; c += blockDim.x) {
      bs->rn2[c0 + c] = tot[c];
      bs->tn2[c0 + c] = tot[NB + c];
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// out_j = sum_{i < k} V_i C[i][j] for j < m (and the same with W into Wout if given):
// the collapsed basis of a restart, or the returned Ritz vectors.
__global__ void __launch_bounds__(kVecThreads)
block_combine_kernel(const double* __restrict__ V, const double* __restrict__ W, int64_t ldv,
                     int64_t n, int k, int m, const BlockSmall* bs, double* __restrict__ Vout,
                     double* __restrict__ Wout, int64_t ldo) {
  __shared__ double cs[KMAX][2 * kBlockMax];
  for (int e = threadIdx.x; e < KMAX * 2 * kBlockMax; e += blockDim.x) {
    const int i = e / (2 * kBlockMax), j = e - (e / (2 * kBlockMax)) * (2 * kBlockMax);
    cs[i][j] = (i < k && j < m) ? bs->C[i * KMAX + j] : 0.0;
  }
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a[2 * kBlockMax], b[2 * kBlockMax];
#pragma unroll
    for (int j = 0; j < 2 * kBlockMax; ++j) a[j] = b[j] = 0.0;
    for (int i = 0; i < k; ++i) {
      const double v = V[i * ldv + e];
      const double w = Wout ? W[i * ldv + e] : 0.0;
#pragma unroll
      for (int j = 0; j < 2 * kBlockMax; ++j) {
        a[j] = fma(cs[i][j], v, a[j]);
        b[j] = fma(cs[i][j], w, b[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2 * kBlockMax; ++j) {
      if (j < m) {
        Vout[j * ldo + e] = a[j];
        if (Wout) Wout[j * ldo + e] = b[j];
      }
    }
  }
}

// before the Gram-Schmidt of correction c (raw = 0) or of its raw residual (raw = 1)
__global__ void set_tnorm_before_kernel(DevSmall* small, const BlockSmall* bs, int c, int raw) {
  small->tnorm2_before = raw ? bs->rn2[c] : bs->tn2[c];
  small->flags = 0;
}

// ||t||^2 of a start vector into tnorm2_before (the breakdown test of finish_kernel), and
// the flags cleared
__global__ void __launch_bounds__(kVecThreads)
start_norm_kernel(const double* __restrict__ t, int64_t n, DevSmall* small,
                  double* __restrict__ partials, unsigned int* counter) {
  double acc[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    acc[0] = fma(t[e], t[e], acc[0]);
  block_partials<0, 1>(acc, 0, partials);
  if (Ticket::last_block(counter)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      small->tnorm2_before = tot[0];
      small->tnorm2 = tot[0];
      small->flags = 0;
      *counter = 0u;
    }
  }
}

template <int NB>
void launch_block_residual_nb(const VecWork& vw, const double* V, const double* W,
                              const double* D, int64_t ldv, int64_t n, int k, double* T,
                              double* R, const DevSmall* small, BlockSmall* bs, cudaStream_t st) {
  block_residual_kernel<NB><<<vw.grid, kVecThreads, 0, st>>>(V, W, D, ldv, n, k, 0, T, R, ldv,
                                                            small, bs, vw.partials, vw.counter);
}

dmrg_status launch_block_residual(const VecWork& vw, const double* V, const double* W,
                                  const double* D, int64_t ldv, int64_t n, int k, int nb,
                                  double* T, double* R, const DevSmall* small, BlockSmall* bs,
                                  cudaStream_t st) {
  switch (nb) {
    case 1: launch_block_residual_nb<1>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 2: launch_block_residual_nb<2>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 3: launch_block_residual_nb<3>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 4: launch_block_residual_nb<4>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 5: launch_block_residual_nb<5>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 6: launch_block_residual_nb<6>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 7: launch_block_residual_nb<7>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    case 8: launch_block_residual_nb<8>(vw, V, W, D, ldv, n, k, T, R, small, bs, st); break;
    default:
      set_error("internal: block size %d", nb);
      return DMRG_ERR_INVALID_ARG;
  }
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

struct BlockState {
  dmrg_plan* plan = nullptr;
  cudaStream_t st = nullptr;
  int64_t n = 0, ldv = 0;
  int ms = 0, b = 0;
  double* V = nullptr;   // ms columns
  double* W = nullptr;
  double* T = nullptr;   // b corrections
  double* R = nullptr;   // b raw residuals
  double* S = nullptr;   // 2 b columns of V scratch for a restart
  double* SW = nullptr;  // 2 b columns of W scratch
  DevSmall* small = nullptr;
  DevSmall* hsmall = nullptr;
  BlockSmall* bs = nullptr;
  BlockSmall* hbs = nullptr;
  VecWork vw;
  dmrg_precision aprec = DMRG_PREC_FP64;
  int projections = 0, restarts = 0, iters = 0, sweeps = 0;

  ~BlockState() {
    cudaFree(V);
    cudaFree(W);
    cudaFree(T);
    cudaFree(R);
    cudaFree(S);
    cudaFree(SW);
    cudaFree(small);
    cudaFree(bs);
    cudaFreeHost(hsmall);
    cudaFreeHost(hbs);
    vec_work_destroy(&vw);
  }

  dmrg_status sync_read() {
    DMRG_CUDA_TRY(cudaMemcpyAsync(hsmall, small, sizeof(DevSmall), cudaMemcpyDeviceToHost, st));
    DMRG_CUDA_TRY(cudaMemcpyAsync(hbs, bs, sizeof(BlockSmall), cudaMemcpyDeviceToHost, st));
    DMRG_CUDA_TRY(cudaStreamSynchronize(st));
    return tc_error_status(plan);
  }

  double* col(double* base, int j) const { return base + (int64_t)j * ldv; }

  // t (in column kcur of V, tnorm2_before set) orthogonalised twice against V(:, :kcur)
  // and normalised; returns through *ok whether it survived (no breakdown)
  dmrg_status orthonormalise(int kcur, bool* ok) {
    double* t = col(V, kcur);
    if (kcur > 0) {
      DMRG_TRY(launch_overlap(vw, V, ldv, n, kcur, t, small->s[0], small, -1, st));
      DMRG_TRY(launch_cgs(vw, V, ldv, n, kcur, t, small, 0, 1, st, 0));
      DMRG_TRY(launch_cgs(vw, V, ldv, n, kcur, t, small, 1, 2, st, 1));
    }
    DMRG_TRY(launch_finish(t, n, small, st));
    DMRG_TRY(sync_read());
    if (hsmall->flags & 2) {
      set_error("non-finite vector in the block Davidson iteration");
      return DMRG_ERR_NUMERIC;
    }
    *ok = !(hsmall->flags & 1);
    return DMRG_OK;
  }
};

}  // namespace
}  // namespace dmrg

using namespace dmrg;

extern "C" dmrg_status dmrg_davidson_solve_block(dmrg_plan* plan, int32_t nev, int32_t block,
                                                 const double* X0, int64_t ldx0, double* X_out,
                                                 int64_t ldx_out, double* energies,
                                                 double* resnorms, dmrg_solve_info* info,
                                                 void* stream) {
  if (!plan || !X0 || !X_out || !energies) {
    set_error("dmrg_davidson_solve_block: NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  const int ms = plan->opt.max_subspace;
  if (block < 1 || block > kBlockMax || nev < 1 || nev > block || 2 * block > ms ||
      ldx0 < plan->n || ldx_out < plan->n) {
    set_error("dmrg_davidson_solve_block: need 1 <= nev <= block <= %d, 2 block <= max_subspace "
              "(%d), ldx0 and ldx_out >= n", kBlockMax, ms);
    return DMRG_ERR_INVALID_ARG;
  }
  if (plan->n == 0) {
    set_error("empty superblock (n = 0)");
    return DMRG_ERR_SHAPE;
  }
  if (plan->n < block) {
    set_error("dmrg_davidson_solve_block: block %d exceeds the dimension %lld", block,
              (long long)plan->n);
    return DMRG_ERR_INVALID_ARG;
  }
  BlockState s;
  s.plan = plan;
  s.st = (cudaStream_t)stream;
  s.n = plan->n;
  s.ldv = round_up(plan->n, 32);
  s.ms = ms;
  s.b = block;
  const dmrg_precision p = plan->opt.prec;
  s.aprec = (p == DMRG_PREC_FP64 || p == DMRG_PREC_FP64_TC) ? p : plan->opt.anchor_prec;
  const size_t colb = sizeof(double) * (size_t)s.ldv;
  if (cudaMalloc((void**)&s.V, colb * ms) != cudaSuccess ||
      cudaMalloc((void**)&s.W, colb * ms) != cudaSuccess ||
      cudaMalloc((void**)&s.T, colb * block) != cudaSuccess ||
      cudaMalloc((void**)&s.R, colb * block) != cudaSuccess ||
      cudaMalloc((void**)&s.S, colb * 2 * block) != cudaSuccess ||
      cudaMalloc((void**)&s.SW, colb * 2 * block) != cudaSuccess ||
      cudaMalloc((void**)&s.small, sizeof(DevSmall)) != cudaSuccess ||
      cudaMalloc((void**)&s.bs, sizeof(BlockSmall)) != cudaSuccess ||
      cudaMallocHost((void**)&s.hsmall, sizeof(DevSmall)) != cudaSuccess ||
      cudaMallocHost((void**)&s.hbs, sizeof(BlockSmall)) != cudaSuccess) {
    cudaGetLastError();
    set_error("allocation of the block Davidson workspace failed");
    return DMRG_ERR_OOM;
  }
  DMRG_TRY(vec_work_create(&s.vw));
  cudaStream_t st = s.st;
  DMRG_CUDA_TRY(cudaMemsetAsync(s.V, 0, colb * ms, st));
  DMRG_CUDA_TRY(cudaMemsetAsync(s.W, 0, colb * ms, st));
  DMRG_CUDA_TRY(cudaMemsetAsync(s.small, 0, sizeof(DevSmall), st));
  DMRG_CUDA_TRY(cudaMemsetAsync(s.bs, 0, sizeof(BlockSmall), st));
  const int64_t n = s.n, ldv = s.ldv;

  // ---- start block, orthonormalised column by column
  int k = 0;
  for (int j = 0; j < block; ++j) {
    DMRG_CUDA_TRY(cudaMemcpyAsync(s.col(s.V, k), X0 + (int64_t)j * ldx0, sizeof(double) * n,
                                  cudaMemcpyDeviceToDevice, st));
    start_norm_kernel<<<s.vw.grid, kVecThreads, 0, st>>>(s.col(s.V, k), n, s.small, s.vw.partials,
                                                        s.vw.counter);
    DMRG_LAUNCH_CHECK();
    bool ok = false;
    DMRG_TRY(s.orthonormalise(k, &ok));
    if (!ok) {
      set_error("dmrg_davidson_solve_block: start block is rank deficient (column %d)", j);
      return DMRG_ERR_INVALID_ARG;
    }
    ++k;
  }

  int done = 0;
  std::vector<double> Yprev;  // previous Ritz coefficients, kprev x b, column-major
  int kprev = 0;
  bool converged = false;
  std::vector<double> theta(block), rn(block);
  dmrg_status err = DMRG_OK;
  for (int it = 0; it < plan->opt.max_iter && err == DMRG_OK; ++it) {
    // projections and overlaps of the new columns
    for (int c = done; c < k && err == DMRG_OK; ++c) {
      err = dmrg_project_prec(plan, s.aprec, s.col(s.V, c), s.col(s.W, c), st);
      ++s.projections;
    }
    for (int c = done; c < k && err == DMRG_OK; ++c)
      err = launch_overlap(s.vw, s.V, ldv, n, k, s.col(s.W, c), nullptr, s.small, c, st);
    if (err != DMRG_OK) break;
    done = k;
    if ((err = launch_all_eig(s.small, k, st)) != DMRG_OK) break;
    if ((err = launch_block_residual(s.vw, s.V, s.W, plan->D, ldv, n, k, block, s.T, s.R,
                                     s.small, s.bs, st)) != DMRG_OK)
      break;
    if ((err = s.sync_read()) != DMRG_OK) break;
    ++s.iters;
    s.sweeps += s.hsmall->jacobi_sweeps;
    bool all = true;
    for (int c = 0; c < block; ++c) {
      theta[c] = s.hsmall->theta[c];
      rn[c] = sqrt(std::max(0.0, s.hbs->rn2[c]));
      if (!std::isfinite(theta[c]) || !std::isfinite(rn[c])) {
        set_error("non-finite Ritz pair in the block Davidson iteration %d", s.iters);
        err = DMRG_ERR_NUMERIC;
      }
      if (c < nev && !(rn[c] <= plan->opt.tol)) all = false;
    }
    if (err != DMRG_OK) break;
    // the b lowest Ritz coefficient vectors (column-major k x b)
    std::vector<double> Y((size_t)k * block);
    for (int c = 0; c < block; ++c)
      for (int j = 0; j < k; ++j) Y[(size_t)c * k + j] = s.hsmall->Q[j * KMAX + c];
    if (all) {
      converged = true;
      // X_out = V Y(:, :nev)
      for (int j = 0; j < KMAX * KMAX; ++j) s.hbs->C[j] = 0.0;
      for (int c = 0; c < nev; ++c)
        for (int j = 0; j < k; ++j) s.hbs->C[j * KMAX + c] = Y[(size_t)c * k + j];
      DMRG_CUDA_TRY(cudaMemcpyAsync(s.bs->C, s.hbs->C, sizeof(s.hbs->C), cudaMemcpyHostToDevice, st));
      block_combine_kernel<<<s.vw.grid, kVecThreads, 0, st>>>(s.V, nullptr, ldv, n, k, nev, s.bs,
                                                             X_out, nullptr, ldx_out);
      DMRG_LAUNCH_CHECK();
      break;
    }
    std::vector<int> idx;
    for (int c = 0; c < block; ++c)
      if (!(rn[c] <= plan->opt.tol)) idx.push_back(c);
    if (k + (int)idx.size() > ms) {
      // collapse to the Ritz block and as much of the previous one as leaves room
      const int keep_prev = plan->opt.restart_keep == 2 ? ms - block - (int)idx.size() : 0;
      std::vector<std::vector<double>> C;
      for (int c = 0; c < block; ++c) C.emplace_back(Y.begin() + (size_t)c * k, Y.begin() + (size_t)(c + 1) * k);
      if (kprev > 0) {
        for (int c = 0; c < std::min(keep_prev, block); ++c) {
          std::vector<double> v(k, 0.0);
          for (int j = 0; j < kprev && j < k; ++j) v[j] = Yprev[(size_t)c * kprev + j];
          for (int pass = 0; pass < 2; ++pass)
            for (const auto& q : C) {
              double a = 0.0;
              for (int j = 0; j < k; ++j) a += q[j] * v[j];
              for (int j = 0; j < k; ++j) v[j] -= a * q[j];
            }
          double nv = 0.0;
          for (int j = 0; j < k; ++j) nv += v[j] * v[j];
          nv = sqrt(nv);
          if (nv > 1e-8) {
            for (int j = 0; j < k; ++j) v[j] /= nv;
            C.push_back(v);
          }
        }
      }
      const int kc = (int)C.size();
      for (int j = 0; j < KMAX * KMAX; ++j) s.hbs->C[j] = 0.0;
      for (int c = 0; c < kc; ++c)
        for (int j = 0; j < k; ++j) s.hbs->C[j * KMAX + c] = C[c][j];
      // B <- C^T B C (host, from the B read back with this iteration's state)
      std::vector<double> Bn((size_t)KMAX * KMAX, 0.0);
      for (int a = 0; a < kc; ++a)
        for (int c = 0; c < kc; ++c) {
          double v = 0.0;
          for (int i = 0; i < k; ++i) {
            double bi = 0.0;
            for (int j = 0; j < k; ++j) bi += s.hsmall->B[i * KMAX + j] * C[c][j];
            v += C[a][i] * bi;
          }
          Bn[(size_t)a * KMAX + c] = v;
        }
      for (int a = 0; a < kc; ++a)  // exactly symmetric
        for (int c = 0; c < a; ++c) Bn[(size_t)a * KMAX + c] = Bn[(size_t)c * KMAX + a];
      DMRG_CUDA_TRY(cudaMemcpyAsync(s.bs->C, s.hbs->C, sizeof(s.hbs->C), cudaMemcpyHostToDevice, st));
      block_combine_kernel<<<s.vw.grid, kVecThreads, 0, st>>>(s.V, s.W, ldv, n, k, kc, s.bs, s.S,
                                                             s.SW, ldv);
      DMRG_LAUNCH_CHECK();
      DMRG_CUDA_TRY(cudaMemcpyAsync(s.V, s.S, colb * kc, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s.W, s.SW, colb * kc, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s.small->B, Bn.data(), sizeof(double) * KMAX * KMAX,
                                    cudaMemcpyHostToDevice, st));
      // the Ritz block in the new basis: C^T Y = the first b unit vectors
      std::vector<double> Yn((size_t)kc * block, 0.0);
      for (int c = 0; c < block; ++c)
        for (int a = 0; a < kc; ++a) {
          double v = 0.0;
          for (int j = 0; j < k; ++j) v += C[a][j] * Y[(size_t)c * k + j];
          Yn[(size_t)c * kc + a] = v;
        }
      Y.swap(Yn);
      k = done = kc;
      ++s.restarts;
    }
    Yprev = Y;
    kprev = k;
    int added = 0;
    for (int c : idx) {
      // the correction, else (if it collapses in Gram-Schmidt) the raw residual, else none
      bool ok = false;
      for (int raw = 0; raw < 2 && !ok && err == DMRG_OK; ++raw) {
        DMRG_CUDA_TRY(cudaMemcpyAsync(s.col(s.V, k), s.col(raw ? s.R : s.T, c), sizeof(double) * n,
                                      cudaMemcpyDeviceToDevice, st));
        set_tnorm_before_kernel<<<1, 1, 0, st>>>(s.small, s.bs, c, raw);
        DMRG_LAUNCH_CHECK();
        err = s.orthonormalise(k, &ok);
      }
      if (err != DMRG_OK) break;
      if (!ok) continue;
      ++k;
      ++added;
    }
    if (err != DMRG_OK) break;
    if (added == 0) {
      set_error("block Davidson basis breakdown at iteration %d", s.iters);
      err = DMRG_ERR_NUMERIC;
      break;
    }
  }
  if (err == DMRG_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("block solve: %s", cudaGetErrorString(cudaGetLastError()));
    err = DMRG_ERR_CUDA;
  }
  for (int c = 0; c < nev; ++c) {
    energies[c] = theta[c];
    if (resnorms) resnorms[c] = rn[c];
  }
  if (info) {
    info->energy = theta[0];
    info->resnorm = rn[0];
    info->iters = s.iters;
    info->projections = 0;
    info->fp64_projections = s.projections;
    info->restarts = s.restarts;
    info->small_eig_sweeps = s.sweeps;
    info->converged = converged ? 1 : 0;
    info->anchor_updates = 0;
  }
  if (err == DMRG_OK && !converged) {
    set_error("block Davidson did not converge in %d iterations", s.iters);
    err = DMRG_ERR_NOT_CONVERGED;
  }
  return err;
}
