// The small projected eigenproblem of Algorithm 3 (line 4): the lowest eigenpair (lambda, y)
// of the symmetric k x k matrix B = V^T H V, k <= 24, computed by one CTA.
//
// This part executes FP64 at about 2 FMA per clock per SM, so a cyclic Jacobi solve in
// FP64 (~10^4 FP64 operations per sweep at k = 20, several sweeps) costs ~100 us per call,
// as much as a BF16x3 projection.  The solver therefore splits the work:
//   1. cyclic Jacobi in FP32 on the FP32 units (round-robin ordering: the k/2 rotations of a
//      step are disjoint; every 2 x 2 block of J^T A J is updated by one thread), warm-
//      started from the previous call's eigendecomposition: B_k differs from B_{k-1} by its
//      last row and column, so in the basis diag(Q_{k-1}, 1) it is diagonal except for that
//      row and column (an arrowhead), which a few sweeps finish;
//   2. refinement of the lowest pair in FP64 on B itself, with the FP32 eigenvectors U and
//      eigenvalues theta as the approximate inverse:
//          lambda = y^T B y / y^T y,  rho = B y - lambda y,
//          y <- y - sum_{i != b} u_i (u_i^T rho) / (theta_i - lambda)
//      (b the lowest index); each step multiplies the error by about the FP32
//      decomposition error over the eigenvalue gap, until ||rho|| reaches the FP64 level;
//   3. if ||rho|| does not reach that level (eigenvalues closer than the FP32 resolution),
//      a cold Jacobi solve with FP64 rotations replaces steps 1-2.
// Jacobi rotation (p, q): tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c zeroes a_pq of J^T A J (the symmetric
// Schur decomposition of the 2 x 2 block).
#include <math.h>

#include "internal.h"

namespace dmrg {
namespace {

constexpr int kEigThreads = 256;  // >= KMAX^2 / 2: two Q items per thread suffice
constexpr double kEps = 1.1102230246251565e-16;  // 2^-53

// player at position j of step `step` of the round-robin tournament over kk (even)
// players: position 0 stays, the others rotate; pairs are positions (i, kk - 1 - i)
__device__ __forceinline__ int rr_player(int j, int step, int kk) {
  return j == 0 ? 0 : 1 + (j - 1 + step) % (kk - 1);
}

// Rotation parameters of pair (p, q) from the current A.  FP32: the exact annihilating
// rotation in FP32.  FP64: the angle in FP32 (it only needs to be close to the
// annihilating one; the next sweep removes what is left), c and s in FP64 from the same
// t, so c^2 + s^2 = 1 to FP64 rounding (two Newton steps for 1 / sqrt(1 + t^2) from the
// FP32 estimate).
__device__ __forceinline__ float absval(float x) { return fabsf(x); }
__device__ __forceinline__ double absval(double x) { return fabs(x); }

template <typename T>
__device__ __forceinline__ void rotation(T app, T aqq, T apq, T& c, T& s) {
  const float tau = (float)(aqq - app) / (2.0f * (float)apq);
  const float tf = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
  if constexpr (sizeof(T) == 4) {
    c = rsqrtf(1.0f + tf * tf);
    s = tf * c;
  } else {
    const double t = (double)tf;
    const double u = fma(t, t, 1.0);
    double cc = (double)rsqrtf((float)u);
    cc = cc * fma(-0.5 * u, cc * cc, 1.5);
    cc = cc * fma(-0.5 * u, cc * cc, 1.5);
    c = cc;
    s = t * cc;
  }
}

// Round-robin schedule of one sweep, computed once per call: pair i of step t is
// (sp[t][i], sq[t][i]) with sp < sq; players >= k are dummies (no rotation).
struct Schedule {
  uint8_t sp[KMAX][KMAX / 2], sq[KMAX][KMAX / 2];
  __device__ void build(int kk) {
    const int half = kk / 2;
    for (int e = threadIdx.x; e < (kk - 1) * half; e += blockDim.x) {
      const int t = e / half, i = e - t * half;
      int p = rr_player(i, t, kk), q = rr_player(kk - 1 - i, t, kk);
      if (p > q) { const int w = p; p = q; q = w; }
      sp[t][i] = (uint8_t)p;
      sq[t][i] = (uint8_t)q;
    }
  }
};

// Cyclic Jacobi on A (k x k in shared memory, rows and columns k..kk-1 zero), accumulating
// Q <- Q J.  A rotation is skipped when a_pq^2 <= rel2 |a_pp a_qq| + abs2; sweeps stop
// after one without rotations.  Returns the number of sweeps.  All threads call it.  Each
// thread owns fixed work items for the whole solve (no index arithmetic per step): at
// most one 2 x 2 block (I, J) of J^T A J and two (row, pair) items of Q J.
template <typename T>
__device__ int jacobi_sweeps(T (*A)[KMAX + 1], T (*Q)[KMAX + 1], int k, T rel2, T abs2,
                             int max_sweeps, const Schedule& sch, T* cs, T* sn, int* rotated) {
  const int tid = threadIdx.x;
  const int kk = (k + 1) & ~1;
  const int half = kk / 2;
  const bool has_blk = tid < half * half;
  const int bI = has_blk ? tid / half : 0, bJ = has_blk ? tid - (tid / half) * half : 0;
  int qr[2], qj[2];
  bool has_q[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = tid + u * (int)blockDim.x;
    has_q[u] = e < k * half;
    qr[u] = has_q[u] ? e / half : 0;
    qj[u] = has_q[u] ? e - (e / half) * half : 0;
  }
  int sweep = 0;
  for (; sweep < max_sweeps && k > 1; ++sweep) {
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int step = 0; step < kk - 1; ++step) {
      if (tid < half) {
        const int p = sch.sp[step][tid], q = sch.sq[step][tid];
        T c = (T)1, s = (T)0;
        if (q < k) {
          const T apq = A[p][q], app = A[p][p], aqq = A[q][q];
          if (apq != (T)0 && apq * apq > rel2 * absval(app * aqq) + abs2) {
            rotation<T>(app, aqq, apq, c, s);
            *rotated = 1;
          }
        }
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // A <- J^T A J: the 2 x 2 block (rows of pair I, columns of pair J) depends only on
      // itself, so each thread updates its block in place
      if (has_blk) {
        const T sI = sn[bI], sJ = sn[bJ];
        if (sI != (T)0 || sJ != (T)0) {
          const int a0 = sch.sp[step][bI], a1 = sch.sq[step][bI];
          const int b0 = sch.sp[step][bJ], b1 = sch.sq[step][bJ];
          const T cI = cs[bI], cJ = cs[bJ];
          const T x00 = A[a0][b0], x01 = A[a0][b1], x10 = A[a1][b0], x11 = A[a1][b1];
          const T y00 = cI * x00 - sI * x10, y01 = cI * x01 - sI * x11;
          const T y10 = sI * x00 + cI * x10, y11 = sI * x01 + cI * x11;
          T z01 = sJ * y00 + cJ * y01, z10 = cJ * y10 - sJ * y11;
          if (sizeof(T) == 4 && bI == bJ) z01 = z10 = (T)0;  // the FP32 rotation annihilates a_pq
          A[a0][b0] = cJ * y00 - sJ * y01;
          A[a0][b1] = z01;
          A[a1][b0] = z10;
          A[a1][b1] = sJ * y10 + cJ * y11;
        }
      }
      // Q <- Q J
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!has_q[u]) continue;
        const T sJ = sn[qj[u]];
        if (sJ == (T)0) continue;
        const int b0 = sch.sp[step][qj[u]], b1 = sch.sq[step][qj[u]];
        const T cJ = cs[qj[u]];
        const T q0 = Q[qr[u]][b0], q1 = Q[qr[u]][b1];
        Q[qr[u]][b0] = cJ * q0 - sJ * q1;
        Q[qr[u]][b1] = sJ * q0 + cJ * q1;
      }
      __syncthreads();
    }
    const int any = *rotated;
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  return sweep;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kEigThreads) small_eig_kernel(DevSmall* small, int k) {
  __shared__ double Bs[KMAX][KMAX + 1];
  __shared__ float A32[KMAX][KMAX + 1];
  __shared__ float Q32[KMAX][KMAX + 1];
  __shared__ float cs32[KMAX / 2], sn32[KMAX / 2];
  __shared__ double A64[KMAX][KMAX + 1];
  __shared__ double Q64[KMAX][KMAX + 1];
  __shared__ double cs64[KMAX / 2], sn64[KMAX / 2];
  __shared__ Schedule sch;
  __shared__ int rotated, best, refined_ok;
  __shared__ double yref[KMAX];
  __shared__ double lam_ref;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long c0 = clock64();
  const bool warm = k > 1 && small->qk == k - 1;

  // the previous call's eigenvector (restarts keep the previous Ritz vector); thread tid
  // also writes y[tid] at the end, after this read
  if (tid < KMAX) small->y_prev[tid] = small->y[tid];
  sch.build((k + 1) & ~1);
  // ---- B, and the FP32 start: the arrowhead in the previous eigenbasis, or B itself
  for (int e = tid; e < KMAX * KMAX; e += blockDim.x) {
    const int r = e / KMAX, c = e - (e / KMAX) * KMAX;
    const double b = (r < k && c < k) ? small->B[r * KMAX + c] : 0.0;
    Bs[r][c] = b;
    float q = (r == c) ? 1.0f : 0.0f;
    if (warm && r < k - 1 && c < k - 1) q = (float)small->Q[r * KMAX + c];
    Q32[r][c] = q;
  }
  __syncthreads();
  for (int e = tid; e < KMAX * KMAX; e += blockDim.x) {
    const int r = e / KMAX, c = e - (e / KMAX) * KMAX;
    float a = 0.0f;
    if (r < k && c < k) {
      if (!warm) {
        a = (float)Bs[r][c];
      } else if (r < k - 1 && c < k - 1) {
        a = r == c ? (float)small->theta[r] : 0.0f;
      } else if (r == k - 1 && c == k - 1) {
        a = (float)Bs[k - 1][k - 1];
      } else {  // arrow: (Q^T b)_i, b = B(0:k-1, k-1)
        const int i = r < k - 1 ? r : c;
        float z = 0.0f;
        for (int m = 0; m < k - 1; ++m) z = fmaf(Q32[m][i], (float)Bs[m][k - 1], z);
        a = z;
      }
    }
    A32[r][c] = a;
  }
  __syncthreads();

  // ---- 1. FP32 Jacobi; rotations stop at the FP32 resolution of the largest diagonal
  __shared__ float scale32;
  if (tid == 0) {
    float sc = 0.0f;
    for (int i = 0; i < k; ++i) sc = fmaxf(sc, fabsf(A32[i][i]));
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) sc = fmaxf(sc, fabsf(A32[i][j]));
    scale32 = sc;
  }
  __syncthreads();
  const float tol32 = 2e-7f * scale32;
  int sweeps = jacobi_sweeps<float>(A32, Q32, k, 0.0f, tol32 * tol32, 30, sch, cs32, sn32, &rotated);
  if (tid == 0) {
    int b = 0;
    for (int i = 1; i < k; ++i)
      if (A32[i][i] < A32[b][b]) b = i;
    best = b;
    refined_ok = 0;
  }
  __syncthreads();
  const long long c1 = clock64();

  // ---- 2. FP64 refinement of the lowest pair.  B y is split over the 8 warps (warp w adds
  // the columns j = w, w + 8, w + 16 for row = lane; the FP64 pipe of each SM sub-partition
  // works in parallel), the rest runs in warp 0 (lane i owns row i).  B y, the Rayleigh
  // quotient and rho are FP64; the correction U D^-1 U^T rho only has to be accurate
  // relative to the (small) error it removes, so it runs in FP32.  y is normalised at the end.
  __shared__ double ysh[KMAX], wpart[kEigThreads / 32][KMAX];
  __shared__ int ref_stop;
  constexpr int kWarps = kEigThreads / 32;
  static_assert(kWarps == 8, "the partial sums below combine 8 warps");
  const int b = best;
  const bool act = lane < k;
  double scale = 0.0;
  for (int i = 0; i < k; ++i) scale = fmax(scale, fabs((double)A32[i][i]));
  scale = fmax(scale, 1e-300);
  const double tol = 8.0 * kEps * scale * sqrt((double)k);
  const double accept = 64.0 * kEps * scale * sqrt((double)k);
  double y = 0.0, lam = 0.0, rel2 = INFINITY, yy = 1.0;
  if (warp == 0) {
    y = act ? (double)Q32[lane][b] : 0.0;
    if (act) ysh[lane] = y;
    if (lane == 0) ref_stop = 0;
  }
  const double theta = act ? (double)A32[lane][lane] : 0.0;
  for (int it = 0; it < 6; ++it) {
    __syncthreads();  // ysh, ref_stop
    if (ref_stop) break;
    if (act) {
      double part = 0.0;
      for (int j = warp; j < k; j += kWarps) part = fma(Bs[lane][j], ysh[j], part);
      wpart[warp][lane] = part;
    }
    __syncthreads();
    if (warp == 0) {
      double w = 0.0;
      if (act) {
        double w0 = wpart[0][lane] + wpart[1][lane], w1 = wpart[2][lane] + wpart[3][lane];
        double w2 = wpart[4][lane] + wpart[5][lane], w3 = wpart[6][lane] + wpart[7][lane];
        w = (w0 + w1) + (w2 + w3);
      }
      double s_yy = y * y, s_yw = y * w;  // two reductions in one shuffle tree
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s_yy += __shfl_xor_sync(0xffffffffu, s_yy, o);
        s_yw += __shfl_xor_sync(0xffffffffu, s_yw, o);
      }
      yy = s_yy;
      lam = s_yw / yy;
      const double rho = act ? fma(-lam, y, w) : 0.0;
      rel2 = warp_sum(rho * rho) / yy;  // ||rho||^2 / ||y||^2
      if (rel2 <= tol * tol || it == 5) {
        if (lane == 0) ref_stop = 1;
      } else {
        const float rf = (float)rho;
        float c = 0.0f;
        for (int j = 0; j < k; ++j) {
          const float rj = __shfl_sync(0xffffffffu, rf, j);
          if (act) c = fmaf(Q32[j][lane], rj, c);
        }
        const double d = theta - lam;
        c = (!act || lane == b || fabs(d) < 1e-6 * scale) ? 0.0f : c / (float)d;
        float dy = 0.0f;
        for (int i = 0; i < k; ++i) {
          const float ci = __shfl_sync(0xffffffffu, c, i);
          if (act) dy = fmaf(Q32[lane][i], ci, dy);
        }
        y -= (double)dy;
        if (act) ysh[lane] = y;
      }
    }
  }
  if (warp == 0) {
    if (act) yref[lane] = y / sqrt(yy);
    if (lane == 0) {
      lam_ref = lam;
      refined_ok = (rel2 <= accept * accept) ? 1 : 0;
    }
  }
  __syncthreads();

  const long long c2 = clock64();
  if (refined_ok) {
    if (tid == 0) {
      small->lambda = lam_ref;
      small->jacobi_sweeps = sweeps;
      small->qk = k;
      small->eig_cycles[0] = c1 - c0;
      small->eig_cycles[1] = c2 - c1;
      small->eig_cycles[2] = clock64() - c0;
    }
    for (int e = tid; e < k * k; e += blockDim.x) {
      const int r = e / k, c = e - (e / k) * k;
      small->Q[r * KMAX + c] = (double)Q32[r][c];
    }
    if (tid < k) small->theta[tid] = (double)A32[tid][tid];
    if (tid < KMAX) small->y[tid] = tid < k ? yref[tid] : 0.0;
    return;
  }

  // ---- 3. fallback: cold Jacobi with FP64 rotations
  for (int e = tid; e < KMAX * KMAX; e += blockDim.x) {
    const int r = e / KMAX, c = e - (e / KMAX) * KMAX;
    A64[r][c] = Bs[r][c];
    Q64[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __shared__ double scale64;
  if (tid == 0) {
    double sc = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) sc = fmax(sc, fabs(Bs[i][j]));
    scale64 = sc;
  }
  __syncthreads();
  const double abs64 = 1e-17 * scale64;
  sweeps += jacobi_sweeps<double>(A64, Q64, k, 1e-30, abs64 * abs64, 40, sch, cs64, sn64, &rotated);
  if (tid == 0) {
    int b = 0;
    for (int i = 1; i < k; ++i)
      if (A64[i][i] < A64[b][b]) b = i;
    best = b;
    small->eig_fallbacks += 1;
    small->eig_cycles[0] = c1 - c0;
    small->eig_cycles[1] = c2 - c1;
    small->eig_cycles[2] = clock64() - c0;
    small->lambda = A64[b][b];
    small->jacobi_sweeps = sweeps;
    small->qk = k;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int r = e / k, c = e - (e / k) * k;
    small->Q[r * KMAX + c] = Q64[r][c];
  }
  if (tid < k) small->theta[tid] = A64[tid][tid];
  if (tid < KMAX) small->y[tid] = tid < k ? Q64[tid][best] : 0.0;
}

// All eigenpairs of the k x k symmetric B in FP64, in ascending order (the block iteration
// needs the b lowest pairs, not only the lowest): a cold cyclic Jacobi solve with FP64
// rotations on B, then the eigenvalues sorted; theta[j] is the j-th smallest and column j
// of Q (Q[r * KMAX + j]) its eigenvector.
__global__ void __launch_bounds__(kEigThreads) all_eig_kernel(DevSmall* small, int k) {
  __shared__ double A64[KMAX][KMAX + 1];
  __shared__ double Q64[KMAX][KMAX + 1];
  __shared__ double cs64[KMAX / 2], sn64[KMAX / 2];
  __shared__ Schedule sch;
  __shared__ int rotated;
  __shared__ int order[KMAX];
  __shared__ double scale64;
  const int tid = threadIdx.x;
  sch.build((k + 1) & ~1);
  for (int e = tid; e < KMAX * KMAX; e += blockDim.x) {
    const int r = e / KMAX, c = e - (e / KMAX) * KMAX;
    A64[r][c] = (r < k && c < k) ? small->B[r * KMAX + c] : 0.0;
    Q64[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double sc = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) sc = fmax(sc, fabs(A64[i][j]));
    scale64 = sc;
  }
  __syncthreads();
  const double abs64 = 1e-17 * scale64;
  const int sweeps = jacobi_sweeps<double>(A64, Q64, k, 1e-30, abs64 * abs64, 40, sch, cs64, sn64, &rotated);
  if (tid == 0) {
    // ascending order of the diagonal (selection sort of at most 24 values)
    for (int i = 0; i < k; ++i) order[i] = i;
    for (int i = 0; i < k; ++i) {
      int m = i;
      for (int j = i + 1; j < k; ++j)
        if (A64[order[j]][order[j]] < A64[order[m]][order[m]]) m = j;
      const int w = order[i];
      order[i] = order[m];
      order[m] = w;
    }
    small->jacobi_sweeps = sweeps;
    small->qk = 0;  // not a warm start for the single-vector solver
  }
  __syncthreads();
  for (int e = tid; e < KMAX * KMAX; e += blockDim.x) {
    const int r = e / KMAX, c = e - (e / KMAX) * KMAX;
    small->Q[e] = (r < k && c < k) ? Q64[r][order[c]] : 0.0;
  }
  if (tid < KMAX) small->theta[tid] = tid < k ? A64[order[tid]][order[tid]] : 0.0;
}

}  // namespace

dmrg_status launch_all_eig(DevSmall* small, int k, cudaStream_t st) {
  all_eig_kernel<<<1, kEigThreads, 0, st>>>(small, k);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

dmrg_status launch_jacobi(DevSmall* small, int k, cudaStream_t st) {
  small_eig_kernel<<<1, kEigThreads, 0, st>>>(small, k);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

}  // namespace dmrg
