// The Davidson iteration of Algorithm 3 on the GPU, driven by a thin host loop.
//
// Per iteration (k basis columns, the newest one not yet projected):
//   projection     W(:,k-1) = H V(:,k-1)                     (line 2; plan precision)
//   overlap        B(:,k-1) = V^T W(:,k-1), mirrored into row k-1  (line 3)
//   jacobi         (lambda, y) = lowest eigenpair of B            (line 4)
//   residual       r = W y - lambda V y, ||r||, t = r/(lambda - D), V^T t   (lines 5-6, 9)
//   [host]         read ||r||, lambda; decide convergence / restart (line 7)
//   cgs x2         t -= V (V^T t), twice                         (lines 11-12)
//   finish         t /= ||t||, append                            (line 13)
// Readings where the paper is silent are the ones of the FP64 oracle: diagonal
// correction with a 1e-8 denominator guard, classical Gram-Schmidt applied twice with a
// fall-back to the raw residual on breakdown, restart to the Ritz vector when the basis
// holds max_subspace columns (20 in Sec. 6.1), stop on ||r||_2 <= tol.
//
// Low-precision projections (TF32, BF16X3, BF16X2) carry an error of order eps * ||H||,
// which bounds how small the computed residual can get.  The mixed mode therefore anchors the
// iteration with float64 projections: the basis is collapsed to the Ritz vector x, which
// is projected in FP64, so lambda = x^T H x is an FP64 Rayleigh quotient and the residual
// W(:,0) - lambda x is exact.  Only such an exact residual can end the iteration.  Later
// low-precision columns only carry the error of the correction x - x_anchor, which
// shrinks as the iteration converges; the coupling of the anchor with them is taken from
// the exact column.  An anchor is taken when the computed residual approaches the
// estimated low-precision floor eps ||H|| ||y(1:)||, when it falls below tol, and at a
// subspace-limit restart close to the floor or after a stalled phase (other restarts are
// plain ones keeping W y).
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "internal.h"

using namespace dmrg;

struct dmrg_davidson_state {
  dmrg_plan* plan = nullptr;
  int64_t n = 0, ldv = 0;
  int kmax = 20;
  double* V = nullptr;     // (kmax + 1) columns (split arithmetic: column 0 only)
  double* W = nullptr;     // kmax columns (split arithmetic: column 0 only)
  bool f32 = false;        // split arithmetic: columns >= 1 of V and W stored in FP32
  float* V32 = nullptr;    // kmax + 1 FP32 columns (column 0 unused)
  float* W32 = nullptr;    // kmax FP32 columns (column 0 unused)
  double* tbuf = nullptr;  // split arithmetic: the new direction t while it is formed
  double* D = nullptr;     // padded diag(H_SB)
  double* xbuf = nullptr;  // Ritz vector at a restart
  double* wbuf = nullptr;  // W y at a restart
  double* pbuf = nullptr;  // second kept vector of a two-vector restart
  double* wpbuf = nullptr; // its W combination
  DevSmall* small = nullptr;
  DevSmall* hsmall = nullptr;  // pinned mirror
  VecWork vw;
  int k = 1;
  int iters = 0, projections = 0, fp64_projections = 0, restarts = 0;
  double lambda = NAN, rnorm = INFINITY;
  bool converged = false;
  bool mixed = false;
  bool anchor_pending = false;
  double anchor_rnorm = INFINITY;
  int ritz_k = 1;  // columns that small->y refers to; 0: V(:,0) holds the Ritz vector
  bool anchored = false;  // column 0 of W is an FP64 projection (mixed mode)
  int plain_restarts = 0; // subspace-limit restarts since the last FP64 anchor
  int sweeps = 0;         // Jacobi sweeps over all iterations
  double floor_est = 0.0; // estimated low-precision residual floor (mixed mode)
  double restart_rnorm = INFINITY;  // residual at the last subspace-limit restart
  double baked_err = 0.0; // low-precision error folded into W(:,0) by plain restarts
  double cur_err = 0.0;   // low-precision error of the current W y
  bool cur_anchor = false;  // this iteration projects an FP64 anchor
  int knew = 1;             // basis size after a restart decided in phase_b
  bool did_restart = false;
  bool proj_fp64 = false;   // this iteration's projection is FP64-accurate
  bool ws_complete = false; // every workspace buffer was allocated (it may go to the plan)
  bool w0_ready = false;    // W(:,0) of the pending anchor was formed by the anchor update
  int anchor_updates = 0;   // anchors formed from the previous one (diagnostics)
};

namespace {

// DMRG_TRACE=1 in the environment prints one line per Davidson iteration to stderr
bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("DMRG_TRACE");
    on = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return on == 1;
}

dmrg_status read_small(dmrg_davidson_state* s, cudaStream_t st) {
  DMRG_CUDA_TRY(cudaMemcpyAsync(s->hsmall, s->small, sizeof(DevSmall), cudaMemcpyDeviceToHost, st));
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  return tc_error_status(s->plan);
}

// vector passes: FP64 units, double-float arithmetic on the FP32 units (vec_df.cu), or,
// in the mixed modes, FP64 for the anchor column and FP32 for the others (vec_split.cu)
int vec_mode(const dmrg_davidson_state* s) {
  const int a = s->plan->opt.vector_arith;
  if (a == DMRG_VEC_SPLIT) return s->mixed ? DMRG_VEC_SPLIT : DMRG_VEC_FP64;
  return a;
}
// the FP64 work column of the new direction t (basis column k without split storage)
double* tcol_of(dmrg_davidson_state* s, int k) { return s->f32 ? s->tbuf : s->V + (int64_t)k * s->ldv; }

// overlap with vec64 (FP64) or, with split storage, vec32 (an FP32 basis column)
dmrg_status ov(dmrg_davidson_state* s, int k, const double* vec64, const float* vec32,
               double* s_out, int Bcol, cudaStream_t st, const double* w0 = nullptr) {
  switch (vec_mode(s)) {
    case DMRG_VEC_SPLIT:
      return launch_overlap_split(s->vw, s->V, s->V32, s->ldv, s->n, k, vec64, vec32, s_out, s->small,
                                  Bcol, st, w0);
    case DMRG_VEC_DOUBLE_FLOAT:
      return launch_overlap_df(s->vw, s->V, s->ldv, s->n, k, vec64, s_out, s->small, Bcol, st, w0);
    default:
      return launch_overlap(s->vw, s->V, s->ldv, s->n, k, vec64, s_out, s->small, Bcol, st, w0);
  }
}
dmrg_status res(dmrg_davidson_state* s, int k, double* tcol, int mode, cudaStream_t st) {
  switch (vec_mode(s)) {
    case DMRG_VEC_SPLIT:
      return launch_residual_split(s->vw, s->V, s->W, s->V32, s->W32, s->D, s->ldv, s->n, k, tcol,
                                   s->small, mode, st);
    case DMRG_VEC_DOUBLE_FLOAT:
      return launch_residual_df(s->vw, s->V, s->W, s->D, s->ldv, s->n, k, tcol, s->small, mode, st);
    default:
      return launch_residual(s->vw, s->V, s->W, s->D, s->ldv, s->n, k, tcol, s->small, mode, st);
  }
}
dmrg_status cgs(dmrg_davidson_state* s, int k, double* tcol, int sin, int sout, int second,
                cudaStream_t st) {
  switch (vec_mode(s)) {
    case DMRG_VEC_SPLIT:
      return launch_cgs_split(s->vw, s->V, s->V32, s->ldv, s->n, k, tcol, s->small, sin, sout, st, second);
    case DMRG_VEC_DOUBLE_FLOAT:
      return launch_cgs_df(s->vw, s->V, s->ldv, s->n, k, tcol, s->small, sin, sout, st, second);
    default:
      return launch_cgs(s->vw, s->V, s->ldv, s->n, k, tcol, s->small, sin, sout, st, second);
  }
}

// normalise t; with split storage it is also appended as FP32 basis column k
dmrg_status fin(dmrg_davidson_state* s, int k, double* tcol, cudaStream_t st) {
  if (vec_mode(s) == DMRG_VEC_SPLIT)
    return launch_finish_split(s->vw, s->V, tcol, s->n, k, s->small, s->V32 + (int64_t)k * s->ldv, st);
  return launch_finish(tcol, s->n, s->small, st);
}

// x (and wx) = V y over the first k columns, into padded buffers
dmrg_status ritz(dmrg_davidson_state* s, int k, double* x, double* wx, cudaStream_t st) {
  if (s->f32)
    return launch_ritz_split(s->vw, s->V, s->W, s->V32, s->W32, s->ldv, s->n, k, s->small, x, wx, st);
  return launch_ritz(s->V, s->W, s->ldv, s->n, k, s->small, x, wx, st);
}

dmrg_status project_col(dmrg_davidson_state* s, int col, bool fp64, cudaStream_t st) {
  // FP64-accurate projections (FP64 mode, or an anchor of a mixed mode) use FP64 units
  // or the FP64-emulating tensor-core path, as the options say
  dmrg_precision prec = s->plan->opt.prec;
  if (s->f32 && col > 0) {
    // a low-precision column in FP32 storage (anchors are always column 0)
    if (fp64) {
      set_error("internal: FP64 projection of an FP32 basis column");
      return DMRG_ERR_INVALID_ARG;
    }
    DMRG_TRY(launch_project_tc32(s->plan, prec, s->V32 + (int64_t)col * s->ldv,
                                 s->W32 + (int64_t)col * s->ldv, st));
    s->projections++;
    return DMRG_OK;
  }
  if (fp64) prec = s->plan->opt.prec == DMRG_PREC_FP64_TC ? DMRG_PREC_FP64_TC : s->plan->opt.anchor_prec;
  DMRG_TRY(dmrg_project_prec(s->plan, prec, s->V + col * s->ldv, s->W + col * s->ldv, st));
  if (prec == DMRG_PREC_FP64 || prec == DMRG_PREC_FP64_TC) s->fp64_projections++;
  else s->projections++;
  return DMRG_OK;
}

}  // namespace

namespace dmrg {

void workspace_free(SolveWorkspace* w) {
  if (!w) return;
  cudaFree(w->V);
  cudaFree(w->W);
  cudaFree(w->V32);
  cudaFree(w->W32);
  cudaFree(w->tbuf);
  cudaFree(w->D);
  cudaFree(w->xbuf);
  cudaFree(w->wbuf);
  cudaFree(w->pbuf);
  cudaFree(w->wpbuf);
  cudaFree(w->small);
  cudaFreeHost(w->hsmall);
  vec_work_destroy(&w->vw);
  delete w;
}

}  // namespace dmrg

extern "C" {

dmrg_status dmrg_state_create(dmrg_plan* plan, const double* x0, void* stream,
                              dmrg_davidson_state** out) {
  if (!plan || !out || (!x0 && plan->n)) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (plan->n == 0) {
    set_error("empty superblock (n = 0)");
    return DMRG_ERR_SHAPE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  auto* s = new (std::nothrow) dmrg_davidson_state();
  if (!s) {
    set_error("host allocation failed");
    return DMRG_ERR_OOM;
  }
  s->plan = plan;
  s->n = plan->n;
  s->ldv = round_up(plan->n, 32);
  s->kmax = plan->opt.max_subspace;
  s->mixed = plan->opt.prec != DMRG_PREC_FP64 && plan->opt.prec != DMRG_PREC_FP64_TC &&
             plan->opt.fp64_refine;
  s->f32 = s->mixed && plan->opt.vector_arith == DMRG_VEC_SPLIT;
  auto fail = [&](dmrg_status e) { dmrg_state_destroy(s); return e; };
  const size_t col = sizeof(double) * (size_t)s->ldv;
  const size_t col32 = sizeof(float) * (size_t)s->ldv;
  const int cV = s->f32 ? 1 : s->kmax + 1, cW = s->f32 ? 1 : s->kmax;
  // the two spare vectors serve the two-vector restart and the anchor update (mixed modes)
  const bool keep2 = plan->opt.restart_keep == 2 || s->mixed;
  dmrg::SolveWorkspace* cached = nullptr;
  {
    std::lock_guard<std::mutex> g(plan->ws_mu);
    cached = plan->ws_cache;
    plan->ws_cache = nullptr;
  }
  if (cached && cached->ldv == s->ldv && cached->kmax == s->kmax && cached->f32 == s->f32 &&
      cached->keep2 == keep2) {
    // the previous state's buffers, same shape: no allocation
    s->V = cached->V;
    s->W = cached->W;
    s->V32 = cached->V32;
    s->W32 = cached->W32;
    s->tbuf = cached->tbuf;
    s->D = cached->D;
    s->xbuf = cached->xbuf;
    s->wbuf = cached->wbuf;
    s->pbuf = cached->pbuf;
    s->wpbuf = cached->wpbuf;
    s->small = cached->small;
    s->hsmall = cached->hsmall;
    s->vw = cached->vw;
    delete cached;
  } else {
    dmrg::workspace_free(cached);
    if (cudaMalloc((void**)&s->V, col * cV) != cudaSuccess ||
        cudaMalloc((void**)&s->W, col * cW) != cudaSuccess ||
        (s->f32 && (cudaMalloc((void**)&s->V32, col32 * (s->kmax + 1)) != cudaSuccess ||
                    cudaMalloc((void**)&s->W32, col32 * s->kmax) != cudaSuccess ||
                    cudaMalloc((void**)&s->tbuf, col) != cudaSuccess)) ||
        cudaMalloc((void**)&s->D, col) != cudaSuccess ||
        cudaMalloc((void**)&s->xbuf, col) != cudaSuccess ||
        cudaMalloc((void**)&s->wbuf, col) != cudaSuccess ||
        (keep2 && (cudaMalloc((void**)&s->pbuf, col) != cudaSuccess ||
                   cudaMalloc((void**)&s->wpbuf, col) != cudaSuccess)) ||
        cudaMalloc((void**)&s->small, sizeof(DevSmall)) != cudaSuccess ||
        cudaMallocHost((void**)&s->hsmall, sizeof(DevSmall)) != cudaSuccess) {
      cudaGetLastError();
      set_error("allocation of the Davidson workspace (%zu bytes) failed",
                col * (2 * s->kmax + 6));
      return fail(DMRG_ERR_OOM);
    }
    const dmrg_status ev = vec_work_create(&s->vw);
    if (ev != DMRG_OK) return fail(ev);
  }
  s->ws_complete = true;
  dmrg_status e = DMRG_OK;
  if (cudaMemsetAsync(s->V, 0, col * cV, st) != cudaSuccess ||
      cudaMemsetAsync(s->W, 0, col * cW, st) != cudaSuccess ||
      (s->f32 && (cudaMemsetAsync(s->V32, 0, col32 * (s->kmax + 1), st) != cudaSuccess ||
                  cudaMemsetAsync(s->W32, 0, col32 * s->kmax, st) != cudaSuccess ||
                  cudaMemsetAsync(s->tbuf, 0, col, st) != cudaSuccess)) ||
      cudaMemsetAsync(s->D, 0, col, st) != cudaSuccess ||
      cudaMemsetAsync(s->xbuf, 0, col, st) != cudaSuccess ||
      cudaMemsetAsync(s->wbuf, 0, col, st) != cudaSuccess ||
      cudaMemsetAsync(s->small, 0, sizeof(DevSmall), st) != cudaSuccess ||
      cudaMemcpyAsync(s->D, plan->D, sizeof(double) * s->n, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess) {
    set_error("workspace initialisation failed");
    return fail(DMRG_ERR_CUDA);
  }
  if ((e = launch_normalize(s->vw, x0, s->V, s->n, s->small, st)) != DMRG_OK) return fail(e);
  if ((e = read_small(s, st)) != DMRG_OK) return fail(e);
  if (!(s->hsmall->nrm2 > 0.0) || !std::isfinite(s->hsmall->nrm2)) {
    set_error("start vector has zero or non-finite norm");
    return fail(DMRG_ERR_INVALID_ARG);
  }
  s->k = 1;
  *out = s;
  return DMRG_OK;
}

void dmrg_state_destroy(dmrg_davidson_state* s) {
  if (!s) return;
  if (s->ws_complete && s->plan) {
    // hand the buffers to the plan for the next state, once no kernel uses them (the
    // device-wide wait is the one a cudaFree would make)
    auto* w = new (std::nothrow) dmrg::SolveWorkspace();
    if (w && cudaDeviceSynchronize() == cudaSuccess) {
      w->ldv = s->ldv;
      w->kmax = s->kmax;
      w->f32 = s->f32;
      w->keep2 = s->plan->opt.restart_keep == 2 || s->mixed;
      w->V = s->V;
      w->W = s->W;
      w->V32 = s->V32;
      w->W32 = s->W32;
      w->tbuf = s->tbuf;
      w->D = s->D;
      w->xbuf = s->xbuf;
      w->wbuf = s->wbuf;
      w->pbuf = s->pbuf;
      w->wpbuf = s->wpbuf;
      w->small = s->small;
      w->hsmall = s->hsmall;
      w->vw = s->vw;
      {
        std::lock_guard<std::mutex> g(s->plan->ws_mu);
        std::swap(w, s->plan->ws_cache);
      }
      dmrg::workspace_free(w);  // the workspace this one displaced, if any
      delete s;
      return;
    }
    cudaGetLastError();
    delete w;
  }
  cudaFree(s->V);
  cudaFree(s->W);
  cudaFree(s->V32);
  cudaFree(s->W32);
  cudaFree(s->tbuf);
  cudaFree(s->D);
  cudaFree(s->xbuf);
  cudaFree(s->wbuf);
  cudaFree(s->pbuf);
  cudaFree(s->wpbuf);
  cudaFree(s->small);
  cudaFreeHost(s->hsmall);
  vec_work_destroy(&s->vw);
  delete s;
}

}  // extern "C"

namespace {

// A Davidson iteration runs in three host phases so that a batch of problems can share
// each host synchronisation:
//   phase_a  enqueue projection, overlap, Jacobi, residual; copy the small state back
//   phase_b  (after a sync) read lambda, ||r||; decide convergence / anchor / restart;
//            enqueue Gram-Schmidt and normalisation; copy the small state back
//   phase_c  (after a sync) check for a basis breakdown, append the new column
// phase_a in three parts, so that a batch can group the low-precision projections:
// begin decides the projection arithmetic (true: a low-precision one), project runs it,
// end enqueues the rest of the phase
// Digits of the FP64_TC split for the anchor update of a collapse at basis size k, or 0
// for a full projection of the new anchor.  The update applies when column 0 of V and W is
// an FP64-accurate pair (an anchor, no plain restart since), the anchors run on the
// FP64_TC path, and the update is cheaper: with ||d|| = ||y(1:)|| (orthonormal columns),
// the leading `digits` digits of both stages give an error of about 2^(4 - 7 digits) ||H||
// ||d|| (truncation of the operands and of the stage-1 results, with a margin of 8), held
// below 2^-46 ||H||, the accuracy of a full FP64_TC projection.
int anchor_update_digits(const dmrg_davidson_state* s, int k) {
  if (!s->mixed || !s->anchored || s->plain_restarts != 0 || k < 2) return 0;
  if (s->plan->opt.anchor_prec != DMRG_PREC_FP64_TC || !s->plan->opt.anchor_update) return 0;
  double t2 = 0.0;
  for (int j = 1; j < k; ++j) t2 += s->hsmall->y[j] * s->hsmall->y[j];
  const double ytail = std::sqrt(t2);
  if (!(ytail > 0.0)) return 2;
  const int digits = (int)std::ceil((50.0 + std::log2(ytail)) / 7.0);
  if (digits >= 7) return 0;
  return std::max(2, digits);
}

bool phase_a_begin(dmrg_davidson_state* s) {
  const bool anchor = s->mixed && s->anchor_pending;
  if (anchor) s->anchored = true;
  s->cur_anchor = anchor;
  const bool fp64 = !s->mixed && (s->plan->opt.prec == DMRG_PREC_FP64 ||
                                   s->plan->opt.prec == DMRG_PREC_FP64_TC);
  s->proj_fp64 = fp64 || anchor;
  s->anchor_pending = false;
  return !s->proj_fp64;
}

dmrg_status phase_a_project(dmrg_davidson_state* s, cudaStream_t st) {
  if (s->w0_ready) {  // the anchor's projection was formed in phase_b
    s->w0_ready = false;
    return DMRG_OK;
  }
  return project_col(s, s->k - 1, s->proj_fp64, st);
}

dmrg_status phase_a_end(dmrg_davidson_state* s, cudaStream_t st) {
  const int64_t ldv = s->ldv;
  const int k = s->k, col = k - 1;
  // after an FP64 anchor, the anchor row of B comes from the exact column W(:,0)
  const double* w0 = (s->mixed && s->anchored) ? s->W : nullptr;
  if (s->f32 && col > 0) DMRG_TRY(ov(s, k, nullptr, s->W32 + col * ldv, nullptr, col, st, w0));
  else DMRG_TRY(ov(s, k, s->W + col * ldv, nullptr, nullptr, col, st, w0));
  DMRG_TRY(launch_jacobi(s->small, k, st));
  DMRG_TRY(res(s, k, tcol_of(s, k), 0, st));
  DMRG_CUDA_TRY(cudaMemcpyAsync(s->hsmall, s->small, sizeof(DevSmall), cudaMemcpyDeviceToHost, st));
  return DMRG_OK;
}

dmrg_status phase_a(dmrg_davidson_state* s, cudaStream_t st) {
  phase_a_begin(s);
  DMRG_TRY(phase_a_project(s, st));
  return phase_a_end(s, st);
}

dmrg_status phase_b(dmrg_davidson_state* s, cudaStream_t st, bool* need_c) {
  *need_c = false;
  DMRG_TRY(tc_error_status(s->plan));
  const int64_t ldv = s->ldv, n = s->n;
  const int k = s->k;
  const bool anchor = s->cur_anchor;
  const bool fp64 = !s->mixed && (s->plan->opt.prec == DMRG_PREC_FP64 ||
                                   s->plan->opt.prec == DMRG_PREC_FP64_TC);
  double* tcol = tcol_of(s, k);
  s->iters++;
  s->sweeps += s->hsmall->jacobi_sweeps;
  s->lambda = s->hsmall->lambda;
  s->rnorm = std::sqrt(std::max(0.0, s->hsmall->rnorm2));
  if (s->hsmall->flags & 2 || !std::isfinite(s->lambda)) {
    set_error("non-finite residual or eigenvalue at iteration %d", s->iters);
    return DMRG_ERR_NUMERIC;
  }
  const double tol = s->plan->opt.tol;
  const bool exact = !s->mixed || anchor;  // residual computed from FP64 projections only
  const bool lowprec_plain = !fp64 && !s->mixed;
  if (s->mixed && k == 1) s->anchor_rnorm = s->rnorm;
  s->ritz_k = k;
  if (s->rnorm <= tol && (exact || lowprec_plain)) {
    s->converged = true;
    return DMRG_OK;
  }
  bool do_anchor = false, do_restart = false;
  if (s->mixed) {
    // estimated floor of the low-precision residual: eps * ||H|| * ||y(1:)||, the error
    // the low-precision columns contribute to W y (||y(1:)|| = 1 before the first anchor;
    // ||H|| from the extreme Ritz values); anchor when the computed residual has come
    // within a factor 10 of it, or below tol, or (optional) below refine_ratio times the
    // last exact residual
    const DevSmall& h = *s->hsmall;
    double hnorm = 0.0, ytail = 0.0;
    for (int j = 0; j < k; ++j) hnorm = std::max(hnorm, std::fabs(h.theta[j]));
    for (int j = 1; j < k; ++j) ytail += h.y[j] * h.y[j];
    ytail = s->anchored ? std::sqrt(ytail) : 1.0;
    // relative error of one low-precision projection, measured against FP64 at the full
    // workload sizes (BF16x3: 5e-6 of max|y|, FP32 accumulation over K ~ 1e3; BF16x2:
    // operands to 2^-18 and the dropped x1 y1 product, 3e-5; TF32: 1e-3)
    const dmrg_precision lp = s->plan->opt.prec;
    const double eps = lp == DMRG_PREC_TF32 ? 2e-3 : lp == DMRG_PREC_BF16X2 ? 3e-5 : 5e-6;
    // a plain restart folds the current low-precision error of W y into W(:,0): it stays
    // in the floor until the next FP64 anchor
    const double floor_est = eps * hnorm * ytail + s->baked_err;
    s->floor_est = floor_est;
    s->cur_err = eps * hnorm * ytail;
    const double ratio = s->plan->opt.refine_ratio;
    if (s->rnorm <= tol || (k > 1 && s->rnorm <= 10.0 * floor_est) ||
        (k > 1 && ratio > 0.0 && s->rnorm <= ratio * s->anchor_rnorm))
      do_anchor = true;
    if (trace_on())
      fprintf(stderr, "dmrg it %4d k %2d %s lambda % .15f r %.3e floor %.3e ytail %.2e sweeps %d "
              "eig cycles %lld/%lld/%lld fallbacks %d%s\n",
              s->iters, k, anchor ? "FP64" : "lp  ", s->lambda, s->rnorm, floor_est, ytail,
              h.jacobi_sweeps, (long long)h.eig_cycles[0], (long long)h.eig_cycles[1],
              (long long)h.eig_cycles[2], h.eig_fallbacks, do_anchor ? "  -> anchor" : "");
  } else if (trace_on()) {
    fprintf(stderr, "dmrg it %4d k %2d lambda % .15f r %.3e sweeps %d fallbacks %d\n", s->iters, k,
            s->lambda, s->rnorm, s->hsmall->jacobi_sweeps, s->hsmall->eig_fallbacks);
  }
  if (k == s->kmax && !do_anchor) {
    // subspace limit: a plain restart keeps W y, whose low-precision error is of the
    // order of the current floor.  It becomes an FP64 anchor instead when the residual
    // is already within a factor 100 of the floor, or when it has not halved since the
    // previous subspace-limit restart (a stalled low-precision phase)
    if (s->mixed && (s->rnorm <= 100.0 * s->floor_est || s->rnorm > 0.5 * s->restart_rnorm))
      do_anchor = true;
    else
      do_restart = true;
    s->restart_rnorm = s->rnorm;
  }
  if (do_anchor) {
    // collapse to the normalised Ritz vector; its projection is redone FP64-accurately
    DMRG_TRY(ritz(s, k, s->xbuf, nullptr, st));
    const int digits = anchor_update_digits(s, k);
    if (digits > 0) {
      // anchor update: x = y_0 v_0 + d with H v_0 = W(:,0) exact (FP64-accurate, no plain
      // restart since), so H x = y_0 W(:,0) + H d, and H d needs accuracy relative to ||d||
      // only: it runs with the leading `digits` digits of the FP64_TC split
      const double y0 = s->hsmall->y[0];
      DMRG_TRY(launch_axpby(s->vw, s->xbuf, -y0, s->V, s->pbuf, n, st));        // d
      DMRG_TRY(launch_project_oz(s->plan, s->pbuf, s->wpbuf, st, digits));       // H d
      DMRG_TRY(launch_axpby(s->vw, s->wpbuf, y0, s->W, s->wbuf, n, st));        // H x
      DMRG_TRY(launch_normalize(s->vw, s->xbuf, s->V, n, s->small, st));
      DMRG_TRY(launch_scale_copy(s->vw, s->wbuf, s->W, n, s->small, st));        // / ||x||
      s->fp64_projections++;
      s->anchor_updates++;
      s->w0_ready = true;
      if (trace_on()) fprintf(stderr, "dmrg anchor update with %d digits\n", digits);
    } else {
      DMRG_TRY(launch_normalize(s->vw, s->xbuf, s->V, n, s->small, st));
    }
    s->k = 1;
    s->restarts++;
    s->anchor_pending = true;
    s->plain_restarts = 0;
    s->restart_rnorm = INFINITY;
    s->baked_err = 0.0;
    s->ritz_k = 0;
    return DMRG_OK;
  }
  int knew = k;
  // two-vector restart (restart_keep = 2): keep x and the previous iteration's Ritz vector,
  // orthogonalised against x in coefficient space (c2 = y_prev - y (y . y_prev), twice)
  double c2[KMAX] = {0.0};
  bool keep2 = false;
  if (do_restart && s->plan->opt.restart_keep == 2 && k >= 2) {
    const DevSmall& h = *s->hsmall;
    for (int j = 0; j < k - 1; ++j) c2[j] = h.y_prev[j];
    for (int pass = 0; pass < 2; ++pass) {
      double a = 0.0;
      for (int j = 0; j < k; ++j) a += h.y[j] * c2[j];
      for (int j = 0; j < k; ++j) c2[j] -= a * h.y[j];
    }
    double nrm = 0.0;
    for (int j = 0; j < k; ++j) nrm += c2[j] * c2[j];
    nrm = std::sqrt(nrm);
    if (nrm > 1e-8) {
      keep2 = true;
      for (int j = 0; j < k; ++j) c2[j] /= nrm;
    }
  }
  if (keep2) {
    // V = [x, p], W = [W y, W c2]; B(0,0) = lambda here, B(:,1) from an overlap after p is
    // re-orthonormalised against x in FP64 (the low-precision columns of the old basis are
    // orthonormal only to FP32 in the split arithmetic); the correction t is kept
    DevSmall& h = *s->hsmall;
    for (int j = 0; j < KMAX; ++j) {
      h.C[0][j] = j < k ? h.y[j] : 0.0;
      h.C[1][j] = j < k ? c2[j] : 0.0;
    }
    for (int j = 0; j < KMAX * KMAX; ++j) h.B[j] = 0.0;
    h.B[0] = s->lambda;
    for (int j = 0; j < KMAX; ++j) h.y[j] = j == 0 ? 1.0 : 0.0;
    h.qk = 0;  // the next small eigenproblem starts cold
    DMRG_CUDA_TRY(cudaMemcpyAsync(s->small, s->hsmall, sizeof(DevSmall), cudaMemcpyHostToDevice, st));
    const size_t bytes = sizeof(double) * n;
    const double* w0 = (s->mixed && s->anchored) ? s->W : nullptr;
    if (s->f32) {
      // p orthonormalised against x in FP64 before it is rounded into FP32 column 1
      DMRG_TRY(launch_ritz2_split(s->vw, s->V, s->W, s->V32, s->W32, ldv, n, k, s->small, s->xbuf,
                                  s->pbuf, s->wbuf, s->wpbuf, st));
      DMRG_TRY(launch_orth_pair(s->vw, s->pbuf, s->wpbuf, s->xbuf, s->wbuf, n, s->small, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->V, s->xbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->W, s->wbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_TRY(launch_convert32(s->vw, s->pbuf, s->V32 + ldv, n, st));
      DMRG_TRY(launch_convert32(s->vw, s->wpbuf, s->W32 + ldv, n, st));
      DMRG_TRY(ov(s, 2, nullptr, s->W32 + ldv, nullptr, 1, st, w0));
    } else {
      DMRG_TRY(launch_ritz2(s->V, s->W, ldv, n, k, s->small, s->xbuf, s->pbuf, s->wbuf, s->wpbuf, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->V, s->xbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->V + ldv, s->pbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->W, s->wbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->W + ldv, s->wpbuf, bytes, cudaMemcpyDeviceToDevice, st));
      DMRG_TRY(launch_orth_pair(s->vw, s->V + ldv, s->W + ldv, s->V, s->W, n, s->small, st));
      DMRG_TRY(ov(s, 2, s->W + ldv, nullptr, nullptr, 1, st, w0));
    }
    knew = 2;
    s->restarts++;
    s->plain_restarts++;
    s->baked_err += s->cur_err;
    s->ritz_k = 0;
    DMRG_TRY(ov(s, knew, tcol, nullptr, s->small->s[0], -1, st));
  } else if (do_restart) {
    // V = [x], W = [W y], B = [lambda]; the correction t (column k) is kept
    DMRG_TRY(ritz(s, k, s->xbuf, s->wbuf, st));
    DMRG_CUDA_TRY(cudaMemcpyAsync(s->V, s->xbuf, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    DMRG_CUDA_TRY(cudaMemcpyAsync(s->W, s->wbuf, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    DMRG_TRY(launch_set_B00(s->small, st));
    knew = 1;
    s->restarts++;
    s->plain_restarts++;
    s->baked_err += s->cur_err;
    s->ritz_k = 0;
    DMRG_TRY(ov(s, knew, tcol, nullptr, s->small->s[0], -1, st));
  }
  s->knew = knew;
  s->did_restart = do_restart;  // (after a restart y = e_1 in the new basis)
  // classical Gram-Schmidt (second pass only when needed), then normalise
  DMRG_CUDA_TRY(cudaMemsetAsync(&s->small->flags, 0, sizeof(int32_t), st));
  DMRG_TRY(cgs(s, knew, tcol, 0, 1, 0, st));
  DMRG_TRY(cgs(s, knew, tcol, 1, 2, 1, st));
  DMRG_TRY(fin(s, knew, tcol, st));
  DMRG_CUDA_TRY(cudaMemcpyAsync(s->hsmall, s->small, sizeof(DevSmall), cudaMemcpyDeviceToHost, st));
  *need_c = true;
  return DMRG_OK;
}

dmrg_status phase_c(dmrg_davidson_state* s, cudaStream_t st) {
  const int64_t ldv = s->ldv;
  const int k = s->k, knew = s->knew;
  double* tcol = tcol_of(s, k);
  if (s->hsmall->flags & 1) {
    // breakdown: fall back to the raw residual r (mode 1 writes t = r); after a restart
    // the basis is [x] with W = [W y], so r = W(:,0) - lambda V(:,0)
    if (s->did_restart) {
      static const double e1[KMAX] = {1.0};
      DMRG_CUDA_TRY(cudaMemcpyAsync(s->small->y, e1, sizeof(e1), cudaMemcpyHostToDevice, st));
    }
    DMRG_TRY(res(s, knew, tcol, 1, st));
    DMRG_CUDA_TRY(cudaMemsetAsync(&s->small->flags, 0, sizeof(int32_t), st));
    DMRG_TRY(cgs(s, knew, tcol, 0, 1, 0, st));
    DMRG_TRY(cgs(s, knew, tcol, 1, 2, 1, st));
    DMRG_TRY(fin(s, knew, tcol, st));
    DMRG_TRY(read_small(s, st));
    if (s->hsmall->flags & 1) {
      set_error("Davidson basis breakdown at iteration %d (||r|| = %g)", s->iters, s->rnorm);
      return DMRG_ERR_NUMERIC;
    }
  }
  if (knew != k && !s->f32) {  // (split storage: the normalisation wrote column knew)
    DMRG_CUDA_TRY(cudaMemcpyAsync(s->V + (int64_t)knew * ldv, tcol, sizeof(double) * ldv,
                                  cudaMemcpyDeviceToDevice, st));
  }
  s->k = knew + 1;
  return DMRG_OK;
}

}  // namespace

extern "C" {

dmrg_status dmrg_davidson_step(dmrg_davidson_state* s, void* stream, int32_t* converged) {
  if (!s) {
    set_error("NULL state");
    return DMRG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (converged) *converged = s->converged ? 1 : 0;
  if (s->converged) return DMRG_OK;
  DMRG_TRY(phase_a(s, st));
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  bool need_c = false;
  DMRG_TRY(phase_b(s, st, &need_c));
  if (need_c) {
    DMRG_CUDA_TRY(cudaStreamSynchronize(st));
    DMRG_TRY(phase_c(s, st));
  }
  if (converged) *converged = s->converged ? 1 : 0;
  return DMRG_OK;
}

dmrg_status dmrg_state_get_info(const dmrg_davidson_state* s, dmrg_solve_info* info) {
  if (!s || !info) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  info->energy = s->lambda;
  info->resnorm = s->rnorm;
  info->iters = s->iters;
  info->projections = s->projections;
  info->fp64_projections = s->fp64_projections;
  info->restarts = s->restarts;
  info->small_eig_sweeps = s->sweeps;
  info->converged = s->converged ? 1 : 0;
  info->anchor_updates = s->anchor_updates;
  return DMRG_OK;
}

dmrg_status dmrg_state_ritz(dmrg_davidson_state* s, double* x_out, void* stream) {
  if (!s || !x_out) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  if (s->ritz_k == 0) {  // the basis was collapsed onto the Ritz vector
    DMRG_CUDA_TRY(cudaMemcpyAsync(x_out, s->V, sizeof(double) * s->n, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
    return DMRG_OK;
  }
  if (s->f32) {  // (padded work buffer first: x_out holds exactly n elements)
    DMRG_TRY(ritz(s, s->ritz_k, s->xbuf, nullptr, (cudaStream_t)stream));
    DMRG_CUDA_TRY(cudaMemcpyAsync(x_out, s->xbuf, sizeof(double) * s->n, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
    return DMRG_OK;
  }
  return launch_ritz(s->V, s->W, s->ldv, s->n, s->ritz_k, s->small, x_out, nullptr,
                     (cudaStream_t)stream);
}

dmrg_status dmrg_davidson_solve(dmrg_plan* plan, const double* x0, double* x_out,
                                dmrg_solve_info* info, void* stream) {
  if (!plan || !x0 || !x_out) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  dmrg_davidson_state* s = nullptr;
  DMRG_TRY(dmrg_state_create(plan, x0, stream, &s));
  dmrg_status e = DMRG_OK;
  int32_t conv = 0;
  while (!conv && s->iters < plan->opt.max_iter) {
    e = dmrg_davidson_step(s, stream, &conv);
    if (e != DMRG_OK) break;
  }
  if (e == DMRG_OK) e = dmrg_state_ritz(s, x_out, stream);
  if (info) dmrg_state_get_info(s, info);
  if (e == DMRG_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    set_error("solve: %s", cudaGetErrorString(cudaGetLastError()));
    e = DMRG_ERR_CUDA;
  }
  if (e == DMRG_OK && !conv) {
    set_error("Davidson did not converge in %d iterations (||r|| = %g)", s->iters, s->rnorm);
    e = DMRG_ERR_NOT_CONVERGED;
  }
  dmrg_state_destroy(s);
  return e;
}

dmrg_status dmrg_davidson_solve_host(dmrg_plan* plan, const double* x0_host,
                                     double* x_out_host, dmrg_solve_info* info, void* stream) {
  if (!plan || !x0_host || !x_out_host) {
    set_error("NULL argument");
    return DMRG_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *dx0 = nullptr, *dx = nullptr;
  {
    // the device vectors of the previous call, if no other call holds them
    std::lock_guard<std::mutex> g(plan->ws_mu);
    std::swap(dx0, plan->io_x0);
    std::swap(dx, plan->io_x);
  }
  const size_t bytes = sizeof(double) * (size_t)plan->n;
  if ((!dx0 && cudaMalloc((void**)&dx0, bytes) != cudaSuccess) ||
      (!dx && cudaMalloc((void**)&dx, bytes) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(dx0);
    cudaFree(dx);
    set_error("allocation of the solve vectors failed");
    return DMRG_ERR_OOM;
  }
  dmrg_status e = DMRG_OK;
  if (cudaMemcpyAsync(dx0, x0_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_error("host-to-device copy of x0 failed");
    e = DMRG_ERR_CUDA;
  }
  if (e == DMRG_OK) e = dmrg_davidson_solve(plan, dx0, dx, info, stream);
  bool idle = false;
  if (e == DMRG_OK || e == DMRG_ERR_NOT_CONVERGED) {
    if (cudaMemcpyAsync(x_out_host, dx, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("device-to-host copy of x failed");
      e = DMRG_ERR_CUDA;
    } else {
      idle = true;
    }
  }
  if (idle) {
    // nothing of this call is in flight: the vectors go back to the plan
    std::lock_guard<std::mutex> g(plan->ws_mu);
    if (!plan->io_x0 && !plan->io_x) {
      plan->io_x0 = dx0;
      plan->io_x = dx;
      dx0 = dx = nullptr;
    }
  }
  cudaFree(dx0);
  cudaFree(dx);
  return e;
}

dmrg_status dmrg_plan_trim(dmrg_plan* plan) {
  if (!plan) {
    set_error("NULL plan");
    return DMRG_ERR_INVALID_ARG;
  }
  dmrg::SolveWorkspace* w = nullptr;
  double *a = nullptr, *b = nullptr;
  {
    std::lock_guard<std::mutex> g(plan->ws_mu);
    std::swap(w, plan->ws_cache);
    std::swap(a, plan->io_x0);
    std::swap(b, plan->io_x);
  }
  dmrg::workspace_free(w);
  cudaFree(a);
  cudaFree(b);
  return DMRG_OK;
}

dmrg_status dmrg_gemv_trans(const double* V, int64_t ldv, int64_t n, int32_t k,
                            const double* w, double* s, void* stream) {
  if ((n > 0 && (!V || !w)) || !s || n < 0 || k < 1 || k > DMRG_MAX_SUBSPACE || ldv < n) {
    set_error("dmrg_gemv_trans: bad argument (k must be in [1, %d], ldv >= n)", DMRG_MAX_SUBSPACE);
    return DMRG_ERR_INVALID_ARG;
  }
  return launch_gemv_trans_public(V, ldv, n, k, w, s, (cudaStream_t)stream);
}


dmrg_status dmrg_davidson_solve_batched(dmrg_plan* const* plans, int32_t nb,
                                        const double* const* x0, double* const* x_out,
                                        dmrg_solve_info* infos, void* stream) {
  if (nb < 0 || (nb > 0 && (!plans || !x0 || !x_out))) {
    set_error("dmrg_davidson_solve_batched: bad argument");
    return DMRG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < nb; ++i) {
    if (!plans[i] || !x0[i] || !x_out[i]) {
      set_error("dmrg_davidson_solve_batched: NULL plan or vector at index %d", i);
      return DMRG_ERR_INVALID_ARG;
    }
  }
  if (nb == 0) return DMRG_OK;
  cudaStream_t caller = (cudaStream_t)stream;
  std::vector<cudaStream_t> sts(nb, nullptr);
  std::vector<dmrg_davidson_state*> states(nb, nullptr);
  std::vector<char> active(nb, 1);
  std::vector<dmrg_status> status(nb, DMRG_OK);
  cudaEvent_t start_ev = nullptr;
  dmrg_status err = DMRG_OK;
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(start_ev, caller) != cudaSuccess) {
    set_error("dmrg_davidson_solve_batched: event creation failed");
    cudaEventDestroy(start_ev);
    return DMRG_ERR_CUDA;
  }
  // one stream per distinct plan: a plan's projection scratch (operand images,
  // intermediates) is shared by every projection made with it, so problems that share a
  // plan are kept in order on one stream; problems with their own plans overlap
  std::vector<cudaStream_t> owned;
  std::vector<const dmrg_plan*> owner;
  for (int i = 0; i < nb && err == DMRG_OK; ++i) {
    int found = -1;
    for (size_t u = 0; u < owner.size(); ++u)
      if (owner[u] == plans[i]) found = (int)u;
    if (found < 0) {
      cudaStream_t ns = nullptr;
      if (cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(ns, start_ev, 0) != cudaSuccess) {
        set_error("dmrg_davidson_solve_batched: stream creation failed");
        if (ns) cudaStreamDestroy(ns);
        err = DMRG_ERR_CUDA;
        break;
      }
      owned.push_back(ns);
      owner.push_back(plans[i]);
      found = (int)owned.size() - 1;
    }
    sts[i] = owned[found];
    err = dmrg_state_create(plans[i], x0[i], sts[i], &states[i]);
  }
  // Grouped projections: when every problem has its own plan and all plans project in the
  // same tensor-core precision, the low-precision projections of one lockstep phase run as
  // one pack launch and one launch per GEMM stage on a batch stream (TcBatch); FP64 and
  // FP64-accurate anchor projections stay on the problems' streams.
  TcBatch* batch = nullptr;
  cudaStream_t bst = nullptr;
  cudaEvent_t bdone = nullptr;
  std::vector<cudaEvent_t> ready(nb, nullptr);
  const dmrg_precision p0 = nb > 0 ? plans[0]->opt.prec : DMRG_PREC_FP64;
  bool group = err == DMRG_OK && nb >= 2 && (int)owned.size() == nb && tc_lowprec(p0);
  for (int i = 0; i < nb && group; ++i) group = plans[i]->opt.prec == p0;
  if (group) {
    if (cudaStreamCreateWithFlags(&bst, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(bst, start_ev, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&bdone, cudaEventDisableTiming) != cudaSuccess) {
      set_error("dmrg_davidson_solve_batched: stream creation failed");
      err = DMRG_ERR_CUDA;
    }
    for (int i = 0; i < nb && err == DMRG_OK; ++i)
      if (cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming) != cudaSuccess) {
        set_error("dmrg_davidson_solve_batched: event creation failed");
        err = DMRG_ERR_CUDA;
      }
    if (err == DMRG_OK) err = tc_batch_create(plans, nb, p0, bst, &batch);
  }
  std::vector<const double*> bx(nb, nullptr);
  std::vector<double*> by(nb, nullptr);
  std::vector<const float*> bx32(nb, nullptr);
  std::vector<float*> by32(nb, nullptr);
  std::vector<char> lp(nb, 0);
  // lockstep: every phase is enqueued for all active problems before one wait for all
  for (int it = 0; err == DMRG_OK; ++it) {
    bool any = false, any_lp = false;
    for (int i = 0; i < nb; ++i) {
      lp[i] = 0;
      if (!active[i]) continue;
      if (states[i]->converged || states[i]->iters >= plans[i]->opt.max_iter) {
        active[i] = 0;
        continue;
      }
      any = true;
      dmrg_davidson_state* s = states[i];
      const bool is_lp = phase_a_begin(s);
      if (batch && is_lp) {
        lp[i] = 1;
        any_lp = true;
        const int64_t c = s->k - 1;
        bx[i] = s->V + c * s->ldv;
        by[i] = s->W + c * s->ldv;
        bx32[i] = (s->f32 && c > 0) ? s->V32 + c * s->ldv : nullptr;
        by32[i] = (s->f32 && c > 0) ? s->W32 + c * s->ldv : nullptr;
        if (cudaEventRecord(ready[i], sts[i]) != cudaSuccess ||
            cudaStreamWaitEvent(bst, ready[i], 0) != cudaSuccess) {
          set_error("dmrg_davidson_solve_batched: event record failed");
          err = DMRG_ERR_CUDA;
        }
        continue;
      }
      status[i] = phase_a_project(s, sts[i]);
      if (status[i] == DMRG_OK) status[i] = phase_a_end(s, sts[i]);
      if (status[i] != DMRG_OK) active[i] = 0;
    }
    if (err != DMRG_OK) break;
    if (any_lp) {
      err = tc_batch_project(batch, bx.data(), by.data(), bx32.data(), by32.data(), lp.data(), bst);
      if (err == DMRG_OK && cudaEventRecord(bdone, bst) != cudaSuccess) {
        set_error("dmrg_davidson_solve_batched: event record failed");
        err = DMRG_ERR_CUDA;
      }
      for (int i = 0; i < nb && err == DMRG_OK; ++i) {
        if (!lp[i]) continue;
        states[i]->projections++;
        if (cudaStreamWaitEvent(sts[i], bdone, 0) != cudaSuccess) {
          set_error("dmrg_davidson_solve_batched: stream wait failed");
          err = DMRG_ERR_CUDA;
          break;
        }
        status[i] = phase_a_end(states[i], sts[i]);
        if (status[i] != DMRG_OK) active[i] = 0;
      }
      if (err != DMRG_OK) break;
    }
    if (!any) break;
    std::vector<char> need_c(nb, 0);
    for (int i = 0; i < nb; ++i) {
      if (!active[i]) continue;
      if (cudaStreamSynchronize(sts[i]) != cudaSuccess) {
        set_error("dmrg_davidson_solve_batched: %s", cudaGetErrorString(cudaGetLastError()));
        err = DMRG_ERR_CUDA;
        break;
      }
      bool c = false;
      if (batch && tc_batch_error(batch) != DMRG_OK) {
        err = DMRG_ERR_CUDA;
        break;
      }
      status[i] = phase_b(states[i], sts[i], &c);
      need_c[i] = c;
      if (status[i] != DMRG_OK) active[i] = 0;
    }
    if (err != DMRG_OK) break;
    for (int i = 0; i < nb; ++i) {
      if (!active[i] || !need_c[i]) continue;
      if (cudaStreamSynchronize(sts[i]) != cudaSuccess) {
        set_error("dmrg_davidson_solve_batched: %s", cudaGetErrorString(cudaGetLastError()));
        err = DMRG_ERR_CUDA;
        break;
      }
      status[i] = phase_c(states[i], sts[i]);
      if (status[i] != DMRG_OK) active[i] = 0;
    }
  }
  bool all_converged = true;
  for (int i = 0; i < nb; ++i) {
    if (!states[i]) {
      all_converged = false;
      continue;
    }
    dmrg_status r = dmrg_state_ritz(states[i], x_out[i], sts[i]);
    if (status[i] == DMRG_OK) status[i] = r;
    if (infos) {
      dmrg_state_get_info(states[i], &infos[i]);
      infos[i].converged = states[i]->converged ? 1 : 0;
    }
    if (!states[i]->converged) all_converged = false;
    if (err == DMRG_OK && status[i] != DMRG_OK) err = status[i];
  }
  for (cudaStream_t os : owned) {
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, os);
      cudaStreamWaitEvent(caller, done, 0);
      cudaEventDestroy(done);
    }
    cudaStreamSynchronize(os);
  }
  if (bst) cudaStreamSynchronize(bst);
  tc_batch_destroy(batch);
  for (cudaEvent_t e : ready)
    if (e) cudaEventDestroy(e);
  if (bdone) cudaEventDestroy(bdone);
  if (bst) cudaStreamDestroy(bst);
  for (int i = 0; i < nb; ++i) dmrg_state_destroy(states[i]);
  for (cudaStream_t os : owned) cudaStreamDestroy(os);
  cudaEventDestroy(start_ev);
  if (err == DMRG_OK && !all_converged) {
    set_error("dmrg_davidson_solve_batched: at least one problem did not converge");
    err = DMRG_ERR_NOT_CONVERGED;
  }
  return err;
}

}  // extern "C"
