// Error reporting, option defaults and the small C-ABI helpers.
#include <stdarg.h>

#include <atomic>
#include <stdio.h>

#include "internal.h"

namespace dmrg {

static thread_local char g_last_error[1024] = "";
static std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

}  // namespace dmrg

extern "C" {

void dmrg_options_default(dmrg_options* opt) {
  if (!opt) return;
  opt->prec = DMRG_PREC_FP64;
  opt->tol = 1e-10;
  opt->max_iter = 1000;
  opt->max_subspace = 20;
  opt->restart_keep = 2;
  opt->fp64_refine = 1;
  opt->refine_ratio = 0.0;
  opt->anchor_prec = DMRG_PREC_FP64;
  opt->vector_arith = DMRG_VEC_SPLIT;
  opt->autotune = 1;
  opt->graphs = 1;
  opt->anchor_update = 1;
}

const char* dmrg_status_string(dmrg_status s) {
  switch (s) {
    case DMRG_OK: return "ok";
    case DMRG_ERR_INVALID_ARG: return "invalid argument";
    case DMRG_ERR_SHAPE: return "shape mismatch";
    case DMRG_ERR_OOM: return "out of memory";
    case DMRG_ERR_CUDA: return "CUDA error";
    case DMRG_ERR_NOT_CONVERGED: return "not converged";
    case DMRG_ERR_NUMERIC: return "numerical breakdown";
    case DMRG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* dmrg_last_error(void) { return dmrg::g_last_error; }

int64_t dmrg_kernel_launches(void) { return dmrg::g_launches.load(); }

int32_t dmrg_precision_available(dmrg_precision prec) {
  if (prec == DMRG_PREC_FP64) return 1;
  return dmrg::tc_available(prec) ? 1 : 0;
}

const char* dmrg_version(void) { return "dmrg-gb300 0.1 (sm_103a)"; }

}  // extern "C"
