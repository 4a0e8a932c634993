// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "dmrg.h"

namespace dmrg {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);

#define DMRG_CUDA_TRY(expr)                                                          \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ::dmrg::set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,   \
                        __LINE__);                                                   \
      return DMRG_ERR_CUDA;                                                          \
    }                                                                                \
  } while (0)

#define DMRG_TRY(expr)                \
  do {                                \
    dmrg_status s_ = (expr);          \
    if (s_ != DMRG_OK) return s_;     \
  } while (0)

// Kernel launches are counted and checked with cudaGetLastError right after the launch.
void note_launch();
// adds n (may be negative) to the launch count: the kernels of a replayed CUDA graph count
// as launches, the captured ones do not
void note_launches(int64_t n);
#define DMRG_LAUNCH_CHECK()                  \
  do {                                       \
    ::dmrg::note_launch();                   \
    DMRG_CUDA_TRY(cudaGetLastError());       \
  } while (0)

#ifdef __CUDACC__
// Programmatic dependent launch, device side: wait until the grids this one depends on have
// completed and their writes are visible (returns at once for a grid launched without the
// attribute); allow the next grid in the stream to be scheduled (it still waits for this
// one to complete before it reads anything).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// Launch with programmatic dependent launch allowed: the kernel may be scheduled while the
// previous kernel in the stream is finishing, so it must execute griddepcontrol.wait before
// it touches memory that earlier work writes (every kernel launched this way does so first).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- operand addressing
// Operands of the FP64 projection GEMMs are addressed relative to one of four base
// pointers that change from call to call: the operator arena owned by the plan, the
// input vector X, the stage-1 intermediates T and the output vector Y.
enum Space : int32_t { SP_ARENA = 0, SP_X = 1, SP_T = 2, SP_Y = 3 };

struct Bases {
  const double* p[4];
};

// Element (r, c) of an operand sits at base[space] + off + r * rs + c * cs.
struct Operand {
  int64_t off;
  int64_t rs, cs;
  int32_t space;
  int32_t pad_;
};

// One K-segment of a job: C += alpha * P[M x K] * Q[K x N].
struct Seg64 {
  Operand P, Q;
  int32_t K;
  int32_t pad_;
  double alpha;
};

// One output matrix C[M x N] (row stride ldc) written as the sum of its segments plus
// axpy * X(axpy operand) (the term whose two factors are identities).
struct Job64 {
  Operand C;
  Operand Xaxpy;
  double axpy;
  int32_t M, N;
  int32_t seg_begin, seg_end;
};

struct Tile64 {
  int32_t job;
  int32_t m0, n0;
  int32_t pad_;
};

constexpr int kTileM = 64;
constexpr int kTileN = 64;
constexpr int kTileK = 16;

// ---------------------------------------------------------------- plan
struct Record {
  int32_t term;
  int32_t a_blk, b_blk;  // index into the block table of each side, -1 = identity
  int32_t pin, pout;     // input / output pair index
  int32_t i, j, k, l;    // sectors
  int64_t di, dj, dk, dl;
  double coef;
  int32_t a_first;       // 1: T = A X then T B^T; 0: U = X B^T then A U
  int64_t inter_off;     // offset of T or U in the intermediate buffer
};

struct HostBlock {
  int32_t idx_in, idx_out;
  int64_t rows, cols;
  int64_t arena_off;     // row-major, ld = cols
};

// Records whose block factors are both identities add coef * X(pin) to Y(pout).  In the
// LR form pin == pout, and the GEMM epilogues add the term in place; in the l-1-1-r form
// the site factors can move the state to another segment of the same dimensions, and a
// pass after the last GEMM stage adds those terms (one group per output segment, entries
// in record order).
struct SegAxpyGroup {
  int64_t dst_off, size;
  int32_t beg, end;
};
struct SegAxpyEntry {
  int64_t src_off;
  double coef;
};

struct TcPlan;           // tensor-core (low precision) part, see gemm_tc.cu
struct OzPlan;           // FP64-accurate tensor-core part, see gemm_oz.cu
struct SolveWorkspace;   // buffers of one Davidson state, see davidson.cu

}  // namespace dmrg

struct dmrg_plan {
  int device = 0;
  dmrg_options opt{};
  int64_t n = 0;
  std::vector<int64_t> dimL, dimR;
  std::vector<int32_t> pair_i, pair_k;
  std::vector<int64_t> pair_off;  // npairs + 1
  std::vector<std::vector<dmrg::HostBlock>> opsL, opsR;
  std::vector<dmrg_term> terms;
  std::vector<dmrg::Record> records;
  int64_t flops = 0;

  double* arena = nullptr;        // operator blocks
  size_t arena_elems = 0;
  std::vector<double> arena_host; // staging copy (freed after upload)
  double* T = nullptr;            // stage-1 intermediates
  size_t T_elems = 0;
  double* D = nullptr;            // diag(H_SB)

  dmrg::Job64* d_jobs = nullptr;
  dmrg::Seg64* d_segs = nullptr;
  dmrg::Tile64* d_tiles1 = nullptr;
  dmrg::Tile64* d_tiles2 = nullptr;
  int64_t ntiles1 = 0, ntiles2 = 0;
  size_t device_bytes = 0;

  dmrg::SegAxpyGroup* d_sax_groups = nullptr;  // cross-segment identity terms (l-1-1-r form)
  dmrg::SegAxpyEntry* d_sax_entries = nullptr;
  int32_t n_sax_groups = 0;
  int64_t sax_max_size = 0;

  dmrg::TcPlan* tc[3] = {nullptr, nullptr, nullptr};  // TF32, BF16x3, BF16x2; built on first use
  dmrg::OzPlan* oz = nullptr;                 // FP64 emulation; built on first use

  // buffers kept between solves (released by dmrg_plan_trim and dmrg_plan_destroy): the
  // workspace of the last finished Davidson state, and the two device vectors of
  // dmrg_davidson_solve_host; ws_mu guards the three pointers
  std::mutex ws_mu;
  dmrg::SolveWorkspace* ws_cache = nullptr;
  double* io_x0 = nullptr;
  double* io_x = nullptr;
};

namespace dmrg {
// gemm_fp64.cu
dmrg_status launch_project_fp64(dmrg_plan* plan, const double* x, double* y,
                                cudaStream_t stream);
// gemm_tc.cu
dmrg_status launch_project_tc(dmrg_plan* plan, dmrg_precision prec, const double* x,
                              double* y, cudaStream_t stream);
// the same with an FP32 vector in and out (the low-precision basis columns of a mixed
// solve with split vector arithmetic)
dmrg_status launch_project_tc32(dmrg_plan* plan, dmrg_precision prec, const float* x, float* y,
                                cudaStream_t stream);
// builds the tensor-core plan of prec if needed and times its tile schedules
dmrg_status tune_project_tc(dmrg_plan* plan, dmrg_precision prec, cudaStream_t stream);
dmrg_status set_schedule_tc(dmrg_plan* plan, dmrg_precision prec, int stage1, int stage2,
                            cudaStream_t stream);
// chosen schedule per GEMM stage (-1: no tensor-core plan) and the tuning times (us)
void tc_schedule_stats(const dmrg_plan* plan, int32_t sched[2], float us[2][DMRG_TILE_SCHEDULES]);
// grouped launch of the low-precision projections of several distinct plans
struct TcBatch;
dmrg_status tc_batch_create(dmrg_plan* const* plans, int nb, dmrg_precision prec,
                            cudaStream_t stream, TcBatch** out);
// y[i] = H_i x[i] for every i with active[i]; x[i], y[i] are device vectors of plan i, or,
// where x32 (and y32) are given and x32[i] is not NULL, FP32 vectors x32[i], y32[i]
dmrg_status tc_batch_project(TcBatch* b, const double* const* x, double* const* y,
                             const float* const* x32, float* const* y32, const char* active,
                             cudaStream_t stream);
dmrg_status tc_batch_error(const TcBatch* b);
void tc_batch_destroy(TcBatch* b);
void destroy_tc(dmrg_plan* plan);
bool tc_available(dmrg_precision prec);
// slot of a low-precision tensor-core plan in dmrg_plan::tc (TF32 0, BF16X3 1, BF16X2 2)
inline int tc_slot(dmrg_precision prec) {
  return prec == DMRG_PREC_TF32 ? 0 : prec == DMRG_PREC_BF16X3 ? 1 : 2;
}
inline bool tc_lowprec(dmrg_precision prec) {
  return prec == DMRG_PREC_TF32 || prec == DMRG_PREC_BF16X3 || prec == DMRG_PREC_BF16X2;
}
dmrg_status tc_error_status(dmrg_plan* plan);
// gemm_oz.cu
// y = H x with the leading `digits` (2..7) base-128 digits of every operand (7: FP64-accurate;
// fewer: relative accuracy ~2^(-7 digits + 1), for inputs small against what they correct)
dmrg_status launch_project_oz(dmrg_plan* plan, const double* x, double* y, cudaStream_t stream,
                              int digits = 7);
void destroy_oz(dmrg_plan* plan);
dmrg_status oz_error_status(dmrg_plan* plan);

// vec.cu -- Davidson vector kernels (the small eigenproblem: eig.cu)
constexpr int KMAX = DMRG_MAX_SUBSPACE;
constexpr int kVecThreads = 256;

struct DevSmall {
  double B[KMAX * KMAX];  // projected matrix, row-major
  double y[KMAX];         // lowest eigenvector of B
  double s[3][KMAX];      // Gram-Schmidt coefficients
  double lambda;
  double rnorm2;          // ||r||^2 of the current Ritz pair
  double tnorm2_before;   // ||t||^2 before orthogonalisation
  double tnorm2;          // ||t||^2 after the latest Gram-Schmidt pass
  double nrm2;            // generic norm result
  int32_t flags;          // bit 0: breakdown, bit 1: non-finite, bit 2: second
                          // Gram-Schmidt pass ran
  int32_t jacobi_sweeps;
  double Q[KMAX * KMAX];  // eigenvectors of the last k x k B (row-major, columns)
  double theta[KMAX];     // its eigenvalues
  int32_t qk;             // order of the stored decomposition (0: none)
  int32_t eig_fallbacks;  // small eigenproblems that needed the FP64 Jacobi fallback
  int64_t eig_cycles[3];  // last small eigenproblem: SM clock cycles of setup + FP32
                          // Jacobi, of the FP64 refinement, and in total (diagnostics)
  double y_prev[KMAX];    // lowest eigenvector of the previous small eigenproblem
  double C[2][KMAX];      // restart coefficients: new basis = [V C0, V C1]
};

struct VecWork {
  double* partials = nullptr;   // [grid x slots]
  unsigned int* counter = nullptr;
  int grid = 0;
};

dmrg_status vec_work_create(VecWork* w);
void vec_work_destroy(VecWork* w);

// The device and pinned buffers of one Davidson state (davidson.cu).  A finished state
// hands them to its plan, and the next state of the same shape takes them over, so that
// repeated solves allocate nothing and replay the projection graphs captured for the same
// column pointers.
struct SolveWorkspace {
  int64_t ldv = 0;
  int kmax = 0;
  bool f32 = false, keep2 = false;  // keep2: the spare vectors pbuf and wpbuf exist
  double *V = nullptr, *W = nullptr;
  float *V32 = nullptr, *W32 = nullptr;
  double *tbuf = nullptr, *D = nullptr, *xbuf = nullptr, *wbuf = nullptr;
  double *pbuf = nullptr, *wpbuf = nullptr;
  DevSmall* small = nullptr;
  DevSmall* hsmall = nullptr;
  VecWork vw;
};
void workspace_free(SolveWorkspace* w);

// s_out[j] = V_j . w for j < k (V column-major, ldv); if Bcol >= 0 also fills row and
// column Bcol of small->B.
dmrg_status launch_overlap(const VecWork& w, const double* V, int64_t ldv, int64_t n,
                           int k, const double* vec, double* s_out, DevSmall* small,
                           int Bcol, cudaStream_t st, const double* w0 = nullptr);
dmrg_status launch_jacobi(DevSmall* small, int k, cudaStream_t st);
// all eigenpairs of B (k x k) in FP64, ascending: theta[j] and column j of Q
dmrg_status launch_all_eig(DevSmall* small, int k, cudaStream_t st);
// r = W y - lambda V y, t = r / (lambda - D) (mode 0) or t = r (mode 1) into tcol;
// reductions: rnorm2, s[0] = V^T t, tnorm2_before.
dmrg_status launch_residual(const VecWork& w, const double* V, const double* W,
                            const double* D, int64_t ldv, int64_t n, int k, double* tcol,
                            DevSmall* small, int mode, cudaStream_t st);
// t -= V s[sin]; s[sout] = V^T t; tnorm2 = ||t||^2
dmrg_status launch_cgs(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                       double* tcol, DevSmall* small, int sin, int sout, cudaStream_t st,
                       int second = 0);
// flags breakdown (tnorm2 < 1e-20 tnorm2_before) else t /= ||t||
dmrg_status launch_finish(double* tcol, int64_t n, DevSmall* small, cudaStream_t st);
// x = V y, optionally wy = W y (n elements, written unpadded)
dmrg_status launch_ritz(const double* V, const double* W, int64_t ldv, int64_t n, int k,
                        const DevSmall* small, double* x_out, double* wy_out,
                        cudaStream_t st);
// nrm2 = ||src||^2 then dst = src / ||src|| (dst padded to ldv with zeros by caller)
dmrg_status launch_normalize(const VecWork& w, const double* src, double* dst, int64_t n,
                             DevSmall* small, cudaStream_t st);
dmrg_status launch_set_B00(DevSmall* small, cudaStream_t st);
// out = a + c b (n elements)
dmrg_status launch_axpby(const VecWork& w, const double* a, double c, const double* b, double* out,
                         int64_t n, cudaStream_t st);
// dst = src / sqrt(small->nrm2) (the norm of the last launch_normalize)
dmrg_status launch_scale_copy(const VecWork& w, const double* src, double* dst, int64_t n,
                              const DevSmall* small, cudaStream_t st);
// two-vector restart: x = V C0, p = V C1, wx = W C0, wp = W C1 (n elements each)
dmrg_status launch_ritz2(const double* V, const double* W, int64_t ldv, int64_t n, int k,
                         const DevSmall* small, double* x, double* p, double* wx, double* wp,
                         cudaStream_t st);
// p -= a x and wp -= a wx with a = small->s[2][0], then p and wp scaled by 1 / ||p||
dmrg_status launch_orth_pair(const VecWork& w, double* p, double* wp, const double* x,
                             const double* wx, int64_t n, DevSmall* small, cudaStream_t st);
// vec_df.cu -- the same passes in double-float (FP32 pair) arithmetic
dmrg_status launch_overlap_df(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                              const double* vec, double* s_out, DevSmall* small, int Bcol,
                              cudaStream_t st, const double* w0 = nullptr);
dmrg_status launch_residual_df(const VecWork& w, const double* V, const double* W,
                               const double* D, int64_t ldv, int64_t n, int k, double* tcol,
                               DevSmall* small, int mode, cudaStream_t st);
dmrg_status launch_cgs_df(const VecWork& w, const double* V, int64_t ldv, int64_t n, int k,
                          double* tcol, DevSmall* small, int sin, int sout, cudaStream_t st,
                          int second = 0);
// vec_split.cu -- mixed modes with split arithmetic: column 0 of the basis in FP64 (V0, W0),
// the low-precision columns j >= 1 stored in FP32 (V32 + j * ldv, W32 + j * ldv); the new
// direction t is an FP64 work vector (tcol) until it is appended
dmrg_status launch_overlap_split(const VecWork& w, const double* V0, const float* V32, int64_t ldv,
                                 int64_t n, int k, const double* vec64, const float* vec32,
                                 double* s_out, DevSmall* small, int Bcol, cudaStream_t st,
                                 const double* w0 = nullptr);
dmrg_status launch_residual_split(const VecWork& w, const double* V0, const double* W0,
                                  const float* V32, const float* W32, const double* D,
                                  int64_t ldv, int64_t n, int k, double* tcol, DevSmall* small,
                                  int mode, cudaStream_t st);
dmrg_status launch_cgs_split(const VecWork& w, const double* V0, const float* V32, int64_t ldv,
                             int64_t n, int k, double* tcol, DevSmall* small, int sin, int sout,
                             cudaStream_t st, int second = 0);
// flags breakdown, else t = (t - s[1][0] v_0) / norm unless the second pass ran (k >= 2),
// and out32 = t rounded to FP32
dmrg_status launch_finish_split(const VecWork& w, const double* V0, double* tcol, int64_t n,
                                int k, DevSmall* small, float* out32, cudaStream_t st);
// dst = src rounded to nearest FP32 (n elements rounded up to even; padded buffers)
dmrg_status launch_convert32(const VecWork& w, const double* src, float* dst, int64_t n,
                             cudaStream_t st);
// x = V y (and wx = W y if wx): column 0 in FP64, the FP32 tail summed in FP32 (padded
// outputs: n rounded up to even elements are written)
dmrg_status launch_ritz_split(const VecWork& w, const double* V0, const double* W0,
                              const float* V32, const float* W32, int64_t ldv, int64_t n, int k,
                              const DevSmall* small, double* x, double* wx, cudaStream_t st);
// two-vector restart: x = V C0, p = V C1, wx = W C0, wp = W C1 (padded outputs)
dmrg_status launch_ritz2_split(const VecWork& w, const double* V0, const double* W0,
                               const float* V32, const float* W32, int64_t ldv, int64_t n, int k,
                               const DevSmall* small, double* x, double* p, double* wx,
                               double* wp, cudaStream_t st);
dmrg_status launch_gemv_trans_public(const double* V, int64_t ldv, int64_t n, int k,
                                     const double* w, double* s, cudaStream_t st);

// plan.cu
dmrg_status compute_diagonal(dmrg_plan* plan, double* d, cudaStream_t st);
// y(pout) += coef x(pin) for the cross-segment identity terms (no-op without any); FP64
// vectors, or FP32 ones when x32 is given
dmrg_status launch_seg_axpy(const dmrg_plan* plan, const double* x, double* y, const float* x32,
                            float* y32, cudaStream_t st);

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace dmrg
