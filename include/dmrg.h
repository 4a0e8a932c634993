/*
 * dmrg.h -- C ABI of the GB300 library for the DMRG superblock Davidson path.
 *
 * The library finds the lowest eigenpair of a superblock Hamiltonian written in the LR
 * form of Sec. 4.1,
 *
 *     H_SB = sum_a coef_a  A_a (x) B_a                                   (Eq. 9)
 *
 * restricted to one symmetry sector Q (Sec. 3), with the projection evaluated as the
 * sector-decomposed matrix products
 *
 *     X'_{jl} += coef_a * A_{a, i->j} X_{ik} B_{a, k->l}^T                (Eq. 11)
 *
 * and the Davidson iteration of Algorithm 3 (Sec. 5) around it.
 *
 * Conventions used by every call:
 *
 *  - Vector layout.  A superblock vector of length n is the concatenation, in the order
 *    of the pair list (pair_i[p], pair_k[p]), of the dense row-major segments X_{ik} of
 *    shape [dimL[i], dimR[k]]; element psi(a, b) of segment p sits at
 *    x[offset_p + a * dimR[k] + b], offset_p being the sum of the sizes of the earlier
 *    segments.  The reshape of Eq. 10 is therefore the row-major one (left index slow).
 *  - Operator blocks map input sector idx_in to output sector idx_out and are dense
 *    row-major [rows = dim(idx_out), cols = dim(idx_in)] matrices with leading
 *    dimension ld >= cols, in float64.  Block data may live in host or device memory
 *    (dmrg_superblock_desc.data_location); the plan copies what it needs at creation,
 *    so the caller may free the descriptor and the block data afterwards.
 *  - Vectors passed to dmrg_project / dmrg_davidson_* (x, y, x0, x_out, d) are device
 *    pointers to float64 arrays of n elements owned by the caller, unless a call says
 *    otherwise (the *_host variants take host pointers).  They are borrowed for the
 *    duration of the call only.
 *  - Streams.  A stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue their work on it; the calls named *_solve*, the *_host
 *    variants and dmrg_davidson_step return only when their results are complete.
 *  - Errors.  No exception crosses the ABI.  Every call returns a dmrg_status;
 *    dmrg_last_error() gives a thread-local message for the last failure.  A CUDA error
 *    maps to DMRG_ERR_CUDA.  Invalid sizes or indices map to DMRG_ERR_INVALID_ARG or
 *    DMRG_ERR_SHAPE before any device work is enqueued.
 *  - Single GPU.  A plan lives on the device that was current when it was created; use
 *    it with that device current.
 *  - A plan owns the scratch of its projections (operand images, intermediates): calls
 *    that use the same plan must be ordered (one stream, or events); create one plan per
 *    problem to run problems concurrently.
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DMRG_OK = 0,
  DMRG_ERR_INVALID_ARG = 1,   /* null pointer, negative size, index out of range      */
  DMRG_ERR_SHAPE = 2,         /* block shape or pair table inconsistent with sectors  */
  DMRG_ERR_OOM = 3,           /* device or host allocation failed                      */
  DMRG_ERR_CUDA = 4,          /* a CUDA runtime or kernel error                        */
  DMRG_ERR_NOT_CONVERGED = 5, /* Davidson hit max_iter; best pair and info are filled  */
  DMRG_ERR_NUMERIC = 6,       /* NaN/Inf in a residual or a basis breakdown            */
  DMRG_ERR_UNSUPPORTED = 7    /* option not available in this build                    */
} dmrg_status;

/* Arithmetic of the projection GEMMs.  FP64: float64 operands and accumulation on the
 * FP64 units.  TF32: operands rounded to TF32 on the tensor cores, FP32 accumulation.
 * BF16X3: every operand split into three BF16 terms x = x0 + x1 + x2, the six products
 * with i + j <= 2 accumulated in FP32 on the tensor cores.  BF16X2: the shorter split
 * x = x0 + x1 (two BF16 terms, about 17 significant bits) with the three products
 * x0 y0 + x0 y1 + x1 y0 accumulated in FP32 on the tensor cores: half the tensor work and
 * two thirds of the operand bytes of BF16X3, at a larger projection error (meant for the
 * mixed Davidson iteration, whose FP64-accurate anchors decide the answer).  FP64_TC:
 * FP64-accurate products on the tensor cores: every operand row chunk (256 K elements) is
 * split into a power-of-two scale and seven integer base-128 digits held exactly in BF16;
 * digit products sharing a scale are summed exactly in FP32 and the scaled sums are
 * combined in FP32-pair (about 48-bit) arithmetic, then converted to float64.  The Davidson
 * vector work (overlaps, Gram-Schmidt, Rayleigh quotient, residual, small eigenproblem)
 * keeps float64 accuracy in every mode. */
typedef enum {
  DMRG_PREC_FP64 = 0,
  DMRG_PREC_TF32 = 1,
  DMRG_PREC_BF16X3 = 2,
  DMRG_PREC_FP64_TC = 3,
  DMRG_PREC_BF16X2 = 4
} dmrg_precision;

enum { DMRG_HOST_DATA = 0, DMRG_DEVICE_DATA = 1 };
enum { DMRG_IDENTITY_OP = -1 };
enum { DMRG_MAX_SUBSPACE = 24 };
enum { DMRG_TILE_SCHEDULES = 27 };  /* candidate tile schedules per tensor-core GEMM stage */

/* One dense block A_{q_in -> q_out} of an operator (Sec. 4.1, around Eq. 11). */
typedef struct {
  int32_t idx_in, idx_out;  /* sector indices on this side (left or right)        */
  int64_t rows, cols, ld;   /* rows = dim(idx_out), cols = dim(idx_in), ld >= cols */
  const double* data;       /* row-major; host or device per data_location        */
} dmrg_block;

typedef struct {
  int32_t nblocks;
  const dmrg_block* blocks; /* at most one block per (idx_in, idx_out)            */
} dmrg_operator;

/* coef * (A_{a_op} (x) B_{b_op}); an op index of DMRG_IDENTITY_OP is the identity. */
typedef struct {
  double coef;
  int32_t a_op, b_op;
} dmrg_term;

typedef struct {
  int32_t nL, nR;                 /* number of enlarged-left / enlarged-right sectors */
  const int64_t* dimL;            /* host arrays of sector dimensions                 */
  const int64_t* dimR;
  int32_t npairs;                 /* valid (i, k) pairs of sector Q, storage order    */
  const int32_t* pair_i;          /* host arrays of length npairs                     */
  const int32_t* pair_k;
  int32_t nopsL, nopsR;
  const dmrg_operator* opsL;      /* host array of operators (blocks may be device)   */
  const dmrg_operator* opsR;
  int32_t nterms;
  const dmrg_term* terms;         /* host array                                       */
  int32_t data_location;          /* DMRG_HOST_DATA or DMRG_DEVICE_DATA               */
} dmrg_superblock_desc;

/* A superblock in the l-1-1-r form of Sec. 4.2:
 *
 *     H_SB = sum_a coef_a  A_a^(l) (x) a_a (x) b_a (x) B_a^(r)              (Eq. 12)
 *
 * with A on block l, a and b on the two middle sites, B on block r, and the projection of
 * Eq. 13 (Algorithm 2 per term).  Every site state is a sector of its own (its quantum
 * numbers differ from the others'), so a site operator is a dense q x q matrix.  A vector
 * is the concatenation, in the order of the segment list, of the row-major segments
 * (i, s1, s2, k) of shape [diml[i], dimr[k]]: element psi(a, b) of segment g sits at
 * x[offset_g + a * dimr[k] + b]. */
typedef struct {
  double coef;
  int32_t l_op, s1_op, s2_op, r_op; /* DMRG_IDENTITY_OP: the identity on that subsystem */
} dmrg_term4;

typedef struct {
  int32_t nl, nr;                   /* sectors of block l and of block r               */
  const int64_t* diml;              /* host arrays of their dimensions                 */
  const int64_t* dimr;
  int32_t q;                        /* states of one site (at most 64)                 */
  int32_t nsegs;                    /* valid (i, s1, s2, k), storage order             */
  const int32_t* seg_l;             /* host arrays of length nsegs                     */
  const int32_t* seg_s1;
  const int32_t* seg_s2;
  const int32_t* seg_r;
  int32_t nopsl, nopsr;
  const dmrg_operator* opsl;        /* block operators of l and r (blocks host or
                                       device per data_location)                       */
  const dmrg_operator* opsr;
  int32_t nsops;
  const double* sops;               /* host: nsops site matrices, each q x q row-major
                                       with element [s_out * q + s_in]                 */
  int32_t nterms;
  const dmrg_term4* terms;          /* host array                                      */
  int32_t data_location;            /* DMRG_HOST_DATA or DMRG_DEVICE_DATA              */
} dmrg_l11r_desc;

/* Arithmetic of the Davidson vector passes (overlap, residual, Gram-Schmidt; the paper
   runs them in FP64, Sec. 6.1).  GB300 executes about 0.55 T FP64 FMA/s against 6.8 TB/s
   of HBM, so the FP64 passes are bound by the FP64 units.
   DMRG_VEC_FP64          FP64 units throughout.
   DMRG_VEC_DOUBLE_FLOAT  double-float (FP32 pairs, ~48 bits) on the FP32 units; measured
                          slower than FP64 at the sizes tested, kept as an option.
   DMRG_VEC_SPLIT         mixed modes only (TF32/BF16X3/BF16X2 with fp64_refine): column 0
                          (the FP64 anchor) in FP64, the low-precision columns in FP32
                          arithmetic, whose rounding stays far below their projection
                          error; anchor iterations and the convergence test stay FP64.
                          In FP64 and FP64_TC solves this is DMRG_VEC_FP64.             */
typedef enum {
  DMRG_VEC_FP64 = 0,
  DMRG_VEC_DOUBLE_FLOAT = 1,
  DMRG_VEC_SPLIT = 2
} dmrg_vector_arith;

typedef struct {
  dmrg_precision prec;   /* projection arithmetic inside Davidson (default FP64)          */
  double tol;            /* stop when ||H x - lambda x||_2 <= tol, ||x|| = 1 (1e-10)      */
  int32_t max_iter;      /* Davidson iterations before DMRG_ERR_NOT_CONVERGED (1000)      */
  int32_t max_subspace;  /* basis size that triggers a restart, <= 24 (20, Sec. 6.1)     */
  int32_t restart_keep;  /* vectors kept at a subspace-limit restart: 1 (the Ritz vector)
                            or 2 (also the previous iteration's Ritz vector, orthonormalised
                            against it; default); FP64 anchors of the mixed modes keep 1  */
  int32_t fp64_refine;   /* low-precision modes: re-anchor with FP64 projections (1)      */
  double refine_ratio;   /* if > 0, also re-anchor when the low-precision residual has
                            fallen by this factor below the last FP64 residual (0: only
                            the adaptive floor test and the subspace limit re-anchor)     */
  dmrg_precision anchor_prec; /* FP64-accurate projections of the mixed modes: DMRG_PREC_FP64
                            (FP64 units, default) or DMRG_PREC_FP64_TC (tensor cores,
                            FP64-accurate digit products; about 17x faster)              */
  int32_t vector_arith;  /* arithmetic of the Davidson vector passes (dmrg_vector_arith);
                            vectors are float64 in memory in every mode (default
                            DMRG_VEC_SPLIT)                                              */
  int32_t autotune;      /* 1 (default): the first TF32/BF16X3/BF16X2 projection of a plan times
                            the candidate tile schedules of both tensor-core GEMM stages
                            and keeps the fastest (that call synchronizes its stream and
                            must not be captured in a CUDA graph; dmrg_plan_autotune does
                            it ahead of time); 0: descending-cost schedule              */
  int32_t graphs;        /* 1 (default): a TF32/BF16X3/BF16X2 projection is replayed from a
                            CUDA graph of its launch sequence (pack, both GEMM stages, the
                            split-K reduction), captured on first use for each pair of
                            vector pointers and tile schedules on a stream owned by the
                            plan; a call made while the caller's stream is being captured
                            launches the kernels directly into that capture; 0: direct
                            launches always.  The results are identical either way.       */
  int32_t anchor_update; /* 1 (default): with anchor_prec = DMRG_PREC_FP64_TC, an anchor taken
                            while column 0 of the basis is still the previous anchor (no
                            plain restart since) is formed as H x = y_0 W(:,0) + H d,
                            d = x - y_0 v_0, with H d computed from the leading digits of
                            the FP64_TC split that its norm needs (error held below 2^-46
                            ||H||, as for a full FP64_TC projection); 0: every anchor
                            projects x in full.                                          */
} dmrg_options;

typedef struct {
  double energy;            /* lambda of the returned pair (FP64 Rayleigh quotient)       */
  double resnorm;           /* ||H x - lambda x||_2 of the returned pair                  */
  int32_t iters;            /* Davidson iterations                                        */
  int32_t projections;      /* projections in the plan's precision                        */
  int32_t fp64_projections; /* FP64 projections (all of them in FP64 mode)                */
  int32_t restarts;         /* basis collapses (subspace limit or re-anchoring)           */
  int32_t small_eig_sweeps; /* Jacobi sweeps of the projected eigenproblem, all iterations */
  int32_t converged;        /* 1 if ||r|| <= tol was reached                               */
  int32_t anchor_updates;   /* anchors formed by the anchor update (included in
                               fp64_projections)                                          */
} dmrg_solve_info;

typedef struct {
  int64_t n;                /* superblock dimension                                       */
  int64_t records;          /* transition pairs of Eq. 11                                 */
  int64_t flops;            /* algorithmic FLOPs of one projection (cheaper order, non-
                               identity factors only)                                      */
  int64_t tiles_stage1, tiles_stage2;
  int64_t device_bytes;     /* device memory owned by the plan                            */
  int32_t tc_schedule[2];   /* tile schedule of tensor-core GEMM stages 1 and 2,
                               (3 s + w) 3 + o: order o of the tile list that the CTAs take
                               tiles from (0: descending estimated time; 1: stage 1 grouped
                               by vector segment, stage 2 by right sector; 2: stage 1
                               grouped by operator block, stage 2 by left sector), BF16
                               tile width w (0: 128 columns; 1: 256 columns for tiles below
                               half the mean work per SM; 2: 256 wherever possible) and
                               stage-2 K split s (0: none; 1, 2: tiles above 2/3, 2/5 of the
                               mean time per SM split into parts); -1 before a low-precision
                               plan exists                                                 */
  float tc_tune_us[2][DMRG_TILE_SCHEDULES]; /* autotuner: median time of each schedule per
                               stage (us), 0 if not tuned or not a candidate               */
} dmrg_plan_stats;

typedef struct dmrg_plan dmrg_plan;
typedef struct dmrg_davidson_state dmrg_davidson_state;

/* Fills the defaults listed above. */
void dmrg_options_default(dmrg_options* opt);

/* Builds the operation records of Sec. 7 (Algorithm 5, line 1: records and their FLOP
 * workload) and uploads the operator blocks to a device arena owned by the plan; also
 * computes diag(H_SB) for the Davidson correction.  desc and its arrays are read during
 * the call only.  opt may be NULL (defaults).  On success *out owns device memory until
 * dmrg_plan_destroy. */
dmrg_status dmrg_plan_create(const dmrg_superblock_desc* desc, const dmrg_options* opt,
                             void* stream, dmrg_plan** out);
/* Plan of a superblock in the l-1-1-r form (Sec. 4.2, Eqs. 12-13; the paper describes the
 * form and leaves its implementation open).  Every call that takes a plan (projections in
 * every precision, the Davidson solves, autotuning, batched solves) works on it as on an
 * LR plan; the vector layout is that of dmrg_l11r_desc.  The site factors are single
 * elements of their matrices (each site state is a sector), so stages 2 and 3 of
 * Algorithm 2 become coefficients of the records, and each record is the product of a
 * block of l, a segment and a block of r: the largest matrices are those of the blocks,
 * O(m^2), instead of the O((mq)^2) enlarged blocks of the LR form.  Same ownership and
 * error rules as dmrg_plan_create. */
dmrg_status dmrg_plan_create_l11r(const dmrg_l11r_desc* desc, const dmrg_options* opt,
                                  void* stream, dmrg_plan** out);
/* Frees the plan and everything it owns (the buffers kept by dmrg_plan_trim included). */
void dmrg_plan_destroy(dmrg_plan* plan);
/* A finished Davidson state (dmrg_state_destroy, and so the end of every solve) leaves its
 * device and pinned buffers with its plan, and the next state of the same shape takes them
 * over; dmrg_davidson_solve_host keeps its two device vectors the same way.  Repeated
 * solves on one plan therefore allocate nothing after the first.  The kept workspace is
 * (2 max_subspace + 6) n doubles for FP64 solves and about half of that for mixed solves
 * with split vector arithmetic.  This call frees all of it now (the plan stays usable;
 * the next solve allocates again); a state that is running holds its own buffers and is
 * not affected.  DMRG_ERR_INVALID_ARG for a NULL plan. */
dmrg_status dmrg_plan_trim(dmrg_plan* plan);
dmrg_status dmrg_plan_get_stats(const dmrg_plan* plan, dmrg_plan_stats* stats);

/* Tile-schedule autotuner of the tensor-core projection (prec DMRG_PREC_TF32,
 * DMRG_PREC_BF16X3 or DMRG_PREC_BF16X2): builds the operand images if needed, times every
 * candidate schedule of each GEMM stage on this GPU (L2 flushed before each timing) and
 * keeps the fastest; the results appear in dmrg_plan_stats (for the plan's own precision
 * when its tensor-core plan exists, else for the first one built).  The paper has no
 * counterpart (its records are dispatched to streams by Algorithms 6-7).  Synchronizes the
 * stream; allocates and frees 256 MB of scratch. */
dmrg_status dmrg_plan_autotune(dmrg_plan* plan, dmrg_precision prec, void* stream);

/* Fixes the tile schedules of the tensor-core projection in precision prec (DMRG_PREC_TF32,
 * DMRG_PREC_BF16X3 or DMRG_PREC_BF16X2) to stage1 and stage2 (indices as in
 * dmrg_plan_stats.tc_schedule; stage 1 takes no K split, TF32 only 128-column tiles) and
 * keeps the first projection from autotuning; builds the operand images if needed and
 * synchronizes the stream.
 * DMRG_ERR_INVALID_ARG for an index that is not a candidate of its stage. */
dmrg_status dmrg_plan_set_tile_schedule(dmrg_plan* plan, dmrg_precision prec, int32_t stage1,
                                        int32_t stage2, void* stream);

/* y = H_SB x (Eq. 11 summed over all records), in the given precision.  x and y are
 * device arrays of n float64 and must not overlap.  Enqueued on stream. */
dmrg_status dmrg_project(dmrg_plan* plan, const double* x, double* y, void* stream);
dmrg_status dmrg_project_prec(dmrg_plan* plan, dmrg_precision prec, const double* x,
                              double* y, void* stream);
/* y = H_SB x on the FP64_TC path with the leading `digits` (2..7) base-128 digits of every
 * operand and stage-1 result (7: the FP64-accurate DMRG_PREC_FP64_TC projection; d digits
 * cost d (d + 1) / 2 digit-pair products instead of 28 and give a relative accuracy of about
 * 2^(1 - 7 d) of the row-chunk scales).  The paper has no counterpart: the Davidson anchor
 * update uses it for the projection of a small correction (dmrg_options.anchor_update).
 * Same layout, stream and overlap rules as dmrg_project; DMRG_ERR_INVALID_ARG for digits
 * outside [2, 7]. */
dmrg_status dmrg_project_digits(dmrg_plan* plan, int32_t digits, const double* x, double* y,
                                void* stream);

/* d = diag(H_SB) (device array of n float64), the Davidson preconditioner input. */
dmrg_status dmrg_diagonal(dmrg_plan* plan, double* d, void* stream);

/* s[j] = sum_e V[j * ldv + e] * w[e] for j < k: the "asymmetric" matrix-vector product
 * V^T w of Sec. 6.1 (Algorithm 3 lines 3 and 11) on a tall-skinny column-major V of n
 * rows and k <= 24 columns.  V, w, s are device pointers; ldv >= n.  Enqueued. */
dmrg_status dmrg_gemv_trans(const double* V, int64_t ldv, int64_t n, int32_t k,
                            const double* w, double* s, void* stream);

/* Allocation-free variant of dmrg_gemv_trans (the paper has no counterpart: it exists for
 * callers that cannot let a library allocate device memory, such as an application whose
 * own allocator owns all device memory, or a latency-critical loop where cudaMalloc and
 * cudaFree would synchronise the device).  Same arguments and result as dmrg_gemv_trans;
 * no cudaMalloc, cudaFree or other allocating routine is called.  The cross-block partial
 * sums live in one fixed scratch array inside the library (196,864 bytes, held by every GPU
 * that loads the library until the process exits); k above 24, the column count that array
 * holds, is rejected with DMRG_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current, so make that first
 * call before any stream capture.  All calls on a device share the array and it keeps the
 * last call's contents (the counter that must start at zero is cleared by every call);
 * calls that overlap on the GPU, e.g. from unordered streams, race on it.  Enqueued on
 * stream. */
dmrg_status dmrg_gemv_trans_noalloc(const double* V, int64_t ldv, int64_t n, int32_t k,
                                    const double* w, double* s, void* stream);

/* Davidson state: basis V, projections W, the small matrix B of Algorithm 3, started
 * from x0 (device, n float64, normalised by the call). */
dmrg_status dmrg_state_create(dmrg_plan* plan, const double* x0, void* stream,
                              dmrg_davidson_state** out);
/* Waits for the device to finish (as a cudaFree would) and hands the state's buffers to
 * its plan for the next state (dmrg_plan_trim frees them). */
void dmrg_state_destroy(dmrg_davidson_state* st);
/* One iteration of Algorithm 3.  Synchronises the stream; *converged is set to 1 when
 * the residual of the current Ritz pair is below tol. */
dmrg_status dmrg_davidson_step(dmrg_davidson_state* st, void* stream, int32_t* converged);
dmrg_status dmrg_state_get_info(const dmrg_davidson_state* st, dmrg_solve_info* info);
/* x_out = current Ritz vector V y (device, n float64).  Enqueued. */
dmrg_status dmrg_state_ritz(dmrg_davidson_state* st, double* x_out, void* stream);

/* Full Davidson solve from x0 (device) into x_out (device); info may be NULL.  Returns
 * DMRG_ERR_NOT_CONVERGED with x_out and info filled when max_iter is reached. */
dmrg_status dmrg_davidson_solve(dmrg_plan* plan, const double* x0, double* x_out,
                                dmrg_solve_info* info, void* stream);
/* Many independent superblock problems (each with its own plan, sector spectrum and size)
 * solved together: every Davidson iteration of all unconverged problems is enqueued, each
 * problem on its own stream, before one host wait for the whole batch, so small problems
 * overlap on the GPU and share the host round trips.  plans, x0 and x_out are host arrays
 * of nb pointers (x0[i], x_out[i] device vectors of plans[i]'s n); infos, if not NULL, has
 * nb entries.  Problems that share a plan run in order on one stream (a plan's scratch is
 * shared); give problems their own plans to let them overlap.  Work is ordered after the
 * caller's stream and the caller's stream waits for it.  Returns DMRG_ERR_NOT_CONVERGED if any problem stopped at its max_iter (the others'
 * results are valid; see infos[i].converged), or the first error met. */
dmrg_status dmrg_davidson_solve_batched(dmrg_plan* const* plans, int32_t nb,
                                        const double* const* x0, double* const* x_out,
                                        dmrg_solve_info* infos, void* stream);
/* Lowest nev eigenpairs by the block Davidson-Liu iteration that Sec. 6 names as the
 * block extension of Algorithm 3: every iteration adds the corrections of the unconverged
 * ones among the `block` lowest Ritz pairs (block >= nev), each orthonormalised (classical
 * Gram-Schmidt twice) against the basis and the corrections added before it; when they do
 * not fit in max_subspace columns the basis is collapsed to the current Ritz block and (with
 * restart_keep = 2) as much of the previous one as leaves room.  Projections are
 * FP64-accurate: the plan's precision if it is DMRG_PREC_FP64 or DMRG_PREC_FP64_TC, else its
 * anchor_prec; the vector passes are FP64.  X0: device, column-major n x block start block
 * (leading dimension ldx0 >= n), orthonormalised by the call (DMRG_ERR_INVALID_ARG if it is
 * rank deficient).  X_out: device, column-major n x nev (ldx_out >= n), the Ritz vectors of
 * the nev lowest pairs in ascending order.  energies (host, nev): their Ritz values;
 * resnorms (host, nev, may be NULL): ||H x - theta x||_2.  info (may be NULL): iters,
 * fp64_projections (all projections), restarts, converged; energy and resnorm of the lowest
 * pair.  Needs 1 <= nev <= block <= 8 and 2 block <= max_subspace.  Synchronizes the stream;
 * DMRG_ERR_NOT_CONVERGED with everything filled when max_iter is reached. */
dmrg_status dmrg_davidson_solve_block(dmrg_plan* plan, int32_t nev, int32_t block,
                                      const double* X0, int64_t ldx0, double* X_out,
                                      int64_t ldx_out, double* energies, double* resnorms,
                                      dmrg_solve_info* info, void* stream);

/* Same, with x0 and x_out in host memory: the host-to-device copy of x0 and the
 * device-to-host copy of x_out are part of the call. */
dmrg_status dmrg_davidson_solve_host(dmrg_plan* plan, const double* x0_host,
                                     double* x_out_host, dmrg_solve_info* info,
                                     void* stream);

/* 1 if projections in this precision are available in this build, else 0. */
int32_t dmrg_precision_available(dmrg_precision prec);

/* Number of kernels this library has launched in this process (all devices). */
int64_t dmrg_kernel_launches(void);

const char* dmrg_status_string(dmrg_status s);
const char* dmrg_last_error(void);
/* Library version string. */
const char* dmrg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DMRG_GB300_H */
