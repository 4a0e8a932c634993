// Low-precision projection on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// Eq. 11 is evaluated in the same two stages as the FP64 path (stage 1: one GEMM per
// record with two proper factors; stage 2: one GEMM per output segment whose K dimension
// concatenates every record writing that segment), but every GEMM runs as
//     D[128 x N] (FP32, in TMEM) += A_tile[128 x K] . B_tile[N x K]^T,  N = 128 or 256
// with both operands K-major in shared memory.  Three arithmetics:
//   TF32   : operands stored as FP32 rounded to TF32, one product per K step;
//   BF16x3 : every operand stored as three BF16 planes x = x0 + x1 + x2 (24 significant
//            bits); the six products x_i y_j with i + j <= 2 are accumulated in FP32;
//   BF16x2 : two BF16 planes x = x0 + x1 (about 17 significant bits); the three products
//            x0 y0 + x0 y1 + x1 y0 are accumulated in FP32.
//
// Operand tiles are "images": the exact shared-memory byte image of a 128-row x 32-element
// K-major tile in a swizzled canonical layout (BF16x3: 64-byte rows, 512-byte atoms; TF32:
// 128-byte rows, 1024-byte atoms; see Layout), zero-padded to whole tiles, with the planes
// of one (row tile, K tile) contiguous.  A tile therefore arrives in shared memory with ONE
// bulk asynchronous copy (cp.async.bulk, the TMA engine) and no bounds logic.  Operator
// blocks are packed once per plan (they are fixed during Davidson, Sec. 7); the Davidson
// vector is packed per projection in two forms (A-form: rows = left index; B-form: rows =
// right index); stage-1 epilogues write their results directly as images for stage 2.  The
// record order "X B^T first" is computed transposed, U^T = B X^T, so that every epilogue
// writes its accumulator rows as image rows.
//
// Kernel structure (persistent, one CTA per SM, 192 threads):
//   warp 0     producer: takes output tiles from the launch's tile list (the first one
//              blockIdx.x, the following ones from a global atomic counter, i.e. greedy
//              list scheduling in list order), publishes each tile index in a small
//              shared-memory ring for the other roles, and issues the bulk copies of its A
//              and B tiles into a ring of shared-memory stages
//   warp 1     allocates the TMEM accumulators (two of 128 or 256 FP32 columns) and one
//              lane issues tcgen05.mma; tcgen05.commit releases stages and publishes
//              accumulators
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes
//              32 (w % 4) .. + 31), then either an image of the result (stage 1) or FP64 Y
//              plus the identity-identity term (stage 2, from 16-lane loads so that the
//              stores write 64-byte row segments).  A stage-2 tile whose K range is
//              split into parts writes its FP32 partial sums to a scratch slot of its own;
//              a small kernel after the stage adds the slots in part order and writes Y,
//              so the result does not depend on which CTA ran which part.
// Every mbarrier wait is bounded (2 s of %globaltimer); on a timeout the kernel records an
// error code, stops issuing work, waits (bounded) for its own copies and MMAs, frees TMEM
// and returns.
#include <cuda_bf16.h>
#include <stdio.h>

#include <algorithm>
#include <functional>
#include <vector>
#include <map>
#include <tuple>

#include "internal.h"

namespace dmrg {

struct TcSeg {
  int64_t p_off, q_off;   // byte offsets of the first tile of the operand images
  int32_t p_buf, q_buf;   // which image buffer
  int32_t p_nkt, q_nkt;   // K tiles per row tile in each image
  int32_t nkt;            // K tiles of this segment
  int32_t pad_;
};

struct TcJob {
  int32_t seg_begin, seg_end;
  int32_t M, N;
  int32_t out_fp64;       // 0: write an image (stage 1), 1: write FP64 Y (stage 2)
  int32_t out_nkt;        // K tiles of the output image (stage 1)
  int64_t out_off;        // byte offset of the output image, or element offset in Y
  int64_t x_off;          // element offset of X for the identity-identity term
  double axpy;
};

struct TcTile {
  int32_t job, mt, nt, pad_;  // pad_: problem index in a grouped launch
  int32_t wide;               // 1: 256 output columns (row tiles nt and nt + 1 of B)
  int32_t kb, ke;             // K tiles [kb, ke) of the job's segments taken in order
  int32_t part, nparts;       // split K (FP64-output tiles only): part of nparts > 1
  int32_t red;                // split K: partial-sum slots red .. red + nparts - 1; -1 if
                              // not split
};

inline TcTile make_tile(int job, int mt, int nt, int prob, int wide, int kb, int ke) {
  return TcTile{job, mt, nt, prob, wide, kb, ke, 0, 1, -1};
}

struct PackJob {
  int64_t src_off;        // element offset in the FP64 source
  int64_t rs, cs;         // element (r, k) at src[src_off + r * rs + k * cs]
  int64_t dst_off;        // byte offset of the image
  int32_t R, K;
  int32_t nkt;
  int32_t src_space;      // 0: operator arena, 1: vector X
  double scale;
};

struct PackChunk {
  int32_t job, rt, kt, pad_;
};

enum TcBuf { TB_OPS = 0, TB_XA = 1, TB_XB = 2, TB_INTER = 3 };

// Per-problem pointers of a grouped launch over several plans (TcBatch): tiles and pack
// chunks carry the problem index; problems with active == 0 are skipped.
struct TcPtrs {
  const double* arena;
  const double* x;
  double* y;
  const float* x32;     // FP32 vector in and out instead of x, y when not NULL
  float* y32;
  const uint8_t* ops;
  uint8_t* xa;          // A-form and B-form vector images (one buffer)
  uint8_t* inter;
  int32_t active, pad_;
};

// Tile schedules: the tile shapes, the K split and the order of the tile list.  The CTAs
// of a launch take tiles from the list greedily (CTA b starts with tile b; each CTA that
// finishes a tile takes the next untaken one), so the list order is a priority order.
// Schedule c = (3 s + w) 3 + o combines order o:
//   0  tiles in descending estimated time (longest first: list scheduling in LPT order)
//   1  stage 1: jobs grouped by the vector image they read (all records of one (i, k)
//      segment and form together), tiles column-major; stage 2: output segments grouped
//      by their right sector l
//   2  stage 1: jobs grouped by the operator block image they read, tiles row-major;
//      stage 2: output segments grouped by their left sector j
// (groups in descending total cost, jobs within a group in descending cost), tile width
// policy w (BF16x3 only; TF32 tiles are always 128 x 128):
//   0  all tiles 128 columns
//   1  256 columns where the job has two B row tiles left and the tile's work stays below
//      half of the mean work per SM (wide tiles halve the B-operand traffic per FLOP, but
//      a long wide tile can become the critical path of the stage)
//   2  256 columns wherever possible
// and K split policy s (stage 2 only):
//   0  none
//   1  tiles estimated above 2/3 (s = 2: 2/5) of the mean time per SM are cut into parts
//      of whole K tiles below that bound; the parts are list entries of their own, and
//      a reduction launch after the stage adds their partial sums
// Schedules without a K split compute each output element with the same arithmetic, so
// their results are identical; a split changes the FP32 summation order of the split tiles
// (partial sums added in part order), which is deterministic for a given schedule.
constexpr int kOrders = 3, kWidths = 3, kSplits = 3;
constexpr int kSchedules = kOrders * kWidths * kSplits;
constexpr int kSlotFloats = 128 * 256;  // one split-K partial-sum slot (128 x 256 FP32)

struct TcPlan {
  dmrg_precision prec = DMRG_PREC_BF16X3;
  int planes = 3, kt_elems = 32;
  int64_t chunk = 0;  // bytes of one plane of one image tile
  uint8_t* buf[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t buf_bytes[4] = {0, 0, 0, 0};
  PackJob* d_xpack_jobs = nullptr;
  PackChunk* d_xpack_chunks = nullptr;
  int64_t n_xpack_chunks = 0;
  TcJob* d_jobs = nullptr;
  TcSeg* d_segs = nullptr;
  // candidate tile schedules of each stage (kSchedules, see build_tc); the kernels run
  // schedule sched[stage]
  TcTile* d_tiles[2][kSchedules] = {};
  int64_t ntiles[2][kSchedules] = {};
  bool valid[2][kSchedules] = {};  // candidates of each stage (TF32: narrow; stage 1: no split)
  int64_t ntiles1 = 0, ntiles2 = 0;  // tiles of schedule 0 (all narrow)
  int* d_ctr = nullptr;        // tile-list counters: 2 per stage, zero between launches
  float* d_partial = nullptr;  // split-K partial sums: nslots slots of kSlotFloats
  int64_t nslots = 0;
  TcTile* d_groups[kSchedules] = {};  // split-K tiles of each stage-2 schedule (part 0)
  int64_t ngroups[kSchedules] = {};
  int sched[2] = {0, 0};
  bool tuned = false;
  float tune_us[2][kSchedules] = {};
  int* d_err = nullptr;   // device view of a mapped host word: kernel error codes
  int* h_err = nullptr;
  int sms = 0;
  // host copies for grouped launches over several plans (TcBatch)
  std::vector<TcJob> h_jobs;
  std::vector<TcSeg> h_segs;
  std::vector<std::pair<int64_t, int>> h_order[2];  // (cost per tile, job), descending
  std::vector<PackJob> h_xjobs;
  std::vector<PackChunk> h_xchunks;
  // CUDA graphs of the projection's launch sequence (pack, both GEMM stages, the split-K
  // reduction), one per (x, y, x32, y32) vector pair under the current tile schedules,
  // captured on a plan-owned stream and replayed on the caller's stream; dropped when the
  // schedules change
  using GraphKey = std::tuple<const void*, const void*, const void*, const void*>;
  std::map<GraphKey, std::pair<cudaGraphExec_t, int>> graphs;  // -> (exec, kernel launches)
  cudaStream_t cap_st = nullptr;
};

// drops every captured projection graph of a tensor-core plan
void drop_graphs(TcPlan* t) {
  for (auto& g : t->graphs) cudaGraphExecDestroy(g.second.first);
  t->graphs.clear();
}

namespace tc {

constexpr int kThreads = 192;
constexpr int kRing = 8;  // tile indices in flight between the producer and the other roles

#include "tc_ptx.cuh"
#include "cvt.cuh"


// ---------------------------------------------------------------- packing kernel
// One CTA packs one image tile (128 rows x 128 bytes x planes) of one pack job from FP64.
template <int PLANES, bool TF32>
__global__ void __launch_bounds__(256)
pack_kernel(const PackChunk* __restrict__ chunks, const PackJob* __restrict__ jobs,
            const double* __restrict__ arena, const double* __restrict__ x,
            uint8_t* __restrict__ dst, const TcPtrs* __restrict__ ptrs,
            const float* __restrict__ x32) {
  using L = Layout<TF32>;
  constexpr int EPG = TF32 ? 4 : 8;  // elements per 16-byte group
  constexpr int KT = L::KT;
  grid_dep_wait();
  const PackChunk ch = chunks[blockIdx.x];
  if (ptrs) {  // grouped launch: the chunk's problem
    const TcPtrs& pt = ptrs[ch.pad_];
    if (!pt.active) return;
    arena = pt.arena;
    x = pt.x;
    x32 = pt.x32;
    dst = pt.xa;
  }
  const PackJob jb = jobs[ch.job];
  const double* src = (jb.src_space ? x : arena) + jb.src_off;
  // an FP32 vector (the low-precision basis columns of a mixed solve) is read as it is
  const float* src32 = (jb.src_space && x32) ? x32 + jb.src_off : nullptr;
  uint8_t* base = dst + jb.dst_off + ((int64_t)ch.rt * jb.nkt + ch.kt) * PLANES * L::CHUNK;
  const bool kfast = jb.cs == 1;
  for (int idx = threadIdx.x; idx < kRows * L::GROUPS; idx += blockDim.x) {
    int r, g;
    if (kfast) { g = idx % L::GROUPS; r = idx / L::GROUPS; }
    else { r = idx & (kRows - 1); g = idx >> 7; }
    const int64_t grow = (int64_t)ch.rt * kRows + r;
    const int k0 = ch.kt * KT + g * EPG;
    // operands are rounded to FP32 first (one conversion, no further FP64 arithmetic:
    // FP64 throughput is low on this part, and so is the hardware conversion, so the
    // rounding is done with integer operations); the three BF16 terms of an FP32 value
    // represent it exactly
    const bool scaled = jb.scale != 1.0;
    float v[EPG];
#pragma unroll
    for (int e = 0; e < EPG; ++e) {
      const int k = k0 + e;
      const bool in = grow < jb.R && k < jb.K;
      const int64_t at = grow * jb.rs + (int64_t)k * jb.cs;
      if (src32) {
        v[e] = in ? src32[at] : 0.0f;
      } else {
        const double a = in ? src[at] : 0.0;
        v[e] = scaled ? (float)(jb.scale * a) : f64_to_f32_rn(a);
      }
    }
    const uint32_t off = L::off(r, g);
    if constexpr (TF32) {
      uint4 q;
      q.x = __float_as_uint(to_tf32(v[0]));
      q.y = __float_as_uint(to_tf32(v[1]));
      q.z = __float_as_uint(to_tf32(v[2]));
      q.w = __float_as_uint(to_tf32(v[3]));
      *reinterpret_cast<uint4*>(base + off) = q;
    } else {
      __nv_bfloat16 h[3][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float a = v[e];
        const __nv_bfloat16 h0 = __float2bfloat16_rn(a);
        const float r1 = a - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(h1);
        h[0][e] = h0;
        h[1][e] = h1;
        h[2][e] = __float2bfloat16_rn(r2);
      }
#pragma unroll
      for (int p = 0; p < PLANES; ++p) {
        uint4 q;
        q.x = pack2_bf16(h[p][0], h[p][1]);
        q.y = pack2_bf16(h[p][2], h[p][3]);
        q.z = pack2_bf16(h[p][4], h[p][5]);
        q.w = pack2_bf16(h[p][6], h[p][7]);
        *reinterpret_cast<uint4*>(base + p * L::CHUNK + off) = q;
      }
    }
  }
  grid_dep_launch();
}

// products of plane pairs per K step: TF32 1, BF16x2 3, BF16x3 6
template <int PLANES>
__host__ __device__ constexpr int kProducts() {
  return PLANES == 3 ? 6 : PLANES == 2 ? 3 : 1;
}

// ---------------------------------------------------------------- grouped GEMM kernel
// WIDE: tiles may be 256 columns wide (N = 256 MMA, B operand = two 128-row image tiles,
// each plane of B in a 2 x CHUNK slot so that its 256 rows are contiguous; TMEM holds two
// 256-column accumulators).  Otherwise every tile is 128 x 128.
template <int PLANES, int STAGES, bool TF32, bool WIDE>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const TcTile* __restrict__ tiles, int ntiles, const TcJob* __restrict__ jobs,
               const TcSeg* __restrict__ segs, const uint8_t* __restrict__ b0,
               const uint8_t* __restrict__ b1, const uint8_t* __restrict__ b2,
               const uint8_t* __restrict__ b3, uint8_t* __restrict__ out_img,
               double* __restrict__ y, const double* __restrict__ x, int* __restrict__ gerr,
               const TcPtrs* __restrict__ ptrs, int gemm_stage, int* __restrict__ tile_ctr,
               float* __restrict__ partial, float* __restrict__ y32,
               const float* __restrict__ x32) {
  using L = Layout<TF32>;
  constexpr uint32_t kStageA = PLANES * L::CHUNK;             // A operand of one stage
  constexpr uint32_t kSlotB = (WIDE ? 2 : 1) * L::CHUNK;      // one plane of B
  constexpr uint32_t kStage = kStageA + PLANES * kSlotB;
  constexpr int kAccCols = WIDE ? 256 : 128;                  // columns of one accumulator
  constexpr uint32_t kTmemCols = 2 * kAccCols;
  constexpr int KT = L::KT;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ __align__(8) uint64_t tq_full[kRing], tq_empty[kRing];
  __shared__ int tile_ring[kRing];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull_bar[a]), 1);
      mbar_init(smem_u32(&tempty_bar[a]), 128);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    for (int r = 0; r < kRing; ++r) {
      mbar_init(smem_u32(&tq_full[r]), 1);
      mbar_init(smem_u32(&tq_empty[r]), 5);  // one lane of the MMA warp and of each epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  grid_dep_wait();  // inputs of this launch are written by the previous one
  // grouped launch (ptrs != NULL): the operand buffers and outputs of each tile are those
  // of its problem (tile.pad_), and tiles of inactive problems are skipped by all roles
  auto active = [&](const TcTile& tile) { return !ptrs || ptrs[tile.pad_].active != 0; };
  // consumer side of the tile ring: the next tile index, -1 at the end (or on abort);
  // called by a whole warp (the MMA warp, each epilogue warp: one arrival per warp)
  auto next_tile = [&](int& slot, uint32_t& phase, bool whole_warp, int code) -> int {
    const bool ok = whole_warp ? mbar_wait_warp(smem_u32(&tq_full[slot]), phase, &abort_flag, gerr, code)
                               : mbar_wait(smem_u32(&tq_full[slot]), phase, &abort_flag, gerr, code);
    if (!ok) return -1;
    const int t = tile_ring[slot];
    if (whole_warp) __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(smem_u32(&tq_empty[slot]));
    if (++slot == kRing) { slot = 0; phase ^= 1; }
    return t;
  };

  if (warp == 0) {
    // ------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t issued = 0;
      int rslot = 0;
      uint32_t rphase = 0;
      for (int t = blockIdx.x;;) {
        // publish the tile (-1: none left) to the MMA and epilogue warps
        if (!mbar_wait(smem_u32(&tq_empty[rslot]), rphase ^ 1, &abort_flag, gerr, 5)) break;
        const bool done = t >= ntiles || abort_flag;
        tile_ring[rslot] = done ? -1 : t;
        mbar_arrive(smem_u32(&tq_full[rslot]));
        if (++rslot == kRing) { rslot = 0; rphase ^= 1; }
        if (done) {
          grid_dep_launch();  // no tile left to take: the next launch may be scheduled
          break;
        }
        // the following tile, taken now and used once this one's copies are issued
        const int t_next = (int)gridDim.x + atomicAdd(tile_ctr, 1);
        const TcTile tile = tiles[t];
        t = t_next;
        if (!active(tile)) continue;
        const uint8_t* bufs[4] = {b0, b1, b2, b3};
        if (ptrs) {
          const TcPtrs& pt = ptrs[tile.pad_];
          bufs[0] = pt.ops;
          bufs[1] = bufs[2] = pt.xa;
          bufs[3] = gemm_stage == 2 ? pt.inter : nullptr;
        }
        const TcJob job = jobs[tile.job];
        int kbase = 0;  // K tiles of the job's earlier segments
        for (int si = job.seg_begin; si < job.seg_end && !abort_flag; ++si) {
          const TcSeg sg = segs[si];
          const int k_lo = max(tile.kb - kbase, 0), k_hi = min(tile.ke - kbase, sg.nkt);
          kbase += sg.nkt;
          const uint8_t* P = bufs[sg.p_buf] + sg.p_off + (int64_t)tile.mt * sg.p_nkt * kStageA;
          const uint8_t* Q = bufs[sg.q_buf] + sg.q_off + (int64_t)tile.nt * sg.q_nkt * kStageA;
          const bool wide = WIDE && tile.wide;
          for (int kt = k_lo; kt < k_hi; ++kt) {
            if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, gerr, 1)) break;
            const uint32_t sa = smem_u32(smem + stage * kStage);
            const uint32_t fb = smem_u32(&full_bar[stage]);
            const uint8_t* q0 = Q + (int64_t)kt * kStageA;
            mbar_expect_tx(fb, kStageA + (wide ? 2u : 1u) * PLANES * L::CHUNK);
            bulk_g2s(sa, P + (int64_t)kt * kStageA, kStageA, fb);
            if constexpr (WIDE) {
              // plane p of B rows 0-127 (and 128-255) into the slot of plane p
#pragma unroll
              for (int pl = 0; pl < PLANES; ++pl) {
                bulk_g2s(sa + kStageA + pl * kSlotB, q0 + pl * L::CHUNK, L::CHUNK, fb);
                if (wide)
                  bulk_g2s(sa + kStageA + pl * kSlotB + L::CHUNK,
                           q0 + (int64_t)sg.q_nkt * kStageA + pl * L::CHUNK, L::CHUNK, fb);
              }
            } else {
              bulk_g2s(sa + kStageA, q0, kStageA, fb);
            }
            ++issued;
            if (++stage == STAGES) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (abort_flag) {
        // wait (bounded) for the copies still in flight: the last min(issued, STAGES) loads
        int s = stage;
        uint32_t ph = phase;
        for (int i = 0; i < STAGES && i < issued; ++i) {
          if (--s < 0) { s = STAGES - 1; ph ^= 1; }
          const uint64_t t0 = gtime();
          while (!mbar_try_wait(smem_u32(&full_bar[s]), ph) && gtime() - t0 < kWaitNs) {}
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    // The whole warp runs the loop in step (its control flow and the descriptors stay
    // warp-uniform); lane 0 alone issues the MMAs and the commits that track them.
    const bool leader = lane == 0;
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool any = false;
    constexpr uint32_t idesc128 = instr_desc<TF32, 128>();
    constexpr uint32_t idesc256 = instr_desc<TF32, 256>();
    int rslot = 0;
    uint32_t rphase = 0;
    while (!abort_flag) {
      const int t = next_tile(rslot, rphase, true, 6);
      if (t < 0) break;
      const TcTile tile = tiles[t];
      if (!active(tile) || tile.kb >= tile.ke) continue;
      const TcJob job = jobs[tile.job];
      const uint32_t idesc = (WIDE && tile.wide) ? idesc256 : idesc128;
      if (!mbar_wait_warp(smem_u32(&tempty_bar[acc]), acc_phase ^ 1, &abort_flag, gerr, 2)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * kAccCols);
      uint32_t accumulate = 0;
      int kbase = 0;
      for (int si = job.seg_begin; si < job.seg_end && !abort_flag; ++si) {
        const int nkt = segs[si].nkt;
        const int k_lo = max(tile.kb - kbase, 0), k_hi = min(tile.ke - kbase, nkt);
        kbase += nkt;
        for (int kt = k_lo; kt < k_hi; ++kt) {
          if (!mbar_wait_warp(smem_u32(&full_bar[stage]), phase, &abort_flag, gerr, 3)) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * kStage);
          const uint32_t sb = sa + kStageA;
#pragma unroll
          for (int pr = 0; pr < kProducts<PLANES>(); ++pr) {
            // plane pairs (pa, pb) with pa + pb < PLANES: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
            const int pa = pr == 0 ? 0 : pr == 1 ? 0 : pr == 2 ? 1 : pr == 3 ? 0 : pr == 4 ? 1 : 2;
            const int pb = pr == 0 ? 0 : pr == 1 ? 1 : pr == 2 ? 0 : pr == 3 ? 2 : pr == 4 ? 1 : 0;
#pragma unroll
            for (int kk = 0; kk < L::ROWB / 32; ++kk) {  // one MMA per 32 bytes of K
              const uint64_t ad = L::desc(sa + pa * L::CHUNK + kk * 32);
              const uint64_t bd = L::desc(sb + pb * kSlotB + kk * 32);
              if (leader) mma<TF32>(d_tmem, ad, bd, idesc, accumulate);
              accumulate = 1;
            }
          }
          if (leader) tc_commit(smem_u32(&empty_bar[stage]));
          __syncwarp();
          any = true;
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (leader) tc_commit(smem_u32(&tfull_bar[acc]));
      __syncwarp();
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
    if (any && leader) {
      // all MMAs issued by this thread complete before TMEM is released
      tc_commit(smem_u32(&drain_bar));
      const uint64_t t0 = gtime();
      while (!mbar_try_wait(smem_u32(&drain_bar), 0) && gtime() - t0 < kWaitNs) {}
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2..5)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    int rslot = 0;
    uint32_t rphase = 0;
    for (;;) {
      const int t = next_tile(rslot, rphase, true, 7);
      if (t < 0) break;
      const TcTile tile = tiles[t];
      if (!active(tile)) continue;
      uint8_t* o_img = out_img;
      double* o_y = y;
      const double* i_x = x;
      float* o_y32 = y32;
      const float* i_x32 = x32;
      if (ptrs) {
        const TcPtrs& pt = ptrs[tile.pad_];
        o_img = gemm_stage == 1 ? pt.inter : nullptr;
        o_y = pt.y;
        i_x = pt.x;
        o_y32 = pt.y32;
        i_x32 = pt.x32;
      }
      const TcJob job = jobs[tile.job];
      const bool has = tile.kb < tile.ke;
      const bool split = tile.nparts > 1;
      if (has) {
        if (!mbar_wait(smem_u32(&tfull_bar[acc]), acc_phase, &abort_flag, gerr, 4)) break;
        tc_fence_after();
      }
      const int ncols = (WIDE && tile.wide) ? 256 : 128;
      if (job.out_fp64) {
        // FP64 Y (or the FP32 partial sums of a split part) from 16-lane TMEM loads: four
        // consecutive threads hold eight consecutive columns of one row, so each store
        // instruction writes 64-byte row segments instead of one element of 32 rows
        for (int c0 = 0; c0 < ncols; c0 += 32) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t v[16];
            if (has) {
              tmem_ld16x256_x4(tmem_base + ((uint32_t)(quarter * 32 + half * 16) << 16) +
                                   (uint32_t)(acc * kAccCols + c0), v);
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
              const int r = quarter * 32 + half * 16 + hr * 8 + (lane >> 2);
              const int64_t mr = (int64_t)tile.mt * kRows + r;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int cc = c0 + 8 * j + 2 * (lane & 3);  // column in the tile
                const float f0 = __uint_as_float(v[4 * j + 2 * hr]);
                const float f1 = __uint_as_float(v[4 * j + 2 * hr + 1]);
                if (split) {
                  // partial sums of this part: slot red + part, row-major 128 x 256
                  *reinterpret_cast<float2*>(partial + (int64_t)(tile.red + tile.part) * kSlotFloats +
                                             r * 256 + cc) = make_float2(f0, f1);
                } else if (mr < job.M && o_y32) {
                  // FP32 output (a low-precision basis column of a mixed solve)
                  const int n = tile.nt * kRows + cc;
                  float* yp = o_y32 + job.out_off + mr * job.N + n;
                  float e0 = f0, e1 = f1;
                  if (job.axpy != 0.0) {
                    const float* xp = i_x32 + job.x_off + mr * job.N + n;
                    const float a = (float)job.axpy;
                    if (n < job.N) e0 = fmaf(a, xp[0], e0);
                    if (n + 1 < job.N) e1 = fmaf(a, xp[1], e1);
                  }
                  if (n + 1 < job.N && (reinterpret_cast<uintptr_t>(yp) & 7) == 0) {
                    *reinterpret_cast<float2*>(yp) = make_float2(e0, e1);
                  } else {
                    if (n < job.N) yp[0] = e0;
                    if (n + 1 < job.N) yp[1] = e1;
                  }
                } else if (mr < job.M) {
                  const int n = tile.nt * kRows + cc;
                  double* yp = o_y + job.out_off + mr * job.N + n;
                  double d0 = f32_to_f64(f0), d1 = f32_to_f64(f1);  // exact, integer ops
                  if (job.axpy != 0.0) {
                    const double* xp = i_x + job.x_off + mr * job.N + n;
                    if (n < job.N) d0 = fma(job.axpy, xp[0], d0);
                    if (n + 1 < job.N) d1 = fma(job.axpy, xp[1], d1);
                  }
                  if (n + 1 < job.N && (reinterpret_cast<uintptr_t>(yp) & 15) == 0) {
                    *reinterpret_cast<double2*>(yp) = make_double2(d0, d1);
                  } else {
                    if (n < job.N) yp[0] = d0;
                    if (n + 1 < job.N) yp[1] = d1;
                  }
                }
              }
            }
          }
        }
      } else {
        for (int c0 = 0; c0 < ncols; c0 += 32) {
          uint32_t v[32];
          if (has) {
            tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * kAccCols + c0), v);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0u;
          }
          const int n0 = tile.nt * kRows + c0;
          const int kt = n0 / KT;
          if (kt < job.out_nkt) {
            uint8_t* tb = o_img + job.out_off + ((int64_t)tile.mt * job.out_nkt + kt) * PLANES * L::CHUNK;
            if constexpr (TF32) {
#pragma unroll
              for (int g = 0; g < 8; ++g) {
                uint4 q;
                q.x = __float_as_uint(to_tf32(__uint_as_float(v[4 * g + 0])));
                q.y = __float_as_uint(to_tf32(__uint_as_float(v[4 * g + 1])));
                q.z = __float_as_uint(to_tf32(__uint_as_float(v[4 * g + 2])));
                q.w = __float_as_uint(to_tf32(__uint_as_float(v[4 * g + 3])));
                *reinterpret_cast<uint4*>(tb + L::off(row, g)) = q;
              }
            } else {
              const int gbase = (n0 % KT) / 8;
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                uint32_t w0[4], w1[4], w2[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  __nv_bfloat16 h[2][3];
#pragma unroll
                  for (int u = 0; u < 2; ++u) {
                    const float f = __uint_as_float(v[8 * g + 2 * e + u]);
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(f);
                    const float r1 = f - __bfloat162float(h0);
                    const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
                    const float r2 = r1 - __bfloat162float(h1);
                    h[u][0] = h0;
                    h[u][1] = h1;
                    h[u][2] = __float2bfloat16_rn(r2);
                  }
                  w0[e] = pack2_bf16(h[0][0], h[1][0]);
                  w1[e] = pack2_bf16(h[0][1], h[1][1]);
                  w2[e] = pack2_bf16(h[0][2], h[1][2]);
                }
                const uint32_t off = L::off(row, gbase + g);
                *reinterpret_cast<uint4*>(tb + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
                *reinterpret_cast<uint4*>(tb + L::CHUNK + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
                if constexpr (PLANES == 3)
                  *reinterpret_cast<uint4*>(tb + 2 * L::CHUNK + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
              }
            }
          }
        }
      }
      if (has) {
        tc_fence_before();
        mbar_arrive(smem_u32(&tempty_bar[acc]));
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0) {
    // every CTA has taken its last tile: the last one to finish zeroes the tile counter
    // for the next launch
    __threadfence();
    if (atomicAdd(tile_ctr + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(tile_ctr, 0);
      atomicExch(tile_ctr + 1, 0);
    }
  }
}

// Split K: sums the FP32 partial sums of each split tile in part order (slots red ..
// red + nparts - 1, row-major 128 x 256) and writes FP64 Y plus the identity-identity
// term.  32 CTAs of 256 threads per split tile, 4 consecutive values per thread.
__global__ void __launch_bounds__(256)
split_reduce_kernel(const TcTile* __restrict__ groups, const TcJob* __restrict__ jobs,
                    const float* __restrict__ partial, double* __restrict__ y,
                    const double* __restrict__ x, float* __restrict__ y32,
                    const float* __restrict__ x32) {
  grid_dep_wait();
  const TcTile g = groups[blockIdx.x >> 5];
  const TcJob job = jobs[g.job];
  const int idx = (((int)blockIdx.x & 31) * 256 + (int)threadIdx.x) * 4;
  const int row = idx >> 8, col = idx & 255;
  const int64_t m = (int64_t)g.mt * kRows + row;
  if (col < (g.wide ? 256 : 128) && m < job.M) {
    const float* src = partial + (int64_t)g.red * kSlotFloats + idx;
    float4 s = __ldcg(reinterpret_cast<const float4*>(src));
    for (int p = 1; p < g.nparts; ++p) {
      const float4 q = __ldcg(reinterpret_cast<const float4*>(src + (int64_t)p * kSlotFloats));
      s.x += q.x;
      s.y += q.y;
      s.z += q.z;
      s.w += q.w;
    }
    const float v[4] = {s.x, s.y, s.z, s.w};
    const int n0 = g.nt * kRows + col;
    if (y32) {
      float* yr = y32 + job.out_off + m * job.N;
      const float* xr = x32 + job.x_off + m * job.N;
      const float a = (float)job.axpy;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n = n0 + e;
        if (n < job.N) yr[n] = job.axpy != 0.0 ? fmaf(a, xr[n], v[e]) : v[e];
      }
    } else {
      double* yr = y + job.out_off + m * job.N;
      const double* xr = x + job.x_off + m * job.N;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int n = n0 + e;
        if (n < job.N) {
          double val = f32_to_f64(v[e]);  // exact, integer ops
          if (job.axpy != 0.0) val = fma(job.axpy, xr[n], val);
          yr[n] = val;
        }
      }
    }
  }
  grid_dep_launch();
}

template <int PLANES, int STAGES, bool TF32, bool WIDE>
constexpr size_t smem_bytes() {
  return (size_t)STAGES * (PLANES * Layout<TF32>::CHUNK * (WIDE ? 3 : 2)) + 1024;
}

}  // namespace tc

// ======================================================================== host side
namespace {

using tc::kRows;

int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

struct ImageAlloc {
  int64_t bytes = 0;
  int64_t chunk = 0;  // bytes of one plane of one image tile
  int64_t add(int64_t rows, int64_t K, int planes, int kt_elems, int* nkt_out) {
    const int nrt = ceil_div(rows, kRows), nkt = ceil_div(K, kt_elems);
    *nkt_out = nkt;
    const int64_t off = bytes;
    bytes += (int64_t)nrt * nkt * planes * chunk;
    return off;
  }
};

template <typename T>
dmrg_status upload_vec(T** dst, const std::vector<T>& v, cudaStream_t st) {
  *dst = nullptr;
  if (v.empty()) return DMRG_OK;
  DMRG_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * v.size()));
  DMRG_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return DMRG_OK;
}

void free_tc(TcPlan* t) {
  if (!t) return;
  drop_graphs(t);
  if (t->cap_st) cudaStreamDestroy(t->cap_st);
  for (int b = 0; b < 4; ++b)
    if (b != TB_XB) cudaFree(t->buf[b]);
  if (t->h_err) cudaFreeHost(t->h_err);
  cudaFree(t->d_xpack_jobs);
  cudaFree(t->d_xpack_chunks);
  cudaFree(t->d_jobs);
  cudaFree(t->d_segs);
  cudaFree(t->d_ctr);
  cudaFree(t->d_partial);
  for (TcTile* d : t->d_groups) cudaFree(d);
  for (auto& st : t->d_tiles)
    for (TcTile* d : st) cudaFree(d);
  delete t;
}

template <int PLANES, bool TF32>
dmrg_status launch_pack(const std::vector<PackChunk>& chunks, const PackChunk* d_chunks,
                        const PackJob* d_jobs, const double* arena, const double* x,
                        uint8_t* dst, cudaStream_t st) {
  if (chunks.empty()) return DMRG_OK;
  tc::pack_kernel<PLANES, TF32><<<(unsigned)chunks.size(), 256, 0, st>>>(d_chunks, d_jobs, arena, x, dst,
                                                                          nullptr, nullptr);
  DMRG_LAUNCH_CHECK();
  return DMRG_OK;
}

// Checks that every operand tile a GEMM tile reads and every output it writes lie inside
// the plan's buffers (byte sizes buf_bytes, TB_XB aliasing TB_XA; y has n elements).
bool tc_tiles_in_range(const TcPlan* t, int64_t n, const std::vector<TcJob>& jobs,
                       const std::vector<TcSeg>& segs, const std::vector<TcTile>& tiles,
                       int job_base, int seg_base, char* why, size_t why_len) {
  const int64_t stageA = (int64_t)t->planes * t->chunk;
  auto bytes = [&](int b) { return (int64_t)t->buf_bytes[b == TB_XB ? TB_XA : b]; };
  for (const TcTile& tl : tiles) {
    const TcJob& j = jobs[tl.job - job_base];
    int64_t job_kt = 0;
    for (int si = j.seg_begin; si < j.seg_end; ++si) job_kt += segs[si - seg_base].nkt;
    if (tl.kb < 0 || tl.ke < tl.kb || tl.ke > job_kt) {
      snprintf(why, why_len, "tile (job %d, %d, %d) has K range [%d, %d) outside 0..%lld",
               tl.job, tl.mt, tl.nt, tl.kb, tl.ke, (long long)job_kt);
      return false;
    }
    if (tl.nparts < 1 || (tl.nparts > 1 && (!j.out_fp64 || tl.part < 0 || tl.part >= tl.nparts || tl.red < 0 ||
                          (int64_t)tl.red + tl.nparts > t->nslots))) {
      snprintf(why, why_len, "tile (job %d, %d, %d) has bad split-K fields", tl.job, tl.mt, tl.nt);
      return false;
    }
    for (int si = j.seg_begin; si < j.seg_end; ++si) {
      const TcSeg& sg = segs[si - seg_base];
      const int64_t pe = sg.p_off + ((int64_t)tl.mt * sg.p_nkt + sg.nkt) * stageA;
      const int64_t qe = sg.q_off + ((int64_t)(tl.nt + (tl.wide ? 1 : 0)) * sg.q_nkt + sg.nkt) * stageA;
      if (sg.p_off < 0 || pe > bytes(sg.p_buf) || sg.q_off < 0 || qe > bytes(sg.q_buf)) {
        snprintf(why, why_len, "tile (job %d, %d, %d) segment %d reads outside its operand images",
                 tl.job, tl.mt, tl.nt, si);
        return false;
      }
    }
    if (j.out_fp64) {
      if (j.out_off < 0 || j.out_off + (int64_t)j.M * j.N > n || j.x_off < 0 ||
          j.x_off + (int64_t)j.M * j.N > n) {
        snprintf(why, why_len, "tile (job %d) writes outside y or reads outside x", tl.job);
        return false;
      }
    } else if (j.out_off < 0 ||
               j.out_off + ((int64_t)tl.mt * j.out_nkt + j.out_nkt) * stageA > bytes(TB_INTER)) {
      snprintf(why, why_len, "tile (job %d, %d, %d) writes outside the intermediate images",
               tl.job, tl.mt, tl.nt);
      return false;
    }
  }
  return true;
}

dmrg_status build_tc(dmrg_plan* p, dmrg_precision prec, cudaStream_t st, TcPlan** out) {
  TcPlan* t = new TcPlan();
  t->prec = prec;
  const bool tf32 = prec == DMRG_PREC_TF32;
  t->planes = tf32 ? 1 : prec == DMRG_PREC_BF16X2 ? 2 : 3;
  t->kt_elems = tf32 ? tc::Layout<true>::KT : tc::Layout<false>::KT;
  t->chunk = tf32 ? tc::Layout<true>::CHUNK : tc::Layout<false>::CHUNK;
  const int planes = t->planes, KT = t->kt_elems;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev);
  auto fail = [&](dmrg_status s) { free_tc(t); return s; };

  // ---- operator images, keyed by (side, op, block, scale)
  ImageAlloc ops_alloc;
  ops_alloc.chunk = t->chunk;
  std::vector<PackJob> op_jobs;
  std::map<std::tuple<int, int, int, double>, std::pair<int64_t, int>> op_img;  // -> (off, nkt)
  auto op_image = [&](int side, int op, int blk, double scale) -> std::pair<int64_t, int> {
    auto key = std::make_tuple(side, op, blk, scale);
    auto it = op_img.find(key);
    if (it != op_img.end()) return it->second;
    const HostBlock& hb = side == 0 ? p->opsL[op][blk] : p->opsR[op][blk];
    int nkt = 0;
    const int64_t off = ops_alloc.add(hb.rows, hb.cols, planes, KT, &nkt);
    PackJob j{};
    j.src_off = hb.arena_off;
    j.rs = hb.cols;
    j.cs = 1;
    j.dst_off = off;
    j.R = (int32_t)hb.rows;
    j.K = (int32_t)hb.cols;
    j.nkt = nkt;
    j.src_space = 0;
    j.scale = scale;
    op_jobs.push_back(j);
    op_img[key] = {off, nkt};
    return {off, nkt};
  };

  // ---- vector images (A-form rows = left index, B-form rows = right index)
  const int npairs = (int)p->pair_i.size();
  ImageAlloc xa_alloc;  // both forms share one buffer: A-form tiles, then B-form tiles
  xa_alloc.chunk = t->chunk;
  std::vector<PackJob> x_jobs;
  std::vector<std::pair<int64_t, int>> xa(npairs), xb(npairs);
  for (int q = 0; q < npairs; ++q) {
    const int64_t di = p->dimL[p->pair_i[q]], dk = p->dimR[p->pair_k[q]];
    int nkt = 0;
    int64_t off = xa_alloc.add(di, dk, planes, KT, &nkt);
    xa[q] = {off, nkt};
    if (di * dk > 0) {
      PackJob j{p->pair_off[q], dk, 1, off, (int32_t)di, (int32_t)dk, nkt, 1, 1.0};
      j.dst_off = off;
      x_jobs.push_back(j);
    }
    off = xa_alloc.add(dk, di, planes, KT, &nkt);
    xb[q] = {off, nkt};
    if (di * dk > 0) {
      PackJob j{p->pair_off[q], 1, dk, off, (int32_t)dk, (int32_t)di, nkt, 1, 1.0};
      x_jobs.push_back(j);
    }
  }

  // ---- jobs
  ImageAlloc inter_alloc;
  inter_alloc.chunk = t->chunk;
  std::vector<TcJob> jobs;
  std::vector<TcSeg> segs;
  std::vector<TcTile> tiles1, tiles2;
  std::vector<std::pair<int64_t, int>> inter(p->records.size(), {-1, 0});
  std::vector<std::pair<int64_t, int>> order1, order2;
  auto seg = [](int pbuf, std::pair<int64_t, int> P, int qbuf, std::pair<int64_t, int> Q, int nkt) {
    TcSeg s{};
    s.p_off = P.first;
    s.p_nkt = P.second;
    s.p_buf = pbuf;
    s.q_off = Q.first;
    s.q_nkt = Q.second;
    s.q_buf = qbuf;
    s.nkt = nkt;
    return s;
  };
  for (size_t ri = 0; ri < p->records.size(); ++ri) {
    const Record& r = p->records[ri];
    if (r.a_blk < 0 || r.b_blk < 0) continue;
    const int a_op = p->terms[r.term].a_op, b_op = p->terms[r.term].b_op;
    TcJob job{};
    job.out_fp64 = 0;
    job.axpy = 0.0;
    job.seg_begin = (int32_t)segs.size();
    int nkt_out = 0;
    if (r.a_first) {  // T [dj x dk] = A [dj x di] X [di x dk]
      job.M = (int32_t)r.dj;
      job.N = (int32_t)r.dk;
      const int64_t off = inter_alloc.add(r.dj, r.dk, planes, KT, &nkt_out);
      job.out_off = off;
      job.out_nkt = nkt_out;
      inter[ri] = {off, nkt_out};
      if (r.di > 0)
        segs.push_back(seg(TB_OPS, op_image(0, a_op, r.a_blk, 1.0), TB_XB, xb[r.pin], ceil_div(r.di, KT)));
    } else {          // U^T [dl x di] = (coef B) [dl x dk] X^T [dk x di]
      job.M = (int32_t)r.dl;
      job.N = (int32_t)r.di;
      const int64_t off = inter_alloc.add(r.dl, r.di, planes, KT, &nkt_out);
      job.out_off = off;
      job.out_nkt = nkt_out;
      inter[ri] = {off, nkt_out};
      if (r.dk > 0)
        segs.push_back(seg(TB_OPS, op_image(1, b_op, r.b_blk, r.coef), TB_XA, xa[r.pin], ceil_div(r.dk, KT)));
    }
    job.seg_end = (int32_t)segs.size();
    if (job.M > 0 && job.N > 0) {
      int64_t cost = 0;
      for (int s = job.seg_begin; s < job.seg_end; ++s) cost += segs[s].nkt;
      order1.push_back({cost, (int)jobs.size()});
    }
    jobs.push_back(job);
  }
  std::vector<std::vector<int>> by_out(npairs);
  for (size_t ri = 0; ri < p->records.size(); ++ri) by_out[p->records[ri].pout].push_back((int)ri);
  std::vector<int> stage2_job(npairs, -1);
  for (int q = 0; q < npairs; ++q) {
    const int i = p->pair_i[q], k = p->pair_k[q];
    stage2_job[q] = (int)jobs.size();
    TcJob job{};
    job.M = (int32_t)p->dimL[i];
    job.N = (int32_t)p->dimR[k];
    job.out_fp64 = 1;
    job.out_off = p->pair_off[q];
    job.x_off = p->pair_off[q];
    job.axpy = 0.0;
    job.seg_begin = (int32_t)segs.size();
    for (int ri : by_out[q]) {
      const Record& r = p->records[ri];
      const int a_op = p->terms[r.term].a_op, b_op = p->terms[r.term].b_op;
      if (r.a_blk >= 0 && r.b_blk >= 0) {
        if (r.a_first) {
          if (r.dk > 0)
            segs.push_back(seg(TB_INTER, inter[ri], TB_OPS, op_image(1, b_op, r.b_blk, r.coef), ceil_div(r.dk, KT)));
        } else {
          if (r.di > 0)
            segs.push_back(seg(TB_OPS, op_image(0, a_op, r.a_blk, 1.0), TB_INTER, inter[ri], ceil_div(r.di, KT)));
        }
      } else if (r.a_blk >= 0) {   // (coef A) X_{il}, k == l
        if (r.di > 0)
          segs.push_back(seg(TB_OPS, op_image(0, a_op, r.a_blk, r.coef), TB_XB, xb[r.pin], ceil_div(r.di, KT)));
      } else if (r.b_blk >= 0) {   // X_{jk} (coef B)^T, i == j
        if (r.dk > 0)
          segs.push_back(seg(TB_XA, xa[r.pin], TB_OPS, op_image(1, b_op, r.b_blk, r.coef), ceil_div(r.dk, KT)));
      } else {
        if (r.pin == r.pout) job.axpy += r.coef;  // (other segments: seg_axpy pass)
      }
    }
    job.seg_end = (int32_t)segs.size();
    if (job.M > 0 && job.N > 0) {
      int64_t cost = 0;
      for (int s = job.seg_begin; s < job.seg_end; ++s) cost += segs[s].nkt;
      order2.push_back({cost, (int)jobs.size()});
    }
    jobs.push_back(job);
  }
  auto by_cost = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  };
  std::stable_sort(order1.begin(), order1.end(), by_cost);
  std::stable_sort(order2.begin(), order2.end(), by_cost);
  // work of a 128 x 128 tile of each job (K tiles) and the mean narrow work per SM
  std::vector<int64_t> job_cost(jobs.size(), 0);
  int64_t mean_work[2] = {0, 0};
  for (int g = 0; g < 2; ++g) {
    for (const auto& pr : g == 0 ? order1 : order2) {
      job_cost[pr.second] = pr.first;
      const TcJob& j = jobs[pr.second];
      mean_work[g] += pr.first * ceil_div(j.M, kRows) * ceil_div(j.N, kRows);
    }
    mean_work[g] /= std::max(1, t->sms);
  }
  int wpol = 0, cur_stage = 0;  // width policy and stage of the schedule being built
  auto add_tiles = [&](std::vector<TcTile>& dst, int jb, bool col_major) {
    const TcJob& j = jobs[jb];
    const int nm = ceil_div(j.M, kRows), nn = ceil_div(j.N, kRows);
    const bool may_wide = !tf32 && (wpol == 2 || (wpol == 1 && 4 * job_cost[jb] <= mean_work[cur_stage]));
    auto width = [&](int nt) { return (may_wide && nt + 1 < nn) ? 2 : 1; };
    const int ke = (int)job_cost[jb];
    if (col_major) {
      for (int nt = 0; nt < nn; nt += width(nt))
        for (int mt = 0; mt < nm; ++mt) dst.push_back(make_tile(jb, mt, nt, 0, width(nt) - 1, 0, ke));
    } else {
      for (int mt = 0; mt < nm; ++mt)
        for (int nt = 0; nt < nn; nt += width(nt)) dst.push_back(make_tile(jb, mt, nt, 0, width(nt) - 1, 0, ke));
    }
  };
  // estimated time of a tile in thirds of a 128-column K step: a 256-column K step takes
  // about 1.3 times as long (measured on GB300; the 128-column step waits on its operand
  // copies, the 256-column one is close to the MMA rate)
  auto tile_cost = [](const TcTile& tl) { return (int64_t)(tl.ke - tl.kb) * (tl.wide ? 4 : 3); };
  auto by_tile_cost = [&](std::vector<TcTile>& v) {
    std::stable_sort(v.begin(), v.end(), [&](const TcTile& a, const TcTile& b) {
      return tile_cost(a) > tile_cost(b);
    });
  };
  // K split of the FP64-output tiles estimated above num / den of the mean time per SM
  int64_t slots_used = 0;
  auto split_k = [&](const std::vector<TcTile>& src, int num, int den) {
    int64_t total = 0;
    for (const TcTile& tl : src) total += tile_cost(tl);
    const int64_t cap = std::max<int64_t>(1, total * num / den / std::max(1, t->sms));
    std::vector<TcTile> res;
    int64_t slot = 0;
    for (const TcTile& tl : src) {
      const int nk = tl.ke - tl.kb;
      const int64_t c = tile_cost(tl);
      const int np = (int)std::min<int64_t>({(c + cap - 1) / cap, (int64_t)nk, 8});
      if (!jobs[tl.job].out_fp64 || np < 2) {
        res.push_back(tl);
        continue;
      }
      for (int q = 0; q < np; ++q) {
        TcTile pt = tl;
        pt.kb = tl.kb + (int)((int64_t)nk * q / np);
        pt.ke = tl.kb + (int)((int64_t)nk * (q + 1) / np);
        pt.part = q;
        pt.nparts = np;
        pt.red = (int)slot;
        res.push_back(pt);
      }
      slot += np;
    }
    slots_used = std::max(slots_used, slot);
    return res;
  };
  // jobs (already in descending cost) grouped by key; groups in descending total cost
  auto grouped = [&](const std::vector<std::pair<int64_t, int>>& order,
                     const std::function<int64_t(int)>& key, bool col_major) {
    std::map<int64_t, std::pair<int64_t, std::vector<int>>> groups;
    for (const auto& pr : order) {
      auto& g = groups[key(pr.second)];
      g.first += pr.first;
      g.second.push_back(pr.second);
    }
    std::vector<std::pair<int64_t, int64_t>> gorder;
    for (const auto& g : groups) gorder.push_back({g.second.first, g.first});
    std::stable_sort(gorder.begin(), gorder.end(), [](const auto& a, const auto& b) {
      return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    std::vector<TcTile> res;
    for (const auto& g : gorder)
      for (int jb : groups[g.second].second) add_tiles(res, jb, col_major);
    return res;
  };
  std::vector<TcTile> sched1[kSchedules], sched2[kSchedules];
  // a stage-1 job has one segment (its record), or none when its K dimension is empty
  auto x_key = [&](int jb) -> int64_t {
    const TcJob& j = jobs[jb];
    return j.seg_begin == j.seg_end ? -1 : segs[j.seg_begin].q_off * 4 + segs[j.seg_begin].q_buf;
  };
  auto op_key = [&](int jb) -> int64_t {
    const TcJob& j = jobs[jb];
    return j.seg_begin == j.seg_end ? -1 : segs[j.seg_begin].p_off;
  };
  std::vector<int> job_pair(jobs.size(), -1);
  for (int q = 0; q < npairs; ++q) job_pair[stage2_job[q]] = q;
  for (int c = 0; c < kSchedules; ++c) {
    const int o = c % kOrders, w = (c / kOrders) % kWidths, sp = c / (kOrders * kWidths);
    t->valid[0][c] = sp == 0 && (!tf32 || w == 0);
    t->valid[1][c] = !tf32 || w == 0;
    if (!t->valid[1][c]) continue;
    wpol = w;
    if (sp == 0) {
      cur_stage = 0;
      if (o == 0) for (const auto& pr : order1) add_tiles(sched1[c], pr.second, false);
      if (o == 1) sched1[c] = grouped(order1, x_key, true);
      if (o == 2) sched1[c] = grouped(order1, op_key, false);
      if (o == 0) by_tile_cost(sched1[c]);
    }
    cur_stage = 1;
    if (o == 0) for (const auto& pr : order2) add_tiles(sched2[c], pr.second, false);
    if (o == 1) sched2[c] = grouped(order2, [&](int jb) { return (int64_t)p->pair_k[job_pair[jb]]; }, false);
    if (o == 2) sched2[c] = grouped(order2, [&](int jb) { return (int64_t)p->pair_i[job_pair[jb]]; }, false);
    if (sp > 0) sched2[c] = split_k(sched2[c], 2, sp == 1 ? 3 : 5);
    if (o == 0) by_tile_cost(sched2[c]);
  }
  tiles1 = sched1[0];
  tiles2 = sched2[0];
  // stage-1 N tiles read Q image row tiles; stage-2 image K tiles must cover the segment
  // (image row tiles = ceil(rows / 128) >= tiles; image K tiles = nkt): checked here
  for (const TcSeg& s : segs) {
    if (s.nkt > s.p_nkt || s.nkt > s.q_nkt) {
      set_error("internal: segment K tiles exceed its operand images");
      return fail(DMRG_ERR_SHAPE);
    }
  }

  // ---- device buffers
  t->buf_bytes[TB_OPS] = (size_t)ops_alloc.bytes;
  t->buf_bytes[TB_XA] = (size_t)xa_alloc.bytes;
  t->buf_bytes[TB_INTER] = (size_t)inter_alloc.bytes;
  for (int b = 0; b < 4; ++b) {
    if (t->buf_bytes[b] == 0) continue;
    if (cudaMalloc((void**)&t->buf[b], t->buf_bytes[b]) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of %zu bytes for tensor-core operand images failed", t->buf_bytes[b]);
      return fail(DMRG_ERR_OOM);
    }
    p->device_bytes += t->buf_bytes[b];
  }
  t->buf[TB_XB] = t->buf[TB_XA];  // alias: B-form offsets follow the A-form tiles
  // tile-list counters and the split-K scratch
  t->nslots = slots_used;
  if (cudaMalloc((void**)&t->d_ctr, 4 * sizeof(int)) != cudaSuccess ||
      (t->nslots > 0 &&
       cudaMalloc((void**)&t->d_partial, sizeof(float) * kSlotFloats * (size_t)t->nslots) != cudaSuccess)) {
    cudaGetLastError();
    set_error("cudaMalloc of the tile counters or the split-K scratch failed");
    return fail(DMRG_ERR_OOM);
  }
  p->device_bytes += 4 * sizeof(int) + sizeof(float) * kSlotFloats * t->nslots;
  DMRG_CUDA_TRY(cudaMemsetAsync(t->d_ctr, 0, 4 * sizeof(int), st));
  {
    char why[160];
    for (int c = 0; c < kSchedules; ++c) {
      if (!tc_tiles_in_range(t, p->n, jobs, segs, sched1[c], 0, 0, why, sizeof(why)) ||
          !tc_tiles_in_range(t, p->n, jobs, segs, sched2[c], 0, 0, why, sizeof(why))) {
        set_error("internal: %s", why);
        return fail(DMRG_ERR_SHAPE);
      }
    }
  }
  if (t->buf[TB_INTER]) {
    // intermediate tiles beyond the written rows stay zero
    DMRG_CUDA_TRY(cudaMemsetAsync(t->buf[TB_INTER], 0, t->buf_bytes[TB_INTER], st));
  }
  std::vector<PackChunk> op_chunks, x_chunks;
  for (size_t jb = 0; jb < op_jobs.size(); ++jb)
    for (int rt = 0; rt < ceil_div(op_jobs[jb].R, kRows); ++rt)
      for (int kt = 0; kt < op_jobs[jb].nkt; ++kt) op_chunks.push_back(PackChunk{(int32_t)jb, rt, kt, 0});
  for (size_t jb = 0; jb < x_jobs.size(); ++jb)
    for (int rt = 0; rt < ceil_div(x_jobs[jb].R, kRows); ++rt)
      for (int kt = 0; kt < x_jobs[jb].nkt; ++kt) x_chunks.push_back(PackChunk{(int32_t)jb, rt, kt, 0});
  PackJob* d_opj = nullptr;
  PackChunk* d_opc = nullptr;
  dmrg_status s;
  if ((s = upload_vec(&d_opj, op_jobs, st)) != DMRG_OK) return fail(s);
  if ((s = upload_vec(&d_opc, op_chunks, st)) != DMRG_OK) return fail(s);
  if (tf32) s = launch_pack<1, true>(op_chunks, d_opc, d_opj, p->arena, nullptr, t->buf[TB_OPS], st);
  else if (planes == 2) s = launch_pack<2, false>(op_chunks, d_opc, d_opj, p->arena, nullptr, t->buf[TB_OPS], st);
  else s = launch_pack<3, false>(op_chunks, d_opc, d_opj, p->arena, nullptr, t->buf[TB_OPS], st);
  cudaStreamSynchronize(st);
  cudaFree(d_opj);
  cudaFree(d_opc);
  if (s != DMRG_OK) return fail(s);
  if ((s = upload_vec(&t->d_xpack_jobs, x_jobs, st)) != DMRG_OK) return fail(s);
  if ((s = upload_vec(&t->d_xpack_chunks, x_chunks, st)) != DMRG_OK) return fail(s);
  t->n_xpack_chunks = (int64_t)x_chunks.size();
  if ((s = upload_vec(&t->d_jobs, jobs, st)) != DMRG_OK) return fail(s);
  if ((s = upload_vec(&t->d_segs, segs, st)) != DMRG_OK) return fail(s);
  for (int c = 0; c < kSchedules; ++c) {
    if ((s = upload_vec(&t->d_tiles[0][c], sched1[c], st)) != DMRG_OK) return fail(s);
    if ((s = upload_vec(&t->d_tiles[1][c], sched2[c], st)) != DMRG_OK) return fail(s);
    std::vector<TcTile> groups;
    for (const TcTile& tl : sched2[c])
      if (tl.nparts > 1 && tl.part == 0) groups.push_back(tl);
    if ((s = upload_vec(&t->d_groups[c], groups, st)) != DMRG_OK) return fail(s);
    t->ngroups[c] = (int64_t)groups.size();
    t->ntiles[0][c] = (int64_t)sched1[c].size();
    t->ntiles[1][c] = (int64_t)sched2[c].size();
  }
  t->ntiles1 = (int64_t)tiles1.size();
  t->ntiles2 = (int64_t)tiles2.size();
  t->h_jobs = jobs;
  t->h_segs = segs;
  t->h_order[0] = order1;
  t->h_order[1] = order2;
  t->h_xjobs = x_jobs;
  t->h_xchunks = x_chunks;
  if (cudaHostAlloc((void**)&t->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&t->d_err, t->h_err, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("mapped host allocation for the kernel error word failed");
    return fail(DMRG_ERR_OOM);
  }
  *t->h_err = 0;
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  *out = t;
  return DMRG_OK;
}

template <int PLANES, int STAGES, bool TF32>
dmrg_status configure_tc() {
  constexpr bool WIDE = !TF32;
  constexpr size_t smem = tc::smem_bytes<PLANES, STAGES, TF32, WIDE>();
  static bool configured[64] = {false};
  int dev = 0;
  DMRG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    DMRG_CUDA_TRY(cudaFuncSetAttribute(tc::tc_gemm_kernel<PLANES, STAGES, TF32, !TF32>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured[dev] = true;
  }
  return DMRG_OK;
}

// The vector of a projection: FP64 x, y, or (x32, y32 set) an FP32 one.
struct VecIO {
  const double* x;
  double* y;
  const float* x32;
  float* y32;
};

// part 0: pack X into its operand images; part 1, 2: the GEMM stages with schedule c
template <int PLANES, int STAGES, bool TF32>
dmrg_status run_tc_part(dmrg_plan* p, TcPlan* t, const VecIO& io, int part, int c,
                        cudaStream_t st) {
  const double* x = io.x;
  double* y = io.y;
  constexpr bool WIDE = !TF32;
  constexpr size_t smem = tc::smem_bytes<PLANES, STAGES, TF32, WIDE>();
  if (part == 0) {
    if (t->n_xpack_chunks > 0) {  // X -> A-form and B-form images
      DMRG_CUDA_TRY(launch_pdl(tc::pack_kernel<PLANES, TF32>, dim3((unsigned)t->n_xpack_chunks), dim3(256),
                               0, st, (const PackChunk*)t->d_xpack_chunks, (const PackJob*)t->d_xpack_jobs,
                               (const double*)p->arena, x, t->buf[TB_XA], (const TcPtrs*)nullptr, io.x32));
      DMRG_LAUNCH_CHECK();
    }
    return DMRG_OK;
  }
  const int64_t nt = t->ntiles[part - 1][c];
  if (nt == 0) return DMRG_OK;
  const int grid = (int)std::min<int64_t>(nt, t->sms);
  DMRG_CUDA_TRY(launch_pdl(
      tc::tc_gemm_kernel<PLANES, STAGES, TF32, WIDE>, dim3(grid), dim3(tc::kThreads), smem, st,
      (const TcTile*)t->d_tiles[part - 1][c], (int)nt, (const TcJob*)t->d_jobs, (const TcSeg*)t->d_segs,
      (const uint8_t*)t->buf[TB_OPS], (const uint8_t*)t->buf[TB_XA], (const uint8_t*)t->buf[TB_XB],
      (const uint8_t*)(part == 1 ? nullptr : t->buf[TB_INTER]), part == 1 ? t->buf[TB_INTER] : nullptr, y, x,
      t->d_err, (const TcPtrs*)nullptr, part, t->d_ctr + 2 * (part - 1), t->d_partial, io.y32, io.x32));
  DMRG_LAUNCH_CHECK();
  if (part == 2 && t->ngroups[c] > 0) {
    DMRG_CUDA_TRY(launch_pdl(tc::split_reduce_kernel, dim3((unsigned)(t->ngroups[c] * 32)), dim3(256), 0, st,
                             (const TcTile*)t->d_groups[c], (const TcJob*)t->d_jobs,
                             (const float*)t->d_partial, y, x, io.y32, io.x32));
    DMRG_LAUNCH_CHECK();
  }
  return DMRG_OK;
}

template <int PLANES, int STAGES, bool TF32>
dmrg_status run_tc_direct(dmrg_plan* p, TcPlan* t, const VecIO& io, cudaStream_t st) {
  DMRG_TRY((run_tc_part<PLANES, STAGES, TF32>(p, t, io, 0, 0, st)));
  DMRG_TRY((run_tc_part<PLANES, STAGES, TF32>(p, t, io, 1, t->sched[0], st)));
  DMRG_TRY((run_tc_part<PLANES, STAGES, TF32>(p, t, io, 2, t->sched[1], st)));
  return launch_seg_axpy(p, io.x, io.y, io.x32, io.y32, st);
}

template <int PLANES, int STAGES, bool TF32>
dmrg_status run_tc(dmrg_plan* p, TcPlan* t, const VecIO& io, cudaStream_t st) {
  DMRG_TRY((configure_tc<PLANES, STAGES, TF32>()));
  if (*t->h_err != 0) {
    set_error("tensor-core projection kernel reported error %d (a bounded wait timed out)",
              *t->h_err);
    return DMRG_ERR_CUDA;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DMRG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  // launched directly when graphs are off, or inside the caller's own stream capture
  if (!p->opt.graphs || cs != cudaStreamCaptureStatusNone)
    return run_tc_direct<PLANES, STAGES, TF32>(p, t, io, st);
  const TcPlan::GraphKey key{io.x, io.y, io.x32, io.y32};
  auto it = t->graphs.find(key);
  if (it == t->graphs.end()) {
    if (!t->cap_st) DMRG_CUDA_TRY(cudaStreamCreateWithFlags(&t->cap_st, cudaStreamNonBlocking));
    const int64_t l0 = dmrg_kernel_launches();
    DMRG_CUDA_TRY(cudaStreamBeginCapture(t->cap_st, cudaStreamCaptureModeThreadLocal));
    dmrg_status s = run_tc_direct<PLANES, STAGES, TF32>(p, t, io, t->cap_st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(t->cap_st, &g);
    const int nk = (int)(dmrg_kernel_launches() - l0);
    note_launches(-nk);  // captured, not launched: replays count them
    if (s != DMRG_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) {
      set_error("capture of the projection graph: %s", cudaGetErrorString(e));
      return DMRG_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      set_error("instantiation of the projection graph: %s", cudaGetErrorString(ei));
      return DMRG_ERR_CUDA;
    }
    if (t->graphs.size() >= 96) drop_graphs(t);  // bounded: a solve uses about 25 vector pairs
    it = t->graphs.emplace(key, std::make_pair(ex, nk)).first;
  }
  DMRG_CUDA_TRY(cudaGraphLaunch(it->second.first, st));
  note_launches(it->second.second);
  return DMRG_OK;
}

// The autotuner: times every schedule of each stage (median of 3 after one untimed run,
// with L2 flushed by a 256 MB write before each timed run, as inside a Davidson
// iteration whose vector passes stream far more than L2) and keeps the fastest.  Stage 2
// reads the intermediates of stage 1, which every schedule writes identically.
template <int PLANES, int STAGES, bool TF32>
dmrg_status tune_tc(dmrg_plan* p, TcPlan* t, const double* x, double* y, cudaStream_t st) {
  DMRG_TRY((configure_tc<PLANES, STAGES, TF32>()));
  constexpr size_t kFlush = size_t(256) << 20;
  void* flush = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (flush) cudaFreeAsync(flush, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMallocAsync(&flush, kFlush, st) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    set_error("autotune: allocation of the L2 flush buffer or events failed");
    return DMRG_ERR_OOM;
  }
  const VecIO io{x, y, nullptr, nullptr};
  dmrg_status s = run_tc_part<PLANES, STAGES, TF32>(p, t, io, 0, 0, st);
  for (int part = 1; part <= 2 && s == DMRG_OK; ++part) {
    float best = 0.0f;
    int arg = 0;
    bool first = true;
    for (int c = 0; c < kSchedules && s == DMRG_OK; ++c) {
      if (!t->valid[part - 1][c]) continue;
      float ms[3] = {0.0f, 0.0f, 0.0f};
      s = run_tc_part<PLANES, STAGES, TF32>(p, t, io, part, c, st);
      for (int r = 0; r < 3 && s == DMRG_OK; ++r) {
        if (cudaMemsetAsync(flush, r + 1, kFlush, st) != cudaSuccess ||
            cudaEventRecord(e0, st) != cudaSuccess) {
          set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
          s = DMRG_ERR_CUDA;
          break;
        }
        s = run_tc_part<PLANES, STAGES, TF32>(p, t, io, part, c, st);
        if (s != DMRG_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms[r], e0, e1) != cudaSuccess) {
          set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
          s = DMRG_ERR_CUDA;
        }
      }
      if (s != DMRG_OK) break;
      std::sort(ms, ms + 3);
      t->tune_us[part - 1][c] = ms[1] * 1000.0f;
      if (first || ms[1] < best) {
        best = ms[1];
        arg = c;
        first = false;
      }
    }
    t->sched[part - 1] = arg;
    drop_graphs(t);
  }
  cleanup();
  if (s == DMRG_OK && *t->h_err != 0) {
    set_error("tensor-core projection kernel reported error %d (a bounded wait timed out)",
              *t->h_err);
    s = DMRG_ERR_CUDA;
  }
  if (s == DMRG_OK) t->tuned = true;
  return s;
}

}  // namespace

// ======================================================================== grouped launch
// One pack launch and one launch per GEMM stage for the low-precision projections of many
// independent plans (batched Davidson solves): the jobs, segments, tiles and pack chunks of
// all plans are concatenated once; every tile and chunk carries its problem index, and a
// small per-call table gives each problem's vector pointers and whether it takes part.
// Tiles of all problems are taken in one descending-cost order (longest first).
struct TcBatch {
  dmrg_precision prec = DMRG_PREC_BF16X3;
  std::vector<dmrg_plan*> plans;
  TcJob* d_jobs = nullptr;
  TcSeg* d_segs = nullptr;
  TcTile* d_tiles[2] = {nullptr, nullptr};
  int64_t ntiles[2] = {0, 0};
  PackJob* d_pjobs = nullptr;
  PackChunk* d_pchunks = nullptr;
  int64_t nchunks = 0;
  TcPtrs* d_ptrs = nullptr;
  int* d_ctr = nullptr;                     // tile-list counters, 2 per stage
  TcPtrs* h_ptrs[2] = {nullptr, nullptr};   // pinned ring: slot r reused after ev[r]
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int slot = 0;
  int* d_err = nullptr;
  int* h_err = nullptr;
  int sms = 0;
};

void tc_batch_destroy(TcBatch* b) {
  if (!b) return;
  cudaFree(b->d_jobs);
  cudaFree(b->d_segs);
  cudaFree(b->d_tiles[0]);
  cudaFree(b->d_tiles[1]);
  cudaFree(b->d_pjobs);
  cudaFree(b->d_pchunks);
  cudaFree(b->d_ptrs);
  cudaFree(b->d_ctr);
  for (int r = 0; r < 2; ++r) {
    if (b->ev[r]) {
      cudaEventSynchronize(b->ev[r]);
      cudaEventDestroy(b->ev[r]);
    }
    if (b->h_ptrs[r]) cudaFreeHost(b->h_ptrs[r]);
  }
  if (b->h_err) cudaFreeHost(b->h_err);
  delete b;
}

dmrg_status tc_batch_create(dmrg_plan* const* plans, int nb, dmrg_precision prec,
                            cudaStream_t st, TcBatch** out) {
  *out = nullptr;
  if (!tc_lowprec(prec)) {
    set_error("internal: grouped launch needs a TF32, BF16X3 or BF16X2 plan");
    return DMRG_ERR_INVALID_ARG;
  }
  const int slot = tc_slot(prec);
  TcBatch* b = new TcBatch();
  b->prec = prec;
  auto fail = [&](dmrg_status e) { tc_batch_destroy(b); return e; };
  std::vector<TcJob> jobs;
  std::vector<TcSeg> segs;
  std::vector<PackJob> pjobs;
  std::vector<PackChunk> pchunks;
  struct Item { int64_t cost; int prob, job; };
  std::vector<Item> items[2];
  for (int i = 0; i < nb; ++i) {
    dmrg_plan* p = plans[i];
    if (!p->tc[slot]) {
      TcPlan* t = nullptr;
      dmrg_status e = build_tc(p, prec, st, &t);
      if (e != DMRG_OK) return fail(e);
      p->tc[slot] = t;
    }
    const TcPlan* t = p->tc[slot];
    b->plans.push_back(p);
    b->sms = t->sms;
    const int job0 = (int)jobs.size(), seg0 = (int)segs.size(), pjob0 = (int)pjobs.size();
    for (TcJob j : t->h_jobs) {
      j.seg_begin += seg0;
      j.seg_end += seg0;
      jobs.push_back(j);
    }
    segs.insert(segs.end(), t->h_segs.begin(), t->h_segs.end());
    for (int g = 0; g < 2; ++g)
      for (const auto& pr : t->h_order[g]) items[g].push_back(Item{pr.first, i, job0 + pr.second});
    pjobs.insert(pjobs.end(), t->h_xjobs.begin(), t->h_xjobs.end());
    for (PackChunk c : t->h_xchunks) {
      c.job += pjob0;
      c.pad_ = i;
      pchunks.push_back(c);
    }
  }
  std::vector<TcTile> tiles[2];
  for (int g = 0; g < 2; ++g) {
    std::stable_sort(items[g].begin(), items[g].end(), [](const Item& a, const Item& c) {
      return a.cost > c.cost;
    });
    // width policy 1 of the single-plan schedules over the whole batch: 256-column tiles
    // for jobs whose wide tile stays below half of the mean work per SM
    int64_t mean = 0;
    for (const Item& it : items[g]) {
      const TcJob& j = jobs[it.job];
      mean += it.cost * ceil_div(j.M, kRows) * ceil_div(j.N, kRows);
    }
    mean /= std::max(1, b->sms);
    for (const Item& it : items[g]) {
      const TcJob& j = jobs[it.job];
      const int nn = ceil_div(j.N, kRows);
      const bool wide_tiles = prec != DMRG_PREC_TF32 && 4 * it.cost <= mean;
      for (int mt = 0; mt < ceil_div(j.M, kRows); ++mt)
        for (int nt = 0; nt < nn;) {
          const int w = (wide_tiles && nt + 1 < nn) ? 2 : 1;
          tiles[g].push_back(make_tile(it.job, mt, nt, it.prob, w - 1, 0, (int)it.cost));
          nt += w;
        }
    }
    b->ntiles[g] = (int64_t)tiles[g].size();
  }
  {
    // every tile of problem i against problem i's own buffers
    std::vector<int> job_base(nb + 1, 0), seg_base(nb + 1, 0);
    for (int i = 0; i < nb; ++i) {
      job_base[i + 1] = job_base[i] + (int)plans[i]->tc[slot]->h_jobs.size();
      seg_base[i + 1] = seg_base[i] + (int)plans[i]->tc[slot]->h_segs.size();
    }
    char why[160];
    for (int g = 0; g < 2; ++g) {
      for (const TcTile& tl : tiles[g]) {
        const int i = tl.pad_;
        if (i < 0 || i >= nb || tl.job < job_base[i] || tl.job >= job_base[i + 1]) {
          set_error("internal: grouped tile with a bad problem or job index");
          return fail(DMRG_ERR_SHAPE);
        }
        const TcPlan* t = plans[i]->tc[slot];
        TcJob j = jobs[tl.job];
        j.seg_begin -= seg_base[i];
        j.seg_end -= seg_base[i];
        std::vector<TcJob> one(1, j);
        TcTile one_tile = tl;
        one_tile.job = 0;
        one_tile.pad_ = 0;
        std::vector<TcTile> onet(1, one_tile);
        if (j.seg_begin < 0 || j.seg_end > (int)t->h_segs.size() ||
            !tc_tiles_in_range(t, plans[i]->n, one, t->h_segs, onet, 0, 0, why, sizeof(why))) {
          set_error("internal: grouped launch, problem %d: %s", i, why);
          return fail(DMRG_ERR_SHAPE);
        }
      }
    }
    for (const PackChunk& c : pchunks) {
      if (c.pad_ < 0 || c.pad_ >= nb || c.job < 0 || c.job >= (int)pjobs.size()) {
        set_error("internal: grouped pack chunk with a bad index");
        return fail(DMRG_ERR_SHAPE);
      }
    }
  }
  dmrg_status e;
  if ((e = upload_vec(&b->d_jobs, jobs, st)) != DMRG_OK) return fail(e);
  if ((e = upload_vec(&b->d_segs, segs, st)) != DMRG_OK) return fail(e);
  if ((e = upload_vec(&b->d_tiles[0], tiles[0], st)) != DMRG_OK) return fail(e);
  if ((e = upload_vec(&b->d_tiles[1], tiles[1], st)) != DMRG_OK) return fail(e);
  if ((e = upload_vec(&b->d_pjobs, pjobs, st)) != DMRG_OK) return fail(e);
  if ((e = upload_vec(&b->d_pchunks, pchunks, st)) != DMRG_OK) return fail(e);
  b->nchunks = (int64_t)pchunks.size();
  if (cudaMalloc((void**)&b->d_ptrs, sizeof(TcPtrs) * std::max(nb, 1)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_ctr, 4 * sizeof(int)) != cudaSuccess ||
      cudaHostAlloc((void**)&b->h_ptrs[0], sizeof(TcPtrs) * std::max(nb, 1), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc((void**)&b->h_ptrs[1], sizeof(TcPtrs) * std::max(nb, 1), cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc((void**)&b->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&b->d_err, b->h_err, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("grouped launch: allocation failed");
    return fail(DMRG_ERR_OOM);
  }
  *b->h_err = 0;
  DMRG_CUDA_TRY(cudaMemsetAsync(b->d_ctr, 0, 4 * sizeof(int), st));
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  *out = b;
  return DMRG_OK;
}

dmrg_status tc_batch_error(const TcBatch* b) {
  if (b && b->h_err && *b->h_err != 0) {
    set_error("grouped tensor-core projection reported error %d (a bounded wait timed out)", *b->h_err);
    return DMRG_ERR_CUDA;
  }
  return DMRG_OK;
}

namespace {
template <int PLANES, int STAGES, bool TF32>
dmrg_status run_batch(TcBatch* b, const TcPtrs* h, cudaStream_t st) {
  constexpr bool WIDE = !TF32;
  constexpr size_t smem = tc::smem_bytes<PLANES, STAGES, TF32, WIDE>();
  DMRG_TRY((configure_tc<PLANES, STAGES, TF32>()));
  if (b->nchunks > 0) {
    tc::pack_kernel<PLANES, TF32><<<(unsigned)b->nchunks, 256, 0, st>>>(
        b->d_pchunks, b->d_pjobs, nullptr, nullptr, nullptr, b->d_ptrs, nullptr);
    DMRG_LAUNCH_CHECK();
  }
  for (int part = 1; part <= 2; ++part) {
    const int64_t nt = b->ntiles[part - 1];
    if (nt == 0) continue;
    const int grid = (int)std::min<int64_t>(nt, b->sms);
    tc::tc_gemm_kernel<PLANES, STAGES, TF32, WIDE><<<grid, tc::kThreads, smem, st>>>(
        b->d_tiles[part - 1], (int)nt, b->d_jobs, b->d_segs, nullptr, nullptr, nullptr, nullptr,
        nullptr, nullptr, nullptr, b->d_err, b->d_ptrs, part, b->d_ctr + 2 * (part - 1), nullptr,
        nullptr, nullptr);
    DMRG_LAUNCH_CHECK();
  }
  for (size_t i = 0; i < b->plans.size(); ++i)  // cross-segment identity terms, per problem
    if (h[i].active)
      DMRG_TRY(launch_seg_axpy(b->plans[i], h[i].x, h[i].y, h[i].x32, h[i].y32, st));
  return DMRG_OK;
}
}  // namespace

dmrg_status tc_batch_project(TcBatch* b, const double* const* x, double* const* y,
                             const float* const* x32, float* const* y32, const char* active,
                             cudaStream_t st) {
  DMRG_TRY(tc_batch_error(b));
  const int slot = tc_slot(b->prec);
  const int r = b->slot;
  b->slot ^= 1;
  // the pinned slot is rewritten only after its previous copy has completed
  DMRG_CUDA_TRY(cudaEventSynchronize(b->ev[r]));
  TcPtrs* h = b->h_ptrs[r];
  bool any = false;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const dmrg_plan* p = b->plans[i];
    const TcPlan* t = p->tc[slot];
    const bool f32 = x32 && x32[i];
    h[i] = TcPtrs{p->arena, f32 ? nullptr : x[i], f32 ? nullptr : y[i], f32 ? x32[i] : nullptr,
                  f32 ? y32[i] : nullptr, t->buf[TB_OPS], t->buf[TB_XA], t->buf[TB_INTER],
                  active[i] ? 1 : 0, 0};
    if (active[i] && (!(f32 ? (const void*)x32[i] : (const void*)x[i]) ||
                      !(f32 ? (void*)y32[i] : (void*)y[i]) || !t->buf[TB_OPS] || !t->buf[TB_XA] ||
                      (t->ntiles1 > 0 && !t->buf[TB_INTER]))) {
      set_error("internal: grouped projection of problem %zu without its buffers", i);
      return DMRG_ERR_INVALID_ARG;
    }
    any = any || active[i];
  }
  if (!any) return DMRG_OK;
  DMRG_CUDA_TRY(cudaMemcpyAsync(b->d_ptrs, h, sizeof(TcPtrs) * b->plans.size(),
                                cudaMemcpyHostToDevice, st));
  DMRG_CUDA_TRY(cudaEventRecord(b->ev[r], st));
  if (b->prec == DMRG_PREC_TF32) return run_batch<1, 6, true>(b, h, st);
  if (b->prec == DMRG_PREC_BF16X2) return run_batch<2, 4, false>(b, h, st);
  return run_batch<3, 3, false>(b, h, st);
}

bool tc_available(dmrg_precision prec) { return tc_lowprec(prec) || prec == DMRG_PREC_FP64_TC; }

void destroy_tc(dmrg_plan* p) {
  if (!p) return;
  for (auto& t : p->tc) {
    free_tc(t);
    t = nullptr;
  }
}

dmrg_status tc_error_status(dmrg_plan* p) {
  DMRG_TRY(oz_error_status(p));
  for (TcPlan* t : p->tc) {
    if (t && t->h_err && *t->h_err != 0) {
      set_error("tensor-core projection kernel reported error %d (a bounded wait timed out)",
                *t->h_err);
      return DMRG_ERR_CUDA;
    }
  }
  return DMRG_OK;
}

namespace {
dmrg_status project_tc_io(dmrg_plan* p, dmrg_precision prec, const VecIO& io, cudaStream_t st) {
  const int slot = tc_slot(prec);
  if (!p->tc[slot]) {
    TcPlan* t = nullptr;
    DMRG_TRY(build_tc(p, prec, st, &t));
    p->tc[slot] = t;
  }
  TcPlan* t = p->tc[slot];
  if (p->opt.autotune && !t->tuned) DMRG_TRY(tune_project_tc(p, prec, st));
  if (prec == DMRG_PREC_TF32) return run_tc<1, 6, true>(p, t, io, st);
  if (prec == DMRG_PREC_BF16X2) return run_tc<2, 4, false>(p, t, io, st);
  return run_tc<3, 3, false>(p, t, io, st);
}
}  // namespace

dmrg_status launch_project_tc(dmrg_plan* p, dmrg_precision prec, const double* x, double* y,
                              cudaStream_t st) {
  return project_tc_io(p, prec, VecIO{x, y, nullptr, nullptr}, st);
}

dmrg_status launch_project_tc32(dmrg_plan* p, dmrg_precision prec, const float* x, float* y,
                                cudaStream_t st) {
  return project_tc_io(p, prec, VecIO{nullptr, nullptr, x, y}, st);
}

dmrg_status tune_project_tc(dmrg_plan* p, dmrg_precision prec, cudaStream_t st) {
  const int slot = tc_slot(prec);
  if (!p->tc[slot]) {
    TcPlan* t = nullptr;
    DMRG_TRY(build_tc(p, prec, st, &t));
    p->tc[slot] = t;
  }
  TcPlan* t = p->tc[slot];
  // input: diag(H_SB) (any vector of the right size times the same); output: scratch
  double* y = nullptr;
  if (cudaMallocAsync((void**)&y, sizeof(double) * (size_t)std::max<int64_t>(p->n, 1), st) != cudaSuccess) {
    cudaGetLastError();
    set_error("autotune: scratch allocation failed");
    return DMRG_ERR_OOM;
  }
  dmrg_status s = prec == DMRG_PREC_TF32     ? tune_tc<1, 6, true>(p, t, p->D, y, st)
                  : prec == DMRG_PREC_BF16X2 ? tune_tc<2, 4, false>(p, t, p->D, y, st)
                                             : tune_tc<3, 3, false>(p, t, p->D, y, st);
  cudaFreeAsync(y, st);
  return s;
}

dmrg_status set_schedule_tc(dmrg_plan* p, dmrg_precision prec, int stage1, int stage2,
                            cudaStream_t st) {
  const int slot = tc_slot(prec);
  if (!p->tc[slot]) {
    TcPlan* t = nullptr;
    DMRG_TRY(build_tc(p, prec, st, &t));
    p->tc[slot] = t;
  }
  TcPlan* t = p->tc[slot];
  const int want[2] = {stage1, stage2};
  for (int g = 0; g < 2; ++g) {
    if (want[g] < 0 || want[g] >= kSchedules || !t->valid[g][want[g]]) {
      set_error("tile schedule %d is not a candidate of GEMM stage %d in this precision",
                want[g], g + 1);
      return DMRG_ERR_INVALID_ARG;
    }
  }
  drop_graphs(t);
  t->sched[0] = stage1;
  t->sched[1] = stage2;
  t->tuned = true;  // fixed: the first projection does not autotune
  return DMRG_OK;
}

void tc_schedule_stats(const dmrg_plan* p, int32_t sched[2], float us[2][DMRG_TILE_SCHEDULES]) {
  static_assert(DMRG_TILE_SCHEDULES == kSchedules, "schedule count of the public stats");
  // the plan's own low-precision arithmetic if built, else the first one built
  const TcPlan* t = tc_lowprec(p->opt.prec) ? p->tc[tc_slot(p->opt.prec)] : nullptr;
  for (int i = 0; i < 3 && !t; ++i) t = p->tc[i];
  for (int g = 0; g < 2; ++g) {
    sched[g] = t ? t->sched[g] : -1;
    for (int c = 0; c < kSchedules; ++c) us[g][c] = t ? t->tune_us[g][c] : 0.0f;
  }
}

}  // namespace dmrg
