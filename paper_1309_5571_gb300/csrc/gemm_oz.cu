// FP64-accurate projection on the tensor cores: exact integer-digit products in BF16.
//
// Each FP64 operand row is split, per chunk of 256 K elements, into a power-of-two scale
// and S = 7 balanced base-128 digits,
//     x = 2^E * sum_{s=1..S} D_s 2^(-7 s),   D_s integers, |D_s| <= 64,
// with E chosen so that |x| 2^-E < 1/2 for the whole row chunk (the error-free splitting
// of the Ozaki scheme, with digits that BF16 represents exactly).  A product of two rows
// then is
//     sum_k P Q = 2^(E_P + E_Q) sum_{s,t} 2^(-7 (s + t)) sum_k D_s E_t .
// Digit products are exact (|D_s E_t| <= 2^12) and their sums over one chunk stay below
// 2^24 even for the 7 digit pairs that share one scale (7 * 256 * 2^12 < 2^24), so the
// tensor cores add them EXACTLY in FP32.  The kernel therefore keeps one TMEM
// accumulator per scale group g = s + t - 2 (pairs with s + t <= S + 1 are kept: the
// dropped ones lie below 2^-56 of the row scale), and after each chunk the epilogue
// scales the S exact group sums by powers of two and adds them into a double-float
// (FP32 hi + FP32 lo, ~48 bits) accumulator per output element; the result is converted
// to FP64 once.  The rest mirrors the low-precision path: two stages (intermediates in
// FP64, re-split for stage 2), operand tiles pre-swizzled into the 64-byte K-major
// layout and moved by single bulk copies.
//
// Tile: 128 output rows (M of the MMA) x 64 columns (N); K tiles of 32 elements in the
// 64-byte swizzled K-major layout, two shared-memory stages of one K tile each (7 digit
// planes of A: 56 KB; of B: 28 KB), so that the copies of one K tile overlap the 56 MMAs of
// the previous one; 7 accumulators x 64 TMEM columns.  Warp roles: warp 0 copies, warp 1
// issues tcgen05.mma, warps 2-9 drain and accumulate (warp w reads TMEM lanes
// 32 (w % 4) .. + 31, columns 32 ((w - 2) / 4) .. + 31).  All waits are bounded (2 s).
#include <cuda_bf16.h>

#include <algorithm>
#include <map>
#include <tuple>

#include "internal.h"

namespace dmrg {

struct OzSeg {
  int64_t p_off, q_off;     // byte offsets of the (row tile 0, K tile 0) image tiles
  int64_t p_eoff, q_eoff;   // element offsets of the exponent tables
  int32_t p_buf, q_buf;     // 0: operators, 1: vector X, 2: stage-1 results
  int32_t p_nkt, q_nkt;     // K tiles of each image
  int32_t nkt;              // K tiles of this segment
  int32_t pad_;
};

struct OzJob {
  int32_t seg_begin, seg_end;
  int32_t M, N;
  int32_t out_y;            // 0: stage-1 result into the FP64 intermediate buffer; 1: Y
  int32_t pad_;
  int64_t out_off;          // element offset of the output matrix (row-major, ld = N)
  int64_t x_off;            // element offset of X for the identity-identity term
  double axpy;
};

struct OzTile {
  int32_t job, mt, nt, pad_;  // nt counts 64-column tiles
};

struct OzSlice {             // FP64 matrix -> digit image + exponent table
  int64_t src_off, rs, cs;   // element (r, k) at src[src_off + r * rs + k * cs]
  int64_t dst_off;           // byte offset of the image
  int64_t exp_off;           // element offset of the exponent table
  int32_t R, K, nkt, nch;    // rows, K, K tiles, K chunks
  int32_t src_space;         // 0: operator arena, 1: X, 2: FP64 intermediates
  int32_t pad_;
  double scale;
};

struct OzSliceItem {
  int32_t job, rt, ch, pad_;
};

struct OzPlan {
  uint8_t* img[3] = {nullptr, nullptr, nullptr};
  int32_t* exps[3] = {nullptr, nullptr, nullptr};
  size_t img_bytes[3] = {0, 0, 0}, exp_elems[3] = {0, 0, 0};
  OzSlice *d_xsl = nullptr, *d_tsl = nullptr;
  OzSliceItem *d_xit = nullptr, *d_tit = nullptr;
  int64_t n_xit = 0, n_tit = 0;
  OzJob* d_jobs = nullptr;
  OzSeg* d_segs = nullptr;
  OzTile *d_tiles1 = nullptr, *d_tiles2 = nullptr;
  int64_t ntiles1 = 0, ntiles2 = 0;
  int* d_err = nullptr;
  int* h_err = nullptr;
  int sms = 0;
};

namespace tc {
#include "tc_ptx.cuh"

using OzL = Layout<false>;                 // 32-element K tiles, 64-byte rows and swizzle
constexpr int S = 7;                       // digits per operand element
constexpr int kN = 64;                     // output columns per tile
constexpr int kKT = OzL::KT;               // elements per K tile
constexpr int kPlane = OzL::CHUNK;         // bytes of one digit plane of one image tile
constexpr int kChunkKT = 256 / kKT;        // K tiles per exponent chunk (256 elements)
constexpr int kOzStages = 2;
constexpr int kOzThreads = 320;            // 2 + 8 warps
constexpr int kOzTmemCols = 512;           // S accumulators x 64 columns (448) -> 512
constexpr uint32_t kStageA = S * kPlane;   // 7 planes x 128 rows x 64 bytes
constexpr uint32_t kStageB = S * kPlane / 2;  // 7 planes x 64 rows x 64 bytes
constexpr uint32_t kStage = kStageA + kStageB;
constexpr size_t kOzSmem = kOzStages * kStage + 1024;

// ---------------------------------------------------------------- digit split
// |x| = M 2^(be - 1075); with E = be_max - 1021 (so |x| 2^-E < 1/2),
// q = round(|x| 2^(7S - E)) = round(M 2^(be - be_max + 7S - 54)) < 2^(7S - 1).
__device__ __forceinline__ void split_digits(double x, int be_max, int (&d)[S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7ff);
  const int rs = be_max - be + 54 - 7 * S;
  unsigned long long q = 0;
  if (be != 0 && rs < 64) {
    const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    q = rs > 0 ? (M + (1ull << (rs - 1))) >> rs : M;
  }
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    int r = (int)(q & 127ull);
    q >>= 7;
    if (r >= 64) {
      r -= 128;
      q += 1;
    }
    d[s] = r;
  }
  d[0] = (int)q;
  if (bits >> 63) {
#pragma unroll
    for (int s = 0; s < S; ++s) d[s] = -d[s];
  }
}

// One CTA per (slice job, row tile, K chunk): per-row exponent of the chunk, then the S
// digit planes of every element of the chunk.
__global__ void __launch_bounds__(256)
oz_slice_kernel(const OzSliceItem* __restrict__ items, const OzSlice* __restrict__ jobs,
                const double* __restrict__ arena, const double* __restrict__ x,
                const double* __restrict__ inter, uint8_t* __restrict__ img,
                int32_t* __restrict__ exps) {
  __shared__ int bemax[kRows];
  const OzSliceItem it = items[blockIdx.x];
  const OzSlice jb = jobs[it.job];
  const double* src = (jb.src_space == 0 ? arena : jb.src_space == 1 ? x : inter) + jb.src_off;
  const int kt0 = it.ch * kChunkKT;
  const int kt1 = min(kt0 + kChunkKT, jb.nkt);
  const int k0 = kt0 * kKT, k1 = min(kt1 * kKT, jb.K);
  const bool scaled = jb.scale != 1.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // pass 1: largest binary exponent of each row over the chunk
  for (int r = warp; r < kRows; r += 8) {
    const int64_t grow = (int64_t)it.rt * kRows + r;
    int m = 0;
    if (grow < jb.R) {
      for (int k = k0 + lane; k < k1; k += 32) {
        double v = src[grow * jb.rs + (int64_t)k * jb.cs];
        if (scaled) v *= jb.scale;
        const int be = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
        m = max(m, be);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      bemax[r] = m;
      exps[jb.exp_off + grow * jb.nch + it.ch] = m == 0 ? -30000 : m - 1021;
    }
  }
  __syncthreads();
  // pass 2: digit planes, one 16-byte group (8 elements) of one row per item
  constexpr int G = OzL::GROUPS;
  const bool kfast = jb.cs == 1;
  const int ngroups = (kt1 - kt0) * G;
  for (int idx = threadIdx.x; idx < kRows * ngroups; idx += blockDim.x) {
    int r, gg;
    if (kfast) { gg = idx % ngroups; r = idx / ngroups; }
    else { r = idx % kRows; gg = idx / kRows; }
    const int kt = kt0 + gg / G, g = gg % G;
    const int64_t grow = (int64_t)it.rt * kRows + r;
    int dig[8][S];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kt * kKT + g * 8 + e;
      double v = 0.0;
      if (grow < jb.R && k < jb.K) {
        v = src[grow * jb.rs + (int64_t)k * jb.cs];
        if (scaled) v *= jb.scale;
      }
      split_digits(v, bemax[r], dig[e]);
    }
    uint8_t* base = img + jb.dst_off + ((int64_t)it.rt * jb.nkt + kt) * S * kPlane + OzL::off(r, g);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      uint4 q;
      q.x = pack2_bf16(__float2bfloat16_rn((float)dig[0][s]), __float2bfloat16_rn((float)dig[1][s]));
      q.y = pack2_bf16(__float2bfloat16_rn((float)dig[2][s]), __float2bfloat16_rn((float)dig[3][s]));
      q.z = pack2_bf16(__float2bfloat16_rn((float)dig[4][s]), __float2bfloat16_rn((float)dig[5][s]));
      q.w = pack2_bf16(__float2bfloat16_rn((float)dig[6][s]), __float2bfloat16_rn((float)dig[7][s]));
      *reinterpret_cast<uint4*>(base + s * kPlane) = q;
    }
  }
}

__device__ __forceinline__ float pow2f(int e) {
  // 2^e as an FP32 power of two, 0 below the normal range
  if (e < -126) return 0.0f;
  if (e > 127) e = 127;
  return __int_as_float((e + 127) << 23);
}

// ---------------------------------------------------------------- grouped GEMM
// The GEMM uses the leading NS <= S digits of each operand (the planes of a tile are stored
// most significant first, so they are its first NS planes): the NS (NS + 1) / 2 digit pairs
// with s + u <= NS - 1 (28 for NS = 7).  Dropping the digits below NS truncates each operand
// to about 7 NS bits of its row-chunk scale; a projection whose input is known to be small
// against the quantity it corrects (the Davidson anchor update) needs no more.
//
// The MMAs of one K tile: the digit pairs (s, u) with s + u <= NS - 1, each into the
// accumulator of its scale group g = s + u, for both 16-element K steps.  The K step is
// the outermost loop and u the innermost, so consecutive MMAs write different
// accumulators; the descriptors are the stage's base descriptors plus constant offsets
// (in 16-byte units; every address stays below 256 KB, so the 14-bit address field does
// not carry).  FIRST: the first K tile of an exponent chunk, in which the first MMA of each
// group (s = 0, first K step) overwrites its accumulator.  Called by the whole MMA warp;
// leader (one lane) issues.
template <int NS, bool FIRST>
__device__ __forceinline__ void issue_ktile(uint32_t tmem_base, uint64_t ad0, uint64_t bd0,
                                            bool leader) {
  constexpr uint32_t idesc = instr_desc<false, kN>();
#pragma unroll
  for (int kk = 0; kk < OzL::ROWB / 32; ++kk) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int u = 0; u < NS - s; ++u) {
        const uint64_t ad = ad0 + (uint64_t)((s * kPlane + kk * 32) >> 4);
        const uint64_t bd = bd0 + (uint64_t)((u * (kPlane / 2) + kk * 32) >> 4);
        if (leader)
          mma<false>(tmem_base + (uint32_t)((s + u) * kN), ad, bd, idesc,
                     (FIRST && kk == 0 && s == 0) ? 0u : 1u);
      }
    }
  }
}

template <int NS>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const OzTile* __restrict__ tiles, int ntiles, const OzJob* __restrict__ jobs,
               const OzSeg* __restrict__ segs, const uint8_t* __restrict__ b0,
               const uint8_t* __restrict__ b1, const uint8_t* __restrict__ b2,
               const int32_t* __restrict__ e0, const int32_t* __restrict__ e1,
               const int32_t* __restrict__ e2, double* __restrict__ inter,
               double* __restrict__ y, const double* __restrict__ x, int* __restrict__ gerr) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[kOzStages], empty_bar[kOzStages];
  __shared__ __align__(8) uint64_t tfull_bar, tempty_bar, drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kOzStages; ++i) {
      mbar_init(smem_u32(&full_bar[i]), 1);
      mbar_init(smem_u32(&empty_bar[i]), 1);
    }
    mbar_init(smem_u32(&tfull_bar), 1);
    mbar_init(smem_u32(&tempty_bar), 256);
    mbar_init(smem_u32(&drain_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kOzTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  const uint8_t* imgs[3] = {b0, b1, b2};
  const int32_t* exs[3] = {e0, e1, e2};

  if (warp == 0) {
    // ------------------------------------------------ producer (kOzStages-deep ring)
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
        const OzTile tile = tiles[t];
        const OzJob job = jobs[tile.job];
        for (int si = job.seg_begin; si < job.seg_end && !abort_flag; ++si) {
          const OzSeg sg = segs[si];
          const uint8_t* P = imgs[sg.p_buf] + sg.p_off + (int64_t)tile.mt * sg.p_nkt * kStageA;
          const uint8_t* Q = imgs[sg.q_buf] + sg.q_off + (int64_t)(tile.nt >> 1) * sg.q_nkt * kStageA +
                             (tile.nt & 1) * (kPlane / 2);
          for (int kt = 0; kt < sg.nkt; ++kt) {
            if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, &abort_flag, gerr, 11)) break;
            const uint32_t sa = smem_u32(smem + stage * kStage);
            const uint32_t fb = smem_u32(&full_bar[stage]);
            mbar_expect_tx(fb, NS * kPlane + NS * (kPlane / 2));
            bulk_g2s(sa, P + (int64_t)kt * kStageA, NS * kPlane, fb);
            const uint8_t* qk = Q + (int64_t)kt * kStageA;
#pragma unroll
            for (int pl = 0; pl < NS; ++pl)
              bulk_g2s(sa + kStageA + pl * (kPlane / 2), qk + pl * kPlane, kPlane / 2, fb);
            ++issued;
            if (++stage == kOzStages) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (abort_flag) {
        // the copies still in flight complete before the CTA exits (bounded)
        int st = stage;
        uint32_t ph = phase;
        for (int i = 0; i < kOzStages && i < issued; ++i) {
          if (--st < 0) { st = kOzStages - 1; ph ^= 1; }
          const uint64_t t0 = gtime();
          while (!mbar_try_wait(smem_u32(&full_bar[st]), ph) && gtime() - t0 < kWaitNs) {}
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    // The whole warp runs the loop in step (its control flow and the descriptors stay
    // warp-uniform); lane 0 alone issues the MMAs and the commits that track them.
    const bool leader = lane == 0;
    int stage = 0;
    uint32_t phase = 0, acc_phase = 0;
    bool any = false;
    for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
      const OzJob job = jobs[tiles[t].job];
      for (int si = job.seg_begin; si < job.seg_end && !abort_flag; ++si) {
        const int nkt = segs[si].nkt;
        for (int c0 = 0; c0 < nkt && !abort_flag; c0 += kChunkKT) {
          if (!mbar_wait_warp(smem_u32(&tempty_bar), acc_phase ^ 1, &abort_flag, gerr, 12)) break;
          tc_fence_after();
          const int c1 = min(c0 + kChunkKT, nkt);
          for (int kt = c0; kt < c1; ++kt) {
            if (!mbar_wait_warp(smem_u32(&full_bar[stage]), phase, &abort_flag, gerr, 13)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + stage * kStage);
            const uint64_t ad0 = OzL::desc(sa), bd0 = OzL::desc(sa + kStageA);
            if (kt == c0) issue_ktile<NS, true>(tmem_base, ad0, bd0, leader);
            else issue_ktile<NS, false>(tmem_base, ad0, bd0, leader);
            if (leader) tc_commit(smem_u32(&empty_bar[stage]));
            __syncwarp();
            any = true;
            if (++stage == kOzStages) { stage = 0; phase ^= 1; }
          }
          if (leader) tc_commit(smem_u32(&tfull_bar));
          __syncwarp();
          acc_phase ^= 1;
        }
      }
    }
    if (any && leader) {
      tc_commit(smem_u32(&drain_bar));
      const uint64_t t0 = gtime();
      while (!mbar_try_wait(smem_u32(&drain_bar), 0) && gtime() - t0 < kWaitNs) {}
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ epilogue (warps 2..9)
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;         // which 32 of the 64 columns
    const int row = quarter * 32 + lane;
    uint32_t acc_phase = 0;
    bool stop = false;
    for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
      const OzTile tile = tiles[t];
      const OzJob job = jobs[tile.job];
      const int64_t m = (int64_t)tile.mt * kRows + row;
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { hi[j] = 0.0f; lo[j] = 0.0f; }
      for (int si = job.seg_begin; si < job.seg_end && !stop; ++si) {
        const OzSeg sg = segs[si];
        const int pch = (sg.p_nkt + kChunkKT - 1) / kChunkKT;
        const int qch = (sg.q_nkt + kChunkKT - 1) / kChunkKT;
        const int32_t* pe = exs[sg.p_buf] + sg.p_eoff + m * pch;
        const int32_t* qe = exs[sg.q_buf] + sg.q_eoff + ((int64_t)tile.nt * kN + half * 32) * qch;
        for (int c0 = 0, ch = 0; c0 < sg.nkt; c0 += kChunkKT, ++ch) {
          if (!mbar_wait(smem_u32(&tfull_bar), acc_phase, &abort_flag, gerr, 14)) { stop = true; break; }
          tc_fence_after();
          const int ep = pe[ch];
          float sc[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) sc[j] = pow2f(ep + qe[j * qch + ch]);
#pragma unroll 1
          for (int g = 0; g < NS; ++g) {
            uint32_t v[32];
            tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * kN + half * 32), v);
            const float gs = pow2f(-7 * (g + 2));
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float a = __uint_as_float(v[j]) * (sc[j] * gs);   // exact: powers of two
              const float s = hi[j] + a;
              const float bp = s - hi[j];
              const float err = (hi[j] - (s - bp)) + (a - bp);
              hi[j] = s;
              lo[j] += err;
            }
          }
          tc_fence_before();
          mbar_arrive(smem_u32(&tempty_bar));
          acc_phase ^= 1;
        }
      }
      if (stop) break;
      if (m < job.M) {
        double* out = (job.out_y ? y : inter) + job.out_off + m * job.N;
        const double* xr = x + job.x_off + m * job.N;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t n = (int64_t)tile.nt * kN + half * 32 + j;
          if (n < job.N) {
            double val = (double)hi[j] + (double)lo[j];
            if (job.axpy != 0.0) val = fma(job.axpy, xr[n], val);
            out[n] = val;
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kOzTmemCols)
                 : "memory");
  }
}

}  // namespace tc

// ======================================================================== host side
namespace {

using tc::kRows;

int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

struct OzAlloc {
  int64_t bytes = 0, exps = 0;
  // image of rows x K: returns (byte offset, exponent offset, nkt)
  std::tuple<int64_t, int64_t, int> add(int64_t rows, int64_t K) {
    const int nrt = cdiv(rows, kRows), nkt = cdiv(K, tc::kKT), nch = cdiv(nkt, tc::kChunkKT);
    const int64_t off = bytes, eoff = exps;
    bytes += (int64_t)nrt * nkt * tc::S * tc::kPlane;
    exps += (int64_t)nrt * kRows * nch;
    return {off, eoff, nkt};
  }
};

template <typename T>
dmrg_status up(T** dst, const std::vector<T>& v, cudaStream_t st) {
  *dst = nullptr;
  if (v.empty()) return DMRG_OK;
  DMRG_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * v.size()));
  DMRG_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return DMRG_OK;
}

void free_oz(OzPlan* o) {
  if (!o) return;
  for (int b = 0; b < 3; ++b) {
    cudaFree(o->img[b]);
    cudaFree(o->exps[b]);
  }
  cudaFree(o->d_xsl);
  cudaFree(o->d_tsl);
  cudaFree(o->d_xit);
  cudaFree(o->d_tit);
  cudaFree(o->d_jobs);
  cudaFree(o->d_segs);
  cudaFree(o->d_tiles1);
  cudaFree(o->d_tiles2);
  if (o->h_err) cudaFreeHost(o->h_err);
  delete o;
}

void slice_items(const std::vector<OzSlice>& jobs, std::vector<OzSliceItem>* items) {
  for (size_t j = 0; j < jobs.size(); ++j)
    for (int rt = 0; rt < cdiv(jobs[j].R, kRows); ++rt)
      for (int ch = 0; ch < jobs[j].nch; ++ch) items->push_back(OzSliceItem{(int32_t)j, rt, ch, 0});
}

dmrg_status build_oz(dmrg_plan* p, cudaStream_t st, OzPlan** out) {
  OzPlan* o = new OzPlan();
  auto fail = [&](dmrg_status s) { free_oz(o); return s; };
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&o->sms, cudaDevAttrMultiProcessorCount, dev);
  if (p->T_elems == 0 && !p->records.empty()) {
    // the FP64 intermediates buffer exists whenever a record has two proper factors
  }
  OzAlloc ops, xs, ts;
  std::vector<OzSlice> op_jobs, x_jobs, t_jobs;
  auto mk = [](int64_t src_off, int64_t rs, int64_t cs, std::tuple<int64_t, int64_t, int> im,
               int64_t R, int64_t K, int space, double scale) {
    OzSlice j{};
    j.src_off = src_off;
    j.rs = rs;
    j.cs = cs;
    j.dst_off = std::get<0>(im);
    j.exp_off = std::get<1>(im);
    j.nkt = std::get<2>(im);
    j.nch = cdiv(j.nkt, tc::kChunkKT);
    j.R = (int32_t)R;
    j.K = (int32_t)K;
    j.src_space = space;
    j.scale = scale;
    return j;
  };
  // operator images keyed by (side, op, block, scale)
  std::map<std::tuple<int, int, int, double>, std::tuple<int64_t, int64_t, int>> opimg;
  auto op_image = [&](int side, int op, int blk, double scale) {
    auto key = std::make_tuple(side, op, blk, scale);
    auto it = opimg.find(key);
    if (it != opimg.end()) return it->second;
    const HostBlock& hb = side == 0 ? p->opsL[op][blk] : p->opsR[op][blk];
    auto im = ops.add(hb.rows, hb.cols);
    op_jobs.push_back(mk(hb.arena_off, hb.cols, 1, im, hb.rows, hb.cols, 0, scale));
    opimg[key] = im;
    return im;
  };
  const int npairs = (int)p->pair_i.size();
  std::vector<std::tuple<int64_t, int64_t, int>> xa(npairs), xb(npairs);
  for (int q = 0; q < npairs; ++q) {
    const int64_t di = p->dimL[p->pair_i[q]], dk = p->dimR[p->pair_k[q]];
    xa[q] = xs.add(di, dk);
    xb[q] = xs.add(dk, di);
    if (di * dk > 0) {
      x_jobs.push_back(mk(p->pair_off[q], dk, 1, xa[q], di, dk, 1, 1.0));
      x_jobs.push_back(mk(p->pair_off[q], 1, dk, xb[q], dk, di, 1, 1.0));
    }
  }
  std::vector<OzJob> jobs;
  std::vector<OzSeg> segs;
  std::vector<OzTile> tiles1, tiles2;
  std::vector<std::tuple<int64_t, int64_t, int>> timg(p->records.size());
  auto seg = [](int pb, std::tuple<int64_t, int64_t, int> P, int qb,
                std::tuple<int64_t, int64_t, int> Q, int nkt) {
    OzSeg s{};
    s.p_off = std::get<0>(P);
    s.p_eoff = std::get<1>(P);
    s.p_nkt = std::get<2>(P);
    s.q_off = std::get<0>(Q);
    s.q_eoff = std::get<1>(Q);
    s.q_nkt = std::get<2>(Q);
    s.p_buf = pb;
    s.q_buf = qb;
    s.nkt = nkt;
    return s;
  };
  std::vector<std::pair<int64_t, int>> order1, order2;
  for (size_t ri = 0; ri < p->records.size(); ++ri) {
    const Record& r = p->records[ri];
    if (r.a_blk < 0 || r.b_blk < 0) continue;
    const int a_op = p->terms[r.term].a_op, b_op = p->terms[r.term].b_op;
    OzJob job{};
    job.out_y = 0;
    job.out_off = r.inter_off;
    job.seg_begin = (int32_t)segs.size();
    if (r.a_first) {  // T [dj x dk] = A X
      job.M = (int32_t)r.dj;
      job.N = (int32_t)r.dk;
      if (r.di > 0) segs.push_back(seg(0, op_image(0, a_op, r.a_blk, 1.0), 1, xb[r.pin], cdiv(r.di, tc::kKT)));
      timg[ri] = ts.add(r.dj, r.dk);
      t_jobs.push_back(mk(r.inter_off, r.dk, 1, timg[ri], r.dj, r.dk, 2, 1.0));
    } else {          // U^T [dl x di] = (coef B) X^T
      job.M = (int32_t)r.dl;
      job.N = (int32_t)r.di;
      if (r.dk > 0) segs.push_back(seg(0, op_image(1, b_op, r.b_blk, r.coef), 1, xa[r.pin], cdiv(r.dk, tc::kKT)));
      timg[ri] = ts.add(r.dl, r.di);
      t_jobs.push_back(mk(r.inter_off, r.di, 1, timg[ri], r.dl, r.di, 2, 1.0));
    }
    job.seg_end = (int32_t)segs.size();
    if (job.M > 0 && job.N > 0) order1.push_back({(int64_t)(r.a_first ? r.di : r.dk), (int)jobs.size()});
    jobs.push_back(job);
  }
  std::vector<std::vector<int>> by_out(npairs);
  for (size_t ri = 0; ri < p->records.size(); ++ri) by_out[p->records[ri].pout].push_back((int)ri);
  for (int q = 0; q < npairs; ++q) {
    const int i = p->pair_i[q], k = p->pair_k[q];
    OzJob job{};
    job.M = (int32_t)p->dimL[i];
    job.N = (int32_t)p->dimR[k];
    job.out_y = 1;
    job.out_off = p->pair_off[q];
    job.x_off = p->pair_off[q];
    job.seg_begin = (int32_t)segs.size();
    int64_t cost = 0;
    for (int ri : by_out[q]) {
      const Record& r = p->records[ri];
      const int a_op = p->terms[r.term].a_op, b_op = p->terms[r.term].b_op;
      if (r.a_blk >= 0 && r.b_blk >= 0) {
        if (r.a_first) {
          if (r.dk > 0) segs.push_back(seg(2, timg[ri], 0, op_image(1, b_op, r.b_blk, r.coef), cdiv(r.dk, tc::kKT)));
        } else {
          if (r.di > 0) segs.push_back(seg(0, op_image(0, a_op, r.a_blk, 1.0), 2, timg[ri], cdiv(r.di, tc::kKT)));
        }
      } else if (r.a_blk >= 0) {
        if (r.di > 0) segs.push_back(seg(0, op_image(0, a_op, r.a_blk, r.coef), 1, xb[r.pin], cdiv(r.di, tc::kKT)));
      } else if (r.b_blk >= 0) {
        if (r.dk > 0) segs.push_back(seg(1, xa[r.pin], 0, op_image(1, b_op, r.b_blk, r.coef), cdiv(r.dk, tc::kKT)));
      } else {
        if (r.pin == r.pout) job.axpy += r.coef;  // (other segments: seg_axpy pass)
      }
    }
    job.seg_end = (int32_t)segs.size();
    for (int s = job.seg_begin; s < job.seg_end; ++s) cost += segs[s].nkt;
    if (job.M > 0 && job.N > 0) order2.push_back({cost, (int)jobs.size()});
    jobs.push_back(job);
  }
  for (const OzSeg& s : segs) {
    if (s.nkt > s.p_nkt || s.nkt > s.q_nkt) {
      set_error("internal: digit segment K tiles exceed its operand images");
      return fail(DMRG_ERR_SHAPE);
    }
  }
  auto by_cost = [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  };
  std::stable_sort(order1.begin(), order1.end(), by_cost);
  std::stable_sort(order2.begin(), order2.end(), by_cost);
  for (auto& pr : order1)
    for (int mt = 0; mt < cdiv(jobs[pr.second].M, kRows); ++mt)
      for (int nt = 0; nt < cdiv(jobs[pr.second].N, tc::kN); ++nt) tiles1.push_back(OzTile{pr.second, mt, nt, 0});
  for (auto& pr : order2)
    for (int mt = 0; mt < cdiv(jobs[pr.second].M, kRows); ++mt)
      for (int nt = 0; nt < cdiv(jobs[pr.second].N, tc::kN); ++nt) tiles2.push_back(OzTile{pr.second, mt, nt, 0});

  // buffers
  OzAlloc* allocs[3] = {&ops, &xs, &ts};
  for (int b = 0; b < 3; ++b) {
    o->img_bytes[b] = (size_t)allocs[b]->bytes;
    o->exp_elems[b] = (size_t)allocs[b]->exps;
    if (o->img_bytes[b] && (cudaMalloc((void**)&o->img[b], o->img_bytes[b]) != cudaSuccess ||
                            cudaMalloc((void**)&o->exps[b], sizeof(int32_t) * o->exp_elems[b]) != cudaSuccess)) {
      cudaGetLastError();
      set_error("cudaMalloc for the FP64-emulation operand images failed");
      return fail(DMRG_ERR_OOM);
    }
    p->device_bytes += o->img_bytes[b] + sizeof(int32_t) * o->exp_elems[b];
  }
  dmrg_status s;
  std::vector<OzSliceItem> op_items, x_items, t_items;
  slice_items(op_jobs, &op_items);
  slice_items(x_jobs, &x_items);
  slice_items(t_jobs, &t_items);
  if (!op_items.empty()) {
    OzSlice* dj = nullptr;
    OzSliceItem* di = nullptr;
    if ((s = up(&dj, op_jobs, st)) != DMRG_OK) return fail(s);
    if ((s = up(&di, op_items, st)) != DMRG_OK) { cudaFree(dj); return fail(s); }
    tc::oz_slice_kernel<<<(unsigned)op_items.size(), 256, 0, st>>>(di, dj, p->arena, nullptr, nullptr,
                                                                 o->img[0], o->exps[0]);
    note_launch();
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);
    cudaFree(dj);
    cudaFree(di);
    if (e != cudaSuccess) {
      set_error("oz_slice_kernel: %s", cudaGetErrorString(e));
      return fail(DMRG_ERR_CUDA);
    }
  }
  if ((s = up(&o->d_xsl, x_jobs, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_xit, x_items, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_tsl, t_jobs, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_tit, t_items, st)) != DMRG_OK) return fail(s);
  o->n_xit = (int64_t)x_items.size();
  o->n_tit = (int64_t)t_items.size();
  if ((s = up(&o->d_jobs, jobs, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_segs, segs, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_tiles1, tiles1, st)) != DMRG_OK) return fail(s);
  if ((s = up(&o->d_tiles2, tiles2, st)) != DMRG_OK) return fail(s);
  o->ntiles1 = (int64_t)tiles1.size();
  o->ntiles2 = (int64_t)tiles2.size();
  if (cudaHostAlloc((void**)&o->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&o->d_err, o->h_err, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("mapped host allocation for the kernel error word failed");
    return fail(DMRG_ERR_OOM);
  }
  *o->h_err = 0;
  DMRG_CUDA_TRY(cudaStreamSynchronize(st));
  *out = o;
  return DMRG_OK;
}

}  // namespace

dmrg_status oz_error_status(dmrg_plan* p) {
  if (p->oz && p->oz->h_err && *p->oz->h_err != 0) {
    set_error("FP64-emulation projection kernel reported error %d (a bounded wait timed out)",
              *p->oz->h_err);
    return DMRG_ERR_CUDA;
  }
  return DMRG_OK;
}

void destroy_oz(dmrg_plan* p) {
  if (!p) return;
  free_oz(p->oz);
  p->oz = nullptr;
}

namespace {

// the two GEMM launches of a projection with the leading NS digits of every operand
template <int NS>
dmrg_status launch_oz_gemms(dmrg_plan* p, const double* x, double* y, cudaStream_t st) {
  OzPlan* o = p->oz;
  static bool configured[64] = {false};
  int dev = 0;
  DMRG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    DMRG_CUDA_TRY(cudaFuncSetAttribute(tc::oz_gemm_kernel<NS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kOzSmem));
    configured[dev] = true;
  }
  if (o->n_xit > 0) {
    tc::oz_slice_kernel<<<(unsigned)o->n_xit, 256, 0, st>>>(o->d_xit, o->d_xsl, p->arena, x, p->T,
                                                          o->img[1], o->exps[1]);
    DMRG_LAUNCH_CHECK();
  }
  if (o->ntiles1 > 0) {
    const int grid = (int)std::min<int64_t>(o->ntiles1, o->sms);
    tc::oz_gemm_kernel<NS><<<grid, tc::kOzThreads, tc::kOzSmem, st>>>(
        o->d_tiles1, (int)o->ntiles1, o->d_jobs, o->d_segs, o->img[0], o->img[1], nullptr,
        o->exps[0], o->exps[1], nullptr, p->T, y, x, o->d_err);
    DMRG_LAUNCH_CHECK();
  }
  if (o->n_tit > 0) {
    tc::oz_slice_kernel<<<(unsigned)o->n_tit, 256, 0, st>>>(o->d_tit, o->d_tsl, p->arena, x, p->T,
                                                          o->img[2], o->exps[2]);
    DMRG_LAUNCH_CHECK();
  }
  if (o->ntiles2 > 0) {
    const int grid = (int)std::min<int64_t>(o->ntiles2, o->sms);
    tc::oz_gemm_kernel<NS><<<grid, tc::kOzThreads, tc::kOzSmem, st>>>(
        o->d_tiles2, (int)o->ntiles2, o->d_jobs, o->d_segs, o->img[0], o->img[1], o->img[2],
        o->exps[0], o->exps[1], o->exps[2], p->T, y, x, o->d_err);
    DMRG_LAUNCH_CHECK();
  }
  return DMRG_OK;
}

}  // namespace

dmrg_status launch_project_oz(dmrg_plan* p, const double* x, double* y, cudaStream_t st,
                              int digits) {
  if (digits < 2 || digits > tc::S) {
    set_error("internal: FP64_TC digit count %d outside [2, %d]", digits, tc::S);
    return DMRG_ERR_INVALID_ARG;
  }
  if (!p->oz) {
    OzPlan* o = nullptr;
    DMRG_TRY(build_oz(p, st, &o));
    p->oz = o;
  }
  DMRG_TRY(oz_error_status(p));
  switch (digits) {
    case 2: DMRG_TRY(launch_oz_gemms<2>(p, x, y, st)); break;
    case 3: DMRG_TRY(launch_oz_gemms<3>(p, x, y, st)); break;
    case 4: DMRG_TRY(launch_oz_gemms<4>(p, x, y, st)); break;
    case 5: DMRG_TRY(launch_oz_gemms<5>(p, x, y, st)); break;
    case 6: DMRG_TRY(launch_oz_gemms<6>(p, x, y, st)); break;
    default: DMRG_TRY(launch_oz_gemms<7>(p, x, y, st)); break;
  }
  return launch_seg_axpy(p, x, y, nullptr, nullptr, st);
}

}  // namespace dmrg
