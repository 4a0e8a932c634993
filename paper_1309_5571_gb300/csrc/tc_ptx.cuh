// PTX wrappers for the tcgen05 / TMEM / mbarrier / bulk-copy kernels (shared by the
// tensor-core projection kernels).  Included inside namespace dmrg::tc.
#pragma once

constexpr int kRows = 128;                 // rows of an image tile, M of the MMA
constexpr int kChunk = 128 * 128;          // bytes of one plane of one image tile
constexpr uint64_t kWaitNs = 2000000000ull;

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity.  Returns false on abort or timeout.
static __device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       int* gerr, int code) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort_flag) return false;
      const uint64_t t = gtime();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kWaitNs) {
        *abort_flag = 1;
        atomicCAS(gerr, 0, code);
        return false;
      }
    }
  }
}
// The same wait made by every lane of a warp, with one outcome for all lanes (false if any
// lane saw an abort or a timeout), so that the warp leaves it converged.
static __device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity,
                                                      volatile int* abort_flag, int* gerr,
                                                      int code) {
  const bool ok = mbar_wait(bar, parity, abort_flag, gerr, code);
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled layout;
// 8-row core-matrix groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor: FP32 accumulate, A/B format (1 = BF16 in kind::f16,
// 2 = TF32 in kind::tf32), both K-major, M = 128, N (default 128).
template <bool TF32, int N = kRows>
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 16 TMEM lanes x 32 columns: thread t receives, for each 8-column group j = 0..3, the
// column pair 8 j + 2 (t % 4) + {0, 1} of lane t / 4 (v[4 j], v[4 j + 1]) and of lane
// t / 4 + 8 (v[4 j + 2], v[4 j + 3]), so that four consecutive threads hold eight
// consecutive columns of one row
__device__ __forceinline__ void tmem_ld16x256_x4(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ uint32_t pack2_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// byte offset of the 16-byte group g of row r inside one plane of an image tile
__host__ __device__ __forceinline__ uint32_t swz(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

// Operand image layout.  An image tile is 128 rows x one K-tile of 32 elements, K-major:
//   BF16x3 planes: 64-byte rows, 64-byte swizzle (8-row atoms of 512 bytes; the 16-byte
//                  group g of row r sits at group g ^ ((r >> 1) & 3) of its row), 8 KB
//   TF32:          128-byte rows, 128-byte swizzle (1024-byte atoms, g ^ (r & 7)), 16 KB
// so that a pipeline stage of BF16x3 holds three planes of A (24 KB) and three planes of a
// 128- or 256-row B (up to 48 KB), and three such 72 KB stages fit in shared memory.
template <bool TF32>
struct Layout {
  static constexpr int ROWB = TF32 ? 128 : 64;  // bytes per image row
  static constexpr int GROUPS = ROWB / 16;      // 16-byte groups per row
  static constexpr int KT = 32;                 // elements per K-tile
  static constexpr int CHUNK = kRows * ROWB;    // bytes of one plane of one image tile
  __host__ __device__ static uint32_t off(int r, int g) {
    if constexpr (TF32) return swz(r, g);
    else return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((g ^ ((r >> 1) & 3)) << 4));
  }
  // shared-memory matrix descriptor of a K-major operand in this layout (descriptor
  // version 1; stride byte offset = distance between 8-row atoms)
  __device__ static uint64_t desc(uint32_t addr) {
    if constexpr (TF32) {
      return smem_desc(addr);
    } else {
      uint64_t d = 0;
      d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
      d |= (uint64_t)(16u >> 4) << 16;
      d |= (uint64_t)(512u >> 4) << 32;
      d |= (uint64_t)1 << 46;
      d |= (uint64_t)4 << 61;  // 64-byte swizzle
      return d;
    }
  }
};
