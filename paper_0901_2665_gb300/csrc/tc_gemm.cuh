// tcgen05 GEMM for sm_103a: D (128 x BN per CTA, fp32 in TMEM) =
// sum_k A[m, k] B[n, k] with A and B K-major operands loaded by TMA into
// 128-byte-swizzled shared memory, one elected thread issuing
// tcgen05.mma (M = 128, N = BN; kind::tf32 on fp32 operands, kind::f16 on
// BF16 operands or on split BF16 pairs, see KIND below), and a
// caller-supplied epilogue that reads the accumulator back with tcgen05.ld.
//
// Warp roles (192 threads): warp 0 = TMA producer, warp 1 = TMEM owner and
// MMA issuer, warps 2-5 = epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
// Every mbarrier wait is bounded; on expiry the kernel records DEV_TIMEOUT in
// the status word, stops issuing work and still releases its TMEM.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"

namespace feast {
namespace tc {

constexpr int kBlockM = 128;
constexpr int kBlockK = 32;                      // fp32 elements per 128-byte swizzle row
constexpr int kATileBytes = kBlockM * kBlockK * 4;   // 16 KB
constexpr int kThreads = 192;
constexpr long long kWaitLimit = 1LL << 26;      // polls before a wait gives up (~1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and DEV_TIMEOUT recorded) when `limit` polls are
// used up or another role of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, int* status,
                                                volatile int* abort_flag, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(status, (int)DEV_TIMEOUT);
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status, volatile int* abort_flag) {
  return mbar_wait_limit(bar, parity, status, abort_flag, kWaitLimit);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// 3-D tiled TMA load / store (coordinates innermost first).  A store reads
// shared memory through the async proxy: the writing threads fence first.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// waits until the committed stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// waits until the committed stores are complete
__device__ __forceinline__ void bulk_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Programmatic dependent launch: wait until the grid this one was launched
// after (with programmatic stream serialisation) has completed and its
// memory is visible; then let the next such grid start its own prologue.
// Both are no-ops for a grid launched the ordinary way.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1; the leading byte offset is unused for this layout.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1u) << 16;
  d |= static_cast<uint64_t>(1024u >> 4) << 32;
  d |= static_cast<uint64_t>(1u) << 46;
  d |= static_cast<uint64_t>(2u) << 61;
  return d;
}

// Instruction descriptor for kind::tf32: fp32 accumulator, TF32 A and B,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// BF16 A and B (kind::f16, K = 16 per instruction, 32 bytes like TF32's 8).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive fp32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round an fp32 value to TF32 (10 explicit mantissa bits, nearest).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split bf16 pairs (the KIND 2 operand layout of k_tc_gemm): a row keeps the
// byte size of its fp32 form; each 128-byte block of 32 K-columns holds their
// bf16 leading parts hi = bf16(x) (nearest), then their trailing parts
// lo = bf16(x - hi).  K-column c's leading part is bf16 element
// 64 (c / 32) + c % 32 of the row, its trailing part 32 elements further.
__device__ __forceinline__ void store_pair(float* row, int kcol, float x) {
  __nv_bfloat16* r = reinterpret_cast<__nv_bfloat16*>(row) + ((kcol >> 5) << 6) + (kcol & 31);
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  r[0] = hi;
  r[32] = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Leading and trailing parts of two values, packed (first value low).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Four consecutive K-columns kcol..kcol+3 (kcol a multiple of 4, the row
// 16-byte aligned): two 8-byte stores.
__device__ __forceinline__ void store_pair4(float* row, int kcol, float4 x) {
  uint2 h, l;
  split2(x.x, x.y, h.x, l.x);
  split2(x.z, x.w, h.y, l.y);
  uint2* r = reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(row) + ((kcol >> 5) << 6) + (kcol & 31));
  r[0] = h;
  r[8] = l;   // 32 bf16 further
}

// Geometry of a batched launch: grid (n tiles, m tiles, batch).  The A tile
// of CTA (x, tm, e) starts at row a_row0 + e*a_batch + tm*128 of A's tensor
// map, the B tile at row b_row0 + e*b_batch + tn*BN with tn = x + tn_base,
// moved past tn_skip; nk K-blocks of 32.
struct Geom {
  int a_row0, a_batch;
  int b_row0, b_batch;
  int nk;
  int tn_base = 0;    // first n tile of the launch
  int tn_skip = -1;   // n tile left out (the grid's x covers the others), -1 = none
  unsigned long long node_mask = 0;   // != 0: the batch index of CTA z is the z-th set bit (a compacted batch)
  // split > 0: batch indices b >= split take their A tile at row
  // a_row0_hi + (b - split) a_batch (a second set of A rows, e.g. the
  // other end of a two-ended elimination)
  int split = 0;
  int a_row0_hi = 0;
  // active != nullptr: a CTA whose node is inactive (active[b], b the batch
  // index, or b - split above the split) leaves at once: a launch of fixed
  // shape, as a CUDA graph replays it, over the nodes a device-side decision
  // selects
  const int* active = nullptr;
};

// Position of the z-th set bit (z from 0) of a 64-bit mask.
__device__ __forceinline__ int nth_set_bit(unsigned long long mask, int z) {
  const unsigned lo = static_cast<unsigned>(mask), hi = static_cast<unsigned>(mask >> 32);
  const int c = __popc(lo);
  return z < c ? static_cast<int>(__fns(lo, 0, z + 1)) : 32 + static_cast<int>(__fns(hi, 0, z - c + 1));
}

template <int BN, int STAGES>
struct Smem {
  static constexpr int kBTileBytes = BN * kBlockK * 4;
  static constexpr int kStageBytes = kATileBytes + kBTileBytes;
  static constexpr int kTmemCols = BN < 32 ? 32 : BN;
  static constexpr size_t kPipeBytes = (size_t)STAGES * kStageBytes;
  static constexpr size_t kBytes = 1024 /*align slack*/ + kPipeBytes + 256;
};

// Epilogues may ask for shared memory of their own (static constexpr size_t
// kExtraSmem, 1024-byte aligned, after the pipeline).  They then provide a
// prologue, epi.prologue(e, tm, tn, ept, extra, status, abort_flag), that the
// epilogue threads run at kernel start while the main loop is under way, and
// take the accumulator through epi.run(e, tm, tn, row, lane_taddr, ept, stage,
// extra, status, abort_flag) instead of operator() (stage: the pipeline
// shared memory, free once the accumulator is complete).
template <class E, class = void>
struct EpiExtra {
  static constexpr size_t kBytes = 0;
};
template <class E>
struct EpiExtra<E, std::void_t<decltype(E::kExtraSmem)>> {
  static constexpr size_t kBytes = E::kExtraSmem;
};

// Epilogues may also declare a register block `Pre` and a member
// prefetch(e, tm, tn, row, Pre&) that the epilogue threads run before they
// wait for the accumulator (global loads that the epilogue will need, issued
// while the main loop is under way); the accumulator is then taken through
// epi(e, tm, tn, row, lane_taddr, ept, stage, pre).
template <class E, class = void>
struct EpiPre {
  static constexpr bool kHas = false;
};
template <class E>
struct EpiPre<E, std::void_t<typename E::Pre>> {
  static constexpr bool kHas = true;
};

template <int BN, int STAGES, class Epi>
constexpr size_t smem_bytes() {
  return Smem<BN, STAGES>::kBytes + (EpiExtra<Epi>::kBytes ? 1024 + EpiExtra<Epi>::kBytes : 0);
}

// Named barrier of the 128 epilogue threads (warps 2-5).
__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Epilogue contract: epi(e, tm, tn, row, lane_taddr, ept, stage) with row in
// [0, 128) the accumulator row (TMEM lane) of this thread, lane_taddr the TMEM
// address of that lane at column 0, ept in [0, 128) the thread's index in the
// epilogue group and stage the pipeline shared memory (Smem::kPipeBytes),
// free for reuse once the accumulator is complete.
// KIND 0: fp32 operands read as TF32 (kind::tf32); KIND 1: BF16 operands
// (kind::f16).  A K-block is one 128-byte swizzle row either way: 32 fp32 or
// 64 bf16 elements; geo.nk counts K-blocks.
// KIND 2: split BF16 pairs.  Each 128-byte row holds 32 K-columns as their
// bf16 leading parts x_hi = bf16(x) (bytes 0-63) then their trailing parts
// x_lo = bf16(x - x_hi) (bytes 64-127), so that x_hi + x_lo carries 16
// significant bits, and C += A_hi B_hi + A_hi B_lo + A_lo B_hi: six
// kind::f16 MMAs of K = 16 per K-block (the dropped A_lo B_lo is below the
// pairs' own rounding).  A K-block then covers 32 K-columns, as for TF32.
template <int BN, int STAGES, class Epi, int KIND = 0>
__global__ void __launch_bounds__(kThreads)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Geom geo,
              const __grid_constant__ Epi epi, int* status) {
  using S = Smem<BN, STAGES>;
  constexpr int kStages = STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kATileBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * S::kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfull + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int e = geo.node_mask ? nth_set_bit(geo.node_mask, (int)blockIdx.z) : (int)blockIdx.z;
  const int tm = blockIdx.y;
  int tn = (int)blockIdx.x + geo.tn_base;
  if (geo.tn_skip >= 0 && tn >= geo.tn_skip) ++tn;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, S::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // the set-up above overlaps the previous grid's tail under programmatic
  // dependent launch; everything below may read its results
  grid_dep_wait();
  grid_dep_launch_dependents();
  // a CTA of a node that the device-side refinement left out does nothing
  // (uniform per CTA)
  const bool skip = geo.active && !geo.active[geo.split > 0 && e >= geo.split ? e - geo.split : e];

  if (skip) {
  } else if (warp == 0) {
    if (lane == 0) {
      const bool hi = geo.split > 0 && e >= geo.split;
      const int ay = (hi ? geo.a_row0_hi + (e - geo.split) * geo.a_batch : geo.a_row0 + e * geo.a_batch) + tm * kBlockM;
      const int by = geo.b_row0 + e * geo.b_batch + tn * BN;
      int issued = 0;
      for (int kb = 0; kb < geo.nk; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        if (kb >= kStages && !mbar_wait(&empty[s], ph ^ 1, status, abort_flag)) break;
        mbar_arrive_expect_tx(&full[s], S::kStageBytes);
        constexpr int kElems = KIND == 1 ? 2 * kBlockK : kBlockK;   // map elements (32 bit for KIND 2) per row
        tma_load_2d(sA + s * kATileBytes, &tmA, &full[s], kb * kElems, ay);
        tma_load_2d(sB + s * S::kBTileBytes, &tmB, &full[s], kb * kElems, by);
        issued = kb + 1;
      }
      if (*abort_flag) {
        // drain: wait (bounded) for the last load issued into every stage
        for (int kb = issued - kStages < 0 ? 0 : issued - kStages; kb < issued; ++kb) {
          for (long long it = 0; it < kWaitLimit; ++it)
            if (mbar_try_wait(&full[kb % kStages], (kb / kStages) & 1)) break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = KIND == 0 ? idesc_tf32(kBlockM, BN) : idesc_bf16(kBlockM, BN);
      static_assert(KIND >= 0 && KIND <= 2, "operand kind");
      for (int kb = 0; kb < geo.nk; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        if (!mbar_wait(&full[s], ph, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA + s * kATileBytes);
        const uint32_t b0 = smem_u32(sB + s * S::kBTileBytes);
        if constexpr (KIND == 2) {
          // (A byte offset, B byte offset) of the six 32-byte K steps:
          // hi x hi, hi x lo, lo x hi over both halves of the 32 columns
#pragma unroll
          for (int t = 0; t < 6; ++t) {
            const uint32_t ao = (t >= 4 ? 64u : 0u) + (t & 1) * 32u;
            const uint32_t bo = (t >= 2 && t < 4 ? 64u : 0u) + (t & 1) * 32u;
            mma_bf16(tmem, sdesc_sw128(a0 + ao), sdesc_sw128(b0 + bo), idesc, (kb | t) != 0);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // four 32-byte K steps per 128-byte row
            if constexpr (KIND == 0)
              mma_tf32(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, (kb | kk) != 0);
            else
              mma_bf16(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc, (kb | kk) != 0);
          }
        }
        mma_commit(&empty[s]);
      }
      // always signal: the epilogue (and the TMEM release) wait for every
      // issued MMA to finish, also on the abort path
      mma_commit(tfull);
    }
  } else {
    const int q = warp % 4;
    const int row = q * 32 + lane;
    if constexpr (EpiExtra<Epi>::kBytes > 0)
      epi.prologue(e, tm, tn, static_cast<int>(threadIdx.x) - 64, smem + S::kPipeBytes + 1024, status, abort_flag);
    if constexpr (EpiPre<Epi>::kHas) {
      typename Epi::Pre pre;
      epi.prefetch(e, tm, tn, row, pre);
      mbar_wait(tfull, 0, status, abort_flag);
      tc_fence_after();
      epilogue_sync();   // uniform abort decision, as below
      if (!*abort_flag)
        epi(e, tm, tn, row, tmem + (static_cast<uint32_t>(q * 32) << 16), static_cast<int>(threadIdx.x) - 64, smem,
            pre);
    } else {
    mbar_wait(tfull, 0, status, abort_flag);
    tc_fence_after();
    // one decision for the whole epilogue group: a thread that gave up set
    // the flag before this barrier, so all 128 threads read the same value
    epilogue_sync();
    if constexpr (EpiExtra<Epi>::kBytes > 0) {
      // run() also waits (bounded) for the prologue's copies and checks the
      // abort flag itself, so that no copy is left in flight on abort
      epi.run(e, tm, tn, row, tmem + (static_cast<uint32_t>(q * 32) << 16), static_cast<int>(threadIdx.x) - 64,
              smem, smem + S::kPipeBytes + 1024, status, abort_flag);
    } else if (!*abort_flag) {
      epi(e, tm, tn, row, tmem + (static_cast<uint32_t>(q * 32) << 16), static_cast<int>(threadIdx.x) - 64, smem);
    }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, S::kTmemCols);
  }
}


// ---------------------------------------------------------------------------
// Batched complex TF32 GEMM on row-split fp32 blocks (real parts of a row,
// then its imaginary parts):
//   C_b (M x N complex) = U_b V_b^T,   C[i, j] = sum_k U[i, k] V[j, k],
// with U and V each given by two 3-D tensor maps (real and imaginary part;
// x: column k of the block, y: row, z: batch plane) whose extents end at the
// block, so that TMA fills the ragged edges of every tile with zeros.  Per
// K-block the four parts are staged in 128-byte-swizzled shared memory and
// one thread issues four tcgen05.mma.kind::tf32 per 8-wide K step into three
// TMEM accumulators
//   rr = Ur Vr^T,   ii = Ui Vi^T,   ri = Ur Vi^T + Ui Vr^T,
// so that C = (rr - ii) + i ri (no embedded copy of either operand).  The
// operands are fp32 in memory; the four epilogue warps, idle during the main
// loop, round each staged K-block to TF32 (nearest) in shared memory before
// the MMA reads it -- the tensor cores would otherwise drop the low mantissa
// bits, a biased error that adds up coherently over a long K.  Warp roles,
// bounded waits and the TMEM release on abort as in k_tc_gemm; the epilogue
// is epi(b, tm, tn, row, lane_taddr) and reads C through cload16.
template <int BN, int STAGES>
struct CSmem {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "complex tile width");
  static constexpr int kUBytes = kBlockM * kBlockK * 4;   // 16 KB per part
  static constexpr int kVBytes = BN * kBlockK * 4;
  static constexpr int kStageBytes = 2 * kUBytes + 2 * kVBytes;
  static constexpr int kTmemCols = 3 * BN <= 64 ? 64 : (3 * BN <= 128 ? 128 : (3 * BN <= 256 ? 256 : 512));
  static constexpr size_t kPipeBytes = (size_t)STAGES * kStageBytes;
  static constexpr size_t kBytes = 1024 /*align slack*/ + kPipeBytes + 256;
};

// CTA (tn, tm, b) reads U rows tm*128.. at plane b*uz_mul + uz_add and V rows
// tn*BN.. at plane b*vz_mul + vz_add, nk K-blocks of 32 columns.
struct CGeom {
  int nk;
  int uz_mul, uz_add;
  int vz_mul, vz_add;
};

// C[i, tn*BN + c0 + t] (t < 16) of this thread's row: real and imaginary parts.
template <int BN>
__device__ __forceinline__ void cload16(uint32_t taddr, int c0, float* re, float* im) {
  float ii[16];
  tmem_ld16(taddr + c0, re);
  tmem_ld16(taddr + BN + c0, ii);
  tmem_ld16(taddr + 2 * BN + c0, im);
#pragma unroll
  for (int t = 0; t < 16; ++t) re[t] -= ii[t];
}

template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(kThreads)
    k_cgemm(const __grid_constant__ CUtensorMap mUr, const __grid_constant__ CUtensorMap mUi,
            const __grid_constant__ CUtensorMap mVr, const __grid_constant__ CUtensorMap mVi, CGeom geo,
            const __grid_constant__ Epi epi, int* status) {
  using S = CSmem<BN, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kPipeBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* rounded = empty + STAGES;   // stage rounded to TF32 (128 arrivals)
  uint64_t* tfull = rounded + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfull + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int b = blockIdx.z, tm = blockIdx.y, tn = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&rounded[s], 4 * 32);
    }
    mbar_init(tfull, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, S::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const int uz = b * geo.uz_mul + geo.uz_add, vz = b * geo.vz_mul + geo.vz_add;
      int issued = 0;
      for (int kb = 0; kb < geo.nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1, status, abort_flag)) break;
        uint8_t* st = smem + (size_t)s * S::kStageBytes;
        mbar_arrive_expect_tx(&full[s], S::kStageBytes);
        tma_load_3d(st, &mUr, &full[s], kb * kBlockK, tm * kBlockM, uz);
        tma_load_3d(st + S::kUBytes, &mUi, &full[s], kb * kBlockK, tm * kBlockM, uz);
        tma_load_3d(st + 2 * S::kUBytes, &mVr, &full[s], kb * kBlockK, tn * BN, vz);
        tma_load_3d(st + 2 * S::kUBytes + S::kVBytes, &mVi, &full[s], kb * kBlockK, tn * BN, vz);
        issued = kb + 1;
      }
      if (*abort_flag) {
        // drain: wait (bounded) for the last load issued into every stage
        for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
          for (long long it = 0; it < kWaitLimit; ++it)
            if (mbar_try_wait(&full[kb % STAGES], (kb / STAGES) & 1)) break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kBlockM, BN);
      for (int kb = 0; kb < geo.nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(&rounded[s], ph, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t ur = smem_u32(smem + (size_t)s * S::kStageBytes);
        const uint32_t ui = ur + S::kUBytes;
        const uint32_t vr = ur + 2 * S::kUBytes;
        const uint32_t vi = vr + S::kVBytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {   // four 32-byte K steps per 128-byte row
          const uint32_t acc = (kb | kk) != 0;
          const uint32_t o = kk * 32;
          mma_tf32(tmem, sdesc_sw128(ur + o), sdesc_sw128(vr + o), idesc, acc);
          mma_tf32(tmem + BN, sdesc_sw128(ui + o), sdesc_sw128(vi + o), idesc, acc);
          mma_tf32(tmem + 2 * BN, sdesc_sw128(ur + o), sdesc_sw128(vi + o), idesc, acc);
          mma_tf32(tmem + 2 * BN, sdesc_sw128(ui + o), sdesc_sw128(vr + o), idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      // always signal: the epilogue (and the TMEM release) wait for every
      // issued MMA to finish, also on the abort path
      mma_commit(tfull);
    }
  } else {
    const int q = warp % 4;
    const int row = q * 32 + lane;
    const int et = static_cast<int>(threadIdx.x) - 64;   // 0..127
    // round every staged K-block to TF32 in place, then release it to the MMA
    for (int kb = 0; kb < geo.nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full[s], (kb / STAGES) & 1, status, abort_flag)) break;
      float4* st = reinterpret_cast<float4*>(smem + (size_t)s * S::kStageBytes);
#pragma unroll 4
      for (int x = et; x < S::kStageBytes / 16; x += 128) {
        float4 v = st[x];
        v.x = to_tf32(v.x);
        v.y = to_tf32(v.y);
        v.z = to_tf32(v.z);
        v.w = to_tf32(v.w);
        st[x] = v;
      }
      fence_proxy_async_smem();   // generic-proxy writes -> the tensor cores' reads
      mbar_arrive(&rounded[s]);
    }
    mbar_wait(tfull, 0, status, abort_flag);
    tc_fence_after();
    epilogue_sync();   // one abort decision for the whole epilogue group
    if (!*abort_flag) epi(b, tm, tn, row, tmem + (static_cast<uint32_t>(q * 32) << 16));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, S::kTmemCols);
  }
}

}  // namespace tc
}  // namespace feast
