// Device-side helpers: inline PTX for mbarrier, TMA and tcgen05 (sm_103a), bounded
// waits, and the small integer routines shared by several kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace ozk2 {

// Range checks of the debug build (compiled with -DOZK2_DEBUG): a failed check sets
// kFlagDebug in the call's flag word (ozk2_device_status reports OZK2_ERR_INTERNAL); it
// never traps, so the kernel runs to its end either way.
#ifdef OZK2_DEBUG
#define OZK2_DCHECK(cond, flags)                    \
  do {                                              \
    if (!(cond)) atomicOr((flags), ozk2::kFlagDebug); \
  } while (0)
#else
#define OZK2_DCHECK(cond, flags) \
  do {                           \
  } while (0)
#endif

// Default limit of a device wait in nanoseconds (the host may set another per launch);
// a wait that reaches its limit makes the kernel record kFlagTimeout and return instead
// of hanging.  The waits of an aborting kernel for its own copies and products in
// flight always use this default.
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with the given parity to complete.  Returns false if
// the CTA-wide abort flag is raised or more than limit_ns nanoseconds pass.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31u) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, FP8 E4M3 x E4M3 -> FP32, one 128 x N x 32 step.
__device__ __forceinline__ void mma_fp8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}
// Each lane reads 32 consecutive 32-bit columns of its TMEM lane.
__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// Each lane reads 16 consecutive 32-bit columns of its TMEM lane.
__device__ __forceinline__ void tmem_ld_16cols(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
template <int W>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[W]) {
  static_assert(W == 16 || W == 32, "16 or 32 columns");
  if constexpr (W == 16) tmem_ld_16cols(taddr, r);
  else tmem_ld_32cols(taddr, r);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major tile written by TMA with 128-byte
// swizzling: rows of 128 bytes, 8-row core groups 1024 bytes apart (SBO), start
// address in 16-byte units, descriptor version 1, layout SWIZZLE_128B (= 2).
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1u) << 16;            // LBO (unused for swizzled K-major)
  d |= static_cast<uint64_t>(1024u >> 4) << 32;    // SBO
  d |= static_cast<uint64_t>(1u) << 46;            // version
  d |= static_cast<uint64_t>(2u) << 61;            // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3, both K-major.
__host__ __device__ constexpr uint32_t fp8_idesc(int M, int N) {
  return (1u << 4)                                   // D format F32
         | (0u << 7) | (0u << 10)                    // A, B format E4M3
         | (static_cast<uint32_t>(N >> 3) << 17)     // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);    // M / 16
}

// ---------------------------------------------------------------- grouped launches
// Problem of virtual block b of grouped launch w: the last p with first_block[w] <= b.
__device__ __forceinline__ int batch_problem(const BatchProblem* __restrict__ probs, int count, int w, int64_t b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].first_block[w] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// A grouped launch w over `total` virtual blocks (problem p owns the virtual blocks
// [first_block[w], first_block[w] + nblocks[w])).  Each physical block serves one
// contiguous range of virtual blocks in order: one binary search finds its first
// problem, and it steps to the following ones, so that the per-block cost of finding a
// problem is paid once per physical block.  fn(P, v) runs for each virtual block, v its
// index within problem P; every thread of the block makes the same calls.
template <class F>
__device__ __forceinline__ void for_each_vblock(const BatchProblem* __restrict__ probs, int count, int w,
                                                int64_t total, F&& fn) {
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  int64_t v = static_cast<int64_t>(blockIdx.x) * per;
  const int64_t end = v + per < total ? v + per : total;
  if (v >= end) return;
  int p = batch_problem(probs, count, w, v);
  int64_t first = probs[p].first_block[w];
  int64_t next = p + 1 < count ? probs[p + 1].first_block[w] : total;
  for (; v < end; ++v) {
    while (v >= next) {
      ++p;
      first = next;
      next = p + 1 < count ? probs[p + 1].first_block[w] : total;
    }
    fn(probs[p], v - first);
  }
}

// ---------------------------------------------------------------- integers
// q = a / b, r = a % b for a >= 0 and b > 0: an unsigned 32-bit division when a fits,
// which is several times cheaper than the 64-bit one.
__device__ __forceinline__ void divmod_nonneg(int64_t a, int b, int& q, int& r) {
  if (a <= 0x7FFFFFFFll) {
    const uint32_t ua = static_cast<uint32_t>(a), ub = static_cast<uint32_t>(b);
    const uint32_t uq = ua / ub;
    q = static_cast<int>(uq);
    r = static_cast<int>(ua - uq * ub);
  } else {
    q = static_cast<int>(a / b);
    r = static_cast<int>(a - static_cast<int64_t>(q) * b);
  }
}
// Normalise a value in [-2h, 2(p-1-h)] (a sum of two symmetric residues).
__device__ __forceinline__ int smod_small(int x, int p, int h) {
  x = (x > p - 1 - h) ? x - p : x;
  x = (x < -h) ? x + p : x;
  return x;
}

}  // namespace ozk2
