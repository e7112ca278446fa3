// FP8 tensor-core products of the method on tcgen05 (sm_103a): one persistent kernel,
// three epilogues.
//
//   residue : C'_l = mod(A'_l B'_l, p_l) for an output tile, from digit-plane products
//             held in TMEM and reduced mod p in registers:
//               square p = s^2 : X = A1 B2 + A2 B1 (one accumulator), Z = A2 B2,
//                                C'_l = mod(s X + Z, p)           [Eq. 3matmult-notKaratsuba]
//               Karatsuba      : Dx = Ax Bx, x = 1, 2, 3,
//                                256 D1 + D2 + 16 (D3 - D1 - D2) = 16 (15 D1 - D2 + D3) + D2
//                                                                  [Eq. C'-Karatsuba]
//             Every FP32 accumulator is an exact integer of magnitude <= 2^24
//             (Eq. error-free-FP8-matmult): a Karatsuba product over at most 2^16
//             terms of digits |d| <= 16, or the shared square accumulator over at most
//             2^15.  Longer reductions run in blocks whose residues are added mod p.
//   bound   : Cbar = RU((1 + k 2^-24) Abar Bbar) folded into row / column maxima
//             (Eq. barCupper); Cbar itself is never stored.
//   raw     : D = A B^T in FP32 (a parity hook for the tensor-core path).
//
// Tiles are 128 x 256 (M x N); TMEM holds two 256-column FP32 accumulator slots (the
// whole 512 columns).  A unit (one tile of one modulus) is a sequence of passes over
// the k-block:
//   square p = s^2 : one pass over BOTH slots, the products interleaved per k-step,
//                    X = A1 B2 + A2 B1 -> slot 0, Z = A2 B2 -> slot 1 (A2 and B2 are
//                    loaded while still in L2), C'_l = mod(s X + Z, p);
//   Karatsuba      : three passes over ONE slot each, alternating slots, so the
//                    epilogue drains one slot while the tensor cores fill the other:
//                    D1, park d1 = mod(D1, p); D2, park v = mod(240 d1 - 15 D2, p);
//                    D3, C'_l = mod(v + 16 D3, p)  (256 D1 + D2 + 16 (D3 - D1 - D2)
//                    = 240 D1 - 15 D2 + 16 D3; every operand of mod is below 2^28).
// Parked values are int16 pairs in the epilogue threads' registers (every pass of a
// unit gives a thread the same row and columns).  The bound and raw products are one single-slot pass per unit.  The wide tile halves the
// operand bytes each SM pulls per flop compared with 128 x 128.
//
// Roles (320 threads for single problems, 576 for grouped launches; one persistent CTA
// per SM):
//   warp 0      TMA producer: 128-row A and 256-row B^T boxes of 128 bytes along K
//               (K-major, 128-byte swizzle, zero fill past m, n, k) into a 4-stage
//               ring of 48 KiB stages, mbarrier complete_tx.
//   warp 1      TMEM allocation and the single MMA-issuing thread:
//               tcgen05.mma.cta_group::1.kind::f8f6f4, M = 128, N = 256, K = 32; a pass
//               starts once the epilogue has released the slot(s) it writes.
//   warps 2-9   epilogue (warps 2-17 in grouped launches): warp w reads TMEM lane
//               quadrant w % 4, column half (quarter) (w - 2) / 4, with tcgen05.ld;
//               FP32 math; global stores.
// Every wait is bounded (device.cuh; the limit is a launch parameter); a wait that gives
// up raises a CTA-wide abort flag and the global timeout flag, drains the copies and
// products this CTA has in flight, frees TMEM and returns.  Operands are read only with
// plain (non-multicast) TMA loads of this CTA's own tiles.
#include <cstring>

#include "device.cuh"

namespace ozk2 {
namespace {

constexpr int BM = 128;
constexpr int BK = 128;  // bytes = FP8 elements per k-step (one 128-byte swizzle row)
constexpr int kATileBytes = BM * BK;  // 16 KiB
// Epilogue warps: 8 for single problems, 16 for grouped launches.  Short reductions in
// batches of small problems leave the tensor cores waiting for the epilogue (about 40%
// of the MMA thread's time with 8 warps on the 512-product batch); twice the warps hide
// more of its TMEM-load and store latency there (batch 14.8 -> 13.7 ms), while for
// single problems the extra warps slowed the MMA and TMA threads that share their
// schedulers (8192 x 8192 x 2048: 4.29 -> 4.53 ms).
template <bool GROUPED>
struct Epi {
  static constexpr int kWarps = GROUPED ? 16 : 8;
  static constexpr int kColGroups = kWarps / 4;  // epilogue warps per TMEM lane quadrant
  static constexpr int kThreads = 64 + 32 * kWarps;
  static constexpr int kCW = GROUPED ? 16 : 32;  // columns per TMEM load of the residue epilogue
};
constexpr int kChunkKaratsuba = 65536;  // 2^16 * 16 * 16 = 2^24
constexpr int kChunkSquare = 32768;     // shared accumulator: 2 * 2^15 * 16 * 16 = 2^24
constexpr int kGroupM = 16;             // tile rasterisation: bands of 16 tile rows (2048 rows of A)

// Tile shapes: 128 x 256 (the default) or 128 x 128 (narrow or ragged products, where a
// 256-wide tile would spend much of its tensor work on padding).  Both keep two TMEM
// accumulator slots of TN columns and fill about 192 KiB of shared memory with stages.
template <int TN>
struct Tile {
  static_assert(TN == 256 || TN == 128, "tile widths 256 and 128");
  static constexpr int kStages = TN == 256 ? 4 : 6;
  static constexpr int kBTileBytes = TN * BK;
  static constexpr int kStageBytes = kATileBytes + kBTileBytes;
  static constexpr uint32_t kTmemCols = 2 * TN;
  static constexpr size_t kSmemBytes = 1024 + static_cast<size_t>(kStages) * kStageBytes + 256;
};

struct EpiMod {
  int p[kMaxModuli];
  int half[kMaxModuli];
  int s[kMaxModuli];
  float inv_p[kMaxModuli];
};

struct GemmParams {
  int mode;
  int m, n, k;
  int tiles_m, tiles_n, tiles;
  int num_units;
  int16_t* cres;
  int64_t ldr;
  int64_t res_stride;
  EpiMod mod;
  float factor;
  float* R;
  float* S;
  float* D;
  int64_t ldd;
  uint32_t* flags;
  // bound mode: cbar_ij is also scaled by 2^-colshift_j and 2^-rowshift_i before the
  // maxima (each may be null; values clamped to [-126, 126], below that kFlagRange)
  const int32_t* colshift;
  const int32_t* rowshift;
  unsigned long long wait_ns;  // limit of every device wait (the drains of an abort use the default)
  int stall;                   // fault injection: the MMA thread's first wait never completes
  int split_squares;           // single problems: square moduli in two single-slot passes
};

__device__ __forceinline__ void decode_unit(int tiles_m, int tiles_n, int tiles, int u, int& mod, int& tm,
                                            int& tn) {
  mod = u / tiles;
  const int t = u - mod * tiles;
  const int per_group = kGroupM * tiles_n;
  const int g = t / per_group;
  const int first_m = g * kGroupM;
  const int gsz = min(tiles_m - first_m, kGroupM);
  const int r = t - g * per_group;
  tm = first_m + r % gsz;
  tn = r / gsz;
}

// Everything a role needs about one unit (a tile of one modulus of one problem).  A
// role walks its units in increasing order and keeps one UnitCtx across them: in a
// grouped launch the problem's fields are reloaded only when the problem changes.
struct UnitCtx {
  const CUtensorMap* ta;
  const CUtensorMap* tb;
  int m, n, k;
  int mod, tm, tn;
  int prob = -1;  // grouped: problem of the fields below (-1: none yet)
  int tiles_m, tiles_n, tiles;
  int64_t unit_start, next_start;  // grouped: units [unit_start, next_start) are this problem's
  int16_t* cres;
  int64_t ldr, res_stride;
  float factor;
  float* R;
  float* S;
  bool split;  // square moduli in two single-slot passes
};

template <bool GROUPED>
__device__ __forceinline__ void resolve_unit(const GemmParams& P, const CUtensorMap* tmA, const CUtensorMap* tmB,
                                             const GemmProblem* __restrict__ probs, int nprobs, int u, UnitCtx& c) {
  if constexpr (!GROUPED) {
    c.ta = tmA;
    c.tb = tmB;
    c.m = P.m;
    c.n = P.n;
    c.k = P.k;
    c.prob = 0;
    decode_unit(P.tiles_m, P.tiles_n, P.tiles, u, c.mod, c.tm, c.tn);
    c.cres = P.cres;
    c.ldr = P.ldr;
    c.res_stride = P.res_stride;
    c.factor = P.factor;
    c.R = P.R;
    c.S = P.S;
    c.split = P.split_squares != 0;
  } else {
    if (c.prob < 0 || u >= c.next_start) {
      // the last problem starting at or before u, searched above the current one
      int lo = c.prob < 0 ? 0 : c.prob + 1, hi = nprobs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].unit_start <= u) lo = mid;
        else hi = mid - 1;
      }
      const GemmProblem& G = probs[lo];
      c.ta = &G.ta;
      c.tb = &G.tb;
      c.m = G.m;
      c.n = G.n;
      c.k = G.k;
      c.prob = lo;
      c.tiles_m = G.tiles_m;
      c.tiles_n = G.tiles_n;
      c.tiles = G.tiles;
      c.unit_start = G.unit_start;
      c.next_start = lo + 1 < nprobs ? probs[lo + 1].unit_start : 0x7FFFFFFFFFFFFFFFll;
      c.cres = G.cres;
      c.ldr = G.ldr;
      c.res_stride = G.res_stride;
      c.factor = G.factor;
      c.R = G.R;
      c.S = G.S;
      c.split = G.split != 0;
    }
    decode_unit(c.tiles_m, c.tiles_n, c.tiles, static_cast<int>(u - c.unit_start), c.mod, c.tm, c.tn);
  }
}

// Tensor maps written to global memory before the launch: order the tensormap proxy's
// reads of this map after the generic writes.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// Pass structure of a unit.
struct UnitPlan {
  int chunk_len;  // k per exactness block
  int nchunks;
  int npasses;    // passes per block
};

// split: a square modulus runs as two single-slot passes, X = A1 B2 + A2 B1 (its residue
// parked) and then Z = A2 B2, instead of one pass over both slots; chosen for short
// reductions, where the drain of both slots after a pair pass would leave the tensor
// cores idle.
template <int MODE>
__device__ __forceinline__ UnitPlan plan_of(int k, int mod, bool split) {
  UnitPlan u;
  if (MODE == kModeResidue) {
    const bool square = mod < kNumSquares;
    u.chunk_len = square ? kChunkSquare : kChunkKaratsuba;
    u.npasses = square ? (split ? 2 : 1) : 3;
  } else {
    u.chunk_len = ((k + BK - 1) / BK) * BK;
    u.npasses = 1;
  }
  u.nchunks = (k + u.chunk_len - 1) / u.chunk_len;
  return u;
}

// A pass uses both slots (a square modulus in one pass) or one.
template <int MODE>
__device__ __forceinline__ bool pair_pass(int mod, bool split) {
  return MODE == kModeResidue && mod < kNumSquares && !split;
}

// Products of one pass per k-step, the digit planes (pa, pb) of product x and the
// accumulator (0: the pass's first slot, 1: slot 1 of a pair pass) it adds to.
template <int MODE>
__device__ __forceinline__ int num_products(int mod, int pass, bool split) {
  if (pair_pass<MODE>(mod, split)) return 3;
  if (MODE == kModeResidue && mod < kNumSquares) return pass == 0 ? 2 : 1;  // split square: X, then Z
  return 1;
}

template <int MODE>
__device__ __forceinline__ void product_of(int mod, int pass, int x, bool split, int& pa, int& pb, int& acc) {
  if (MODE != kModeResidue) {
    pa = pb = 0;
    acc = 0;
  } else if (mod < kNumSquares) {
    const int a0 = 2 * mod;  // (A1, B2) -> X, (A2, B1) -> X, (A2, B2) -> Z
    const int xs = split ? (pass == 0 ? x : 2) : x;
    pa = (xs == 0) ? a0 : a0 + 1;
    pb = (xs == 1) ? a0 : a0 + 1;
    acc = (!split && xs == 2) ? 1 : 0;
  } else {
    pa = pb = 2 * kNumSquares + 3 * (mod - kNumSquares) + pass;  // (Ax, Bx) -> Dx
    acc = 0;
  }
}

// Slot bookkeeping shared by the MMA thread and the epilogue, which walk the same pass
// sequence: a single-slot pass takes slot `next` and flips it; a pair pass takes both
// (X in slot 0, Z in slot 1).  uses[j] counts the passes that used slot j before.
struct Slots {
  uint32_t u0 = 0u, u1 = 0u;  // passes that used slot 0 / slot 1
  uint32_t next = 0u;
  __device__ __forceinline__ uint32_t uses(uint32_t j) const { return j ? u1 : u0; }
  __device__ __forceinline__ void bump(uint32_t j) {
    u0 += (j == 0u) ? 1u : 0u;
    u1 += (j == 1u) ? 1u : 0u;
  }
};

// Lane l of the warp ends with the maximum of column l over the 32 lanes.
__device__ __forceinline__ float warp_column_max(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? v[i] : v[i + off];
      const float keep = upper ? v[i + off] : v[i];
      const float got = __shfl_xor_sync(0xffffffffu, send, off);
      v[i] = fmaxf(keep, got);
    }
  }
  return v[0];
}

// The residue epilogue works on pairs of accumulator columns with packed two-wide FP32
// instructions (__ffma2_rn / __fadd2_rn / __fmul2_rn round each component like the
// scalar forms), so its results are those of the element-at-a-time arithmetic below.
constexpr float kMagic = 12582912.0f;  // 1.5 2^23: y + kMagic rounds y to an integer
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 bits2(uint32_t a, uint32_t b) { return make_float2(__uint_as_float(a), __uint_as_float(b)); }

// Per-modulus constants of the epilogue, as pairs.
struct ModPair {
  float2 neg_p, inv_p;
  bool is1024;  // p = 1024, the even modulus: the last step rounds (r + 1/2) / p
};

// x - p q for exact-integer floats |x| <= 2^24, q = RN(x RN(1/p)): x RN(1/p) is within
// 0.003 of x / p for p >= 443, so the remainder, formed exactly by one FMA, lies in
// (-0.51 p, 0.51 p) and is congruent to x.
__device__ __forceinline__ float2 mod_near2(float2 x, const ModPair& m) {
  const float2 q = __fadd2_rn(__ffma2_rn(x, m.inv_p, dup2(kMagic)), dup2(-kMagic));
  return __ffma2_rn(m.neg_p, q, x);
}
// The symmetric remainder, in [-h, p - 1 - h], of exact-integer floats |y| < 2^23: for odd
// p the rounded quotient is then the nearest integer to y / p (never a tie), for p = 1024
// q = RN((y + 1/2) / 1024) = floor((y + 512) / 1024) (the product and sum are exact for
// |y| < 2^12, which holds wherever this form is used: after a first reduction).
__device__ __forceinline__ float2 smod_small2(float2 y, const ModPair& m) {
  if (m.is1024) {
    const float2 t = __ffma2_rn(y, m.inv_p, dup2(0.00048828125f));  // (y + 1/2) / 1024, exact
    const float2 q = __fadd2_rn(__fadd2_rn(t, dup2(kMagic)), dup2(-kMagic));
    return __ffma2_rn(m.neg_p, q, y);
  }
  return mod_near2(y, m);
}
// The symmetric remainder of exact-integer floats |x| <= 2^24: a first reduction to
// |r| < 0.51 p, then the exact one.
__device__ __forceinline__ float2 smod2(float2 x, const ModPair& m) { return smod_small2(mod_near2(x, m), m); }

// Two exact-integer floats |r| < 2^15 as two int16 of one word (first in the low half):
// the low 16 bits of r + 1.5 2^23 are r in two's complement.
__device__ __forceinline__ uint32_t pack2(float2 r) {
  const float2 b = __fadd2_rn(r, dup2(kMagic));
  return __byte_perm(__float_as_uint(b.x), __float_as_uint(b.y), 0x5410);
}
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  return make_float2(static_cast<float>(static_cast<int16_t>(w & 0xFFFFu)), static_cast<float>(static_cast<int16_t>(w >> 16)));
}

// Store 8 int16 residues of one row at columns gc .. gc + 7, packed two per word (adding
// the previous block's residues when `accumulate`), as one 16-byte store when the 8
// columns are all inside the matrix.  The debug build checks that every residue lies in
// the symmetric range [-h, p - 1 - h].
__device__ __forceinline__ void store_residues8(int16_t* dst, int gc, int n, uint32_t (&pk)[4], bool accumulate,
                                                int p, int h, uint32_t* flags) {
  if (accumulate) {
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int j = gc + 2 * z;
      const int a = smod_small(static_cast<int16_t>(pk[z] & 0xFFFFu) + (j < n ? dst[j] : 0), p, h);
      const int b = smod_small(static_cast<int16_t>(pk[z] >> 16) + (j + 1 < n ? dst[j + 1] : 0), p, h);
      pk[z] = (static_cast<uint32_t>(a) & 0xFFFFu) | (static_cast<uint32_t>(b) << 16);
    }
  }
#ifdef OZK2_DEBUG
  bool in_range = true;
#pragma unroll
  for (int z = 0; z < 4; ++z) {
    const int a = static_cast<int16_t>(pk[z] & 0xFFFFu), b = static_cast<int16_t>(pk[z] >> 16);
    in_range = in_range && a >= -h && a <= p - 1 - h && b >= -h && b <= p - 1 - h;
  }
  OZK2_DCHECK(in_range, flags);
#else
  (void)flags;
#endif
  if (gc + 8 <= n) {
    *reinterpret_cast<uint4*>(dst + gc) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (gc + j < n) dst[gc + j] = static_cast<int16_t>((j & 1) ? (pk[j >> 1] >> 16) : (pk[j >> 1] & 0xFFFFu));
  }
}

// GROUPED: the units of all `nprobs` problems of `probs` (tmA, tmB unused).  TN: tile width.
template <int MODE, bool GROUPED, int TN>
__global__ void __launch_bounds__(Epi<GROUPED>::kThreads, 1)
    fp8_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ GemmParams prm, const GemmProblem* __restrict__ probs, int nprobs) {
  constexpr int BN = TN;
  constexpr int kStages = Tile<TN>::kStages;
  constexpr int kStageBytes = Tile<TN>::kStageBytes;
  constexpr uint32_t kTmemCols = Tile<TN>::kTmemCols;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tiles = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;  // [2]: slot filled by the tensor cores
  uint64_t* tempty = tfull + 2;       // [2]: slot drained by the epilogue
  uint64_t* done = tempty + 2;
  uint64_t* never = done + 1;  // nothing arrives here (the injected stall waits on it)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int u_first = static_cast<int>(blockIdx.x);
  const int u_step = static_cast<int>(gridDim.x);
  const unsigned long long wait_ns = prm.wait_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(tfull + j, 1);
      mbar_init(tempty + j, 32 * Epi<GROUPED>::kWarps);
    }
    mbar_init(done, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (!GROUPED && warp == 0 && lane == 0) {
    tma_prefetch_map(&tmA);
    tma_prefetch_map(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0, issued_phase = 0;
      bool ok = true;
      int last_prob = -1;
      UnitCtx uc;
      for (int u = u_first; ok && u < prm.num_units; u += u_step) {
        resolve_unit<GROUPED>(prm, &tmA, &tmB, probs, nprobs, u, uc);
        if (GROUPED && uc.prob != last_prob) {
          tensormap_acquire(uc.ta);
          tensormap_acquire(uc.tb);
          last_prob = uc.prob;
        }
        const int mod = uc.mod;
        const UnitPlan up = plan_of<MODE>(uc.k, mod, uc.split);
        for (int c = 0; ok && c < up.nchunks; ++c) {
          const int k0 = c * up.chunk_len;
          const int ksteps = (min(uc.k, k0 + up.chunk_len) - k0 + BK - 1) / BK;
          for (int ps = 0; ok && ps < up.npasses; ++ps) {
            const int np = num_products<MODE>(mod, ps, uc.split);
            for (int s = 0; ok && s < ksteps; ++s) {
              for (int x = 0; x < np; ++x) {
                if (!mbar_wait_bounded(empty + stage, phase ^ 1u, abort_flag, wait_ns)) {
                  ok = false;
                  break;
                }
                int pa, pb, acc;
                product_of<MODE>(mod, ps, x, uc.split, pa, pb, acc);
                uint8_t* dst = tiles + stage * kStageBytes;
                mbar_arrive_expect_tx(full + stage, kStageBytes);
                tma_load_3d(dst, uc.ta, full + stage, k0 + s * BK, uc.tm * BM, pa);
                tma_load_3d(dst + kATileBytes, uc.tb, full + stage, k0 + s * BK, uc.tn * BN, pb);
                issued |= 1u << stage;
                issued_phase = (issued_phase & ~(1u << stage)) | (phase << stage);
                if (++stage == kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.flags, kFlagTimeout);
        int no_abort = 0;  // let this thread's copies in flight land before exiting
        for (int s = 0; s < kStages; ++s)
          if (issued & (1u << s)) mbar_wait_bounded(full + s, (issued_phase >> s) & 1u, &no_abort, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = fp8_idesc(BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      Slots sl;
      // an injected stall (fault-injection tests): wait for a barrier nothing arrives at,
      // so this wait runs out and the kernel takes its timeout path
      bool ok = prm.stall ? mbar_wait_bounded(never, 0u, abort_flag, wait_ns) : true;
      UnitCtx uc;
      for (int u = u_first; ok && u < prm.num_units; u += u_step) {
        resolve_unit<GROUPED>(prm, &tmA, &tmB, probs, nprobs, u, uc);
        const int mod = uc.mod;
        const UnitPlan up = plan_of<MODE>(uc.k, mod, uc.split);
        for (int c = 0; ok && c < up.nchunks; ++c) {
          const int k0 = c * up.chunk_len;
          const int ksteps = (min(uc.k, k0 + up.chunk_len) - k0 + BK - 1) / BK;
          for (int ps = 0; ok && ps < up.npasses; ++ps) {
            const bool pair = pair_pass<MODE>(mod, uc.split);
            const uint32_t first_slot = pair ? 0u : sl.next;
            for (uint32_t j = 0; j < 2 && ok; ++j) {
              if (!pair && j != first_slot) continue;
              ok = mbar_wait_bounded(tempty + j, (sl.uses(j) & 1u) ^ 1u, abort_flag, wait_ns);
            }
            if (!ok) break;
            tc_fence_after();
            const int np = num_products<MODE>(mod, ps, uc.split);
            for (int s = 0; ok && s < ksteps; ++s) {
              for (int x = 0; x < np; ++x) {
                if (!mbar_wait_bounded(full + stage, phase, abort_flag, wait_ns)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                int pa, pb, acc;
                product_of<MODE>(mod, ps, x, uc.split, pa, pb, acc);
                const bool first = s == 0 && (pair ? (x == 0 || x == 2) : x == 0);  // first into its slot
                const uint32_t dtm = tmem_base + (first_slot + static_cast<uint32_t>(acc)) * static_cast<uint32_t>(BN);
                const uint32_t sa = smem_addr(tiles + stage * kStageBytes);
                const uint64_t adesc = sw128_kmajor_desc(sa);
                const uint64_t bdesc = sw128_kmajor_desc(sa + kATileBytes);
#pragma unroll
                for (int kk = 0; kk < BK / 32; ++kk)
                  mma_fp8(dtm, adesc + 2ull * kk, bdesc + 2ull * kk, idesc, (first && kk == 0) ? 0u : 1u);
                mma_commit(empty + stage);
                if (++stage == kStages) {
                  stage = 0;
                  phase ^= 1u;
                }
              }
            }
            if (pair) {
              if (ok) {
                mma_commit(tfull + 0);
                mma_commit(tfull + 1);
              }
              sl.bump(0u);
              sl.bump(1u);
            } else {
              if (ok) mma_commit(tfull + first_slot);
              sl.bump(first_slot);
              sl.next ^= 1u;
            }
          }
        }
      }
      mma_commit(done);  // every product issued here completes before TMEM is freed
      int no_abort = 0;
      mbar_wait_bounded(done, 0, &no_abort, kWaitLimitNs);
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.flags, kFlagTimeout);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                 // TMEM lane quadrant this warp may access
    const int cgrp = (warp - 2) >> 2;       // column group of the tile
    constexpr int kCols = BN / Epi<GROUPED>::kColGroups;  // columns of this thread
    constexpr int kCW = Epi<GROUPED>::kCW;
    constexpr int kChunks = kCols / kCW;
    const int row = q * 32 + lane;
    const uint32_t tq = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(cgrp * kCols);
    // Residues kept between the passes of a unit (Karatsuba d1, then v; the X residue of
    // a two-pass square modulus), kCW int16 per chunk of kCW columns, two per word.  Every
    // pass of a unit gives this thread the same row and the same kCols columns, so they
    // stay in registers (the chunk loop unrolled).  An earlier form parked them in a
    // CTA-private scratch tile in L2; its round trips made short reductions up to 14%
    // slower.
    uint32_t park[MODE == kModeResidue ? kChunks : 1][kCW / 2];
    Slots sl;  // the MMA thread's pass sequence, replayed
    bool ok = true;
    UnitCtx uc;
    for (int u = u_first; ok && u < prm.num_units; u += u_step) {
      resolve_unit<GROUPED>(prm, &tmA, &tmB, probs, nprobs, u, uc);
      const int mod = uc.mod, tn = uc.tn;
      const UnitPlan up = plan_of<MODE>(uc.k, mod, uc.split);
      const int gi = uc.tm * BM + row;
      for (int c = 0; ok && c < up.nchunks; ++c) {
        for (int ps = 0; ok && ps < up.npasses; ++ps) {
          const bool pair = pair_pass<MODE>(mod, uc.split);
          const uint32_t slot = pair ? 0u : sl.next;
          for (uint32_t j = 0; j < 2 && ok; ++j) {
            if (!pair && j != slot) continue;
            ok = mbar_wait_bounded(tfull + j, sl.uses(j) & 1u, abort_flag, wait_ns);
          }
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          tc_fence_after();
          const uint32_t ts = tq + slot * static_cast<uint32_t>(BN);
          if constexpr (MODE == kModeResidue) {
            const int p = prm.mod.p[mod], h = prm.mod.half[mod], sq = prm.mod.s[mod];
            const ModPair mp{dup2(-static_cast<float>(p)), dup2(prm.mod.inv_p[mod]), p == 1024};
            const bool last = ps == up.npasses - 1;
            int16_t* dst = uc.cres + static_cast<int64_t>(mod) * uc.res_stride + static_cast<int64_t>(gi) * uc.ldr;
            // one chunk of kCW columns; sp: this thread's kCW parked int16 of the chunk, two per
            // word (registers: every index below is known at compile time)
            auto store4 = [](uint32_t* sp, int w, const uint32_t (&pk)[4]) {
#pragma unroll
              for (int z = 0; z < 4; ++z) sp[4 * w + z] = pk[z];
            };
            auto load4 = [](const uint32_t* sp, int w, uint32_t (&pr)[4]) {
#pragma unroll
              for (int z = 0; z < 4; ++z) pr[z] = sp[4 * w + z];
            };
            // single problems: the pass's slot(s) go back to the MMA thread as soon as the last
            // chunk has been read from TMEM, before that chunk's arithmetic and stores (in the
            // grouped kernel the extra live state made it spill, and the release stays at the
            // end of the pass)
            auto release = [&]() {
              tc_fence_before();
              if (pair) {
                mbar_arrive(tempty + 0);
                mbar_arrive(tempty + 1);
              } else {
                mbar_arrive(tempty + slot);
              }
            };
            auto chunk = [&](int cb, uint32_t* sp) {
              const int gc = tn * BN + cgrp * kCols + cb * kCW;
              const bool keep = gi < uc.m;  // this thread's row is inside the matrix
              if (pair) {  // square modulus: X in slot 0, Z in slot 1
                uint32_t vx[kCW], vz[kCW];
                tmem_ld_cols(tq + cb * kCW, vx);
                tmem_ld_cols(tq + BN + cb * kCW, vz);
                tmem_ld_wait();
                if (!GROUPED && cb == kChunks - 1) release();
                // mod(s X + Z, p): X mod p first keeps s (X mod p) + Z below 2^24 (|X| <= 2^24,
                // |Z| <= 2^23), so every step is exact
#pragma unroll
                for (int w = 0; w < kCW / 8; ++w) {
                  uint32_t pk[4];
#pragma unroll
                  for (int z = 0; z < 4; ++z) {
                    const int j = 8 * w + 2 * z;
                    const float2 xr = mod_near2(bits2(vx[j], vx[j + 1]), mp);
                    const float2 y = __ffma2_rn(dup2(static_cast<float>(sq)), xr, bits2(vz[j], vz[j + 1]));
                    pk[z] = pack2(smod2(y, mp));
                  }
                  if (keep) store_residues8(dst, gc + 8 * w, uc.n, pk, c > 0, p, h, prm.flags);
                }
                return;
              }
              uint32_t v[kCW];
              tmem_ld_cols(ts + cb * kCW, v);
              tmem_ld_wait();
              if (!GROUPED && cb == kChunks - 1) release();
              if (mod < kNumSquares) {  // square modulus in two passes
                if (ps == 0) {  // park x = X mod p (|x| < 0.51 p)
#pragma unroll
                  for (int w = 0; w < kCW / 8; ++w) {
                    uint32_t pk[4];
#pragma unroll
                    for (int z = 0; z < 4; ++z) pk[z] = pack2(mod_near2(bits2(v[8 * w + 2 * z], v[8 * w + 2 * z + 1]), mp));
                    store4(sp, w, pk);
                  }
                  return;
                }
                // C' = mod(s x + Z, p), as the one-pass form computes it
#pragma unroll
                for (int w = 0; w < kCW / 8; ++w) {
                  uint32_t pr[4];
                  load4(sp, w, pr);
                  uint32_t pk[4];
#pragma unroll
                  for (int z = 0; z < 4; ++z) {
                    const int j = 8 * w + 2 * z;
                    const float2 y = __ffma2_rn(dup2(static_cast<float>(sq)), unpack2(pr[z]), bits2(v[j], v[j + 1]));
                    pk[z] = pack2(smod2(y, mp));
                  }
                  if (keep) store_residues8(dst, gc + 8 * w, uc.n, pk, c > 0, p, h, prm.flags);
                }
                return;
              }
              if (ps == 0) {  // Karatsuba pass 1: park d1 = mod(D1, p)
#pragma unroll
                for (int w = 0; w < kCW / 8; ++w) {
                  uint32_t pk[4];
#pragma unroll
                  for (int z = 0; z < 4; ++z) pk[z] = pack2(smod2(bits2(v[8 * w + 2 * z], v[8 * w + 2 * z + 1]), mp));
                  store4(sp, w, pk);
                }
                return;
              }
              if (!last) {  // Karatsuba pass 2: park v = mod(240 d1 - 15 D2, p); D2 mod p first
                            // keeps |240 d1 - 15 (D2 mod p)| below 2^17
#pragma unroll
                for (int w = 0; w < kCW / 8; ++w) {
                  uint32_t pr[4];
                  load4(sp, w, pr);
                  uint32_t pk[4];
#pragma unroll
                  for (int z = 0; z < 4; ++z) {
                    const int j = 8 * w + 2 * z;
                    const float2 d2 = mod_near2(bits2(v[j], v[j + 1]), mp);
                    const float2 y = __ffma2_rn(dup2(-15.0f), d2, __fmul2_rn(dup2(240.0f), unpack2(pr[z])));
                    pk[z] = pack2(smod_small2(y, mp));
                  }
                  store4(sp, w, pk);
                }
                return;
              }
              // Karatsuba pass 3: C' = mod(v + 16 D3, p); D3 mod p first (|v + 16 (D3 mod p)| < 2^14)
#pragma unroll
              for (int w = 0; w < kCW / 8; ++w) {
                uint32_t pr[4];
                load4(sp, w, pr);
                uint32_t pk[4];
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                  const int j = 8 * w + 2 * z;
                  const float2 d3 = mod_near2(bits2(v[j], v[j + 1]), mp);
                  pk[z] = pack2(smod_small2(__ffma2_rn(dup2(16.0f), d3, unpack2(pr[z])), mp));
                }
                if (keep) store_residues8(dst, gc + 8 * w, uc.n, pk, c > 0, p, h, prm.flags);
              }
            };
#pragma unroll
            for (int cb = 0; cb < kChunks; ++cb) chunk(cb, park[cb]);
          } else if constexpr (MODE == kModeBound) {
            float rmax = 0.0f;
            // 2^-s for an integer s clamped to [-126, 126] (an upper bound of 2^-s for
            // every s >= -126; smaller s is out of range and flagged)
            auto pow2_neg = [&](int s) {
              if (s < -126) atomicOr(prm.flags, kFlagRange);
              s = max(-126, min(126, s));
              return __int_as_float((127 - s) << 23);
            };
            const float rscale = (GROUPED || !prm.rowshift || gi >= uc.m) ? 1.0f : pow2_neg(prm.rowshift[gi]);
            const bool cshift = !GROUPED && prm.colshift != nullptr;
#pragma unroll 1
            for (int cb = 0; cb < kCols / 32; ++cb) {
              uint32_t v0[32];
              tmem_ld_32cols(ts + cb * 32, v0);
              tmem_ld_wait();
              const int gc = tn * BN + cgrp * kCols + cb * 32;
              float cv[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                float cj = __fmul_ru(uc.factor, __uint_as_float(v0[j]));
                if (cshift && gc + j < uc.n) cj = __fmul_ru(cj, pow2_neg(prm.colshift[gc + j]));
                if (!GROUPED && prm.rowshift) cj = __fmul_ru(cj, rscale);
                cj = (gi < uc.m && gc + j < uc.n) ? cj : 0.0f;
                rmax = fmaxf(rmax, cj);
                cv[j] = cj;
              }
              const float cm = warp_column_max(cv, lane);
              if (gc + lane < uc.n && cm > 0.0f)
                atomicMax(reinterpret_cast<int*>(uc.S) + gc + lane, __float_as_int(cm));
            }
            if (gi < uc.m && rmax > 0.0f) atomicMax(reinterpret_cast<int*>(uc.R) + gi, __float_as_int(rmax));
          } else {
#pragma unroll 1
            for (int cb = 0; cb < kCols / 32; ++cb) {
              uint32_t v0[32];
              tmem_ld_32cols(ts + cb * 32, v0);
              tmem_ld_wait();
              const int gc = tn * BN + cgrp * kCols + cb * 32;
              if (gi < uc.m) {
                float* o = prm.D + static_cast<int64_t>(gi) * prm.ldd;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (gc + j < uc.n) o[gc + j] = __uint_as_float(v0[j]);
              }
            }
          }
          if constexpr (MODE != kModeResidue || GROUPED) {  // else the epilogue released the slot(s) itself
            tc_fence_before();
            if (pair) {
              mbar_arrive(tempty + 0);
              mbar_arrive(tempty + 1);
            } else {
              mbar_arrive(tempty + slot);
            }
          }
          if (pair) {
            sl.bump(0u);
            sl.bump(1u);
          } else {
            sl.bump(slot);
            sl.next ^= 1u;
          }
        }
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (lane == 0) atomicOr(prm.flags, kFlagTimeout);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

template <int MODE, bool GROUPED, int TN>
cudaError_t launch_mode(const GemmParams& prm, const CUtensorMap& ta, const CUtensorMap& tb, int grid,
                        const GemmProblem* probs, int nprobs, cudaStream_t st) {
  static bool configured[64] = {false};
  constexpr size_t smem = Tile<TN>::kSmemBytes;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    cudaError_t err = cudaFuncSetAttribute(fp8_gemm_kernel<MODE, GROUPED, TN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    configured[dev] = true;
  }
  fp8_gemm_kernel<MODE, GROUPED, TN><<<grid, Epi<GROUPED>::kThreads, smem, st>>>(ta, tb, prm, probs, nprobs);
  return cudaGetLastError();
}

template <int MODE, bool GROUPED>
cudaError_t launch_tile(int tn, const GemmParams& prm, const CUtensorMap& ta, const CUtensorMap& tb, int grid,
                        const GemmProblem* probs, int nprobs, cudaStream_t st) {
  if (tn == 128) return launch_mode<MODE, GROUPED, 128>(prm, ta, tb, grid, probs, nprobs, st);
  return launch_mode<MODE, GROUPED, 256>(prm, ta, tb, grid, probs, nprobs, st);
}

int tile_width(int tile_n) { return tile_n == 128 ? 128 : 256; }

void fill_mod(GemmParams& prm, const ModTable& mt) {
  for (int l = 0; l < mt.N; ++l) {
    prm.mod.p[l] = mt.p[l];
    prm.mod.half[l] = mt.half[l];
    prm.mod.s[l] = mt.s[l];
    prm.mod.inv_p[l] = mt.inv_p[l];
  }
}

}  // namespace

cudaError_t launch_fp8_gemm(const GemmArgs& g, const uint8_t* a, int64_t lda8, int planes_a, const uint8_t* b,
                            int64_t ldb8, int planes_b, cudaStream_t st) {
  GemmParams prm{};
  prm.mode = g.mode;
  prm.m = g.m;
  prm.n = g.n;
  prm.k = g.k;
  const int BN = tile_width(g.tile_n);
  prm.tiles_m = (g.m + BM - 1) / BM;
  prm.tiles_n = (g.n + BN - 1) / BN;
  prm.tiles = prm.tiles_m * prm.tiles_n;
  const int nmod = (g.mode == kModeResidue) ? g.mt->N : 1;
  prm.num_units = prm.tiles * nmod;
  prm.cres = g.cres;
  prm.ldr = g.ldr;
  prm.res_stride = g.res_stride;
  if (g.mode == kModeResidue) fill_mod(prm, *g.mt);
  prm.factor = g.factor;
  prm.R = g.R;
  prm.S = g.S;
  prm.D = g.D;
  prm.ldd = g.ldd;
  prm.flags = g.flags;
  prm.colshift = g.colshift;
  prm.rowshift = g.rowshift;
  prm.wait_ns = g.wait_ns;
  prm.stall = g.stall ? 1 : 0;
  prm.split_squares = g.split_squares ? 1 : 0;

  CUtensorMap ta, tb;
  if (!encode_fp8_map(&ta, a, g.k, g.m, planes_a, lda8, g.plane_stride_a, BM, BK)) return cudaErrorInvalidValue;
  if (!encode_fp8_map(&tb, b, g.k, g.n, planes_b, ldb8, g.plane_stride_b, BN, BK)) return cudaErrorInvalidValue;
  const int ctas = g.num_sms < kMaxGemmCtas ? g.num_sms : kMaxGemmCtas;
  const int grid = prm.num_units < ctas ? prm.num_units : ctas;
  switch (g.mode) {
    case kModeResidue:
      return launch_tile<kModeResidue, false>(BN, prm, ta, tb, grid, nullptr, 0, st);
    case kModeBound:
      return launch_tile<kModeBound, false>(BN, prm, ta, tb, grid, nullptr, 0, st);
    default:
      return launch_tile<kModeRaw, false>(BN, prm, ta, tb, grid, nullptr, 0, st);
  }
}

int64_t fp8_gemm_units(int mode, int m, int n, int N, int tile_n) {
  const int BN = tile_width(tile_n);
  const int64_t tiles = static_cast<int64_t>((m + BM - 1) / BM) * ((n + BN - 1) / BN);
  return tiles * (mode == kModeResidue ? N : 1);
}

bool encode_gemm_problem(GemmProblem* gp, const uint8_t* a, const uint8_t* b, int64_t ld8, int planes, int m, int n,
                         int k, int tile_n) {
  const int BN = tile_width(tile_n);
  if (!encode_fp8_map(&gp->ta, a, k, m, planes, ld8, 0, BM, BK)) return false;
  if (!encode_fp8_map(&gp->tb, b, k, n, planes, ld8, 0, BN, BK)) return false;
  gp->m = m;
  gp->n = n;
  gp->k = k;
  gp->tiles_m = (m + BM - 1) / BM;
  gp->tiles_n = (n + BN - 1) / BN;
  gp->tiles = gp->tiles_m * gp->tiles_n;
  return true;
}

cudaError_t launch_fp8_gemm_grouped(const GemmArgs& g, const GemmProblem* probs, int count, int64_t total_units,
                                    cudaStream_t st) {
  if (count < 1 || total_units < 1 || total_units > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  if (g.mode != kModeResidue && g.mode != kModeBound) return cudaErrorInvalidValue;
  GemmParams prm{};
  prm.mode = g.mode;
  prm.num_units = static_cast<int>(total_units);
  prm.flags = g.flags;
  prm.wait_ns = g.wait_ns;
  prm.stall = g.stall ? 1 : 0;
  if (g.mode == kModeResidue) fill_mod(prm, *g.mt);
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  const int ctas = g.num_sms < kMaxGemmCtas ? g.num_sms : kMaxGemmCtas;
  const int grid = prm.num_units < ctas ? prm.num_units : ctas;
  const int BN = tile_width(g.tile_n);
  if (g.mode == kModeResidue)
    return launch_tile<kModeResidue, true>(BN, prm, unused, unused, grid, probs, count, st);
  return launch_tile<kModeBound, true>(BN, prm, unused, unused, grid, probs, count, st);
}

}  // namespace ozk2
