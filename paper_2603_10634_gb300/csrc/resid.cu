// Residues and FP8 digit planes, Sec. III-B / III-C / III-D of the paper (workflow
// steps 4-6 of Sec. IV-B).
//
// For each element, a' = trunc(2^e a) (Eq. def:A'), then for every modulus p_l
//   r = mod(a', p_l)                                  (symmetric remainder)
//   square p = s^2 : d1 = round(r / s), d2 = r - s d1            (Sec. III-D)
//   Karatsuba      : d1 = sign(r) ceil(|r| / 16), d2 = r - 16 d1,
//                    d3 = d1 + d2                                (Sec. III-B)
// and each digit (|d| <= 16, exact in E4M3) is stored as an E4M3 byte in its plane.
//
// a' is never formed as a wide integer or a double.  With a = M 2^E (M the 53-bit
// significand) and t = E + e: a' = M' 2^t', where M' = M >> -t, t' = 0 if t < 0 and
// M' = M, t' = t otherwise.  M' is split once into five signed 11-bit pieces c_j
// (exact floats), and for each modulus
//   x = sum_j c_j w_j,   w_j = 2^(11j) mod p in [-p/2, p/2],   |x| <= 5 (2^11 - 1) 544 < 2^23
// is formed with exact FP32 fused multiply-adds.  For odd p the exact product x (1/p)
// rounded once (see reduce) differs from x / p by at most |x| 2^-24 / p < 1/(2p), less
// than the distance from x / p to any half-integer, so q is the nearest integer to x / p
// and r = x - q p (one exact FMA) is the symmetric remainder with no correction step.
// p = 1024 uses q = floor((x + 512) / 1024), exact.  No conversion instruction is used:
// every rounding is an FP32 add of 1.5 2^23.  When t' > 0 the remainder is
// multiplied by 2^t' mod p (|product| < 2^19) and reduced once more.
//
// Rows of A produce K-major planes directly.  Columns of B are written transposed
// (plane rows are columns of B), so both operands of the tensor-core products are
// K-major.  Each thread owns 8 elements.
#include <algorithm>

#include <cuda_fp8.h>

#include "device.cuh"

namespace ozk2 {
namespace {

constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;
constexpr int kPieces = 5;  // 11-bit pieces of the 53-bit shifted significand
constexpr int kElems = 8;  // elements per thread
constexpr int kPairs = kElems / 2;

// Signed byte pieces of a' (as floats) and t'.
// a: the element's IEEE-754 bits (the kernels move elements as 64-bit integers).
__device__ __forceinline__ void decode_element(unsigned long long bits, int e, float (&c)[kPieces], int& tp,
                                               bool& range_err) {
  const unsigned long long mag = bits & kAbsMask;
  unsigned long long Mp = 0;
  tp = 0;
  if (mag != 0 && mag < kInfBits) {
    const int be = static_cast<int>(mag >> 52);
    const unsigned long long M = be ? ((mag & ((1ull << 52) - 1)) | (1ull << 52)) : mag;
    const int t = (be ? be - 1075 : -1074) + e;
    if (t >= 0) {
      Mp = M;
      tp = t;
    } else {
      Mp = (t <= -64) ? 0ull : (M >> (-t));
    }
    if (tp >= kPow2Table) {
      range_err = true;
      Mp = 0;
      tp = 0;
    }
  }
  // piece b (< 2^11) -> float via the bit pattern of 2^23 + b (exact), sign folded into
  // one FMA: sg (2^23 + b) - sg 2^23 = sg b
  const uint32_t lo = static_cast<uint32_t>(Mp), hi = static_cast<uint32_t>(Mp >> 32);
  const float sg = (bits >> 63) ? -1.0f : 1.0f;
  const float off = -sg * 8388608.0f;
  const uint32_t pieces[kPieces] = {lo & 0x7FFu, (lo >> 11) & 0x7FFu, __funnelshift_r(lo, hi, 22) & 0x7FFu,
                                    (hi >> 1) & 0x7FFu, hi >> 12};
#pragma unroll
  for (int j = 0; j < kPieces; ++j) c[j] = fmaf(sg, __uint_as_float(0x4B000000u | pieces[j]), off);
}

// The arithmetic below runs on element pairs: two elements of the same modulus share
// every constant, so each step is one packed two-wide FP32 instruction of sm_100-class
// GPUs (__ffma2_rn / __fadd2_rn), which rounds each component exactly like the scalar
// fmaf / add.  The digits are therefore bit-identical to an element-at-a-time pass.
using f2 = float2;
__device__ __forceinline__ f2 dup(float v) { return make_float2(v, v); }

struct ModF {
  f2 neg_p, inv_p;
  f2 w[kPieces];
  bool pow2_modulus;  // p = 1024
};

// Rounding to an integer without a conversion instruction: for |y| < 2^22, y + 1.5 2^23
// rounds (to nearest, ties to even) to an integer-valued float, and subtracting
// 1.5 2^23 is exact.  fma(x, inv_p, kMagic) rounds the exact product x (1/p), so the
// quotient estimate carries only the error of inv_p: |x| (1/p) 2^-24 < 1/(2p) for |x| < 2^23.
// Inputs are never -0 (the pieces c_j come out of an exact FMA as +0 when zero), so
// no remainder or digit is -0 (E4M3 0x80).
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23

__device__ __forceinline__ f2 round_magic(f2 y) { return __fadd2_rn(y, dup(-kMagic)); }

__device__ __forceinline__ f2 reduce(f2 x, const ModF& m) {
  if (m.pow2_modulus) {
    // floor((x + 512) / 1024) = round((x + 0.5) / 1024) for integer x (never a tie);
    // (x + 0.5) / 1024 is formed exactly by the inner FMA.
    const f2 q = round_magic(__fadd2_rn(__ffma2_rn(x, dup(0.0009765625f), dup(0.00048828125f)), dup(kMagic)));
    return __ffma2_rn(dup(-1024.0f), q, x);
  }
  const f2 q = round_magic(__ffma2_rn(x, m.inv_p, dup(kMagic)));
  return __ffma2_rn(m.neg_p, q, x);
}

// P2: some element of the warp has t' > 0 (rare: a' >= 2^53), so the remainder takes the
// factor 2^t' mod p.  A template argument rather than a branch, so that the common path
// carries no table loads.
template <bool P2>
__device__ __forceinline__ f2 residue_of(const f2 (&c)[kPieces], int tp0, int tp1, const ModF& m,
                                         const float* pow2) {
  f2 x = c[0];
#pragma unroll
  for (int j = 1; j < kPieces; ++j) x = __ffma2_rn(c[j], m.w[j], x);
  f2 r = reduce(x, m);
  if constexpr (P2)  // + 0 gives +0, never -0
    r = reduce(__ffma2_rn(r, make_float2(pow2[tp0], pow2[tp1]), dup(0.0f)), m);
  return r;
}

// Digits of a residue r (an exact float, never -0); the digits are never -0 either
// (an exact zero from x - x or x + (-x) is +0 in round-to-nearest).
__device__ __forceinline__ void square_digits(f2 r, f2 neg_s, f2 inv_s, f2& d1, f2& d2) {
  d1 = round_magic(__ffma2_rn(r, inv_s, dup(kMagic)));  // round(r / s), ties to even (only s = 32 has ties)
  d2 = __ffma2_rn(neg_s, d1, r);
}
__device__ __forceinline__ void karatsuba_digits(f2 r, f2& d1, f2& d2, f2& d3) {
  // d1 = sign(r) ceil(|r| / 16) = RN(r / 16 + sign(r) 15/32): the sum is exact and never a
  // half-integer for integer r, and a zero result is +0
  const f2 off = make_float2(copysignf(0.46875f, r.x), copysignf(0.46875f, r.y));
  d1 = round_magic(__fadd2_rn(__ffma2_rn(r, dup(0.0625f), off), dup(kMagic)));
  d2 = __ffma2_rn(dup(-16.0f), d1, r);
  d3 = __fadd2_rn(d1, d2);
}

// Four E4M3 bytes, elements in address order: pair lo, then pair hi.
__device__ __forceinline__ uint32_t e4m3x4(f2 lo, f2 hi) {
  const uint32_t a = __nv_cvt_float2_to_fp8x2(lo, __NV_SATFINITE, __NV_E4M3);
  const uint32_t b = __nv_cvt_float2_to_fp8x2(hi, __NV_SATFINITE, __NV_E4M3);
  return a | (b << 16);
}

struct ResidArgs {
  const double* X;
  int64_t ldx;
  int lines;  // rows of A or columns of B
  int k, kp;
  int64_t ldp;  // row pitch of a plane (bytes)
  const int32_t* exps;
  uint8_t* planes;
  int64_t plane_stride;  // lines * ldp
  uint32_t* flags;
};

// The residue kernels' constants in shared memory (the modulus loops index them by a
// loop counter): per modulus the FP32 pairs and the table of 2^t mod p.
struct __align__(16) ModConsts {
  f2 neg_p, inv_p, neg_s, inv_s;
  f2 w[kPieces];
  float is1024, pad;  // p = 1024: the floor-based reduction
};
struct Tables {
  ModConsts c[kMaxModuli];
  float pow2[kMaxModuli * kPow2Table];
};

__device__ __forceinline__ void load_tables(const ModTable& mt, Tables& tb) {
  for (int i = threadIdx.x; i < mt.N * kPow2Table; i += blockDim.x)
    tb.pow2[i] = static_cast<float>(mt.pow2[i / kPow2Table][i % kPow2Table]);
  for (int l = threadIdx.x; l < mt.N; l += blockDim.x) {
    ModConsts& c = tb.c[l];
    c.neg_p = mt.neg_p2[l];
    c.inv_p = mt.inv_p2[l];
    c.neg_s = mt.neg_s2[l];
    c.inv_s = mt.inv_s2[l];
#pragma unroll
    for (int j = 0; j < kPieces; ++j) c.w[j] = mt.w2[l][j];
    c.is1024 = mt.p[l] == 1024 ? 1.0f : 0.0f;
    c.pad = 0.0f;
  }
  __syncthreads();
}

// SQUARE: the modulus is one of the squares, the only kind that contains p = 1024.
template <bool SQUARE>
__device__ __forceinline__ ModF consts_of(const ModConsts& c) {
  ModF m;
  m.neg_p = c.neg_p;
  m.inv_p = c.inv_p;
#pragma unroll
  for (int j = 0; j < kPieces; ++j) m.w[j] = c.w[j];
  m.pow2_modulus = SQUARE && c.is1024 != 0.0f;
  return m;
}

// t' of the thread's 8 elements, one byte each (t' < kPow2Table).
struct TpPack {
  uint32_t w[2];
};
__device__ __forceinline__ int tp_of(const TpPack& p, int t) { return (p.w[t >> 2] >> (8 * (t & 3))) & 0xFF; }

// Digits of the thread's 8 elements (4 pairs) for square modulus l, packed as E4M3
// bytes: words[x][q] holds plane x's bytes of elements 4q .. 4q+3.
template <bool P2>
__device__ __forceinline__ void square_words(const f2 (&c)[kPairs][kPieces], const TpPack& tp,
                                             const Tables& tb, int l, uint32_t (&words)[2][2]) {
  const ModConsts& cs = tb.c[l];
  const ModF m = consts_of<true>(cs);
  const float* pw = tb.pow2 + l * kPow2Table;
  const f2 neg_s = cs.neg_s;
  const f2 inv_s = cs.inv_s;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    f2 d1[2], d2[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pr = 2 * q + u;
      square_digits(residue_of<P2>(c[pr], tp_of(tp, 2 * pr), tp_of(tp, 2 * pr + 1), m, pw), neg_s, inv_s, d1[u], d2[u]);
    }
    words[0][q] = e4m3x4(d1[0], d1[1]);
    words[1][q] = e4m3x4(d2[0], d2[1]);
  }
}

// The same for Karatsuba modulus l (three planes).
template <bool P2>
__device__ __forceinline__ void karatsuba_words(const f2 (&c)[kPairs][kPieces], const TpPack& tp,
                                                const Tables& tb, int l, uint32_t (&words)[3][2]) {
  const ModF m = consts_of<false>(tb.c[l]);
  const float* pw = tb.pow2 + l * kPow2Table;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    f2 d1[2], d2[2], d3[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pr = 2 * q + u;
      karatsuba_digits(residue_of<P2>(c[pr], tp_of(tp, 2 * pr), tp_of(tp, 2 * pr + 1), m, pw), d1[u], d2[u], d3[u]);
    }
    words[0][q] = e4m3x4(d1[0], d1[1]);
    words[1][q] = e4m3x4(d2[0], d2[1]);
    words[2][q] = e4m3x4(d3[0], d3[1]);
  }
}

// Pieces of element t of the thread's 8, into its pair slot; its t' into tp (zeroed
// before the first element) and any_tp.
__device__ __forceinline__ void decode_into(f2 (&c)[kPairs][kPieces], int t, unsigned long long a, int e,
                                            TpPack& tp, int& any_tp, bool& range_err) {
  float v[kPieces];
  int tpt;
  decode_element(a, e, v, tpt, range_err);
  tp.w[t >> 2] |= static_cast<uint32_t>(tpt) << (8 * (t & 3));
  any_tp |= tpt;
#pragma unroll
  for (int j = 0; j < kPieces; ++j) {
    if (t & 1) c[t >> 1][j].y = v[j];
    else c[t >> 1][j].x = v[j];
  }
}

// Destination of a task that owns 8 consecutive bytes of every digit plane: the planes
// are written in order, each store moving the pointer to the next plane.
struct PlaneStore {
  uint8_t* dst;    // the task's bytes in the next plane
  int64_t stride;  // bytes from one plane to the next
  bool active;
  __device__ __forceinline__ void put(const uint32_t (&w)[2]) {
    if (active) *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    dst += stride;
  }
};

// every digit |d| <= 16: E4M3 magnitude code at most 0x58 (= 16)
__device__ __forceinline__ void check_digits(const uint32_t (&w)[2], uint32_t* flags) {
  OZK2_DCHECK(__vcmpgtu4(w[0] & 0x7F7F7F7Fu, 0x58585858u) == 0u && __vcmpgtu4(w[1] & 0x7F7F7F7Fu, 0x58585858u) == 0u,
              flags);
}

// Every digit plane of the thread's 8 elements, one modulus at a time.  The modulus loops
// stay rolled: unrolled over all N moduli, the body outgrew the instruction cache and the
// warps waited on instruction fetch more than on anything else.
template <bool P2>
__device__ __forceinline__ void all_planes(int N, const Tables& tb, const f2 (&c)[kPairs][kPieces],
                                           const TpPack& tp, PlaneStore st, uint32_t* flags) {
  const int nsq = N < kNumSquares ? N : kNumSquares;
  // planes in order: 2 per square modulus, then 3 per Karatsuba modulus
#pragma unroll 1
  for (int l = 0; l < nsq; ++l) {
    uint32_t w[2][2];
    square_words<P2>(c, tp, tb, l, w);
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      check_digits(w[x], flags);
      st.put(w[x]);
    }
  }
#pragma unroll 1
  for (int l = kNumSquares; l < N; ++l) {
    uint32_t w[3][2];
    karatsuba_words<P2>(c, tp, tb, l, w);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      check_digits(w[x], flags);
      st.put(w[x]);
    }
  }
}

// The planes of one task: the P2 form only when some element of the warp needs it.
__device__ __forceinline__ void task_planes(int N, const Tables& tb, const f2 (&c)[kPairs][kPieces],
                                            const TpPack& tp, int any_tp, const PlaneStore& st,
                                            uint32_t* flags) {
  if (__any_sync(0xffffffffu, any_tp != 0)) all_planes<true>(N, tb, c, tp, st, flags);
  else all_planes<false>(N, tb, c, tp, st, flags);
}

// Rows of A.  A warp item covers 2^s lanes x 8 k of 32 / 2^s rows (16 lanes on 128
// consecutive k of two rows, or 4 or 8 lanes per row for rows of at most 64 k; see
// resid_rows_lane_log), so short rows and the ends of rows leave few lanes idle.  Lane
// l owns 8 consecutive elements (four 16-byte loads when the row is 16-byte aligned) and
// writes 8 bytes of each plane.
static_assert(kElems == 8, "the row kernel's item shapes assume 8 elements per lane");

// vblock / vgrid: the block's index among, and the number of, the blocks serving this
// operand (the warps stride over its items).
__device__ __forceinline__ void residues_rows_body(const ResidArgs& a, int N, const Tables& tb, int64_t vblock,
                                                   int64_t vgrid) {
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int ls = resid_rows_lane_log(a.kp);
  const int rpi = 32 >> ls, span = kElems << ls;  // rows per item, k per item
  const int nkw = (a.kp + span - 1) / span;
  const int groups = (a.lines + rpi - 1) / rpi;
  const int64_t items = static_cast<int64_t>(groups) * nkw;
  const int64_t stride = vgrid * warps_per_block;
  const int64_t first = vblock * warps_per_block + (threadIdx.x >> 5);
  if (first >= items) return;
  // (row group, k chunk) of the item, advanced by the stride's quotient and remainder
  // instead of a 64-bit division per item (the stride is at most a few grids of warps)
  int grp, chunk, dgrp, dchunk;
  divmod_nonneg(first, nkw, grp, chunk);
  divmod_nonneg(stride, nkw, dgrp, dchunk);
  // every line of X starts on a 16-byte boundary: 16-byte loads
  const bool vec = (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0 && (a.ldx & 1) == 0;
  bool range_err = false;
  for (; grp < groups; grp += dgrp, chunk += dchunk) {
    if (chunk >= nkw) {
      chunk -= nkw;
      if (++grp >= groups) break;
    }
    const int row = grp * rpi + (lane >> ls);
    const bool row_ok = row < a.lines;
    const int h0 = chunk * span + (lane & ((1 << ls) - 1)) * kElems;
    const unsigned long long* x =
        reinterpret_cast<const unsigned long long*>(a.X + static_cast<int64_t>(row_ok ? row : 0) * a.ldx + h0);
    const int e = row_ok ? a.exps[row] : 0;
    unsigned long long v[kElems];
    if (vec && row_ok && h0 + kElems <= a.k) {
#pragma unroll
      for (int q = 0; q < kElems / 2; ++q) {
        const ulonglong2 d = __ldg(reinterpret_cast<const ulonglong2*>(x) + q);
        v[2 * q] = d.x;
        v[2 * q + 1] = d.y;
      }
    } else {
#pragma unroll
      for (int t = 0; t < kElems; ++t) v[t] = (row_ok && h0 + t < a.k) ? __ldg(x + t) : 0ull;
    }
    f2 c[kPairs][kPieces];
    TpPack tp{};
    int any_tp = 0;
#pragma unroll
    for (int t = 0; t < kElems; ++t) decode_into(c, t, v[t], e, tp, any_tp, range_err);
    const PlaneStore st{a.planes + static_cast<int64_t>(row_ok ? row : 0) * a.ldp + h0, a.plane_stride,
                        row_ok && h0 < a.kp};
    task_planes(N, tb, c, tp, any_tp, st, a.flags);
  }
  if (range_err) atomicOr(a.flags, kFlagRange);
}

// Columns of B through shared memory.  A block converts tiles of kTileCols columns x
// kTileK k: the tile is read row by row (512 contiguous bytes per row of B) into shared
// memory, column-major, then each thread converts 8 consecutive k of one column, so a
// half-warp covers 128 consecutive k of a column and writes one full 128-byte line of
// each plane (the register kernel above writes 32-byte pieces of 8 columns).  Within a
// column, chunk c of 8 elements sits at 64 c bytes with the element order rotated by
// (c >> 1) & 7, so that the 16 lanes reading element t of their chunks hit 16 different
// bank pairs.
constexpr int kTileCols = kResidTileCols, kTileK = kResidTileK;
constexpr int kTilePitch = kTileK + 1;  // doubles per column in shared memory
constexpr size_t kTileBytes = sizeof(double) * kTileCols * kTilePitch;

__device__ __forceinline__ int tile_slot(int h) {  // position of k offset h within its column
  const int c = h >> 3;
  return (c << 3) + ((h & 7) ^ ((c >> 1) & 7));
}

// Tiles t0, t0 + tstride, ... of the operand (tiles numbered with the column tile
// fastest).
__device__ __forceinline__ void residues_cols_tiled_body(const ResidArgs& a, int N, const Tables& tb,
                                                         unsigned long long* tile, int64_t t0, int64_t tstride) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_n = (a.lines + kTileCols - 1) / kTileCols, tiles_k = (a.kp + kTileK - 1) / kTileK;
  const int64_t tiles = static_cast<int64_t>(tiles_n) * tiles_k;
  bool range_err = false;
  for (int64_t t = t0; t < tiles; t += tstride) {
    const int j0 = static_cast<int>(t % tiles_n) * kTileCols;
    const int k0 = static_cast<int>(t / tiles_n) * kTileK;
    // load: warp w reads rows w, w + 8, ...; lane l takes columns l and l + 32
#pragma unroll 4
    for (int r = warp; r < kTileK; r += 8) {
      const int h = k0 + r;
      const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.X + static_cast<int64_t>(h) * a.ldx);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = lane + 32 * u, j = j0 + c;
        tile[c * kTilePitch + tile_slot(r)] = (h < a.k && j < a.lines) ? __ldg(row + j) : 0ull;
      }
    }
    __syncthreads();
    // convert: 4 rounds of 256 (column, 8-k chunk) tasks; a half-warp per column
#pragma unroll 1
    for (int round = 0; round < kTileCols * kTileK / (8 * 256); ++round) {
      const int q = round * 256 + tid;
      const int c = q >> 4, chunk = q & 15;
      const int j = j0 + c, h0 = k0 + chunk * 8;
      const bool active = j < a.lines && h0 < a.kp;
      const int e = j < a.lines ? a.exps[j] : 0;
      const unsigned long long* src = tile + c * kTilePitch + chunk * 8;
      f2 cc[kPairs][kPieces];
      TpPack tp{};
      int any_tp = 0;
#pragma unroll
      for (int u = 0; u < kElems; ++u) {
        decode_into(cc, u, src[u ^ ((chunk >> 1) & 7)], e, tp, any_tp, range_err);
      }
      const PlaneStore st{a.planes + static_cast<int64_t>(j < a.lines ? j : 0) * a.ldp + (h0 < a.kp ? h0 : 0),
                          a.plane_stride, active};
      task_planes(N, tb, cc, tp, any_tp, st, a.flags);
    }
    __syncthreads();  // the tile is reloaded
  }
  if (range_err) atomicOr(a.flags, kFlagRange);
}

__global__ void __launch_bounds__(256, 3) residues_cols_tiled_kernel(ResidArgs a,
                                                                    const __grid_constant__ ModTable mt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tables& tb = *reinterpret_cast<Tables*>(smem_raw + kTileBytes);
  load_tables(mt, tb);
  residues_cols_tiled_body(a, mt.N, tb, reinterpret_cast<unsigned long long*>(smem_raw), blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256, 3) residues_rows_kernel(ResidArgs a, const __grid_constant__ ModTable mt) {
  __shared__ Tables tb;
  load_tables(mt, tb);
  residues_rows_body(a, mt.N, tb, blockIdx.x, gridDim.x);
}

// Grouped: rows of every A; columns of every B (one virtual block per tile).
__global__ void __launch_bounds__(256, 2) residues_rows_batch(const BatchProblem* __restrict__ probs, int count,
                                                           int64_t total, uint32_t* flags,
                                                           const __grid_constant__ ModTable mt) {
  __shared__ Tables tb;
  load_tables(mt, tb);
  for_each_vblock(probs, count, kBkResidRows, total, [&](const BatchProblem& P, int64_t v) {
    const ResidArgs a{P.A, P.lda, P.m, P.k, P.kp, P.ldp, P.e, P.planesA, static_cast<int64_t>(P.m) * P.ldp, flags};
    residues_rows_body(a, mt.N, tb, v, P.nblocks[kBkResidRows]);
  });
}

__global__ void __launch_bounds__(256, 3) residues_cols_batch(const BatchProblem* __restrict__ probs, int count,
                                                           int64_t total, uint32_t* flags,
                                                           const __grid_constant__ ModTable mt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tables& tb = *reinterpret_cast<Tables*>(smem_raw + kTileBytes);
  load_tables(mt, tb);
  for_each_vblock(probs, count, kBkResidCols, total, [&](const BatchProblem& P, int64_t v) {
    const ResidArgs a{P.B, P.ldb, P.n, P.k, P.kp, P.ldp, P.f, P.planesB, static_cast<int64_t>(P.n) * P.ldp, flags};
    residues_cols_tiled_body(a, mt.N, tb, reinterpret_cast<unsigned long long*>(smem_raw), v,
                             P.nblocks[kBkResidCols]);
  });
}

constexpr size_t kColsSmem = kTileBytes + sizeof(Tables);
static_assert(kTileBytes % 16 == 0, "the tables follow the tile on a 16-byte boundary");

// ------------------------------------------------------------------ gradient operands
// The upstream gradient dC (m x n, row-major) of C = A B enters both gradient products
// that reuse the forward's integer matrices, with per-element exponents:
//   G'_ij = trunc(2^(g_i - f_j) dC_ij)  rows i as lines, along j   (dA = dC B^T)
//   H'_ij = trunc(2^(h_j - e_i) dC_ij)  columns j as lines, along i (dB = A^T dC)
// One kernel reads each kTileK x kTileCols tile of dC once into shared memory (the
// layout of the column kernel above: tile rows are rows i of dC, tile columns are
// columns j) and converts it twice: the column pass writes H' exactly as the column
// kernel writes B's planes; the row pass writes G' with 8 consecutive j per task, a
// warp covering 4 rows x 64 columns (64-byte plane pieces).
struct GradArgs {
  const double* dC;
  int64_t lddc;
  int m, n;
  const int32_t* g;  // m: exponents of dC's rows
  const int32_t* f;  // n: the forward's column exponents of B
  const int32_t* h;  // n: exponents of dC's columns
  const int32_t* e;  // m: the forward's row exponents of A
  uint8_t* planesG;  // lines m, pitch ldg, plane stride m * ldg
  int64_t ldg;
  uint8_t* planesH;  // lines n, pitch ldh, plane stride n * ldh
  int64_t ldh;
  uint32_t* flags;
  bool do_g, do_h;  // which of the two outputs to write
};

__global__ void __launch_bounds__(256, 3) grad_residues_kernel(GradArgs a, const __grid_constant__ ModTable mt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned long long* tile = reinterpret_cast<unsigned long long*>(smem_raw);
  Tables& tb = *reinterpret_cast<Tables*>(smem_raw + kTileBytes);
  load_tables(mt, tb);
  const int N = mt.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_n = (a.n + kTileCols - 1) / kTileCols, tiles_m = (a.m + kTileK - 1) / kTileK;
  const int64_t tiles = static_cast<int64_t>(tiles_n) * tiles_m;
  bool range_err = false;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int j0 = static_cast<int>(t % tiles_n) * kTileCols;
    const int i0 = static_cast<int>(t / tiles_n) * kTileK;
#pragma unroll 4
    for (int r = warp; r < kTileK; r += 8) {
      const int i = i0 + r;
      const unsigned long long* row = reinterpret_cast<const unsigned long long*>(a.dC + static_cast<int64_t>(i) * a.lddc);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = lane + 32 * u, j = j0 + c;
        tile[c * kTilePitch + tile_slot(r)] = (i < a.m && j < a.n) ? __ldg(row + j) : 0ull;
      }
    }
    __syncthreads();
    // column pass: H' (lines j, positions i), a half-warp per column
#pragma unroll 1
    for (int round = 0; a.do_h && round < kTileCols * kTileK / (8 * 256); ++round) {
      const int q = round * 256 + tid;
      const int c = q >> 4, chunk = q & 15;
      const int j = j0 + c, ib = i0 + chunk * 8;
      const bool active = j < a.n && ib < a.m;
      const int hj = j < a.n ? a.h[j] : 0;
      const unsigned long long* src = tile + c * kTilePitch + chunk * 8;
      f2 cc[kPairs][kPieces];
      TpPack tp{};
      int any_tp = 0;
#pragma unroll
      for (int u = 0; u < kElems; ++u) {
        const int i = ib + u;
        const int ex = hj - (i < a.m ? a.e[i] : 0);
        decode_into(cc, u, src[u ^ ((chunk >> 1) & 7)], ex, tp, any_tp, range_err);
      }
      const PlaneStore st{a.planesH + static_cast<int64_t>(j < a.n ? j : 0) * a.ldh + (ib < a.m ? ib : 0),
                          static_cast<int64_t>(a.n) * a.ldh, active};
      task_planes(N, tb, cc, tp, any_tp, st, a.flags);
    }
    // row pass: G' (lines i, positions j); warp w, round s: rows 4 (8 s + w) + lane / 8
#pragma unroll 1
    for (int round = 0; a.do_g && round < kTileK * kTileCols / (8 * 256); ++round) {
      const int r = 4 * (8 * round + warp) + (lane >> 3), chunk = lane & 7;
      const int i = i0 + r, jb = j0 + chunk * 8;
      const bool active = i < a.m && jb < a.n;
      const int gi = i < a.m ? a.g[i] : 0;
      f2 cc[kPairs][kPieces];
      TpPack tp{};
      int any_tp = 0;
#pragma unroll
      for (int u = 0; u < kElems; ++u) {
        const int c = chunk * 8 + u, j = jb + u;
        const int ex = gi - (j < a.n ? a.f[j] : 0);
        decode_into(cc, u, tile[c * kTilePitch + tile_slot(r)], ex, tp, any_tp, range_err);
      }
      const PlaneStore st{a.planesG + static_cast<int64_t>(i < a.m ? i : 0) * a.ldg + (jb < a.n ? jb : 0),
                          static_cast<int64_t>(a.m) * a.ldg, active};
      task_planes(N, tb, cc, tp, any_tp, st, a.flags);
    }
    __syncthreads();  // the tile is reloaded
  }
  if (range_err) atomicOr(a.flags, kFlagRange);
}

// dst[p][x][y] = src[p][y][x] for y < lines, x < len: the digit planes of an operand
// (lines x len bytes, K-major) as the planes of its transpose.  A block moves 128 x 128
// byte tiles through shared memory (row pitch 33 words: the words a warp reads along a
// column fall in 32 different banks); each thread then reads a 16 x 4 byte block (16
// rows, 4 columns) as 16 words, transposes it four 4 x 4 blocks at a time with byte
// permutes, and writes 4 destination rows of 16 bytes.
constexpr int kTrTile = 128, kTrPitchW = 33;

// 4 x 4 byte block: in[r] holds bytes (r, 0..3); out[c] gets bytes (0..3, c).
__device__ __forceinline__ void transpose4x4(const uint32_t (&in)[4], uint32_t (&out)[4]) {
  const uint32_t t0 = __byte_perm(in[0], in[1], 0x5140), t1 = __byte_perm(in[0], in[1], 0x7362);
  const uint32_t t2 = __byte_perm(in[2], in[3], 0x5140), t3 = __byte_perm(in[2], in[3], 0x7362);
  out[0] = __byte_perm(t0, t2, 0x5410);
  out[1] = __byte_perm(t0, t2, 0x7632);
  out[2] = __byte_perm(t1, t3, 0x5410);
  out[3] = __byte_perm(t1, t3, 0x7632);
}

__global__ void __launch_bounds__(256) transpose_planes_kernel(const uint8_t* __restrict__ src, int64_t src_pitch,
                                                               int64_t src_stride, int lines, int len,
                                                               uint8_t* __restrict__ dst, int64_t dst_pitch,
                                                               int64_t dst_stride, int planes) {
  __shared__ uint32_t tile[kTrTile * kTrPitchW];
  const int tx = (len + kTrTile - 1) / kTrTile, ty = (lines + kTrTile - 1) / kTrTile;
  const int64_t total = static_cast<int64_t>(tx) * ty * planes;
  const int t = threadIdx.x;
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int p = static_cast<int>(b / (static_cast<int64_t>(tx) * ty));
    const int rem = static_cast<int>(b - static_cast<int64_t>(p) * tx * ty);
    const int y0 = (rem / tx) * kTrTile, x0 = (rem % tx) * kTrTile;
    // load: 128 rows of 128 bytes, 16 bytes per thread and round (inside the source pitch)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = q * 32 + (t >> 3), c16 = (t & 7) * 16;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (y0 + r < lines && x0 + c16 < len)
        v = *reinterpret_cast<const uint4*>(src + p * src_stride + static_cast<int64_t>(y0 + r) * src_pitch + x0 +
                                            c16);
      uint32_t* tw = tile + r * kTrPitchW + c16 / 4;
      tw[0] = v.x;
      tw[1] = v.y;
      tw[2] = v.z;
      tw[3] = v.w;
    }
    __syncthreads();
    // store: destination rows x0 + 4 cw .. + 3, bytes y0 + 16 yb .. + 15
    const int cw = t & 31, yb = t >> 5;
    uint32_t out[4][4];  // out[c][w]: destination row 4 cw + c, word w (4 y's)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      uint32_t in[4], o[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) in[r] = tile[(16 * yb + 4 * w + r) * kTrPitchW + cw];
      transpose4x4(in, o);
#pragma unroll
      for (int c = 0; c < 4; ++c) out[c][w] = o[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = x0 + 4 * cw + c, y = y0 + 16 * yb;
      if (x < len && y < lines)
        *reinterpret_cast<uint4*>(dst + p * dst_stride + static_cast<int64_t>(x) * dst_pitch + y) =
            make_uint4(out[c][0], out[c][1], out[c][2], out[c][3]);
    }
    __syncthreads();
  }
}

// Opt a column kernel into kColsSmem bytes of dynamic shared memory, once per device
// (a launch on a device where this failed reports the error itself).
template <class K>
void allow_cols_smem(K* kernel, bool (&done)[64]) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (!done[dev] && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kColsSmem)) == cudaSuccess)
    done[dev] = true;
}

int grid_for(int64_t warps) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (warps + 7) / 8;
  const int64_t cap = static_cast<int64_t>(sms) * 16;
  return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_residues_rows(const double* A, int64_t lda, int m, int k, int kp, int64_t ldp, const int32_t* e,
                                 const ModTable& mt, uint8_t* planes, uint32_t* flags, cudaStream_t st,
                                 int64_t plane_stride) {
  ResidArgs a{A, lda, m, k, kp, ldp, e, planes, plane_stride ? plane_stride : static_cast<int64_t>(m) * ldp, flags};
  residues_rows_kernel<<<grid_for(resid_rows_items(m, kp)), 256, 0, st>>>(a, mt);
  return cudaGetLastError();
}

cudaError_t launch_residues_cols(const double* B, int64_t ldb, int k, int n, int kp, int64_t ldp, const int32_t* f,
                                 const ModTable& mt, uint8_t* planes, uint32_t* flags, cudaStream_t st,
                                 int64_t plane_stride) {
  ResidArgs a{B, ldb, n, k, kp, ldp, f, planes, plane_stride ? plane_stride : static_cast<int64_t>(n) * ldp, flags};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = static_cast<int64_t>((n + kTileCols - 1) / kTileCols) * ((kp + kTileK - 1) / kTileK);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, 3 * static_cast<int64_t>(sms)));
  static bool done[64] = {};  // per device
  allow_cols_smem(residues_cols_tiled_kernel, done);
  residues_cols_tiled_kernel<<<grid, 256, kColsSmem, st>>>(a, mt);
  return cudaGetLastError();
}

cudaError_t launch_residues_batch(const BatchProblem* probs, int count, int64_t rows_blocks, int64_t cols_blocks,
                                  const ModTable& mt, uint32_t* flags, cudaStream_t st, cudaStream_t st_cols) {
  if (rows_blocks < 1 || cols_blocks < 1 || rows_blocks > 0x7FFFFFFFll || cols_blocks > 0x7FFFFFFFll)
    return cudaErrorInvalidValue;
  static bool done[64] = {};
  allow_cols_smem(residues_cols_batch, done);
  residues_rows_batch<<<grouped_grid(rows_blocks, 3), 256, 0, st>>>(probs, count, rows_blocks, flags, mt);
  residues_cols_batch<<<grouped_grid(cols_blocks, 3), 256, kColsSmem, st_cols>>>(probs, count, cols_blocks, flags,
                                                                                mt);
  return cudaGetLastError();
}

cudaError_t launch_grad_residues(const double* dC, int64_t lddc, int m, int n, const int32_t* g, const int32_t* f,
                                 const int32_t* h, const int32_t* e, uint8_t* planesG, int64_t ldg, uint8_t* planesH,
                                 int64_t ldh, const ModTable& mt, uint32_t* flags, cudaStream_t st) {
  GradArgs a{dC, lddc, m, n, g, f, h, e, planesG, ldg, planesH, ldh, flags, planesG != nullptr, planesH != nullptr};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = static_cast<int64_t>((n + kTileCols - 1) / kTileCols) * ((m + kTileK - 1) / kTileK);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, 3 * static_cast<int64_t>(sms)));
  static bool done[64] = {};  // per device
  allow_cols_smem(grad_residues_kernel, done);
  grad_residues_kernel<<<grid, 256, kColsSmem, st>>>(a, mt);
  return cudaGetLastError();
}

cudaError_t launch_transpose_planes(const uint8_t* src, int64_t src_pitch, int64_t src_stride, int lines, int len,
                                    uint8_t* dst, int64_t dst_pitch, int64_t dst_stride, int planes, cudaStream_t st) {
  if ((src_pitch % 16) || (dst_pitch % 16) || (src_stride % 16) || (dst_stride % 16) || lines < 1 || len < 1 ||
      planes < 1 || src_pitch < ((len + 15) / 16) * 16 || dst_pitch < ((lines + 15) / 16) * 16)
    return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t total = static_cast<int64_t>((len + kTrTile - 1) / kTrTile) * ((lines + kTrTile - 1) / kTrTile) * planes;
  const int grid = static_cast<int>(std::min<int64_t>(total, 8 * static_cast<int64_t>(sms)));
  transpose_planes_kernel<<<grid, 256, 0, st>>>(src, src_pitch, src_stride, lines, len, dst, dst_pitch, dst_stride,
                                                planes);
  return cudaGetLastError();
}

}  // namespace ozk2
