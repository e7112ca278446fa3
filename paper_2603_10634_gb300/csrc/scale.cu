// Scaling, Sec. III-E of the paper (workflow steps 1 and 3 of Sec. IV-B).
//
//   e'_i = 7 - floor(log2 max_h |a_ih|)             (Eq. def:mu'nu', mu'_i = 2^e'_i)
//   Abar_ih = RU_E4M3(2^e'_i |a_ih|)                 (cast to E4M3 in round-up mode)
//   e_i = e'_i + int(P' + delta log2 max_j cbar_ij)  (Eq. mu-computation)
// and the same for the columns of B, whose bound operand is stored transposed
// (n x kp, K-major) so that both GEMM operands are K-major.  Fast mode replaces the bound
// product by the Cauchy-Schwarz bound: the kernels then produce round-up sums of squares
// of the scaled lines instead of Abar / Bbar, and the same exponent rule applies.
// "Rows" kernels serve any operand whose lines are contiguous along k (A, or B^T), the
// "column" kernels any operand whose lines are strided along k (B, or A^T).
//
// Everything up to the exponent rule is integer manipulation of the IEEE-754
// encoding: no FP64 arithmetic and no 2^e' factor is ever formed (e' reaches 1081
// for subnormal rows, beyond the double range).  Non-finite entries count as 0 and
// mark their row / column; a row with no nonzero finite entry gets e' = e = 0.
#include <algorithm>

#include "device.cuh"

namespace ozk2 {
namespace {

// A double's magnitude as two 32-bit words: hi (sign cleared: 11 exponent bits and the
// top 20 fraction bits) and lo (the low 32 fraction bits).  The kernels below work on
// these words with 32-bit integer operations only.
struct Mag {
  uint32_t hi, lo;
};
__device__ __forceinline__ Mag mag_of(double x) {
  return Mag{static_cast<uint32_t>(__double2hiint(x)) & 0x7FFFFFFFu, static_cast<uint32_t>(__double2loint(x))};
}
__device__ __forceinline__ bool nonfinite(Mag m) { return (m.hi >> 20) == 0x7FFu; }

// floor(log2 |x|) + 1075 for a finite nonzero x, a key from 1 (2^-1074) to 2098 that
// orders like |x|; 0 for zero and for a non-finite x, which also sets bad.  No branch,
// so that the loops below keep their loads in flight together.
__device__ __forceinline__ uint32_t log2_key(Mag m, bool& bad) {
  const uint32_t be = m.hi >> 20;
  const uint32_t z = m.hi != 0u ? __clz(m.hi) : 32u + __clz(m.lo);  // leading zeros of the 64-bit magnitude
  bad |= be == 0x7FFu;
  return be == 0x7FFu ? 0u : (be != 0u ? be + 52u : 64u - z);  // normal: floor(log2) = be - 1023
}

// e' = 7 - floor(log2 max |x|) from the key of the line's maximum; 0 for a zero line.
__device__ __forceinline__ int prelim_exponent(uint32_t key) { return key ? 1082 - static_cast<int>(key) : 0; }

// floor(log2 |x|) and the 52 fraction bits of |x| normalised (the top 20 in f20, the rest
// in lo) for a finite nonzero x; subnormals are shifted up (rare, 64-bit operations).
__device__ __forceinline__ int normalise(Mag& m) {
  const int be = static_cast<int>(m.hi >> 20);
  if (be != 0) {
    m.hi &= 0xFFFFFu;
    return be - 1023;
  }
  const unsigned long long f52 = (static_cast<unsigned long long>(m.hi) << 32) | m.lo;
  const int top = 63 - __clzll(f52);
  const unsigned long long n52 = (f52 << (52 - top)) & ((1ull << 52) - 1);
  m.hi = static_cast<uint32_t>(n52 >> 32);
  m.lo = static_cast<uint32_t>(n52);
  return top - 1074;
}

// E4M3 code of the least E4M3 value >= |x| 2^sh, for a finite x with |x| 2^sh < 2^8.
// Positive values below 2^-9 give the smallest subnormal, 2^-9.  E4M3 codes of
// non-negative values increase with the value, so rounding the 3-bit mantissa up may
// carry into the exponent field and stay correct.
__device__ __forceinline__ uint32_t ru_e4m3_scaled(Mag m, int sh) {
  if ((m.hi | m.lo) == 0u) return 0u;
  const int ev = normalise(m) + sh;  // floor(log2) of the scaled value, <= 7
  if (ev >= -6)                      // E4M3 normal range: the top 3 fraction bits, rounded up
    return static_cast<uint32_t>((ev + 7) << 3) + (m.hi >> 17) + (((m.hi & 0x1FFFFu) | m.lo) != 0u ? 1u : 0u);
  if (ev >= -9) {  // E4M3 subnormal k 2^-9, k = ceil(|x| 2^(sh + 9)) in 1..8
    const uint32_t mant = m.hi | (1u << 20);  // the significand's top 21 bits
    const int s = 11 - ev;                    // 18 .. 20
    return (mant >> s) + (((mant & ((1u << s) - 1u)) | m.lo) != 0u ? 1u : 0u);
  }
  return 1u;
}

// RU_fp32(|x| 2^sh) for a finite nonzero x with |x| 2^sh < 2^8: the float bit pattern
// is assembled from the exponent and the top 23 fraction bits, plus one unit when any
// lower bit is set (a carry into the exponent field stays correct).  Results below the
// FP32 normal range are replaced by 2^-126, still an upper bound.
__device__ __forceinline__ float ru_f32_scaled(Mag m, int sh) {
  if ((m.hi | m.lo) == 0u) return 0.0f;
  const int ev = normalise(m) + sh;
  if (ev < -126) return 1.1754943508222875e-38f;  // 2^-126
  const uint32_t bits = (static_cast<uint32_t>(ev + 127) << 23) + ((m.hi << 3) | (m.lo >> 29)) +
                        ((m.lo & 0x1FFFFFFFu) != 0u ? 1u : 0u);
  return __uint_as_float(bits);
}

// Loads a thread keeps in flight per batch (the column kernels take twice as many).
constexpr int kBatch = 4;

// One warp per row of A: row maximum, e'_i, row status, then Abar (m x kp bytes).
// FAST: instead of Abar, the sum of squares s_i = sum_h RU_fp32(2^e'_i |a_ih|)^2 with
// every addition rounded up (an upper bound of ||2^e'_i a_i||_2^2), written to sq[row].
// vblock: the block's index among the blocks of this problem (8 rows each).
template <bool FAST>
__device__ __forceinline__ void scale_rows_body(const double* __restrict__ A, int64_t lda, int m, int k, int kp,
                                                int32_t* __restrict__ eprime, uint8_t* __restrict__ rowstat,
                                                uint8_t* __restrict__ Abar, float* __restrict__ sq,
                                                uint32_t* flags, int64_t vblock) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = static_cast<int>(vblock) * (blockDim.x >> 5) + warp;
  if (row >= m) return;
  const double* a = A + static_cast<int64_t>(row) * lda;
  uint32_t key = 0u;
  bool bad = false;
  for (int h = lane; h < k; h += 32 * kBatch) {
    double v[kBatch];  // the loads of a batch are issued before any is used
#pragma unroll
    for (int u = 0; u < kBatch; ++u) v[u] = h + 32 * u < k ? __ldg(a + h + 32 * u) : 0.0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) key = max(key, log2_key(mag_of(v[u]), bad));
  }
  key = __reduce_max_sync(0xffffffffu, key);
  bad = __any_sync(0xffffffffu, bad);
  const int ep = prelim_exponent(key);
  if (lane == 0) {
    eprime[row] = ep;
    rowstat[row] = static_cast<uint8_t>((key == 0u ? kLineZero : 0) | (bad ? kLineNonfinite : 0));
    if (bad) atomicOr(flags, kFlagNonfinite);
  }
  if constexpr (FAST) {
    float acc = 0.0f;
#pragma unroll 4
    for (int h = lane; h < k; h += 32) {
      const Mag mg = mag_of(__ldg(a + h));
      if (!nonfinite(mg)) {
        const float v = ru_f32_scaled(mg, ep);
        acc = __fmaf_ru(v, v, acc);
      }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) acc = __fadd_ru(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if (lane == 0) sq[row] = acc;
  } else {
    uint8_t* out = Abar + static_cast<int64_t>(row) * kp;
    for (int h0 = lane * 4; h0 < kp; h0 += 256) {
      double v[8];  // two words of 4 bytes, 128 bytes apart; loads first
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int h = h0 + (t >> 2) * 128 + (t & 3);
        v[t] = h < k ? __ldg(a + h) : 0.0;
      }
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        uint32_t word = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const Mag mg = mag_of(v[4 * g + t]);
          if (!nonfinite(mg)) word |= ru_e4m3_scaled(mg, ep) << (8 * t);
        }
        if (h0 + 128 * g < kp) *reinterpret_cast<uint32_t*>(out + h0 + 128 * g) = word;
      }
    }
  }
}

template <bool FAST>
__global__ void __launch_bounds__(256) scale_rows_kernel(const double* __restrict__ A, int64_t lda, int m, int k,
                                                         int kp, int32_t* __restrict__ eprime,
                                                         uint8_t* __restrict__ rowstat, uint8_t* __restrict__ Abar,
                                                         float* __restrict__ sq, uint32_t* flags) {
  scale_rows_body<FAST>(A, lda, m, k, kp, eprime, rowstat, Abar, sq, flags, blockIdx.x);
}

constexpr int kColRows = 256;

// Column maxima of |B| (as log2 keys) and non-finite flags.  Block (bx, by): columns
// 256 bx .. 256 bx + 255, rows rpb by .. rpb by + rpb - 1.
__device__ __forceinline__ void colmax_body(const double* __restrict__ B, int64_t ldb, int k, int n,
                                            uint32_t* __restrict__ colmax, uint32_t* __restrict__ colbad, int bx,
                                            int by, int rpb) {
  const int j = bx * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int h0 = by * rpb;
  const int h1 = min(k, h0 + rpb);
  uint32_t key = 0u;
  bool bad = false;
  for (int h = h0; h < h1; h += 2 * kBatch) {
    double v[2 * kBatch];  // the loads of a batch are issued before any is used
#pragma unroll
    for (int u = 0; u < 2 * kBatch; ++u) v[u] = h + u < h1 ? __ldg(B + static_cast<int64_t>(h + u) * ldb + j) : 0.0;
#pragma unroll
    for (int u = 0; u < 2 * kBatch; ++u) key = max(key, log2_key(mag_of(v[u]), bad));
  }
  if (key) atomicMax(colmax + j, key);
  if (bad) atomicOr(colbad + j, 1u);
}

__global__ void __launch_bounds__(256) colmax_kernel(const double* __restrict__ B, int64_t ldb, int k, int n,
                                                     uint32_t* __restrict__ colmax, uint32_t* __restrict__ colbad,
                                                     int rpb) {
  colmax_body(B, ldb, k, n, colmax, colbad, blockIdx.x, blockIdx.y, rpb);
}

// Bbar^T (n x kp bytes): thread (column j, 32 consecutive h) writes 32 bytes of row j.
// FAST: instead, the partial sum of squares of the 32 elements (rounded up) goes to
// part[hb * n + j]; sumsq_reduce_kernel adds the partials of a column in a fixed order.
template <bool FAST>
__device__ __forceinline__ void scale_cols_body(const double* __restrict__ B, int64_t ldb, int k, int n, int kp,
                                                const uint32_t* __restrict__ colmax,
                                                const uint32_t* __restrict__ colbad, int32_t* __restrict__ fprime,
                                                uint8_t* __restrict__ colstat, uint8_t* __restrict__ BbarT,
                                                float* __restrict__ part, uint32_t* flags, int bx, int hb) {
  const int j = bx * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t key = colmax[j];
  const bool bad = colbad[j] != 0;
  const int fp = prelim_exponent(key);
  if (hb == 0) {
    fprime[j] = fp;
    colstat[j] = static_cast<uint8_t>((key == 0u ? kLineZero : 0) | (bad ? kLineNonfinite : 0));
    if (bad) atomicOr(flags, kFlagNonfinite);
  }
  if constexpr (FAST) {
    float acc = 0.0f;
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      const int h = hb * 32 + t;
      if (h < k) {
        const Mag mg = mag_of(__ldg(B + static_cast<int64_t>(h) * ldb + j));
        if (!nonfinite(mg)) {
          const float v = ru_f32_scaled(mg, fp);
          acc = __fmaf_ru(v, v, acc);
        }
      }
    }
    part[static_cast<int64_t>(hb) * n + j] = acc;
  } else {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = 0;
#pragma unroll
    for (int t0 = 0; t0 < 32; t0 += 2 * kBatch) {
      double v[2 * kBatch];  // loads first
#pragma unroll
      for (int u = 0; u < 2 * kBatch; ++u) {
        const int h = hb * 32 + t0 + u;
        v[u] = h < k ? __ldg(B + static_cast<int64_t>(h) * ldb + j) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 2 * kBatch; ++u) {
        const Mag mg = mag_of(v[u]);
        const int t = t0 + u;
        if (!nonfinite(mg)) w[t >> 2] |= ru_e4m3_scaled(mg, fp) << (8 * (t & 3));
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(BbarT + static_cast<int64_t>(j) * kp + hb * 32);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

template <bool FAST>
__global__ void __launch_bounds__(256) scale_cols_kernel(const double* __restrict__ B, int64_t ldb, int k, int n,
                                                         int kp, const uint32_t* __restrict__ colmax,
                                                         const uint32_t* __restrict__ colbad,
                                                         int32_t* __restrict__ fprime, uint8_t* __restrict__ colstat,
                                                         uint8_t* __restrict__ BbarT, float* __restrict__ part,
                                                         uint32_t* flags) {
  scale_cols_body<FAST>(B, ldb, k, n, kp, colmax, colbad, fprime, colstat, BbarT, part, flags, blockIdx.x,
                        blockIdx.y);
}

// s_j = sum over blocks of part[hb][j], every addition rounded up, in block order.
__device__ __forceinline__ void sumsq_body(const float* __restrict__ part, int nblocks, int n,
                                           float* __restrict__ sq, int64_t vblock) {
  const int j = static_cast<int>(vblock) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float acc = 0.0f;
  for (int hb = 0; hb < nblocks; ++hb) acc = __fadd_ru(acc, part[static_cast<int64_t>(hb) * n + j]);
  sq[j] = acc;
}

__global__ void sumsq_reduce_kernel(const float* __restrict__ part, int nblocks, int n, float* __restrict__ sq) {
  sumsq_body(part, nblocks, n, sq, blockIdx.x);
}

// e = e' + floor(RD(P' + RD(delta * log2 R))) [Eq. mu-computation].  log2 is the FP32
// rounding of the double-precision log2 (a correctly rounded FP32 log2 except in
// vanishingly rare ties); P' + delta log2 R is evaluated in FP32 round-down.
__device__ __forceinline__ int final_exponent(int ep, uint8_t stat, float rmax, float pprime,
                                              float delta) {
  if (stat & kLineZero) return 0;
  if (!(rmax > 0.0f)) return ep + static_cast<int>(floorf(pprime));
  const float lg = __double2float_rn(log2(static_cast<double>(rmax)));
  const float t1 = __fmul_rd(delta, lg);
  const float t2 = __fadd_rd(pprime, t1);
  return ep + static_cast<int>(floorf(t2));
}

__device__ __forceinline__ void exponents_body(int m, int n, const int32_t* __restrict__ eprime,
                                               const int32_t* __restrict__ fprime,
                                               const uint8_t* __restrict__ rowstat,
                                               const uint8_t* __restrict__ colstat, const float* __restrict__ R,
                                               const float* __restrict__ S, float pprime, float delta,
                                               int32_t* __restrict__ e, int32_t* __restrict__ f, int64_t vblock) {
  const int t = static_cast<int>(vblock) * blockDim.x + threadIdx.x;
  if (t < m) {
    e[t] = final_exponent(eprime[t], rowstat[t], R[t], pprime, delta);
  } else if (t < m + n) {
    const int j = t - m;
    f[j] = final_exponent(fprime[j], colstat[j], S[j], pprime, delta);
  }
}

__global__ void exponents_kernel(int m, int n, const int32_t* __restrict__ eprime,
                                 const int32_t* __restrict__ fprime, const uint8_t* __restrict__ rowstat,
                                 const uint8_t* __restrict__ colstat, const float* __restrict__ R,
                                 const float* __restrict__ S, float pprime, float delta, int32_t* __restrict__ e,
                                 int32_t* __restrict__ f) {
  exponents_body(m, n, eprime, fprime, rowstat, colstat, R, S, pprime, delta, e, f, blockIdx.x);
}

// Exponent of a line whose product partner's integers are fixed (the gradient products
// that reuse the forward's A' or B'): g = g' + floor(RD(Q + RD(d log2 R))) with
// Q = RD(log2(P - 1) - 1) and d = -(1 + 2^-21) for log2 R >= 0, -(1 - 2^-21) below, so
// that d log2 R stays below -log2 R whatever the FP32 rounding of the logarithm; then
// 2 2^(g - g') R <= P - 1.  A zero line gets 0; R = 0 gives g' + floor(Q); an infinite
// R (its shifted bound overflowed FP32) is out of range.
__device__ __forceinline__ int reuse_exponent(int gp, uint8_t stat, float rmax, float q, uint32_t* flags) {
  if (stat & kLineZero) return 0;
  if (!(rmax > 0.0f)) return gp + static_cast<int>(floorf(q));
  if (!(rmax < INFINITY)) {
    atomicOr(flags, kFlagRange);
    return gp - 256;
  }
  const float lg = __double2float_rn(log2(static_cast<double>(rmax)));
  const float d = lg >= 0.0f ? -(1.0f + 0x1p-21f) : -(1.0f - 0x1p-21f);
  const float t1 = __fmul_rd(d, lg);
  const float t2 = __fadd_rd(q, t1);
  return gp + static_cast<int>(floorf(t2));
}

// g_i for the m rows (prelim gp, status rstat, bound R) and h_j for the n columns.
__global__ void reuse_exponents_kernel(int m, const int32_t* __restrict__ gp, const uint8_t* __restrict__ rstat,
                                       const float* __restrict__ R, int32_t* __restrict__ g, int n,
                                       const int32_t* __restrict__ hp, const uint8_t* __restrict__ cstat,
                                       const float* __restrict__ S, int32_t* __restrict__ h, float q,
                                       uint32_t* flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) {
    g[t] = reuse_exponent(gp[t], rstat[t], R[t], q, flags);
  } else if (t < m + n) {
    const int j = t - m;
    h[j] = reuse_exponent(hp[j], cstat[j], S[j], q, flags);
  }
}

// ------------------------------------------------------------------ grouped launches
template <bool FAST>
__global__ void __launch_bounds__(256) scale_rows_batch(const BatchProblem* __restrict__ probs, int count,
                                                        int64_t total, uint32_t* flags) {
  for_each_vblock(probs, count, kBkScaleRows, total, [&](const BatchProblem& P, int64_t v) {
    scale_rows_body<FAST>(P.A, P.lda, P.m, P.k, P.kp, P.eprime, P.rowstat, P.Abar, P.R, flags, v);
  });
}

__global__ void __launch_bounds__(256) colmax_batch(const BatchProblem* __restrict__ probs, int count,
                                                    int64_t total) {
  for_each_vblock(probs, count, kBkColmax, total, [&](const BatchProblem& P, int64_t v) {
    const int gx = (P.n + 255) / 256;
    int by, bx;
    divmod_nonneg(v, gx, by, bx);
    colmax_body(P.B, P.ldb, P.k, P.n, P.colmaxB, P.colbadB, bx, by, kColRows);
  });
}

template <bool FAST>
__global__ void __launch_bounds__(256) scale_cols_batch(const BatchProblem* __restrict__ probs, int count,
                                                        int64_t total, uint32_t* flags) {
  for_each_vblock(probs, count, kBkScaleCols, total, [&](const BatchProblem& P, int64_t v) {
    const int gx = (P.n + 255) / 256;
    int hb, bx;
    divmod_nonneg(v, gx, hb, bx);
    scale_cols_body<FAST>(P.B, P.ldb, P.k, P.n, P.kp, P.colmaxB, P.colbadB, P.fprime, P.colstat, P.BbarT, P.partB,
                          flags, bx, hb);
  });
}

__global__ void __launch_bounds__(256) sumsq_batch(const BatchProblem* __restrict__ probs, int count, int64_t total) {
  for_each_vblock(probs, count, kBkSumsq, total, [&](const BatchProblem& P, int64_t v) {
    sumsq_body(P.partB, P.kp / 32, P.n, P.S, v);
  });
}

__global__ void __launch_bounds__(256) exponents_batch(const BatchProblem* __restrict__ probs, int count,
                                                       int64_t total, float pprime, float delta) {
  for_each_vblock(probs, count, kBkExponents, total, [&](const BatchProblem& P, int64_t v) {
    exponents_body(P.m, P.n, P.eprime, P.fprime, P.rowstat, P.colstat, P.R, P.S, pprime, delta, P.e, P.f, v);
  });
}

bool grid_ok(int64_t blocks) { return blocks > 0 && blocks <= 0x7FFFFFFFll; }

}  // namespace

void batch_block_counts(int m, int n, int k, int kp, bool fast, int64_t (&nb)[kBatchKernels]) {
  const int64_t gx = (n + 255) / 256;
  nb[kBkScaleRows] = (m + 7) / 8;
  nb[kBkColmax] = gx * ((k + kColRows - 1) / kColRows);
  nb[kBkScaleCols] = gx * (kp / 32);
  nb[kBkSumsq] = fast ? gx : 0;
  nb[kBkExponents] = (static_cast<int64_t>(m) + n + 255) / 256;
  nb[kBkResidRows] = (resid_rows_items(m, kp) + 127) / 128;  // up to 16 items per warp
  // one block per tile of the column residue kernel
  nb[kBkResidCols] = static_cast<int64_t>((n + kResidTileCols - 1) / kResidTileCols) *
                     ((kp + kResidTileK - 1) / kResidTileK);
  nb[kBkCrt] = (static_cast<int64_t>(m) * ((n + 1) / 2) + 4095) / 4096;  // up to 16 items per thread
}

cudaError_t launch_scale_batch(const BatchProblem* probs, int count, const int64_t (&total)[kBatchKernels],
                               bool fast, uint32_t* flags, cudaStream_t st, cudaStream_t st_cols) {
  for (int w : {int(kBkScaleRows), int(kBkColmax), int(kBkScaleCols), int(kBkExponents)})
    if (!grid_ok(total[w])) return cudaErrorInvalidValue;
  if (fast && !grid_ok(total[kBkSumsq])) return cudaErrorInvalidValue;
  const int64_t tr = total[kBkScaleRows], tm = total[kBkColmax], tc = total[kBkScaleCols];
  if (fast)
    scale_rows_batch<true><<<grouped_grid(tr, 8), 256, 0, st>>>(probs, count, tr, flags);
  else
    scale_rows_batch<false><<<grouped_grid(tr, 8), 256, 0, st>>>(probs, count, tr, flags);
  colmax_batch<<<grouped_grid(tm, 8), 256, 0, st_cols>>>(probs, count, tm);
  if (fast) {
    scale_cols_batch<true><<<grouped_grid(tc, 8), 256, 0, st_cols>>>(probs, count, tc, flags);
    sumsq_batch<<<grouped_grid(total[kBkSumsq], 8), 256, 0, st_cols>>>(probs, count, total[kBkSumsq]);
  } else {
    scale_cols_batch<false><<<grouped_grid(tc, 8), 256, 0, st_cols>>>(probs, count, tc, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_exponents_batch(const BatchProblem* probs, int count, int64_t total_blocks, float pprime,
                                   float delta, cudaStream_t st) {
  if (!grid_ok(total_blocks)) return cudaErrorInvalidValue;
  exponents_batch<<<grouped_grid(total_blocks, 8), 256, 0, st>>>(probs, count, total_blocks, pprime, delta);
  return cudaGetLastError();
}

cudaError_t launch_scale_rows(const double* A, int64_t lda, int m, int k, int kp, int32_t* eprime,
                              uint8_t* rowstat, uint8_t* Abar, float* sq, bool fast, uint32_t* flags,
                              cudaStream_t st) {
  const int rows_per_block = 8;
  const int grid = (m + rows_per_block - 1) / rows_per_block;
  if (fast)
    scale_rows_kernel<true><<<grid, 256, 0, st>>>(A, lda, m, k, kp, eprime, rowstat, Abar, sq, flags);
  else
    scale_rows_kernel<false><<<grid, 256, 0, st>>>(A, lda, m, k, kp, eprime, rowstat, Abar, sq, flags);
  return cudaGetLastError();
}

cudaError_t launch_colmax(const double* B, int64_t ldb, int k, int n, uint32_t* colmax,
                          uint32_t* colbad, cudaStream_t st) {
  // rows per block: enough blocks for about four per SM, 16 to kColRows rows each
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t gx = (n + 255) / 256;
  int64_t rpb = (static_cast<int64_t>(k) * gx + 4 * sms - 1) / (4 * sms);
  rpb = std::min<int64_t>(kColRows, std::max<int64_t>(16, (rpb + 15) / 16 * 16));
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>((k + rpb - 1) / rpb));
  colmax_kernel<<<grid, 256, 0, st>>>(B, ldb, k, n, colmax, colbad, static_cast<int>(rpb));
  return cudaGetLastError();
}

cudaError_t launch_scale_cols(const double* B, int64_t ldb, int k, int n, int kp,
                              const uint32_t* colmax, const uint32_t* colbad,
                              int32_t* fprime, uint8_t* colstat, uint8_t* BbarT, float* part, float* sq,
                              bool fast, uint32_t* flags, cudaStream_t st) {
  dim3 grid((n + 255) / 256, kp / 32);
  if (fast) {
    scale_cols_kernel<true><<<grid, 256, 0, st>>>(B, ldb, k, n, kp, colmax, colbad, fprime, colstat, BbarT, part,
                                                  flags);
    sumsq_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, kp / 32, n, sq);
  } else {
    scale_cols_kernel<false><<<grid, 256, 0, st>>>(B, ldb, k, n, kp, colmax, colbad, fprime, colstat, BbarT,
                                                   part, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_exponents(int m, int n, const int32_t* eprime, const int32_t* fprime,
                             const uint8_t* rowstat, const uint8_t* colstat, const float* R,
                             const float* S, float pprime, float delta, int32_t* e, int32_t* f,
                             cudaStream_t st) {
  const int total = m + n;
  exponents_kernel<<<(total + 255) / 256, 256, 0, st>>>(m, n, eprime, fprime, rowstat, colstat, R, S,
                                                        pprime, delta, e, f);
  return cudaGetLastError();
}

cudaError_t launch_reuse_exponents(int m, const int32_t* gp, const uint8_t* rstat, const float* R, int32_t* g, int n,
                                   const int32_t* hp, const uint8_t* cstat, const float* S, int32_t* h, float q,
                                   uint32_t* flags, cudaStream_t st) {
  const int total = m + n;
  if (total <= 0) return cudaSuccess;
  reuse_exponents_kernel<<<(total + 255) / 256, 256, 0, st>>>(m, gp, rstat, R, g, n, hp, cstat, S, h, q, flags);
  return cudaGetLastError();
}

}  // namespace ozk2
