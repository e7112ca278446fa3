// CRT reconstruction and inverse scaling, Sec. II of the paper (Eqs. CRT_finalreduction
// and inversescaling; workflow steps 9-10 of Sec. IV-B).
//
//   C'_ij = mod(sum_l w_l C'_l,ij, P),  w_l = q_l P / p_l,  symmetric in [-P/2, P/2)
//   C_ij  = RN(C'_ij 2^-(e_i + f_j))
//
// The sum is formed exactly in integer arithmetic from the signed residues c_l in
// [-p_l/2, p_l/2): sum_l c_l w_l differs from the sum over the non-negative residues by
// multiples of p_l w_l = q_l P, so it is the same mod P.  The weights are split into
// balanced 32-bit limbs (each in [-2^31, 2^31)), and limb t of sum_l c_l w_l accumulates
// in a 64-bit integer (each term below 2^46 in magnitude, N <= 20 terms), one signed wide
// multiply-add per limb.  The quotient Q = round(V / P) comes from the fixed-point
// estimate sum_l c_l round(2^16 w_l / P) (error below 0.05); V - Q P is normalised to L
// signed 32-bit limbs.  When the estimate is at least 0.3 away from a rounding boundary
// the result is already in [-P/2, P/2); otherwise one exact comparison with +-P/2
// corrects it.  The double is then assembled bit by bit with round-to-nearest-even at the
// right position, which gives the correctly rounded value including gradual underflow
// and overflow to infinity: for a normal result from more than 53 bits (the common case)
// from a 96-bit window at the leading limb, otherwise bit by bit over all limbs.  No FP64
// arithmetic is used.
#include "device.cuh"

namespace ozk2 {
namespace {

template <int L>
__device__ __forceinline__ uint32_t limb_at(const uint32_t (&x)[L], int idx) {
  uint32_t r = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) r = (idx == t) ? x[t] : r;
  return r;
}

// x <- x + sign * y over L limbs (two's complement); returns nothing, wraps mod 2^32L.
template <int L>
__device__ __forceinline__ void add_limbs(uint32_t (&x)[L], const uint32_t* y, bool subtract) {
  uint64_t carry = subtract ? 1u : 0u;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const uint64_t yt = subtract ? static_cast<uint64_t>(~y[t]) : static_cast<uint64_t>(y[t]);
    const uint64_t s = static_cast<uint64_t>(x[t]) + (yt & 0xFFFFFFFFull) + carry;
    x[t] = static_cast<uint32_t>(s);
    carry = s >> 32;
  }
}

template <int L>
__device__ __forceinline__ bool is_negative(const uint32_t (&x)[L]) {
  return (x[L - 1] >> 31) != 0;
}

template <int L>
__device__ __forceinline__ double crt_finish(uint32_t (&v)[L], bool exact_check, int scale, bool nan_out,
                                             const CrtTable& ct) {
  // v = V - Q P in two's complement; |v| < 1.5 P.  Bring it into [-P/2, P/2).
  if (exact_check) {
    uint32_t tst[L];
#pragma unroll
    for (int t = 0; t < L; ++t) tst[t] = v[t];
    if (!is_negative<L>(v)) {
      add_limbs<L>(tst, ct.halfP, true);  // v - P/2 >= 0  ->  v -= P
      if (!is_negative<L>(tst)) add_limbs<L>(v, ct.P, true);
    } else {
      add_limbs<L>(tst, ct.halfP, false);  // v + P/2 < 0  ->  v += P
      if (is_negative<L>(tst)) add_limbs<L>(v, ct.P, false);
    }
  }
  if (nan_out) return __longlong_as_double(0x7FF8000000000000ll);
  const bool neg = is_negative<L>(v);
  if (neg) {  // magnitude
    uint64_t c = 1;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const uint64_t s = static_cast<uint64_t>(~v[t]) + c;
      v[t] = static_cast<uint32_t>(s);
      c = s >> 32;
    }
  }
  // the top nonzero limb, the two below it and whether anything lies lower still
  uint32_t top = 0u, mid = 0u, low = 0u, rest = 0u, below = 0u;  // below: OR of v[0 .. t - 3]
  int ti = -1;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    if (v[t] != 0u) {
      top = v[t];
      mid = t >= 1 ? v[t >= 1 ? t - 1 : 0] : 0u;
      low = t >= 2 ? v[t >= 2 ? t - 2 : 0] : 0u;
      rest = below;
      ti = t;
    }
    if (t >= 2) below |= v[t >= 2 ? t - 2 : 0];
  }
  if (ti < 0) return 0.0;
  const int nbits = 32 * ti + 32 - __clz(top);
  if (nbits > 53 && nbits - 53 >= scale - 1074) {
    // the common case, a normal result from more than 53 bits: the 96-bit window
    // (top : mid : low) shifted left to its leading one holds the 53 significand bits,
    // the round bit and most of the sticky bits
    const int sh = __clz(top);
    const uint32_t w2 = __funnelshift_l(mid, top, sh), w1 = __funnelshift_l(low, mid, sh), w0 = low << sh;
    uint64_t mant = (static_cast<uint64_t>(w2) << 21) | (w1 >> 11);
    const bool round_bit = (w1 >> 10) & 1u;
    const bool sticky = ((w1 & 0x3FFu) | w0 | rest) != 0u;
    if (round_bit && (sticky || (mant & 1ull))) mant += 1;
    const int ebias = nbits - 53 - scale + 1074;  // exponent field before the implicit bit
    uint64_t bits = (ebias >= 2047) ? 0x7FF0000000000000ull : (static_cast<uint64_t>(ebias) << 52) + mant;
    if ((bits >> 52) >= 2047) bits = 0x7FF0000000000000ull;
    if (neg) bits |= 0x8000000000000000ull;
    return __longlong_as_double(static_cast<long long>(bits));
  }
  // position (bit index of C') of the result's last significand bit
  const int rpos = max(nbits - 53, scale - 1074);
  uint64_t mant;
  if (rpos <= 0) {
    const uint64_t lo = static_cast<uint64_t>(v[0]) | (L > 1 ? (static_cast<uint64_t>(v[1 < L ? 1 : 0]) << 32) : 0ull);
    mant = lo << (-rpos);  // C' < 2^53 here: exact
  } else {
    const int w = rpos >> 5, sh = rpos & 31;
    const uint64_t two = static_cast<uint64_t>(limb_at<L>(v, w)) |
                         (static_cast<uint64_t>(limb_at<L>(v, w + 1)) << 32);
    mant = two >> sh;
    if (sh) mant |= static_cast<uint64_t>(limb_at<L>(v, w + 2)) << (64 - sh);
    const int rb = rpos - 1;  // round bit position
    const uint32_t round_bit = (limb_at<L>(v, rb >> 5) >> (rb & 31)) & 1u;
    bool sticky = false;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      const int lo_bit = 32 * t;
      if (lo_bit + 32 <= rb) sticky |= v[t] != 0;
      else if (lo_bit < rb) sticky |= (v[t] & ((1u << (rb - lo_bit)) - 1u)) != 0;
    }
    if (round_bit && (sticky || (mant & 1ull))) mant += 1;
  }
  const int ebias = rpos - scale + 1074;  // exponent field before the implicit bit
  uint64_t bits;
  if (ebias >= 2047) {
    bits = 0x7FF0000000000000ull;
  } else {
    bits = (static_cast<uint64_t>(ebias) << 52) + mant;
    if ((bits >> 52) >= 2047) bits = 0x7FF0000000000000ull;
  }
  if (neg) bits |= 0x8000000000000000ull;
  return __longlong_as_double(static_cast<long long>(bits));
}

// 32-bit limbs of the signed results for N moduli (bit length of P plus a sign bit,
// at least 4): N <= 13 -> 4, N <= 17 -> 5, N <= 20 -> 6.
__host__ __device__ constexpr int limbs_for(int N) { return N <= 13 ? 4 : (N <= 17 ? 5 : 6); }

// Thread (row i, 2 consecutive columns).  One instance per N, so the modulus loop is
// unrolled and the N residue loads of a thread can be issued together.
template <int N>
__device__ __forceinline__ void crt_body(const int16_t* __restrict__ cres, int64_t ldr, int64_t rstride, int m,
                                         int n, const int32_t* __restrict__ e, const int32_t* __restrict__ f,
                                         const uint8_t* __restrict__ rowstat, const uint8_t* __restrict__ colstat,
                                         double* __restrict__ C, int64_t ldc, const CrtTable& ct, int64_t vblock,
                                         int64_t vgrid) {
  constexpr int L = limbs_for(N);
  const int nq = (n + 1) >> 1;
  const int64_t total = static_cast<int64_t>(m) * nq;
  const int64_t stride = vgrid * blockDim.x;
  const int64_t first = vblock * blockDim.x + threadIdx.x;
  if (first >= total) return;
  // (row, column pair) of the item, advanced by the stride's own quotient and remainder
  // instead of a 64-bit division per item (the stride is at most a few grids of threads)
  int i, jq, di, dj;
  divmod_nonneg(first, nq, i, jq);
  divmod_nonneg(stride, nq, di, dj);
  for (; i < m; i += di, jq += dj) {
    if (jq >= nq) {
      jq -= nq;
      if (++i >= m) break;
    }
    const int j0 = jq * 2;
    const int16_t* src = cres + static_cast<int64_t>(i) * ldr + j0;
    // sum_l C'_l w_l with the signed residues: it differs from the sum over the residues
    // made non-negative by multiples of p_l w_l = q_l P, so it is the same mod P
    int64_t acc[2][L];
    int32_t est[2] = {0, 0};
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int t = 0; t < L; ++t) acc[z][t] = 0;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const uint32_t raw = __ldg(reinterpret_cast<const unsigned int*>(src + static_cast<int64_t>(l) * rstride));
      const int cz[2] = {static_cast<int16_t>(raw & 0xFFFFu), static_cast<int16_t>(raw >> 16)};
#pragma unroll
      for (int z = 0; z < 2; ++z) {
#pragma unroll
        for (int t = 0; t < L; ++t) acc[z][t] += static_cast<int64_t>(cz[z]) * ct.wb[l][t];
        est[z] += cz[z] * ct.frac16[l];
      }
    }
    const int ei = e[i];
    const bool rbad = rowstat != nullptr && (rowstat[i] & kLineNonfinite);
    double* out = C + static_cast<int64_t>(i) * ldc;
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      const int j = j0 + z;
      if (j < n) {
        // Q = round(est / 2^16); est / 2^16 is within 0.05 of V / P
        const int32_t q = (est[z] + 0x8000) >> 16;                  // arithmetic shift: floor
        const int32_t off = est[z] - q * 65536;                      // in [-2^15, 2^15)
        const bool exact_check = (off > 19660 || off < -19660);      // |est - Q| > 0.3
        // v = V - Q P from the 64-bit limb sums, normalised to 32-bit limbs
        uint32_t v[L];
        int64_t carry = 0;
#pragma unroll
        for (int t = 0; t < L; ++t) {
          const int64_t x = carry + acc[z][t] - static_cast<int64_t>(q) * static_cast<int64_t>(ct.P[t]);
          v[t] = static_cast<uint32_t>(x);
          carry = x >> 32;  // arithmetic: signed carry
        }
        const bool bad = rbad || (colstat != nullptr && (colstat[j] & kLineNonfinite));
        out[j] = crt_finish<L>(v, exact_check, ei + f[j], bad, ct);
      }
    }
  }
}

template <int N>
__global__ void __launch_bounds__(256, 2)
    crt_kernel(const int16_t* __restrict__ cres, int64_t ldr, int64_t rstride, int m, int n,
               const int32_t* __restrict__ e, const int32_t* __restrict__ f,
               const uint8_t* __restrict__ rowstat, const uint8_t* __restrict__ colstat,
               double* __restrict__ C, int64_t ldc, const __grid_constant__ CrtTable ct) {
  crt_body<N>(cres, ldr, rstride, m, n, e, f, rowstat, colstat, C, ldc, ct, blockIdx.x, gridDim.x);
}

template <int N>
__global__ void __launch_bounds__(256, 2)
    crt_batch(const BatchProblem* __restrict__ probs, int count, int64_t total, const __grid_constant__ CrtTable ct) {
  for_each_vblock(probs, count, kBkCrt, total, [&](const BatchProblem& P, int64_t v) {
    crt_body<N>(P.cres, P.ldr, static_cast<int64_t>(P.m) * P.ldr, P.m, P.n, P.e, P.f, P.rowstat, P.colstat, P.C,
                P.ldc, ct, v, P.nblocks[kBkCrt]);
  });
}

template <int N>
cudaError_t launch_N(const int16_t* cres, int64_t ldr, int64_t rs, int m, int n, const int32_t* e,
                     const int32_t* f, const uint8_t* rowstat, const uint8_t* colstat, double* C,
                     int64_t ldc, const CrtTable& ct, cudaStream_t st) {
  const int64_t threads = static_cast<int64_t>(m) * ((n + 1) / 2);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (threads + 255) / 256;
  if (blocks > static_cast<int64_t>(sms) * 16) blocks = static_cast<int64_t>(sms) * 16;
  if (blocks < 1) blocks = 1;
  crt_kernel<N><<<static_cast<int>(blocks), 256, 0, st>>>(cres, ldr, rs, m, n, e, f, rowstat, colstat, C, ldc, ct);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_batch_N(const BatchProblem* probs, int count, int64_t blocks, const CrtTable& ct,
                           cudaStream_t st) {
  crt_batch<N><<<grouped_grid(blocks, 8), 256, 0, st>>>(probs, count, blocks, ct);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_crt_batch(const BatchProblem* probs, int count, int64_t total_blocks, const CrtTable& ct,
                             cudaStream_t st) {
  if (ct.limbs > limbs_for(ct.N) || total_blocks < 1 || total_blocks > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  switch (ct.N) {
#define OZK2_CASE(nn) \
  case nn:            \
    return launch_batch_N<nn>(probs, count, total_blocks, ct, st);
    OZK2_CASE(1) OZK2_CASE(2) OZK2_CASE(3) OZK2_CASE(4) OZK2_CASE(5) OZK2_CASE(6) OZK2_CASE(7)
    OZK2_CASE(8) OZK2_CASE(9) OZK2_CASE(10) OZK2_CASE(11) OZK2_CASE(12) OZK2_CASE(13) OZK2_CASE(14)
    OZK2_CASE(15) OZK2_CASE(16) OZK2_CASE(17) OZK2_CASE(18) OZK2_CASE(19) OZK2_CASE(20)
#undef OZK2_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_crt(const int16_t* cres, int64_t ldr, int64_t res_stride, int m, int n,
                       const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                       const uint8_t* colstat, double* C, int64_t ldc, const CrtTable& ct,
                       cudaStream_t st) {
  if (ct.limbs > limbs_for(ct.N)) return cudaErrorInvalidValue;
  switch (ct.N) {
#define OZK2_CASE(nn) \
  case nn:            \
    return launch_N<nn>(cres, ldr, res_stride, m, n, e, f, rowstat, colstat, C, ldc, ct, st);
    OZK2_CASE(1) OZK2_CASE(2) OZK2_CASE(3) OZK2_CASE(4) OZK2_CASE(5) OZK2_CASE(6) OZK2_CASE(7)
    OZK2_CASE(8) OZK2_CASE(9) OZK2_CASE(10) OZK2_CASE(11) OZK2_CASE(12) OZK2_CASE(13) OZK2_CASE(14)
    OZK2_CASE(15) OZK2_CASE(16) OZK2_CASE(17) OZK2_CASE(18) OZK2_CASE(19) OZK2_CASE(20)
#undef OZK2_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ozk2
