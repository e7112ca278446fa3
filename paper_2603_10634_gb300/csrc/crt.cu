// CRT reconstruction and inverse scaling, Sec. II of the paper (Eqs. CRT_finalreduction
// and inversescaling; workflow steps 9-10 of Sec. IV-B).
//
//   C'_ij = mod(sum_l w_l C'_l,ij, P),  w_l = q_l P / p_l,  symmetric in [-P/2, P/2)
//   C_ij  = RN(C'_ij 2^-(e_i + f_j))
//
// The sum is formed exactly in integer arithmetic: with u_l = C'_l mod p_l in [0, p_l),
// limb t of sum_l u_l w_l is accumulated in a 64-bit integer (each term < 2^43, N <= 20
// terms), the quotient Q = round(V / P) is estimated in FP32 from sum_l u_l (w_l / P)
// (error < 0.05), V - Q P is normalised to L signed 32-bit limbs and corrected once
// into [-P/2, P/2).  The double is then assembled bit by bit with round-to-nearest-even
// at the right position, which gives the correctly rounded value including gradual
// underflow and overflow to infinity.  No FP64 arithmetic is used.
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
__device__ __forceinline__ double crt_finish(int64_t (&acc)[L], float est, int scale, bool nan_out,
                                             const CrtTable& ct) {
  const int64_t q = static_cast<int64_t>(__float2int_rn(est));
#pragma unroll
  for (int t = 0; t < L; ++t) acc[t] -= q * static_cast<int64_t>(ct.P[t]);
  uint32_t v[L];
  int64_t carry = 0;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const int64_t x = acc[t] + carry;
    v[t] = static_cast<uint32_t>(x);
    carry = x >> 32;  // arithmetic shift: signed carry
  }
  // |v| < 0.55 P here; one correction brings it into [-P/2, P/2)
  {
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
  int nbits = 0;
#pragma unroll
  for (int t = L - 1; t >= 0; --t)
    if (nbits == 0 && v[t] != 0) nbits = 32 * t + 32 - __clz(v[t]);
  if (nbits == 0) return 0.0;
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

// Thread (row i, 4 consecutive columns).
template <int L>
__global__ void __launch_bounds__(256) crt_kernel(const int16_t* __restrict__ cres, int64_t ldr,
                                                  int64_t rstride, int m, int n,
                                                  const int32_t* __restrict__ e,
                                                  const int32_t* __restrict__ f,
                                                  const uint8_t* __restrict__ rowstat,
                                                  const uint8_t* __restrict__ colstat,
                                                  double* __restrict__ C, int64_t ldc,
                                                  const __grid_constant__ CrtTable ct) {
  const int nq = (n + 3) >> 2;
  const int64_t total = static_cast<int64_t>(m) * nq;
  for (int64_t it = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; it < total;
       it += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(it / nq);
    const int j0 = static_cast<int>(it % nq) * 4;
    int64_t acc[4][L];
    float est[4];
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      est[z] = 0.0f;
#pragma unroll
      for (int t = 0; t < L; ++t) acc[z][t] = 0;
    }
    const int16_t* src = cres + static_cast<int64_t>(i) * ldr + j0;
    for (int l = 0; l < ct.N; ++l) {
      const uint2 raw = *reinterpret_cast<const uint2*>(src + static_cast<int64_t>(l) * rstride);
      const int p = ct.p[l];
      const int cz[4] = {static_cast<int16_t>(raw.x & 0xFFFFu), static_cast<int16_t>(raw.x >> 16),
                         static_cast<int16_t>(raw.y & 0xFFFFu), static_cast<int16_t>(raw.y >> 16)};
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const uint32_t u = static_cast<uint32_t>(cz[z] < 0 ? cz[z] + p : cz[z]);
#pragma unroll
        for (int t = 0; t < L; ++t) acc[z][t] += static_cast<int64_t>(static_cast<uint64_t>(u) * ct.w[l][t]);
        est[z] = fmaf(static_cast<float>(u), ct.frac[l], est[z]);
      }
    }
    const int ei = e[i];
    const bool rbad = rowstat != nullptr && (rowstat[i] & kLineNonfinite);
    double* out = C + static_cast<int64_t>(i) * ldc;
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int j = j0 + z;
      if (j < n) {
        const bool bad = rbad || (colstat != nullptr && (colstat[j] & kLineNonfinite));
        out[j] = crt_finish<L>(acc[z], est[z], ei + f[j], bad, ct);
      }
    }
  }
}

template <int L>
cudaError_t launch_L(const int16_t* cres, int64_t ldr, int64_t rs, int m, int n, const int32_t* e,
                     const int32_t* f, const uint8_t* rowstat, const uint8_t* colstat, double* C,
                     int64_t ldc, const CrtTable& ct, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t threads = static_cast<int64_t>(m) * ((n + 3) / 4);
  int64_t blocks = (threads + 255) / 256;
  if (blocks > static_cast<int64_t>(sms) * 16) blocks = static_cast<int64_t>(sms) * 16;
  if (blocks < 1) blocks = 1;
  crt_kernel<L><<<static_cast<int>(blocks), 256, 0, st>>>(cres, ldr, rs, m, n, e, f, rowstat, colstat,
                                                         C, ldc, ct);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_crt(const int16_t* cres, int64_t ldr, int64_t res_stride, int m, int n,
                       const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                       const uint8_t* colstat, double* C, int64_t ldc, const CrtTable& ct,
                       cudaStream_t st) {
  switch (ct.limbs) {
    case 1:
    case 2:
    case 3:
    case 4:
      return launch_L<4>(cres, ldr, res_stride, m, n, e, f, rowstat, colstat, C, ldc, ct, st);
    case 5:
      return launch_L<5>(cres, ldr, res_stride, m, n, e, f, rowstat, colstat, C, ldc, ct, st);
    case 6:
      return launch_L<6>(cres, ldr, res_stride, m, n, e, f, rowstat, colstat, C, ldc, ct, st);
    default:
      return launch_L<7>(cres, ldr, res_stride, m, n, e, f, rowstat, colstat, C, ldc, ct, st);
  }
}

}  // namespace ozk2
