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
// a' is never materialised as a wide integer or a double: with a = M 2^E (M the
// 53-bit significand) and t = E + e, a' = M' 2^t' where M' = M >> -t, t' = 0 if t < 0
// and M' = M, t' = t otherwise.  Then
//   a' mod p = (sum_j c_j (2^16j mod p)) * (2^t' mod p)  mod p,
// with c_j the 16-bit pieces of M' and 2^t' mod p read from a per-modulus table.
// Every partial value stays below 2^28.1, where the float-estimated remainder of
// smod_i32 is exact.
//
// Rows of A produce K-major planes directly.  Columns of B are written transposed
// (plane rows are columns of B), so both operands of the tensor-core products are
// K-major.  Each thread owns 16 elements: it decodes them once into two registers
// each, then loops over the moduli.
#include <cuda_fp8.h>

#include "device.cuh"

namespace ozk2 {
namespace {

constexpr unsigned long long kAbsMask = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

// Packed element: x = bits 0..31 of M', y = bits 32..52 of M' | t' << 21 | sign << 31.
__device__ __forceinline__ uint2 encode_element(double a, int e, bool& range_err) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(a));
  const unsigned long long mag = bits & kAbsMask;
  uint2 r = make_uint2(0u, 0u);
  if (mag == 0 || mag >= kInfBits) return r;
  const int be = static_cast<int>(mag >> 52);
  unsigned long long M;
  int E;
  if (be == 0) {
    M = mag;
    E = -1074;
  } else {
    M = (mag & ((1ull << 52) - 1)) | (1ull << 52);
    E = be - 1075;
  }
  const int t = E + e;
  unsigned long long Mp;
  int tp;
  if (t >= 0) {
    Mp = M;
    tp = t;
  } else {
    Mp = (t <= -64) ? 0ull : (M >> (-t));
    tp = 0;
  }
  if (Mp == 0) return r;
  if (tp >= kPow2Table) {
    range_err = true;
    return r;
  }
  r.x = static_cast<uint32_t>(Mp);
  r.y = static_cast<uint32_t>(Mp >> 32) | (static_cast<uint32_t>(tp) << 21) |
        (static_cast<uint32_t>(bits >> 63) << 31);
  return r;
}

struct ModConsts {
  int p, h, w1, w2, w3;
  float inv_p;
};

// Symmetric residue of the signed integer a' = +-M' 2^t' encoded in v.  The sign is
// applied before the reduction, so the result needs no correction afterwards.
__device__ __forceinline__ int residue_of(uint2 v, const ModConsts& c, const int16_t* pow2,
                                          bool use_pow2) {
  const uint32_t c0 = v.x & 0xFFFFu, c1 = v.x >> 16, c2 = v.y & 0xFFFFu, c3 = (v.y >> 16) & 0x1Fu;
  int x = static_cast<int>(c0 + c1 * static_cast<uint32_t>(c.w1) + c2 * static_cast<uint32_t>(c.w2) +
                           c3 * static_cast<uint32_t>(c.w3));  // < 2^28.1
  if (use_pow2) {
    const int tp = static_cast<int>((v.y >> 21) & 63u);
    x = smod_i32(x, c.p, c.h, c.inv_p) * static_cast<int>(pow2[tp]);  // |x| < 2^19.2
  }
  const int neg = -static_cast<int>(v.y >> 31);  // 0 or -1
  x = (x ^ neg) - neg;
  return smod_i32(x, c.p, c.h, c.inv_p);
}

// Digits of residue r as floats (exact small integers, never -0).
__device__ __forceinline__ void square_digits(int r, int s, float inv_s, float& d1, float& d2) {
  const float rf = static_cast<float>(r);
  d1 = __fadd_rn(rintf(rf * inv_s), 0.0f);
  d2 = fmaf(-static_cast<float>(s), d1, rf);
}
__device__ __forceinline__ void karatsuba_digits(int r, float& d1, float& d2, float& d3) {
  const float rf = static_cast<float>(r);
  d1 = copysignf(ceilf(fabsf(rf) * 0.0625f), rf);
  d2 = fmaf(-16.0f, d1, rf);
  d3 = d1 + d2;
}

__device__ __forceinline__ uint32_t e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return lo | (hi << 16);
}

struct ResidArgs {
  const double* X;
  int64_t ldx;
  int lines;  // rows of A or columns of B
  int k, kp;
  const int32_t* exps;
  uint8_t* planes;
  int64_t plane_stride;  // lines * kp
  uint32_t* flags;
};

__device__ __forceinline__ void load_table(const ModTable& mt, int16_t* pow2_s) {
  const int total = mt.N * kPow2Table;
  for (int i = threadIdx.x; i < total; i += blockDim.x)
    pow2_s[i] = mt.pow2[i / kPow2Table][i % kPow2Table];
  __syncthreads();
}

__device__ __forceinline__ ModConsts consts_of(const ModTable& mt, int l) {
  ModConsts c;
  c.p = mt.p[l];
  c.h = mt.half[l];
  c.w1 = mt.w16[l][1];
  c.w2 = mt.w16[l][2];
  c.w3 = mt.w16[l][3];
  c.inv_p = mt.inv_p[l];
  return c;
}

// Rows of A.  One warp covers 512 consecutive k of one row: lane l owns elements
// base + 128 g + 4 l + {0..3}, g = 0..3, so loads and 4-byte plane stores coalesce.
constexpr int kRowGroups = 4;
constexpr int kRowSpan = 128 * kRowGroups;

__global__ void __launch_bounds__(256) residues_rows_kernel(ResidArgs a,
                                                            const __grid_constant__ ModTable mt) {
  __shared__ int16_t pow2_s[kMaxModuli * kPow2Table];
  load_table(mt, pow2_s);
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int nkw = (a.kp + kRowSpan - 1) / kRowSpan;
  const int64_t items = static_cast<int64_t>(a.lines) * nkw;
  bool range_err = false;
  for (int64_t it = static_cast<int64_t>(blockIdx.x) * warps_per_block + (threadIdx.x >> 5);
       it < items; it += static_cast<int64_t>(gridDim.x) * warps_per_block) {
    const int row = static_cast<int>(it / nkw);
    const int base = static_cast<int>(it % nkw) * kRowSpan;
    const double* x = a.X + static_cast<int64_t>(row) * a.ldx;
    const int e = a.exps[row];
    uint2 v[4 * kRowGroups];
    uint32_t any_tp = 0;
#pragma unroll
    for (int g = 0; g < kRowGroups; ++g) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int h = base + g * 128 + lane * 4 + t;
        const double val = (h < a.k) ? __ldg(x + h) : 0.0;
        v[g * 4 + t] = encode_element(val, e, range_err);
        any_tp |= v[g * 4 + t].y & (63u << 21);
      }
    }
    const bool use_pow2 = __any_sync(0xffffffffu, any_tp != 0);
    uint8_t* rowp = a.planes + static_cast<int64_t>(row) * a.kp;
    for (int l = 0; l < mt.N; ++l) {
      const ModConsts c = consts_of(mt, l);
      const int16_t* pw = pow2_s + l * kPow2Table;
      uint8_t* pl = rowp + static_cast<int64_t>(mt.plane0[l]) * a.plane_stride;
      if (l < kNumSquares) {
        const int s = mt.s[l];
        const float inv_s = mt.inv_s[l];
#pragma unroll
        for (int g = 0; g < kRowGroups; ++g) {
          float d1[4], d2[4];
#pragma unroll
          for (int t = 0; t < 4; ++t)
            square_digits(residue_of(v[g * 4 + t], c, pw, use_pow2), s, inv_s, d1[t], d2[t]);
          const int h = base + g * 128 + lane * 4;
          if (h < a.kp) {
            *reinterpret_cast<uint32_t*>(pl + h) = e4m3x4(d1[0], d1[1], d1[2], d1[3]);
            *reinterpret_cast<uint32_t*>(pl + a.plane_stride + h) = e4m3x4(d2[0], d2[1], d2[2], d2[3]);
          }
        }
      } else {
#pragma unroll
        for (int g = 0; g < kRowGroups; ++g) {
          float d1[4], d2[4], d3[4];
#pragma unroll
          for (int t = 0; t < 4; ++t)
            karatsuba_digits(residue_of(v[g * 4 + t], c, pw, use_pow2), d1[t], d2[t], d3[t]);
          const int h = base + g * 128 + lane * 4;
          if (h < a.kp) {
            *reinterpret_cast<uint32_t*>(pl + h) = e4m3x4(d1[0], d1[1], d1[2], d1[3]);
            *reinterpret_cast<uint32_t*>(pl + a.plane_stride + h) = e4m3x4(d2[0], d2[1], d2[2], d2[3]);
            *reinterpret_cast<uint32_t*>(pl + 2 * a.plane_stride + h) = e4m3x4(d3[0], d3[1], d3[2], d3[3]);
          }
        }
      }
    }
  }
  if (range_err) atomicOr(a.flags, kFlagRange);
}

// Columns of B.  A warp covers 16 columns x 32 consecutive h: lanes 2jj and 2jj+1 take
// column j0 + jj, rows h0..h0+15 and h0+16..h0+31.  Loads read two 128-byte row
// segments per instruction; each lane pair writes one full 32-byte sector of row j of
// every plane.
__global__ void __launch_bounds__(256) residues_cols_kernel(ResidArgs a,
                                                            const __grid_constant__ ModTable mt) {
  __shared__ int16_t pow2_s[kMaxModuli * kPow2Table];
  load_table(mt, pow2_s);
  const int lane = threadIdx.x & 31;
  const int jj = lane >> 1, half = lane & 1;
  const int warps_per_block = blockDim.x >> 5;
  const int ncg = (a.lines + 15) / 16;  // column groups of 16
  const int nkb = a.kp / 32;
  const int64_t items = static_cast<int64_t>(ncg) * nkb;
  bool range_err = false;
  for (int64_t it = static_cast<int64_t>(blockIdx.x) * warps_per_block + (threadIdx.x >> 5);
       it < items; it += static_cast<int64_t>(gridDim.x) * warps_per_block) {
    const int hb = static_cast<int>(it / ncg);
    const int j = static_cast<int>(it % ncg) * 16 + jj;
    const bool active = j < a.lines;
    const int e = active ? a.exps[j] : 0;
    const int h0 = hb * 32 + half * 16;
    uint2 v[16];
    uint32_t any_tp = 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int h = h0 + t;
      const double val = (active && h < a.k) ? __ldg(a.X + static_cast<int64_t>(h) * a.ldx + j) : 0.0;
      v[t] = encode_element(val, e, range_err);
      any_tp |= v[t].y & (63u << 21);
    }
    const bool use_pow2 = __any_sync(0xffffffffu, any_tp != 0);
    uint8_t* colp = a.planes + static_cast<int64_t>(active ? j : 0) * a.kp + h0;
    for (int l = 0; l < mt.N; ++l) {
      const ModConsts c = consts_of(mt, l);
      const int16_t* pw = pow2_s + l * kPow2Table;
      uint8_t* pl = colp + static_cast<int64_t>(mt.plane0[l]) * a.plane_stride;
      if (l < kNumSquares) {
        const int s = mt.s[l];
        const float inv_s = mt.inv_s[l];
        uint32_t w1[4], w2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float d1[4], d2[4];
#pragma unroll
          for (int t = 0; t < 4; ++t)
            square_digits(residue_of(v[q * 4 + t], c, pw, use_pow2), s, inv_s, d1[t], d2[t]);
          w1[q] = e4m3x4(d1[0], d1[1], d1[2], d1[3]);
          w2[q] = e4m3x4(d2[0], d2[1], d2[2], d2[3]);
        }
        if (active) {
          *reinterpret_cast<uint4*>(pl) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
          *reinterpret_cast<uint4*>(pl + a.plane_stride) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        }
      } else {
        uint32_t w1[4], w2[4], w3[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float d1[4], d2[4], d3[4];
#pragma unroll
          for (int t = 0; t < 4; ++t)
            karatsuba_digits(residue_of(v[q * 4 + t], c, pw, use_pow2), d1[t], d2[t], d3[t]);
          w1[q] = e4m3x4(d1[0], d1[1], d1[2], d1[3]);
          w2[q] = e4m3x4(d2[0], d2[1], d2[2], d2[3]);
          w3[q] = e4m3x4(d3[0], d3[1], d3[2], d3[3]);
        }
        if (active) {
          *reinterpret_cast<uint4*>(pl) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
          *reinterpret_cast<uint4*>(pl + a.plane_stride) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
          *reinterpret_cast<uint4*>(pl + 2 * a.plane_stride) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
        }
      }
    }
  }
  if (range_err) atomicOr(a.flags, kFlagRange);
}

int grid_for(int64_t work_items, int per_block) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (work_items + per_block - 1) / per_block;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_residues_rows(const double* A, int64_t lda, int m, int k, int kp,
                                 const int32_t* e, const ModTable& mt, uint8_t* planes,
                                 uint32_t* flags, cudaStream_t st) {
  ResidArgs a{A, lda, m, k, kp, e, planes, static_cast<int64_t>(m) * kp, flags};
  const int64_t warps = static_cast<int64_t>(m) * ((kp + kRowSpan - 1) / kRowSpan);
  residues_rows_kernel<<<grid_for(warps, 8), 256, 0, st>>>(a, mt);
  return cudaGetLastError();
}

cudaError_t launch_residues_cols(const double* B, int64_t ldb, int k, int n, int kp,
                                 const int32_t* f, const ModTable& mt, uint8_t* planes,
                                 uint32_t* flags, cudaStream_t st) {
  ResidArgs a{B, ldb, n, k, kp, f, planes, static_cast<int64_t>(n) * kp, flags};
  const int64_t warps = static_cast<int64_t>((n + 15) / 16) * (kp / 32);
  residues_cols_kernel<<<grid_for(warps, 8), 256, 0, st>>>(a, mt);
  return cudaGetLastError();
}

}  // namespace ozk2
