// FP8 tensor-core products of the method on tcgen05 (sm_103a), one kernel, three
// epilogues:
//
//   residue : for modulus l and an output tile, three products into three TMEM
//             accumulators, then C'_l = mod(., p_l) in registers and an int16 store.
//               square p = s^2 : X = A1 B2, Y = A2 B1, Z = A2 B2,
//                                C'_l = mod(s (X + Y) + Z, p)     [Eq. 3matmult-notKaratsuba]
//               Karatsuba      : Dx = Ax Bx (x = 1, 2, 3),
//                                C'_l = mod(256 D1 + D2 + 16 (D3 - D1 - D2), p)
//                                     = mod(16 mod(15 D1 + D3 - D2, p) + D2, p)  [Eq. C'-Karatsuba]
//             Every accumulator holds one product over at most 2^16 terms of digits
//             |d| <= 16, so its FP32 value is an exact integer of magnitude <= 2^24
//             (Eq. error-free-FP8-matmult).  Longer reductions are split into 2^16
//             blocks whose residues are added mod p.
//   bound   : Cbar = RU((1 + k 2^-24) Abar Bbar) folded into row / column maxima
//             (Eq. barCupper); Cbar itself is never stored.
//   raw     : D = A B^T in FP32 (a parity hook for the tensor-core path).
//
// Structure: persistent CTAs (one per SM), 192 threads in three roles.
//   warp 0      TMA producer: 128 x 128 byte tiles of A and B^T (K-major, 128-byte
//               swizzle) into a 6-stage shared-memory ring, mbarrier complete_tx.
//   warp 1      TMEM allocation (512 columns) and the single MMA-issuing thread:
//               tcgen05.mma kind::f8f6f4, M = N = 128, K = 32 per instruction.
//   warps 2-5   epilogue: tcgen05.ld of their TMEM lane quadrant, integer math,
//               global stores.
// Every wait is bounded (device.cuh); a wait that gives up raises a CTA-wide abort
// flag and the global timeout flag, drains the copies and products this CTA has in
// flight, frees TMEM and returns.
#include "device.cuh"

namespace ozk2 {
namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 128;  // bytes = FP8 elements per k-step (one 128-byte swizzle row)
constexpr int kStages = 6;
constexpr int kTileBytes = BM * BK;  // 16 KiB (BN == BM)
constexpr int kStageBytes = 2 * kTileBytes;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr int kChunk = 65536;  // exactness block of the residue products
constexpr int kGroupM = 8;     // tile rasterisation: bands of 8 tile rows
constexpr size_t kSmemBytes = 1024 + static_cast<size_t>(kStages) * kStageBytes + 256;

struct EpiMod {
  int p[kMaxModuli];
  int half[kMaxModuli];
  int s[kMaxModuli];
  float inv_p[kMaxModuli];
};

struct GemmParams {
  int m, n, k;
  int tiles_m, tiles_n, tiles;
  int num_units;
  int kchunks;
  int chunk_len;
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
};

__device__ __forceinline__ void decode_unit(const GemmParams& P, int u, int& mod, int& tm, int& tn) {
  mod = u / P.tiles;
  const int t = u - mod * P.tiles;
  const int per_group = kGroupM * P.tiles_n;
  const int g = t / per_group;
  const int first_m = g * kGroupM;
  const int gsz = min(P.tiles_m - first_m, kGroupM);
  const int r = t - g * per_group;
  tm = first_m + r % gsz;
  tn = r / gsz;
}

// Digit planes of product x of modulus `mod` (plane layout of the residue kernels).
__device__ __forceinline__ void planes_of(int mode, int mod, int x, int& pa, int& pb) {
  if (mode != kModeResidue) {
    pa = pb = 0;
  } else if (mod < kNumSquares) {
    const int a0 = 2 * mod;  // (A1, B2), (A2, B1), (A2, B2)
    pa = (x == 0) ? a0 : a0 + 1;
    pb = (x == 1) ? a0 : a0 + 1;
  } else {
    pa = pb = 12 + 3 * (mod - kNumSquares) + x;  // (Ax, Bx)
  }
}

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

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    fp8_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ GemmParams prm) {
  constexpr int NPROD = (MODE == kModeResidue) ? 3 : 1;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* tiles = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;
  uint64_t* tempty = tfull + 1;
  uint64_t* done = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4 * 32);
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
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
      for (int u = blockIdx.x; ok && u < prm.num_units; u += gridDim.x) {
        int mod, tm, tn;
        decode_unit(prm, u, mod, tm, tn);
        for (int c = 0; ok && c < prm.kchunks; ++c) {
          const int k0 = c * prm.chunk_len;
          const int k1 = min(prm.k, k0 + prm.chunk_len);
          const int ksteps = (k1 - k0 + BK - 1) / BK;
          for (int s = 0; ok && s < ksteps; ++s) {
#pragma unroll
            for (int x = 0; x < NPROD; ++x) {
              if (!mbar_wait_bounded(empty + stage, phase ^ 1u, abort_flag)) {
                ok = false;
                break;
              }
              int pa, pb;
              planes_of(MODE, mod, x, pa, pb);
              uint8_t* dst = tiles + stage * kStageBytes;
              mbar_arrive_expect_tx(full + stage, kStageBytes);
              tma_load_3d(dst, &tmA, full + stage, k0 + s * BK, tm * BM, pa);
              tma_load_3d(dst + kTileBytes, &tmB, full + stage, k0 + s * BK, tn * BN, pb);
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
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.flags, kFlagTimeout);
        // let the copies this thread issued land before the CTA exits
        int no_abort = 0;
        for (int s = 0; s < kStages; ++s)
          if (issued & (1u << s)) mbar_wait_bounded(full + s, (issued_phase >> s) & 1u, &no_abort);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = fp8_idesc(BM, BN);
      int stage = 0;
      uint32_t phase = 0, rc = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < prm.num_units; u += gridDim.x) {
        for (int c = 0; ok && c < prm.kchunks; ++c) {
          if (!mbar_wait_bounded(tempty, (rc & 1u) ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int k0 = c * prm.chunk_len;
          const int k1 = min(prm.k, k0 + prm.chunk_len);
          const int ksteps = (k1 - k0 + BK - 1) / BK;
          for (int s = 0; ok && s < ksteps; ++s) {
#pragma unroll
            for (int x = 0; x < NPROD; ++x) {
              if (!mbar_wait_bounded(full + stage, phase, abort_flag)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_addr(tiles + stage * kStageBytes);
              const uint64_t adesc = sw128_kmajor_desc(sa);
              const uint64_t bdesc = sw128_kmajor_desc(sa + kTileBytes);
              const uint32_t dtm = tmem_base + static_cast<uint32_t>(x * BN);
#pragma unroll
              for (int kk = 0; kk < BK / 32; ++kk)
                mma_fp8(dtm, adesc + 2ull * kk, bdesc + 2ull * kk, idesc, (s | kk) != 0 ? 1u : 0u);
              mma_commit(empty + stage);
              if (++stage == kStages) {
                stage = 0;
                phase ^= 1u;
              }
            }
          }
          if (ok) mma_commit(tfull);
          ++rc;
        }
      }
      // every product issued here must be complete before TMEM is released
      mma_commit(done);
      int no_abort = 0;
      mbar_wait_bounded(done, 0, &no_abort);
      if (!ok) {
        *abort_flag = 1;
        atomicOr(prm.flags, kFlagTimeout);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int row = q * 32 + lane;
    const uint32_t tq = tmem_base + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t rc = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < prm.num_units; u += gridDim.x) {
      int mod, tm, tn;
      decode_unit(prm, u, mod, tm, tn);
      const int gi = tm * BM + row;
      for (int c = 0; ok && c < prm.kchunks; ++c) {
        ok = mbar_wait_bounded(tfull, rc & 1u, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        if constexpr (MODE == kModeResidue) {
          const int p = prm.mod.p[mod], h = prm.mod.half[mod], sq = prm.mod.s[mod];
          const float ip = prm.mod.inv_p[mod];
          const bool square = mod < kNumSquares;
          int16_t* dst = prm.cres + static_cast<int64_t>(mod) * prm.res_stride +
                         static_cast<int64_t>(gi) * prm.ldr;
#pragma unroll 1
          for (int cb = 0; cb < BN / 32; ++cb) {
            uint32_t v0[32], v1[32], v2[32];
            tmem_ld_32cols(tq + cb * 32, v0);
            tmem_ld_32cols(tq + BN + cb * 32, v1);
            tmem_ld_32cols(tq + 2 * BN + cb * 32, v2);
            tmem_ld_wait();
            const int gc = tn * BN + cb * 32;
            int res[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int a = __float2int_rn(__uint_as_float(v0[j]));
              const int b = __float2int_rn(__uint_as_float(v1[j]));
              const int d = __float2int_rn(__uint_as_float(v2[j]));
              int r;
              if (square) {
                r = smod_i32(sq * (a + b) + d, p, h, ip);
              } else {
                const int t = smod_i32(15 * a + d - b, p, h, ip);
                r = smod_i32(16 * t + b, p, h, ip);
              }
              res[j] = r;
            }
            if (gi < prm.m) {
              if (gc + 32 <= prm.n) {
                uint4* o = reinterpret_cast<uint4*>(dst + gc);
                if (c > 0) {
#pragma unroll
                  for (int w = 0; w < 4; ++w) {
                    const uint4 pv = o[w];
                    const uint32_t pr[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
                    for (int z = 0; z < 4; ++z) {
                      res[w * 8 + 2 * z] = smod_small(res[w * 8 + 2 * z] + static_cast<int16_t>(pr[z] & 0xFFFFu), p, h);
                      res[w * 8 + 2 * z + 1] = smod_small(res[w * 8 + 2 * z + 1] + static_cast<int16_t>(pr[z] >> 16), p, h);
                    }
                  }
                }
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                  uint32_t pk[4];
#pragma unroll
                  for (int z = 0; z < 4; ++z)
                    pk[z] = (static_cast<uint32_t>(res[w * 8 + 2 * z]) & 0xFFFFu) |
                            (static_cast<uint32_t>(res[w * 8 + 2 * z + 1]) << 16);
                  o[w] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  if (gc + j < prm.n) {
                    int r = res[j];
                    if (c > 0) r = smod_small(r + dst[gc + j], p, h);
                    dst[gc + j] = static_cast<int16_t>(r);
                  }
                }
              }
            }
          }
        } else if constexpr (MODE == kModeBound) {
          float rmax = 0.0f;
#pragma unroll 1
          for (int cb = 0; cb < BN / 32; ++cb) {
            uint32_t v0[32];
            tmem_ld_32cols(tq + cb * 32, v0);
            tmem_ld_wait();
            const int gc = tn * BN + cb * 32;
            float cv[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float cb_ = __fmul_ru(prm.factor, __uint_as_float(v0[j]));
              cb_ = (gi < prm.m && gc + j < prm.n) ? cb_ : 0.0f;
              rmax = fmaxf(rmax, cb_);
              cv[j] = cb_;
            }
            const float cm = warp_column_max(cv, lane);
            if (gc + lane < prm.n && cm > 0.0f)
              atomicMax(reinterpret_cast<int*>(prm.S) + gc + lane, __float_as_int(cm));
          }
          if (gi < prm.m && rmax > 0.0f) atomicMax(reinterpret_cast<int*>(prm.R) + gi, __float_as_int(rmax));
        } else {
#pragma unroll 1
          for (int cb = 0; cb < BN / 32; ++cb) {
            uint32_t v0[32];
            tmem_ld_32cols(tq + cb * 32, v0);
            tmem_ld_wait();
            const int gc = tn * BN + cb * 32;
            if (gi < prm.m) {
              float* o = prm.D + static_cast<int64_t>(gi) * prm.ldd;
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (gc + j < prm.n) o[gc + j] = __uint_as_float(v0[j]);
            }
          }
        }
        tc_fence_before();
        mbar_arrive(tempty);
        ++rc;
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

template <int MODE>
cudaError_t launch_mode(const GemmParams& prm, const CUtensorMap& ta, const CUtensorMap& tb, int grid,
                        cudaStream_t st) {
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    cudaError_t err = cudaFuncSetAttribute(fp8_gemm_kernel<MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(kSmemBytes));
    if (err != cudaSuccess) return err;
    configured[dev] = true;
  }
  fp8_gemm_kernel<MODE><<<grid, kThreads, kSmemBytes, st>>>(ta, tb, prm);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp8_gemm(const GemmArgs& g, const uint8_t* a, int64_t lda8, int planes_a,
                            const uint8_t* b, int64_t ldb8, int planes_b, cudaStream_t st) {
  GemmParams prm{};
  prm.m = g.m;
  prm.n = g.n;
  prm.k = g.k;
  prm.tiles_m = (g.m + BM - 1) / BM;
  prm.tiles_n = (g.n + BN - 1) / BN;
  prm.tiles = prm.tiles_m * prm.tiles_n;
  const int nmod = (g.mode == kModeResidue) ? g.mt->N : 1;
  prm.num_units = prm.tiles * nmod;
  prm.chunk_len = (g.mode == kModeResidue) ? kChunk : ((g.k + BK - 1) / BK) * BK;
  prm.kchunks = (g.k + prm.chunk_len - 1) / prm.chunk_len;
  prm.cres = g.cres;
  prm.ldr = g.ldr;
  prm.res_stride = g.res_stride;
  if (g.mode == kModeResidue) {
    for (int l = 0; l < g.mt->N; ++l) {
      prm.mod.p[l] = g.mt->p[l];
      prm.mod.half[l] = g.mt->half[l];
      prm.mod.s[l] = g.mt->s[l];
      prm.mod.inv_p[l] = g.mt->inv_p[l];
    }
  }
  prm.factor = g.factor;
  prm.R = g.R;
  prm.S = g.S;
  prm.D = g.D;
  prm.ldd = g.ldd;
  prm.flags = g.flags;

  CUtensorMap ta, tb;
  if (!encode_fp8_map(&ta, a, g.k, g.m, planes_a, lda8, BM)) return cudaErrorInvalidValue;
  if (!encode_fp8_map(&tb, b, g.k, g.n, planes_b, ldb8, BN)) return cudaErrorInvalidValue;
  const int grid = prm.num_units < g.num_sms ? prm.num_units : g.num_sms;
  switch (g.mode) {
    case kModeResidue:
      return launch_mode<kModeResidue>(prm, ta, tb, grid, st);
    case kModeBound:
      return launch_mode<kModeBound>(prm, ta, tb, grid, st);
    default:
      return launch_mode<kModeRaw>(prm, ta, tb, grid, st);
  }
}

}  // namespace ozk2
