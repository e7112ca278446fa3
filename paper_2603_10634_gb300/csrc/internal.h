// Internal declarations shared by the host code and the kernels of libozk2.
//
// Parameter blocks are passed to kernels by value (no __constant__ state), so calls
// with different N on different streams never interfere.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ozk2 {

constexpr int kMaxModuli = 20;
constexpr int kMaxLimbs = 8;    // 32-bit limbs of the CRT arithmetic (N <= 20 needs 6)
constexpr int kPow2Table = 64;  // 2^t mod p for t in [0, 64)
constexpr int kNumSquares = 6;  // squares lead the hybrid list (Sec. III-D)

// Device flag bits (a uint32 word in every workspace)
constexpr uint32_t kFlagTimeout = 1u;    // a bounded device wait gave up
constexpr uint32_t kFlagRange = 2u;      // a scaled value exceeded the supported range
constexpr uint32_t kFlagNonfinite = 4u;  // NaN / Inf input seen
constexpr uint32_t kFlagDebug = 8u;      // a range check of the debug build (OZK2_DEBUG) failed

// Line status bits (one byte per row of A / column of B)
constexpr uint8_t kLineZero = 1;       // no nonzero finite entry
constexpr uint8_t kLineNonfinite = 2;  // holds NaN or Inf

// Per-modulus constants for the residue, GEMM-epilogue and CRT kernels.
struct ModTable {
  int N;
  int num_planes;                 // M_N (Sec. IV-B Eq. M)
  int p[kMaxModuli];              // modulus
  int half[kMaxModuli];           // floor(p / 2)
  int s[kMaxModuli];              // sqrt(p) for squares, 16 for Karatsuba moduli
  int plane0[kMaxModuli];         // first digit plane of the modulus
  float inv_p[kMaxModuli];        // RN(1 / p)
  float inv_s[kMaxModuli];        // RN(1 / s)
  float w11[kMaxModuli][5];       // 2^(11 j) mod p, symmetric representative, j = 0..4
  int16_t pow2[kMaxModuli][kPow2Table];  // 2^t mod p, symmetric representative
  // The residue kernels' constants as duplicated FP32 pairs (they work on element
  // pairs): -p, RN(1/p), -s, RN(1/s) and w11.
  float2 neg_p2[kMaxModuli], inv_p2[kMaxModuli], neg_s2[kMaxModuli], inv_s2[kMaxModuli];
  float2 w2[kMaxModuli][5];
};

struct CrtTable {
  int N;
  int limbs;                               // L, 32-bit limbs of the signed result
  int p[kMaxModuli];
  int32_t wb[kMaxModuli][kMaxLimbs];       // w_l = q_l P / p_l mod P in balanced 32-bit limbs:
                                           // w_l = sum_t wb[l][t] 2^(32 t), wb in [-2^31, 2^31)
  int32_t frac16[kMaxModuli];              // round(2^16 w_l / P) (quotient estimate)
  uint32_t P[kMaxLimbs];
  uint32_t halfP[kMaxLimbs];               // P / 2 (P is even: 1024 is a modulus)
};

// Row pitch in bytes of the digit planes for kp (a multiple of 32) bytes of data per row.
// Packed: rows padded away from power-of-two pitches measured no change in the DRAM
// traffic of the residue products (the L2 hashes such strides well).
__host__ __device__ inline int64_t plane_pitch(int64_t kp) { return kp; }

// Host-side fault injection and the device wait limit (api.cu).  A fault kind is armed
// by ozk2_debug_inject_fault or the OZK2_FAULT environment variable and fires once.
enum FaultKind { kFaultNone = 0, kFaultAlloc = 1, kFaultLaunch = 2, kFaultStall = 3 };
bool take_fault(int kind);        // true (and disarmed) if `kind` is the armed fault
unsigned long long wait_limit_ns();

// Entry points for ozk2_dgemm_noalloc (api.cu), returning ozk2_status codes: the argument
// checks of ozk2_dgemm, and ozk2_dgemm_ws in a workspace of this library (whose memory
// type needs no check).
int validate_dgemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                   const double* C, int64_t ldc, int N);
int dgemm_library_ws(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double* C, int64_t ldc, int N, void* ws, size_t ws_bytes, cudaStream_t st);

// Host-side constant generation (moduli.cpp)
bool build_mod_table(int N, ModTable* mt);
bool build_crt_table(int N, CrtTable* ct);
int hybrid_moduli(int N, int* out);  // returns N or -1
float p_prime_f32(int N);            // RD_fp32((log2(P - 1) - 1) / 2)
float delta_f32();                   // RD_fp32(-1 / (2 - 2^-21))
float reuse_budget_f32(int N);       // RD_fp32(log2(P - 1) - 1), the budget of one side
float bound_factor_f32(int64_t k);   // RU_fp32(1 + k 2^-24)

// ---------------------------------------------------------------------------
// Kernel launchers (each returns the cudaError_t of its launch)
// ---------------------------------------------------------------------------

// scale.cu.  "rows": lines contiguous along k; "cols": lines strided along k.  With
// fast = true the kernels write sums of squares (sq) instead of bound operands.
cudaError_t launch_scale_rows(const double* A, int64_t lda, int m, int k, int kp,
                              int32_t* eprime, uint8_t* rowstat, uint8_t* Abar, float* sq,
                              bool fast, uint32_t* flags, cudaStream_t st);
// colmax: per column, floor(log2 max |b|) + 1075 (0 for a zero column), accumulated
// with atomicMax into a zeroed array.
cudaError_t launch_colmax(const double* B, int64_t ldb, int k, int n,
                          uint32_t* colmax, uint32_t* colbad, cudaStream_t st);
cudaError_t launch_scale_cols(const double* B, int64_t ldb, int k, int n, int kp,
                              const uint32_t* colmax, const uint32_t* colbad,
                              int32_t* fprime, uint8_t* colstat, uint8_t* BbarT, float* part,
                              float* sq, bool fast, uint32_t* flags, cudaStream_t st);
cudaError_t launch_exponents(int m, int n, const int32_t* eprime, const int32_t* fprime,
                             const uint8_t* rowstat, const uint8_t* colstat,
                             const float* R, const float* S, float pprime, float delta,
                             int32_t* e, int32_t* f, cudaStream_t st);
// Exponents of dC's rows (g from R) and columns (h from S) for the gradient products
// that reuse the forward's integer matrices: the whole budget q = reuse_budget_f32(N).
cudaError_t launch_reuse_exponents(int m, const int32_t* gp, const uint8_t* rstat, const float* R, int32_t* g, int n,
                                   const int32_t* hp, const uint8_t* cstat, const float* S, int32_t* h, float q,
                                   uint32_t* flags, cudaStream_t st);

// resid.cu.  Planes: M_N planes of lines x kp bytes, row pitch ldp bytes (>= kp, a
// multiple of 16), plane stride plane_stride bytes (0: lines * ldp; larger when the
// lines converted are a slice of a taller operand).
cudaError_t launch_residues_rows(const double* A, int64_t lda, int m, int k, int kp, int64_t ldp,
                                 const int32_t* e, const ModTable& mt, uint8_t* planes,
                                 uint32_t* flags, cudaStream_t st, int64_t plane_stride = 0);
cudaError_t launch_residues_cols(const double* B, int64_t ldb, int k, int n, int kp, int64_t ldp,
                                 const int32_t* f, const ModTable& mt, uint8_t* planes,
                                 uint32_t* flags, cudaStream_t st, int64_t plane_stride = 0);

// Gradient operands (resid.cu): the digit planes of G'_ij = trunc(2^(g_i - f_j) dC_ij)
// (m lines along j, pitch ldg) and of H'_ij = trunc(2^(h_j - e_i) dC_ij) (n lines along i,
// pitch ldh) from one read of dC; a null plane pointer skips that output.
cudaError_t launch_grad_residues(const double* dC, int64_t lddc, int m, int n, const int32_t* g, const int32_t* f,
                                 const int32_t* h, const int32_t* e, uint8_t* planesG, int64_t ldg, uint8_t* planesH,
                                 int64_t ldh, const ModTable& mt, uint32_t* flags, cudaStream_t st);
// dst[p][x][y] = src[p][y][x], y < lines, x < len (pitches and strides multiples of 16;
// src_pitch >= len and dst_pitch >= lines, both rounded up to 16).
cudaError_t launch_transpose_planes(const uint8_t* src, int64_t src_pitch, int64_t src_stride, int lines, int len,
                                    uint8_t* dst, int64_t dst_pitch, int64_t dst_stride, int planes, cudaStream_t st);

// gemm.cu
enum GemmMode { kModeResidue = 0, kModeBound = 1, kModeRaw = 2 };

struct GemmArgs {
  int mode;
  int m, n, k;
  int num_sms;
  // residue products
  int16_t* cres;
  int64_t ldr;          // int16 elements per row of a residue plane
  int64_t res_stride;   // elements between residue planes
  const ModTable* mt;
  // bound product
  float factor;
  float* R;
  float* S;
  const int32_t* colshift;  // optional: maxima of cbar_ij 2^-colshift_j (single problems)
  const int32_t* rowshift;  // optional: maxima of cbar_ij 2^-rowshift_i
  // raw product
  float* D;
  int64_t ldd;
  uint32_t* flags;
  // bytes between digit planes of A / B; 0 means rows * row stride (packed planes).  A
  // row block of a larger plane set passes the full set's plane stride.
  int64_t plane_stride_a;
  int64_t plane_stride_b;
  unsigned long long wait_ns;  // limit of each device wait (wait_limit_ns())
  bool stall;                  // fault injection: the kernel's first MMA wait never completes
  int tile_n;                  // output tile width: 128, or 256 (any other value)
  bool split_squares;          // residue products: square moduli in two single-slot passes
};
// A operand: `planes_a` digit planes (K-major, m x k bytes, row stride lda8 bytes, plane
// stride plane_stride_a); B operand the same with n rows.
constexpr int kMaxGemmCtas = 192;  // persistent GEMM CTAs at most
cudaError_t launch_fp8_gemm(const GemmArgs& g, const uint8_t* a, int64_t lda8, int planes_a,
                            const uint8_t* b, int64_t ldb8, int planes_b, cudaStream_t st);

// crt.cu
cudaError_t launch_crt(const int16_t* cres, int64_t ldr, int64_t res_stride, int m, int n,
                       const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                       const uint8_t* colstat, double* C, int64_t ldc, const CrtTable& ct,
                       cudaStream_t st);

// ---------------------------------------------------------------------------
// Grouped launches: one launch of a kernel serves every problem of a batch.  Problem p
// owns blocks [first_block[w], first_block[w] + nblocks[w]) of grouped launch w; a block
// finds its problem by binary search over first_block[w].
// ---------------------------------------------------------------------------
enum BatchKernel {
  kBkScaleRows = 0,  // rows of A
  kBkColmax,         // columns of B: maxima
  kBkScaleCols,      // columns of B: Bbar^T or partial sums of squares
  kBkSumsq,          // columns of B: sums of squares (fast mode)
  kBkExponents,
  kBkResidRows,
  kBkResidCols,
  kBkCrt,
  kBatchKernels
};

struct BatchProblem {
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  int m, n, k, kp;
  int64_t ldp;  // digit-plane row pitch
  int64_t ldr;
  int32_t* eprime;
  int32_t* fprime;
  int32_t* e;
  int32_t* f;
  uint8_t* rowstat;
  uint8_t* colstat;
  uint8_t* Abar;
  uint8_t* BbarT;
  float* R;
  float* S;
  float* partB;
  uint32_t* colmaxB;  // log2 keys of the column maxima
  uint32_t* colbadB;
  uint8_t* planesA;
  uint8_t* planesB;
  int16_t* cres;
  int64_t first_block[kBatchKernels];
  int64_t nblocks[kBatchKernels];
};

// Tile of the column residue kernel: kResidTileCols columns x kResidTileK k per block
// (one block per tile in a grouped launch).
constexpr int kResidTileCols = 64, kResidTileK = 128;

// Items of the row residue kernel: a warp covers 2^s lanes x 8 k of 32 / 2^s rows, s = 4
// (128 consecutive k of two rows) for kp > 64, else the smallest s with 2^s 8 >= kp (kp is
// a multiple of 32): the last item of a row then leaves at most 120 of its k idle.
__host__ __device__ constexpr int resid_rows_lane_log(int kp) {
  return kp <= 32 ? 2 : (kp <= 64 ? 3 : 4);
}
__host__ __device__ constexpr int64_t resid_rows_items(int lines, int kp) {
  return static_cast<int64_t>((lines + (32 >> resid_rows_lane_log(kp)) - 1) / (32 >> resid_rows_lane_log(kp))) *
         ((kp + (8 << resid_rows_lane_log(kp)) - 1) / (8 << resid_rows_lane_log(kp)));
}

// Physical blocks of a grouped launch over `total` virtual blocks: at most four waves of
// per_sm resident blocks per SM (each physical block walks a contiguous range).
inline int grouped_grid(int64_t total, int per_sm) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = static_cast<int64_t>(sms) * per_sm * 4;
  return static_cast<int>(total < cap ? total : cap);
}

// Blocks of each grouped launch for one problem (the same decomposition the
// single-problem launchers use, without their grid caps).
void batch_block_counts(int m, int n, int k, int kp, bool fast, int64_t (&nblocks)[kBatchKernels]);

// The row kernels (A) run on st, the column kernels (B) on st_cols.
cudaError_t launch_scale_batch(const BatchProblem* probs, int count, const int64_t (&total)[kBatchKernels],
                               bool fast, uint32_t* flags, cudaStream_t st, cudaStream_t st_cols);
cudaError_t launch_exponents_batch(const BatchProblem* probs, int count, int64_t total_blocks, float pprime,
                                   float delta, cudaStream_t st);
cudaError_t launch_residues_batch(const BatchProblem* probs, int count, int64_t rows_blocks,
                                  int64_t cols_blocks, const ModTable& mt, uint32_t* flags, cudaStream_t st,
                                  cudaStream_t st_cols);
cudaError_t launch_crt_batch(const BatchProblem* probs, int count, int64_t total_blocks, const CrtTable& ct,
                             cudaStream_t st);

// One problem of a grouped GEMM launch: its operand maps and outputs.  Units (tile x
// modulus) of all problems are numbered consecutively from unit_start.
struct GemmProblem {  // CUtensorMap carries the 64-byte alignment TMA needs
  CUtensorMap ta;
  CUtensorMap tb;
  int m, n, k;
  int tiles_m, tiles_n, tiles;
  int64_t unit_start;
  int16_t* cres;
  int64_t ldr;
  int64_t res_stride;
  float factor;
  float* R;
  float* S;
  int split;  // residue products: square moduli in two single-slot passes
};
// Units of one problem in a GEMM of mode `mode` with N moduli and tiles of width tile_n.
int64_t fp8_gemm_units(int mode, int m, int n, int N, int tile_n);
// g supplies mode, num_sms, mt and flags; the problems (device memory, built on
// the host with encode_gemm_problem) supply everything else.
cudaError_t launch_fp8_gemm_grouped(const GemmArgs& g, const GemmProblem* probs, int count, int64_t total_units,
                                    cudaStream_t st);
// Fills the maps and tiling of one problem (the rest is the caller's); every problem of
// a grouped launch uses the launch's tile width (GemmArgs::tile_n).
bool encode_gemm_problem(GemmProblem* gp, const uint8_t* a, const uint8_t* b, int64_t ld8, int planes, int m,
                         int n, int k, int tile_n);

// tensor maps (api.cu)
// Boxes of box_rows x box_cols bytes (box_cols 128 or 64, swizzled to match).
bool encode_fp8_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows,
                    int64_t planes, int64_t row_stride_bytes, int64_t plane_stride_bytes,
                    int box_rows, int box_cols);

}  // namespace ozk2
