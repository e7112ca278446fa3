// C ABI of libozk2 (declared in include/ozk2.h): argument validation, the workspace,
// TMA descriptors, constant tables, and the order of the kernels of one emulated DGEMM:
//
//   scale rows of A | column maxima of B | scale columns of B   (Sec. III-E, Eq. def:mu'nu')
//   bound product Abar Bbar -> row / column maxima               (Eq. barCupper)
//   exponents e, f                                                (Eq. mu-computation)
//   residues and FP8 digits of A' and B'                          (Sec. III-B..III-D)
//   3N digit products + mod-reduce -> C'_l                        (Eqs. 3matmult, C'-Karatsuba)
//   CRT + inverse scaling -> C                                    (Eqs. CRT_finalreduction,
//                                                                  inversescaling)
// All kernels are launched on the caller's stream; nothing here runs on the CPU
// except bookkeeping.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "ozk2.h"

namespace ozk2 {
namespace {

constexpr int64_t kMaxDim = int64_t(1) << 20;

// ------------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// ------------------------------------------------------------------ device checks
struct DeviceInfo {
  bool probed = false;
  bool supported = false;
  int num_sms = 0;
};
std::mutex g_dev_mutex;
DeviceInfo g_dev[64];

bool device_info(int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  DeviceInfo& d = g_dev[dev];
  if (!d.probed) {
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    d.supported = (major == 10 && minor == 3);  // the kernels are built for sm_103a only
    d.num_sms = sms;
    d.probed = true;
  }
  *num_sms = d.num_sms;
  return d.supported;
}

// ------------------------------------------------------------------ constant tables
struct Tables {
  bool built = false;
  ModTable mt;
  CrtTable ct;
  float pprime;
};
std::mutex g_tab_mutex;
Tables g_tables[kMaxModuli + 1];

const Tables* tables_for(int N) {
  std::lock_guard<std::mutex> lk(g_tab_mutex);
  Tables& t = g_tables[N];
  if (!t.built) {
    if (!build_mod_table(N, &t.mt) || !build_crt_table(N, &t.ct)) return nullptr;
    t.pprime = p_prime_f32(N);
    t.built = true;
  }
  return &t;
}

// ------------------------------------------------------------------ operands
// The lines of an operand are the rows of op(A) (m of them) or the columns of op(B)
// (n of them); each line has k elements.  A line is contiguous along k for A and for
// B^T, strided (by ld) for B and for A^T.
struct Operand {
  const double* ptr;
  int64_t ld;
  bool kcontig;
};

Operand operand_a(ozk2_op transa, const double* A, int64_t lda) { return Operand{A, lda, transa == OZK2_OP_N}; }
Operand operand_b(ozk2_op transb, const double* B, int64_t ldb) { return Operand{B, ldb, transb == OZK2_OP_T}; }

// Sub-operand of lines [first, ...).
Operand shift_lines(const Operand& o, int64_t first) {
  Operand r = o;
  r.ptr = o.kcontig ? o.ptr + first * o.ld : o.ptr + first;
  return r;
}

// ------------------------------------------------------------------ workspace layout
struct Layout {
  int64_t kp, ldr;
  int planes;
  size_t flags, R, S, colmaxA, colbadA, colmaxB, colbadB, zero_end;
  size_t eprime, fprime, e, f, rowstat, colstat;
  size_t Abar, BbarT, partA, partB, planesA, planesB, cres, scratch, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int64_t m, int64_t n, int64_t k, int N, bool fast) {
  Layout L;
  L.kp = ((k + 31) / 32) * 32;
  L.ldr = ((n + 7) / 8) * 8;
  L.planes = (N <= kNumSquares) ? 2 * N : 3 * N - kNumSquares;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.flags = take(256);
  L.R = take(4 * size_t(m));
  L.S = take(4 * size_t(n));
  L.colmaxA = take(8 * size_t(m));
  L.colbadA = take(4 * size_t(m));
  L.colmaxB = take(8 * size_t(n));
  L.colbadB = take(4 * size_t(n));
  L.zero_end = o;
  L.eprime = take(4 * size_t(m));
  L.fprime = take(4 * size_t(n));
  L.e = take(4 * size_t(m));
  L.f = take(4 * size_t(n));
  L.rowstat = take(size_t(m));
  L.colstat = take(size_t(n));
  L.Abar = fast ? o : take(size_t(m) * L.kp);
  L.BbarT = fast ? o : take(size_t(n) * L.kp);
  L.partA = fast ? take(4 * size_t(m) * (L.kp / 32)) : o;
  L.partB = fast ? take(4 * size_t(n) * (L.kp / 32)) : o;
  L.planesA = take(size_t(L.planes) * m * L.kp);
  L.planesB = take(size_t(L.planes) * n * L.kp);
  L.cres = take(2 * size_t(N) * m * L.ldr);
  L.scratch = take(fp8_gemm_scratch_bytes(kMaxGemmCtas));
  L.total = o;
  return L;
}

struct Ctx {
  int m, n, k, N;
  bool fast;
  bool timed = true;  // record the per-phase timing events (sequential calls only)
  Layout L;
  uint8_t* ws;
  const Tables* tab;
  int num_sms;
  cudaStream_t st;
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

// ------------------------------------------------------------------ library-owned workspace
struct OwnedWs {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_ws_mutex;
OwnedWs g_ws[64];

uint8_t* owned_workspace(size_t need, ozk2_status* err) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_ws_mutex);
  OwnedWs& w = g_ws[dev];
  if (w.bytes < need) {
    if (w.ptr) cudaFree(w.ptr);
    w.ptr = nullptr;
    w.bytes = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      *err = OZK2_ERR_ALLOC;
      return nullptr;
    }
    cudaMemset(p, 0, 256);
    w.ptr = p;
    w.bytes = need;
  }
  return static_cast<uint8_t*>(w.ptr);
}

// ------------------------------------------------------------------ timing
struct Timing {
  bool enabled = false;
  bool have = false;
  int dev = -1;
  cudaEvent_t ev[7] = {};
};
Timing g_timing;
std::mutex g_timing_mutex;
thread_local int t_launches = 0;

void mark(Ctx& c, int idx) {
  if (!g_timing.enabled || !c.timed) return;
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_timing.dev != dev) {
    for (auto& e : g_timing.ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : g_timing.ev) cudaEventCreate(&e);
    g_timing.dev = dev;
  }
  cudaEventRecord(g_timing.ev[idx], c.st);
  if (idx == 6) g_timing.have = true;
}

#define OZK2_TRY(expr)                      \
  do {                                      \
    cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) return OZK2_ERR_CUDA; \
  } while (0)

// ------------------------------------------------------------------ phases
// Zero the bound maxima and column reductions of a call (and its flag word when
// clear_flags: the first block of a call; later blocks keep what earlier blocks
// recorded).
ozk2_status zero_scratch(Ctx& c, bool clear_flags) {
  const Layout& L = c.L;
  if (clear_flags)
    OZK2_TRY(cudaMemsetAsync(c.ws, 0, L.zero_end, c.st));
  else
    OZK2_TRY(cudaMemsetAsync(c.ws + L.R, 0, L.zero_end - L.R, c.st));
  return OZK2_OK;
}

// Which operand a scaling launch serves.
struct Side {
  size_t eprime, stat, bar, sq, part, colmax, colbad;
};
Side side_a(const Layout& L) { return Side{L.eprime, L.rowstat, L.Abar, L.R, L.partA, L.colmaxA, L.colbadA}; }
Side side_b(const Layout& L) { return Side{L.fprime, L.colstat, L.BbarT, L.S, L.partB, L.colmaxB, L.colbadB}; }

// e'/status and either the E4M3 bound operand (accurate) or the sums of squares (fast)
// of lines [first, first + lines) of one operand (`op` points at line `first`).
ozk2_status scale_operand(Ctx& c, const Operand& op, int64_t first, int lines, const Side& sd) {
  const Layout& L = c.L;
  const int64_t kb = L.kp / 32;
  int32_t* ep = c.at<int32_t>(sd.eprime) + first;
  uint8_t* stat = c.at<uint8_t>(sd.stat) + first;
  uint8_t* bar = c.at<uint8_t>(sd.bar) + first * L.kp;
  float* sq = c.at<float>(sd.sq) + first;
  if (op.kcontig) {
    OZK2_TRY(launch_scale_rows(op.ptr, op.ld, lines, c.k, int(L.kp), ep, stat, bar, sq, c.fast,
                               c.at<uint32_t>(L.flags), c.st));
    t_launches += 1;
  } else {
    unsigned long long* cm = c.at<unsigned long long>(sd.colmax) + first;
    uint32_t* cb = c.at<uint32_t>(sd.colbad) + first;
    OZK2_TRY(launch_colmax(op.ptr, op.ld, c.k, lines, cm, cb, c.st));
    OZK2_TRY(launch_scale_cols(op.ptr, op.ld, c.k, lines, int(L.kp), cm, cb, ep, stat, bar,
                               c.at<float>(sd.part) + first * kb, sq, c.fast, c.at<uint32_t>(L.flags), c.st));
    t_launches += c.fast ? 3 : 2;
  }
  return OZK2_OK;
}

// Bound product (accurate mode) and the exponents e, f.
ozk2_status bound_and_exponents(Ctx& c) {
  const Layout& L = c.L;
  mark(c, 1);
  if (!c.fast) {
    GemmArgs g{};
    g.mode = kModeBound;
    g.m = c.m;
    g.n = c.n;
    g.k = c.k;
    g.num_sms = c.num_sms;
    g.factor = bound_factor_f32(c.k);
    g.R = c.at<float>(L.R);
    g.S = c.at<float>(L.S);
    g.flags = c.at<uint32_t>(L.flags);
    OZK2_TRY(launch_fp8_gemm(g, c.at<uint8_t>(L.Abar), L.kp, 1, c.at<uint8_t>(L.BbarT), L.kp, 1, c.st));
    t_launches += 1;
  }
  mark(c, 2);
  OZK2_TRY(launch_exponents(c.m, c.n, c.at<int32_t>(L.eprime), c.at<int32_t>(L.fprime), c.at<uint8_t>(L.rowstat),
                            c.at<uint8_t>(L.colstat), c.at<float>(L.R), c.at<float>(L.S), c.tab->pprime,
                            delta_f32(), c.at<int32_t>(L.e), c.at<int32_t>(L.f), c.st));
  t_launches += 1;
  mark(c, 3);
  return OZK2_OK;
}

ozk2_status phase_scales(Ctx& c, const Operand& a, const Operand& b, bool clear_flags) {
  ozk2_status s;
  if ((s = zero_scratch(c, clear_flags)) != OZK2_OK) return s;
  if ((s = scale_operand(c, a, 0, c.m, side_a(c.L))) != OZK2_OK) return s;
  if ((s = scale_operand(c, b, 0, c.n, side_b(c.L))) != OZK2_OK) return s;
  return bound_and_exponents(c);
}

cudaError_t residues_operand(Ctx& c, const Operand& op, int lines, const int32_t* ex, uint8_t* planes) {
  if (op.kcontig)
    return launch_residues_rows(op.ptr, op.ld, lines, c.k, int(c.L.kp), ex, c.tab->mt, planes,
                                c.at<uint32_t>(c.L.flags), c.st);
  return launch_residues_cols(op.ptr, op.ld, c.k, lines, int(c.L.kp), ex, c.tab->mt, planes,
                              c.at<uint32_t>(c.L.flags), c.st);
}

ozk2_status phase_residues(Ctx& c, const Operand& a, const Operand& b, const int32_t* e, const int32_t* f,
                           uint8_t* planesA, uint8_t* planesB) {
  OZK2_TRY(residues_operand(c, a, c.m, e, planesA));
  OZK2_TRY(residues_operand(c, b, c.n, f, planesB));
  t_launches += 2;
  mark(c, 4);
  return OZK2_OK;
}

// Residue products C'_l for output rows [i0, i0 + rows).
ozk2_status products_rows(Ctx& c, int64_t i0, int rows) {
  const Layout& L = c.L;
  GemmArgs g{};
  g.mode = kModeResidue;
  g.m = rows;
  g.n = c.n;
  g.k = c.k;
  g.num_sms = c.num_sms;
  g.cres = c.at<int16_t>(L.cres) + i0 * L.ldr;
  g.ldr = L.ldr;
  g.res_stride = int64_t(c.m) * L.ldr;
  g.scratch = c.at<uint32_t>(L.scratch);
  g.mt = &c.tab->mt;
  g.flags = c.at<uint32_t>(L.flags);
  g.plane_stride_a = int64_t(c.m) * L.kp;
  g.plane_stride_b = int64_t(c.n) * L.kp;
  OZK2_TRY(launch_fp8_gemm(g, c.at<uint8_t>(L.planesA) + i0 * L.kp, L.kp, L.planes, c.at<uint8_t>(L.planesB), L.kp,
                           L.planes, c.st));
  t_launches += 1;
  return OZK2_OK;
}

ozk2_status phase_products(Ctx& c) {
  ozk2_status s = products_rows(c, 0, c.m);
  if (s != OZK2_OK) return s;
  mark(c, 5);
  return OZK2_OK;
}

// CRT and inverse scaling of output rows [i0, i0 + rows) into C (which points at row i0).
ozk2_status crt_rows(Ctx& c, int64_t i0, int rows, const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                     const uint8_t* colstat, double* C, int64_t ldc) {
  const Layout& L = c.L;
  OZK2_TRY(launch_crt(c.at<int16_t>(L.cres) + i0 * L.ldr, L.ldr, int64_t(c.m) * L.ldr, rows, c.n, e + i0, f,
                      rowstat ? rowstat + i0 : nullptr, colstat, C, ldc, c.tab->ct, c.st));
  t_launches += 1;
  return OZK2_OK;
}

ozk2_status phase_crt(Ctx& c, const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                      const uint8_t* colstat, double* C, int64_t ldc) {
  ozk2_status s = crt_rows(c, 0, c.m, e, f, rowstat, colstat, C, ldc);
  if (s != OZK2_OK) return s;
  mark(c, 6);
  return OZK2_OK;
}

ozk2_status check_sizes(int64_t m, int64_t n, int64_t k, int N) {
  if (m < 0 || n < 0 || k < 0 || N < 1 || N > kMaxModuli) return OZK2_ERR_INVALID_VALUE;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return OZK2_ERR_UNSUPPORTED;
  return OZK2_OK;
}

bool valid_op(int op) { return op == OZK2_OP_N || op == OZK2_OP_T; }
bool valid_mode(int mode) { return mode == OZK2_MODE_ACCURATE || mode == OZK2_MODE_FAST; }

ozk2_status validate(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                     const double* B, int64_t ldb, const double* C, int64_t ldc, int N) {
  ozk2_status s = check_sizes(m, n, k, N);
  if (s != OZK2_OK) return s;
  if (!valid_op(transa) || !valid_op(transb)) return OZK2_ERR_INVALID_VALUE;
  const int64_t min_lda = transa == OZK2_OP_N ? k : m;
  const int64_t min_ldb = transb == OZK2_OP_N ? n : k;
  if (lda < std::max<int64_t>(1, min_lda) || ldb < std::max<int64_t>(1, min_ldb) || ldc < std::max<int64_t>(1, n))
    return OZK2_ERR_INVALID_VALUE;
  if (m == 0 || n == 0) return OZK2_OK;  // nothing is read or written
  if (!C || (k > 0 && (!A || !B))) return OZK2_ERR_INVALID_VALUE;
  return OZK2_OK;
}

// validate() for the scaling hook, which writes no C.
ozk2_status validate_operands(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                              int64_t lda, const double* B, int64_t ldb, int N) {
  static double dummy;
  return validate(transa, transb, m, n, k, A, lda, B, ldb, &dummy, std::max<int64_t>(1, n), N);
}

// `extra`: bytes the caller needs after the layout (256-aligned, at offset L.total).
ozk2_status setup(Ctx& c, int64_t m, int64_t n, int64_t k, int N, bool fast, void* ws, size_t ws_bytes,
                  cudaStream_t st, size_t extra = 0) {
  c.m = int(m);
  c.n = int(n);
  c.k = int(k);
  c.N = N;
  c.fast = fast;
  c.st = st;
  if (!device_info(&c.num_sms)) return OZK2_ERR_UNSUPPORTED;
  if (!encode_fn()) return OZK2_ERR_CUDA;
  c.tab = tables_for(N);
  if (!c.tab) return OZK2_ERR_INTERNAL;
  c.L = make_layout(m, n, k, N, fast);
  if (ws) {
    if (ws_bytes < c.L.total + extra || (reinterpret_cast<uintptr_t>(ws) & 255u)) return OZK2_ERR_INVALID_VALUE;
    c.ws = static_cast<uint8_t*>(ws);
  } else {
    ozk2_status err = OZK2_OK;
    c.ws = owned_workspace(c.L.total + extra, &err);
    if (!c.ws) return err;
  }
  return OZK2_OK;
}

// One emulated product over whole operands (no blocking); arguments already validated,
// m, n, k > 0.
ozk2_status run_one(const Operand& a, const Operand& b, int64_t m, int64_t n, int64_t k, double* C, int64_t ldc,
                    int N, bool fast, bool first, void* ws, size_t ws_bytes, cudaStream_t st) {
  Ctx c;
  ozk2_status s = setup(c, m, n, k, N, fast, ws, ws_bytes, st);
  if (s != OZK2_OK) return s;
  mark(c, 0);
  const Layout& L = c.L;
  if ((s = phase_scales(c, a, b, first)) != OZK2_OK) return s;
  if ((s = phase_residues(c, a, b, c.at<int32_t>(L.e), c.at<int32_t>(L.f), c.at<uint8_t>(L.planesA),
                          c.at<uint8_t>(L.planesB))) != OZK2_OK)
    return s;
  if ((s = phase_products(c)) != OZK2_OK) return s;
  return phase_crt(c, c.at<int32_t>(L.e), c.at<int32_t>(L.f), c.at<uint8_t>(L.rowstat), c.at<uint8_t>(L.colstat), C,
                   ldc);
}

int64_t block_or_all(int64_t b, int64_t total) { return (b <= 0 || b >= total) ? total : b; }

size_t workspace_bytes(int64_t m, int64_t n, int64_t k, int N, bool fast, int64_t bm, int64_t bn) {
  return make_layout(block_or_all(bm, m), block_or_all(bn, n), k, N, fast).total;
}

ozk2_status dgemm_general(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                          int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int N, int mode,
                          int64_t block_m, int64_t block_n, void* ws, size_t ws_bytes, cudaStream_t st) {
  t_launches = 0;
  if (!valid_mode(mode) || block_m < 0 || block_n < 0) return OZK2_ERR_INVALID_VALUE;
  ozk2_status s = validate(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, N);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0) return OZK2_OK;
  if (k == 0) {
    OZK2_TRY(cudaMemset2DAsync(C, size_t(ldc) * 8, 0, size_t(n) * 8, size_t(m), st));
    return OZK2_OK;
  }
  const bool fast = mode == OZK2_MODE_FAST;
  const Operand a = operand_a(transa, A, lda);
  const Operand b = operand_b(transb, B, ldb);
  const int64_t bm = block_or_all(block_m, m), bn = block_or_all(block_n, n);
  for (int64_t i0 = 0; i0 < m; i0 += bm) {
    for (int64_t j0 = 0; j0 < n; j0 += bn) {
      const int64_t mm = std::min(bm, m - i0), nn = std::min(bn, n - j0);
      s = run_one(shift_lines(a, i0), shift_lines(b, j0), mm, nn, k, C + i0 * ldc + j0, ldc, N, fast,
                  i0 == 0 && j0 == 0, ws, ws_bytes, st);
      if (s != OZK2_OK) return s;
    }
  }
  return OZK2_OK;
}

// ------------------------------------------------------------------ host buffers
// Device staging of a host-buffer call: A and B as stored (packed), and C.
struct Staging {
  size_t A, B, C, total;
};

Staging make_staging(int64_t m, int64_t n, int64_t k) {
  Staging g;
  size_t o = 0;
  g.A = o;
  o = align256(o + 8 * size_t(m) * size_t(k));
  g.B = o;
  o = align256(o + 8 * size_t(k) * size_t(n));
  g.C = o;
  o = align256(o + 8 * size_t(m) * size_t(n));
  g.total = o;
  return g;
}

constexpr int kHostChunks = 4;  // A arrives in this many line chunks
constexpr int kHostBlocks = 4;  // at most this many output row blocks stream back
constexpr int kHostEvents = 2 + kHostChunks + kHostBlocks + 1;

struct CopyEngine {
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[kHostEvents] = {};
};
std::mutex g_copy_mutex;
CopyEngine g_copy[64];

// The library's copy stream and events of the current device (created on first use).
CopyEngine* copy_engine(ozk2_status* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *err = OZK2_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_copy_mutex);
  CopyEngine& e = g_copy[dev];
  if (!e.cs) {
    if (cudaStreamCreateWithFlags(&e.cs, cudaStreamNonBlocking) != cudaSuccess) {
      *err = OZK2_ERR_CUDA;
      e.cs = nullptr;
      return nullptr;
    }
    for (auto& ev : e.ev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        *err = OZK2_ERR_CUDA;
        return nullptr;
      }
  }
  return &e;
}

// Copy lines [i0, i1) of an operand stored on the host to its packed device copy.
// kcontig lines are rows of the stored matrix (ld elements apart), otherwise columns.
cudaError_t copy_lines_h2d(double* dst, const double* src, int64_t ld, bool kcontig, int64_t lines, int64_t k,
                           int64_t i0, int64_t i1, cudaStream_t cs) {
  if (i1 <= i0) return cudaSuccess;
  if (kcontig)
    return cudaMemcpy2DAsync(dst + i0 * k, size_t(k) * 8, src + i0 * ld, size_t(ld) * 8, size_t(k) * 8,
                             size_t(i1 - i0), cudaMemcpyHostToDevice, cs);
  return cudaMemcpy2DAsync(dst + i0, size_t(lines) * 8, src + i0, size_t(ld) * 8, size_t(i1 - i0) * 8, size_t(k),
                           cudaMemcpyHostToDevice, cs);
}

// C = op(A) op(B) from host buffers: B and then A (in line chunks) go up on the copy
// stream while the scaling of what has arrived runs on `st`; after the exponents and
// residues, the residue products and the CRT run in output row blocks, and block b
// streams back while block b + 1 is computed.  The device arithmetic is exactly that
// of the device-buffer call, so the results are bit-identical.
ozk2_status run_host(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* hA,
                     int64_t lda, const double* hB, int64_t ldb, double* hC, int64_t ldc, int N, bool fast,
                     void* ws, size_t ws_bytes, cudaStream_t st) {
  ozk2_status s;
  CopyEngine* ce = copy_engine(&s);
  if (!ce) return s;
  Ctx c;
  const Staging G = make_staging(m, n, k);
  if ((s = setup(c, m, n, k, N, fast, ws, ws_bytes, st, G.total)) != OZK2_OK) return s;
  c.timed = false;  // phases overlap with copies
  const Layout& L = c.L;
  double* dA = c.at<double>(L.total + G.A);
  double* dB = c.at<double>(L.total + G.B);
  double* dC = c.at<double>(L.total + G.C);
  const bool a_kc = transa == OZK2_OP_N, b_kc = transb == OZK2_OP_T;
  const Operand a = operand_a(transa, dA, a_kc ? k : m);
  const Operand b = operand_b(transb, dB, b_kc ? k : n);
  cudaStream_t cs = ce->cs;
  cudaEvent_t* ev = ce->ev;
  cudaEvent_t ev_start = ev[0], ev_b = ev[1], *ev_a = ev + 2, *ev_blk = ev + 2 + kHostChunks,
              ev_done = ev[kHostEvents - 1];

  // nothing is copied into the workspace before earlier work on `st` is done with it
  OZK2_TRY(cudaEventRecord(ev_start, st));
  OZK2_TRY(cudaStreamWaitEvent(cs, ev_start, 0));
  OZK2_TRY(copy_lines_h2d(dB, hB, ldb, b_kc, n, k, 0, n, cs));
  OZK2_TRY(cudaEventRecord(ev_b, cs));
  const int64_t chunk = (m + kHostChunks - 1) / kHostChunks;
  for (int q = 0; q < kHostChunks; ++q) {
    OZK2_TRY(copy_lines_h2d(dA, hA, lda, a_kc, m, k, std::min(m, q * chunk), std::min(m, (q + 1) * chunk), cs));
    OZK2_TRY(cudaEventRecord(ev_a[q], cs));
  }

  if ((s = zero_scratch(c, true)) != OZK2_OK) return s;
  OZK2_TRY(cudaStreamWaitEvent(st, ev_b, 0));
  if ((s = scale_operand(c, b, 0, int(n), side_b(L))) != OZK2_OK) return s;
  for (int q = 0; q < kHostChunks; ++q) {
    const int64_t i0 = std::min(m, q * chunk), i1 = std::min(m, (q + 1) * chunk);
    OZK2_TRY(cudaStreamWaitEvent(st, ev_a[q], 0));
    if (i1 > i0 && (s = scale_operand(c, shift_lines(a, i0), i0, int(i1 - i0), side_a(L))) != OZK2_OK) return s;
  }
  if ((s = bound_and_exponents(c)) != OZK2_OK) return s;
  if ((s = phase_residues(c, a, b, c.at<int32_t>(L.e), c.at<int32_t>(L.f), c.at<uint8_t>(L.planesA),
                          c.at<uint8_t>(L.planesB))) != OZK2_OK)
    return s;

  // output row blocks: a multiple of the 128-row tile, each at least ~8 waves of tiles
  const int64_t units = ((m + 127) / 128) * ((n + 255) / 256) * N;
  const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(kHostBlocks, units / (8 * int64_t(c.num_sms))));
  const int64_t rb = ((m + nblk - 1) / nblk + 127) / 128 * 128;
  int used = 0;
  for (int64_t i0 = 0; i0 < m; i0 += rb, ++used) {
    const int rows = int(std::min(rb, m - i0));
    if ((s = products_rows(c, i0, rows)) != OZK2_OK) return s;
    if ((s = crt_rows(c, i0, rows, c.at<int32_t>(L.e), c.at<int32_t>(L.f), c.at<uint8_t>(L.rowstat),
                      c.at<uint8_t>(L.colstat), dC + i0 * n, n)) != OZK2_OK)
      return s;
    OZK2_TRY(cudaEventRecord(ev_blk[used], st));
    OZK2_TRY(cudaStreamWaitEvent(cs, ev_blk[used], 0));
    OZK2_TRY(cudaMemcpy2DAsync(hC + i0 * ldc, size_t(ldc) * 8, dC + i0 * n, size_t(n) * 8, size_t(n) * 8,
                               size_t(rows), cudaMemcpyDeviceToHost, cs));
  }
  // the call is complete on `st` once the last block is back on the host
  OZK2_TRY(cudaEventRecord(ev_done, cs));
  OZK2_TRY(cudaStreamWaitEvent(st, ev_done, 0));
  return OZK2_OK;
}

size_t host_workspace_bytes(int64_t m, int64_t n, int64_t k, int N, bool fast) {
  return make_layout(m, n, k, N, fast).total + make_staging(m, n, k).total;
}

}  // namespace

bool encode_fp8_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int64_t planes,
                    int64_t row_stride_bytes, int64_t plane_stride_bytes, int box_rows, int box_cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || cols < 1 || rows < 1 || planes < 1 || (box_cols != 128 && box_cols != 64)) return false;
  if (plane_stride_bytes == 0) plane_stride_bytes = row_stride_bytes * rows;
  if (planes > 1 && plane_stride_bytes < row_stride_bytes * rows) return false;
  const cuuint64_t dims[3] = {cuuint64_t(cols), cuuint64_t(rows), cuuint64_t(planes)};
  const cuuint64_t strides[2] = {cuuint64_t(row_stride_bytes), cuuint64_t(plane_stride_bytes)};
  const cuuint32_t box[3] = {cuuint32_t(box_cols), cuuint32_t(box_rows), 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapSwizzle sw = (box_cols == 128) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace ozk2

using namespace ozk2;

extern "C" {

ozk2_status ozk2_dgemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                       double* C, int64_t ldc, int num_moduli, ozk2_stream_t stream) {
  return dgemm_general(OZK2_OP_N, OZK2_OP_N, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, OZK2_MODE_ACCURATE, 0, 0,
                       nullptr, 0, reinterpret_cast<cudaStream_t>(stream));
}

ozk2_status ozk2_dgemm_ws(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double* C, int64_t ldc, int num_moduli, void* workspace, size_t workspace_bytes,
                          ozk2_stream_t stream) {
  if (!workspace) return OZK2_ERR_INVALID_VALUE;
  return dgemm_general(OZK2_OP_N, OZK2_OP_N, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, OZK2_MODE_ACCURATE, 0, 0,
                       workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

ozk2_status ozk2_dgemm_ex(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                          int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int num_moduli,
                          ozk2_mode mode, int64_t block_m, int64_t block_n, void* workspace, size_t workspace_bytes,
                          ozk2_stream_t stream) {
  return dgemm_general(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode, block_m, block_n, workspace,
                       workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

ozk2_status ozk2_dgemm_host(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int num_moduli,
                            ozk2_mode mode, void* workspace, size_t workspace_bytes, ozk2_stream_t stream) {
  t_launches = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!valid_mode(mode)) return OZK2_ERR_INVALID_VALUE;
  ozk2_status s = validate(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0) return OZK2_OK;
  if (k == 0) {  // C = 0 once earlier work on the stream (which may target C) is done
    if (cudaStreamSynchronize(st) != cudaSuccess) return OZK2_ERR_CUDA;
    for (int64_t i = 0; i < m; ++i) std::memset(C + i * ldc, 0, size_t(n) * 8);
    return OZK2_OK;
  }
  return run_host(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode == OZK2_MODE_FAST, workspace,
                  workspace_bytes, st);
}

size_t ozk2_workspace_size_host(int64_t m, int64_t n, int64_t k, int num_moduli, ozk2_mode mode) {
  if (check_sizes(m, n, k, num_moduli) != OZK2_OK || !valid_mode(mode)) return 0;
  return host_workspace_bytes(m, n, k, num_moduli, mode == OZK2_MODE_FAST);
}

size_t ozk2_workspace_size(int64_t m, int64_t n, int64_t k, int num_moduli) {
  if (check_sizes(m, n, k, num_moduli) != OZK2_OK) return 0;
  return workspace_bytes(m, n, k, num_moduli, false, 0, 0);
}

size_t ozk2_workspace_size_ex(int64_t m, int64_t n, int64_t k, int num_moduli, ozk2_mode mode, int64_t block_m,
                              int64_t block_n) {
  if (check_sizes(m, n, k, num_moduli) != OZK2_OK || !valid_mode(mode) || block_m < 0 || block_n < 0) return 0;
  return workspace_bytes(m, n, k, num_moduli, mode == OZK2_MODE_FAST, block_m, block_n);
}

const char* ozk2_status_string(ozk2_status s) {
  switch (s) {
    case OZK2_OK: return "OZK2_OK";
    case OZK2_ERR_INVALID_VALUE: return "OZK2_ERR_INVALID_VALUE";
    case OZK2_ERR_UNSUPPORTED: return "OZK2_ERR_UNSUPPORTED";
    case OZK2_ERR_ALLOC: return "OZK2_ERR_ALLOC";
    case OZK2_ERR_CUDA: return "OZK2_ERR_CUDA";
    case OZK2_ERR_INTERNAL: return "OZK2_ERR_INTERNAL";
    case OZK2_ERR_TIMEOUT: return "OZK2_ERR_TIMEOUT";
    case OZK2_ERR_NONFINITE: return "OZK2_ERR_NONFINITE";
    case OZK2_ERR_RANGE: return "OZK2_ERR_RANGE";
  }
  return "OZK2_UNKNOWN_STATUS";
}

ozk2_status ozk2_device_status(void* workspace, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return OZK2_ERR_CUDA;
  void* ws = workspace;
  if (!ws) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OZK2_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    ws = g_ws[dev].ptr;
  }
  if (!ws) return OZK2_OK;
  uint32_t flags = 0;
  if (cudaMemcpy(&flags, ws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZK2_ERR_CUDA;
  if (cudaMemset(ws, 0, 4) != cudaSuccess) return OZK2_ERR_CUDA;
  if (flags & kFlagTimeout) return OZK2_ERR_TIMEOUT;
  if (flags & kFlagRange) return OZK2_ERR_RANGE;
  if (flags & kFlagNonfinite) return OZK2_ERR_NONFINITE;
  return OZK2_OK;
}

int ozk2_moduli(int num_moduli, int32_t* p_out) {
  int mods[kMaxModuli];
  if (!p_out || hybrid_moduli(num_moduli, mods) != num_moduli) return -1;
  for (int i = 0; i < num_moduli; ++i) p_out[i] = mods[i];
  return num_moduli;
}

void ozk2_set_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_timing_mutex);
  g_timing.enabled = enable != 0;
  g_timing.have = false;
}

int ozk2_get_timing(float* ms, int max) {
  std::lock_guard<std::mutex> lk(g_timing_mutex);
  if (!g_timing.have || !ms) return -1;
  if (cudaEventSynchronize(g_timing.ev[6]) != cudaSuccess) return -1;
  int w = 0;
  for (int i = 0; i < 6 && w < max; ++i, ++w) cudaEventElapsedTime(&ms[i], g_timing.ev[i], g_timing.ev[i + 1]);
  return w;
}

int ozk2_last_launch_count(void) { return t_launches; }

ozk2_status ozk2_debug_fp8_gemm(int64_t m, int64_t n, int64_t k, const uint8_t* A8, int64_t lda8, const uint8_t* B8,
                                int64_t ldb8, float* D, int64_t ldd, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (m < 0 || n < 0 || k < 0) return OZK2_ERR_INVALID_VALUE;
  if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return OZK2_ERR_UNSUPPORTED;
  if (m == 0 || n == 0) return OZK2_OK;
  if (!D || ldd < n) return OZK2_ERR_INVALID_VALUE;
  if (k == 0) {
    OZK2_TRY(cudaMemset2DAsync(D, size_t(ldd) * 4, 0, size_t(n) * 4, size_t(m), st));
    return OZK2_OK;
  }
  if (!A8 || !B8 || lda8 < k || ldb8 < k || (lda8 % 16) || (ldb8 % 16) ||
      (reinterpret_cast<uintptr_t>(A8) & 15u) || (reinterpret_cast<uintptr_t>(B8) & 15u))
    return OZK2_ERR_INVALID_VALUE;
  int sms = 0;
  if (!device_info(&sms)) return OZK2_ERR_UNSUPPORTED;
  if (!encode_fn()) return OZK2_ERR_CUDA;
  GemmArgs g{};
  g.mode = kModeRaw;
  g.m = int(m);
  g.n = int(n);
  g.k = int(k);
  g.num_sms = sms;
  g.D = D;
  g.ldd = ldd;
  ozk2_status err = OZK2_OK;
  uint8_t* ws = owned_workspace(256, &err);  // flag word only
  if (!ws) return err;
  g.flags = reinterpret_cast<uint32_t*>(ws);
  OZK2_TRY(launch_fp8_gemm(g, A8, lda8, 1, B8, ldb8, 1, st));
  return OZK2_OK;
}

ozk2_status ozk2_debug_scales_ex(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                                 int64_t lda, const double* B, int64_t ldb, int num_moduli, ozk2_mode mode,
                                 int32_t* e, int32_t* f, int32_t* eprime, int32_t* fprime, float* R, float* S,
                                 uint8_t* Abar, uint8_t* BbarT, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!valid_mode(mode)) return OZK2_ERR_INVALID_VALUE;
  ozk2_status s = validate_operands(transa, transb, m, n, k, A, lda, B, ldb, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0 || k == 0 || !A || !B) return OZK2_ERR_INVALID_VALUE;
  const bool fast = mode == OZK2_MODE_FAST;
  Ctx c;
  if ((s = setup(c, m, n, k, num_moduli, fast, nullptr, 0, st)) != OZK2_OK) return s;
  if ((s = phase_scales(c, operand_a(transa, A, lda), operand_b(transb, B, ldb), true)) != OZK2_OK) return s;
  const Layout& L = c.L;
  auto cp = [&](void* dst, size_t off, size_t bytes) -> cudaError_t {
    if (!dst) return cudaSuccess;
    return cudaMemcpyAsync(dst, c.ws + off, bytes, cudaMemcpyDeviceToDevice, st);
  };
  OZK2_TRY(cp(e, L.e, 4 * size_t(m)));
  OZK2_TRY(cp(f, L.f, 4 * size_t(n)));
  OZK2_TRY(cp(eprime, L.eprime, 4 * size_t(m)));
  OZK2_TRY(cp(fprime, L.fprime, 4 * size_t(n)));
  OZK2_TRY(cp(R, L.R, 4 * size_t(m)));
  OZK2_TRY(cp(S, L.S, 4 * size_t(n)));
  if (!fast) {
    OZK2_TRY(cp(Abar, L.Abar, size_t(m) * L.kp));
    OZK2_TRY(cp(BbarT, L.BbarT, size_t(n) * L.kp));
  }
  return OZK2_OK;
}

ozk2_status ozk2_debug_scales(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                              int64_t ldb, int num_moduli, int32_t* e, int32_t* f, int32_t* eprime, int32_t* fprime,
                              float* R, float* S, uint8_t* Abar, uint8_t* BbarT, ozk2_stream_t stream) {
  return ozk2_debug_scales_ex(OZK2_OP_N, OZK2_OP_N, m, n, k, A, lda, B, ldb, num_moduli, OZK2_MODE_ACCURATE, e, f,
                              eprime, fprime, R, S, Abar, BbarT, stream);
}

ozk2_status ozk2_debug_residue_planes(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                                      int64_t ldb, int num_moduli, const int32_t* e, const int32_t* f,
                                      uint8_t* planesA, uint8_t* planesB, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = check_sizes(m, n, k, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0 || k == 0 || !A || !B || !e || !f || !planesA || !planesB || lda < k || ldb < n)
    return OZK2_ERR_INVALID_VALUE;
  Ctx c;
  if ((s = setup(c, m, n, k, num_moduli, false, nullptr, 0, st)) != OZK2_OK) return s;
  return phase_residues(c, operand_a(OZK2_OP_N, A, lda), operand_b(OZK2_OP_N, B, ldb), e, f, planesA, planesB);
}

ozk2_status ozk2_debug_residue_products(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                                        const double* B, int64_t ldb, int num_moduli, const int32_t* e,
                                        const int32_t* f, int16_t* Cres, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = check_sizes(m, n, k, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0 || k == 0 || !A || !B || !e || !f || !Cres || lda < k || ldb < n)
    return OZK2_ERR_INVALID_VALUE;
  Ctx c;
  if ((s = setup(c, m, n, k, num_moduli, false, nullptr, 0, st)) != OZK2_OK) return s;
  const Layout& L = c.L;
  if ((s = phase_residues(c, operand_a(OZK2_OP_N, A, lda), operand_b(OZK2_OP_N, B, ldb), e, f,
                          c.at<uint8_t>(L.planesA), c.at<uint8_t>(L.planesB))) != OZK2_OK)
    return s;
  if ((s = phase_products(c)) != OZK2_OK) return s;
  OZK2_TRY(cudaMemcpy2DAsync(Cres, size_t(n) * 2, c.ws + L.cres, size_t(L.ldr) * 2, size_t(n) * 2,
                             size_t(num_moduli) * size_t(m), cudaMemcpyDeviceToDevice, st));
  return OZK2_OK;
}

ozk2_status ozk2_debug_crt(int64_t m, int64_t n, int num_moduli, const int16_t* Cres, const int32_t* e,
                           const int32_t* f, double* C, int64_t ldc, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = check_sizes(m, n, 1, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0) return OZK2_OK;
  if (!Cres || !e || !f || !C || ldc < n) return OZK2_ERR_INVALID_VALUE;
  Ctx c;
  if ((s = setup(c, m, n, 1, num_moduli, false, nullptr, 0, st)) != OZK2_OK) return s;
  const Layout& L = c.L;
  OZK2_TRY(cudaMemcpy2DAsync(c.ws + L.cres, size_t(L.ldr) * 2, Cres, size_t(n) * 2, size_t(n) * 2,
                             size_t(num_moduli) * size_t(m), cudaMemcpyDeviceToDevice, st));
  return phase_crt(c, e, f, nullptr, nullptr, C, ldc);
}

}  // extern "C"
