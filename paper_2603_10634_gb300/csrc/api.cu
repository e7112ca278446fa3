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
// All kernels are launched on the caller's stream (a host-buffer call moves its data on
// a library copy stream); nothing here runs on the CPU except bookkeeping.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

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

// ------------------------------------------------------------------ fault injection, wait limit
// One armed fault kind (kFaultNone when none), set by ozk2_debug_inject_fault or, once at
// first use, by the environment variable OZK2_FAULT (alloc | launch | stall).
std::mutex g_fault_mutex;
int g_fault = kFaultNone;
bool g_fault_env_read = false;

int fault_kind_of(const char* s) {
  if (!s) return kFaultNone;
  if (!std::strcmp(s, "alloc")) return kFaultAlloc;
  if (!std::strcmp(s, "launch")) return kFaultLaunch;
  if (!std::strcmp(s, "stall")) return kFaultStall;
  return kFaultNone;
}

// With g_fault_mutex held.
void read_fault_env() {
  if (g_fault_env_read) return;
  g_fault_env_read = true;
  const int k = fault_kind_of(std::getenv("OZK2_FAULT"));
  if (k != kFaultNone) g_fault = k;
}

std::atomic<unsigned long long> g_wait_ns{0};  // 0: the default limit of the kernels

// ------------------------------------------------------------------ tile width
// The FP8 products run in 128 x 256 or 128 x 128 output tiles.  ozk2_set_tile_n fixes
// one; 0 (the default) lets the rule below choose: the narrow tile where the wide one
// would pad the product's columns by a quarter or more (ceil(n/256) 256 >= 1.25 ceil(n/128)
// 128), since the wide tile otherwise runs the tensor cores more efficiently.
std::atomic<int> g_tile_n{0};

int64_t padded(int64_t n, int64_t t) { return ((n + t - 1) / t) * t; }

int tile_rule(int64_t padded256, int64_t padded128) { return 4 * padded256 >= 5 * padded128 ? 128 : 256; }

// Square moduli run as two single-slot passes (X, then Z) when the reduction is at most
// this long (ozk2_set_square_split).  Off by default: measured on the 512-product batch,
// the 65536 x 1024 x 1024 product and square sizes 1024-8192, the split was neutral or
// slower (the drain of both slots after a one-pass square modulus is not what limits
// short reductions).
std::atomic<int64_t> g_split_kmax{0};

int tile_for(int64_t n) {
  const int t = g_tile_n.load();
  return t ? t : tile_rule(padded(n, 256), padded(n, 128));
}

// ------------------------------------------------------------------ workspace checks
// A caller workspace must be device memory of the current device: the FP8 product kernels
// read it through TMA tensor maps, and nothing else (host, managed or another GPU's memory)
// may become the source of those loads.
bool device_memory_here(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
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
  int64_t kp, ldp, ldr;  // kp: bytes of k per row; ldp: digit-plane row pitch
  int planes;
  size_t flags, R, S, colmaxA, colbadA, colmaxB, colbadB, zero_end;
  size_t eprime, fprime, e, f, rowstat, colstat;
  size_t Abar, BbarT, partA, partB, planesA, planesB, cres, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int64_t m, int64_t n, int64_t k, int N, bool fast) {
  Layout L;
  L.kp = ((k + 31) / 32) * 32;
  L.ldp = plane_pitch(L.kp);
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
  L.colmaxA = take(4 * size_t(m));
  L.colbadA = take(4 * size_t(m));
  L.colmaxB = take(4 * size_t(n));
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
  L.planesA = take(size_t(L.planes) * m * L.ldp);
  L.planesB = take(size_t(L.planes) * n * L.ldp);
  L.cres = take(2 * size_t(N) * m * L.ldr);
  L.total = o;
  return L;
}

struct Ctx {
  int m, n, k, N;
  bool fast;
  bool timed = true;  // record the per-phase timing events (sequential calls only)
  uint64_t owned_use = 0;  // > 0: the call runs in the library-owned workspace, its use number
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
  uint64_t uses = 0;  // calls that have taken it
};
std::mutex g_ws_mutex;
OwnedWs g_ws[64];

uint8_t* owned_workspace(size_t need, ozk2_status* err, uint64_t* use = nullptr) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (take_fault(kFaultAlloc)) {  // injected: as if the workspace could not be obtained
    *err = OZK2_ERR_ALLOC;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_ws_mutex);
  OwnedWs& w = g_ws[dev];
  ++w.uses;
  if (use) *use = w.uses;
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
constexpr int kMaxRowBlocks = 5;  // output row blocks of a host-buffer call (4 + the split tail)

struct Timing {
  bool enabled = false;
  bool have = false;
  int dev = -1;
  cudaEvent_t ev[7] = {};
};
Timing g_timing;
std::mutex g_timing_mutex;
thread_local int t_launches = 0;

void timing_events() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_timing.dev != dev) {
    for (auto& e : g_timing.ev)
      if (e) cudaEventDestroy(e);
    for (auto& e : g_timing.ev) cudaEventCreate(&e);
    g_timing.dev = dev;
  }
}

// Phase boundary idx (0..6) of the call, on its stream.
void mark(Ctx& c, int idx) {
  if (!g_timing.enabled || !c.timed) return;
  timing_events();
  cudaEventRecord(g_timing.ev[idx], c.st);
  if (idx == 6) g_timing.have = true;
}

#define OZK2_TRY(expr)                      \
  do {                                      \
    cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) return OZK2_ERR_CUDA; \
  } while (0)

// 2-D copy that is issued as one linear copy when both sides are contiguous.
cudaError_t copy_2d(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                    cudaMemcpyKind kind, cudaStream_t st) {
  if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * height, kind, st);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, st);
}

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
    uint32_t* cm = c.at<uint32_t>(sd.colmax) + first;
    uint32_t* cb = c.at<uint32_t>(sd.colbad) + first;
    OZK2_TRY(launch_colmax(op.ptr, op.ld, c.k, lines, cm, cb, c.st));
    OZK2_TRY(launch_scale_cols(op.ptr, op.ld, c.k, lines, int(L.kp), cm, cb, ep, stat, bar,
                               c.at<float>(sd.part) + first * kb, sq, c.fast, c.at<uint32_t>(L.flags), c.st));
    t_launches += c.fast ? 3 : 2;
  }
  return OZK2_OK;
}

// Launch controls of an FP8 product launch: the device wait limit and the injected
// faults.  Returns false when an injected launch failure replaces this launch.
bool launch_controls(GemmArgs& g) {
  g.wait_ns = wait_limit_ns();
  g.stall = take_fault(kFaultStall);
  return !take_fault(kFaultLaunch);
}

// Bound product (accurate mode) of rows [i0, i0 + rows) of A with all of B: the row
// maxima R_i of those rows, and their share of the column maxima S_j (atomic maxima, so
// the row slices may come in any order).
cudaError_t bound_rows(Ctx& c, int64_t i0, int rows) {
  const Layout& L = c.L;
  GemmArgs g{};
  g.mode = kModeBound;
  g.m = rows;
  g.n = c.n;
  g.k = c.k;
  g.num_sms = c.num_sms;
  g.factor = bound_factor_f32(c.k);
  g.R = c.at<float>(L.R) + i0;
  g.S = c.at<float>(L.S);
  g.flags = c.at<uint32_t>(L.flags);
  g.tile_n = tile_for(c.n);
  if (!launch_controls(g)) return cudaErrorLaunchFailure;
  t_launches += 1;
  return launch_fp8_gemm(g, c.at<uint8_t>(L.Abar) + i0 * L.kp, L.kp, 1, c.at<uint8_t>(L.BbarT), L.kp, 1, c.st);
}

// Exponents e_i of rows [i0, i0 + rows) (Eq. 9); with cols, also every f_j.  Each needs
// its own final maximum (R_i: the bound products of row i with every column; S_j: those
// of column j with every row).
cudaError_t exponents_of(Ctx& c, int64_t i0, int rows, bool cols) {
  const Layout& L = c.L;
  t_launches += 1;
  return launch_exponents(rows, cols ? c.n : 0, c.at<int32_t>(L.eprime) + i0, c.at<int32_t>(L.fprime),
                          c.at<uint8_t>(L.rowstat) + i0, c.at<uint8_t>(L.colstat), c.at<float>(L.R) + i0,
                          c.at<float>(L.S), c.tab->pprime, delta_f32(), c.at<int32_t>(L.e) + i0,
                          c.at<int32_t>(L.f), c.st);
}

// Bound product (accurate mode) and the exponents e, f.
ozk2_status bound_and_exponents(Ctx& c) {
  mark(c, 1);
  if (!c.fast) OZK2_TRY(bound_rows(c, 0, c.m));
  mark(c, 2);
  OZK2_TRY(exponents_of(c, 0, c.m, true));
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

// plane_stride: bytes between the planes (0: lines * pitch; the whole operand's when
// `op`, `ex` and `planes` point at a slice of its lines).
cudaError_t residues_operand(Ctx& c, const Operand& op, int lines, const int32_t* ex, uint8_t* planes,
                             int64_t pitch, int64_t plane_stride = 0) {
  if (op.kcontig)
    return launch_residues_rows(op.ptr, op.ld, lines, c.k, int(c.L.kp), pitch, ex, c.tab->mt, planes,
                                c.at<uint32_t>(c.L.flags), c.st, plane_stride);
  return launch_residues_cols(op.ptr, op.ld, c.k, lines, int(c.L.kp), pitch, ex, c.tab->mt, planes,
                              c.at<uint32_t>(c.L.flags), c.st, plane_stride);
}

// pitch: row pitch of the destination planes (0: the workspace pitch L.ldp).
ozk2_status phase_residues(Ctx& c, const Operand& a, const Operand& b, const int32_t* e, const int32_t* f,
                           uint8_t* planesA, uint8_t* planesB, int64_t pitch = 0) {
  if (pitch == 0) pitch = c.L.ldp;
  OZK2_TRY(residues_operand(c, a, c.m, e, planesA, pitch));
  OZK2_TRY(residues_operand(c, b, c.n, f, planesB, pitch));
  t_launches += 2;
  mark(c, 4);
  return OZK2_OK;
}

// Residue products C'_l for output rows [i0, i0 + rows), on stream `st`.
ozk2_status products_rows(Ctx& c, int64_t i0, int rows, cudaStream_t st) {
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
  g.mt = &c.tab->mt;
  g.flags = c.at<uint32_t>(L.flags);
  g.plane_stride_a = int64_t(c.m) * L.ldp;
  g.plane_stride_b = int64_t(c.n) * L.ldp;
  g.tile_n = tile_for(c.n);
  g.split_squares = c.k <= g_split_kmax.load();
  if (!launch_controls(g)) return OZK2_ERR_CUDA;
  OZK2_TRY(launch_fp8_gemm(g, c.at<uint8_t>(L.planesA) + i0 * L.ldp, L.ldp, L.planes, c.at<uint8_t>(L.planesB),
                           L.ldp, L.planes, st));
  t_launches += 1;
  return OZK2_OK;
}

ozk2_status phase_products(Ctx& c) {
  ozk2_status s = products_rows(c, 0, c.m, c.st);
  if (s != OZK2_OK) return s;
  mark(c, 5);
  return OZK2_OK;
}

// CRT and inverse scaling of output rows [i0, i0 + rows) into C (which points at row i0).
ozk2_status crt_rows(Ctx& c, int64_t i0, int rows, const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                     const uint8_t* colstat, double* C, int64_t ldc, cudaStream_t st) {
  const Layout& L = c.L;
  OZK2_TRY(launch_crt(c.at<int16_t>(L.cres) + i0 * L.ldr, L.ldr, int64_t(c.m) * L.ldr, rows, c.n, e + i0, f,
                      rowstat ? rowstat + i0 : nullptr, colstat, C, ldc, c.tab->ct, st));
  t_launches += 1;
  return OZK2_OK;
}

ozk2_status phase_crt(Ctx& c, const int32_t* e, const int32_t* f, const uint8_t* rowstat,
                      const uint8_t* colstat, double* C, int64_t ldc) {
  ozk2_status s = crt_rows(c, 0, c.m, e, f, rowstat, colstat, C, ldc, c.st);
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
// ws_trusted: `ws` is memory of this library (the static array of ozk2_dgemm_noalloc),
// known to be device memory of the current device.
ozk2_status setup(Ctx& c, int64_t m, int64_t n, int64_t k, int N, bool fast, void* ws, size_t ws_bytes,
                  cudaStream_t st, size_t extra = 0, bool ws_trusted = false) {
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
    if (!ws_trusted && !device_memory_here(ws)) return OZK2_ERR_INVALID_VALUE;
    c.ws = static_cast<uint8_t*>(ws);
  } else {
    ozk2_status err = OZK2_OK;
    c.ws = owned_workspace(c.L.total + extra, &err, &c.owned_use);
    if (!c.ws) return err;
  }
  return OZK2_OK;
}

// ------------------------------------------------------------------ products and CRT
// Copy of finished output row blocks to the host (the host-buffer call).
struct CopyBack {
  double* hC;
  int64_t ldc;
  cudaStream_t cs;
  cudaEvent_t* done;  // one event per row block
};

// Row blocks of a host-buffer call: each at least 16 waves of GEMM units (a persistent
// launch loses up to one wave at its end), at most four, 128-row aligned.  When there
// are several, the last is split a quarter from its end, so that the download left
// after the last CRT is a quarter of a block.  Returns the count; first[b] is the first
// row of block b, first[count] = m.
int row_blocks(const Ctx& c, int64_t (&first)[kMaxRowBlocks + 1]) {
  const int64_t units = ((int64_t(c.m) + 127) / 128) * ((int64_t(c.n) + 255) / 256) * c.N;
  const int64_t nb = std::max<int64_t>(1, std::min<int64_t>(4, units / (16 * int64_t(c.num_sms))));
  const int64_t rb = ((c.m + nb - 1) / nb + 127) / 128 * 128;
  int count = 0;
  for (int64_t i0 = 0; i0 < c.m; i0 += rb) first[count++] = i0;
  if (count > 1) {
    const int64_t last = first[count - 1], rows = c.m - last;
    const int64_t tail = ((rows + 3) / 4 + 127) / 128 * 128;
    if (rows > tail) first[count++] = c.m - tail;
  }
  first[count] = c.m;
  return count;
}

// After the scaling, the exponents and B's residues (all on c.st): A's residues (unless
// `a` is null: already converted), the residue products and the CRT, in order on c.st.
// C (device, row-major, ldc) receives the result.  With cb the products and the CRT run
// in output row blocks, and block b is copied to cb->hC on cb->cs while block b + 1 is
// computed.  (Running the conversion kernels on a second stream beside the persistent
// GEMM was measured and gains nothing: they get too little of an SM next to it.)
ozk2_status products_and_crt(Ctx& c, const Operand* a, double* C, int64_t ldc, const CopyBack* cb) {
  const Layout& L = c.L;
  const int32_t* e = c.at<int32_t>(L.e);
  const int32_t* f = c.at<int32_t>(L.f);
  const uint8_t* rs = c.at<uint8_t>(L.rowstat);
  const uint8_t* cs = c.at<uint8_t>(L.colstat);
  if (a) {
    OZK2_TRY(residues_operand(c, *a, c.m, e, c.at<uint8_t>(L.planesA), L.ldp));
    t_launches += 1;
  }
  mark(c, 4);
  ozk2_status s;
  if (!cb) {
    if ((s = phase_products(c)) != OZK2_OK) return s;
    return phase_crt(c, e, f, rs, cs, C, ldc);
  }
  int64_t first[kMaxRowBlocks + 1];
  const int nb = row_blocks(c, first);
  for (int b = 0; b < nb; ++b) {
    const int64_t i0 = first[b];
    const int rows = int(first[b + 1] - i0);
    if ((s = products_rows(c, i0, rows, c.st)) != OZK2_OK) return s;
    if ((s = crt_rows(c, i0, rows, e, f, rs, cs, C + i0 * ldc, ldc, c.st)) != OZK2_OK) return s;
    OZK2_TRY(cudaEventRecord(cb->done[b], c.st));
    OZK2_TRY(cudaStreamWaitEvent(cb->cs, cb->done[b], 0));
    OZK2_TRY(copy_2d(cb->hC + i0 * cb->ldc, size_t(cb->ldc) * 8, C + i0 * ldc, size_t(ldc) * 8, size_t(c.n) * 8,
                     size_t(rows), cudaMemcpyDeviceToHost, cb->cs));
  }
  return OZK2_OK;
}

// One emulated product over whole operands (no blocking); arguments already validated,
// m, n, k > 0.
ozk2_status run_one(const Operand& a, const Operand& b, int64_t m, int64_t n, int64_t k, double* C, int64_t ldc,
                    int N, bool fast, bool first, void* ws, size_t ws_bytes, cudaStream_t st, bool ws_trusted) {
  Ctx c;
  ozk2_status s = setup(c, m, n, k, N, fast, ws, ws_bytes, st, 0, ws_trusted);
  if (s != OZK2_OK) return s;
  mark(c, 0);
  const Layout& L = c.L;
  if ((s = phase_scales(c, a, b, first)) != OZK2_OK) return s;
  OZK2_TRY(residues_operand(c, b, c.n, c.at<int32_t>(L.f), c.at<uint8_t>(L.planesB), L.ldp));
  t_launches += 1;
  return products_and_crt(c, &a, C, ldc, nullptr);
}

int64_t block_or_all(int64_t b, int64_t total) { return (b <= 0 || b >= total) ? total : b; }

size_t workspace_bytes(int64_t m, int64_t n, int64_t k, int N, bool fast, int64_t bm, int64_t bn) {
  return make_layout(block_or_all(bm, m), block_or_all(bn, n), k, N, fast).total;
}

ozk2_status dgemm_general(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                          int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int N, int mode,
                          int64_t block_m, int64_t block_n, void* ws, size_t ws_bytes, cudaStream_t st,
                          bool ws_trusted = false) {
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
                  i0 == 0 && j0 == 0, ws, ws_bytes, st, ws_trusted);
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
constexpr int kHostEvents = 2 + kHostChunks + kMaxRowBlocks + 1;

struct CopyEngine {
  cudaStream_t up = nullptr, down = nullptr;  // host-to-device and device-to-host copies
  cudaEvent_t ev[kHostEvents] = {};
  // The last host-buffer call in the owned workspace: recorded on its stream once its
  // kernels have read the staged A and B for the last time, with the workspace use
  // number and the staging range of that call.
  cudaEvent_t staged_free = nullptr;
  uint64_t staged_use = 0;
  const uint8_t* staged_at = nullptr;
  size_t staged_bytes = 0;
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
  if (!e.up) {
    if (cudaStreamCreateWithFlags(&e.down, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e.up, cudaStreamNonBlocking) != cudaSuccess) {
      *err = OZK2_ERR_CUDA;
      e.up = nullptr;
      return nullptr;
    }
    for (auto& ev : e.ev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        *err = OZK2_ERR_CUDA;
        return nullptr;
      }
    if (cudaEventCreateWithFlags(&e.staged_free, cudaEventDisableTiming) != cudaSuccess) {
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
    return copy_2d(dst + i0 * k, size_t(k) * 8, src + i0 * ld, size_t(ld) * 8, size_t(k) * 8, size_t(i1 - i0),
                   cudaMemcpyHostToDevice, cs);
  return copy_2d(dst + i0, size_t(lines) * 8, src + i0, size_t(ld) * 8, size_t(i1 - i0) * 8, size_t(k),
                 cudaMemcpyHostToDevice, cs);
}

// C = op(A) op(B) from host buffers.  B goes up first, then A in line chunks, on the copy
// stream.  B's scaling runs once B is in; each chunk of A is then scaled, bounded against
// all of B (accurate mode; its rows' maxima R_i are then final), given its exponents e_i
// and converted to digit planes while the next chunk is still on its way.  Only the
// column exponents f_j wait for the whole of A (S_j is a maximum over every row), and
// with them B's residues.  The residue products and the CRT then run in output row
// blocks, block b streaming back while block b + 1 is computed.  Every kernel does the
// same arithmetic as in the device-buffer call, so the results are bit-identical.
ozk2_status run_host(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* hA,
                     int64_t lda, const double* hB, int64_t ldb, double* hC, int64_t ldc, int N, bool fast,
                     unsigned flags, void* ws, size_t ws_bytes, cudaStream_t st) {
  ozk2_status s;
  CopyEngine* ce = copy_engine(&s);
  if (!ce) return s;
  Ctx c;
  const Staging G = make_staging(m, n, k);
  if ((s = setup(c, m, n, k, N, fast, ws, ws_bytes, st, G.total)) != OZK2_OK) return s;
  // Timed phases on `st`: 0 start, 1 last chunk of A scaled (the uploads done), 2 its
  // bound product, 3 its residues, 4 B's residues (accurate mode), 5 last block's CRT,
  // 6 last block back.
  mark(c, 0);
  const Layout& L = c.L;
  double* dA = c.at<double>(L.total + G.A);
  double* dB = c.at<double>(L.total + G.B);
  double* dC = c.at<double>(L.total + G.C);
  const bool a_kc = transa == OZK2_OP_N, b_kc = transb == OZK2_OP_T;
  const Operand a = operand_a(transa, dA, a_kc ? k : m);
  const Operand b = operand_b(transb, dB, b_kc ? k : n);
  cudaStream_t up = ce->up;
  cudaEvent_t* ev = ce->ev;
  cudaEvent_t ev_start = ev[0], ev_b = ev[1], *ev_a = ev + 2, *ev_blk = ev + 2 + kHostChunks,
              ev_done = ev[kHostEvents - 1];

  // Nothing is copied into the workspace before earlier work on `st` is done with it.
  // With OZK2_HOST_INPUTS_READY, when the previous use of the owned workspace was a host
  // call with the same staging, "done with it" is that call's last read of its staged
  // A and B, so the upload overlaps its residue products.
  const uint8_t* stage = c.ws + L.total;
  const bool early = (flags & OZK2_HOST_INPUTS_READY) && c.owned_use > 0 && ce->staged_use + 1 == c.owned_use &&
                     ce->staged_at == stage && ce->staged_bytes == G.total;
  if (early) {
    OZK2_TRY(cudaStreamWaitEvent(up, ce->staged_free, 0));
  } else {
    OZK2_TRY(cudaEventRecord(ev_start, st));
    OZK2_TRY(cudaStreamWaitEvent(up, ev_start, 0));
  }
  OZK2_TRY(copy_lines_h2d(dB, hB, ldb, b_kc, n, k, 0, n, up));
  OZK2_TRY(cudaEventRecord(ev_b, up));
  const int64_t chunk = (m + kHostChunks - 1) / kHostChunks;
  for (int q = 0; q < kHostChunks; ++q) {
    OZK2_TRY(copy_lines_h2d(dA, hA, lda, a_kc, m, k, std::min(m, q * chunk), std::min(m, (q + 1) * chunk), up));
    OZK2_TRY(cudaEventRecord(ev_a[q], up));
  }

  if ((s = zero_scratch(c, true)) != OZK2_OK) return s;
  OZK2_TRY(cudaStreamWaitEvent(st, ev_b, 0));
  if ((s = scale_operand(c, b, 0, int(n), side_b(L))) != OZK2_OK) return s;
  // fast mode: f_j depends on column j of B alone (Sec. III-E with the Cauchy-Schwarz
  // bound), so B's residues need not wait for A
  auto residues_b = [&]() -> ozk2_status {
    OZK2_TRY(exponents_of(c, 0, 0, true));
    OZK2_TRY(residues_operand(c, b, int(n), c.at<int32_t>(L.f), c.at<uint8_t>(L.planesB), L.ldp));
    t_launches += 1;
    return OZK2_OK;
  };
  if (fast && (s = residues_b()) != OZK2_OK) return s;
  const int64_t planes_a_stride = int64_t(m) * L.ldp;
  for (int q = 0; q < kHostChunks; ++q) {
    const int64_t i0 = std::min(m, q * chunk), i1 = std::min(m, (q + 1) * chunk);
    const bool last = q == kHostChunks - 1;
    OZK2_TRY(cudaStreamWaitEvent(st, ev_a[q], 0));
    if (i1 > i0) {
      const int rows = int(i1 - i0);
      const Operand ai = shift_lines(a, i0);
      if ((s = scale_operand(c, ai, i0, rows, side_a(L))) != OZK2_OK) return s;
      if (last) mark(c, 1);
      if (!fast) OZK2_TRY(bound_rows(c, i0, rows));
      if (last) mark(c, 2);
      OZK2_TRY(exponents_of(c, i0, rows, false));
      OZK2_TRY(residues_operand(c, ai, rows, c.at<int32_t>(L.e) + i0, c.at<uint8_t>(L.planesA) + i0 * L.ldp,
                                L.ldp, planes_a_stride));
      t_launches += 1;
    } else if (last) {
      mark(c, 1);
      mark(c, 2);
    }
  }
  mark(c, 3);
  if (!fast && (s = residues_b()) != OZK2_OK) return s;
  // the staged A and B are not read again by this call
  OZK2_TRY(cudaEventRecord(ce->staged_free, st));
  ce->staged_use = c.owned_use;
  ce->staged_at = stage;
  ce->staged_bytes = G.total;
  // residue products and CRT in output row blocks; each finished block streams back
  const CopyBack cb{hC, ldc, ce->down, ev_blk};
  if ((s = products_and_crt(c, nullptr, dC, n, &cb)) != OZK2_OK) return s;
  mark(c, 5);
  // the call is complete on `st` once the last block is back on the host
  OZK2_TRY(cudaEventRecord(ev_done, ce->down));
  OZK2_TRY(cudaStreamWaitEvent(st, ev_done, 0));
  mark(c, 6);
  return OZK2_OK;
}

size_t host_workspace_bytes(int64_t m, int64_t n, int64_t k, int N, bool fast) {
  return make_layout(m, n, k, N, fast).total + make_staging(m, n, k).total;
}

// ------------------------------------------------------------------ gradients with reuse
// dA = dC B^T and dB = A^T dC for C = A B computed in a caller workspace, reusing that
// call's exponents e, f and digit planes of A' = trunc(diag(2^e) A), B' = trunc(B diag(2^f)):
//   dA: G'_ij = trunc(2^(g_i - f_j) dC_ij); (G' B'^T)_ih = 2^g_i dA_ih (up to truncation)
//   dB: H'_ij = trunc(2^(h_j - e_i) dC_ij); (A'^T H')_hj = 2^h_j dB_hj
// The exponents g, h of dC's side come from FP8 bound products of |dC| with |B| (rows of
// B as lines) and of |A| (columns as lines) with |dC|, whose maxima remove the lines'
// own FP8 scalings (colshift / rowshift), under the budget Q = log2(P - 1) - 1 (B' and A'
// are fixed).  The forward's planes are transposed into the layout the products read.
struct BwLayout {
  int64_t np, mp, ldrk, ldrn;
  int planes;
  size_t flags, R, S, Rk, Sk, colmaxA, colbadA, colmaxC, colbadC, zk, zero_end;
  size_t gp, hp, g, h, t, tA, rstatC, cstatC, rstatB, cstatA;
  size_t Gbar, Bhat, AhatT, HhatT, planesG, planesBT, planesAT, planesH, cresA, cresB, total;
};

BwLayout make_bw_layout(int64_t m, int64_t n, int64_t k, int N) {
  BwLayout L;
  L.np = ((n + 31) / 32) * 32;
  L.mp = ((m + 31) / 32) * 32;
  L.ldrk = ((k + 7) / 8) * 8;
  L.ldrn = ((n + 7) / 8) * 8;
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
  L.Rk = take(4 * size_t(k));
  L.Sk = take(4 * size_t(k));
  L.colmaxA = take(4 * size_t(k));
  L.colbadA = take(4 * size_t(k));
  L.colmaxC = take(4 * size_t(n));
  L.colbadC = take(4 * size_t(n));
  L.zk = take(4 * size_t(k));
  L.zero_end = o;
  L.gp = take(4 * size_t(m));
  L.hp = take(4 * size_t(n));
  L.g = take(4 * size_t(m));
  L.h = take(4 * size_t(n));
  L.t = take(4 * size_t(k));
  L.tA = take(4 * size_t(k));
  L.rstatC = take(size_t(m));
  L.cstatC = take(size_t(n));
  L.rstatB = take(size_t(k));
  L.cstatA = take(size_t(k));
  L.Gbar = take(size_t(m) * L.np);
  L.Bhat = take(size_t(k) * L.np);
  L.AhatT = take(size_t(k) * L.mp);
  L.HhatT = take(size_t(n) * L.mp);
  L.planesG = take(size_t(L.planes) * m * L.np);
  L.planesBT = take(size_t(L.planes) * k * L.np);
  L.planesAT = take(size_t(L.planes) * k * L.mp);
  L.planesH = take(size_t(L.planes) * n * L.mp);
  L.cresA = take(2 * size_t(N) * m * L.ldrk);
  L.cresB = take(2 * size_t(N) * k * L.ldrn);
  L.total = o;
  return L;
}

// One bound product for the gradient exponents (single problem, accurate mode).
cudaError_t bw_bound(const Ctx& c, const uint8_t* a, const uint8_t* b, int64_t pitch, int rows, int cols, int len,
                     float* R, float* S, const int32_t* colshift, const int32_t* rowshift, uint32_t* flags) {
  GemmArgs g{};
  g.mode = kModeBound;
  g.m = rows;
  g.n = cols;
  g.k = len;
  g.num_sms = c.num_sms;
  g.factor = bound_factor_f32(len);
  g.R = R;
  g.S = S;
  g.colshift = colshift;
  g.rowshift = rowshift;
  g.flags = flags;
  g.tile_n = tile_for(cols);
  if (!launch_controls(g)) return cudaErrorLaunchFailure;
  t_launches += 1;
  return launch_fp8_gemm(g, a, pitch, 1, b, pitch, 1, c.st);
}

// Residue products of one gradient: `planes` planes of a (rows lines) and b (cols lines),
// contraction len, row pitch `pitch`, into cres (N x rows x ldr).
cudaError_t bw_products(const Ctx& c, const uint8_t* a, const uint8_t* b, int64_t pitch, int rows, int cols, int len,
                        int16_t* cres, int64_t ldr, uint32_t* flags) {
  GemmArgs g{};
  g.mode = kModeResidue;
  g.m = rows;
  g.n = cols;
  g.k = len;
  g.num_sms = c.num_sms;
  g.cres = cres;
  g.ldr = ldr;
  g.res_stride = int64_t(rows) * ldr;
  g.mt = &c.tab->mt;
  g.flags = flags;
  g.plane_stride_a = int64_t(rows) * pitch;
  g.plane_stride_b = int64_t(cols) * pitch;
  g.tile_n = tile_for(cols);
  g.split_squares = len <= g_split_kmax.load();
  if (!launch_controls(g)) return cudaErrorLaunchFailure;
  t_launches += 1;
  return launch_fp8_gemm(g, a, pitch, c.tab->mt.num_planes, b, pitch, c.tab->mt.num_planes, c.st);
}

ozk2_status run_backward(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                         int64_t ldb, const double* dC, int64_t lddc, double* dA, int64_t ldda, double* dB,
                         int64_t lddb, int N, const void* fws, size_t fws_bytes, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
  Ctx c;
  c.m = int(m);
  c.n = int(n);
  c.k = int(k);
  c.N = N;
  c.st = st;
  if (!device_info(&c.num_sms)) return OZK2_ERR_UNSUPPORTED;
  if (!encode_fn()) return OZK2_ERR_CUDA;
  c.tab = tables_for(N);
  if (!c.tab) return OZK2_ERR_INTERNAL;
  const Layout FL = make_layout(m, n, k, N, false);
  if (!fws || fws_bytes < FL.total || (reinterpret_cast<uintptr_t>(fws) & 255u) || !device_memory_here(fws))
    return OZK2_ERR_INVALID_VALUE;
  const BwLayout L = make_bw_layout(m, n, k, N);
  uint8_t* w;
  if (ws) {
    if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) || !device_memory_here(ws))
      return OZK2_ERR_INVALID_VALUE;
    w = static_cast<uint8_t*>(ws);
  } else {
    ozk2_status err = OZK2_OK;
    w = owned_workspace(L.total, &err);
    if (!w) return err;
  }
  auto at = [w](size_t off) { return w + off; };
  const uint8_t* f8 = static_cast<const uint8_t*>(fws);
  const int32_t* e = reinterpret_cast<const int32_t*>(f8 + FL.e);
  const int32_t* f = reinterpret_cast<const int32_t*>(f8 + FL.f);
  const uint8_t* planesA = f8 + FL.planesA;
  const uint8_t* planesB = f8 + FL.planesB;
  uint32_t* flags = reinterpret_cast<uint32_t*>(at(L.flags));
  const int P = L.planes;
  int32_t* gp = reinterpret_cast<int32_t*>(at(L.gp));
  int32_t* hp = reinterpret_cast<int32_t*>(at(L.hp));
  int32_t* g = reinterpret_cast<int32_t*>(at(L.g));
  int32_t* h = reinterpret_cast<int32_t*>(at(L.h));
  const int32_t* zk = reinterpret_cast<const int32_t*>(at(L.zk));
  OZK2_TRY(cudaMemsetAsync(w, 0, L.zero_end, st));
  const bool wantA = dA != nullptr, wantB = dB != nullptr;
  // bounds and exponents of dC's rows (dA) and columns (dB)
  if (wantA) {
    OZK2_TRY(launch_scale_rows(dC, lddc, c.m, c.n, int(L.np), gp, at(L.rstatC), at(L.Gbar), nullptr, false, flags, st));
    OZK2_TRY(launch_scale_rows(B, ldb, c.k, c.n, int(L.np), reinterpret_cast<int32_t*>(at(L.t)), at(L.rstatB),
                               at(L.Bhat), nullptr, false, flags, st));
    OZK2_TRY(bw_bound(c, at(L.Gbar), at(L.Bhat), L.np, c.m, c.k, c.n, reinterpret_cast<float*>(at(L.R)),
                      reinterpret_cast<float*>(at(L.Sk)), reinterpret_cast<const int32_t*>(at(L.t)), nullptr, flags));
    t_launches += 2;
  }
  if (wantB) {
    uint32_t* cmC = reinterpret_cast<uint32_t*>(at(L.colmaxC));
    uint32_t* cbC = reinterpret_cast<uint32_t*>(at(L.colbadC));
    OZK2_TRY(launch_colmax(dC, lddc, c.m, c.n, cmC, cbC, st));
    OZK2_TRY(launch_scale_cols(dC, lddc, c.m, c.n, int(L.mp), cmC, cbC, hp, at(L.cstatC), at(L.HhatT), nullptr,
                               nullptr, false, flags, st));
    uint32_t* cmA = reinterpret_cast<uint32_t*>(at(L.colmaxA));
    uint32_t* cbA = reinterpret_cast<uint32_t*>(at(L.colbadA));
    OZK2_TRY(launch_colmax(A, lda, c.m, c.k, cmA, cbA, st));
    OZK2_TRY(launch_scale_cols(A, lda, c.m, c.k, int(L.mp), cmA, cbA, reinterpret_cast<int32_t*>(at(L.tA)),
                               at(L.cstatA), at(L.AhatT), nullptr, nullptr, false, flags, st));
    OZK2_TRY(bw_bound(c, at(L.AhatT), at(L.HhatT), L.mp, c.k, c.n, c.m, reinterpret_cast<float*>(at(L.Rk)),
                      reinterpret_cast<float*>(at(L.S)), nullptr, reinterpret_cast<const int32_t*>(at(L.tA)), flags));
    t_launches += 4;
  }
  OZK2_TRY(launch_reuse_exponents(wantA ? c.m : 0, gp, at(L.rstatC), reinterpret_cast<float*>(at(L.R)), g,
                                  wantB ? c.n : 0, hp, at(L.cstatC), reinterpret_cast<float*>(at(L.S)), h,
                                  reuse_budget_f32(N), flags, st));
  // dC's two integer matrices from one read of dC; the forward's planes transposed
  OZK2_TRY(launch_grad_residues(dC, lddc, c.m, c.n, g, f, h, e, wantA ? at(L.planesG) : nullptr, L.np,
                                wantB ? at(L.planesH) : nullptr, L.mp, c.tab->mt, flags, st));
  t_launches += 2;
  if (wantA) {
    OZK2_TRY(launch_transpose_planes(planesB, FL.ldp, int64_t(n) * FL.ldp, c.n, c.k, at(L.planesBT), L.np,
                                     int64_t(k) * L.np, P, st));
    OZK2_TRY(bw_products(c, at(L.planesG), at(L.planesBT), L.np, c.m, c.k, c.n,
                         reinterpret_cast<int16_t*>(at(L.cresA)), L.ldrk, flags));
    OZK2_TRY(launch_crt(reinterpret_cast<int16_t*>(at(L.cresA)), L.ldrk, int64_t(m) * L.ldrk, c.m, c.k, g, zk,
                        at(L.rstatC), at(L.rstatB), dA, ldda, c.tab->ct, st));
    t_launches += 2;
  }
  if (wantB) {
    OZK2_TRY(launch_transpose_planes(planesA, FL.ldp, int64_t(m) * FL.ldp, c.m, c.k, at(L.planesAT), L.mp,
                                     int64_t(k) * L.mp, P, st));
    OZK2_TRY(bw_products(c, at(L.planesAT), at(L.planesH), L.mp, c.k, c.n, c.m,
                         reinterpret_cast<int16_t*>(at(L.cresB)), L.ldrn, flags));
    OZK2_TRY(launch_crt(reinterpret_cast<int16_t*>(at(L.cresB)), L.ldrn, int64_t(k) * L.ldrn, c.k, c.n, zk, h,
                        at(L.cstatA), at(L.cstatC), dB, lddb, c.tab->ct, st));
    t_launches += 2;
  }
  return OZK2_OK;
}

// ------------------------------------------------------------------ batches
// A batch plan: the descriptors of every problem, uploaded once into a device workspace,
// and the totals of each grouped launch.  Executing it issues one launch per phase for
// the whole batch (plus one memset of the bound maxima), with no host work, so it can
// be captured into a CUDA graph.
struct ZeroK {
  double* C;
  int64_t ldc, m, n;
};

struct BatchLayout {
  size_t flags, probs, gbound, gres, zero_begin, zero_end, total;
};

}  // namespace
}  // namespace ozk2

struct ozk2_batch_plan_st {
  int dev = -1;
  int N = 0;
  bool fast = false;
  int cnt = 0;  // problems with m, n, k > 0
  std::vector<ozk2::ZeroK> zero_k;
  uint8_t* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  ozk2::BatchLayout L{};
  int64_t totals[ozk2::kBatchKernels] = {};
  int64_t units_bound = 0;
  // The residue products run in up to two grouped launches: the first res_cnt[0]
  // descriptors in 256-wide tiles, the next res_cnt[1] in 128-wide tiles.
  int res_cnt[2] = {0, 0};
  int64_t res_units[2] = {0, 0};
  int num_sms = 0;
  int tile_n = 256;      // tile width of the residue products (0: both widths)
  int bound_tile = 256;  // tile width of the bound products
  const void* tab = nullptr;  // ozk2::Tables
  uint8_t* host = nullptr;    // pinned copy of the uploaded descriptors
  size_t host_bytes = 0;
  cudaEvent_t uploaded = nullptr;
  // B's scaling and residue kernels run on this second stream beside A's (fork and join
  // through the two events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

namespace ozk2 {
namespace {

ozk2_status validate_batch(int count, const int64_t* m, const int64_t* n, const int64_t* k, const double* const* A,
                           const int64_t* lda, const double* const* B, const int64_t* ldb, double* const* C,
                           const int64_t* ldc, int N, int mode) {
  if (count < 0 || !valid_mode(mode) || N < 1 || N > kMaxModuli) return OZK2_ERR_INVALID_VALUE;
  if (count == 0) return OZK2_OK;
  if (!m || !n || !k || !A || !lda || !B || !ldb || !C || !ldc) return OZK2_ERR_INVALID_VALUE;
  for (int i = 0; i < count; ++i) {
    const ozk2_status s = validate(OZK2_OP_N, OZK2_OP_N, m[i], n[i], k[i], A[i], lda[i], B[i], ldb[i], C[i], ldc[i], N);
    if (s != OZK2_OK) return s;
  }
  return OZK2_OK;
}

bool active_problem(int64_t m, int64_t n, int64_t k) { return m > 0 && n > 0 && k > 0; }

// Offsets of the batch workspace; with `probs`, also the per-problem pointers (relative
// to a null base, rebased by the caller).
BatchLayout batch_layout(int count, const int64_t* m, const int64_t* n, const int64_t* k, int N, bool fast,
                         std::vector<BatchProblem>* probs) {
  BatchLayout L{};
  const int planes = (N <= kNumSquares) ? 2 * N : 3 * N - kNumSquares;
  int cnt = 0;
  for (int i = 0; i < count; ++i) cnt += active_problem(m[i], n[i], k[i]) ? 1 : 0;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.flags = take(256);
  L.probs = take(sizeof(BatchProblem) * size_t(cnt));
  L.gbound = fast ? o : take(sizeof(GemmProblem) * size_t(cnt));
  L.gres = take(sizeof(GemmProblem) * size_t(cnt));
  if (probs) probs->assign(size_t(cnt), BatchProblem{});
  auto P = [&](int j) -> BatchProblem& { return (*probs)[size_t(j)]; };
  auto at = [](size_t off) { return reinterpret_cast<uint8_t*>(off); };
  L.zero_begin = o;
  for (int i = 0, j = 0; i < count; ++i) {
    if (!active_problem(m[i], n[i], k[i])) continue;
    const size_t R = take(4 * size_t(m[i])), S = take(4 * size_t(n[i]));
    const size_t cm = take(4 * size_t(n[i])), cb = take(4 * size_t(n[i]));
    if (probs) {
      P(j).R = reinterpret_cast<float*>(at(R));
      P(j).S = reinterpret_cast<float*>(at(S));
      P(j).colmaxB = reinterpret_cast<uint32_t*>(at(cm));
      P(j).colbadB = reinterpret_cast<uint32_t*>(at(cb));
    }
    ++j;
  }
  L.zero_end = o;
  for (int i = 0, j = 0; i < count; ++i) {
    if (!active_problem(m[i], n[i], k[i])) continue;
    const int64_t mi = m[i], ni = n[i], kp = ((k[i] + 31) / 32) * 32, ldp = plane_pitch(kp),
                  ldr = ((ni + 7) / 8) * 8;
    const size_t ep = take(4 * size_t(mi)), fp = take(4 * size_t(ni)), e = take(4 * size_t(mi)),
                 f = take(4 * size_t(ni)), rs = take(size_t(mi)), cs = take(size_t(ni));
    const size_t abar = fast ? 0 : take(size_t(mi) * kp), bbar = fast ? 0 : take(size_t(ni) * kp);
    const size_t part = fast ? take(4 * size_t(ni) * size_t(kp / 32)) : 0;
    const size_t pa = take(size_t(planes) * mi * ldp), pb = take(size_t(planes) * ni * ldp);
    const size_t cres = take(2 * size_t(N) * mi * ldr);
    if (probs) {
      BatchProblem& q = P(j);
      q.m = int(mi);
      q.n = int(ni);
      q.k = int(k[i]);
      q.kp = int(kp);
      q.ldp = ldp;
      q.ldr = ldr;
      q.eprime = reinterpret_cast<int32_t*>(at(ep));
      q.fprime = reinterpret_cast<int32_t*>(at(fp));
      q.e = reinterpret_cast<int32_t*>(at(e));
      q.f = reinterpret_cast<int32_t*>(at(f));
      q.rowstat = at(rs);
      q.colstat = at(cs);
      q.Abar = fast ? nullptr : at(abar);
      q.BbarT = fast ? nullptr : at(bbar);
      q.partB = fast ? reinterpret_cast<float*>(at(part)) : nullptr;
      q.planesA = at(pa);
      q.planesB = at(pb);
      q.cres = reinterpret_cast<int16_t*>(at(cres));
    }
    ++j;
  }
  L.total = o;
  return L;
}

template <typename T>
T* rebase(T* rel, uint8_t* base) {
  return rel ? reinterpret_cast<T*>(base + reinterpret_cast<uintptr_t>(rel)) : nullptr;
}

void destroy_plan(ozk2_batch_plan plan) {
  if (!plan) return;
  if (plan->uploaded) {
    cudaEventSynchronize(plan->uploaded);
    cudaEventDestroy(plan->uploaded);
  }
  if (plan->host) cudaFreeHost(plan->host);
  if (plan->side) cudaStreamDestroy(plan->side);  // released once its work is done
  if (plan->fork) cudaEventDestroy(plan->fork);
  if (plan->join) cudaEventDestroy(plan->join);
  if (plan->owns_ws && plan->ws) cudaFree(plan->ws);
  delete plan;
}

// Builds the plan and enqueues the descriptor upload on `st`.  ws == nullptr with
// use_owned: the library-owned workspace; ws == nullptr otherwise: a private allocation.
ozk2_status create_plan(ozk2_batch_plan* out, int count, const int64_t* m, const int64_t* n, const int64_t* k,
                        const double* const* A, const int64_t* lda, const double* const* B, const int64_t* ldb,
                        double* const* C, const int64_t* ldc, int N, int mode, void* ws, size_t ws_bytes,
                        bool use_owned, cudaStream_t st) {
  if (!out) return OZK2_ERR_INVALID_VALUE;
  *out = nullptr;
  ozk2_status s = validate_batch(count, m, n, k, A, lda, B, ldb, C, ldc, N, mode);
  if (s != OZK2_OK) return s;
  int sms = 0;
  if (!device_info(&sms)) return OZK2_ERR_UNSUPPORTED;
  if (!encode_fn()) return OZK2_ERR_CUDA;
  const Tables* tab = tables_for(N);
  if (!tab) return OZK2_ERR_INTERNAL;
  const bool fast = mode == OZK2_MODE_FAST;
  ozk2_batch_plan plan = new ozk2_batch_plan_st;
  cudaGetDevice(&plan->dev);
  plan->N = N;
  plan->fast = fast;
  plan->num_sms = sms;
  plan->tab = tab;
  for (int i = 0; i < count; ++i)
    if (m[i] > 0 && n[i] > 0 && k[i] == 0) plan->zero_k.push_back(ZeroK{C[i], ldc[i], m[i], n[i]});
  std::vector<BatchProblem> probs;
  plan->L = batch_layout(count, m, n, k, N, fast, &probs);
  plan->cnt = int(probs.size());
  const BatchLayout& L = plan->L;
  if (ws) {
    if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255u) || !device_memory_here(ws)) {
      destroy_plan(plan);
      return OZK2_ERR_INVALID_VALUE;
    }
    plan->ws = static_cast<uint8_t*>(ws);
  } else if (use_owned) {
    ozk2_status err = OZK2_OK;
    plan->ws = owned_workspace(L.total, &err);
    if (!plan->ws) {
      destroy_plan(plan);
      return err;
    }
  } else {
    void* p = nullptr;
    if (take_fault(kFaultAlloc) || cudaMalloc(&p, L.total) != cudaSuccess) {
      cudaGetLastError();
      destroy_plan(plan);
      return OZK2_ERR_ALLOC;
    }
    plan->ws = static_cast<uint8_t*>(p);
    plan->owns_ws = true;
  }
  plan->ws_bytes = L.total;
  uint8_t* base = plan->ws;
  // operands, pointers, block prefixes; GEMM problems sorted by k (longest units first)
  std::vector<int> order;
  int64_t running[kBatchKernels] = {};
  for (int i = 0, j = 0; i < count; ++i) {
    if (!active_problem(m[i], n[i], k[i])) continue;
    BatchProblem& q = probs[size_t(j)];
    q.A = A[i];
    q.lda = lda[i];
    q.B = B[i];
    q.ldb = ldb[i];
    q.C = C[i];
    q.ldc = ldc[i];
    q.R = rebase(q.R, base);
    q.S = rebase(q.S, base);
    q.colmaxB = rebase(q.colmaxB, base);
    q.colbadB = rebase(q.colbadB, base);
    q.eprime = rebase(q.eprime, base);
    q.fprime = rebase(q.fprime, base);
    q.e = rebase(q.e, base);
    q.f = rebase(q.f, base);
    q.rowstat = rebase(q.rowstat, base);
    q.colstat = rebase(q.colstat, base);
    q.Abar = rebase(q.Abar, base);
    q.BbarT = rebase(q.BbarT, base);
    q.partB = rebase(q.partB, base);
    q.planesA = rebase(q.planesA, base);
    q.planesB = rebase(q.planesB, base);
    q.cres = rebase(q.cres, base);
    batch_block_counts(q.m, q.n, q.k, q.kp, fast, q.nblocks);
    for (int w = 0; w < kBatchKernels; ++w) {
      q.first_block[w] = running[w];
      running[w] += q.nblocks[w];
    }
    order.push_back(j);
    ++j;
  }
  for (int w = 0; w < kBatchKernels; ++w) plan->totals[w] = running[w];
  // Tile widths.  The setting (ozk2_set_tile_n) fixes one for every product of the plan.
  // Otherwise each problem's residue products take the rule of single calls (tile_for):
  // narrow or ragged problems run in 128-wide tiles and the rest in 256-wide ones, in
  // two grouped launches (wide first), which spends less tensor work on padding than one
  // width for the whole batch.  The bound products (1-2% of a plan) run in one launch
  // with the rule applied to the batch's total padded work (sum of m k ceil(n / t) t).
  const int tset = g_tile_n.load();
  {
    int64_t w256 = 0, w128 = 0;
    for (const BatchProblem& q : probs) {
      w256 += int64_t(q.m) * q.k * padded(q.n, 256) / 64;
      w128 += int64_t(q.m) * q.k * padded(q.n, 128) / 64;
    }
    plan->bound_tile = tset ? tset : tile_rule(w256, w128);
  }
  std::vector<int> narrow(probs.size());  // 1: the problem's residue products use 128-wide tiles
  for (size_t i = 0; i < probs.size(); ++i)
    narrow[i] = (tset ? tset : tile_rule(padded(probs[i].n, 256), padded(probs[i].n, 128))) == 128 ? 1 : 0;
  // grouped by tile width, longest reductions first within a group
  std::stable_sort(order.begin(), order.end(), [&probs, &narrow](int a, int b) {
    return narrow[a] != narrow[b] ? narrow[a] < narrow[b] : probs[a].k > probs[b].k;
  });
  std::vector<GemmProblem> gres(probs.size()), gbound(fast ? 0 : probs.size());
  const int64_t split_kmax = g_split_kmax.load();
  int64_t ubound = 0;
  for (size_t r = 0; r < order.size(); ++r) {
    const BatchProblem& q = probs[size_t(order[r])];
    const int grp = narrow[size_t(order[r])];
    const int tile = grp ? 128 : 256;
    GemmProblem& g = gres[r];
    std::memset(&g, 0, sizeof(g));
    if (!encode_gemm_problem(&g, q.planesA, q.planesB, q.ldp, tab->mt.num_planes, q.m, q.n, q.k, tile)) {
      destroy_plan(plan);
      return OZK2_ERR_INTERNAL;
    }
    // the products of one problem are addressed like those of a single call, but the
    // planes of the B operand have n rows: the map was encoded with the packed strides
    g.unit_start = plan->res_units[grp];  // units are numbered within each grouped launch
    g.split = q.k <= split_kmax ? 1 : 0;
    g.cres = q.cres;
    g.ldr = q.ldr;
    g.res_stride = int64_t(q.m) * q.ldr;
    plan->res_units[grp] += fp8_gemm_units(kModeResidue, q.m, q.n, N, tile);
    plan->res_cnt[grp] += 1;
    if (!fast) {
      GemmProblem& b = gbound[r];
      std::memset(&b, 0, sizeof(b));
      if (!encode_gemm_problem(&b, q.Abar, q.BbarT, q.kp, 1, q.m, q.n, q.k, plan->bound_tile)) {
        destroy_plan(plan);
        return OZK2_ERR_INTERNAL;
      }
      b.unit_start = ubound;
      b.factor = bound_factor_f32(q.k);
      b.R = q.R;
      b.S = q.S;
      ubound += fp8_gemm_units(kModeBound, q.m, q.n, N, plan->bound_tile);
    }
  }
  plan->units_bound = ubound;
  plan->tile_n = plan->res_cnt[0] > 0 && plan->res_cnt[1] > 0 ? 0 : (plan->res_cnt[1] > 0 ? 128 : 256);
  if (plan->cnt > 0) {
    if (plan->res_units[0] > 0x7FFFFFFFll || plan->res_units[1] > 0x7FFFFFFFll) {
      destroy_plan(plan);
      return OZK2_ERR_UNSUPPORTED;
    }
    // one pinned staging copy of everything the device reads: problems, then the maps
    const size_t nb = (L.gres - L.probs) + sizeof(GemmProblem) * probs.size();
    if (take_fault(kFaultAlloc) || cudaMallocHost(reinterpret_cast<void**>(&plan->host), nb) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->uploaded, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      destroy_plan(plan);
      return OZK2_ERR_ALLOC;
    }
    if (cudaStreamCreateWithFlags(&plan->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&plan->join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      destroy_plan(plan);
      return OZK2_ERR_CUDA;
    }
    plan->host_bytes = nb;
    std::memset(plan->host, 0, nb);
    std::memcpy(plan->host, probs.data(), sizeof(BatchProblem) * probs.size());
    if (!fast) std::memcpy(plan->host + (L.gbound - L.probs), gbound.data(), sizeof(GemmProblem) * gbound.size());
    std::memcpy(plan->host + (L.gres - L.probs), gres.data(), sizeof(GemmProblem) * gres.size());
    if (cudaMemcpyAsync(base + L.probs, plan->host, nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(plan->uploaded, st) != cudaSuccess) {
      destroy_plan(plan);
      return OZK2_ERR_CUDA;
    }
  }
  *out = plan;
  return OZK2_OK;
}

ozk2_status execute_plan(ozk2_batch_plan plan, cudaStream_t st) {
  t_launches = 0;
  if (!plan) return OZK2_ERR_INVALID_VALUE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->dev) return OZK2_ERR_INVALID_VALUE;
  for (const ZeroK& z : plan->zero_k)
    OZK2_TRY(cudaMemset2DAsync(z.C, size_t(z.ldc) * 8, 0, size_t(z.n) * 8, size_t(z.m), st));
  if (plan->cnt == 0) return OZK2_OK;
  const BatchLayout& L = plan->L;
  const Tables* tab = static_cast<const Tables*>(plan->tab);
  uint8_t* ws = plan->ws;
  const BatchProblem* probs = reinterpret_cast<const BatchProblem*>(ws + L.probs);
  uint32_t* flags = reinterpret_cast<uint32_t*>(ws + L.flags);
  OZK2_TRY(cudaMemsetAsync(ws + L.flags, 0, 256, st));
  OZK2_TRY(cudaMemsetAsync(ws + L.zero_begin, 0, L.zero_end - L.zero_begin, st));
  // A's and B's conversions are independent until the bound product and again until the
  // residue products: B's run on the plan's second stream, forked from and joined back to
  // `st` by events (a CUDA graph captured from `st` keeps the same dependencies), so each
  // grouped launch's tail overlaps the other operand's work
  auto fork = [&]() -> cudaError_t {
    cudaError_t e = cudaEventRecord(plan->fork, st);
    return e != cudaSuccess ? e : cudaStreamWaitEvent(plan->side, plan->fork, 0);
  };
  auto join = [&]() -> cudaError_t {
    cudaError_t e = cudaEventRecord(plan->join, plan->side);
    return e != cudaSuccess ? e : cudaStreamWaitEvent(st, plan->join, 0);
  };
  OZK2_TRY(fork());
  OZK2_TRY(launch_scale_batch(probs, plan->cnt, plan->totals, plan->fast, flags, st, plan->side));
  OZK2_TRY(join());
  t_launches += plan->fast ? 4 : 3;
  GemmArgs g{};
  g.num_sms = plan->num_sms;
  g.flags = flags;
  g.tile_n = plan->bound_tile;
  if (!plan->fast) {
    g.mode = kModeBound;
    if (!launch_controls(g)) return OZK2_ERR_CUDA;
    OZK2_TRY(launch_fp8_gemm_grouped(g, reinterpret_cast<const GemmProblem*>(ws + L.gbound), plan->cnt,
                                     plan->units_bound, st));
    t_launches += 1;
  }
  OZK2_TRY(launch_exponents_batch(probs, plan->cnt, plan->totals[kBkExponents], tab->pprime, delta_f32(), st));
  OZK2_TRY(fork());
  OZK2_TRY(launch_residues_batch(probs, plan->cnt, plan->totals[kBkResidRows], plan->totals[kBkResidCols], tab->mt,
                                 flags, st, plan->side));
  OZK2_TRY(join());
  g.mode = kModeResidue;
  g.mt = &tab->mt;
  const GemmProblem* gres = reinterpret_cast<const GemmProblem*>(ws + L.gres);
  for (int grp = 0, first = 0; grp < 2; first += plan->res_cnt[grp], ++grp) {
    if (plan->res_cnt[grp] == 0) continue;
    g.tile_n = grp ? 128 : 256;
    if (!launch_controls(g)) return OZK2_ERR_CUDA;
    OZK2_TRY(launch_fp8_gemm_grouped(g, gres + first, plan->res_cnt[grp], plan->res_units[grp], st));
    t_launches += 1;
  }
  OZK2_TRY(launch_crt_batch(probs, plan->cnt, plan->totals[kBkCrt], tab->ct, st));
  t_launches += 4;
  return OZK2_OK;
}

}  // namespace

bool take_fault(int kind) {
  std::lock_guard<std::mutex> lk(g_fault_mutex);
  read_fault_env();
  if (kind == kFaultNone || g_fault != kind) return false;
  g_fault = kFaultNone;
  return true;
}

unsigned long long wait_limit_ns() {
  const unsigned long long v = g_wait_ns.load();
  return v ? v : 4000000000ull;
}

int validate_dgemm(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                   const double* C, int64_t ldc, int N) {
  return validate(OZK2_OP_N, OZK2_OP_N, m, n, k, A, lda, B, ldb, C, ldc, N);
}

int dgemm_library_ws(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double* C, int64_t ldc, int N, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!ws) return OZK2_ERR_INTERNAL;
  return dgemm_general(OZK2_OP_N, OZK2_OP_N, m, n, k, A, lda, B, ldb, C, ldc, N, OZK2_MODE_ACCURATE, 0, 0, ws,
                       ws_bytes, st, true);
}

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
  return ozk2_dgemm_host_ex(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode, 0u, workspace,
                            workspace_bytes, stream);
}

ozk2_status ozk2_dgemm_host_ex(ozk2_op transa, ozk2_op transb, int64_t m, int64_t n, int64_t k, const double* A,
                               int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int num_moduli,
                               ozk2_mode mode, unsigned flags, void* workspace, size_t workspace_bytes,
                               ozk2_stream_t stream) {
  t_launches = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!valid_mode(mode) || (flags & ~unsigned(OZK2_HOST_INPUTS_READY))) return OZK2_ERR_INVALID_VALUE;
  ozk2_status s = validate(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli);
  if (s != OZK2_OK) return s;
  if (m == 0 || n == 0) return OZK2_OK;
  if (k == 0) {  // C = 0 once earlier work on the stream (which may target C) is done
    if (cudaStreamSynchronize(st) != cudaSuccess) return OZK2_ERR_CUDA;
    for (int64_t i = 0; i < m; ++i) std::memset(C + i * ldc, 0, size_t(n) * 8);
    return OZK2_OK;
  }
  return run_host(transa, transb, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode == OZK2_MODE_FAST, flags,
                  workspace, workspace_bytes, st);
}

size_t ozk2_workspace_size_host(int64_t m, int64_t n, int64_t k, int num_moduli, ozk2_mode mode) {
  if (check_sizes(m, n, k, num_moduli) != OZK2_OK || !valid_mode(mode)) return 0;
  return host_workspace_bytes(m, n, k, num_moduli, mode == OZK2_MODE_FAST);
}

size_t ozk2_workspace_size_batched(int count, const int64_t* m, const int64_t* n, const int64_t* k, int num_moduli,
                                   ozk2_mode mode) {
  if (count < 0 || !valid_mode(mode) || num_moduli < 1 || num_moduli > kMaxModuli) return 0;
  if (count > 0 && (!m || !n || !k)) return 0;
  for (int i = 0; i < count; ++i)
    if (check_sizes(m[i], n[i], k[i], num_moduli) != OZK2_OK) return 0;
  return batch_layout(count, m, n, k, num_moduli, mode == OZK2_MODE_FAST, nullptr).total;
}

ozk2_status ozk2_batch_plan_create(ozk2_batch_plan* plan, int count, const int64_t* m, const int64_t* n,
                                   const int64_t* k, const double* const* A, const int64_t* lda,
                                   const double* const* B, const int64_t* ldb, double* const* C,
                                   const int64_t* ldc, int num_moduli, ozk2_mode mode, void* workspace,
                                   size_t workspace_bytes, ozk2_stream_t stream) {
  return create_plan(plan, count, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode, workspace, workspace_bytes,
                     false, reinterpret_cast<cudaStream_t>(stream));
}

ozk2_status ozk2_batch_plan_execute(ozk2_batch_plan plan, ozk2_stream_t stream) {
  return execute_plan(plan, reinterpret_cast<cudaStream_t>(stream));
}

void* ozk2_batch_plan_workspace(ozk2_batch_plan plan) { return plan ? plan->ws : nullptr; }

void ozk2_batch_plan_destroy(ozk2_batch_plan plan) { destroy_plan(plan); }

ozk2_status ozk2_dgemm_batched(int count, const int64_t* m, const int64_t* n, const int64_t* k,
                               const double* const* A, const int64_t* lda, const double* const* B,
                               const int64_t* ldb, double* const* C, const int64_t* ldc, int num_moduli,
                               ozk2_mode mode, void* workspace, size_t workspace_bytes, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = validate_batch(count, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode);
  if (s != OZK2_OK || count == 0) return s;
  ozk2_batch_plan plan = nullptr;
  s = create_plan(&plan, count, m, n, k, A, lda, B, ldb, C, ldc, num_moduli, mode, workspace,
                              workspace_bytes, true, st);
  if (s != OZK2_OK) return s;
  s = execute_plan(plan, st);
  destroy_plan(plan);  // waits for the descriptor upload only
  return s;
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
  if (flags & kFlagDebug) return OZK2_ERR_INTERNAL;
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

int ozk2_debug_timeline(float* ms, int max) {
  std::lock_guard<std::mutex> lk(g_timing_mutex);
  if (!g_timing.have || !ms || max < 6) return -1;
  if (cudaEventSynchronize(g_timing.ev[6]) != cudaSuccess) return -1;
  int w = 0;
  for (int i = 1; i <= 6 && w < max; ++i) cudaEventElapsedTime(&ms[w++], g_timing.ev[0], g_timing.ev[i]);
  return w;
}

int ozk2_last_launch_count(void) { return t_launches; }

size_t ozk2_workspace_size_backward(int64_t m, int64_t n, int64_t k, int num_moduli) {
  if (check_sizes(m, n, k, num_moduli) != OZK2_OK) return 0;
  return make_bw_layout(m, n, k, num_moduli).total;
}

ozk2_status ozk2_dgemm_backward(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                                int64_t ldb, const double* dC, int64_t lddc, double* dA, int64_t ldda, double* dB,
                                int64_t lddb, int num_moduli, const void* forward_workspace,
                                size_t forward_workspace_bytes, void* workspace, size_t workspace_bytes,
                                ozk2_stream_t stream) {
  t_launches = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = check_sizes(m, n, k, num_moduli);
  if (s != OZK2_OK) return s;
  if (lda < std::max<int64_t>(1, k) || ldb < std::max<int64_t>(1, n) || lddc < std::max<int64_t>(1, n) ||
      (dA && ldda < std::max<int64_t>(1, k)) || (dB && lddb < std::max<int64_t>(1, n)))
    return OZK2_ERR_INVALID_VALUE;
  // empty shapes: dA (m x k) and dB (k x n) are zero where their reduction is empty
  if (m == 0 || n == 0 || k == 0) {
    if (dA && m > 0 && k > 0) OZK2_TRY(cudaMemset2DAsync(dA, size_t(ldda) * 8, 0, size_t(k) * 8, size_t(m), st));
    if (dB && k > 0 && n > 0) OZK2_TRY(cudaMemset2DAsync(dB, size_t(lddb) * 8, 0, size_t(n) * 8, size_t(k), st));
    return OZK2_OK;
  }
  if (!A || !B || !dC || (!dA && !dB)) return OZK2_ERR_INVALID_VALUE;
  return run_backward(m, n, k, A, lda, B, ldb, dC, lddc, dA, ldda, dB, lddb, num_moduli, forward_workspace,
                      forward_workspace_bytes, workspace, workspace_bytes, st);
}

ozk2_status ozk2_debug_backward_exponents(int64_t m, int64_t n, int64_t k, int num_moduli, const void* workspace,
                                          int32_t* g, int32_t* h, ozk2_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ozk2_status s = check_sizes(m, n, k, num_moduli);
  if (s != OZK2_OK) return s;
  const BwLayout L = make_bw_layout(m, n, k, num_moduli);
  const uint8_t* w = static_cast<const uint8_t*>(workspace);
  if (!w) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OZK2_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    if (g_ws[dev].bytes < L.total) return OZK2_ERR_INVALID_VALUE;
    w = static_cast<const uint8_t*>(g_ws[dev].ptr);
  }
  if (g) OZK2_TRY(cudaMemcpyAsync(g, w + L.g, 4 * size_t(m), cudaMemcpyDeviceToDevice, st));
  if (h) OZK2_TRY(cudaMemcpyAsync(h, w + L.h, 4 * size_t(n), cudaMemcpyDeviceToDevice, st));
  return OZK2_OK;
}

uint64_t ozk2_set_wait_limit(uint64_t ns) { return static_cast<uint64_t>(g_wait_ns.exchange(ns)); }

int ozk2_set_tile_n(int tile_n) {
  if (tile_n != 0 && tile_n != 128 && tile_n != 256) return -1;
  return g_tile_n.exchange(tile_n);
}

int ozk2_batch_plan_tile_n(ozk2_batch_plan plan) { return plan ? plan->tile_n : -1; }

int64_t ozk2_set_square_split(int64_t kmax) { return kmax < 0 ? g_split_kmax.load() : g_split_kmax.exchange(kmax); }

int ozk2_debug_inject_fault(int kind) {
  std::lock_guard<std::mutex> lk(g_fault_mutex);
  read_fault_env();
  const int prev = g_fault;
  if (kind > kFaultStall) return -1;
  if (kind >= 0) g_fault = kind;
  return prev;
}

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
  g.tile_n = tile_for(n);
  if (!launch_controls(g)) return OZK2_ERR_CUDA;
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
  return phase_residues(c, operand_a(OZK2_OP_N, A, lda), operand_b(OZK2_OP_N, B, ldb), e, f, planesA, planesB,
                        c.L.kp);  // the caller's planes are packed (pitch kp)
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
