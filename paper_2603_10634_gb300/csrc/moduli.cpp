// Host-side constants of the method: the hybrid moduli (Sec. III-D), the per-modulus
// tables of the residue and epilogue kernels, the CRT weights q_l P / p_l mod P
// (Sec. II, Eq. CRT_finalreduction) as 32-bit limbs, and the FP32 constants P' and
// delta of the exponent rule (Sec. III-E).  Arbitrary-precision integers are a
// little-endian vector of 32-bit limbs.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace ozk2 {
namespace {

using Big = std::vector<uint32_t>;

int gcd_int(int a, int b) {
  while (b) {
    const int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

void trim(Big& x) {
  while (!x.empty() && x.back() == 0) x.pop_back();
}

Big mul_small(const Big& x, uint32_t s) {
  Big r(x.size() + 1, 0);
  uint64_t carry = 0;
  for (size_t i = 0; i < x.size(); ++i) {
    const uint64_t v = static_cast<uint64_t>(x[i]) * s + carry;
    r[i] = static_cast<uint32_t>(v);
    carry = v >> 32;
  }
  r[x.size()] = static_cast<uint32_t>(carry);
  trim(r);
  return r;
}

// quotient of x / s and the remainder
Big div_small(const Big& x, uint32_t s, uint32_t* rem) {
  Big q(x.size(), 0);
  uint64_t r = 0;
  for (size_t i = x.size(); i-- > 0;) {
    const uint64_t cur = (r << 32) | x[i];
    q[i] = static_cast<uint32_t>(cur / s);
    r = cur % s;
  }
  trim(q);
  if (rem) *rem = static_cast<uint32_t>(r);
  return q;
}

int bit_length(const Big& x) {
  if (x.empty()) return 0;
  const uint32_t top = x.back();
  int b = 0;
  while ((top >> b) != 0 && b < 32) ++b;
  return 32 * static_cast<int>(x.size() - 1) + b;
}

Big sub_one(Big x) {
  for (size_t i = 0; i < x.size(); ++i) {
    if (x[i] != 0) {
      --x[i];
      break;
    }
    x[i] = 0xFFFFFFFFu;
  }
  trim(x);
  return x;
}

// value of x as a double (relative error about 2^-53), with x = m 2^e split off to
// avoid overflow: returns m in [1, 2) scaled and sets e.
double top_as_double(const Big& x, int* e2) {
  const int bl = bit_length(x);
  // the top 64 bits, aligned
  uint64_t top = 0;
  for (int b = bl - 1, taken = 0; b >= 0 && taken < 64; --b, ++taken) {
    const uint32_t bit = (x[b >> 5] >> (b & 31)) & 1u;
    top = (top << 1) | bit;
  }
  const int taken = bl < 64 ? bl : 64;
  *e2 = bl - taken;
  return static_cast<double>(top);
}

int modinv(int a, int p) {
  // extended Euclid; a and p coprime
  long long t = 0, nt = 1, r = p, nr = a % p;
  while (nr) {
    const long long qq = r / nr;
    long long tmp = t - qq * nt;
    t = nt;
    nt = tmp;
    tmp = r - qq * nr;
    r = nr;
    nr = tmp;
  }
  if (t < 0) t += p;
  return static_cast<int>(t);
}

float round_down_f32(double x) {
  float f = static_cast<float>(x);
  if (static_cast<double>(f) > x) f = std::nextafterf(f, -INFINITY);
  return f;
}
float round_up_f32(double x) {
  float f = static_cast<float>(x);
  if (static_cast<double>(f) < x) f = std::nextafterf(f, INFINITY);
  return f;
}

std::once_flag g_moduli_once;
int g_moduli[kMaxModuli];

void build_moduli_list() {
  int count = 0;
  // pairwise-coprime squares, descending from 33^2; the first six lead the list
  for (int s = 33; s >= 2 && count < kNumSquares; --s) {
    bool ok = true;
    for (int i = 0; i < count; ++i) ok = ok && gcd_int(s * s, g_moduli[i]) == 1;
    if (ok) g_moduli[count++] = s * s;
  }
  // then pairwise-coprime integers, descending from 513
  for (int c = 513; c >= 2 && count < kMaxModuli; --c) {
    bool ok = true;
    for (int i = 0; i < count; ++i) ok = ok && gcd_int(c, g_moduli[i]) == 1;
    if (ok) g_moduli[count++] = c;
  }
}

Big product_of(int N) {
  Big P{1u};
  for (int i = 0; i < N; ++i) P = mul_small(P, static_cast<uint32_t>(g_moduli[i]));
  return P;
}

}  // namespace

int hybrid_moduli(int N, int* out) {
  if (N < 1 || N > kMaxModuli) return -1;
  std::call_once(g_moduli_once, build_moduli_list);
  for (int i = 0; i < N; ++i) out[i] = g_moduli[i];
  return N;
}

bool build_mod_table(int N, ModTable* mt) {
  int mods[kMaxModuli];
  if (hybrid_moduli(N, mods) != N) return false;
  std::memset(mt, 0, sizeof(*mt));
  mt->N = N;
  mt->num_planes = (N <= kNumSquares) ? 2 * N : 3 * N - kNumSquares;
  for (int l = 0; l < N; ++l) {
    const int p = mods[l];
    mt->p[l] = p;
    mt->half[l] = p / 2;
    mt->s[l] = (l < kNumSquares) ? static_cast<int>(std::lround(std::sqrt(static_cast<double>(p)))) : 16;
    mt->plane0[l] = (l < kNumSquares) ? 2 * l : 2 * kNumSquares + 3 * (l - kNumSquares);
    mt->inv_p[l] = static_cast<float>(1.0 / p);
    mt->inv_s[l] = static_cast<float>(1.0 / mt->s[l]);
    const int h = p / 2;
    auto sym = [p, h](int v) { return v > p - 1 - h ? v - p : v; };  // [-h, p-1-h]
    int v = 1 % p;
    for (int t = 0; t < kPow2Table; ++t) {
      mt->pow2[l][t] = static_cast<int16_t>(sym(v));
      if (t % 11 == 0 && t / 11 < 5) mt->w11[l][t / 11] = static_cast<float>(sym(v));
      v = (2 * v) % p;
    }
    auto pair = [](float x) { return make_float2(x, x); };
    mt->neg_p2[l] = pair(-static_cast<float>(p));
    mt->inv_p2[l] = pair(mt->inv_p[l]);
    mt->neg_s2[l] = pair(-static_cast<float>(mt->s[l]));
    mt->inv_s2[l] = pair(mt->inv_s[l]);
    for (int j = 0; j < 5; ++j) mt->w2[l][j] = pair(mt->w11[l][j]);
  }
  return true;
}

bool build_crt_table(int N, CrtTable* ct) {
  int mods[kMaxModuli];
  if (hybrid_moduli(N, mods) != N) return false;
  std::memset(ct, 0, sizeof(*ct));
  const Big P = product_of(N);
  const int bl = bit_length(P);
  const int limbs = (bl + 1 + 31) / 32;  // signed values |x| < P/2 ... < 2^(32 L - 1)
  if (limbs > kMaxLimbs) return false;
  ct->N = N;
  ct->limbs = limbs;
  int eP;
  const double Ptop = top_as_double(P, &eP);
  for (int l = 0; l < N; ++l) {
    const int p = mods[l];
    ct->p[l] = p;
    uint32_t rem = 0;
    const Big Pl = div_small(P, static_cast<uint32_t>(p), nullptr);
    div_small(Pl, static_cast<uint32_t>(p), &rem);
    const int q = modinv(static_cast<int>(rem), p);
    const Big w = mul_small(Pl, static_cast<uint32_t>(q));  // < P, already reduced
    // balanced limbs: a limb of 2^31 or more becomes limb - 2^32 and carries 1 upwards
    int64_t carry = 0;
    for (int t = 0; t < limbs; ++t) {
      int64_t u = (t < static_cast<int>(w.size()) ? static_cast<int64_t>(w[t]) : 0) + carry;
      carry = u >= (int64_t(1) << 31) ? 1 : 0;
      u -= carry << 32;
      ct->wb[l][t] = static_cast<int32_t>(u);
    }
    if (carry != 0) return false;  // w_l < P < 2^(32 L - 1): the top limb never carries out
    int ew;
    const double wtop = w.empty() ? 0.0 : top_as_double(w, &ew);
    ct->frac16[l] = w.empty() ? 0 : static_cast<int32_t>(std::llround(std::ldexp(wtop / Ptop, ew - eP + 16)));
  }
  for (size_t t = 0; t < P.size(); ++t) ct->P[t] = P[t];
  uint32_t dummy;
  const Big half = div_small(P, 2u, &dummy);
  for (size_t t = 0; t < half.size(); ++t) ct->halfP[t] = half[t];
  return true;
}

float p_prime_f32(int N) {
  int mods[kMaxModuli];
  if (hybrid_moduli(N, mods) != N) return NAN;
  const Big Pm1 = sub_one(product_of(N));
  int e2;
  const double top = top_as_double(Pm1, &e2);
  const double lg = std::log2(top) + e2;
  return round_down_f32((lg - 1.0) / 2.0);
}

float reuse_budget_f32(int N) {
  int mods[kMaxModuli];
  if (hybrid_moduli(N, mods) != N) return NAN;
  const Big Pm1 = sub_one(product_of(N));
  int e2;
  const double top = top_as_double(Pm1, &e2);
  const double lg = std::log2(top) + e2;
  return round_down_f32(lg - 1.0);
}

float delta_f32() { return round_down_f32(-1.0 / (2.0 - std::ldexp(1.0, -21))); }

float bound_factor_f32(int64_t k) { return round_up_f32(1.0 + std::ldexp(static_cast<double>(k), -24)); }

}  // namespace ozk2
