// Exact fixed-point sums of fp64 values, rounded once to fp64: the dot products
// of the cluster form.
//
// A group of terms is brought to a common scale E (the largest exponent field
// among them): term v = (-1)^s m 2^(e - 1075) becomes the integer
// X = (-1)^s floor(m 2^(e - E + kGuard)), |X| < 2^63, i.e. v in units of
// 2^(E - 1075 - kGuard) truncated toward zero (an error below one unit, 2^-kGuard
// of the last mantissa bit of the group's largest term).  Integer sums are exact
// and do not depend on order; a sum at scale E moves to a larger scale E' by an
// arithmetic right shift of E' - E bits (again below one unit).  The final integer
// is rounded once to the nearest fp64 value, ties to even, with subnormal results
// and overflow to infinity as IEEE 754 defines them.  A non-finite term makes the
// sum NaN.
//
// GB300's fp64 pipe issues one warp instruction per ~64 clocks per SM
// sub-partition, so a tree of fp64 adds in one warp costs that per level; these
// integer steps run on the integer pipes and the warp-wide sums are single
// redux.sync instructions.  The functions compile for the host too (tested there
// against exact rational arithmetic).
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define CG_EXACT_HD __host__ __device__ __forceinline__
#else
#define CG_EXACT_HD inline
#endif

namespace cg_exact {

constexpr int kGuard = 10;  // fraction bits kept below the largest term's last mantissa bit

typedef __int128 i128;
typedef unsigned __int128 u128;

CG_EXACT_HD unsigned long long bits_of(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  std::memcpy(&b, &v, sizeof b);
  return b;
#endif
}

CG_EXACT_HD double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
#endif
}

CG_EXACT_HD int clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// A finite fp64 value as (-1)^neg m 2^(e - 1075) with m < 2^53 and e >= 1
// (subnormals and zero take e = 1, m without the hidden bit); bad for Inf / NaN.
struct Parts {
  unsigned long long m;
  int e;
  bool neg, bad;
};

CG_EXACT_HD Parts parts(double v) {
  const unsigned long long b = bits_of(v);
  const int f = (int)((b >> 52) & 0x7FF);
  Parts p;
  p.neg = (b >> 63) != 0;
  p.bad = f == 0x7FF;
  p.m = p.bad ? 0ull : (b & ((1ull << 52) - 1)) | (f ? (1ull << 52) : 0ull);
  p.e = (f == 0 || p.bad) ? 1 : f;
  return p;
}

// The term in units of 2^(E - 1075 - kGuard), truncated toward zero (E >= p.e).
CG_EXACT_HD long long to_fixed(const Parts& p, int E) {
  const int d = E - p.e;
  unsigned long long x;
  if (d <= kGuard) x = p.m << (kGuard - d);
  else if (d - kGuard >= 64) x = 0;
  else x = p.m >> (d - kGuard);
  return p.neg ? -(long long)x : (long long)x;
}

// x 2^-s, rounded toward minus infinity (the move to a larger scale).
CG_EXACT_HD i128 shift_down(i128 x, int s) { return s >= 127 ? (x < 0 ? (i128)-1 : (i128)0) : (x >> s); }

CG_EXACT_HD double ll_to_double(long long x) {
#ifdef __CUDA_ARCH__
  return __ll2double_rn(x);
#else
  return (double)x;  // round to nearest even: the default rounding mode
#endif
}

// T 2^(E - 1075 - kGuard) rounded to the nearest fp64 value, ties to even, for
// |T| < 2^120 and scales where no result can be subnormal or infinite (the
// integer then passes through the hardware's correctly rounded int64 -> fp64
// conversion, times an exact power of two); false elsewhere.  An integer of more
// than 63 bits is first shifted right with the lost bits ORed into its last bit
// (a sticky bit: with 10 or more bits beyond the 53 kept, rounding is unchanged).
CG_EXACT_HD bool to_fp64_fast(i128 T, int E, double* out) {
  if (E < 63 + kGuard || E > 1900) return false;
  const bool neg = T < 0;
  u128 M = neg ? (u128)0 - (u128)T : (u128)T;
  int s = 0;
  const unsigned long long hi = (unsigned long long)(M >> 63);
  if (hi) {
    s = 64 - clz64(hi);  // M >> s < 2^63
    const bool sticky = (M & (((u128)1 << s) - 1)) != 0;
    M = (M >> s) | (u128)(sticky ? 1 : 0);
  }
  const long long m = (long long)(unsigned long long)M;
  const double d = ll_to_double(neg ? -m : m);
  *out = d * double_of((unsigned long long)(E - 1075 - kGuard + s + 1023) << 52);
  return true;
}

CG_EXACT_HD double to_fp64_int(i128 T, int E, bool bad);

// T 2^(E - 1075 - kGuard) rounded to the nearest fp64 value, ties to even; NaN if bad.
CG_EXACT_HD double to_fp64(i128 T, int E, bool bad) {
  double f;
  if (!bad && T != 0 && to_fp64_fast(T, E, &f)) return f;
  return to_fp64_int(T, E, bad);
}

// The same rounding with integer instructions only (the result's bits built from
// the integer), for code whose fp64 pipe is the bottleneck.
CG_EXACT_HD double to_fp64_int(i128 T, int E, bool bad) {
  if (bad) return double_of(0x7FF8000000000000ull);
  if (T == 0) return 0.0;
  const bool neg = T < 0;
  const u128 M = neg ? (u128)0 - (u128)T : (u128)T;
  const unsigned long long hi = (unsigned long long)(M >> 64), lo = (unsigned long long)M;
  const int nb = hi ? 128 - clz64(hi) : 64 - clz64(lo);  // bit length of M
  // as a normal number: 1.f 2^(nb - 1 + E - 1075 - kGuard), biased exponent eb
  int eb = nb + E - kGuard - 53;
  // right shift of M onto the result's integer mantissa: 53 bits when normal,
  // units of 2^-1074 when subnormal
  const int sh = eb >= 1 ? nb - 53 : 1 + kGuard - E;
  unsigned long long m;
  if (sh <= 0) {
    m = (unsigned long long)(M << (-sh));  // exact
  } else if (sh >= 128) {
    m = 0;  // M < 2^127 <= half a unit
  } else {
    m = (unsigned long long)(M >> sh);
    const u128 rem = M - ((u128)m << sh), half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
  }
  unsigned long long b;
  if (eb >= 1) {
    if (m == (1ull << 53)) {  // rounded up to the next binade
      m >>= 1;
      ++eb;
    }
    b = eb >= 2047 ? 0x7FF0000000000000ull : ((unsigned long long)eb << 52) | (m & ((1ull << 52) - 1));
  } else {
    b = m;  // subnormal; m = 2^52 is the smallest normal number
  }
  if (neg) b |= 1ull << 63;
  return double_of(b);
}

// An integer sum of |value| < 2^69 packed with its scale and NaN flag into 16 bytes:
// lo = the low 64 bits, hi = bits 64.. (40-bit two's complement) | bad << 40 | E << 41.
CG_EXACT_HD void pack(i128 S, int E, bool bad, unsigned long long* lo, unsigned long long* hi) {
  *lo = (unsigned long long)S;
  *hi = ((unsigned long long)(S >> 64) & ((1ull << 40) - 1)) | ((unsigned long long)bad << 40) |
        ((unsigned long long)E << 41);
}

CG_EXACT_HD i128 unpack(unsigned long long lo, unsigned long long hi, int* E, bool* bad) {
  *E = (int)(hi >> 41);
  *bad = ((hi >> 40) & 1ull) != 0;
  const long long h = (long long)(hi << 24) >> 24;  // sign-extend the 40-bit high part
  return (i128)(((u128)(i128)h << 64) | (u128)lo);
}

}  // namespace cg_exact
