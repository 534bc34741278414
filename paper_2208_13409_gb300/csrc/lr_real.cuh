// lr_real.cuh -- arithmetic types of the step kernels.
//
// GB300 executes FP64 at 1/64 of its FP32 rate (304 DFMA against 19456 FFMA
// lanes per clock), so besides native double the kernels can run on a
// double-float type: a value is the unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi)/2, about 48 significand bits, carried entirely by the
// FP32 pipe.  The error-free transformations are the classical ones:
//   two-sum (Knuth, TAOCP vol. 2, 4.2.2): s = a+b, e = (a-(s-bb)) + (b-bb);
//   fast two-sum (Dekker 1971) when |a| >= |b|: s = a+b, e = b-(s-a);
//   two-product with a fused multiply-add: p = a*b, e = fma(a, b, -p);
// and the double-length operations built from them follow Dekker 1971 and
// the double-double algorithms of Hida, Li and Bailey (2001), here on floats.
// Every rounding step uses __fadd_rn/__fmul_rn/__fmaf_rn so the compiler
// cannot contract or reorder them.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

struct __align__(8) df64 {
  float hi, lo;
  __host__ __device__ df64() {}
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(float h) : hi(h), lo(0.0f) {}
};

namespace dfops {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df64 add(df64 x, df64 y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  df64 r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df64 neg(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 mul(df64 x, df64 y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df64 r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// x / y: two quotient digits from an approximate reciprocal of y.hi, the
// second removing the remainder of the first (long division in base 2^24):
// about 2^-46, the pair's own precision near 2^-48.
__device__ __forceinline__ df64 div(df64 x, df64 y) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(y.hi));
  float q1 = __fmul_rn(x.hi, r0);
  df64 rem = add(x, neg(mul(y, df64(q1))));
  float q2 = __fmul_rn(rem.hi, r0);
  df64 q;
  fast_two_sum(q1, q2, q.hi, q.lo);
  return q;
}
// sqrt(x): float square root, then one Newton correction in double length:
// s' = s + (x - s^2) / (2 s).
__device__ __forceinline__ df64 sqrt_(df64 x) {
  if (!(x.hi > 0.0f)) return df64(0.0f, 0.0f);
  float s = __fsqrt_rn(x.hi);
  df64 ss = mul(df64(s), df64(s));
  df64 d = add(x, neg(ss));
  float c = __fmul_rn(d.hi, __frcp_rn(__fmul_rn(2.0f, s)));
  df64 r;
  fast_two_sum(s, c, r.hi, r.lo);
  return r;
}

}  // namespace dfops

__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return dfops::add(a, b); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return dfops::add(a, dfops::neg(b)); }
__device__ __forceinline__ df64 operator-(df64 a) { return dfops::neg(a); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return dfops::mul(a, b); }
__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return dfops::div(a, b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { a = a * b; return a; }
// Comparisons of normalised pairs: hi decides unless the his are equal.
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

// ---- uniform helpers over double, float and df64
template <class R> struct RealOps;
// mul/add: rounded operations the compiler may not fuse into a multiply-add
// (used where two kernels must give bit-identical results).
// Predicates and ordering of doubles on the integer units.  A double
// comparison issues on the FP64 pipe, the binding resource of the native
// double kernels (one warp instruction holds it for 16 clocks), while these
// take a few integer operations on the bit pattern.  They have IEEE 754
// semantics exactly: false when an operand is NaN, -0 equal to +0.
namespace dbits {
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
// +inf's pattern; a NaN's magnitude lies above it.
constexpr unsigned long long kInf = 0x7ff0000000000000ULL;
// x > 0: the patterns 1 .. kInf (smallest subnormal .. +inf) shifted down by one.
__device__ __forceinline__ bool pos(double x) { return (unsigned long long)(bits(x) - 1) < kInf; }
// x < 0: the patterns of -smallest subnormal .. -inf, sign bit set, likewise.
__device__ __forceinline__ bool neg(double x) {
  return (unsigned long long)bits(x) - 0x8000000000000001ULL < kInf;
}
__device__ __forceinline__ bool zero(double x) { return (bits(x) << 1) == 0; }
// -x when f, x otherwise, and |x|: the sign bit alone (a negation written
// as such costs an FP64 add).
__device__ __forceinline__ double flip(bool f, double x) {
  return __longlong_as_double(bits(x) ^ ((long long)f << 63));
}
__device__ __forceinline__ double absb(double x) { return __longlong_as_double(bits(x) & 0x7fffffffffffffffLL); }
__device__ __forceinline__ bool finite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool nan_b(long long v) { return ((unsigned long long)v << 1) > (kInf << 1); }
// Sign-magnitude to two's-complement order: negative patterns have their
// magnitude bits flipped, so signed integer order is numeric order (with -0
// just below +0, which lt treats as equal).
__device__ __forceinline__ long long okey(long long v) { return v ^ ((v >> 63) & 0x7fffffffffffffffLL); }
__device__ __forceinline__ bool lt(double a, double b) {
  long long u = bits(a), v = bits(b);
  bool ord = !(nan_b(u) | nan_b(v));
  bool zz = ((u | v) << 1) == 0;
  return ord & !zz & (okey(u) < okey(v));
}
// Exact double of a float that is normal or zero, from its bits (integer
// units; a subnormal float, which the seeds below never produce, reads as 0).
__device__ __forceinline__ double f2d_exact(float f) {
  unsigned b = __float_as_uint(f), e8 = (b >> 23) & 0xffu;
  unsigned hi = e8 ? (b & 0x80000000u) | ((e8 + 896u) << 20) | ((b & 0x7fffffu) >> 3) : (b & 0x80000000u);
  return __hiloint2double((int)hi, (int)(e8 ? b << 29 : 0u));
}
// n / d with three FP64 operations.  The significands of n and d (in [1, 2))
// are split into float pairs hi + lo (24 + about 24 bits); on the float pipe
// a reciprocal seed r of d's (rcp.approx) takes one Newton-Raphson step in
// double-float arithmetic, r (1 + e) with e = 1 - d r from fused
// multiply-adds (about 2^-44), and the significand quotient q0 = n r (1 + e)
// is formed as an unevaluated float pair by Dekker's exact product with a
// fused multiply-add (T. J. Dekker, Numer. Math. 18, 1971).  In FP64: one
// exact addition joins the pair, the exponents are applied on the integer
// units, and one Markstein correction q0 + (n - d q0) r with its residual
// from a fused multiply-add (P. W. Markstein, IBM J. Res. Dev. 34(1), 1990)
// takes the relative error to about 2^-66 before the last rounding: the
// result is the correctly rounded quotient unless n/d lies that close to a
// rounding midpoint (then it is one ulp off).  About seven FP64 operations
// for the division instruction sequence, which still handles d zero,
// subnormal, infinite, NaN or of magnitude >= 2^1020, n subnormal, infinite
// or NaN, and quotients outside the normal range; n = +-0 gives the IEEE
// signed zero.
__device__ __forceinline__ double ddiv(double n, double d) {
  unsigned hn = (unsigned)__double2hiint(n), ln = (unsigned)__double2loint(n);
  unsigned hd = (unsigned)__double2hiint(d), ld = (unsigned)__double2loint(d);
  unsigned en = (hn >> 20) & 0x7ffu, ed = (hd >> 20) & 0x7ffu;
  if (ed - 1u >= 2043u || en - 1u >= 2046u) {
    if (en == 0u && ((hn << 1) | ln) == 0u && ed - 1u < 2043u)
      return __hiloint2double((int)((hn ^ hd) & 0x80000000u), 0);
    return n / d;
  }
  // significands: hi = the top 23 fraction bits (exact), lo = the other 29
  // (rounded to float)
  float nh = __uint_as_float(0x3f800000u | ((hn & 0xfffffu) << 3) | (ln >> 29));
  float nl = __uint2float_rn(ln & 0x1fffffffu) * 0x1p-52f;
  float dh = __uint_as_float(0x3f800000u | ((hd & 0xfffffu) << 3) | (ld >> 29));
  float dl = __uint2float_rn(ld & 0x1fffffffu) * 0x1p-52f;
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(dh));  // in (0.5, 1]
  float e = __fmaf_rn(-dh, r0, 1.0f);
  e = __fmaf_rn(-dl, r0, e);
  float c = __fmul_rn(r0, e);             // 1/(dh + dl) = r0 + c to about 2^-44
  float p = __fmul_rn(nh, r0);
  float pe = __fmaf_rn(nh, r0, -p);       // nh r0 = p + pe exactly
  pe = __fmaf_rn(nh, c, pe);
  pe = __fmaf_rn(nl, r0, pe);
  double q0 = f2d_exact(p) + f2d_exact(pe);  // exact: the pair fits in 53 bits; q0 in (0.25, 2)
  // q = sign q0 2^(en - ed)
  unsigned hq = (unsigned)__double2hiint(q0);
  int fq = (int)((hq >> 20) & 0x7ffu) + (int)en - (int)ed;
  if (fq < 1 || fq > 2046) return n / d;
  hq = ((hn ^ hd) & 0x80000000u) | ((unsigned)fq << 20) | (hq & 0xfffffu);
  double q = __hiloint2double((int)hq, __double2loint(q0));
  // r = sign(d) r0 2^(1023 - ed): r0's exponent field (126 or 127) gives r's
  // as fe - 127 + 2046 - ed, within [2, 2045] for ed in [1, 2043]
  unsigned fb = __float_as_uint(r0);
  unsigned hr = (hd & 0x80000000u) | (((fb >> 23) + 1919u - ed) << 20) | ((fb & 0x7fffffu) >> 3);
  double r = __hiloint2double((int)hr, (int)(fb << 29));
  return fma(fma(-d, q, n), r, q);
}
// sqrt(x) with three FP64 operations, the same way: x = m 4^k with m in
// [1, 4) split into a float pair; on the float pipe a reciprocal-square-root
// seed y of m's high part (rsqrt.approx) gives s = m y, and one Newton step
// s + (m - s s) y/2, residual by a fused multiply-add, leaves sqrt(m) as an
// unevaluated float pair to about 2^-44.  In FP64: one exact addition joins
// the pair, 2^k is applied on the integer units, and one correction
// s + (x - s s) y/2 (residual from a fused multiply-add) takes the error to
// about 2^-66 before the last rounding (correctly rounded but near
// midpoints).  About seven and a half FP64 operations for the square-root
// instruction sequence, which still handles x zero, subnormal, negative,
// infinite, NaN or in the top binade.
__device__ __forceinline__ double dsqrt(double x) {
  unsigned hx = (unsigned)__double2hiint(x), lx = (unsigned)__double2loint(x);
  unsigned ex = hx >> 20;  // the sign bit included: negative x gives ex >= 2048
  if (ex - 1u >= 2045u) return sqrt(x);
  // x = m 2^e, m in [1, 2); e = 2k + p, p in {0, 1}: x = (m 2^p) 4^k
  int e = (int)ex - 1023;
  int p = e & 1, k = (e - p) / 2;
  float mh = __uint_as_float(((127u + (unsigned)p) << 23) | ((hx & 0xfffffu) << 3) | (lx >> 29));
  float ml = __uint2float_rn(lx & 0x1fffffffu) * (p ? 0x1p-51f : 0x1p-52f);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(mh));  // in (0.5, 1]
  float sh = __fmul_rn(mh, yf);
  float t = __fmaf_rn(-sh, sh, mh);        // mh - sh^2, the square exact inside the fma
  float sl = __fmul_rn(__fadd_rn(t, ml), __fmul_rn(0.5f, yf));
  double s = f2d_exact(sh) + f2d_exact(sl);  // exact; sqrt(m) to about 2^-44, in [1, 2)
  // s 2^k: s's exponent field (1023, or 1024 if it rounded up to 2) + k
  unsigned hs = (unsigned)__double2hiint(s);
  hs = (((hs >> 20) + (unsigned)k) << 20) | (hs & 0xfffffu);
  s = __hiloint2double((int)hs, __double2loint(s));
  // h = yf 2^(-k-1) = y/2: exponent field (fe - 127) - k - 1 + 1023, within [510, 1533]
  unsigned fb = __float_as_uint(yf);
  unsigned hh = ((unsigned)((int)(fb >> 23) - 127 - k - 1 + 1023) << 20) | ((fb & 0x7fffffu) >> 3);
  double h = __hiloint2double((int)hh, (int)(fb << 29));
  return fma(fma(-s, s, x), h, s);
}
}  // namespace dbits

template <> struct RealOps<double> {
  __device__ static __forceinline__ double c(float v) { return (double)v; }
  __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static __forceinline__ double abs(double x) { return dbits::absb(x); }
  __device__ static __forceinline__ double flip(bool f, double x) { return dbits::flip(f, x); }
  __device__ static __forceinline__ double sqrt(double x) { return dbits::dsqrt(x); }
  __device__ static __forceinline__ double rcp(double x) { return dbits::ddiv(1.0, x); }
  __device__ static __forceinline__ double div(double a, double b) { return dbits::ddiv(a, b); }
  __device__ static __forceinline__ bool finite(double x) { return dbits::finite(x); }
  __device__ static __forceinline__ bool pos(double x) { return dbits::pos(x); }
  __device__ static __forceinline__ bool neg(double x) { return dbits::neg(x); }
  __device__ static __forceinline__ bool zero(double x) { return dbits::zero(x); }
  __device__ static __forceinline__ bool lt(double a, double b) { return dbits::lt(a, b); }
  __host__ __device__ static __forceinline__ double todouble(double x) { return x; }
};
template <> struct RealOps<float> {
  __device__ static __forceinline__ float c(float v) { return v; }
  __device__ static __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ static __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static __forceinline__ float abs(float x) { return fabsf(x); }
  __device__ static __forceinline__ float flip(bool f, float x) { return f ? -x : x; }
  __device__ static __forceinline__ float sqrt(float x) { return sqrtf(x); }
  // reciprocal and quotient to about two ulps (the bulk mode's accuracy is
  // set by float storage, not by these)
  __device__ static __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  __device__ static __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
  __device__ static __forceinline__ bool finite(float x) { return isfinite(x); }
  __device__ static __forceinline__ bool pos(float x) { return x > 0.0f; }
  __device__ static __forceinline__ bool neg(float x) { return x < 0.0f; }
  __device__ static __forceinline__ bool zero(float x) { return x == 0.0f; }
  __device__ static __forceinline__ bool lt(float a, float b) { return a < b; }
  __host__ __device__ static __forceinline__ double todouble(float x) { return (double)x; }
};
template <> struct RealOps<df64> {
  __device__ static __forceinline__ df64 c(float v) { return df64(v, 0.0f); }
  __device__ static __forceinline__ df64 mul(df64 a, df64 b) { return dfops::mul(a, b); }
  __device__ static __forceinline__ df64 add(df64 a, df64 b) { return dfops::add(a, b); }
  __device__ static __forceinline__ df64 abs(df64 x) { return x.hi < 0.0f ? dfops::neg(x) : x; }
  __device__ static __forceinline__ df64 flip(bool f, df64 x) { return f ? dfops::neg(x) : x; }
  __device__ static __forceinline__ df64 sqrt(df64 x) { return dfops::sqrt_(x); }
  __device__ static __forceinline__ df64 rcp(df64 x) { return dfops::div(df64(1.0f, 0.0f), x); }
  __device__ static __forceinline__ df64 div(df64 a, df64 b) { return dfops::div(a, b); }
  __device__ static __forceinline__ bool finite(df64 x) { return isfinite(x.hi) && isfinite(x.lo); }
  __device__ static __forceinline__ bool pos(df64 x) { return x.hi > 0.0f; }
  __device__ static __forceinline__ bool neg(df64 x) { return x.hi < 0.0f; }
  __device__ static __forceinline__ bool zero(df64 x) { return x.hi == 0.0f; }
  __device__ static __forceinline__ bool lt(df64 a, df64 b) { return a < b; }
  __host__ __device__ static __forceinline__ double todouble(df64 x) { return (double)x.hi + (double)x.lo; }
};

// Conversions from double (host: exact splitting, used for constants and at
// the API boundary).
template <class R> __host__ __device__ inline R from_double(double v);
template <> __host__ __device__ inline double from_double<double>(double v) { return v; }
template <> __host__ __device__ inline float from_double<float>(double v) { return (float)v; }
template <> __host__ __device__ inline df64 from_double<df64>(double v) {
  float h = (float)v;
  float l = (float)(v - (double)h);
  return df64(h, l);
}

template <class R> __device__ __forceinline__ R rmin(R a, R b) { return RealOps<R>::lt(b, a) ? b : a; }
template <class R> __device__ __forceinline__ R rmax(R a, R b) { return RealOps<R>::lt(a, b) ? b : a; }
