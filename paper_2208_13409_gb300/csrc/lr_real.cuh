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
// x / y: three quotient digits from an approximate reciprocal of y.hi, each
// removing the remainder of the previous ones (long division in base 2^24).
__device__ __forceinline__ df64 div(df64 x, df64 y) {
  float r0 = __frcp_rn(y.hi);
  float q1 = __fmul_rn(x.hi, r0);
  df64 rem = add(x, neg(mul(y, df64(q1))));
  float q2 = __fmul_rn(rem.hi, r0);
  rem = add(rem, neg(mul(y, df64(q2))));
  float q3 = __fmul_rn(rem.hi, r0);
  df64 q;
  fast_two_sum(q1, q2, q.hi, q.lo);
  return add(q, df64(q3));
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
// n / d by Newton-Raphson refinement of the quotient with fused
// multiply-add residuals (P. W. Markstein, IBM J. Res. Dev. 34(1), 1990):
// a float reciprocal r of d's significand, scaled to d's exponent, seeds
// q = n r, and each step adds e r to q, with e = n - d q from one fused
// multiply-add.  The seed is within about 2^-22 of 1/d, so two steps leave
// a relative error near 2^-66 before the last rounding: the result is the
// correctly rounded quotient unless n/d lies that close to a rounding
// midpoint (then it is one ulp off).  Five FP64 operations against about
// seven for the division instruction sequence, which still handles d zero,
// subnormal, infinite, NaN or of magnitude >= 2^1020.  Other differences
// from IEEE division: a quotient that overflows, or n infinite, gives NaN
// rather than an infinity, and -0 / d gives +0.
__device__ __forceinline__ double ddiv(double n, double d) {
  unsigned hd = (unsigned)__double2hiint(d), ld = (unsigned)__double2loint(d);
  unsigned ed = (hd >> 20) & 0x7ffu;
  if (ed - 1u >= 2043u) return n / d;
  // |d|'s significand in [1, 2) to float precision (truncated), its reciprocal
  float m = __uint_as_float(0x3f800000u | ((hd & 0xfffffu) << 3) | (ld >> 29));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(m));
  // r = sign(d) rf 2^(1023 - ed): rf's exponent field fe (126 or 127) gives
  // r's as fe - 127 + 2046 - ed, within [2, 2045] for ed in [1, 2043]
  unsigned fb = __float_as_uint(rf);
  unsigned hr = (hd & 0x80000000u) | (((fb >> 23) + 1919u - ed) << 20) | ((fb & 0x7fffffu) >> 3);
  double r = __hiloint2double((int)hr, (int)(fb << 29));
  double q = n * r;
  double e = fma(-d, q, n);
  q = fma(e, r, q);
  e = fma(-d, q, n);
  return fma(e, r, q);
}
// sqrt(x) by the same refinement with a reciprocal-square-root seed: y, a
// float approximation of 1/sqrt(x) (from x's significand, with the
// exponent's parity folded in), gives s = x y and h = y/2; each step adds
// (x - s s) h to s, the residual from one fused multiply-add.  The seed is
// within about 2^-22, one step leaves about 2^-43 and the second about
// 2^-66 before the last rounding (correctly rounded but near midpoints).
// Five FP64 operations against about seven and a half for the square-root
// instruction sequence, which still handles x zero, subnormal, negative,
// infinite, NaN or in the top binade.
__device__ __forceinline__ double dsqrt(double x) {
  unsigned hx = (unsigned)__double2hiint(x), lx = (unsigned)__double2loint(x);
  unsigned ex = hx >> 20;  // the sign bit included: negative x gives ex >= 2048
  if (ex - 1u >= 2045u) return sqrt(x);
  // x = m 2^e, m in [1, 2); e = 2k + p, p in {0, 1}: x = (m 2^p) 4^k
  int e = (int)ex - 1023;
  int p = e & 1, k = (e - p) / 2;
  float mf = __uint_as_float(((127u + (unsigned)p) << 23) | ((hx & 0xfffffu) << 3) | (lx >> 29));
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(mf));  // in (0.5, 1]
  // y = yf 2^-k: exponent field (fe - 127) - k + 1023, within [511, 1534]
  unsigned fb = __float_as_uint(yf);
  unsigned hy = ((unsigned)((int)(fb >> 23) - 127 - k + 1023) << 20) | ((fb & 0x7fffffu) >> 3);
  double y = __hiloint2double((int)hy, (int)(fb << 29));
  double h = __hiloint2double((int)(hy - (1u << 20)), (int)(fb << 29));  // y / 2
  double s = x * y;
  double r = fma(-s, s, x);
  s = fma(r, h, s);
  r = fma(-s, s, x);
  return fma(r, h, s);
}
}  // namespace dbits

template <> struct RealOps<double> {
  __device__ static __forceinline__ double c(float v) { return (double)v; }
  __device__ static __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ static __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static __forceinline__ double abs(double x) { return dbits::absb(x); }
  __device__ static __forceinline__ double flip(bool f, double x) { return dbits::flip(f, x); }
  __device__ static __forceinline__ double sqrt(double x) { return dbits::dsqrt(x); }
  __device__ static __forceinline__ double rcp(double x) { return 1.0 / x; }
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
  __device__ static __forceinline__ float rcp(float x) { return 1.0f / x; }
  __device__ static __forceinline__ float div(float a, float b) { return a / b; }
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
