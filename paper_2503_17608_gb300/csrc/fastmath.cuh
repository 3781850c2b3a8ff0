// Table-driven binary64 logarithm, exponential and sine/cosine of 2 pi u,
// after P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic" (ACM TOMS 15, 1989) and "... of the logarithm
// function ..." (ACM TOMS 16, 1990): a table lookup reduces the argument to a
// few thousandths, where a short polynomial is accurate to the last bit (the
// sine/cosine use the same idea with the angle-addition formulas).
//
// Why: on GB300 an FP64 warp instruction holds its sub-partition's FP64 pipe
// for ~64 cycles whatever the number of active lanes, so the latency of a
// track step is set by how many FP64 instructions it issues. These versions
// issue about 12 each (the reduction and the table index use integer
// instructions), fewer than the general-purpose library routines, and stay
// within 1.2 ulp of the correctly rounded result. Arguments outside the
// reduced range (non-positive, subnormal, non-finite for log; |x| >= 708
// for exp) go to the library routine.
//
// The tables are computed on the host from the definitions (extended
// precision), copied to device memory once per context, and read through the
// read-only data cache.
#pragma once

#include <cmath>
#include <cstdint>

namespace celer {

constexpr int kLogTable = 256;  // reduced mantissa m in [0.75, 1.5), 256 intervals
constexpr int kExpTable = 64;   // 2^(j/64)
constexpr int kMtLog = 0;                              // kLogTable x {1/c, L_hi, L_lo, 0}
constexpr int kMtExp = kMtLog + 4 * kLogTable;         // kExpTable x {T_hi, T_lo}
constexpr int kSinTable = 256;  // sin, cos of 2 pi j / 256
constexpr int kMtSin = kMtExp + 2 * kExpTable;         // (kSinTable + 1) x {sin, cos}
constexpr int kMtConst = kMtSin + 2 * (kSinTable + 1); // constants below
constexpr int kMtLn2Hi = kMtConst + 0;                 // ln 2 rounded to a multiple of 2^-42
constexpr int kMtLn2Lo = kMtConst + 1;                 // ln 2 - kMtLn2Hi
constexpr int kMtInvC = kMtConst + 2;                  // 64 / ln 2
constexpr int kMtCHi = kMtConst + 3;                   // ln 2 / 64 rounded to a multiple of 2^-42
constexpr int kMtCLo = kMtConst + 4;                   // ln 2 / 64 - kMtCHi
constexpr int kMt2PiHi = kMtConst + 5;                 // 2 pi
constexpr int kMt2PiLo = kMtConst + 6;                 // 2 pi - kMt2PiHi
constexpr int kMtStepInv = kMtConst + 7;               // 256 / (2 pi)
constexpr int kMtStepHi = kMtConst + 8;                // 2 pi / 256 rounded to a multiple of 2^-35 (30 bits)
constexpr int kMtStepLo = kMtConst + 9;                // 2 pi / 256 - kMtStepHi
constexpr int kMathTableSize = kMtConst + 10;          // doubles

// Fill the table (kMathTableSize doubles). Host code, extended precision.
//  log: interval j of the reduced mantissa has centre c_j (c = 1 exactly for
//  the two intervals next to 1, so that log x near 1 keeps full relative
//  accuracy), 1/c_j rounded to binary64, and L_j = -log(rounded 1/c_j) split
//  into a head that is a multiple of 2^-42 and a tail.
//  exp: T_j = 2^(j/64) as a head and a tail.
//  sin/cos: sin and cos of 2 pi j / 256, j = 0 .. 256.
inline void build_math_table(double* out) {
  typedef long double ld;
  const ld ln2 = logl(2.0L);
  auto head42 = [](ld v) { return (double)(nearbyintl(v * 0x1p42L) / 0x1p42L); };
  for (int j = 0; j < kLogTable; ++j) {
    ld c;
    if (j == 127 || j == 128) {
      c = 1.0L;
    } else if (j < 128) {
      c = 0.75L + ((ld)j + 0.5L) / 512.0L;  // m in [0.75, 1): intervals of 1/512
    } else {
      c = 1.0L + ((ld)(j - 128) + 0.5L) / 256.0L;  // m in [1, 1.5): intervals of 1/256
    }
    const double invc = (double)(1.0L / c);
    const ld L = -logl((ld)invc);
    const double hi = head42(L);
    out[kMtLog + 4 * j + 0] = invc;
    out[kMtLog + 4 * j + 1] = hi;
    out[kMtLog + 4 * j + 2] = (double)(L - (ld)hi);
    out[kMtLog + 4 * j + 3] = 0.0;
  }
  for (int j = 0; j < kExpTable; ++j) {
    const ld T = exp2l((ld)j / 64.0L);
    const double hi = (double)T;
    out[kMtExp + 2 * j + 0] = hi;
    out[kMtExp + 2 * j + 1] = (double)(T - (ld)hi);
  }
  const double l2hi = head42(ln2);
  out[kMtLn2Hi] = l2hi;
  out[kMtLn2Lo] = (double)(ln2 - (ld)l2hi);
  out[kMtInvC] = (double)(64.0L / ln2);
  const double chi = head42(ln2 / 64.0L);
  out[kMtCHi] = chi;
  out[kMtCLo] = (double)(ln2 / 64.0L - (ld)chi);
  const ld twopi = 8.0L * atanl(1.0L);
  for (int j = 0; j <= kSinTable; ++j) {
    const ld a = twopi * (ld)j / (ld)kSinTable;
    out[kMtSin + 2 * j + 0] = (double)sinl(a);
    out[kMtSin + 2 * j + 1] = (double)cosl(a);
  }
  const double tp = (double)twopi;
  out[kMt2PiHi] = tp;
  out[kMt2PiLo] = (double)(twopi - (ld)tp);
  const ld step = twopi / (ld)kSinTable;
  out[kMtStepInv] = (double)(1.0L / step);
  const double shi = (double)(nearbyintl(step * 0x1p35L) / 0x1p35L);
  out[kMtStepHi] = shi;
  out[kMtStepLo] = (double)(step - (ld)shi);
  for (int i = kMtStepLo + 1; i < kMathTableSize; ++i) out[i] = 0.0;
}

#ifdef __CUDACC__
// log x = k ln 2 + L_j + log1p(r), x = 2^k m with m in [0.75, 1.5) taken from
// the bits (x - bits(0.75) gives k in the exponent field and the interval j
// in the next 8 bits), r = m / c_j - 1 = fma(m, 1/c_j, -1), |r| < 2^-8.
// k ln2_hi + L_hi is exact (both multiples of 2^-42, below 2^10).
// The elementary functions below are called, not inlined: the step kernels
// reach them from many sites, and one shared copy keeps the instruction cache
// free for the step code (inlined copies measured 6-9 % slower).
static __device__ __noinline__ double fast_log(double x, const double* __restrict__ mt) {
  const long long ix = __double_as_longlong(x);
  if ((unsigned long long)(ix - 0x0010000000000000ll) >= 0x7FE0000000000000ull) return log(x);
  const long long tmp = ix - 0x3FE8000000000000ll;
  const int k = (int)(tmp >> 52);
  const int j = (int)((tmp >> 44) & (kLogTable - 1));
  const double m = __longlong_as_double(ix - ((long long)k << 52));
  const double2 cl = __ldg(reinterpret_cast<const double2*>(mt + kMtLog + 4 * j));
  const double llo = __ldg(mt + kMtLog + 4 * j + 2);
  const double r = fma(m, cl.x, -1.0);
  // log1p(r) = r - r^2/2 + r^3/3 - ... + r^7/7 (truncation < 2^-59 relative)
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(r, q, 0.2);
  q = fma(r, q, -0.25);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  const double p = fma(r * r, q, r);
  const double kd = (double)k;
  const double hi = fma(kd, __ldg(mt + kMtLn2Hi), cl.y);
  const double lo = fma(kd, __ldg(mt + kMtLn2Lo), llo) + p;
  return hi + lo;
}

// exp x = 2^(n/64) exp(r), n = round(64 x / ln 2) read from the low bits of
// x 64/ln2 + 1.5 2^52, r = x - n ln2/64 in two exact-then-rounded steps,
// |r| <= ln2/128; 2^(n/64) = 2^(n >> 6) T_(n & 63), the power of two added
// to the exponent field (|x| < 708 keeps the result normal).
static __device__ __noinline__ double fast_exp(double x, const double* __restrict__ mt) {
  // |x| < 708 on the bit pattern (NaN and inf fail it, as in FP64)
  if ((unsigned long long)(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll) >= 0x4086200000000000ull) return exp(x);
  constexpr double kShift = 0x1.8p52;
  const double t = fma(x, __ldg(mt + kMtInvC), kShift);
  const int n = (int)(uint32_t)__double_as_longlong(t);
  const double nd = t - kShift;
  const double rh = fma(-nd, __ldg(mt + kMtCHi), x);
  const double r = fma(-nd, __ldg(mt + kMtCLo), rh);
  // exp(r) - 1 = r + r^2/2 + ... + r^6/720 (truncation < 2^-64 relative)
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(r, q, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double2 T = __ldg(reinterpret_cast<const double2*>(mt + kMtExp + 2 * (n & (kExpTable - 1))));
  const double y = T.x + fma(T.x, p, T.y);
  return __longlong_as_double(__double_as_longlong(y) + ((long long)(n >> 6) << 52));
}
// sin and cos of 2 pi u for u in [0, 1] (an azimuth from a uniform draw):
// j = nearest multiple of 1/256, r = u - j/256 exact, |r| <= 2^-9, theta =
// 2 pi r (|theta| < 0.0123), then the angle-addition formulas with the
// tabulated sin, cos of 2 pi j/256 and short Taylor series for theta
// (truncation below 2^-70). Arguments outside [0, 1] go to sincospi.
static __device__ __noinline__ void fast_sincos_2pi(double u, const double* __restrict__ mt, double* s, double* c) {
  if (!(u >= 0.0 && u <= 1.0)) {
    sincospi(2.0 * u, s, c);
    return;
  }
  const int j = __double2int_rn(u * (double)kSinTable);
  const double r = u - (double)j * (1.0 / kSinTable);
  const double th = fma(r, __ldg(mt + kMt2PiHi), r * __ldg(mt + kMt2PiLo));
  const double t2 = th * th;
  // sin th = th + th^3 (-1/6 + t2 (1/120 - t2/5040)); cos th - 1 = t2 (-1/2 + t2 (1/24 - t2/720))
  const double sp = fma(t2, fma(t2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0);
  const double sn = fma(th * t2, sp, th);
  const double cm1 = t2 * fma(t2, fma(t2, -1.0 / 720.0, 1.0 / 24.0), -0.5);
  const double2 sc = __ldg(reinterpret_cast<const double2*>(mt + kMtSin + 2 * j));
  *s = sc.x + fma(sc.x, cm1, sc.y * sn);
  *c = sc.y + fma(sc.y, cm1, -sc.x * sn);
}

// sin and cos of an angle x (|x| < 1e5; others go to sincos): j = nearest
// multiple of 2 pi / 256, r = x - j 2pi/256 in two steps (Cody and Waite: the
// head has 30 bits, so j head is exact for |j| < 2^22 and the first step is
// exact), |r| <= pi/256, then the table and the series of fast_sincos_2pi
// with theta = r.
static __device__ __noinline__ void fast_sincos(double x, const double* __restrict__ mt, double* s, double* c) {
  if (!(fabs(x) < 1e5)) {
    sincos(x, s, c);
    return;
  }
  const double jd = rint(x * __ldg(mt + kMtStepInv));
  const int j = (int)jd;
  const double th = fma(-jd, __ldg(mt + kMtStepLo), fma(-jd, __ldg(mt + kMtStepHi), x));
  const double t2 = th * th;
  const double sp = fma(t2, fma(t2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0);
  const double sn = fma(th * t2, sp, th);
  const double cm1 = t2 * fma(t2, fma(t2, -1.0 / 720.0, 1.0 / 24.0), -0.5);
  const double2 sc = __ldg(reinterpret_cast<const double2*>(mt + kMtSin + 2 * (j & (kSinTable - 1))));
  *s = sc.x + fma(sc.x, cm1, sc.y * sn);
  *c = sc.y + fma(sc.y, cm1, -sc.x * sn);
}
#endif

}  // namespace celer
