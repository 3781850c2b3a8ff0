// Device functions of the transport: counter-based random numbers, table
// interpolation, geometry (straight line and exact helix in a uniform field),
// and the sampling of the discrete interactions.
//
// The paper fixes no physics model (it profiles the stepping loop of an EM
// transport code); the model here is the simplified EM set of the benchmark
// workloads: Klein-Nishina Compton, a power-law photoelectric effect, pair
// production with local deposition of the pair's kinetic energy, Moller delta
// rays, a 1/k bremsstrahlung spectrum and restricted continuous loss. All of
// it is binary64: the workloads fix FP64.
#pragma once

#include "common.cuh"
#include "fastmath.cuh"

namespace celer {

constexpr double kMe = 0.51099895;        // electron mass, MeV
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;
constexpr double kFieldK = 2.99792458;    // curvature [1/cm] = kFieldK * B[T] / p[MeV/c]
constexpr double kPairThreshold = 1.022;  // MeV, as in the photon model definition
constexpr double kAlphaR = 0.2;           // range step function: fraction of range
constexpr double kFinalR = 0.1;           // range step function: final range, cm
constexpr double kInf = __builtin_huge_val();
// Attempts after which a rejection sampler gives up (never reached for finite
// inputs: the acceptance probability is at least ~0.4 per attempt).
constexpr int kMaxAttempts = 4096;
// Compare-and-swap rounds a group of lanes may spend claiming buffer entries
// (each failed round means another group succeeded).
constexpr int kMaxCasAttempts = 1 << 16;
// Relative margins above which a step-limit candidate cannot be the shorter
// one after rounding: 1 + 2^-50 for a single quotient d / u tested as
// |d| > s |u| margin, 1 + 2^-48 for the range limit's lower bound (a few
// more roundings).
constexpr double kLimitMargin = 1.0 + 0x1p-50;
constexpr double kRangeMargin = 1.0 + 0x1p-48;
// Longest wait at a grid barrier of the persistent loop (~1 s at 2 GHz).
constexpr long long kBarrierTimeoutCycles = 2000000000ll;

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32 -> 64-bit
// products whose high words are mixed with the other two counter words and
// the round key; the key advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// One Philox block as a called function: a track's draws happen at many
// sites of the step kernels, and one shared copy of the ten rounds keeps the
// instruction cache free for the step code (inlined copies measured 3-4 %
// slower).
static __device__ __noinline__ uint4 philox_block(uint4 c, uint2 k) { return philox4x32_10(c, k); }

// u = (floor(w / 2^12) + 1/2) 2^-52 in [2^-53, 1 - 2^-53], built from the
// exponent bits of 1.0 and one exact subtraction (Sterbenz).
__device__ __forceinline__ double unit_from_bits(unsigned long long w) {
  return __longlong_as_double(0x3FF0000000000000ull | (w >> 12)) - (1.0 - 0x1p-53);
}

// A track's random stream: key (seed, event), counter (tid lo, tid hi,
// index / 2, 0); even indices take output words 0-1, odd ones 2-3. The
// Philox block of the last even index is cached so that each pair of draws
// costs one Philox evaluation.
struct TrackRng {
  uint2 key;
  unsigned long long tid;
  uint32_t ctr;
  uint32_t cached_block;
  uint4 cached;

  __device__ TrackRng(uint32_t seed, uint32_t event, unsigned long long tid_, uint32_t ctr_)
      : key(make_uint2(seed, event)), tid(tid_), ctr(ctr_), cached_block(0xFFFFFFFFu) {}

  __device__ __forceinline__ unsigned long long raw() {
    const uint32_t block = ctr >> 1;
    if (block != cached_block) {
      cached = philox_block(make_uint4((uint32_t)tid, (uint32_t)(tid >> 32), block, 0u), key);
      cached_block = block;
    }
    const unsigned long long w = (ctr & 1u) ? ((unsigned long long)cached.w << 32 | cached.z)
                                            : ((unsigned long long)cached.y << 32 | cached.x);
    ++ctr;
    return w;
  }
  __device__ __forceinline__ double uniform() { return unit_from_bits(raw()); }
};

// Comparisons of doubles on their bit patterns (integer instructions instead
// of the FP64 pipe). For x, y >= +0 (+inf included) x < y iff bits(x) <
// bits(y) as signed integers; a negative x (-0 included) has negative bits,
// below every y >= +0, and a positive NaN has bits above +inf. Each use
// states why its operands qualify and why a NaN gives the outcome of the
// FP64 comparison.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }

// ------------------------------------------------------------------ tables
struct GridPos {
  int bin;
  double frac;
};

// Grid coordinate (ln E - ln E_min) / dl, bin clamped to [0, n - 2].
__device__ __forceinline__ GridPos grid_pos(double E, double lnEmin, double inv_dl, const double* mt) {
  const double x = (fast_log(E, mt) - lnEmin) * inv_dl;
  int b = __double2int_rd(x);  // (int)floor(x), one conversion
  b = b < 0 ? 0 : (b > kGrid - 2 ? kGrid - 2 : b);
  return GridPos{b, x - (double)b};
}

// Linear interpolation in ln E; each entry holds (value, next value - value).
__device__ __forceinline__ double interp(const double2* col, GridPos g) {
  const double2 v = col[g.bin];
  return fma(g.frac, v.y, v.x);
}

// Inverse of the range interpolation: the largest bin i <= n - 2 with
// R_i <= r, then ln E linear in R inside it. r <= R_0: the track stopped.
// Ranges are non-negative, so the search compares their bit patterns as
// integers (same order as the values) and keeps the FP64 pipe free.
__device__ __forceinline__ double inverse_range(const double2* R, double r, double lnEmin, double dl,
                                                const double* mt) {
  const long long rb = __double_as_longlong(r);
  if (rb <= __double_as_longlong(R[0].x)) return 0.0;  // r <= R_0 > 0 on the bits (r may be negative)
  int lo = 0;
#pragma unroll
  for (int step = 128; step > 0; step >>= 1) {
    const int probe = lo + step;
    if (probe <= kGrid - 2 && __double_as_longlong(R[probe].x) <= rb) lo = probe;
  }
  const double2 v = R[lo];
  const double lnE = lnEmin + lo * dl + (r - v.x) / v.y * dl;
  return fast_exp(lnE, mt);
}

// ------------------------------------------------------------- kinematics
// An FP64 warp instruction occupies a GB300 sub-partition's FP64 pipe for
// the same time whatever its active lanes, so the kinematics below take
// reciprocal square roots once instead of a square root and divisions.

// Rotate (ux, uy, uz) by polar cosine cost and azimuth 2 pi u_phi about
// itself: frame e1 = (u x z)/|u x z|, e2 = u x e1 (e1 = x near the poles),
// then renormalised. The input is a unit vector to rounding, so the result's
// squared norm q is 1 + O(1e-16) and one Newton step from 1, 1.5 - q/2, is
// 1/sqrt(q) to O((q - 1)^2).
__device__ __forceinline__ void rotate_dir(double& ux, double& uy, double& uz, double cost, double u_phi,
                                           const double* mt) {
  const double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  double sp, cp;
  fast_sincos_2pi(u_phi, mt, &sp, &cp);
  double e1x, e1y, e1z, e2x, e2y, e2z;
  if ((dbits(uz) & 0x7FFFFFFFFFFFFFFFll) < dbits(1.0 - 1e-10)) {  // |uz| < 1 - 1e-10 on the bits
    const double q = ux * ux + uy * uy;
    const double inv_n = rsqrt(q);
    e1x = uy * inv_n;
    e1y = -ux * inv_n;
    e1z = 0.0;
    e2x = uz * ux * inv_n;
    e2y = uz * uy * inv_n;
    e2z = -q * inv_n;
  } else {
    const double q = uz * uz + uy * uy;
    const double inv_n = rsqrt(q);
    e1x = 1.0;
    e1y = 0.0;
    e1z = 0.0;
    e2x = 0.0;
    e2y = uz * inv_n;
    e2z = -uy * inv_n;
  }
  const double vx = cost * ux + sint * (cp * e1x + sp * e2x);
  const double vy = cost * uy + sint * (cp * e1y + sp * e2y);
  const double vz = cost * uz + sint * (cp * e1z + sp * e2z);
  const double inv = fma(-0.5, fma(vx, vx, fma(vy, vy, vz * vz)), 1.5);
  ux = vx * inv;
  uy = vy * inv;
  uz = vz * inv;
}

// Signed curvature of a charged track in B along z: the transverse
// direction turns by kappa * s over a path s; kappa = q B k / p and its
// inverse p / (q B k) from one reciprocal square root of p^2.
struct Curvature {
  double kappa, inv_kappa;
};
__device__ __forceinline__ Curvature curvature(uint8_t ptype, double E, double Bz) {
  const double q = (ptype == ELECTRON) ? -1.0 : 1.0;
  const double p2 = E * (E + 2.0 * kMe);
  const double r = rsqrt(p2);
  const double qbk = q * Bz * kFieldK;
  return Curvature{qbk * r, (p2 * r) / qbk};
}

// Exact helix for du/ds = kappa (u x z), with 1 - cos(phi) = 2 sin^2(phi/2).
__device__ __forceinline__ void helix_move(Curvature c, double s, double& x, double& y, double& z, double& ux,
                                           double& uy, double uz, const double* mt) {
  const double phi = c.kappa * s;
  double hs, hc;
  fast_sincos(0.5 * phi, mt, &hs, &hc);
  const double sphi = 2.0 * hs * hc;
  const double omc = 2.0 * hs * hs;
  const double cphi = 1.0 - omc;
  const double ox = ux, oy = uy;
  x += (ox * sphi + oy * omc) * c.inv_kappa;
  y += (oy * sphi - ox * omc) * c.inv_kappa;
  z += uz * s;
  ux = ox * cphi + oy * sphi;
  uy = oy * cphi - ox * sphi;
}

// Numerical field propagation (Sec. 3.3): a field step of length s takes
// n = ceil(s |kappa| / 0.1) equal substeps (at most 0.1 rad of turn each, at
// least one) of classical fourth-order Runge-Kutta for the transverse motion,
// dx/ds = ux, dy/ds = uy, dux/ds = kappa uy, duy/ds = -kappa ux; z advances
// by uz s exactly; the transverse direction is rescaled at the end to its
// length at the start.
constexpr double kRkTurn = 0.1;
__device__ __forceinline__ int rk_substeps(double kappa, double s) {
  const int n = (int)ceil(s * fabs(kappa) / kRkTurn);
  return n < 1 ? 1 : n;
}
__device__ __forceinline__ void rk_move(double kappa, double s, int n, double& x, double& y, double& z, double& ux,
                                        double& uy, double uz) {
  const double q0 = ux * ux + uy * uy;
  const double h = s / n;
  double X = x, Y = y, U = ux, V = uy;
  for (int i = 0; i < n; ++i) {
    const double c1 = kappa * V, d1 = -kappa * U;
    const double U2 = U + 0.5 * h * c1, V2 = V + 0.5 * h * d1;
    const double c2 = kappa * V2, d2 = -kappa * U2;
    const double U3 = U + 0.5 * h * c2, V3 = V + 0.5 * h * d2;
    const double c3 = kappa * V3, d3 = -kappa * U3;
    const double U4 = U + h * c3, V4 = V + h * d3;
    const double c4 = kappa * V4, d4 = -kappa * U4;
    X += h / 6.0 * (U + 2.0 * U2 + 2.0 * U3 + U4);
    Y += h / 6.0 * (V + 2.0 * V2 + 2.0 * V3 + V4);
    U += h / 6.0 * (c1 + 2.0 * c2 + 2.0 * c3 + c4);
    V += h / 6.0 * (d1 + 2.0 * d2 + 2.0 * d3 + d4);
  }
  const double q = U * U + V * V;
  if (q > 0.0) {
    const double f = sqrt(q0 / q);
    U *= f;
    V *= f;
  }
  x = X;
  y = Y;
  z += uz * s;
  ux = U;
  uy = V;
}

// Smallest turn angle t in [0, 2 pi) with sin(sigma t + beta) = d.
__device__ __forceinline__ double first_turn(double d, double beta, double sigma) {
  const double a1 = asin(d);
  const double a2 = kPi - a1;
  double t1 = fmod(sigma * (a1 - beta), kTwoPi);
  if (t1 < 0.0) t1 += kTwoPi;
  double t2 = fmod(sigma * (a2 - beta), kTwoPi);
  if (t2 < 0.0) t2 += kTwoPi;
  return fmin(t1, t2);
}

// Path length along the helix to the first side plane (|x| = hx, |y| = hy),
// from the intersection of its transverse circle with each plane; kInf when
// the circle stays inside.
static __device__ __noinline__ double helix_side_distance(Curvature c, double x, double y, double ux, double uy,
                                                          double hx, double hy) {
  CELER_LANES(LS_HELIX_SIDE);
  const double A2 = ux * ux + uy * uy;
  if (dbits(A2) == 0ll) return kInf;  // A2 >= +0
  const double inv_A = rsqrt(A2);
  const double A = A2 * inv_A;
  const double kappa = c.kappa;
  const double inv_K = fabs(c.inv_kappa);
  const double sigma = kappa > 0.0 ? 1.0 : -1.0;
  const double xc = x + uy * c.inv_kappa;
  const double yc = y - ux * c.inv_kappa;
  const double rho = A * inv_K;
  if (xc + rho < hx && xc - rho > -hx && yc + rho < hy && yc - rho > -hy) return kInf;
  double tmin = kInf;
  const double bx = atan2(-uy, ux);
  const double by = atan2(ux, uy);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double X = i == 0 ? hx : -hx;
    const double d = kappa * (X - xc) * inv_A;
    if ((dbits(d) & 0x7FFFFFFFFFFFFFFFll) <= dbits(1.0)) tmin = fmin(tmin, first_turn(d, bx, sigma));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double Y = i == 0 ? hy : -hy;
    const double d = kappa * (Y - yc) * inv_A;
    if ((dbits(d) & 0x7FFFFFFFFFFFFFFFll) <= dbits(1.0)) tmin = fmin(tmin, first_turn(d, by, sigma));
  }
  return tmin == kInf ? kInf : tmin * inv_K;
}

// ------------------------------------------------------------- interactions
// The rejection samplers below decide each attempt in FP32 and fall back to
// FP64 only near the acceptance boundary. An FP64 warp instruction holds a
// GB300 sub-partition's FP64 pipe for 64 cycles, an FP32 one for about two,
// so an FP64 attempt (~40 instructions with its exp or sqrt) costs ~2,500
// cycles and an FP32 one a few hundred. Only the accepted attempt's value is
// computed in FP64, by the same expressions as the plain FP64 sampler, so
// the samples are bit-identical to it:
//  * the FP32 quantities are evaluated from cancellation-free forms
//    (1 - eps by expm1 or an algebraic rewrite, 2b - a likewise) with
//    relative errors below 2^-16 of the values the FP64 expressions
//    approximate, and the FP64 expressions are within 2^-19 of them
//    whenever 1 - eps >= 2^-30 and 2b - a >= 2^-30 (2k + 1) eps, which the
//    filter checks;
//  * a decision is taken in FP32 only if the two sides differ by more than
//    kFilterMargin = 2^-12 relative, far above both error bounds, so both
//    evaluations take the same decision; otherwise (probability ~2^-11 per
//    attempt) the FP64 test of the plain sampler decides.
// The filter covers k = E/m in [1e-4, 1e6] (Compton) and x = Tcut/T in
// [1e-8, 1/2) (Moller); other inputs take the plain FP64 sampler.
constexpr float kFilterMargin = 0x1p-12f;
constexpr float kFilterTiny = 0x1p-30f;

// n 2^-53 in FP32 for 1 <= n < 2^53, truncated to 24 bits (relative error
// below 2^-23), by integer operations only: with the draw word w,
// n = 2 (w >> 12) + 1 gives the draw u and 2^53 - n gives 1 - u.
__device__ __forceinline__ float f32_scaled_2m53(unsigned long long n) {
  const int lz = __clzll((long long)n);  // 11 .. 63
  const unsigned m24 = (unsigned)((n << lz) >> 40);
  return __uint_as_float(((unsigned)(137 - lz) << 23) | (m24 & 0x7FFFFFu));
}
__device__ __forceinline__ unsigned long long draw_numerator(unsigned long long w) { return ((w >> 12) << 1) | 1ull; }
constexpr unsigned long long k2p53 = 1ull << 53;

// A positive normal double in the FP32 exponent range, truncated to FP32
// (relative error below 2^-23) by integer operations.
__device__ __forceinline__ float f32_trunc(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = ((hi >> 20) & 0x7FFu) - 1023u + 127u;
  return __uint_as_float((e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// Klein-Nishina sampling of eps = E'/E by Butcher and Messel's
// composition-rejection: branch 1 samples eps from 1/eps (eps = eps0^u), branch
// 2 samples eps^2 uniformly; both are accepted with 1 - eps sin^2 / (1 + eps^2).
// Three draws per attempt. Returns eps; cost receives the scattering cosine;
// ok is cleared if the attempt limit was hit. With a = 1 - eps and b = k eps,
// t = 1 - cos = a / b and sin^2 = a (2b - a) / b^2, so the test
// u3 <= 1 - eps sin^2 / (1 + eps^2) is taken multiplied through by the
// positive b^2 (1 + eps^2), without divisions; t is divided out once, for
// the accepted attempt. This is the plain FP64 form; sample_compton below
// gives the same results with FP32 filtering.
static __device__ __noinline__ double sample_compton_fp64(double E, TrackRng& rng, double& cost, bool& ok,
                                                          const double* mt) {
  const double k = E / kMe;
  const double eps0 = 1.0 / (1.0 + 2.0 * k);
  const double eps0sq = eps0 * eps0;
  const double a1 = -fast_log(eps0, mt);
  const double w = 1.0 - eps0sq;
  double eps = 1.0, t = 0.0;
  ok = false;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    const double u1 = rng.uniform();
    const double u2 = rng.uniform();
    const double u3 = rng.uniform();
    if (u1 * (a1 + 0.5 * w) < a1) {
      eps = fast_exp(-a1 * u2, mt);
    } else {
      eps = sqrt(fma(w, u2, eps0sq));
    }
    const double a = 1.0 - eps;
    const double b = k * eps;
    const double B = b * b * (1.0 + eps * eps);
    if (eps * a * (2.0 * b - a) <= (1.0 - u3) * B) {
      t = a / b;
      ok = true;
      break;
    }
  }
  cost = 1.0 - t;
  return eps;
}

// FP32-filtered Compton sampler (same draws, same results as
// sample_compton_fp64). Per attempt, with u = u1..u3 and v = 1 - u:
//  branch: u1 (a1 + a2) < a1;
//  branch 1: x = a1 u2, eps = e^-x, a = -expm1(-x), 2b - a = (2k + 1) eps - 1
//    = expm1(a1 v2) (since (2k + 1) e^-a1 = 1 up to the FP64 roundings of
//    eps0 and a1, an absolute 2^-47.7 (2k + 1) eps);
//  branch 2: eps = sqrt(eps0^2 + w u2), w = 1 - eps0^2, a = w v2 / (1 + eps),
//    2b - a = (2k + 1) w u2 / (eps + eps0);
//  accept: eps a (2b - a) <= v3 b^2 (1 + eps^2).
// The loop keeps only the accepted attempt's draw and branch; its FP64 value
// is computed once after the loop, where the warp has reconverged (inside
// the loop, lanes accepting at different attempts would each run it).
static __device__ __noinline__ double sample_compton(double E, TrackRng& rng, double& cost, bool& ok,
                                                     const double* mt) {
  const double k = E / kMe;
  // 1e-4 <= k <= 1e6 on the bits (negative and NaN k fall outside)
  if ((unsigned long long)(dbits(k) - dbits(1e-4)) > (unsigned long long)(dbits(1e6) - dbits(1e-4)))
    return sample_compton_fp64(E, rng, cost, ok, mt);
  const double eps0 = 1.0 / (1.0 + 2.0 * k);
  const double eps0sq = eps0 * eps0;
  const double a1 = -fast_log(eps0, mt);
  const double w = 1.0 - eps0sq;
  const float kf = f32_trunc(k), e0f = f32_trunc(eps0), e0sqf = f32_trunc(eps0sq), a1f = f32_trunc(a1);
  const float wf = f32_trunc(w);
  const float k21f = fmaf(2.0f, kf, 1.0f);
  const float sf = fmaf(0.5f, wf, a1f);
  unsigned long long w2_acc = 0;
  int branch_acc = 0;
  ok = false;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    CELER_LANES(LS_COMPTON_TRY);
    const unsigned long long w1 = rng.raw(), w2 = rng.raw(), w3 = rng.raw();
    int branch = 0;   // 1 or 2 once decided
    int verdict = -1; // 1 accept, 0 reject, -1 undecided
    {
      const unsigned long long n2 = draw_numerator(w2);
      const float u1f = f32_scaled_2m53(draw_numerator(w1));
      const float u2f = f32_scaled_2m53(n2), v2f = f32_scaled_2m53(k2p53 - n2);
      const float v3f = f32_scaled_2m53(k2p53 - draw_numerator(w3));
      const float p = u1f * sf;
      if (p < a1f * (1.0f - kFilterMargin)) {
        branch = 1;
      } else if (p > a1f * (1.0f + kFilterMargin)) {
        branch = 2;
      }
      if (branch != 0) {
        float ef, af, cf;
        if (branch == 1) {
          const float x = a1f * u2f;
          ef = expf(-x);
          af = -expm1f(-x);
          cf = expm1f(a1f * v2f);
        } else {
          ef = sqrtf(fmaf(wf, u2f, e0sqf));
          af = wf * v2f / (1.0f + ef);
          cf = k21f * wf * u2f / (ef + e0f);
        }
        if (af >= kFilterTiny && cf >= kFilterTiny * k21f * ef) {
          const float bf = kf * ef;
          const float L = ef * af * cf;
          const float R = v3f * (bf * bf) * fmaf(ef, ef, 1.0f);
          if (L < R * (1.0f - kFilterMargin)) {
            verdict = 1;
          } else if (L > R * (1.0f + kFilterMargin)) {
            verdict = 0;
          }
        }
      }
    }
    if (verdict == 0) continue;
    if (verdict < 0) {  // the plain FP64 attempt
      const double u2 = unit_from_bits(w2);
      if (branch == 0) branch = (unit_from_bits(w1) * (a1 + 0.5 * w) < a1) ? 1 : 2;
      const double e = branch == 1 ? fast_exp(-a1 * u2, mt) : sqrt(fma(w, u2, eps0sq));
      const double a = 1.0 - e;
      const double b = k * e;
      const double B = b * b * (1.0 + e * e);
      if (!(e * a * (2.0 * b - a) <= (1.0 - unit_from_bits(w3)) * B)) continue;
    }
    w2_acc = w2;
    branch_acc = branch;
    ok = true;
    break;
  }
  double eps = 1.0, t = 0.0;
  if (ok) {
    const double u2 = unit_from_bits(w2_acc);
    eps = branch_acc == 1 ? fast_exp(-a1 * u2, mt) : sqrt(fma(w, u2, eps0sq));
    t = (1.0 - eps) / (k * eps);
  }
  cost = 1.0 - t;
  return eps;
}

// Moller: eps = T_delta / T in [x, 1/2] from the 1/eps^2 proposal, accepted
// with eps^2 B(eps) normalised by its maximum (9g^2 - 10g + 5)/4 at eps = 1/2.
// The test u2 <= norm f(eps) is taken multiplied by the positive (1 - eps)^2.
// Plain FP64 form; sample_moller below gives the same results.
static __device__ __noinline__ double sample_moller_fp64(double T, double Tcut, TrackRng& rng, bool& ok) {
  const double x = Tcut / T;
  const double y = 1.0 - 2.0 * x;
  const double g = T / kMe + 1.0;
  const double g2 = g * g;
  const double norm = 4.0 / (9.0 * g2 - 10.0 * g + 5.0);
  ok = false;
  double eps = 0.5;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    const double u1 = rng.uniform();
    const double u2 = rng.uniform();
    eps = x / fma(-u1, y, 1.0);
    const double om = 1.0 - eps;
    const double eom = eps * om;
    const double fom2 = (g - 1.0) * (g - 1.0) * eom * eom - (2.0 * g2 + 2.0 * g - 1.0) * eom + g2;
    if (u2 * (om * om) <= norm * fom2) {
      ok = true;
      break;
    }
  }
  return eps;
}

// FP32-filtered Moller sampler (same draws, same results as
// sample_moller_fp64). The proposal's denominator 1 - u1 (1 - 2x) is taken as
// v1 + 2x u1 (no cancellation); the polynomial (g-1)^2 eom^2 - (2g^2 + 2g - 1)
// eom + g^2 is at least 1/7 of the sum of its terms' magnitudes for g >= 1
// and eom <= 1/4, and 9g^2 - 10g + 5 at least 1/6 of its terms', so their
// FP32 relative errors stay below 2^-16; g - 1 = T/m is formed directly.
// g, g^2 and the normalisation are needed in FP64 only for an undecided
// attempt; the accepted attempt's eps is computed once, after the loop.
static __device__ __noinline__ double sample_moller(double T, double Tcut, TrackRng& rng, bool& ok) {
  const double x = Tcut / T;
  // 1e-8 <= x < 1/2 on the bits (negative and NaN x fall outside)
  if ((unsigned long long)(dbits(x) - dbits(1e-8)) >= (unsigned long long)(dbits(0.5) - dbits(1e-8)))
    return sample_moller_fp64(T, Tcut, rng, ok);
  const double y = 1.0 - 2.0 * x;
  const float tmf = f32_trunc(T) * (float)(1.0 / kMe);  // g - 1
  const float gf = tmf + 1.0f;
  const float g2f = gf * gf;
  const float normf = 4.0f / fmaf(9.0f, g2f, fmaf(-10.0f, gf, 5.0f));
  const float c1f = tmf * tmf;
  const float c2f = fmaf(2.0f, g2f, fmaf(2.0f, gf, -1.0f));
  const float xf = f32_trunc(x);
  const float txf = 2.0f * xf;
  double g = 0.0, g2 = 0.0, norm = 0.0;
  bool fp64_ready = false;
  unsigned long long w1_acc = 0;
  ok = false;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    CELER_LANES(LS_MOLLER_TRY);
    const unsigned long long w1 = rng.raw(), w2 = rng.raw();
    int verdict = -1;
    {
      const unsigned long long n1 = draw_numerator(w1);
      const float u1f = f32_scaled_2m53(n1), v1f = f32_scaled_2m53(k2p53 - n1);
      const float u2f = f32_scaled_2m53(draw_numerator(w2));
      const float ef = xf / fmaf(u1f, txf, v1f);
      const float omf = 1.0f - ef;
      const float eomf = ef * omf;
      const float L = u2f * (omf * omf);
      const float R = normf * (fmaf(c1f * eomf, eomf, -c2f * eomf) + g2f);
      if (L < R * (1.0f - kFilterMargin)) {
        verdict = 1;
      } else if (L > R * (1.0f + kFilterMargin)) {
        verdict = 0;
      }
    }
    if (verdict == 0) continue;
    if (verdict < 0) {  // the plain FP64 attempt
      if (!fp64_ready) {
        g = T / kMe + 1.0;
        g2 = g * g;
        norm = 4.0 / (9.0 * g2 - 10.0 * g + 5.0);
        fp64_ready = true;
      }
      const double e = x / fma(-unit_from_bits(w1), y, 1.0);
      const double om = 1.0 - e;
      const double eom = e * om;
      const double fom2 = (g - 1.0) * (g - 1.0) * eom * eom - (2.0 * g2 + 2.0 * g - 1.0) * eom + g2;
      if (!(unit_from_bits(w2) * (om * om) <= norm * fom2)) continue;
    }
    w1_acc = w1;
    ok = true;
    break;
  }
  return ok ? x / fma(-unit_from_bits(w1_acc), y, 1.0) : 0.5;
}

}  // namespace celer
