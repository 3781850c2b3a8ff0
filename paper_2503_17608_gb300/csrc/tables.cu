// Cross-section, stopping-power and range tables, built on the device at
// context creation.
//
// Every table is sampled on 200 log-spaced energies from 1 keV to 10 GeV and
// interpolated linearly in ln E by the step kernels. Columns per material:
// Compton (n_e times the Klein-Nishina total cross-section), photoelectric
// (0.15/cm (E/30 keV)^-3.5 scaled by (n_e/n_e,w)(Z/Z_w)^3), pair
// (0.0096/cm ln(E/1.022 MeV) above threshold scaled by (n_e/n_e,w)(Z/Z_w)),
// Moller (n_e times the closed-form delta-ray cross-section above the cut),
// bremsstrahlung (ln(T/k_cut)/X0 for the 1/k spectrum) and the range
// R(E) = E_0 / (2 S(E_0)) + integral of dE / S with S the restricted
// collision plus restricted radiative stopping power, integrated bin by bin
// with 16-point Gauss-Legendre quadrature in ln E.
#include "tables.h"

#include "physics.cuh"

namespace celer {

namespace {

constexpr double kRe = 2.8179403262e-13;  // classical electron radius, cm
constexpr double kPeMu0 = 0.15, kPeE0 = 0.030, kPePower = -3.5;
constexpr double kPairMu0 = 0.0096;
constexpr int kRaw = 6;  // raw columns: 5 cross-sections + stopping power

__device__ double kn_total(double E) {
  const double k = E / kMe;
  const double a = 1.0 + 2.0 * k;
  const double L = log(a);
  const double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k);
  const double t2 = L / (2.0 * k);
  const double t3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * kPi * kRe * kRe * (t1 + t2 - t3);
}

__device__ double moller_total(double T, double Tcut) {
  if (T <= 2.0 * Tcut) return 0.0;
  const double x = Tcut / T;
  const double g = T / kMe + 1.0;
  const double g2 = g * g;
  const double b2 = 1.0 - 1.0 / g2;
  const double br = (g - 1.0) * (g - 1.0) / g2 * (0.5 - x) + 1.0 / x - 1.0 / (1.0 - x) -
                    (2.0 * g - 1.0) / g2 * log((1.0 - x) / x);
  return 2.0 * kPi * kRe * kRe / (b2 * (g - 1.0)) * br;
}

// Restricted collision stopping power (Berger-Seltzer form for electrons,
// energy transfers below min(Tcut, T/2), no density effect) plus restricted
// radiative loss min(T, k_cut) / X0.
__device__ double stopping_power(double T, const MaterialData& m, double Tcut, double kcut) {
  const double tau = T / kMe;
  const double g2 = (tau + 1.0) * (tau + 1.0);
  const double b2 = tau * (tau + 2.0) / g2;
  const double d = fmin(Tcut / kMe, 0.5 * tau);
  const double Im = m.I / kMe;
  const double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d) +
                   (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / g2;
  const double col = 2.0 * kPi * kRe * kRe * kMe * m.ne / b2 * (log(2.0 * (tau + 2.0) / (Im * Im)) + F);
  return col + fmin(T, kcut) / m.X0;
}

__global__ void k_table_values(TableBuild tb, double* raw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int mat = blockIdx.y;
  if (i >= kGrid) return;
  const MaterialData m = tb.mats[mat];
  const double E = exp(tb.lnEmin + i * tb.dl);
  const int P = tb.processes;
  double* r = raw + (size_t)mat * kRaw * kGrid;
  r[0 * kGrid + i] = (P & PROC_COMPTON) ? m.ne * kn_total(E) : 0.0;
  r[1 * kGrid + i] = (P & PROC_PE) ? m.f_pe * kPeMu0 * pow(E / kPeE0, kPePower) : 0.0;
  r[2 * kGrid + i] = ((P & PROC_PAIR) && E > kPairThreshold) ? m.f_pair * kPairMu0 * log(E / kPairThreshold) : 0.0;
  r[3 * kGrid + i] = (P & PROC_MOLLER) ? m.ne * moller_total(E, tb.cut_moller) : 0.0;
  r[4 * kGrid + i] = ((P & PROC_BREMS) && E > tb.cut_brems) ? log(E / tb.cut_brems) / m.X0 : 0.0;
  r[5 * kGrid + i] = (P & PROC_ELOSS) ? stopping_power(E, m, tb.cut_moller, tb.cut_brems) : 0.0;
}

// One block per material: per-bin integrals of E/S(E) d(ln E) in parallel,
// then a sequential running sum from R_0 = E_0 / (2 S_0).
__global__ void k_table_range(TableBuild tb, const double* raw, double* range) {
  __shared__ double gx[16], gw[16];
  __shared__ double seg[kGrid];
  const int mat = blockIdx.x;
  const MaterialData m = tb.mats[mat];
  if (threadIdx.x < 16) {
    // Gauss-Legendre node i of P_16 by Newton iteration from the Tricomi guess
    const int n = 16, i = threadIdx.x;
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double deriv = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pm1 = 1.0, p = z;
      for (int k = 2; k <= n; ++k) {
        const double pn = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
        pm1 = p;
        p = pn;
      }
      deriv = n * (z * p - pm1) / (z * z - 1.0);
      const double dz = p / deriv;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    double pm1 = 1.0, p = z;
    for (int k = 2; k <= n; ++k) {
      const double pn = ((2.0 * k - 1.0) * z * p - (k - 1.0) * pm1) / k;
      pm1 = p;
      p = pn;
    }
    deriv = n * (z * p - pm1) / (z * z - 1.0);
    gx[i] = z;
    gw[i] = 2.0 / ((1.0 - z * z) * deriv * deriv);
  }
  __syncthreads();
  double* R = range + (size_t)mat * kGrid;
  if (!(tb.processes & PROC_ELOSS)) {
    for (int i = threadIdx.x; i < kGrid; i += blockDim.x) R[i] = 0.0;
    return;
  }
  for (int i = threadIdx.x; i < kGrid - 1; i += blockDim.x) {
    const double a = tb.lnEmin + i * tb.dl;
    double sum = 0.0;
    for (int j = 0; j < 16; ++j) {
      const double E = exp(a + 0.5 * (1.0 + gx[j]) * tb.dl);
      sum += gw[j] * E / stopping_power(E, m, tb.cut_moller, tb.cut_brems);
    }
    seg[i] = 0.5 * tb.dl * sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* S = raw + (size_t)mat * kRaw * kGrid + 5 * kGrid;
    double acc = exp(tb.lnEmin) / (2.0 * S[0]);
    R[0] = acc;
    for (int i = 0; i < kGrid - 1; ++i) {
      acc = acc + seg[i];
      R[i + 1] = acc;
    }
  }
}

// Pack (value, next - value) pairs: columns Compton, PE, pair, Moller, brems, range.
__global__ void k_table_pack(int n_mat, const double* raw, const double* range, double2* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;
  const int mat = blockIdx.z;
  if (i >= kGrid || mat >= n_mat) return;
  const double* src = (col < 5) ? raw + ((size_t)mat * kRaw + col) * kGrid : range + (size_t)mat * kGrid;
  const double v = src[i];
  const double nxt = (i + 1 < kGrid) ? src[i + 1] : v;
  out[((size_t)mat * kCols + col) * kGrid + i] = make_double2(v, nxt - v);
}

}  // namespace

cudaError_t build_tables(const TableBuild& tb, double2* d_tables, double* d_scratch, cudaStream_t stream) {
  double* raw = d_scratch;
  double* range = d_scratch + (size_t)tb.n_mat * kRaw * kGrid;
  k_table_values<<<dim3((kGrid + 127) / 128, tb.n_mat), 128, 0, stream>>>(tb, raw);
  k_table_range<<<tb.n_mat, 256, 0, stream>>>(tb, raw, range);
  k_table_pack<<<dim3((kGrid + 127) / 128, kCols, tb.n_mat), 128, 0, stream>>>(tb.n_mat, raw, range, d_tables);
  return cudaGetLastError();
}

size_t table_scratch_doubles(int n_mat) { return (size_t)n_mat * (kRaw + 1) * kGrid; }

}  // namespace celer
