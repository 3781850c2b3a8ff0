/*
 * Physics definitions of the oracle -- TEST INFRASTRUCTURE.
 *
 * The paper fixes no physics model (it profiles the stepping loop of an EM
 * transport code, Sec. 2-3); the model below is the simplified EM set the
 * benchmark workloads specify, written out plainly in binary64:
 *   - Compton scattering: Klein-Nishina total cross-section (closed form) and
 *     the Butcher-Messel composition-rejection sampling of eps = E'/E;
 *   - photoelectric: mu = 0.15/cm (E / 30 keV)^-3.5 for water;
 *   - pair production: mu = 0.0096/cm ln(E / 1.022 MeV) above 1.022 MeV;
 *   - photon processes in other materials scaled from water: Compton by the
 *     electron density, photoelectric by (ne/ne_w)(Z/Z_w)^3 (per-atom Z^4),
 *     pair by (ne/ne_w)(Z/Z_w) (per-atom Z^2);
 *   - Moller delta rays above a cut: closed-form per-electron cross-section
 *     and rejection sampling from a 1/eps^2 proposal;
 *   - bremsstrahlung with a 1/k photon spectrum: mu = ln(T/k_cut)/X0;
 *   - continuous loss: restricted collision stopping power (Berger-Seltzer
 *     form for electrons, no density effect) plus restricted radiative loss
 *     min(T, k_cut)/X0; range by 16-point Gauss-Legendre quadrature of 1/S;
 *   - motion in a uniform field along z: exact helix, or Runge-Kutta substeps
 *     with a cap on the substeps of one step (Sec. 3.3).
 */
#include "oracle.h"

#include <math.h>

#define OM_ME 0.51099895
#define OM_RE 2.8179403262e-13
#define OM_NA 6.02214076e23
#define OM_PI 3.14159265358979323846
#define OM_FIELD_K 2.99792458 /* curvature [1/cm] = K * B[T] / p[MeV/c] */
#define OM_RK_TURN 0.1        /* largest turn angle of one Runge-Kutta substep, rad */

double om_electron_density(const om_material* m) {
  if (m->ne > 0.0) return m->ne;
  return OM_NA * m->rho * m->Z / m->A;
}

/* Klein-Nishina total cross-section per electron [cm^2], k = E / m_e c^2. */
double om_sigma_kn(double E) {
  double k = E / OM_ME;
  double a = 1.0 + 2.0 * k;
  double L = log(a);
  double term1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - L / k);
  double term2 = L / (2.0 * k);
  double term3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * OM_PI * OM_RE * OM_RE * (term1 + term2 - term3);
}

/* Moller cross-section per target electron [cm^2] for producing a delta ray
 * with kinetic energy above Tcut from an electron of kinetic energy T
 * (integral of the Moller differential cross-section over eps = T_delta/T in
 * [Tcut/T, 1/2]). Zero when T <= 2 Tcut. */
double om_sigma_moller(double T, double Tcut) {
  if (T <= 2.0 * Tcut) return 0.0;
  double x = Tcut / T;
  double g = T / OM_ME + 1.0;
  double g2 = g * g;
  double b2 = 1.0 - 1.0 / g2;
  double bracket = (g - 1.0) * (g - 1.0) / g2 * (0.5 - x) + 1.0 / x - 1.0 / (1.0 - x)
                   - (2.0 * g - 1.0) / g2 * log((1.0 - x) / x);
  return 2.0 * OM_PI * OM_RE * OM_RE / (b2 * (g - 1.0)) * bracket;
}

/* Restricted collision stopping power of electrons [MeV/cm]: energy lost per
 * unit path to ionisation with energy transfers below min(Tcut, T/2); no
 * density-effect correction. */
double om_dedx_collision(double T, double Tcut, double ne, double I) {
  double tau = T / OM_ME;
  double g = tau + 1.0;
  double g2 = g * g;
  double b2 = tau * (tau + 2.0) / g2;
  double d = Tcut / OM_ME;
  if (d > 0.5 * tau) d = 0.5 * tau;
  double Im = I / OM_ME;
  double F = -1.0 - b2 + log((tau - d) * d) + tau / (tau - d)
             + (0.5 * d * d + (2.0 * tau + 1.0) * log(1.0 - d / tau)) / g2;
  double bracket = log(2.0 * (tau + 2.0) / (Im * Im)) + F;
  return 2.0 * OM_PI * OM_RE * OM_RE * OM_ME * ne / b2 * bracket;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
void om_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(OM_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Butcher-Messel sampling of the Klein-Nishina distribution. Per attempt three
 * draws (u1 branch, u2 value, u3 rejection); the scattered energy fraction is
 * eps, the photon scattering cosine 1 - (1 - eps) / (k eps). */
void om_sample_compton(double E, om_rng* r, double* eps_out, double* cost_out) {
  double k = E / OM_ME;
  double eps0 = 1.0 / (1.0 + 2.0 * k);
  double eps0sq = eps0 * eps0;
  double a1 = -log(eps0);
  double a2 = 0.5 * (1.0 - eps0sq);
  double eps, t;
  for (;;) {
    double u1 = om_draw(r);
    double u2 = om_draw(r);
    double u3 = om_draw(r);
    if (u1 * (a1 + a2) < a1) {
      eps = exp(-a1 * u2);
    } else {
      eps = sqrt(eps0sq + (1.0 - eps0sq) * u2);
    }
    t = (1.0 - eps) / (k * eps);
    double sint2 = t * (2.0 - t);
    double g = 1.0 - eps * sint2 / (1.0 + eps * eps);
    if (u3 <= g) break;
  }
  *eps_out = eps;
  *cost_out = 1.0 - t;
}

/* Moller: eps = T_delta / T in [x, 1/2], x = Tcut / T, from the proposal
 * 1/eps^2 (inverse CDF eps = x / (1 - u1 (1 - 2x))) accepted with probability
 * eps^2 B(eps) / max, where B is the Moller bracket. Two draws per attempt. */
double om_sample_moller(double T, double Tcut, om_rng* r) {
  double x = Tcut / T;
  double g = T / OM_ME + 1.0;
  double g2 = g * g;
  double norm = 4.0 / (9.0 * g2 - 10.0 * g + 5.0);
  for (;;) {
    double u1 = om_draw(r);
    double u2 = om_draw(r);
    double eps = x / (1.0 - u1 * (1.0 - 2.0 * x));
    double om = 1.0 - eps;
    double f = (g - 1.0) * (g - 1.0) * eps * eps - (2.0 * g2 + 2.0 * g - 1.0) * eps / om
               + g2 / (om * om);
    if (u2 <= norm * f) return eps;
  }
}

/* 1/k spectrum on [kcut, T]: k = kcut (T/kcut)^u, capped at T. One draw. */
double om_sample_brems(double T, double kcut, om_rng* r) {
  double u = om_draw(r);
  double k = kcut * exp(u * log(T / kcut));
  if (k > T) k = T;
  return k;
}

void om_sample_isotropic(om_rng* r, double dir[3]) {
  double cost = 2.0 * om_draw(r) - 1.0;
  double phi = 2.0 * OM_PI * om_draw(r);
  double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  dir[0] = sint * cos(phi);
  dir[1] = sint * sin(phi);
  dir[2] = cost;
}

/* Rotate direction u by polar cosine cost and azimuth phi. Frame: if
 * |u_z| < 1 - 1e-10, e1 = (u x z)/|u x z| and e2 = u x e1; otherwise e1 = x
 * and e2 = (u x x)/|u x x|. Result renormalised. */
void om_rotate(const double u[3], double cost, double phi, double out[3]) {
  double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  double cp = cos(phi), sp = sin(phi);
  double e1[3], e2[3];
  if (fabs(u[2]) < 1.0 - 1e-10) {
    double n = sqrt(u[0] * u[0] + u[1] * u[1]);
    e1[0] = u[1] / n;
    e1[1] = -u[0] / n;
    e1[2] = 0.0;
    e2[0] = u[2] * u[0] / n;
    e2[1] = u[2] * u[1] / n;
    e2[2] = -n;
  } else {
    double n = sqrt(u[2] * u[2] + u[1] * u[1]);
    e1[0] = 1.0;
    e1[1] = 0.0;
    e1[2] = 0.0;
    e2[0] = 0.0;
    e2[1] = u[2] / n;
    e2[2] = -u[1] / n;
  }
  double v[3];
  for (int i = 0; i < 3; ++i) v[i] = cost * u[i] + sint * (cp * e1[i] + sp * e2[i]);
  double inv = 1.0 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 3; ++i) out[i] = v[i] * inv;
}

/* Signed curvature kappa [1/cm] of a charged track in B along z: the
 * transverse direction turns by phi = kappa * s over path length s. */
double om_curvature(int ptype, double E, double Bz) {
  double q = (ptype == OM_ELECTRON) ? -1.0 : 1.0;
  double p = sqrt(E * (E + 2.0 * OM_ME));
  return q * Bz * OM_FIELD_K / p;
}

/* Exact helix: du/ds = kappa (u x z). With phi = kappa s and
 * 1 - cos(phi) = 2 sin^2(phi/2):
 *   x += (ux sin(phi) + uy (1 - cos(phi))) / kappa
 *   y += (uy sin(phi) - ux (1 - cos(phi))) / kappa
 *   z += uz s,  (ux, uy) rotated by -phi. */
void om_helix_move(double kappa, double s, double pos[3], double dir[3]) {
  double phi = kappa * s;
  double hs = sin(0.5 * phi), hc = cos(0.5 * phi);
  double sphi = 2.0 * hs * hc;
  double omc = 2.0 * hs * hs;
  double cphi = 1.0 - omc;
  double ux = dir[0], uy = dir[1];
  pos[0] += (ux * sphi + uy * omc) / kappa;
  pos[1] += (uy * sphi - ux * omc) / kappa;
  pos[2] += dir[2] * s;
  dir[0] = ux * cphi + uy * sphi;
  dir[1] = uy * cphi - ux * sphi;
}

/* Numerical field propagation (paper Sec. 3.3: the curved path is divided
 * into substeps, each found by numerical integration of the equation of
 * motion). A field step of length s takes n = ceil(s |kappa| / 0.1) equal
 * substeps, i.e. at most 0.1 rad of turn each (at least one). */
int om_rk_substeps(double kappa, double s) {
  double a = s * fabs(kappa) / OM_RK_TURN;
  int n = (int)ceil(a);
  return n < 1 ? 1 : n;
}

/* Classical fourth-order Runge-Kutta for the transverse motion in B along z,
 * dx/ds = ux, dy/ds = uy, dux/ds = kappa uy, duy/ds = -kappa ux, over n equal
 * substeps of length s / n; z advances by uz s exactly (uz is constant). The
 * transverse direction is rescaled at the end to its length at the start
 * (Runge-Kutta does not keep it). */
void om_rk_move(double kappa, double s, int n, double pos[3], double dir[3]) {
  double x = pos[0], y = pos[1], ux = dir[0], uy = dir[1];
  const double q0 = ux * ux + uy * uy;
  const double h = s / n;
  for (int i = 0; i < n; ++i) {
    double c1 = kappa * uy, d1 = -kappa * ux;
    double ux2 = ux + 0.5 * h * c1, uy2 = uy + 0.5 * h * d1;
    double c2 = kappa * uy2, d2 = -kappa * ux2;
    double ux3 = ux + 0.5 * h * c2, uy3 = uy + 0.5 * h * d2;
    double c3 = kappa * uy3, d3 = -kappa * ux3;
    double ux4 = ux + h * c3, uy4 = uy + h * d3;
    double c4 = kappa * uy4, d4 = -kappa * ux4;
    x += h / 6.0 * (ux + 2.0 * ux2 + 2.0 * ux3 + ux4);
    y += h / 6.0 * (uy + 2.0 * uy2 + 2.0 * uy3 + uy4);
    ux += h / 6.0 * (c1 + 2.0 * c2 + 2.0 * c3 + c4);
    uy += h / 6.0 * (d1 + 2.0 * d2 + 2.0 * d3 + d4);
  }
  double q = ux * ux + uy * uy;
  if (q > 0.0) {
    double f = sqrt(q0 / q);
    ux *= f;
    uy *= f;
  }
  pos[0] = x;
  pos[1] = y;
  pos[2] += dir[2] * s;
  dir[0] = ux;
  dir[1] = uy;
}

/* Smallest turn angle t in [0, 2 pi) with sin(sigma t + beta) = d. */
static double first_turn(double d, double beta, double sigma) {
  double a1 = asin(d);
  double a2 = OM_PI - a1;
  double best = INFINITY;
  double cand[2] = {a1, a2};
  for (int i = 0; i < 2; ++i) {
    double t = fmod(sigma * (cand[i] - beta), 2.0 * OM_PI);
    if (t < 0.0) t += 2.0 * OM_PI;
    if (t < best) best = t;
  }
  return best;
}

/* Path length to the first crossing of the side planes |x| = hx, |y| = hy by
 * the helix (circle-line intersection in the transverse plane); INFINITY if
 * the circle stays inside. */
double om_helix_side_distance(double kappa, const double pos[3], const double dir[3],
                              double hx, double hy, int* hit) {
  double ux = dir[0], uy = dir[1];
  double A = sqrt(ux * ux + uy * uy);
  *hit = 0;
  if (A == 0.0) return INFINITY;
  double K = fabs(kappa);
  double sigma = kappa > 0.0 ? 1.0 : -1.0;
  double xc = pos[0] + uy / kappa;
  double yc = pos[1] - ux / kappa;
  double rho = A / K;
  if (xc + rho < hx && xc - rho > -hx && yc + rho < hy && yc - rho > -hy) return INFINITY;
  double tmin = INFINITY;
  double planes[2] = {hx, -hx};
  for (int i = 0; i < 2; ++i) {
    double d = kappa * (planes[i] - xc) / A;
    if (fabs(d) <= 1.0) {
      double t = first_turn(d, atan2(-uy, ux), sigma);
      if (t < tmin) tmin = t;
    }
  }
  double yplanes[2] = {hy, -hy};
  for (int i = 0; i < 2; ++i) {
    double d = kappa * (yplanes[i] - yc) / A;
    if (fabs(d) <= 1.0) {
      double t = first_turn(d, atan2(ux, uy), sigma);
      if (t < tmin) tmin = t;
    }
  }
  if (tmin == INFINITY) return INFINITY;
  *hit = 1;
  return tmin / K;
}
