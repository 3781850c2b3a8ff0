/*
 * History-based transport of the oracle -- TEST INFRASTRUCTURE.
 *
 * Sec. 2 of the paper contrasts two ways to organise Monte Carlo transport:
 * following each particle from birth through boundary crossings and
 * interactions to its end (history based, the CPU way), versus applying one
 * action at a time to an array of tracks (step based, the GPU way). This file
 * is the first: a plain loop over primaries, a depth-first stack of tracks
 * per primary, and one full step (step limit, propagation, interaction) at a
 * time per track. The CUDA path implements the second; both produce the same
 * per-history results because each track's random stream depends only on
 * (seed, event, track id, draw index).
 *
 * One step of a track:
 *   1. if its number of mean free paths is unset, n_mfp = -ln u;
 *   2. total macroscopic cross-section mu from tables linear in ln E;
 *      s_int = n_mfp / mu;
 *   3. charged with continuous loss: range R(E); range step limit
 *      s_rng = R if R <= 0.1 cm else 0.2 R + 0.1 (1 - 0.2)(2 - 0.1/R);
 *   4. distance to the layer's z-planes and the side planes (straight line, or
 *      exact helix for charged tracks in a field);
 *   5. s = min, ties resolved boundary > range > interaction;
 *      n_mfp -= s mu;
 *   6. move; charged: E_post = R^-1(R(E) - s), the loss deposited in the
 *      layer the step was taken in;
 *   7. boundary: next layer, or escape (energy tallied as escaped);
 *      E_post below the tracking cut: deposited, track ends;
 *      interaction: process chosen with u mu over the cumulative
 *      cross-sections at the pre-step energy, kinematics at E_post;
 *      kinematically closed (Moller T <= 2 Tcut, brems T <= k_cut): null
 *      collision. Survivors get a fresh n_mfp at their next step.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OM_ME 0.51099895
#define OM_PI 3.14159265358979323846
#define OM_NA 6.02214076e23

/* photon model constants (water reference) */
#define NE_WATER 3.343e23
#define Z_WATER 7.42
#define PE_MU0 0.15
#define PE_E0 0.030
#define PE_POWER -3.5
#define PAIR_MU0 0.0096
#define PAIR_THRESHOLD 1.022

/* energy grid */
#define GRID_EMIN 1e-3
#define GRID_EMAX 1e4

/* range step function */
#define ALPHA_R 0.2
#define FINAL_R 0.1

typedef struct {
  double ne, Z, X0, I;
  double f_pe, f_pair;
  double table[OM_NCOL][OM_NGRID];
} om_mat;

struct om_world {
  int n_mat;
  om_mat* mats;
  int L;           /* total layers */
  double* zb;      /* L + 1 boundaries */
  int* layer_mat;  /* L */
  double hx, hy, Bz;
  int field_substep_cap;
  double cut_track, cut_moller, cut_brems;
  int processes;
  int tally_mode, nbins;
  double zscale;
  uint32_t seed;
  double lnEmin, dl, inv_dl;
};

/* ------------------------------------------------------------------ world */

static void build_tables(om_world* w, om_mat* m) {
  double gx[16], gw[16];
  om_gauss_legendre(16, gx, gw);
  int P = w->processes;
  for (int i = 0; i < OM_NGRID; ++i) {
    double lnE = w->lnEmin + i * w->dl;
    double E = exp(lnE);
    m->table[OM_COL_COMPTON][i] = (P & OM_PROC_COMPTON) ? m->ne * om_sigma_kn(E) : 0.0;
    m->table[OM_COL_PE][i] = (P & OM_PROC_PE) ? m->f_pe * PE_MU0 * pow(E / PE_E0, PE_POWER) : 0.0;
    m->table[OM_COL_PAIR][i] =
        ((P & OM_PROC_PAIR) && E > PAIR_THRESHOLD) ? m->f_pair * PAIR_MU0 * log(E / PAIR_THRESHOLD) : 0.0;
    m->table[OM_COL_MOLLER][i] = (P & OM_PROC_MOLLER) ? m->ne * om_sigma_moller(E, w->cut_moller) : 0.0;
    m->table[OM_COL_BREMS][i] =
        ((P & OM_PROC_BREMS) && E > w->cut_brems) ? log(E / w->cut_brems) / m->X0 : 0.0;
    m->table[OM_COL_DEDX][i] = 0.0;
    m->table[OM_COL_RANGE][i] = 0.0;
  }
  if (!(P & OM_PROC_ELOSS)) return;
  /* S(E) = restricted collision + restricted radiative loss */
  for (int i = 0; i < OM_NGRID; ++i) {
    double E = exp(w->lnEmin + i * w->dl);
    double rad = (E < w->cut_brems ? E : w->cut_brems) / m->X0;
    m->table[OM_COL_DEDX][i] = om_dedx_collision(E, w->cut_moller, m->ne, m->I) + rad;
  }
  /* R(E_0) = E_0 / (2 S(E_0)); R(E_{i+1}) = R(E_i) + int dE / S over the bin,
   * 16-point Gauss-Legendre in ln E with S from its closed form */
  double* R = m->table[OM_COL_RANGE];
  R[0] = exp(w->lnEmin) / (2.0 * m->table[OM_COL_DEDX][0]);
  for (int i = 0; i + 1 < OM_NGRID; ++i) {
    double a = w->lnEmin + i * w->dl;
    double sum = 0.0;
    for (int j = 0; j < 16; ++j) {
      double t = a + 0.5 * (1.0 + gx[j]) * w->dl;
      double E = exp(t);
      double rad = (E < w->cut_brems ? E : w->cut_brems) / m->X0;
      double S = om_dedx_collision(E, w->cut_moller, m->ne, m->I) + rad;
      sum += gw[j] * E / S;
    }
    R[i + 1] = R[i] + 0.5 * w->dl * sum;
  }
}

om_world* om_world_create(const om_problem* p, char* err, int errlen) {
  if (p->n_materials <= 0 || p->n_layers <= 0 || p->n_periods <= 0) {
    snprintf(err, errlen, "empty geometry");
    return NULL;
  }
  om_world* w = (om_world*)calloc(1, sizeof(om_world));
  w->n_mat = p->n_materials;
  w->mats = (om_mat*)calloc((size_t)w->n_mat, sizeof(om_mat));
  w->L = p->n_layers * p->n_periods;
  w->zb = (double*)calloc((size_t)w->L + 1, sizeof(double));
  w->layer_mat = (int*)calloc((size_t)w->L, sizeof(int));
  w->zb[0] = 0.0;
  for (int i = 0; i < w->L; ++i) {
    int j = i % p->n_layers;
    w->layer_mat[i] = p->layer_material[j];
    w->zb[i + 1] = w->zb[i] + p->layer_thickness[j];
  }
  w->hx = p->half_x;
  w->hy = p->half_y;
  w->Bz = p->Bz;
  w->field_substep_cap = p->field_substep_cap > 0 ? p->field_substep_cap : 0;
  w->cut_track = p->cut_track;
  w->cut_moller = p->cut_moller;
  w->cut_brems = p->cut_brems;
  w->processes = p->processes;
  w->tally_mode = p->tally_mode;
  w->nbins = (p->tally_mode == OM_TALLY_LAYERS) ? w->L : p->n_zbins;
  w->zscale = (double)w->nbins / (w->zb[w->L] - w->zb[0]);
  w->seed = p->seed;
  w->lnEmin = log(GRID_EMIN);
  w->dl = log(GRID_EMAX / GRID_EMIN) / (OM_NGRID - 1);
  w->inv_dl = 1.0 / w->dl;
  for (int m = 0; m < w->n_mat; ++m) {
    const om_material* src = &p->materials[m];
    om_mat* dst = &w->mats[m];
    dst->ne = om_electron_density(src);
    dst->Z = src->Z;
    dst->X0 = src->X0;
    dst->I = src->I;
    double zr = src->Z / Z_WATER;
    dst->f_pe = dst->ne / NE_WATER * zr * zr * zr;
    dst->f_pair = dst->ne / NE_WATER * zr;
    build_tables(w, dst);
  }
  return w;
}

void om_world_destroy(om_world* w) {
  if (!w) return;
  free(w->mats);
  free(w->zb);
  free(w->layer_mat);
  free(w);
}

int om_world_nbins(const om_world* w) { return w->nbins; }
int om_world_nlayers(const om_world* w) { return w->L; }
void om_world_boundaries(const om_world* w, double* zb) { memcpy(zb, w->zb, sizeof(double) * (w->L + 1)); }

void om_world_table(const om_world* w, int mat, int col, double* out) {
  memcpy(out, w->mats[mat].table[col], sizeof(double) * OM_NGRID);
}

void om_world_grid(const om_world* w, double* lnE) {
  for (int i = 0; i < OM_NGRID; ++i) lnE[i] = w->lnEmin + i * w->dl;
}

/* Grid coordinate x = (ln E - ln E_min) / dl; bin = floor(x) clamped to
 * [0, n-2]; fraction x - bin (may fall outside [0, 1] at the grid ends). */
static void grid_coord(const om_world* w, double E, int* bin, double* frac) {
  double x = (log(E) - w->lnEmin) * w->inv_dl;
  int b = (int)floor(x);
  if (b < 0) b = 0;
  if (b > OM_NGRID - 2) b = OM_NGRID - 2;
  *bin = b;
  *frac = x - b;
}

static double interp(const double* t, int b, double f) { return t[b] + f * (t[b + 1] - t[b]); }

double om_world_lookup(const om_world* w, int mat, int col, double E) {
  int b;
  double f;
  grid_coord(w, E, &b, &f);
  return interp(w->mats[mat].table[col], b, f);
}

/* Exact inverse of the range interpolation: the largest bin i <= n-2 with
 * R_i <= r, then ln E linear in R within it. r at or below R_0: stopped. */
static double inv_range(const om_world* w, const double* R, double r) {
  if (r <= R[0]) return 0.0;
  int lo = 0, hi = OM_NGRID - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (R[mid] <= r)
      lo = mid;
    else
      hi = mid;
  }
  double lnE = w->lnEmin + lo * w->dl + (r - R[lo]) / (R[lo + 1] - R[lo]) * w->dl;
  return exp(lnE);
}

double om_world_inv_range(const om_world* w, int mat, double r) {
  return inv_range(w, w->mats[mat].table[OM_COL_RANGE], r);
}

int om_world_initial_layer(const om_world* w, double z, double uz) {
  int L = w->L;
  if (z >= w->zb[L]) return L - 1;
  int i = 0;
  while (i < L - 1 && !(z < w->zb[i + 1])) ++i;
  if (z == w->zb[i] && uz < 0.0 && i > 0) --i;
  return i;
}

/* Cross-sections of the particle at E in material mat, in the fixed process
 * order (photon: Compton, photoelectric, pair; electron: Moller, brems). The
 * pair cross-section is exactly zero at or below 1.022 MeV whatever the
 * interpolation across the threshold bin gives. Returns the count. */
static int cross_sections(const om_world* w, int mat, int ptype, double E, double mu[3]) {
  int b;
  double f;
  grid_coord(w, E, &b, &f);
  const om_mat* m = &w->mats[mat];
  if (ptype == OM_GAMMA) {
    mu[0] = interp(m->table[OM_COL_COMPTON], b, f);
    mu[1] = interp(m->table[OM_COL_PE], b, f);
    mu[2] = (E > PAIR_THRESHOLD) ? interp(m->table[OM_COL_PAIR], b, f) : 0.0;
    return 3;
  }
  mu[0] = interp(m->table[OM_COL_MOLLER], b, f);
  mu[1] = interp(m->table[OM_COL_BREMS], b, f);
  return 2;
}

/* Process selection: the first i with u * mu < mu_1 + ... + mu_i; if rounding
 * leaves none, the last process with a nonzero cross-section. */
static int select_from(const double* mu, int n, double mu_tot, double u) {
  double target = u * mu_tot;
  double acc = 0.0;
  int last = -1;
  for (int i = 0; i < n; ++i) {
    acc += mu[i];
    if (mu[i] > 0.0) last = i;
    if (target < acc) return i;
  }
  return last;
}

int om_select_process(const om_world* w, int mat, int ptype, double E, double u) {
  double mu[3];
  int n = cross_sections(w, mat, ptype, E, mu);
  double tot = 0.0;
  for (int i = 0; i < n; ++i) tot += mu[i];
  int i = select_from(mu, n, tot, u);
  if (i < 0) return -1;
  return (ptype == OM_GAMMA) ? i : OM_SEL_MOLLER + i;
}

/* -------------------------------------------------------------- transport */

typedef struct {
  om_track* data;
  size_t n, cap;
} track_stack;

static void stack_push(track_stack* s, const om_track* t) {
  if (s->n == s->cap) {
    s->cap = s->cap ? 2 * s->cap : 256;
    s->data = (om_track*)realloc(s->data, s->cap * sizeof(om_track));
  }
  s->data[s->n++] = *t;
}

typedef struct {
  double* edep;       /* nbins, may be NULL */
  double edep_total;
  double escaped;
  uint64_t steps, secondaries;
  double path;
  track_stack* stack; /* NULL: secondaries are counted, not kept */
} tally;

static int tally_bin(const om_world* w, int layer, double z) {
  if (w->tally_mode == OM_TALLY_LAYERS) return layer;
  int b = (int)floor((z - w->zb[0]) * w->zscale);
  if (b < 0) b = 0;
  if (b > w->nbins - 1) b = w->nbins - 1;
  return b;
}

static void deposit(const om_world* w, tally* tl, int layer, double z, double e) {
  tl->edep_total += e;
  if (tl->edep) tl->edep[tally_bin(w, layer, z)] += e;
}

static void push_secondary(const om_world* w, tally* tl, om_rng* r, const om_track* parent,
                           int ptype, double E, const double dir[3]) {
  if (E < w->cut_track) {
    deposit(w, tl, parent->layer, parent->z, E);
    return;
  }
  om_track s;
  s.E = E;
  s.x = parent->x;
  s.y = parent->y;
  s.z = parent->z;
  s.ux = dir[0];
  s.uy = dir[1];
  s.uz = dir[2];
  s.nmfp = -1.0;
  s.ptype = ptype;
  s.layer = parent->layer;
  s.tid = om_draw_raw(r);
  s.ctr = 0;
  tl->secondaries += 1;
  if (tl->stack) stack_push(tl->stack, &s);
}

enum { GEO_NONE = 0, GEO_ZUP, GEO_ZDOWN, GEO_SIDE };
enum { ACT_GEOM = 0, ACT_RANGE, ACT_INTERACT, ACT_TRAPPED, ACT_FIELD };

/* One step of one track. Returns 0 when the track ends, 1 when it lives on,
 * and sets *escaped_flag when it left the world. */
static int step_track(const om_world* w, uint32_t event, om_track* t, tally* tl, int* escaped_flag) {
  om_rng r = {w->seed, event, t->tid, t->ctr};
  *escaped_flag = 0;
  if (t->nmfp < 0.0) t->nmfp = -log(om_draw(&r));

  int mat = w->layer_mat[t->layer];
  double mu[3];
  int nproc = cross_sections(w, mat, t->ptype, t->E, mu);
  double mu_tot = 0.0;
  for (int i = 0; i < nproc; ++i) mu_tot += mu[i];
  double s_int = (mu_tot > 0.0) ? t->nmfp / mu_tot : INFINITY;

  int charged = (t->ptype != OM_GAMMA);
  int eloss = charged && (w->processes & OM_PROC_ELOSS);
  double R = 0.0, s_rng = INFINITY;
  if (eloss) {
    int b;
    double f;
    grid_coord(w, t->E, &b, &f);
    R = interp(w->mats[mat].table[OM_COL_RANGE], b, f);
    s_rng = (R <= FINAL_R) ? R : ALPHA_R * R + FINAL_R * (1.0 - ALPHA_R) * (2.0 - FINAL_R / R);
  }

  /* geometry: z-planes (exact along the helix too, u_z is constant) */
  int helix = charged && (w->Bz != 0.0);
  double kappa = helix ? om_curvature(t->ptype, t->E, w->Bz) : 0.0;
  double s_geo = INFINITY;
  int geo = GEO_NONE;
  if (t->uz > 0.0) {
    s_geo = (w->zb[t->layer + 1] - t->z) / t->uz;
    geo = GEO_ZUP;
  } else if (t->uz < 0.0) {
    s_geo = (w->zb[t->layer] - t->z) / t->uz;
    geo = GEO_ZDOWN;
  }
  double s_side = INFINITY;
  if (helix) {
    double pos[3] = {t->x, t->y, t->z}, dir[3] = {t->ux, t->uy, t->uz};
    int hit;
    s_side = om_helix_side_distance(kappa, pos, dir, w->hx, w->hy, &hit);
  } else {
    if (t->ux > 0.0) s_side = fmin(s_side, (w->hx - t->x) / t->ux);
    if (t->ux < 0.0) s_side = fmin(s_side, (-w->hx - t->x) / t->ux);
    if (t->uy > 0.0) s_side = fmin(s_side, (w->hy - t->y) / t->uy);
    if (t->uy < 0.0) s_side = fmin(s_side, (-w->hy - t->y) / t->uy);
  }
  if (s_side < s_geo) {
    s_geo = s_side;
    geo = GEO_SIDE;
  }
  if (s_geo < 0.0) s_geo = 0.0;

  double s = s_geo;
  int act = ACT_GEOM;
  if (s_rng < s) {
    s = s_rng;
    act = ACT_RANGE;
  }
  if (s_int < s) {
    s = s_int;
    act = ACT_INTERACT;
  }
  if (s == INFINITY) act = ACT_TRAPPED;
  /* Runge-Kutta field propagation with a substep cap (Sec. 3.3): a step
   * needing more than `cap` substeps of 0.1 rad of turn is cut to cap of them
   * and ends without a boundary crossing or an interaction ("paused");
   * the track goes on from there at its next step. */
  const int cap = w->field_substep_cap;
  if (helix && cap > 0 && act != ACT_TRAPPED && s * fabs(kappa) > 0.1 * cap) {
    s = 0.1 * cap / fabs(kappa);
    act = ACT_FIELD;
  }

  if (act == ACT_TRAPPED) {
    /* no finite step limit (possible only with processes switched off): the
     * track ends where it is and its energy counts as deposited */
    deposit(w, tl, t->layer, t->z, t->E);
    tl->steps += 1;
    t->ctr = r.ctr;
    return 0;
  }

  t->nmfp -= s * mu_tot;

  /* propagation */
  int old_layer = t->layer;
  if (helix) {
    double pos[3] = {t->x, t->y, t->z}, dir[3] = {t->ux, t->uy, t->uz};
    if (cap > 0)
      om_rk_move(kappa, s, act == ACT_FIELD ? cap : om_rk_substeps(kappa, s), pos, dir);
    else
      om_helix_move(kappa, s, pos, dir);
    t->x = pos[0];
    t->y = pos[1];
    t->z = pos[2];
    t->ux = dir[0];
    t->uy = dir[1];
    t->uz = dir[2];
  } else {
    t->x += s * t->ux;
    t->y += s * t->uy;
    t->z += s * t->uz;
  }
  tl->steps += 1;
  tl->path += s;
  if (eloss) {
    double E_post = inv_range(w, w->mats[mat].table[OM_COL_RANGE], R - s);
    deposit(w, tl, old_layer, t->z, t->E - E_post);
    t->E = E_post;
  }

  /* post-step */
  if (act == ACT_GEOM) {
    int out = 0;
    if (geo == GEO_ZUP) {
      t->layer += 1;
      if (t->layer >= w->L) {
        out = 1;
      } else {
        t->z = w->zb[t->layer];
      }
    } else if (geo == GEO_ZDOWN) {
      t->z = w->zb[t->layer];
      t->layer -= 1;
      if (t->layer < 0) out = 1;
    } else {
      out = 1;
    }
    if (out) {
      tl->escaped += t->E;
      *escaped_flag = 1;
      t->ctr = r.ctr;
      return 0;
    }
  }
  if (t->E < w->cut_track) {
    deposit(w, tl, t->layer, t->z, t->E);
    t->ctr = r.ctr;
    return 0;
  }
  if (act != ACT_INTERACT) {
    t->ctr = r.ctr;
    return 1;
  }

  /* discrete interaction, process chosen with the pre-step cross-sections */
  int proc = select_from(mu, nproc, mu_tot, om_draw(&r));
  if (t->ptype != OM_GAMMA) proc += OM_SEL_MOLLER;
  double dir[3] = {t->ux, t->uy, t->uz};
  int alive = 1;
  switch (proc) {
    case OM_SEL_COMPTON: {
      double eps, cost;
      om_sample_compton(t->E, &r, &eps, &cost);
      double phi = 2.0 * OM_PI * om_draw(&r);
      double E1 = eps * t->E;
      deposit(w, tl, t->layer, t->z, t->E - E1);
      double nd[3];
      om_rotate(dir, cost, phi, nd);
      t->ux = nd[0];
      t->uy = nd[1];
      t->uz = nd[2];
      t->E = E1;
      break;
    }
    case OM_SEL_PE:
      deposit(w, tl, t->layer, t->z, t->E);
      alive = 0;
      break;
    case OM_SEL_PAIR: {
      deposit(w, tl, t->layer, t->z, t->E - 2.0 * OM_ME);
      double d1[3], d2[3];
      om_sample_isotropic(&r, d1);
      d2[0] = -d1[0];
      d2[1] = -d1[1];
      d2[2] = -d1[2];
      push_secondary(w, tl, &r, t, OM_GAMMA, OM_ME, d1);
      push_secondary(w, tl, &r, t, OM_GAMMA, OM_ME, d2);
      alive = 0;
      break;
    }
    case OM_SEL_MOLLER: {
      double T = t->E;
      if (T <= 2.0 * w->cut_moller) break; /* null collision */
      double eps = om_sample_moller(T, w->cut_moller, &r);
      double Td = eps * T;
      double cost = sqrt(Td * (T + 2.0 * OM_ME) / (T * (Td + 2.0 * OM_ME)));
      if (cost > 1.0) cost = 1.0;
      double phi = 2.0 * OM_PI * om_draw(&r);
      double dd[3];
      om_rotate(dir, cost, phi, dd);
      double p = sqrt(T * (T + 2.0 * OM_ME));
      double pd = sqrt(Td * (Td + 2.0 * OM_ME));
      double v[3];
      for (int i = 0; i < 3; ++i) v[i] = p * dir[i] - pd * dd[i];
      double inv = 1.0 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      t->ux = v[0] * inv;
      t->uy = v[1] * inv;
      t->uz = v[2] * inv;
      t->E = T - Td;
      push_secondary(w, tl, &r, t, OM_ELECTRON, Td, dd);
      break;
    }
    case OM_SEL_BREMS: {
      double T = t->E;
      if (T <= w->cut_brems) break; /* null collision */
      double k = om_sample_brems(T, w->cut_brems, &r);
      t->E = T - k;
      push_secondary(w, tl, &r, t, OM_GAMMA, k, dir);
      break;
    }
    default:
      break;
  }
  if (alive && t->E < w->cut_track) {
    deposit(w, tl, t->layer, t->z, t->E);
    alive = 0;
  }
  t->nmfp = -1.0;
  t->ctr = r.ctr;
  return alive;
}

static void run_primary(const om_world* w, const om_primary* p, om_history* h, double* edep,
                        track_stack* stack) {
  tally tl;
  memset(&tl, 0, sizeof(tl));
  tl.edep = edep;
  tl.stack = stack;
  stack->n = 0;
  om_track t;
  t.E = p->E;
  t.x = p->x;
  t.y = p->y;
  t.z = p->z;
  t.ux = p->ux;
  t.uy = p->uy;
  t.uz = p->uz;
  t.nmfp = -1.0;
  t.ptype = p->ptype;
  t.layer = om_world_initial_layer(w, p->z, p->uz);
  t.tid = p->tid;
  t.ctr = 0;
  stack_push(stack, &t);
  while (stack->n > 0) {
    om_track cur = stack->data[--stack->n];
    int esc;
    while (step_track(w, p->event, &cur, &tl, &esc)) {
    }
  }
  h->steps = tl.steps;
  h->secondaries = tl.secondaries;
  h->escaped = tl.escaped;
  h->path = tl.path;
}

typedef struct {
  const om_world* w;
  const om_primary* prim;
  uint64_t n;
  om_history* hist;
  double* edep;
  atomic_ullong next;
} run_job;

static void* worker(void* arg) {
  run_job* job = (run_job*)arg;
  track_stack stack = {NULL, 0, 0};
  int nb = job->w->nbins;
  for (;;) {
    uint64_t first = atomic_fetch_add(&job->next, 16);
    if (first >= job->n) break;
    uint64_t last = first + 16 < job->n ? first + 16 : job->n;
    for (uint64_t i = first; i < last; ++i) {
      run_primary(job->w, &job->prim[i], &job->hist[i], job->edep ? job->edep + i * (uint64_t)nb : NULL,
                  &stack);
    }
  }
  free(stack.data);
  return NULL;
}

int om_run(const om_world* w, const om_primary* prim, uint64_t n, int n_threads, om_history* hist,
           double* edep) {
  if (n_threads < 1) n_threads = 1;
  if (edep) memset(edep, 0, sizeof(double) * n * (uint64_t)w->nbins);
  run_job job;
  job.w = w;
  job.prim = prim;
  job.n = n;
  job.hist = hist;
  job.edep = edep;
  atomic_init(&job.next, 0);
  if (n_threads == 1) {
    worker(&job);
    return 0;
  }
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, worker, &job);
  for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
  free(th);
  return 0;
}

int om_transport_track(const om_world* w, uint32_t event, om_track* t, uint64_t max_steps, uint64_t* steps,
                       double* path, double* edep_total, double* escaped, uint64_t* n_secondaries) {
  tally tl;
  memset(&tl, 0, sizeof(tl));
  int esc = 0, status = 2;
  while (tl.steps < max_steps) {
    if (!step_track(w, event, t, &tl, &esc)) {
      status = esc ? 1 : 0;
      break;
    }
  }
  *steps = tl.steps;
  *path = tl.path;
  *edep_total = tl.edep_total;
  *escaped = tl.escaped;
  *n_secondaries = tl.secondaries;
  return status;
}
