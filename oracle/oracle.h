/*
 * CPU oracle for step-based EM Monte Carlo transport -- TEST INFRASTRUCTURE.
 *
 * This library is a plain, slow, history-based transport written to check the
 * CUDA path. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never calls it. It shares no code with
 * the CUDA path: the two meet only through the seeded workload generators,
 * which hold no transport arithmetic.
 *
 * Structure (the contrast case of Sec. 2 of the paper): each primary is
 * followed from birth to death, then its secondaries, depth first, one track
 * at a time on one CPU thread; primaries are spread over threads. Each track
 * draws random numbers from its own counter-based Philox4x32-10 stream keyed
 * by (seed, event) with the counter (track id, draw index), so every
 * per-history result is a deterministic function of (seed, event, primary)
 * and does not depend on scheduling.
 *
 * Physics (Compton, photoelectric, pair, Moller, 1/k bremsstrahlung,
 * restricted continuous loss, exact helix in a uniform field) is not defined
 * by the paper, which fixes no physics model; every definition used here is a
 * modelling choice shared with the CUDA path by specification, not by code.
 *
 * Units: MeV, cm, tesla.
 */
#ifndef CELER_ORACLE_H
#define CELER_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OM_GAMMA = 0, OM_ELECTRON = 1, OM_POSITRON = 2 };
enum {
  OM_PROC_COMPTON = 1, OM_PROC_PE = 2, OM_PROC_PAIR = 4,
  OM_PROC_MOLLER = 8, OM_PROC_BREMS = 16, OM_PROC_ELOSS = 32
};
enum { OM_TALLY_ZBINS = 0, OM_TALLY_LAYERS = 1 };
/* table columns */
enum {
  OM_COL_COMPTON = 0, OM_COL_PE, OM_COL_PAIR, OM_COL_MOLLER, OM_COL_BREMS,
  OM_COL_DEDX, OM_COL_RANGE, OM_NCOL
};
/* process indices returned by om_select_process */
enum { OM_SEL_COMPTON = 0, OM_SEL_PE = 1, OM_SEL_PAIR = 2, OM_SEL_MOLLER = 3, OM_SEL_BREMS = 4 };

#define OM_NGRID 200

typedef struct {
  double Z, A, rho, ne, X0, I;
} om_material;

typedef struct {
  int n_materials;
  const om_material* materials;
  int n_layers;               /* layers in one period */
  const int* layer_material;
  const double* layer_thickness;
  int n_periods;
  double half_x, half_y;
  double Bz;
  double cut_track, cut_moller, cut_brems;
  int processes;
  int tally_mode;
  int n_zbins;
  uint32_t seed;
  int field_substep_cap; /* 0: exact helix; > 0: Runge-Kutta substeps, at most this many per step */
} om_problem;

typedef struct {
  double E, x, y, z, ux, uy, uz;
  int32_t ptype;
  uint32_t event;
  uint64_t tid;
} om_primary;

typedef struct {
  uint64_t steps;        /* track-steps of the primary and all its descendants */
  uint64_t secondaries;  /* secondary tracks created (those above the tracking cut) */
  double escaped;        /* energy leaving the world */
  double path;           /* summed step lengths */
} om_history;

typedef struct {
  uint32_t seed, event;
  uint64_t tid;
  uint32_t ctr;
} om_rng;

typedef struct {
  double E, x, y, z, ux, uy, uz, nmfp;
  int32_t ptype, layer;
  uint64_t tid;
  uint32_t ctr;
} om_track;

typedef struct om_world om_world;

/* ---- world ---- */
om_world* om_world_create(const om_problem* p, char* err, int errlen);
void om_world_destroy(om_world* w);
int om_world_nbins(const om_world* w);
int om_world_nlayers(const om_world* w);
void om_world_boundaries(const om_world* w, double* zb /* nlayers+1 */);
void om_world_table(const om_world* w, int mat, int col, double* out /* OM_NGRID */);
double om_world_lookup(const om_world* w, int mat, int col, double E);
double om_world_inv_range(const om_world* w, int mat, double r);
void om_world_grid(const om_world* w, double* lnE /* OM_NGRID */);
int om_world_initial_layer(const om_world* w, double z, double uz);

/* ---- transport ---- */
int om_run(const om_world* w, const om_primary* prim, uint64_t n, int n_threads,
           om_history* hist /* n */, double* edep /* n * nbins */);
/* Follow one track (secondaries counted but not followed). Returns 0 = absorbed
 * or stopped, 1 = escaped, 2 = step limit reached. */
int om_transport_track(const om_world* w, uint32_t event, om_track* t, uint64_t max_steps,
                       uint64_t* steps, double* path, double* edep_total, double* escaped,
                       uint64_t* n_secondaries);

/* ---- random numbers ---- */
void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t om_raw_word(uint32_t seed, uint32_t event, uint64_t tid, uint32_t index);
double om_uniform(uint64_t w);
double om_draw(om_rng* r);
uint64_t om_draw_raw(om_rng* r);

/* ---- physics ---- */
double om_sigma_kn(double E);
double om_sigma_moller(double T, double Tcut);
double om_dedx_collision(double T, double Tcut, double ne, double I);
double om_electron_density(const om_material* m);
void om_gauss_legendre(int n, double* x, double* w);
void om_sample_compton(double E, om_rng* r, double* eps, double* cost);
double om_sample_moller(double T, double Tcut, om_rng* r);
double om_sample_brems(double T, double kcut, om_rng* r);
void om_sample_isotropic(om_rng* r, double dir[3]);
void om_rotate(const double u[3], double cost, double phi, double out[3]);
void om_helix_move(double kappa, double s, double pos[3], double dir[3]);
int om_rk_substeps(double kappa, double s);
void om_rk_move(double kappa, double s, int n, double pos[3], double dir[3]);
double om_helix_side_distance(double kappa, const double pos[3], const double dir[3],
                              double hx, double hy, int* hit);
double om_curvature(int ptype, double E, double Bz);
int om_select_process(const om_world* w, int mat, int ptype, double E, double u);

#ifdef __cplusplus
}
#endif
#endif
