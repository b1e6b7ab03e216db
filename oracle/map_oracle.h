/*
 * map_oracle.h -- plain FP64 CPU oracle of the EGLM-MHD block step (TEST INFRASTRUCTURE).
 *
 * This is the slow, obviously-correct restatement of the method of Jiang, Fang & Chen,
 * "A new MHD code with adaptive mesh refinement and parallelization for astrophysics"
 * (arXiv:1204.5849).  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Data convention: 9 variables (rho, rho v, B, e, psi), FP64, one array per block of
 * shape [9][NZ][NY][NX] with NX = NY = nb + 4, NZ = nb + 4 in 3D and 1 in 2D (two ghost
 * layers).  Leaf interiors cross this API as [9][nz][nb][nb] with nz = nb (3D) or 1 (2D).
 *
 * Parity unpinned (no value printed by the paper or fixed by a closed form or invariant
 * reaches them on their own): which speeds the two neighbouring g terms inside MMC's limiter
 * ratio use where the speed varies (the face speeds of h and of the face's own g terms are
 * pinned by closed forms, the ratio's structure by Sweby's form at constant speed, and the
 * speeds' locality and symmetry by invariants).
 */
#ifndef MAP_ORACLE_H
#define MAP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double gamma, c_cfl;
  int ch_mode;      /* 0: c_h = alpha_g, 1: c_h = c_cfl*min dx/dt (literal), 2: fixed */
  double ch;        /* fixed c_h */
  int cp_mode;      /* 0: c_p from c_d, 1: fixed c_p */
  double c_d, cp;
  double eta;       /* uniform resistivity */
  int eglm;         /* 1: EGLM non-conservative sources on; 0: GLM */
  int scheme;       /* 0 MMC, 1 LF, 2 WENO */
  int limiter;      /* 0 minmod, 1 van Leer, 2 literal Roe form, 3 phi = 1, 4 phi = 0 (2-4: MMC only) */
  double dt_override; /* > 0: use this dt */
  int reflux;       /* 1: coarse fluxes at coarse/fine faces replaced by the fine ones */
  int riemann;      /* interface flux of LF and WENO: 0 f_m (Lax-Friedrichs), 1 HLLC, 2 HLLD */
  int conduction;   /* thermal conduction: 0 off, 1 isotropic, 2 along B (kappa0 T^(5/2)) */
  double kappa0;
  int subcycle;     /* 1: conduction subcycled within each step; 0: it bounds dt */
  double grad_t_max;/* > 0: face temperature gradients clipped to +-grad_t_max */
} orc_params;

typedef struct {
  int nbase[3];
  double lo[3], hi[3];
  int bc[3][2];     /* 0 periodic, 1 outflow (zero gradient) */
} orc_problem;

typedef struct {
  int var_mask;     /* 1 rho, 2 p, 4 |J| */
  double thr, coarsen_thr;
  double bias, filter; /* B = 0.6, F = 0.05 */
  double eps_rho, eps_p, eps_b;
  double ratio, xi; /* R, xi */
  int max_level;
} orc_refine;

typedef struct orc_mesh orc_mesh;

/* leaves: n x 5 ints (problem, level, i, j, k).  Returns NULL and sets *err on invalid input. */
orc_mesh* orc_create(int ndim, int nb, int nprob, const orc_problem* probs, int nleaves,
                     const int* leaves, int* err);
void orc_destroy(orc_mesh* m);
int orc_nleaves(const orc_mesh* m);
int orc_set_leaf(orc_mesh* m, int leaf, const double* interior);
int orc_get_leaf(const orc_mesh* m, int leaf, double* interior);
int orc_get_leaf_ghosted(const orc_mesh* m, int leaf, double* padded);
int orc_fill_ghosts(orc_mesh* m);
int orc_cfl(orc_mesh* m, const orc_params* p, double* dt_out);
int orc_get_speeds(const orc_mesh* m, double* out /* [nprob][5]: dt ch cp damp alpha_g */);
int orc_step(orc_mesh* m, const orc_params* p);
/* Thermal conduction alone over dt (Sec. 3.6), with its own time step and subcycle. */
int orc_conduct(orc_mesh* m, const orc_params* p, double dt);
/* Conduction time step per problem of the last reduction (orc_cfl or orc_conduct). */
int orc_get_dtc(const orc_mesh* m, double* out);
int orc_flags(orc_mesh* m, const orc_params* p, const orc_refine* r, signed char* flags,
              double* est_max);
int orc_conservation(const orc_mesh* m, double* sums);
orc_mesh* orc_regrid(orc_mesh* m, int nleaves, const int* leaves, int* err);

/* Floating-point operation counters of the counting build (liboracle_flops.so): out3 =
 * {ring-cell work, per-face work counted from both sides, interior-cell work}; reset = 1
 * zeroes them.  Returns 1 in the counting build, 0 (and zeros) in the normal one. */
int orc_flop_counts(unsigned long long* out3, int reset);

/* one MMC/LF step of a single ghost-filled block with given dt, c_h and damping factor */
int orc_block_step(int ndim, int nb, const orc_params* p, const double* dx, double dt,
                   double ch, double damp, const double* padded_in, double* interior_out);

/* point-wise pieces, exposed for the pins */
void orc_flux(int d, const double* w, double gamma, double ch, double* f);
double orc_alpha(int d, const double* w, double gamma);
void orc_hllc_flux(int d, const double* a, const double* b, double gamma, double ch, double* f);
void orc_hlld_flux(int d, const double* a, const double* b, double gamma, double ch, double* f);
void orc_lf_flux(int d, const double* a, const double* b, double gamma, double ch, double* f);
double orc_limiter(int kind, double a, double b);
void orc_weno_faces(double um, double u0, double up, double* minus_right, double* plus_left);
double orc_prolong_1d(double um, double u0, double up, int odd);

#ifdef __cplusplus
}
#endif
#endif
