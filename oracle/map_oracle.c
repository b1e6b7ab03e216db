/*
 * map_oracle.c -- plain FP64 CPU oracle of the EGLM-MHD block step.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg load this library.  It shares no code with the CUDA library and is written for
 * readability: every quantity is recomputed where the paper's formula uses it, with no
 * blocking, fusion or caching beyond temporary arrays for a stage state.
 *
 * Sections and equations cited are those of Jiang, Fang & Chen (arXiv:1204.5849):
 *   Sec. 2  EGLM-MHD equations (MHD-1 .. MHD-5), total energy, c_h and c_p.
 *   Sec. 3  Equ:basic update; 3.1 MMC; 3.2 LF (limiter1/2, minmod, Equ:LFFlux);
 *           3.3 WENO + TVD Runge-Kutta; 3.5 resistivity; 3.7 multi-D and the CFL step.
 *   Sec. 4.3 boundary conditions (restriction, same-level exchange, prolongation formula).
 *   Sec. 4.5 regrid error estimator.
 * Readings where the paper is silent or garbled are stated at the place they are used.
 *
 * MMC's face speeds (Sec. 3.1, "the relevant range of u and u~"; here one u-speed and one
 * u~-speed per face, from its two cells, used for every split term of that face's flux) are
 * pinned where the mathematics fixes them, on states whose speed varies along every axis:
 * with phi = 0 the scheme is Rusanov's with the speed of the face's two cells, and with
 * phi = 1 its flux is a closed four-flux form whose alpha~ comes from u~_i, u~_{i+1}.  With a
 * constant speed it is Sweby's flux-limited Lax-Wendroff (minmod, van Leer, the literal
 * phi(r)).  Locality is pinned too: one step changes nothing beyond two cells of a perturbed
 * cell, and the mirror and transpose symmetries exclude one-sided speeds.
 * Long runs on a static two-level mesh are pinned by conservation, by an error between the
 * all-coarse and all-fine meshes' and by the convergence order; a long run that regrids as
 * it goes by conservation through every regrid and an error within 25 % of the mesh refined
 * everywhere.
 * Parity unpinned: which speeds the two neighbouring g terms inside the limiter's ratio use
 * when the speed varies (here the face's own; a reading the paper leaves open).
 */
#include "map_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Flop counting (built only into the separate counting library, see build.py): each
 * routine adds the floating-point operations it executes (+ - * / sqrt exp log, one each;
 * comparisons, fabs, min/max and negation are not counted) to one of three counters:
 * 0 per-cell work on the one-cell ring around the interior (slopes, predictor),
 * 1 per-face work, which the update loops evaluate once from each side of a face,
 * 2 per-interior-cell work (update, sources, Runge-Kutta combination, damping).
 * The predictor of MMC is counted as executed (each face from both sides) under 0. */
#ifdef ORACLE_COUNT_FLOPS
static unsigned long long g_flops[4];   /* [3]: outside the step (checks, ghost fill) */
static int g_flcat = 2;
#define FLOPS(n) (g_flops[g_flcat] += (unsigned long long)(n))
#define FLCAT(c) (g_flcat = (c))
#else
#define FLOPS(n) ((void)0)
#define FLCAT(c) ((void)0)
#endif

int orc_flop_counts(unsigned long long* out3, int reset) {
#ifdef ORACLE_COUNT_FLOPS
  for (int q = 0; q < 3; ++q) {
    out3[q] = g_flops[q];
    if (reset) g_flops[q] = 0;
  }
  return 1;
#else
  for (int q = 0; q < 3; ++q) out3[q] = 0;
  (void)reset;
  return 0;
#endif
}

#define NV 9
enum { RHO = 0, MX = 1, MY = 2, MZ = 3, BX = 4, BY = 5, BZ = 6, EN = 7, PSI = 8 };
#define NG 2

typedef struct {
  int problem, level, ijk[3];
  int leaf;       /* caller's leaf index, or -1 for an internal (parent) block */
  int parent;
  int child[8];
  double* u;      /* [NV][NZ][NY][NX] */
  double* u1;     /* second state (WENO stage) */
} oblk;

struct orc_mesh {
  int ndim, nb, NX, NY, NZ, S;
  int nprob;
  orc_problem* probs;
  int nblocks;
  oblk* b;
  int nleaves;
  int* leaf_block;
  int maxlev;
  int* order; /* blocks sorted by key */
  double *dt, *ch, *cp, *damp, *alpha_g;
  double* dtc;    /* thermal-conduction time step of the last CFL reduction */
  int have_dt;
};

/* ------------------------------------------------------------------------------------ */
/* Physics: primitives, fluxes, fast speed (Sec. 2 and Sec. 3).                           */

static double pressure(const double* w, double gamma) {
  /* e = p/(gamma-1) + rho v^2/2 + B^2/2  (Sec. 2)  =>  p = (gamma-1)(e - m^2/(2 rho) - B^2/2) */
  double m2 = w[MX] * w[MX] + w[MY] * w[MY] + w[MZ] * w[MZ];
  double b2 = w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ];
  FLOPS(17);
  return (gamma - 1.0) * (w[EN] - 0.5 * m2 / w[RHO] - 0.5 * b2);
}

/* Flux of the EGLM-MHD system in direction d (eqs. MHD-1..MHD-5 without sources). */
void orc_flux(int d, const double* w, double gamma, double ch, double* f) {
  double rho = w[RHO];
  double v[3] = {w[MX] / rho, w[MY] / rho, w[MZ] / rho};
  double B[3] = {w[BX], w[BY], w[BZ]};
  double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  double p = pressure(w, gamma);
  double pt = p + 0.5 * b2;
  double vb = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  f[RHO] = w[MX + d];
  for (int j = 0; j < 3; ++j) {
    f[MX + j] = w[MX + d] * v[j] - B[d] * B[j];
    if (j == d) f[MX + j] += pt;
  }
  for (int j = 0; j < 3; ++j) f[BX + j] = (j == d) ? w[PSI] : v[d] * B[j] - B[d] * v[j];
  f[EN] = v[d] * (w[EN] + pt) - B[d] * vb;
  f[PSI] = ch * ch * B[d];
  FLOPS(37);
}

/* Local maximum speed in direction d: |v_d| + fast magnetosonic speed (reading of the
 * "local maximum eigenvalue", Sec. 3.1/3.2, which the paper does not write out).
 * The pressure is clamped at zero inside this formula only. */
double orc_alpha(int d, const double* w, double gamma) {
  double rho = w[RHO];
  double p = pressure(w, gamma);
  if (p < 0.0) p = 0.0;
  double a2 = gamma * p / rho;
  double b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) / rho;
  double bd2 = w[BX + d] * w[BX + d] / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bd2;
  if (disc < 0.0) disc = 0.0;
  double cf = sqrt(0.5 * (s + sqrt(disc)));
  FLOPS(21);
  return fabs(w[MX + d] / rho) + cf;
}

/* Dissipation speed of component v in direction d: the (B_d, psi) pair is the linear
 * GLM subsystem with speeds +-c_h; every other component uses the local MHD speed. */
static double comp_speed(int v, int d, double alpha, double ch) {
  return (v == BX + d || v == PSI) ? ch : alpha;
}

/* Lax-Friedrichs flux f_m(a,b) = (f(a) + f(b) - alpha (b - a))/2 (Equ:LFFlux), with
 * alpha = max of the two states' local speeds. */
void orc_lf_flux(int d, const double* a, const double* b, double gamma, double ch, double* f) {
  double fa[NV], fb[NV];
  orc_flux(d, a, gamma, ch, fa);
  orc_flux(d, b, gamma, ch, fb);
  double aa = orc_alpha(d, a, gamma), ab = orc_alpha(d, b, gamma);
  double alpha = aa > ab ? aa : ab;
  for (int v = 0; v < NV; ++v) {
    double s = comp_speed(v, d, alpha, ch);
    f[v] = 0.5 * ((fa[v] + fb[v]) - s * (b[v] - a[v]));
  }
  FLOPS(5 * NV);
}

/* Fast magnetosonic speed along d (the c_f of orc_alpha, without |v_d|). */
static double fast_speed(int d, const double* w, double gamma) {
  double rho = w[RHO];
  double p = pressure(w, gamma);
  if (p < 0.0) p = 0.0;
  double a2 = gamma * p / rho;
  double b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) / rho;
  double bd2 = w[BX + d] * w[BX + d] / rho;
  double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * bd2;
  if (disc < 0.0) disc = 0.0;
  FLOPS(19);
  return sqrt(0.5 * (s + sqrt(disc)));
}

/* HLLC flux for MHD (the approximate Riemann solver of Gurski that the paper uses for LF
 * and WENO in 2D/3D, Sec. 3.2-3.3; the paper does not print it).  Steps:
 * 1. The linear (B_d, psi) subsystem keeps its exact upwind flux, as in f_m:
 *    F(B_d) = (psi_a + psi_b - c_h (B_d,b - B_d,a))/2, F(psi) = c_h^2 B_m, with the interface
 *    normal field B_m = (B_d,a + B_d,b)/2 - (psi_b - psi_a)/(2 c_h) (the plain mean if c_h = 0).
 * 2. Both states take B_d = B_m at unchanged gas pressure: E' = E + (B_m^2 - B_d^2)/2.
 * 3. Speed bounds S_L = min(u_a - c_f,a, u_b - c_f,b), S_R = max(u_a + c_f,a, u_b + c_f,b)
 *    (u = v_d, c_f the fast speed along d of the modified states).
 * 4. S_L >= 0: F(a'); S_R <= 0: F(b'); otherwise the star state on the side of the contact
 *    speed S_M = (rho u)_HLL / rho_HLL, with, for K the side taken and S_K its bound,
 *      rho* = rho_K (S_K - u_K)/(S_K - S_M),  m*_d = rho* S_M,
 *      p_T* = p_T,K + rho_K (S_K - u_K)(S_M - u_K),
 *      B*_t = B_t of the HLL state,  B*_d = B_m,
 *      m*_t = rho* v_t,K - B_m (B*_t - B_t,K)/(S_K - S_M),
 *      E* = (E_K (S_K - u_K) - p_T,K u_K + p_T* S_M + B_m (v_K.B_K - v*.B*))/(S_K - S_M)
 *    (Rankine-Hugoniot across S_K), and F = F(K') + S_K (U* - U_K') for rho, m, B_t and E. */
void orc_hllc_flux(int d, const double* a, const double* b, double gamma, double ch, double* f) {
  double bm;
  if (ch > 0.0) bm = 0.5 * (a[BX + d] + b[BX + d]) - (b[PSI] - a[PSI]) / (2.0 * ch);
  else bm = 0.5 * (a[BX + d] + b[BX + d]);
  double w[2][NV], F[2][NV], u[2], cf[2], pt[2];
  for (int k = 0; k < 2; ++k) {
    const double* q = k ? b : a;
    for (int v = 0; v < NV; ++v) w[k][v] = q[v];
    const double p = pressure(q, gamma);
    w[k][BX + d] = bm;
    w[k][EN] = q[EN] + 0.5 * (bm * bm - q[BX + d] * q[BX + d]);
    orc_flux(d, w[k], gamma, ch, F[k]);
    u[k] = w[k][MX + d] / w[k][RHO];
    cf[k] = fast_speed(d, w[k], gamma);
    pt[k] = p + 0.5 * (w[k][BX] * w[k][BX] + w[k][BY] * w[k][BY] + w[k][BZ] * w[k][BZ]);
    FLOPS(15);
  }
  const double sl = fmin(u[0] - cf[0], u[1] - cf[1]);
  const double sr = fmax(u[0] + cf[0], u[1] + cf[1]);
  FLOPS(4);
  if (sl >= 0.0) {
    for (int v = 0; v < NV; ++v) f[v] = F[0][v];
  } else if (sr <= 0.0) {
    for (int v = 0; v < NV; ++v) f[v] = F[1][v];
  } else {
    const double ra = w[0][RHO], rb = w[1][RHO];
    const double sm = (rb * u[1] * (sr - u[1]) - ra * u[0] * (sl - u[0]) - pt[1] + pt[0]) /
                      (rb * (sr - u[1]) - ra * (sl - u[0]));
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;     /* tangential dimensions */
    double bt[3];
    bt[d] = bm;
    for (int t = 0; t < 2; ++t) {
      const int j = t ? t2 : t1;
      bt[j] = (sr * w[1][BX + j] - sl * w[0][BX + j] - (F[1][BX + j] - F[0][BX + j])) / (sr - sl);
    }
    const int k = sm >= 0.0 ? 0 : 1;
    const double sk = k ? sr : sl;
    const double* wk = w[k];
    const double uk = u[k], dk = sk - uk, ds = sk - sm;
    const double rs = wk[RHO] * dk / ds;
    const double pts = pt[k] + wk[RHO] * dk * (sm - uk);
    double us[NV];
    us[RHO] = rs;
    us[MX + d] = rs * sm;
    double vb_k = 0.0, vb_s = sm * bm;
    for (int j = 0; j < 3; ++j) vb_k += (wk[MX + j] / wk[RHO]) * wk[BX + j];
    for (int t = 0; t < 2; ++t) {
      const int j = t ? t2 : t1;
      us[MX + j] = rs * (wk[MX + j] / wk[RHO]) - bm * (bt[j] - wk[BX + j]) / ds;
      vb_s += (us[MX + j] / rs) * bt[j];
    }
    for (int j = 0; j < 3; ++j) us[BX + j] = bt[j];
    us[EN] = (wk[EN] * dk - pt[k] * uk + pts * sm + bm * (vb_k - vb_s)) / ds;
    us[PSI] = wk[PSI];
    for (int v = 0; v < NV; ++v) f[v] = F[k][v] + sk * (us[v] - wk[v]);
    FLOPS(16 + 2 * 7 + 4 + 5 + 3 * 3 + 2 * 9 + 10 + 2 * NV);
  }
  /* the (B_d, psi) pair: exact upwind flux of the linear GLM subsystem (as in f_m) */
  f[BX + d] = 0.5 * ((a[PSI] + b[PSI]) - ch * (b[BX + d] - a[BX + d]));
  f[PSI] = 0.5 * ((ch * ch * a[BX + d] + ch * ch * b[BX + d]) - ch * (b[PSI] - a[PSI]));
  FLOPS(11);
}

/* HLLD flux for MHD (Miyoshi & Kusano, J. Comput. Phys. 208, 2005), which the paper names
 * among the approximate Riemann solvers of MAP for LF and WENO and compares with HLLC on the
 * Brio-Wu tube (Sec. 3.2, Sec. 5), without printing it.  It resolves five waves: the fast
 * waves S_L, S_R, the rotational (Alfven) waves S*_L, S*_R and the contact S_M, with the
 * normal velocity S_M, the total pressure p_T* and the normal field constant inside the fan.
 * Steps 1-3 are those of orc_hllc_flux: the (B_d, psi) pair keeps the exact upwind flux of
 * its linear system, both states take the interface normal field B_n = B_m at unchanged gas
 * pressure, and the fast-wave bounds are S_L = min(u - c_f), S_R = max(u + c_f).  Then, with
 * d_K = S_K - u_K for the sides K = L (a), R (b):
 * 4. S_M = (d_R rho_R u_R - d_L rho_L u_L - p_T,R + p_T,L) / (d_R rho_R - d_L rho_L),
 *    p_T* = (d_R rho_R p_T,L - d_L rho_L p_T,R + rho_L rho_R d_R d_L (u_R - u_L))
 *           / (d_R rho_R - d_L rho_L).
 * 5. Outer states U*_K: rho* = rho_K d_K/(S_K - S_M), normal velocity S_M, and with
 *    D_K = rho_K d_K (S_K - S_M) - B_n^2, for each tangential direction t,
 *      v*_t = v_t - B_n B_t (S_M - u_K)/D_K,  B*_t = B_t (rho_K d_K^2 - B_n^2)/D_K
 *    (v and B unchanged where D_K vanishes, the fast and Alfven waves then coinciding),
 *      E* = (d_K E_K - p_T,K u_K + p_T* S_M + B_n (v_K.B_K - v*.B*))/(S_K - S_M).
 * 6. Inner states U**_K (sigma = sign B_n, r_K = sqrt(rho*_K); the density is rho*_K):
 *      v**_t = (r_L v*_t,L + r_R v*_t,R + sigma (B*_t,R - B*_t,L))/(r_L + r_R),
 *      B**_t = (r_L B*_t,R + r_R B*_t,L + sigma r_L r_R (v*_t,R - v*_t,L))/(r_L + r_R),
 *      E**_L = E*_L - sigma r_L (v*_L.B*_L - v**.B**),  E**_R = E*_R + sigma r_R (v*_R.B*_R - v**.B**).
 * 7. With S*_L = S_M - |B_n|/r_L and S*_R = S_M + |B_n|/r_R the flux is that of the region
 *    holding the interface: F_L, F_L + S_L (U*_L - U_L), that + S*_L (U**_L - U*_L), the
 *    mirror images on the right, or F_R.  With B_n = 0 the inner region has no width and three
 *    waves remain; their star field B_t (S - u)/(S - S_M) follows the density, where
 *    orc_hllc_flux takes the HLL state's, so the two agree only when B = 0. */
void orc_hlld_flux(int d, const double* a, const double* b, double gamma, double ch, double* f) {
  double bm;
  if (ch > 0.0) bm = 0.5 * (a[BX + d] + b[BX + d]) - (b[PSI] - a[PSI]) / (2.0 * ch);
  else bm = 0.5 * (a[BX + d] + b[BX + d]);
  double w[2][NV], F[2][NV], u[2], cf[2], pt[2];
  for (int k = 0; k < 2; ++k) {
    const double* q = k ? b : a;
    for (int v = 0; v < NV; ++v) w[k][v] = q[v];
    const double p = pressure(q, gamma);
    w[k][BX + d] = bm;
    w[k][EN] = q[EN] + 0.5 * (bm * bm - q[BX + d] * q[BX + d]);
    orc_flux(d, w[k], gamma, ch, F[k]);
    u[k] = w[k][MX + d] / w[k][RHO];
    cf[k] = fast_speed(d, w[k], gamma);
    pt[k] = p + 0.5 * (w[k][BX] * w[k][BX] + w[k][BY] * w[k][BY] + w[k][BZ] * w[k][BZ]);
    FLOPS(15);
  }
  const double sl = fmin(u[0] - cf[0], u[1] - cf[1]);
  const double sr = fmax(u[0] + cf[0], u[1] + cf[1]);
  FLOPS(4);
  if (sl >= 0.0) {
    for (int v = 0; v < NV; ++v) f[v] = F[0][v];
  } else if (sr <= 0.0) {
    for (int v = 0; v < NV; ++v) f[v] = F[1][v];
  } else {
    const int tt[2] = {d == 0 ? 1 : 0, d == 2 ? 1 : 2};      /* tangential dimensions */
    const double sk[2] = {sl, sr};
    const double dl = sl - u[0], dr = sr - u[1];
    const double ra = w[0][RHO], rb = w[1][RHO];
    const double den = dr * rb - dl * ra;
    const double sm = (dr * rb * u[1] - dl * ra * u[0] - pt[1] + pt[0]) / den;
    const double pts = (dr * rb * pt[0] - dl * ra * pt[1] + ra * rb * dr * dl * (u[1] - u[0])) / den;
    double us[2][NV], uss[2][NV], vs[2][3], bs[2][3], rs[2], vbs[2];
    for (int k = 0; k < 2; ++k) {
      const double* wk = w[k];
      const double rho = wk[RHO], dk = sk[k] - u[k], ds = sk[k] - sm;
      rs[k] = rho * dk / ds;
      const double D = rho * dk * ds - bm * bm;
      const int flat = fabs(D) <= 1e-12 * (fabs(rho * dk * ds) + bm * bm);
      double vb = 0.0;
      for (int j = 0; j < 3; ++j) vb += (wk[MX + j] / rho) * wk[BX + j];
      vs[k][d] = sm;
      bs[k][d] = bm;
      for (int t = 0; t < 2; ++t) {
        const int j = tt[t];
        const double vt = wk[MX + j] / rho, bt = wk[BX + j];
        vs[k][j] = flat ? vt : vt - bm * bt * (sm - u[k]) / D;
        bs[k][j] = flat ? bt : bt * (rho * dk * dk - bm * bm) / D;
      }
      vbs[k] = vs[k][0] * bs[k][0] + vs[k][1] * bs[k][1] + vs[k][2] * bs[k][2];
      us[k][RHO] = rs[k];
      for (int j = 0; j < 3; ++j) {
        us[k][MX + j] = rs[k] * vs[k][j];
        us[k][BX + j] = bs[k][j];
      }
      us[k][EN] = (dk * wk[EN] - pt[k] * u[k] + pts * sm + bm * (vb - vbs[k])) / ds;
      us[k][PSI] = wk[PSI];
      FLOPS(6 + 6 + 2 * 8 + 5 + 6 + 10);
    }
    const double sgn = bm > 0.0 ? 1.0 : (bm < 0.0 ? -1.0 : 0.0);
    const double rl = sqrt(rs[0]), rr = sqrt(rs[1]);
    const double ssl = sm - fabs(bm) / rl, ssr = sm + fabs(bm) / rr;
    double vss[3], bss[3];
    vss[d] = sm;
    bss[d] = bm;
    for (int t = 0; t < 2; ++t) {
      const int j = tt[t];
      vss[j] = (rl * vs[0][j] + rr * vs[1][j] + sgn * (bs[1][j] - bs[0][j])) / (rl + rr);
      bss[j] = (rl * bs[1][j] + rr * bs[0][j] + sgn * rl * rr * (vs[1][j] - vs[0][j])) / (rl + rr);
    }
    const double vbss = vss[0] * bss[0] + vss[1] * bss[1] + vss[2] * bss[2];
    for (int k = 0; k < 2; ++k) {
      uss[k][RHO] = rs[k];
      for (int j = 0; j < 3; ++j) {
        uss[k][MX + j] = rs[k] * vss[j];
        uss[k][BX + j] = bss[j];
      }
      uss[k][EN] = k == 0 ? us[0][EN] - sgn * rl * (vbs[0] - vbss) : us[1][EN] + sgn * rr * (vbs[1] - vbss);
      uss[k][PSI] = w[k][PSI];
    }
    FLOPS(2 + 4 + 2 * 16 + 5 + 2 * 8);
    if (ssl >= 0.0) {
      for (int v = 0; v < NV; ++v) f[v] = F[0][v] + sl * (us[0][v] - w[0][v]);
    } else if (sm >= 0.0) {
      for (int v = 0; v < NV; ++v) f[v] = F[0][v] + sl * (us[0][v] - w[0][v]) + ssl * (uss[0][v] - us[0][v]);
    } else if (ssr >= 0.0) {
      for (int v = 0; v < NV; ++v) f[v] = F[1][v] + sr * (us[1][v] - w[1][v]) + ssr * (uss[1][v] - us[1][v]);
    } else {
      for (int v = 0; v < NV; ++v) f[v] = F[1][v] + sr * (us[1][v] - w[1][v]);
    }
    FLOPS(5 * NV);
  }
  /* the (B_d, psi) pair: exact upwind flux of the linear GLM subsystem (as in f_m) */
  f[BX + d] = 0.5 * ((a[PSI] + b[PSI]) - ch * (b[BX + d] - a[BX + d]));
  f[PSI] = 0.5 * ((ch * ch * a[BX + d] + ch * ch * b[BX + d]) - ch * (b[PSI] - a[PSI]));
  FLOPS(11);
}

/* Interface flux of LF and WENO: f_m (Equ:LFFlux), HLLC or HLLD. */
static void riemann_flux(int riemann, int d, const double* a, const double* b, double gamma, double ch,
                         double* f) {
  if (riemann == 1) orc_hllc_flux(d, a, b, gamma, ch, f);
  else if (riemann == 2) orc_hlld_flux(d, a, b, gamma, ch, f);
  else orc_lf_flux(d, a, b, gamma, ch, f);
}

static double minmod(double a, double b) {
  /* minmod(a,b) = sgn(a) max(0, min(|a|, sgn(a) b))  (eq. minmod, Sec. 3.2) */
  if (a > 0.0) { double m = a < b ? a : b; return m > 0.0 ? m : 0.0; }
  if (a < 0.0) { double m = -a < -b ? -a : -b; return m > 0.0 ? -m : 0.0; }
  return 0.0;
}

/* Limiter as a function of two differences.
 * kind 0 minmod, 1 van Leer (harmonic mean when a, b agree in sign, else 0), 2 the
 * literal form of Sec. 3.1, phi(r) b with phi(r) = r for |r| <= 1 and 1 otherwise, 3 no
 * limiting, phi = 1 (returns b; a test option that turns MMC into its unlimited form), 4
 * phi = 0 (returns 0; a test option that leaves MMC with its first-order part h alone).
 * For MMC, phi(r) g with r = a/b equals this function of (a, b) (division free); a zero
 * denominator gives 0.  Kinds 2, 3 and 4 are MMC options only. */
double orc_limiter(int kind, double a, double b) {
  if (kind == 0) return minmod(a, b);
  if (kind == 3) return b;
  if (kind == 4) return 0.0;
  if (kind == 1) {
    FLOPS(1);
    if (!(a * b > 0.0)) return 0.0;
    FLOPS(4);
    return (2.0 * a * b) / (a + b);
  }
  if (b == 0.0) return 0.0;
  return (fabs(a) <= fabs(b)) ? a : b;
}

/* Two-stencil WENO reconstructions of Sec. 3.3 around cell 0: the left state of face
 * +1/2 (u^-_{i+1/2}) and the right state of face -1/2 (u^+_{i-1/2}).  The printed
 * denominator of u^+ repeats a_{i-1/2}; it is read as a_{i+1/2} + 2 a_{i-1/2}, the mirror
 * of u^-. */
void orc_weno_faces(double um, double u0, double up, double* minus_right, double* plus_left) {
  const double eps = 1e-12;
  double dp = up - u0, dm = u0 - um;
  double ap = 1.0 / ((eps + dp * dp) * (eps + dp * dp));
  double am = 1.0 / ((eps + dm * dm) * (eps + dm * dm));
  double wm = 0.5 * (u0 + up), vm = 0.5 * (3.0 * u0 - um);
  double wp = 0.5 * (3.0 * u0 - up), vp = 0.5 * (u0 + um);
  FLOPS(38);
  *minus_right = (2.0 * ap * wm + am * vm) / (2.0 * ap + am);
  *plus_left = (ap * wp + 2.0 * am * vp) / (ap + 2.0 * am);
}

/* Conservative linear prolongation along one axis (Sec. 4.3, Matsumoto 2007): fine cell
 * value from the coarse cell and its two neighbours; odd = fine cell on the + side. */
double orc_prolong_1d(double um, double u0, double up, int odd) {
  FLOPS(4);
  return u0 + minmod(up - u0, u0 - um) * (odd ? 0.25 : -0.25);
}

/* ------------------------------------------------------------------------------------ */
/* Block geometry helpers.                                                                 */

typedef struct {
  int ndim, nb, NX, NY, NZ, S;
  int off[3];
} geom;

static geom make_geom(int ndim, int nb) {
  geom g;
  g.ndim = ndim; g.nb = nb;
  g.NX = nb + 2 * NG; g.NY = nb + 2 * NG; g.NZ = ndim == 3 ? nb + 2 * NG : 1;
  g.S = g.NX * g.NY * g.NZ;
  g.off[0] = 1; g.off[1] = g.NX; g.off[2] = g.NX * g.NY;
  return g;
}

static int cidx(const geom* g, int k, int j, int i) { return (k * g->NY + j) * g->NX + i; }

static void load(const geom* g, const double* u, int c, double* w) {
  for (int v = 0; v < NV; ++v) w[v] = u[v * g->S + c];
}

/* Region "margin m": padded indices [m, N-m) in every active dimension. */
#define FOR_REGION(g, m, k, j, i)                                                    \
  for (int k = ((g)->ndim == 3 ? (m) : 0); k < ((g)->ndim == 3 ? (g)->NZ - (m) : 1); ++k) \
    for (int j = (m); j < (g)->NY - (m); ++j)                                         \
      for (int i = (m); i < (g)->NX - (m); ++i)

/* ------------------------------------------------------------------------------------ */
/* Source terms.                                                                           */

/* EGLM non-conservative sources of a state array at cell c (eqs. MHD-2 and MHD-4):
 *   momentum -(div B) B,  energy -B . grad psi,
 * with central differences (reading: the discretisation is not stated). */
static void eglm_source(const geom* g, const double* u, int c, const double* dx, double* s) {
  double divb = 0.0, bgpsi = 0.0;
  for (int d = 0; d < g->ndim; ++d) {
    int o = g->off[d];
    divb += (u[(BX + d) * g->S + c + o] - u[(BX + d) * g->S + c - o]) / (2.0 * dx[d]);
  }
  for (int d = 0; d < g->ndim; ++d) {
    int o = g->off[d];
    double gpsi = (u[PSI * g->S + c + o] - u[PSI * g->S + c - o]) / (2.0 * dx[d]);
    bgpsi += u[(BX + d) * g->S + c] * gpsi;
  }
  for (int j = 0; j < 3; ++j) s[MX + j] += -divb * u[(BX + j) * g->S + c];
  s[EN] += -bgpsi;
  FLOPS(9 * g->ndim + 7);
}

/* central difference of field f (one component, stride S) along d, 0 outside ndim */
static double cdiff(const geom* g, const double* f, int c, int d, const double* dx) {
  if (d >= g->ndim) return 0.0;
  int o = g->off[d];
  FLOPS(3);
  return (f[c + o] - f[c - o]) / (2.0 * dx[d]);
}

/* Current density J = curl B (Sec. 3.5, central differences) on the margin-1 region. */
static void current_density(const geom* g, const double* u, const double* dx, double* J) {
  const double* bx = u + BX * g->S;
  const double* by = u + BY * g->S;
  const double* bz = u + BZ * g->S;
  memset(J, 0, sizeof(double) * 3 * g->S);
  FOR_REGION(g, 1, k, j, i) {
    int c = cidx(g, k, j, i);
    J[0 * g->S + c] = cdiff(g, bz, c, 1, dx) - cdiff(g, by, c, 2, dx);
    J[1 * g->S + c] = cdiff(g, bx, c, 2, dx) - cdiff(g, bz, c, 0, dx);
    J[2 * g->S + c] = cdiff(g, by, c, 0, dx) - cdiff(g, bx, c, 1, dx);
    FLOPS(3);
  }
}

/* Resistive terms at interior cell c (Sec. 3.5): R = -curl(eta J) and
 * R_e = -div((eta J) x B), written as the paper's central differences (the missing "+"
 * signs between the three R_e terms are read as sums). */
static void resistive_source(const geom* g, const double* u, const double* J, int c,
                             const double* dx, double eta, double* s) {
  const double* jx = J;
  const double* jy = J + g->S;
  const double* jz = J + 2 * g->S;
  /* eta uniform: derivatives of eta J are eta times derivatives of J */
  double rx = eta * cdiff(g, jy, c, 2, dx) - eta * cdiff(g, jz, c, 1, dx);
  double ry = eta * cdiff(g, jz, c, 0, dx) - eta * cdiff(g, jx, c, 2, dx);
  double rz = eta * cdiff(g, jx, c, 1, dx) - eta * cdiff(g, jy, c, 0, dx);
  /* R_e = d/dx(eta(Jz By - Jy Bz)) + d/dy(eta(Jx Bz - Jz Bx)) + d/dz(eta(Jy Bx - Jx By)) */
  double re = 0.0;
  for (int d = 0; d < g->ndim; ++d) {
    int o = g->off[d];
    double q[2];
    for (int sgn = 0; sgn < 2; ++sgn) {
      int cc = sgn ? c + o : c - o;
      double Bx = u[BX * g->S + cc], By = u[BY * g->S + cc], Bz = u[BZ * g->S + cc];
      double Jx = jx[cc], Jy = jy[cc], Jz = jz[cc];
      double t;
      if (d == 0) t = Jz * By - Jy * Bz;
      else if (d == 1) t = Jx * Bz - Jz * Bx;
      else t = Jy * Bx - Jx * By;
      q[sgn] = eta * t;
    }
    re += (q[1] - q[0]) / (2.0 * dx[d]);
  }
  s[BX] += rx;
  s[BY] += ry;
  s[BZ] += rz;
  s[EN] += re;
  FLOPS(13 + 12 * g->ndim);
}

/* ------------------------------------------------------------------------------------ */
/* Schemes on one ghost-filled block.  "out" is a padded array; its interior is written.  */

typedef struct {
  double gamma, ch, dt, eta;
  int eglm, limiter;
  double dx[3];
  int riemann;    /* interface flux of LF and WENO: 0 f_m (Lax-Friedrichs), 1 HLLC, 2 HLLD */
  double* freg;   /* face register of the block (reflux), or NULL */
  double fw;      /* weight of this update's fluxes in the register (1, or 1/2 per RK2 stage) */
} stepctx;

/* Face register (reflux, Sec. 4.2 step (2)): the flux through every boundary face cell of a
 * block, summed over the step's flux evaluations with weight fw.  Layout
 * [side][NV][nb][nb], side = 2d (low face of dimension d) or 2d + 1 (high face); the face
 * cell is indexed t0 + nb t1 by its interior coordinates in the two other dimensions, in
 * increasing dimension order (t1 = 0 in 2D). */
static void record_face(const geom* g, const stepctx* s, int d, int side, int k, int j, int i,
                        const double* f) {
  if (!s->freg) return;
  int x = i - NG, y = j - NG, z = g->ndim == 3 ? k - NG : 0;
  int t0 = d == 0 ? y : x, t1 = d == 2 ? y : z;
  size_t nb2 = (size_t)g->nb * g->nb;
  double* r = s->freg + (size_t)(2 * d + side) * NV * nb2 + (size_t)t1 * g->nb + t0;
  for (int v = 0; v < NV; ++v) r[v * nb2] += s->fw * f[v];
}

/* Interior coordinate of padded cell (k, j, i) along d. */
static int icoord(int d, int k, int j, int i) { return (d == 0 ? i : d == 1 ? j : k) - NG; }

/* MMC (Sec. 3.1).  Split fluxes f^+- = (f +- alpha u)/2.  Reading of the local speeds:
 * each face i+1/2 carries alpha = max(alpha(u_i), alpha(u_{i+1})) and
 * alpha~ = max(alpha(u~_i), alpha(u~_{i+1})); every split term entering that face's flux
 * (h and the four g's) is evaluated with the speeds of that face, so a face flux needs
 * u_{i-1..i+2} and u~_{i..i+1} only and the scheme stays conservative (one flux per face).
 * The (B_d, psi) pair uses c_h for both. */
static double splitp(double f, double a, double u) { FLOPS(3); return 0.5 * (f + a * u); }
static double splitm(double f, double a, double u) { FLOPS(3); return 0.5 * (f - a * u); }

static void mmc_h(const geom* g, const stepctx* s, int d, const double* u, int cl, double* h) {
  double wl[NV], wr[NV], fl[NV], fr[NV];
  load(g, u, cl, wl);
  load(g, u, cl + g->off[d], wr);
  orc_flux(d, wl, s->gamma, s->ch, fl);
  orc_flux(d, wr, s->gamma, s->ch, fr);
  double al = orc_alpha(d, wl, s->gamma), ar = orc_alpha(d, wr, s->gamma);
  double alpha = al > ar ? al : ar;
  for (int v = 0; v < NV; ++v) {
    double a = comp_speed(v, d, alpha, s->ch);
    h[v] = splitp(fl[v], a, wl[v]) + splitm(fr[v], a, wr[v]);
  }
  FLOPS(NV);
}

static void mmc_face(const geom* g, const stepctx* s, int d, const double* u, const double* ut,
                     int ci, double* fhat) {
  int o = g->off[d];
  double w[4][NV], t[2][NV], fu[4][NV], ft[2][NV];
  for (int q = 0; q < 4; ++q) {
    load(g, u, ci + (q - 1) * o, w[q]);
    orc_flux(d, w[q], s->gamma, s->ch, fu[q]);
  }
  for (int q = 0; q < 2; ++q) {
    load(g, ut, ci + q * o, t[q]);
    orc_flux(d, t[q], s->gamma, s->ch, ft[q]);
  }
  /* w[1] = u_i, w[2] = u_{i+1}; t[0] = u~_i, t[1] = u~_{i+1} */
  double a1 = orc_alpha(d, w[1], s->gamma), a2 = orc_alpha(d, w[2], s->gamma);
  double alpha = a1 > a2 ? a1 : a2;
  double b1 = orc_alpha(d, t[0], s->gamma), b2 = orc_alpha(d, t[1], s->gamma);
  double alphat = b1 > b2 ? b1 : b2;
  for (int v = 0; v < NV; ++v) {
    double a = comp_speed(v, d, alpha, s->ch);
    double at = comp_speed(v, d, alphat, s->ch);
    double h = splitp(fu[1][v], a, w[1][v]) + splitm(fu[2][v], a, w[2][v]);
    double gp_l = splitp(ft[0][v], at, t[0][v]) - splitp(fu[0][v], a, w[0][v]); /* g+_{i-1/2} */
    double gp_c = splitp(ft[1][v], at, t[1][v]) - splitp(fu[1][v], a, w[1][v]); /* g+_{i+1/2} */
    double gm_c = splitm(fu[2][v], a, w[2][v]) - splitm(ft[0][v], at, t[0][v]); /* g-_{i+1/2} */
    double gm_r = splitm(fu[3][v], a, w[3][v]) - splitm(ft[1][v], at, t[1][v]); /* g-_{i+3/2} */
    fhat[v] = h + 0.5 * (orc_limiter(s->limiter, gp_l, gp_c) - orc_limiter(s->limiter, gm_r, gm_c));
  }
  FLOPS(8 * NV);
}

static void mmc_block(const geom* g, const stepctx* s, const double* u, double* out) {
  double* ut = (double*)calloc((size_t)NV * g->S, sizeof(double));
  double* J = (double*)calloc((size_t)3 * g->S, sizeof(double));
  /* predictor u~ = u - sum_d dt/dx_d (h_{i+1/2} - h_{i-1/2})  on the margin-1 region */
  FLCAT(0);
  FOR_REGION(g, 1, k, j, i) {
    int c = cidx(g, k, j, i);
    double acc[NV], hp[NV], hm[NV];
    load(g, u, c, acc);
    for (int d = 0; d < g->ndim; ++d) {
      mmc_h(g, s, d, u, c, hp);
      mmc_h(g, s, d, u, c - g->off[d], hm);
      double lam = s->dt / s->dx[d];
      for (int v = 0; v < NV; ++v) acc[v] -= lam * (hp[v] - hm[v]);
      FLOPS(1 + 3 * NV);
    }
    for (int v = 0; v < NV; ++v) ut[v * g->S + c] = acc[v];
  }
  FLCAT(0);
  if (s->eta > 0.0) current_density(g, u, s->dx, J);
  FLCAT(2);
  /* corrector: u^{n+1} = u - sum_d dt/dx_d (fhat_{i+1/2} - fhat_{i-1/2}) + dt S(u^n) */
  FOR_REGION(g, NG, k, j, i) {
    int c = cidx(g, k, j, i);
    double acc[NV], fp[NV], fm[NV], src[NV] = {0};
    load(g, u, c, acc);
    for (int d = 0; d < g->ndim; ++d) {
      FLCAT(1);
      mmc_face(g, s, d, u, ut, c, fp);
      mmc_face(g, s, d, u, ut, c - g->off[d], fm);
      FLCAT(2);
      if (icoord(d, k, j, i) == 0) record_face(g, s, d, 0, k, j, i, fm);
      if (icoord(d, k, j, i) == g->nb - 1) record_face(g, s, d, 1, k, j, i, fp);
      double lam = s->dt / s->dx[d];
      for (int v = 0; v < NV; ++v) acc[v] -= lam * (fp[v] - fm[v]);
      FLOPS(1 + 3 * NV);
    }
    if (s->eglm) eglm_source(g, u, c, s->dx, src);
    if (s->eta > 0.0) resistive_source(g, u, J, c, s->dx, s->eta, src);
    for (int v = 0; v < NV; ++v) out[v * g->S + c] = acc[v] + s->dt * src[v];
    FLOPS(2 * NV);
  }
  free(ut);
  free(J);
}

/* LF (Sec. 3.2): MUSCL-Hancock half step with limited slopes of the conserved variables
 * (limiter1), physical fluxes of the cell's own face states, then f_m (Equ:LFFlux) of the
 * u~ face states built with the same slopes (limiter2).  Sources: EGLM at half weight from
 * u^n in the predictor and full weight from u~ in the update; resistivity at full weight
 * from u^n in the update (its stencil needs two cells beyond u~'s one-cell ring). */
static void lf_block(const geom* g, const stepctx* s, const double* u, double* out) {
  double* ut = (double*)calloc((size_t)NV * g->S, sizeof(double));
  double* phi = (double*)calloc((size_t)3 * NV * g->S, sizeof(double));
  double* J = (double*)calloc((size_t)3 * g->S, sizeof(double));
  /* slopes phi_d = limiter(u_i - u_{i-1}, u_{i+1} - u_i) on the margin-1 region */
  FLCAT(0);
  FOR_REGION(g, 1, k, j, i) {
    int c = cidx(g, k, j, i);
    for (int d = 0; d < g->ndim; ++d) {
      int o = g->off[d];
      for (int v = 0; v < NV; ++v) {
        const double* f = u + v * g->S;
        phi[(d * NV + v) * g->S + c] = orc_limiter(s->limiter, f[c] - f[c - o], f[c + o] - f[c]);
        FLOPS(2);
      }
    }
  }
  /* predictor u~_i = u_i - dt/(2dx) (f(u^-_{i+1/2}) - f(u^+_{i-1/2})) + dt/2 S_EGLM(u) */
  FOR_REGION(g, 1, k, j, i) {
    int c = cidx(g, k, j, i);
    double acc[NV], w[NV], wm[NV], wp[NV], fm[NV], fp[NV], src[NV] = {0};
    load(g, u, c, w);
    for (int v = 0; v < NV; ++v) acc[v] = w[v];
    for (int d = 0; d < g->ndim; ++d) {
      for (int v = 0; v < NV; ++v) {
        double ph = phi[(d * NV + v) * g->S + c];
        wp[v] = w[v] + 0.5 * ph; /* u^-_{i+1/2} */
        wm[v] = w[v] - 0.5 * ph; /* u^+_{i-1/2} */
      }
      orc_flux(d, wp, s->gamma, s->ch, fp);
      orc_flux(d, wm, s->gamma, s->ch, fm);
      double lamh = (0.5 * s->dt) / s->dx[d];
      for (int v = 0; v < NV; ++v) acc[v] -= lamh * (fp[v] - fm[v]);
      FLOPS(4 * NV + 2 + 3 * NV);
    }
    if (s->eglm) eglm_source(g, u, c, s->dx, src);
    for (int v = 0; v < NV; ++v) ut[v * g->S + c] = acc[v] + (0.5 * s->dt) * src[v];
    FLOPS(3 * NV);
  }
  if (s->eta > 0.0) current_density(g, u, s->dx, J);
  FLCAT(2);
  FOR_REGION(g, NG, k, j, i) {
    int c = cidx(g, k, j, i);
    double acc[NV], src[NV] = {0};
    load(g, u, c, acc);
    for (int d = 0; d < g->ndim; ++d) {
      int o = g->off[d];
      double fl[NV], fr[NV];
      /* face i+1/2: left u~_i + phi_i/2, right u~_{i+1} - phi_{i+1}/2; face i-1/2 alike */
      FLCAT(1);
      for (int side = 0; side < 2; ++side) {
        int cl = side ? c : c - o;
        double a[NV], b[NV];
        for (int v = 0; v < NV; ++v) {
          a[v] = ut[v * g->S + cl] + 0.5 * phi[(d * NV + v) * g->S + cl];
          b[v] = ut[v * g->S + cl + o] - 0.5 * phi[(d * NV + v) * g->S + cl + o];
        }
        FLOPS(4 * NV);
        riemann_flux(s->riemann, d, a, b, s->gamma, s->ch, side ? fr : fl);
      }
      FLCAT(2);
      if (icoord(d, k, j, i) == 0) record_face(g, s, d, 0, k, j, i, fl);
      if (icoord(d, k, j, i) == g->nb - 1) record_face(g, s, d, 1, k, j, i, fr);
      double lam = s->dt / s->dx[d];
      for (int v = 0; v < NV; ++v) acc[v] -= lam * (fr[v] - fl[v]);
      FLOPS(1 + 3 * NV);
    }
    if (s->eglm) eglm_source(g, ut, c, s->dx, src);
    if (s->eta > 0.0) resistive_source(g, u, J, c, s->dx, s->eta, src);
    for (int v = 0; v < NV; ++v) out[v * g->S + c] = acc[v] + s->dt * src[v];
    FLOPS(2 * NV);
  }
  free(ut);
  free(phi);
  free(J);
}

/* WENO right-hand side L(w) on the interior (Sec. 3.3 + Sec. 3.7, dimension by dimension
 * from the same state, summed): L = -sum_d (fhat_{i+1/2} - fhat_{i-1/2})/dx_d + S(w). */
static void weno_rhs(const geom* g, const stepctx* s, const double* w, double* L) {
  double* J = (double*)calloc((size_t)3 * g->S, sizeof(double));
  FLCAT(0);
  if (s->eta > 0.0) current_density(g, w, s->dx, J);
  FLCAT(2);
  FOR_REGION(g, NG, k, j, i) {
    int c = cidx(g, k, j, i);
    double acc[NV] = {0}, src[NV] = {0};
    for (int d = 0; d < g->ndim; ++d) {
      int o = g->off[d];
      double fl[NV], fr[NV];
      FLCAT(1);
      for (int side = 0; side < 2; ++side) {
        int cl = side ? c : c - o; /* face between cl and cl+o */
        double a[NV], b[NV], dummy;
        for (int v = 0; v < NV; ++v) {
          const double* f = w + v * g->S;
          orc_weno_faces(f[cl - o], f[cl], f[cl + o], &a[v], &dummy);
          orc_weno_faces(f[cl], f[cl + o], f[cl + 2 * o], &dummy, &b[v]);
        }
        riemann_flux(s->riemann, d, a, b, s->gamma, s->ch, side ? fr : fl);
      }
      FLCAT(2);
      if (icoord(d, k, j, i) == 0) record_face(g, s, d, 0, k, j, i, fl);
      if (icoord(d, k, j, i) == g->nb - 1) record_face(g, s, d, 1, k, j, i, fr);
      for (int v = 0; v < NV; ++v) acc[v] -= (fr[v] - fl[v]) / s->dx[d];
      FLOPS(3 * NV);
    }
    if (s->eglm) eglm_source(g, w, c, s->dx, src);
    if (s->eta > 0.0) resistive_source(g, w, J, c, s->dx, s->eta, src);
    for (int v = 0; v < NV; ++v) L[v * g->S + c] = acc[v] + src[v];
    FLOPS(NV);
  }
  free(J);
}

/* ------------------------------------------------------------------------------------ */
/* Mesh: blocks, lookup, validation.                                                        */

static int key_cmp(const oblk* a, const oblk* b) {
  if (a->problem != b->problem) return a->problem < b->problem ? -1 : 1;
  if (a->level != b->level) return a->level < b->level ? -1 : 1;
  for (int d = 2; d >= 0; --d)
    if (a->ijk[d] != b->ijk[d]) return a->ijk[d] < b->ijk[d] ? -1 : 1;
  return 0;
}

static orc_mesh* g_sort_mesh;
static int order_cmp(const void* x, const void* y) {
  return key_cmp(&g_sort_mesh->b[*(const int*)x], &g_sort_mesh->b[*(const int*)y]);
}

static int anc_cmp(const void* x, const void* y) {
  return key_cmp((const oblk*)x, (const oblk*)y);
}

static int lookup(const orc_mesh* m, int p, int L, int i, int j, int k) {
  oblk key;
  key.problem = p; key.level = L; key.ijk[0] = i; key.ijk[1] = j; key.ijk[2] = k;
  int lo = 0, hi = m->nblocks - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    int c = key_cmp(&m->b[m->order[mid]], &key);
    if (c == 0) return m->order[mid];
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int nblk_dim(const orc_mesh* m, int p, int L, int d) {
  if (d >= m->ndim) return 1;
  return m->probs[p].nbase[d] << L;
}

static int add_block(orc_mesh* m, int* cap, int p, int L, const int* ijk, int leaf) {
  if (m->nblocks == *cap) {
    *cap = *cap ? 2 * *cap : 64;
    m->b = (oblk*)realloc(m->b, sizeof(oblk) * (size_t)*cap);
  }
  oblk* o = &m->b[m->nblocks];
  memset(o, 0, sizeof(*o));
  o->problem = p; o->level = L;
  for (int d = 0; d < 3; ++d) o->ijk[d] = ijk[d];
  o->leaf = leaf; o->parent = -1;
  for (int c = 0; c < 8; ++c) o->child[c] = -1;
  return m->nblocks++;
}

static void rebuild_order(orc_mesh* m) {
  free(m->order);
  m->order = (int*)malloc(sizeof(int) * (size_t)(m->nblocks ? m->nblocks : 1));
  for (int q = 0; q < m->nblocks; ++q) m->order[q] = q;
  g_sort_mesh = m;
  qsort(m->order, (size_t)m->nblocks, sizeof(int), order_cmp);
}

/* 2:1 balance across faces, edges and corners: the region next to a leaf at level L is
 * covered at level L-1, L or L+1 (no leaf two levels apart touches another). */
static int check_balance(const orc_mesh* m) {
  int nd = m->ndim;
  for (int q = 0; q < m->nblocks; ++q) {
    const oblk* o = &m->b[q];
    if (o->leaf < 0) continue;
    int L = o->level, p = o->problem;
    for (int oz = (nd == 3 ? -1 : 0); oz <= (nd == 3 ? 1 : 0); ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          int off[3] = {ox, oy, oz}, nbc[3];
          int outside = 0;
          for (int d = 0; d < 3; ++d) {
            int n = nblk_dim(m, p, L, d);
            nbc[d] = o->ijk[d] + off[d];
            if (nbc[d] < 0 || nbc[d] >= n) {
              if (m->probs[p].bc[d][nbc[d] < 0 ? 0 : 1] == 0) nbc[d] = (nbc[d] % n + n) % n;
              else outside = 1;
            }
          }
          if (outside) continue;
          int nbq = lookup(m, p, L, nbc[0], nbc[1], nbc[2]);
          if (nbq >= 0) {
            const oblk* nbk = &m->b[nbq];
            if (nbk->leaf >= 0) continue;
            /* neighbour refined: its children touching this block must be leaves */
            for (int c = 0; c < (1 << nd); ++c) {
              int bits[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
              int touching = 1;
              for (int d = 0; d < nd; ++d) {
                if (off[d] == 1 && bits[d] != 0) touching = 0;
                if (off[d] == -1 && bits[d] != 1) touching = 0;
              }
              if (!touching) continue;
              int ch = nbk->child[c];
              if (ch < 0 || m->b[ch].leaf < 0) return -1;
            }
          } else {
            if (L == 0) return -1;
            int cq = lookup(m, p, L - 1, nbc[0] >> 1, nbc[1] >> 1, nd == 3 ? nbc[2] >> 1 : 0);
            if (cq < 0 || m->b[cq].leaf < 0) return -1;
          }
        }
  }
  return 0;
}

orc_mesh* orc_create(int ndim, int nb, int nprob, const orc_problem* probs, int nleaves,
                     const int* leaves, int* err) {
  *err = 0;
  if ((ndim != 2 && ndim != 3) || nb < 4 || nprob < 1 || nleaves < 1) { *err = -1; return NULL; }
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  geom g = make_geom(ndim, nb);
  m->ndim = ndim; m->nb = nb; m->NX = g.NX; m->NY = g.NY; m->NZ = g.NZ; m->S = g.S;
  m->nprob = nprob;
  m->probs = (orc_problem*)malloc(sizeof(orc_problem) * (size_t)nprob);
  memcpy(m->probs, probs, sizeof(orc_problem) * (size_t)nprob);
  m->nleaves = nleaves;
  m->leaf_block = (int*)malloc(sizeof(int) * (size_t)nleaves);
  int cap = 0;
  /* leaves */
  for (int l = 0; l < nleaves; ++l) {
    const int* q = leaves + 5 * l;
    int p = q[0], L = q[1];
    int ijk[3] = {q[2], q[3], ndim == 3 ? q[4] : 0};
    if (p < 0 || p >= nprob || L < 0 || L > 20) { *err = -1; orc_destroy(m); return NULL; }
    for (int d = 0; d < 3; ++d) {
      int n = (d < ndim) ? (probs[p].nbase[d] << L) : 1;
      if (ijk[d] < 0 || ijk[d] >= n) { *err = -1; orc_destroy(m); return NULL; }
    }
    m->leaf_block[l] = add_block(m, &cap, p, L, ijk, l);
    if (L > m->maxlev) m->maxlev = L;
  }
  rebuild_order(m);
  for (int q = 1; q < m->nblocks; ++q)
    if (key_cmp(&m->b[m->order[q - 1]], &m->b[m->order[q]]) == 0) { *err = -2; orc_destroy(m); return NULL; }
  /* ancestors: every block above a leaf, once */
  {
    int na = 0, acap = 0;
    oblk* anc = NULL;
    for (int l = 0; l < nleaves; ++l) {
      oblk c = m->b[m->leaf_block[l]];
      while (c.level > 0) {
        c.level -= 1;
        for (int d = 0; d < 3; ++d) c.ijk[d] >>= 1;
        if (na == acap) { acap = acap ? 2 * acap : 256; anc = (oblk*)realloc(anc, sizeof(oblk) * (size_t)acap); }
        anc[na++] = c;
      }
    }
    /* sort ancestors by key, drop duplicates, reject ancestors that are leaves */
    qsort(anc, (size_t)na, sizeof(oblk), anc_cmp);
    for (int a = 0; a < na; ++a) {
      if (lookup(m, anc[a].problem, anc[a].level, anc[a].ijk[0], anc[a].ijk[1], anc[a].ijk[2]) >= 0) {
        free(anc); *err = -3; orc_destroy(m); return NULL;
      }
    }
    for (int a = 0; a < na; ++a) {
      if (a > 0 && key_cmp(&anc[a - 1], &anc[a]) == 0) continue;
      add_block(m, &cap, anc[a].problem, anc[a].level, anc[a].ijk, -1);
    }
    free(anc);
  }
  rebuild_order(m);
  for (int q = 0; q < m->nblocks; ++q) {
    oblk* c = &m->b[q];
    if (c->level == 0) continue;
    int par = lookup(m, c->problem, c->level - 1, c->ijk[0] >> 1, c->ijk[1] >> 1, c->ijk[2] >> 1);
    int cb = (c->ijk[0] & 1) | ((c->ijk[1] & 1) << 1) | ((c->ijk[2] & 1) << 2);
    m->b[par].child[cb] = q;
    c->parent = par;
  }
  /* completeness: each parent has all children, each base block exists */
  for (int q = 0; q < m->nblocks; ++q) {
    if (m->b[q].leaf >= 0) continue;
    for (int c = 0; c < (1 << ndim); ++c)
      if (m->b[q].child[c] < 0) { *err = -4; orc_destroy(m); return NULL; }
  }
  for (int p = 0; p < nprob; ++p) {
    int nz = ndim == 3 ? probs[p].nbase[2] : 1;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < probs[p].nbase[1]; ++j)
        for (int i = 0; i < probs[p].nbase[0]; ++i)
          if (lookup(m, p, 0, i, j, k) < 0) { *err = -4; orc_destroy(m); return NULL; }
  }
  if (check_balance(m) != 0) { *err = -5; orc_destroy(m); return NULL; }
  for (int q = 0; q < m->nblocks; ++q) {
    m->b[q].u = (double*)calloc((size_t)NV * m->S, sizeof(double));
    m->b[q].u1 = (double*)calloc((size_t)NV * m->S, sizeof(double));
  }
  m->dt = (double*)calloc((size_t)nprob, sizeof(double));
  m->ch = (double*)calloc((size_t)nprob, sizeof(double));
  m->cp = (double*)calloc((size_t)nprob, sizeof(double));
  m->damp = (double*)calloc((size_t)nprob, sizeof(double));
  m->alpha_g = (double*)calloc((size_t)nprob, sizeof(double));
  m->dtc = (double*)calloc((size_t)nprob, sizeof(double));
  return m;
}

void orc_destroy(orc_mesh* m) {
  if (!m) return;
  for (int q = 0; q < m->nblocks; ++q) { free(m->b[q].u); free(m->b[q].u1); }
  free(m->b); free(m->order); free(m->leaf_block); free(m->probs);
  free(m->dt); free(m->ch); free(m->cp); free(m->damp); free(m->alpha_g); free(m->dtc);
  free(m);
}

int orc_nleaves(const orc_mesh* m) { return m->nleaves; }

static geom mesh_geom(const orc_mesh* m) { return make_geom(m->ndim, m->nb); }

static void block_dx(const orc_mesh* m, const oblk* o, double* dx) {
  const orc_problem* pr = &m->probs[o->problem];
  for (int d = 0; d < 3; ++d) {
    int n = (d < m->ndim) ? (pr->nbase[d] << o->level) * m->nb : 1;
    dx[d] = (pr->hi[d] - pr->lo[d]) / (double)n;
  }
}

int orc_set_leaf(orc_mesh* m, int leaf, const double* in) {
  if (leaf < 0 || leaf >= m->nleaves) return -1;
  geom g = mesh_geom(m);
  double* u = m->b[m->leaf_block[leaf]].u;
  int nz = m->ndim == 3 ? m->nb : 1, n = m->nb, q = 0;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          u[v * g.S + cidx(&g, m->ndim == 3 ? k + NG : 0, j + NG, i + NG)] = in[q++];
  return 0;
}

int orc_get_leaf(const orc_mesh* m, int leaf, double* out) {
  if (leaf < 0 || leaf >= m->nleaves) return -1;
  geom g = mesh_geom(m);
  const double* u = m->b[m->leaf_block[leaf]].u;
  int nz = m->ndim == 3 ? m->nb : 1, n = m->nb, q = 0;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          out[q++] = u[v * g.S + cidx(&g, m->ndim == 3 ? k + NG : 0, j + NG, i + NG)];
  return 0;
}

int orc_get_leaf_ghosted(const orc_mesh* m, int leaf, double* out) {
  if (leaf < 0 || leaf >= m->nleaves) return -1;
  memcpy(out, m->b[m->leaf_block[leaf]].u, sizeof(double) * (size_t)NV * m->S);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Boundary conditions (Sec. 4.3).                                                          */

/* (1) parents are the average of their children (equal volumes), bottom-up. */
static void restrict_all(orc_mesh* m) {
  geom g = mesh_geom(m);
  int nd = m->ndim, nb = m->nb, nz = nd == 3 ? nb : 1;
  for (int L = m->maxlev - 1; L >= 0; --L) {
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* P = &m->b[q];
      if (P->level != L || P->leaf >= 0) continue;
      for (int v = 0; v < NV; ++v)
        for (int k = 0; k < nz; ++k)
          for (int j = 0; j < nb; ++j)
            for (int i = 0; i < nb; ++i) {
              int G[3] = {P->ijk[0] * nb + i, P->ijk[1] * nb + j, nd == 3 ? P->ijk[2] * nb + k : 0};
              double sum = 0.0;
              for (int dz = 0; dz < (nd == 3 ? 2 : 1); ++dz)
                for (int dy = 0; dy < 2; ++dy)
                  for (int dx = 0; dx < 2; ++dx) {
                    int F[3] = {2 * G[0] + dx, 2 * G[1] + dy, nd == 3 ? 2 * G[2] + dz : 0};
                    int cb = ((F[0] / nb) & 1) | (((F[1] / nb) & 1) << 1) |
                             ((nd == 3 ? (F[2] / nb) & 1 : 0) << 2);
                    const oblk* C = &m->b[P->child[cb]];
                    int lc = cidx(&g, nd == 3 ? F[2] - C->ijk[2] * nb + NG : 0,
                                  F[1] - C->ijk[1] * nb + NG, F[0] - C->ijk[0] * nb + NG);
                    sum += C->u[v * g.S + lc];
                  }
              P->u[v * g.S + cidx(&g, nd == 3 ? k + NG : 0, j + NG, i + NG)] =
                  sum / (double)(1 << nd);
            }
    }
  }
}

/* The value of the level-L representation of problem p at global cell G: periodic wrap or
 * zero-gradient clamp outside the domain, then the level-L block's cell if the level
 * exists there, otherwise the conservative minmod prolongation (Sec. 4.3) of the covering
 * level-(L-1) leaf, whose own ghosts are already filled. */
static int sample(const orc_mesh* m, int p, int L, const int* Gin, double* w) {
  geom g = mesh_geom(m);
  int nd = m->ndim, nb = m->nb;
  int G[3] = {Gin[0], Gin[1], Gin[2]};
  for (int d = 0; d < nd; ++d) {
    int N = (m->probs[p].nbase[d] << L) * nb;
    if (G[d] < 0 || G[d] >= N) {
      int side = G[d] < 0 ? 0 : 1;
      if (m->probs[p].bc[d][side] == 0) G[d] = ((G[d] % N) + N) % N;
      else G[d] = side ? N - 1 : 0;
    }
  }
  int q = lookup(m, p, L, G[0] / nb, G[1] / nb, nd == 3 ? G[2] / nb : 0);
  if (q >= 0) {
    const oblk* o = &m->b[q];
    int c = cidx(&g, nd == 3 ? G[2] - o->ijk[2] * nb + NG : 0, G[1] - o->ijk[1] * nb + NG,
                 G[0] - o->ijk[0] * nb + NG);
    load(&g, o->u, c, w);
    return 0;
  }
  if (L == 0) return -1;
  int Gc[3] = {G[0] >> 1, G[1] >> 1, nd == 3 ? G[2] >> 1 : 0};
  int qc = lookup(m, p, L - 1, Gc[0] / nb, Gc[1] / nb, nd == 3 ? Gc[2] / nb : 0);
  if (qc < 0 || m->b[qc].leaf < 0) return -1;
  const oblk* o = &m->b[qc];
  int c = cidx(&g, nd == 3 ? Gc[2] - o->ijk[2] * nb + NG : 0, Gc[1] - o->ijk[1] * nb + NG,
               Gc[0] - o->ijk[0] * nb + NG);
  for (int v = 0; v < NV; ++v) {
    const double* f = o->u + v * g.S;
    double val = f[c];
    for (int d = 0; d < nd; ++d) {
      int off = g.off[d];
      val += minmod(f[c + off] - f[c], f[c] - f[c - off]) * ((G[d] & 1) ? 0.25 : -0.25);
    }
    w[v] = val;
  }
  return 0;
}

int orc_fill_ghosts(orc_mesh* m) {
  geom g = mesh_geom(m);
  int nd = m->ndim, nb = m->nb;
  FLCAT(3);
  restrict_all(m);
  int status = 0;
  for (int L = 0; L <= m->maxlev; ++L) {
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->level != L || o->leaf < 0) continue;
      FOR_REGION(&g, 0, k, j, i) {
        int interior = (i >= NG && i < nb + NG && j >= NG && j < nb + NG &&
                        (nd == 2 || (k >= NG && k < nb + NG)));
        if (interior) continue;
        int G[3] = {o->ijk[0] * nb + i - NG, o->ijk[1] * nb + j - NG,
                    nd == 3 ? o->ijk[2] * nb + k - NG : 0};
        double w[NV];
        if (sample(m, o->problem, L, G, w) != 0) { status = -1; continue; }
        int c = cidx(&g, k, j, i);
        for (int v = 0; v < NV; ++v) o->u[v * g.S + c] = w[v];
      }
    }
  }
  FLCAT(2);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Time step (Sec. 3.7 and Sec. 2: c_h, c_p).                                               */

/* Temperature T = p / rho (p clamped at 0) and conductivity kappa = kappa0 T^(5/2). */
static double temperature(const double* w, double gamma) {
  double p = pressure(w, gamma);
  if (p < 0.0) p = 0.0;
  return p / w[RHO];
}

static double kappa_of(double T, double kappa0) { return kappa0 * (T * T * sqrt(T)); }

/* The rate in the conduction time step: kappa T / p, written kappa / rho (equal for p > 0,
 * and finite at p = 0). */
static double conduction_rate(const double* w, const orc_params* pr) {
  return kappa_of(temperature(w, pr->gamma), pr->kappa0) / w[RHO];
}

int orc_cfl(orc_mesh* m, const orc_params* pr, double* dt_out) {
  geom g = mesh_geom(m);
  int nd = m->ndim;
  for (int p = 0; p < m->nprob; ++p) {
    double ag = 0.0, mindx = INFINITY, kmax = 0.0;
    for (int q = 0; q < m->nblocks; ++q) {
      const oblk* o = &m->b[q];
      if (o->leaf < 0 || o->problem != p) continue;
      double dx[3];
      block_dx(m, o, dx);
      for (int d = 0; d < nd; ++d) if (dx[d] < mindx) mindx = dx[d];
      FOR_REGION(&g, NG, k, j, i) {
        double w[NV];
        load(&g, o->u, cidx(&g, k, j, i), w);
        for (int d = 0; d < nd; ++d) {
          double a = orc_alpha(d, w, pr->gamma);
          if (a > ag || a != a) ag = a;
        }
        if (pr->conduction) {
          const double kt = conduction_rate(w, pr);
          if (kt > kmax || kt != kt) kmax = kt;
        }
      }
    }
    /* alpha_g: global maximal wave speed; a fixed c_h is a signal speed too */
    double sig = ag;
    if (pr->ch_mode == 2 && pr->ch > sig) sig = pr->ch;
    double dt = pr->c_cfl * mindx / ((double)nd * sig);
    if (pr->eta > 0.0) {
      double dtr = pr->c_cfl * mindx * mindx / (2.0 * (double)nd * pr->eta);
      if (dtr < dt) dt = dtr;
    }
    /* thermal conduction (Sec. 3.6): dt_c = c_cfl min(dx)^2 / (n_dim max(kappa T / p)); without
     * the subcycle it bounds the step itself */
    double dtc = INFINITY;
    if (pr->conduction && kmax > 0.0) dtc = pr->c_cfl * mindx * mindx / ((double)nd * kmax);
    if (pr->conduction && !pr->subcycle && dtc < dt) dt = dtc;
    if (pr->dt_override > 0.0) dt = pr->dt_override;
    m->dtc[p] = dtc;
    double ch;
    if (pr->ch_mode == 0) ch = ag;
    else if (pr->ch_mode == 1) ch = pr->c_cfl * mindx / dt;
    else ch = pr->ch;
    double cp = pr->cp_mode == 0 ? sqrt(-dt * ch * ch / log(pr->c_d)) : pr->cp;
    double damp = cp > 0.0 ? exp(-dt * ch * ch / (cp * cp)) : 1.0;
    m->dt[p] = dt; m->ch[p] = ch; m->cp[p] = cp; m->damp[p] = damp; m->alpha_g[p] = ag;
    if (dt_out) dt_out[p] = dt;
  }
  m->have_dt = 1;
  for (int p = 0; p < m->nprob; ++p)
    if (!isfinite(m->dt[p]) || !(m->dt[p] > 0.0)) return -2;
  return 0;
}

int orc_get_speeds(const orc_mesh* m, double* out) {
  for (int p = 0; p < m->nprob; ++p) {
    out[5 * p + 0] = m->dt[p]; out[5 * p + 1] = m->ch[p]; out[5 * p + 2] = m->cp[p];
    out[5 * p + 3] = m->damp[p]; out[5 * p + 4] = m->alpha_g[p];
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* One step over all leaves.                                                                */

static int check_state(const orc_mesh* m, double gamma) {
  geom g = mesh_geom(m);
  int status = 0;
  for (int q = 0; q < m->nblocks; ++q) {
    const oblk* o = &m->b[q];
    if (o->leaf < 0) continue;
    FOR_REGION(&g, NG, k, j, i) {
      double w[NV];
      load(&g, o->u, cidx(&g, k, j, i), w);
      for (int v = 0; v < NV; ++v) if (!isfinite(w[v])) return -2;
      if (w[RHO] <= 0.0 || pressure(w, gamma) < 0.0) status = -3;
    }
  }
  return status;
}

static stepctx make_ctx(const orc_mesh* m, const orc_params* pr, const oblk* o) {
  stepctx s;
  s.gamma = pr->gamma; s.eta = pr->eta; s.eglm = pr->eglm; s.limiter = pr->limiter;
  s.dt = m->dt[o->problem]; s.ch = m->ch[o->problem];
  block_dx(m, o, s.dx);
  s.riemann = pr->riemann;
  s.freg = NULL;
  s.fw = 1.0;
  return s;
}

/* Reflux (Sec. 4.2 step (2), after Berger and Colella): a coarse leaf whose same-level
 * neighbour across a face is refined has updated its cells next to that face with its own
 * flux there, while the fine leaves on the other side used theirs.  The coarse flux of each
 * face cell is replaced by the mean of the 2^(ndim-1) fine fluxes covering it:
 *   u_c += lam (F_fine - F_coarse) on a low face,  u_c -= lam (F_fine - F_coarse) on a high
 * face, lam = dt / dx_d of the coarse block, so every face carries one flux on both sides.
 * Faces are applied in the order (d, low then high); fine means sum in the order
 * (t0, t0+1) and, in 3D, ((f[t1][t0] + f[t1][t0+1]) + (f[t1+1][t0] + f[t1+1][t0+1])). */
static void apply_reflux(orc_mesh* m, const double* freg) {
  const int nd = m->ndim, nb = m->nb, h = nb / 2;
  const size_t nb2 = (size_t)nb * nb, per = (size_t)2 * nd * NV * nb2;
  geom g = mesh_geom(m);
  for (int q = 0; q < m->nblocks; ++q) {
    oblk* o = &m->b[q];
    if (o->leaf < 0) continue;
    const int L = o->level, p = o->problem;
    double dx[3];
    block_dx(m, o, dx);
    for (int d = 0; d < nd; ++d)
      for (int side = 0; side < 2; ++side) {
        int nbc[3] = {o->ijk[0], o->ijk[1], o->ijk[2]};
        nbc[d] += side ? 1 : -1;
        const int n = nblk_dim(m, p, L, d);
        if (nbc[d] < 0 || nbc[d] >= n) {
          if (m->probs[p].bc[d][side] != 0) continue;        /* outflow: no neighbour */
          nbc[d] = (nbc[d] % n + n) % n;
        }
        const int nq = lookup(m, p, L, nbc[0], nbc[1], nbc[2]);
        if (nq < 0 || m->b[nq].leaf >= 0) continue;           /* coarser or same level */
        const oblk* nbk = &m->b[nq];
        const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
        const double lam = m->dt[p] / dx[d];
        const double* rc = freg + (size_t)q * per + (size_t)(2 * d + side) * NV * nb2;
        for (int t1 = 0; t1 < (nd == 3 ? nb : 1); ++t1)
          for (int t0 = 0; t0 < nb; ++t0) {
            int bits[3] = {0, 0, 0};
            bits[d] = side ? 0 : 1;
            bits[da] = t0 / h;
            if (nd == 3) bits[db] = t1 / h;
            const int cq = nbk->child[bits[0] | (bits[1] << 1) | (bits[2] << 2)];
            const double* rf = freg + (size_t)cq * per + (size_t)(2 * d + 1 - side) * NV * nb2;
            const int f0 = 2 * (t0 - bits[da] * h), f1 = nd == 3 ? 2 * (t1 - bits[db] * h) : 0;
            int ci[3];
            ci[d] = side ? nb - 1 : 0;
            ci[da] = t0;
            if (nd == 3) ci[db] = t1;
            const int c = cidx(&g, nd == 3 ? ci[2] + NG : 0, ci[1] + NG, ci[0] + NG);
            for (int v = 0; v < NV; ++v) {
              const double* fv = rf + v * nb2;
              double ff;
              if (nd == 2) ff = 0.5 * (fv[f0] + fv[f0 + 1]);
              else ff = 0.25 * ((fv[(size_t)f1 * nb + f0] + fv[(size_t)f1 * nb + f0 + 1]) +
                                (fv[(size_t)(f1 + 1) * nb + f0] + fv[(size_t)(f1 + 1) * nb + f0 + 1]));
              const double corr = lam * (ff - rc[v * nb2 + (size_t)t1 * nb + t0]);
              o->u[v * g.S + c] = side ? o->u[v * g.S + c] - corr : o->u[v * g.S + c] + corr;
            }
          }
      }
  }
}

static void copy_interior(const geom* g, const double* src, double* dst) {
  FOR_REGION(g, NG, k, j, i) {
    int c = cidx(g, k, j, i);
    for (int v = 0; v < NV; ++v) dst[v * g->S + c] = src[v * g->S + c];
  }
}

/* ------------------------------------------------------------------------------------ */
/* Thermal conduction (Sec. 3.6, and the field-aligned form of the Sec. 5 test).            */

/* One conduction update of the energy of a ghost-filled block over h (interior written to
 * e_out[nz*nb*nb]):  e_i += h sum_d (F_d,i+1/2 - F_d,i-1/2) / dx_d  with
 *   isotropic:     F = sqrt(kappa_i kappa_i+1) (T_i+1 - T_i) / dx_d   (the paper's scheme),
 *   field-aligned: F = sqrt(kappa_i kappa_i+1) b_d (b . grad T)   at the face, b = B_f/|B_f|
 *                  with B_f the mean of the two cells' B, the normal derivative as above and
 *                  each transverse derivative the mean of the two cells' central differences
 *                  (no flux where B_f = 0).
 * A face temperature gradient beyond gradT_max (> 0) is clipped to it.  Boundary face fluxes go
 * to the face register (energy slot) when one is given. */
static void conduction_block(const geom* g, const stepctx* s, const orc_params* pr, const double* u,
                             double h, double* e_out) {
  const int nd = g->ndim, nb = g->nb;
  double* T = (double*)calloc((size_t)g->S, sizeof(double));
  double* K = (double*)calloc((size_t)g->S, sizeof(double));
  FOR_REGION(g, 1, k, j, i) {
    const int c = cidx(g, k, j, i);
    double w[NV];
    load(g, u, c, w);
    T[c] = temperature(w, pr->gamma);
    K[c] = kappa_of(T[c], pr->kappa0);
  }
  int q = 0;
  FOR_REGION(g, NG, k, j, i) {
    const int c = cidx(g, k, j, i);
    double acc = 0.0;
    for (int d = 0; d < nd; ++d) {
      const int o = g->off[d];
      double F[2];
      for (int side = 0; side < 2; ++side) {
        const int cl = side ? c : c - o, cr = cl + o;      /* face between cl and cr */
        double gn = (T[cr] - T[cl]) / s->dx[d];
        if (pr->grad_t_max > 0.0) gn = fmax(-pr->grad_t_max, fmin(pr->grad_t_max, gn));
        const double kf = sqrt(K[cl] * K[cr]);
        if (pr->conduction == 1) {
          F[side] = kf * gn;
        } else {
          double bf[3], b2 = 0.0;
          for (int j2 = 0; j2 < 3; ++j2) {
            bf[j2] = 0.5 * (u[(BX + j2) * g->S + cl] + u[(BX + j2) * g->S + cr]);
            b2 += bf[j2] * bf[j2];
          }
          if (!(b2 > 0.0)) {
            F[side] = 0.0;
          } else {
            double bg = bf[d] * gn;
            for (int t = 0; t < nd; ++t) {
              if (t == d) continue;
              const int ot = g->off[t];
              double gt = 0.5 * ((T[cl + ot] - T[cl - ot]) / (2.0 * s->dx[t]) +
                                 (T[cr + ot] - T[cr - ot]) / (2.0 * s->dx[t]));
              if (pr->grad_t_max > 0.0) gt = fmax(-pr->grad_t_max, fmin(pr->grad_t_max, gt));
              bg += bf[t] * gt;
            }
            F[side] = kf * bf[d] * bg / b2;
          }
        }
      }
      if (icoord(d, k, j, i) == 0 && s->freg) {
        double f9[NV] = {0};
        f9[EN] = -F[0];                    /* as a flux of e along +d: e -= h dF/dx */
        record_face(g, s, d, 0, k, j, i, f9);
      }
      if (icoord(d, k, j, i) == nb - 1 && s->freg) {
        double f9[NV] = {0};
        f9[EN] = -F[1];
        record_face(g, s, d, 1, k, j, i, f9);
      }
      acc += (F[1] - F[0]) / s->dx[d];
    }
    e_out[q++] = u[EN * g->S + c] + h * acc;
  }
  free(T);
  free(K);
}

/* The conduction part of a step over dt: n substeps of dt/n, n = ceil(dt / dt_c) with the
 * subcycle (dt_c of the last CFL reduction, i.e. the state before the MHD update), else one.
 * Each substep refills the ghosts and, on AMR, refluxes the energy at coarse/fine faces. */
static void conduction_step(orc_mesh* m, const orc_params* pr) {
  geom g = mesh_geom(m);
  const int nd = m->ndim, nb = m->nb;
  const int ncell = (nd == 3 ? nb : 1) * nb * nb;
  const size_t per = (size_t)2 * nd * NV * nb * nb;
  int nsub = 1;
  for (int p = 0; p < m->nprob; ++p)
    if (pr->subcycle && m->dtc[p] < m->dt[p]) {
      const int n = (int)ceil(m->dt[p] / m->dtc[p]);
      if (n > nsub) nsub = n;
    }
  double* hsub = (double*)malloc(sizeof(double) * (size_t)m->nprob);
  double* dtsave = (double*)malloc(sizeof(double) * (size_t)m->nprob);
  for (int p = 0; p < m->nprob; ++p) {
    int n = 1;
    if (pr->subcycle && m->dtc[p] < m->dt[p]) n = (int)ceil(m->dt[p] / m->dtc[p]);
    hsub[p] = m->dt[p] / (double)n;
    dtsave[p] = m->dt[p];
  }
  double* enew = (double*)malloc(sizeof(double) * (size_t)m->nblocks * ncell);
  double* freg = (pr->reflux && m->maxlev > 0) ? (double*)malloc((size_t)m->nblocks * per * sizeof(double)) : NULL;
  for (int it = 0; it < nsub; ++it) {
    orc_fill_ghosts(m);
    if (freg) memset(freg, 0, (size_t)m->nblocks * per * sizeof(double));
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->leaf < 0) continue;
      int n = 1;
      if (pr->subcycle && m->dtc[o->problem] < m->dt[o->problem]) n = (int)ceil(m->dt[o->problem] / m->dtc[o->problem]);
      if (it >= n) continue;                       /* this problem needs fewer substeps */
      stepctx s = make_ctx(m, pr, o);
      if (freg) s.freg = freg + (size_t)q * per;
      conduction_block(&g, &s, pr, o->u, hsub[o->problem], enew + (size_t)q * ncell);
    }
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->leaf < 0) continue;
      int n = 1;
      if (pr->subcycle && m->dtc[o->problem] < m->dt[o->problem]) n = (int)ceil(m->dt[o->problem] / m->dtc[o->problem]);
      if (it >= n) continue;
      int c = 0;
      FOR_REGION(&g, NG, k, j, i) o->u[EN * g.S + cidx(&g, k, j, i)] = enew[(size_t)q * ncell + c++];
    }
    if (freg) {
      /* the energy flux of this substep, refluxed with lam = h / dx */
      for (int p = 0; p < m->nprob; ++p) m->dt[p] = hsub[p];
      apply_reflux(m, freg);
      for (int p = 0; p < m->nprob; ++p) m->dt[p] = dtsave[p];
    }
  }
  free(enew);
  free(freg);
  free(hsub);
  free(dtsave);
}

/* The conduction part alone over dt (its time step from the current state), for the pins. */
int orc_conduct(orc_mesh* m, const orc_params* pr, double dt) {
  geom g = mesh_geom(m);
  const int nd = m->ndim;
  for (int p = 0; p < m->nprob; ++p) {
    double mindx = INFINITY, kmax = 0.0;
    for (int q = 0; q < m->nblocks; ++q) {
      const oblk* o = &m->b[q];
      if (o->leaf < 0 || o->problem != p) continue;
      double dx[3];
      block_dx(m, o, dx);
      for (int d = 0; d < nd; ++d) if (dx[d] < mindx) mindx = dx[d];
      FOR_REGION(&g, NG, k, j, i) {
        double w[NV];
        load(&g, o->u, cidx(&g, k, j, i), w);
        const double kt = conduction_rate(w, pr);
        if (kt > kmax || kt != kt) kmax = kt;
      }
    }
    m->dtc[p] = kmax > 0.0 ? pr->c_cfl * mindx * mindx / ((double)nd * kmax) : INFINITY;
    m->dt[p] = dt;
  }
  conduction_step(m, pr);
  return check_state(m, pr->gamma);
}

int orc_get_dtc(const orc_mesh* m, double* out) {
  for (int p = 0; p < m->nprob; ++p) out[p] = m->dtc[p];
  return 0;
}

int orc_step(orc_mesh* m, const orc_params* pr) {
  if (!m->have_dt) return -1;
  geom g = mesh_geom(m);
  /* face registers for reflux, only where a coarse/fine face can exist */
  const size_t per = (size_t)2 * m->ndim * NV * m->nb * m->nb;
  double* freg = (pr->reflux && m->maxlev > 0) ? (double*)calloc((size_t)m->nblocks * per, sizeof(double)) : NULL;
  if (pr->scheme == 0 || pr->scheme == 1) {
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->leaf < 0) continue;
      stepctx s = make_ctx(m, pr, o);
      if (freg) s.freg = freg + (size_t)q * per;
      double* out = (double*)calloc((size_t)NV * g.S, sizeof(double));
      if (pr->scheme == 0) mmc_block(&g, &s, o->u, out);
      else lf_block(&g, &s, o->u, out);
      copy_interior(&g, out, o->u);
      free(out);
    }
  } else if (pr->scheme == 2) {
    /* TVD Runge-Kutta 2 (Sec. 3.3): u1 = u + dt L(u); u^{n+1} = (u + u1 + dt L(u1))/2,
     * with the ghosts of u1 refilled between the stages. */
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->leaf < 0) continue;
      stepctx s = make_ctx(m, pr, o);
      if (freg) s.freg = freg + (size_t)q * per;
      s.fw = 0.5;
      double* L = (double*)calloc((size_t)NV * g.S, sizeof(double));
      weno_rhs(&g, &s, o->u, L);
      FOR_REGION(&g, NG, k, j, i) {
        int c = cidx(&g, k, j, i);
        for (int v = 0; v < NV; ++v) o->u1[v * g.S + c] = o->u[v * g.S + c] + s.dt * L[v * g.S + c];
        FLOPS(2 * NV);
      }
      free(L);
    }
    for (int q = 0; q < m->nblocks; ++q) { double* t = m->b[q].u; m->b[q].u = m->b[q].u1; m->b[q].u1 = t; }
    orc_fill_ghosts(m);
#pragma omp parallel for schedule(dynamic)
    for (int q = 0; q < m->nblocks; ++q) {
      oblk* o = &m->b[q];
      if (o->leaf < 0) continue;
      stepctx s = make_ctx(m, pr, o);
      if (freg) s.freg = freg + (size_t)q * per;
      s.fw = 0.5;
      double* L = (double*)calloc((size_t)NV * g.S, sizeof(double));
      weno_rhs(&g, &s, o->u, L);
      FOR_REGION(&g, NG, k, j, i) {
        int c = cidx(&g, k, j, i);
        for (int v = 0; v < NV; ++v) {
          double un = o->u1[v * g.S + c], us = o->u[v * g.S + c];
          o->u1[v * g.S + c] = 0.5 * ((un + us) + s.dt * L[v * g.S + c]);
        }
        FLOPS(4 * NV);
      }
      free(L);
    }
    for (int q = 0; q < m->nblocks; ++q) { double* t = m->b[q].u; m->b[q].u = m->b[q].u1; m->b[q].u1 = t; }
  } else {
    free(freg);
    return -1;
  }
  if (freg) {
    apply_reflux(m, freg);
    free(freg);
  }
  /* psi damping, exact operator split once per step: psi <- psi exp(-dt c_h^2/c_p^2)
   * (eq. MHD-5 source; equals c_d when c_p comes from the same dt). */
  for (int q = 0; q < m->nblocks; ++q) {
    oblk* o = &m->b[q];
    if (o->leaf < 0) continue;
    double damp = m->damp[o->problem];
    FOR_REGION(&g, NG, k, j, i) {
      o->u[PSI * g.S + cidx(&g, k, j, i)] *= damp;
      FLOPS(1);
    }
  }
  if (pr->conduction) conduction_step(m, pr);
  m->have_dt = 0;
  FLCAT(3);
  const int rc = check_state(m, pr->gamma);
  FLCAT(2);
  return rc;
}

int orc_block_step(int ndim, int nb, const orc_params* pr, const double* dx, double dt,
                   double ch, double damp, const double* in, double* interior_out) {
  if (pr->scheme != 0 && pr->scheme != 1) return -1;
  geom g = make_geom(ndim, nb);
  stepctx s;
  s.gamma = pr->gamma; s.eta = pr->eta; s.eglm = pr->eglm; s.limiter = pr->limiter;
  s.dt = dt; s.ch = ch;
  for (int d = 0; d < 3; ++d) s.dx[d] = dx[d];
  s.riemann = pr->riemann;
  s.freg = NULL;
  s.fw = 1.0;
  double* out = (double*)calloc((size_t)NV * g.S, sizeof(double));
  if (pr->scheme == 0) mmc_block(&g, &s, in, out);
  else lf_block(&g, &s, in, out);
  int nz = ndim == 3 ? nb : 1, q = 0;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          double val = out[v * g.S + cidx(&g, ndim == 3 ? k + NG : 0, j + NG, i + NG)];
          interior_out[q++] = (v == PSI) ? val * damp : val;
        }
  free(out);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Refinement flags (Sec. 4.5).                                                             */

/* The error estimator of one scalar field at cell c:
 *   (B |du|/(|u|+eps) + (1-B) |d2u|/(|du| + F(|u|+eps))) R^(xi (L-1))
 * |du| = sqrt(3)/2 sqrt(sum_d (u_{+1} - u_{-1})^2) (the printed factor is kept),
 * |d2u| = sqrt(sum_d (u_{+1} - 2u + u_{-1})^2), sums over the active dimensions. */
static double estimator(const geom* g, const double* f, int c, double eps, const orc_refine* r,
                        int level) {
  double s1 = 0.0, s2 = 0.0;
  for (int d = 0; d < g->ndim; ++d) {
    int o = g->off[d];
    double d1 = f[c + o] - f[c - o];
    double d2 = f[c + o] - 2.0 * f[c] + f[c - o];
    s1 += d1 * d1;
    s2 += d2 * d2;
  }
  double du = sqrt(3.0) / 2.0 * sqrt(s1);
  double d2u = sqrt(s2);
  double au = fabs(f[c]) + eps;
  double e = r->bias * du / au + (1.0 - r->bias) * d2u / (du + r->filter * au);
  return e * pow(r->ratio, r->xi * (double)(level + 1 - 1));
}

int orc_flags(orc_mesh* m, const orc_params* pr, const orc_refine* r, signed char* flags,
              double* est_max) {
  geom g = mesh_geom(m);
  double* pf = (double*)calloc((size_t)g.S, sizeof(double));
  double* J = (double*)calloc((size_t)3 * g.S, sizeof(double));
  for (int l = 0; l < m->nleaves; ++l) {
    const oblk* o = &m->b[m->leaf_block[l]];
    double dx[3];
    block_dx(m, o, dx);
    double mindx = dx[0];
    for (int d = 1; d < m->ndim; ++d) if (dx[d] < mindx) mindx = dx[d];
    for (int c = 0; c < g.S; ++c) {
      double w[NV];
      load(&g, o->u, c, w);
      pf[c] = pressure(w, pr->gamma);
    }
    if (r->var_mask & 4) current_density(&g, o->u, dx, J);
    double emax = 0.0;
    /* every cell whose +-1 neighbours exist: the interior and the first ghost ring */
    FOR_REGION(&g, 1, k, j, i) {
      int c = cidx(&g, k, j, i);
      if (r->var_mask & 1) {
        double e = estimator(&g, o->u + RHO * g.S, c, r->eps_rho, r, o->level);
        if (e > emax) emax = e;
      }
      if (r->var_mask & 2) {
        double e = estimator(&g, pf, c, r->eps_p, r, o->level);
        if (e > emax) emax = e;
      }
      if (r->var_mask & 4) {
        /* reading for the current sheet: |J| dx / (|B| + eps_B), J by central differences */
        double jx = J[c], jy = J[g.S + c], jz = J[2 * g.S + c];
        double bx = o->u[BX * g.S + c], by = o->u[BY * g.S + c], bz = o->u[BZ * g.S + c];
        double e = sqrt(jx * jx + jy * jy + jz * jz) * mindx /
                   (sqrt(bx * bx + by * by + bz * bz) + r->eps_b);
        if (e > emax) emax = e;
      }
    }
    signed char f = 0;
    if (emax > r->thr && o->level < r->max_level) f = 1;
    else if (emax < r->coarsen_thr && o->level > 0) f = -1;
    flags[l] = f;
    if (est_max) est_max[l] = emax;
  }
  free(pf);
  free(J);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Conservation sums: sum over leaf cells of U * cell volume, per problem.                 */

int orc_conservation(const orc_mesh* m, double* sums) {
  geom g = mesh_geom(m);
  memset(sums, 0, sizeof(double) * (size_t)m->nprob * NV);
  for (int l = 0; l < m->nleaves; ++l) {
    const oblk* o = &m->b[m->leaf_block[l]];
    double dx[3], vol = 1.0;
    block_dx(m, o, dx);
    for (int d = 0; d < m->ndim; ++d) vol *= dx[d];
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      FOR_REGION(&g, NG, k, j, i) s += o->u[v * g.S + cidx(&g, k, j, i)];
      sums[o->problem * NV + v] += s * vol;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Regrid: a new leaf set; kept leaves copy, new children are prolonged from their old leaf
 * parent (same formula as the ghost prolongation, applied to interior cells), new parents
 * take the restriction of their old descendants.  Ghosts of the old mesh must be filled. */

orc_mesh* orc_regrid(orc_mesh* m, int nleaves, const int* leaves, int* err) {
  orc_mesh* n = orc_create(m->ndim, m->nb, m->nprob, m->probs, nleaves, leaves, err);
  if (!n) return NULL;
  geom g = mesh_geom(m);
  int nd = m->ndim, nb = m->nb, nz = nd == 3 ? nb : 1;
  for (int l = 0; l < nleaves; ++l) {
    oblk* o = &n->b[n->leaf_block[l]];
    int q = lookup(m, o->problem, o->level, o->ijk[0], o->ijk[1], o->ijk[2]);
    if (q >= 0) {
      copy_interior(&g, m->b[q].u, o->u);
      continue;
    }
    int pq = o->level > 0 ? lookup(m, o->problem, o->level - 1, o->ijk[0] >> 1, o->ijk[1] >> 1,
                                   nd == 3 ? o->ijk[2] >> 1 : 0) : -1;
    if (pq < 0 || m->b[pq].leaf < 0) { *err = -6; orc_destroy(n); return NULL; }
    const oblk* P = &m->b[pq];
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          int G[3] = {o->ijk[0] * nb + i, o->ijk[1] * nb + j, nd == 3 ? o->ijk[2] * nb + k : 0};
          int c = cidx(&g, nd == 3 ? (G[2] >> 1) - P->ijk[2] * nb + NG : 0,
                       (G[1] >> 1) - P->ijk[1] * nb + NG, (G[0] >> 1) - P->ijk[0] * nb + NG);
          int cf = cidx(&g, nd == 3 ? k + NG : 0, j + NG, i + NG);
          for (int v = 0; v < NV; ++v) {
            const double* f = P->u + v * g.S;
            double val = f[c];
            for (int d = 0; d < nd; ++d) {
              int off = g.off[d];
              val += minmod(f[c + off] - f[c], f[c] - f[c - off]) * ((G[d] & 1) ? 0.25 : -0.25);
            }
            o->u[v * g.S + cf] = val;
          }
        }
  }
  return n;
}
