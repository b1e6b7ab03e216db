// physics.cuh -- point-wise EGLM-MHD physics on the device, templated on the real type.
//
// Equations: Jiang, Fang & Chen (arXiv:1204.5849) Sec. 2, eqs. MHD-1..MHD-5; the local
// speed |v_d| + fast magnetosonic speed (Sec. 3.1/3.2 "local maximum eigenvalue");
// Lax-Friedrichs flux (Equ:LFFlux); minmod (eq. minmod) and van Leer limiters; the
// two-stencil WENO reconstruction (Sec. 3.3).
//
// The double instantiation is compiled without FMA contraction and keeps one expression
// order per formula, so that it rounds like a plain C implementation of the same formulas.
// The float instantiation stores and computes in FP32; the pressure recovery falls back
// to FP64 where the internal energy is a small fraction of e (cancellation).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mapgb {

constexpr int NV = 9;
enum { RHO = 0, MX = 1, MY = 2, MZ = 3, BX = 4, BY = 5, BZ = 6, EN = 7, PSI = 8 };
constexpr int NG = 2;

template <typename T>
struct Phys {
  T gamma;
  T gm1;       // gamma - 1
  T ch;        // GLM speed c_h
  T tau;       // FP64-fix threshold on e_int / e (float only)
};

template <typename T>
__device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }

// a / b.  FP64: the plain quotient (rounds as the same formula written in plain C).  FP32:
// the fast quotient, reciprocal times numerator (within 2 ulp); every FP32 quotient on the
// step path has a denominator (a density, a cell spacing, a sum of slopes, a WENO weight sum)
// far below the 2^126 range where the fast form flushes to zero.
template <typename T>
__device__ __forceinline__ T qdiv(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// p = (gamma-1) (e - m^2/(2 rho) - B^2/2)   (Sec. 2, total energy density)
template <typename T>
__device__ __forceinline__ T pressure(const T* w, const Phys<T>& P) {
  T m2 = w[MX] * w[MX] + w[MY] * w[MY] + w[MZ] * w[MZ];
  T b2 = w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ];
  return P.gm1 * (w[EN] - T(0.5) * m2 / w[RHO] - T(0.5) * b2);
}

// The FP64 recovery of the pressure from FP32 stored values (the fallback of the FP32 form
// where e_int is a small fraction of e).  Out of line: it runs rarely, and kept inline its
// FP64 registers and code weigh on the hot FP32 path around every pressure.
static __device__ __noinline__ float pressure_fp64(float rho, float mx, float my, float mz, float bx, float by,
                                           float bz, float en, float gm1) {
  const double m2d = (double)mx * mx + (double)my * my + (double)mz * mz;
  const double b2d = (double)bx * bx + (double)by * by + (double)bz * bz;
  const double ed = (double)en - 0.5 * m2d / (double)rho - 0.5 * b2d;
  return (float)((double)gm1 * ed);
}

template <>
__device__ __forceinline__ float pressure<float>(const float* w, const Phys<float>& P) {
  float m2 = w[MX] * w[MX] + w[MY] * w[MY] + w[MZ] * w[MZ];
  float b2 = w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ];
  float kin = 0.5f * m2 * qdiv(1.0f, w[RHO]);
  float eint = w[EN] - kin - 0.5f * b2;
  // low internal-energy fraction: recover p in FP64 from the same stored values
  if (eint < P.tau * w[EN]) return pressure_fp64(w[RHO], w[MX], w[MY], w[MZ], w[BX], w[BY], w[BZ], w[EN], P.gm1);
  return P.gm1 * eint;
}

// Physical flux in direction D of the EGLM-MHD system (eqs. MHD-1..MHD-5, no sources),
// given the pressure p of the state.
template <typename T, int D>
__device__ __forceinline__ void flux_p(const T* w, T p, const Phys<T>& P, T* f) {
  T rho = w[RHO];
  T v0, v1, v2;
  if constexpr (std::is_same<T, float>::value) {
    const T ir = qdiv(T(1), rho);   // one reciprocal per state in FP32
    v0 = w[MX] * ir; v1 = w[MY] * ir; v2 = w[MZ] * ir;
  } else {
    v0 = w[MX] / rho; v1 = w[MY] / rho; v2 = w[MZ] / rho;
  }
  T b2 = w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ];
  T pt = p + T(0.5) * b2;
  T vb = v0 * w[BX] + v1 * w[BY] + v2 * w[BZ];
  T vd = D == 0 ? v0 : (D == 1 ? v1 : v2);
  T bd = w[BX + D];
  T md = w[MX + D];
  f[RHO] = md;
  f[MX] = md * v0 - bd * w[BX];
  f[MY] = md * v1 - bd * w[BY];
  f[MZ] = md * v2 - bd * w[BZ];
  f[MX + D] += pt;
  f[BX] = D == 0 ? w[PSI] : vd * w[BX] - bd * v0;
  f[BY] = D == 1 ? w[PSI] : vd * w[BY] - bd * v1;
  f[BZ] = D == 2 ? w[PSI] : vd * w[BZ] - bd * v2;
  f[EN] = vd * (w[EN] + pt) - bd * vb;
  f[PSI] = P.ch * P.ch * bd;
}

// Local speed in direction D: |v_d| + c_f,d with the pressure clamped at 0 here only.
template <typename T, int D>
__device__ __forceinline__ T alpha_p(const T* w, T p, const Phys<T>& P) {
  T rho = w[RHO];
  if (p < T(0)) p = T(0);
  if constexpr (std::is_same<T, float>::value) {
    const T ir = qdiv(T(1), rho);
    T a2 = P.gamma * p * ir;
    T b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) * ir;
    T bd2 = w[BX + D] * w[BX + D] * ir;
    T s = a2 + b2;
    T disc = s * s - T(4) * a2 * bd2;
    if (disc < T(0)) disc = T(0);
    T cf = sqrtf(T(0.5) * (s + sqrtf(disc)));
    return fabsf(w[MX + D] * ir) + cf;
  } else {
    T a2 = P.gamma * p / rho;
    T b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) / rho;
    T bd2 = w[BX + D] * w[BX + D] / rho;
    T s = a2 + b2;
    T disc = s * s - T(4) * a2 * bd2;
    if (disc < T(0)) disc = T(0);
    T cf = sqrt(T(0.5) * (s + sqrt(disc)));
    return fabs(w[MX + D] / rho) + cf;
  }
}

template <typename T>
__device__ __forceinline__ T alpha_dir(int d, const T* w, T p, const Phys<T>& P) {
  return d == 0 ? alpha_p<T, 0>(w, p, P) : (d == 1 ? alpha_p<T, 1>(w, p, P) : alpha_p<T, 2>(w, p, P));
}

// Fast magnetosonic speed along D (c_f of alpha_p without |v_d|); p = pressure of w.
template <typename T, int D>
__device__ __forceinline__ T fast_speed(const T* w, T p, const Phys<T>& P) {
  T rho = w[RHO];
  if (p < T(0)) p = T(0);
  if constexpr (std::is_same<T, float>::value) {
    const T ir = qdiv(T(1), rho);
    T a2 = P.gamma * p * ir;
    T b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) * ir;
    T bd2 = w[BX + D] * w[BX + D] * ir;
    T s = a2 + b2;
    T disc = s * s - T(4) * a2 * bd2;
    if (disc < T(0)) disc = T(0);
    return sqrtf(T(0.5) * (s + sqrtf(disc)));
  } else {
    T a2 = P.gamma * p / rho;
    T b2 = (w[BX] * w[BX] + w[BY] * w[BY] + w[BZ] * w[BZ]) / rho;
    T bd2 = w[BX + D] * w[BX + D] / rho;
    T s = a2 + b2;
    T disc = s * s - T(4) * a2 * bd2;
    if (disc < T(0)) disc = T(0);
    return sqrt(T(0.5) * (s + sqrt(disc)));
  }
}

// HLLC interface flux for MHD (Gurski's solver, which the paper names for LF and WENO in
// 2D/3D, Sec. 3.2-3.3):
// 1. the linear (B_d, psi) pair keeps its exact upwind flux, the same as in f_m, and fixes
//    the interface normal field B_m = (B_d,a + B_d,b)/2 - (psi_b - psi_a)/(2 c_h);
// 2. both states take B_d = B_m at unchanged gas pressure, E' = E + (B_m^2 - B_d^2)/2;
// 3. speed bounds S_L = min(u - c_f), S_R = max(u + c_f) over the two states (u = v_d);
// 4. S_L >= 0 or S_R <= 0: the upwind physical flux; otherwise the star state on the side
//    of the contact speed S_M = (rho u)_HLL / rho_HLL, whose density, normal momentum and
//    total pressure follow from mass and momentum across S_K, tangential B from the HLL
//    state, tangential momentum and energy from the jump conditions across S_K, and
//    F = F_K + S_K (U*_K - U_K).
template <typename T, int D>
__device__ __forceinline__ void hllc_flux(const T* a, const T* b, const Phys<T>& P, T* f) {
  const T ch = P.ch;
  const T bm = ch > T(0) ? T(0.5) * (a[BX + D] + b[BX + D]) - (b[PSI] - a[PSI]) / (T(2) * ch)
                         : T(0.5) * (a[BX + D] + b[BX + D]);
  T w[2][NV], F[2][NV], u[2], cf[2], pt[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T* q = k ? b : a;
    const T p = pressure<T>(q, P);
#pragma unroll
    for (int v = 0; v < NV; ++v) w[k][v] = q[v];
    w[k][BX + D] = bm;
    w[k][EN] = q[EN] + T(0.5) * (bm * bm - q[BX + D] * q[BX + D]);
    const T pw = pressure<T>(w[k], P);
    flux_p<T, D>(w[k], pw, P, F[k]);
    u[k] = w[k][MX + D] / w[k][RHO];
    cf[k] = fast_speed<T, D>(w[k], pw, P);
    pt[k] = p + T(0.5) * (w[k][BX] * w[k][BX] + w[k][BY] * w[k][BY] + w[k][BZ] * w[k][BZ]);
  }
  const T sl = fmin(u[0] - cf[0], u[1] - cf[1]);
  const T sr = fmax(u[0] + cf[0], u[1] + cf[1]);
  if (sl >= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = F[0][v];
  } else if (sr <= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = F[1][v];
  } else {
    const T ra = w[0][RHO], rb = w[1][RHO];
    const T sm = (rb * u[1] * (sr - u[1]) - ra * u[0] * (sl - u[0]) - pt[1] + pt[0]) /
                 (rb * (sr - u[1]) - ra * (sl - u[0]));
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;   // tangential dimensions
    const T bt1 = (sr * w[1][BX + T1] - sl * w[0][BX + T1] - (F[1][BX + T1] - F[0][BX + T1])) / (sr - sl);
    const T bt2 = (sr * w[1][BX + T2] - sl * w[0][BX + T2] - (F[1][BX + T2] - F[0][BX + T2])) / (sr - sl);
    const int k = sm >= T(0) ? 0 : 1;
    const T sk = k ? sr : sl;
    T wk[NV], Fk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wk[v] = k ? w[1][v] : w[0][v];
      Fk[v] = k ? F[1][v] : F[0][v];
    }
    const T uk = k ? u[1] : u[0], ptk = k ? pt[1] : pt[0];
    const T dk = sk - uk, ds = sk - sm;
    const T rs = wk[RHO] * dk / ds;
    const T pts = ptk + wk[RHO] * dk * (sm - uk);
    const T vbk = (wk[MX] / wk[RHO]) * wk[BX] + (wk[MX + 1] / wk[RHO]) * wk[BY] + (wk[MX + 2] / wk[RHO]) * wk[BZ];
    T us[NV];
    us[RHO] = rs;
    us[MX + D] = rs * sm;
    us[MX + T1] = rs * (wk[MX + T1] / wk[RHO]) - bm * (bt1 - wk[BX + T1]) / ds;
    us[MX + T2] = rs * (wk[MX + T2] / wk[RHO]) - bm * (bt2 - wk[BX + T2]) / ds;
    T vbs = sm * bm;
    vbs += (us[MX + T1] / rs) * bt1;
    vbs += (us[MX + T2] / rs) * bt2;
    us[BX + D] = bm;
    us[BX + T1] = bt1;
    us[BX + T2] = bt2;
    us[EN] = (wk[EN] * dk - ptk * uk + pts * sm + bm * (vbk - vbs)) / ds;
    us[PSI] = wk[PSI];
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = Fk[v] + sk * (us[v] - wk[v]);
  }
  f[BX + D] = T(0.5) * ((a[PSI] + b[PSI]) - ch * (b[BX + D] - a[BX + D]));
  f[PSI] = T(0.5) * ((ch * ch * a[BX + D] + ch * ch * b[BX + D]) - ch * (b[PSI] - a[PSI]));
}

// HLLD interface flux for MHD (Miyoshi & Kusano 2005, which the paper names among MAP's
// approximate Riemann solvers for LF and WENO and compares with HLLC on the Brio-Wu tube,
// Sec. 3.2, Sec. 5).  Five waves: the fast bounds S_L, S_R, the rotational (Alfven) waves
// S*_L = S_M - |B_n|/sqrt(rho*_L), S*_R = S_M + |B_n|/sqrt(rho*_R) and the contact S_M, with
// the normal velocity, total pressure and normal field constant inside the fan.
// 1-3. As in hllc_flux: the (B_d, psi) pair keeps its exact upwind flux and fixes the
//      interface normal field B_n = B_m, both states take it at unchanged gas pressure, and
//      the fast bounds are S_L = min(u - c_f), S_R = max(u + c_f).
// 4. S_M and p_T* from mass and normal momentum across S_L and S_R together.
// 5. Outer states on each side: rho* = rho d/(S - S_M) (d = S - u), tangential velocity and
//    field from the jump conditions across S, which divide by D = rho d (S - S_M) - B_n^2
//    (velocity and field kept where D vanishes: the fast and Alfven waves coincide there),
//    energy from the energy jump.
// 6. Inner states: tangential velocity and field as the sqrt(rho*)-weighted combination of
//    the two outer states, which the jump conditions across both Alfven waves fix; energy
//    from the energy jump across each Alfven wave.
// 7. The flux of the region holding the interface: F_K + S_K (U*_K - U_K), plus
//    S*_K (U**_K - U*_K) in the inner region, K the side of the contact.  Only that side's
//    states are built; the inner states need both sides' outer velocity, field and density.
template <typename T, int D>
__device__ __forceinline__ void hlld_flux(const T* a, const T* b, const Phys<T>& P, T* f) {
  const T ch = P.ch;
  const T bm = ch > T(0) ? T(0.5) * (a[BX + D] + b[BX + D]) - (b[PSI] - a[PSI]) / (T(2) * ch)
                         : T(0.5) * (a[BX + D] + b[BX + D]);
  T w[2][NV], F[2][NV], u[2], cf[2], pt[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T* q = k ? b : a;
    const T p = pressure<T>(q, P);
#pragma unroll
    for (int v = 0; v < NV; ++v) w[k][v] = q[v];
    w[k][BX + D] = bm;
    w[k][EN] = q[EN] + T(0.5) * (bm * bm - q[BX + D] * q[BX + D]);
    const T pw = pressure<T>(w[k], P);
    flux_p<T, D>(w[k], pw, P, F[k]);
    u[k] = w[k][MX + D] / w[k][RHO];
    cf[k] = fast_speed<T, D>(w[k], pw, P);
    pt[k] = p + T(0.5) * (w[k][BX] * w[k][BX] + w[k][BY] * w[k][BY] + w[k][BZ] * w[k][BZ]);
  }
  const T sl = fmin(u[0] - cf[0], u[1] - cf[1]);
  const T sr = fmax(u[0] + cf[0], u[1] + cf[1]);
  if (sl >= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = F[0][v];
  } else if (sr <= T(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = F[1][v];
  } else {
    constexpr int T1 = D == 0 ? 1 : 0, T2 = D == 2 ? 1 : 2;   // tangential dimensions
    const T dl = sl - u[0], dr = sr - u[1];
    const T ra = w[0][RHO], rb = w[1][RHO];
    const T den = dr * rb - dl * ra;
    const T sm = (dr * rb * u[1] - dl * ra * u[0] - pt[1] + pt[0]) / den;
    const T pts = (dr * rb * pt[0] - dl * ra * pt[1] + ra * rb * dr * dl * (u[1] - u[0])) / den;
    // outer-state velocity and field (absolute components), density, v*.B*, both sides
    T vs[2][3], bs[2][3], rs[2], vbs[2];
    const T tiny = sizeof(T) == 4 ? T(1e-6) : T(1e-12);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const T rho = w[k][RHO], dk = (k ? sr : sl) - u[k], ds = (k ? sr : sl) - sm;
      rs[k] = rho * dk / ds;
      const T Dk = rho * dk * ds - bm * bm;
      const bool flat = fabs(Dk) <= tiny * (fabs(rho * dk * ds) + bm * bm);
      vs[k][D] = sm;
      bs[k][D] = bm;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = t ? T2 : T1;
        const T vt = w[k][MX + j] / rho, bt = w[k][BX + j];
        vs[k][j] = flat ? vt : vt - bm * bt * (sm - u[k]) / Dk;
        bs[k][j] = flat ? bt : bt * (rho * dk * dk - bm * bm) / Dk;
      }
      vbs[k] = vs[k][0] * bs[k][0] + vs[k][1] * bs[k][1] + vs[k][2] * bs[k][2];
    }
    const int k = sm >= T(0) ? 0 : 1;
    const T sk = k ? sr : sl;
    T wk[NV], Fk[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wk[v] = k ? w[1][v] : w[0][v];
      Fk[v] = k ? F[1][v] : F[0][v];
    }
    const T uk = k ? u[1] : u[0], ptk = k ? pt[1] : pt[0];
    const T dk = sk - uk, ds = sk - sm;
    const T rsk = k ? rs[1] : rs[0], vbsk = k ? vbs[1] : vbs[0];
    T vb = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) vb += (wk[MX + j] / wk[RHO]) * wk[BX + j];
    T us[NV];
    us[RHO] = rsk;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      us[MX + j] = rsk * (k ? vs[1][j] : vs[0][j]);
      us[BX + j] = k ? bs[1][j] : bs[0][j];
    }
    us[EN] = (dk * wk[EN] - ptk * uk + pts * sm + bm * (vb - vbsk)) / ds;
    us[PSI] = wk[PSI];
    const T sgn = bm > T(0) ? T(1) : (bm < T(0) ? T(-1) : T(0));
    const T rl = sqrt(rs[0]), rr = sqrt(rs[1]);
    const T ssk = k ? sm + fabs(bm) / rr : sm - fabs(bm) / rl;
    // left of the contact the inner region lies right of S*_L, right of it left of S*_R
    const bool inner = k ? ssk >= T(0) : ssk < T(0);
    if (inner) {
      T vss[3], bss[3];
      vss[D] = sm;
      bss[D] = bm;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = t ? T2 : T1;
        vss[j] = (rl * vs[0][j] + rr * vs[1][j] + sgn * (bs[1][j] - bs[0][j])) / (rl + rr);
        bss[j] = (rl * bs[1][j] + rr * bs[0][j] + sgn * rl * rr * (vs[1][j] - vs[0][j])) / (rl + rr);
      }
      const T vbss = vss[0] * bss[0] + vss[1] * bss[1] + vss[2] * bss[2];
      T uss[NV];
      uss[RHO] = rsk;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        uss[MX + j] = rsk * vss[j];
        uss[BX + j] = bss[j];
      }
      uss[EN] = k ? us[EN] + sgn * rr * (vbsk - vbss) : us[EN] - sgn * rl * (vbsk - vbss);
      uss[PSI] = wk[PSI];
#pragma unroll
      for (int v = 0; v < NV; ++v) f[v] = Fk[v] + sk * (us[v] - wk[v]) + ssk * (uss[v] - us[v]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) f[v] = Fk[v] + sk * (us[v] - wk[v]);
    }
  }
  f[BX + D] = T(0.5) * ((a[PSI] + b[PSI]) - ch * (b[BX + D] - a[BX + D]));
  f[PSI] = T(0.5) * ((ch * ch * a[BX + D] + ch * ch * b[BX + D]) - ch * (b[PSI] - a[PSI]));
}

// Dissipation speed of component v in direction D: the (B_d, psi) pair uses c_h.
template <int D>
__device__ __forceinline__ bool glm_pair(int v) { return v == BX + D || v == PSI; }

// Lax-Friedrichs flux f_m(a,b) = (f(a) + f(b) - alpha (b - a))/2 (Equ:LFFlux),
// alpha = max of the two states' local speeds; c_h for the (B_d, psi) pair.
template <typename T, int D>
__device__ __forceinline__ void lf_flux(const T* a, const T* b, const Phys<T>& P, T* f) {
  T fa[NV], fb[NV];
  T pa = pressure<T>(a, P), pb = pressure<T>(b, P);
  flux_p<T, D>(a, pa, P, fa);
  flux_p<T, D>(b, pb, P, fb);
  T aa = alpha_p<T, D>(a, pa, P), ab = alpha_p<T, D>(b, pb, P);
  T al = aa > ab ? aa : ab;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T s = glm_pair<D>(v) ? P.ch : al;
    f[v] = T(0.5) * ((fa[v] + fb[v]) - s * (b[v] - a[v]));
  }
}

// minmod(a,b) = sgn(a) max(0, min(|a|, sgn(a) b)), written without branches: the smaller
// magnitude with the common sign where a and b are both positive or both negative, else +0
// (bitwise the value of the branching form for every input, signed zeros and NaN included)
template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
  const T m = fmin(fabs(a), fabs(b));
  const bool pos = a > T(0) && b > T(0);
  const bool neg = a < T(0) && b < T(0);
  return pos ? m : (neg ? -m : T(0));
}

// limiter(a, b): 0 minmod, 1 van Leer (2ab/(a+b) when ab > 0, else 0)
template <typename T, int LIM>
__device__ __forceinline__ T limiter(T a, T b) {
  if (LIM == 0) return minmod<T>(a, b);
  return (a * b > T(0)) ? qdiv(T(2) * a * b, a + b) : T(0);
}

// WENO two-stencil reconstruction around u0 (Sec. 3.3): the left state of the face on
// the + side and the right state of the face on the - side (denominator of the latter
// read as a_{i+1/2} + 2 a_{i-1/2}).
template <typename T>
__device__ __forceinline__ void weno_faces(T um, T u0, T up, T& minus_right, T& plus_left) {
  const T eps = T(1e-12);
  T dp = up - u0, dm = u0 - um;
  T ap = qdiv(T(1), (eps + dp * dp) * (eps + dp * dp));
  T am = qdiv(T(1), (eps + dm * dm) * (eps + dm * dm));
  T wm = T(0.5) * (u0 + up), vm = T(0.5) * (T(3) * u0 - um);
  T wp = T(0.5) * (T(3) * u0 - up), vp = T(0.5) * (u0 + um);
  minus_right = qdiv(T(2) * ap * wm + am * vm, T(2) * ap + am);
  plus_left = qdiv(ap * wp + T(2) * am * vp, ap + T(2) * am);
}

template <typename T>
__device__ __forceinline__ T weno_minus_right(T um, T u0, T up) {
  T a, b;
  weno_faces<T>(um, u0, up, a, b);
  return a;
}

template <typename T>
__device__ __forceinline__ T weno_plus_left(T um, T u0, T up) {
  T a, b;
  weno_faces<T>(um, u0, up, a, b);
  return b;
}

}  // namespace mapgb

// ---- paired FP32 evaluation (sm_100+ f32x2 arithmetic) ---------------------------------
// The two states of a face (or the two half-states u +- phi/2 of the MUSCL-Hancock step)
// are evaluated together, one state per lane of a float2, so each paired instruction does
// the work of two.  Division-free except one reciprocal of rho per state.
namespace mapgb {
namespace pair {

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// van Leer / minmod on two lanes at once
template <int LIM>
__device__ __forceinline__ float2 limiter2(float2 a, float2 b) {
  if (LIM == 0) return make_float2(minmod<float>(a.x, b.x), minmod<float>(a.y, b.y));
  const float2 pr = mul(a, b);
  const float2 s = add(a, b);
  const float2 q = mul(splat(2.0f), pr);
  return make_float2(pr.x > 0.0f ? __fdividef(q.x, s.x) : 0.0f, pr.y > 0.0f ? __fdividef(q.y, s.y) : 0.0f);
}

// pressure of two states (same FP64 fallback rule as pressure<float>); OOL: the FP64
// recovery out of line (as pressure<float> has it) or inline, whichever measures faster in
// the calling kernel (inline in the 3D 16^3 kernels, which sit at their register cap)
template <bool OOL>
__device__ __forceinline__ float2 pressure2(const float2* w, const Phys<float>& P, float2 ir) {
  float2 m2 = mul(w[MX], w[MX]);
  m2 = fma(w[MY], w[MY], m2);
  m2 = fma(w[MZ], w[MZ], m2);
  float2 b2 = mul(w[BX], w[BX]);
  b2 = fma(w[BY], w[BY], b2);
  b2 = fma(w[BZ], w[BZ], b2);
  const float2 kin = mul(mul(splat(0.5f), m2), ir);
  const float2 eint = sub(sub(w[EN], kin), mul(splat(0.5f), b2));
  float2 p = mul(splat(P.gm1), eint);
  if constexpr (OOL) {
    if (eint.x < P.tau * w[EN].x)
      p.x = pressure_fp64(w[RHO].x, w[MX].x, w[MY].x, w[MZ].x, w[BX].x, w[BY].x, w[BZ].x, w[EN].x, P.gm1);
    if (eint.y < P.tau * w[EN].y)
      p.y = pressure_fp64(w[RHO].y, w[MX].y, w[MY].y, w[MZ].y, w[BX].y, w[BY].y, w[BZ].y, w[EN].y, P.gm1);
    return p;
  }
  if (eint.x < P.tau * w[EN].x || eint.y < P.tau * w[EN].y) {
    auto fp64 = [&](const float* q) {
      const double m2d = (double)q[MX] * q[MX] + (double)q[MY] * q[MY] + (double)q[MZ] * q[MZ];
      const double b2d = (double)q[BX] * q[BX] + (double)q[BY] * q[BY] + (double)q[BZ] * q[BZ];
      const double ed = (double)q[EN] - 0.5 * m2d / (double)q[RHO] - 0.5 * b2d;
      return (float)((double)P.gm1 * ed);
    };
    float wx[NV], wy[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { wx[v] = w[v].x; wy[v] = w[v].y; }
    if (eint.x < P.tau * w[EN].x) p.x = fp64(wx);
    if (eint.y < P.tau * w[EN].y) p.y = fp64(wy);
  }
  return p;
}

// physical flux in direction D of two states; if alpha != nullptr also their local speeds
template <int D, bool OOL = true>
__device__ __forceinline__ void flux2(const float2* w, const Phys<float>& P, float2* f, float2* alpha) {
  const float2 ir = make_float2(__fdividef(1.0f, w[RHO].x), __fdividef(1.0f, w[RHO].y));
  const float2 p = pressure2<OOL>(w, P, ir);
  const float2 v0 = mul(w[MX], ir), v1 = mul(w[MY], ir), v2 = mul(w[MZ], ir);
  float2 b2 = mul(w[BX], w[BX]);
  b2 = fma(w[BY], w[BY], b2);
  b2 = fma(w[BZ], w[BZ], b2);
  const float2 pt = fma(splat(0.5f), b2, p);
  float2 vb = mul(v0, w[BX]);
  vb = fma(v1, w[BY], vb);
  vb = fma(v2, w[BZ], vb);
  const float2 vd = D == 0 ? v0 : (D == 1 ? v1 : v2);
  const float2 bd = w[BX + D];
  const float2 md = w[MX + D];
  const float2 nbd = make_float2(-bd.x, -bd.y);
  f[RHO] = md;
  f[MX] = fma(nbd, w[BX], mul(md, v0));
  f[MY] = fma(nbd, w[BY], mul(md, v1));
  f[MZ] = fma(nbd, w[BZ], mul(md, v2));
  f[MX + D] = add(f[MX + D], pt);
  f[BX] = D == 0 ? w[PSI] : fma(nbd, v0, mul(vd, w[BX]));
  f[BY] = D == 1 ? w[PSI] : fma(nbd, v1, mul(vd, w[BY]));
  f[BZ] = D == 2 ? w[PSI] : fma(nbd, v2, mul(vd, w[BZ]));
  f[EN] = fma(nbd, vb, mul(vd, add(w[EN], pt)));
  f[PSI] = mul(splat(P.ch * P.ch), bd);
  if (alpha) {
    const float2 pc = make_float2(p.x > 0.0f ? p.x : 0.0f, p.y > 0.0f ? p.y : 0.0f);
    const float2 a2 = mul(mul(splat(P.gamma), pc), ir);
    const float2 bb = mul(b2, ir);
    const float2 bd2 = mul(mul(bd, bd), ir);
    const float2 s = add(a2, bb);
    float2 disc = fma(mul(splat(-4.0f), a2), bd2, mul(s, s));
    disc.x = disc.x > 0.0f ? disc.x : 0.0f;
    disc.y = disc.y > 0.0f ? disc.y : 0.0f;
    const float2 inner = mul(splat(0.5f), add(s, make_float2(sqrtf(disc.x), sqrtf(disc.y))));
    const float2 vn = mul(md, ir);
    *alpha = make_float2(fabsf(vn.x) + sqrtf(inner.x), fabsf(vn.y) + sqrtf(inner.y));
  }
}

// Lax-Friedrichs flux of the face whose left state is lane x and right state lane y, less
// pt_ref in its normal-momentum component: that component of each state carries the total
// pressure p + B^2/2, and the offset, the same for every face whose fluxes the update
// subtracts, keeps it from taking the FP32 digits of the small terms added to it
template <int D, bool OOL = true>
__device__ __forceinline__ void lf_flux2(const float2* ab, const Phys<float>& P, float* f, float pt_ref = 0.0f) {
  float2 F[NV], al;
  flux2<D, OOL>(ab, P, F, &al);
  F[MX + D] = sub(F[MX + D], splat(pt_ref));
  const float a = al.x > al.y ? al.x : al.y;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float s = glm_pair<D>(v) ? P.ch : a;
    f[v] = 0.5f * ((F[v].x + F[v].y) - s * (ab[v].y - ab[v].x));
  }
}

}  // namespace pair
}  // namespace mapgb
