// step.cuh -- the fused per-block step kernel (scheme update + sources + psi damping).
//
// Schemes (Jiang, Fang & Chen, arXiv:1204.5849):
//   MMC  (Sec. 3.1): u~ = u - sum_d dt/dx_d (h_{i+1/2} - h_{i-1/2}), h = f+_i + f-_{i+1};
//        fhat = h + (phi(r+) g+ - phi(r-) g-)/2 with phi(r) g written division-free.
//   LF   (Sec. 3.2): MUSCL-Hancock half step with limited slopes, then f_m (Equ:LFFlux) of
//        the u~ face states built with the same slopes.
//   WENO (Sec. 3.3): two-stencil reconstruction, f_m, TVD Runge-Kutta 2 (one launch per
//        stage; the ghosts of the stage state are refilled in between).
//   Multi-D (Sec. 3.7): unsplit, all directions from the same state.
// Sources: EGLM -(div B) B and -B.grad psi (eqs. MHD-2, MHD-4), resistive R and R_e
// (Sec. 3.5), psi damping exp(-dt c_h^2/c_p^2) once per step (eq. MHD-5).
//
// Layout: a pool block is [9][NZ][NP][NP] with NP = NB + 4 (two ghost layers); NZ = NP in
// 3D and 1 in 2D.  One CTA owns one block at a time (grid-stride over the block list) and
// has NB*NB threads, thread (tx,ty) owning interior column (tx+2, ty+2).  In 3D the CTA
// marches in z keeping a rolling window in shared memory: four u planes (z-1..z+2), three
// u~ planes (z-1..z+1) and, with resistivity, three planes of J; x- and y-face fluxes of
// the current plane go through one shared buffer, the z-face flux of the column is carried
// in registers from one plane to the next.  In 2D the window is the single plane.
#pragma once
#include <type_traits>

#include "map_internal.hpp"
#include "physics.cuh"

namespace mapgb {

enum { SCH_MMC = 0, SCH_LF = 1, SCH_WENO = 2 };

template <typename T>
struct StepArgsT {
  const T* __restrict__ u_in;
  T* __restrict__ u_out;
  const T* __restrict__ u_base;
  const int* __restrict__ blocks;
  int nblocks;
  const BlockGeo* __restrict__ geo;
  const ProbDyn* __restrict__ dyn;
  T gamma, gm1, tau;
  double eta;
  int eglm;
  int resistive;
  unsigned* err_word;
  double* sums;
  ProbDyn* dyn_next;
};

template <int NDIM, int NB>
struct Geo {
  static constexpr int NP = NB + 4;
  static constexpr int P2 = NP * NP;
  static constexpr int NZ = NDIM == 3 ? NP : 1;
  static constexpr int S = NZ * P2;
  static constexpr int NT = NB * NB;
  static constexpr int UPL = NDIM == 3 ? 4 : 1;
  static constexpr int WPL = NDIM == 3 ? 3 : 1;   // u~ and J planes
  static constexpr int RING = (NB + 2) * (NB + 2);
  static constexpr int NFACE = NB * (NB + 1);
};

template <typename T, int NDIM, int NB, int SCHEME>
__host__ __device__ constexpr size_t step_smem_bytes(bool resistive) {
  using G = Geo<NDIM, NB>;
  size_t n = (size_t)G::UPL * NV * G::P2;                          // u window
  if (SCHEME != SCH_WENO) n += (size_t)G::WPL * NV * G::P2;        // u~ window
  n += (size_t)NV * G::NFACE;                                       // face fluxes
  if (resistive) n += (size_t)G::WPL * 3 * G::P2;                   // J window
  return n * sizeof(T);
}

// ---- small helpers on shared-memory planes -----------------------------------------
template <typename T, int P2>
__device__ __forceinline__ void ldw(const T* plane, int c, T* w) {
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v] = plane[v * P2 + c];
}

// EGLM sources of state field W at cell c (Sec. 2, eqs. MHD-2 and MHD-4), central
// differences: s[MX..MZ] = -(div B) B, s[EN] = -B.grad psi.  pl[-1], pl[0], pl[+1] are the
// planes z-1, z, z+1 (only pl[0] in 2D).
template <typename T, int NDIM, int NP>
__device__ __forceinline__ void eglm_src(const T* const* pl, int c, const T* dx2, T* s) {
  constexpr int P2 = NP * NP;
  const T* p0 = pl[1];
  T divb = T(0);
  divb += (p0[BX * P2 + c + 1] - p0[BX * P2 + c - 1]) / dx2[0];
  divb += (p0[BY * P2 + c + NP] - p0[BY * P2 + c - NP]) / dx2[1];
  if (NDIM == 3) divb += (pl[2][BZ * P2 + c] - pl[0][BZ * P2 + c]) / dx2[2];
  T bg = T(0);
  bg += p0[BX * P2 + c] * ((p0[PSI * P2 + c + 1] - p0[PSI * P2 + c - 1]) / dx2[0]);
  bg += p0[BY * P2 + c] * ((p0[PSI * P2 + c + NP] - p0[PSI * P2 + c - NP]) / dx2[1]);
  if (NDIM == 3) bg += p0[BZ * P2 + c] * ((pl[2][PSI * P2 + c] - pl[0][PSI * P2 + c]) / dx2[2]);
  s[MX] += -divb * p0[BX * P2 + c];
  s[MY] += -divb * p0[BY * P2 + c];
  s[MZ] += -divb * p0[BZ * P2 + c];
  s[EN] += -bg;
}

// Current density J = curl B by central differences (Sec. 3.5) at cell c of plane pl[1].
template <typename T, int NDIM, int NP>
__device__ __forceinline__ void current(const T* const* pl, int c, const T* dx2, T* J) {
  constexpr int P2 = NP * NP;
  const T* p0 = pl[1];
  T dBz_dy = (p0[BZ * P2 + c + NP] - p0[BZ * P2 + c - NP]) / dx2[1];
  T dBz_dx = (p0[BZ * P2 + c + 1] - p0[BZ * P2 + c - 1]) / dx2[0];
  T dBy_dx = (p0[BY * P2 + c + 1] - p0[BY * P2 + c - 1]) / dx2[0];
  T dBx_dy = (p0[BX * P2 + c + NP] - p0[BX * P2 + c - NP]) / dx2[1];
  T dBy_dz = T(0), dBx_dz = T(0);
  if (NDIM == 3) {
    dBy_dz = (pl[2][BY * P2 + c] - pl[0][BY * P2 + c]) / dx2[2];
    dBx_dz = (pl[2][BX * P2 + c] - pl[0][BX * P2 + c]) / dx2[2];
  }
  J[0] = dBz_dy - dBy_dz;
  J[1] = dBx_dz - dBz_dx;
  J[2] = dBy_dx - dBx_dy;
}

// Resistive sources at cell c (Sec. 3.5): R = -curl(eta J), R_e = -div((eta J) x B), from
// J planes jl[0..2] (z-1..z+1) and state planes pl (for B).
template <typename T, int NDIM, int NP>
__device__ __forceinline__ void resist_src(const T* const* jl, const T* const* pl, int c,
                                           const T* dx2, T eta, T* s) {
  constexpr int P2 = NP * NP;
  const T* j0 = jl[1];
  auto cd = [&](const T* const* L, int comp, int d) -> T {
    if (d >= NDIM) return T(0);
    if (d == 0) return (L[1][comp * P2 + c + 1] - L[1][comp * P2 + c - 1]) / dx2[0];
    if (d == 1) return (L[1][comp * P2 + c + NP] - L[1][comp * P2 + c - NP]) / dx2[1];
    return (L[2][comp * P2 + c] - L[0][comp * P2 + c]) / dx2[2];
  };
  (void)j0;
  T rx = eta * cd(jl, 1, 2) - eta * cd(jl, 2, 1);
  T ry = eta * cd(jl, 2, 0) - eta * cd(jl, 0, 2);
  T rz = eta * cd(jl, 0, 1) - eta * cd(jl, 1, 0);
  T re = T(0);
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    T q[2];
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const T* Jp;
      const T* Bp;
      int cc;
      if (d == 0) { Jp = jl[1]; Bp = pl[1]; cc = sg ? c + 1 : c - 1; }
      else if (d == 1) { Jp = jl[1]; Bp = pl[1]; cc = sg ? c + NP : c - NP; }
      else { Jp = sg ? jl[2] : jl[0]; Bp = sg ? pl[2] : pl[0]; cc = c; }
      T Bx = Bp[BX * P2 + cc], By = Bp[BY * P2 + cc], Bz = Bp[BZ * P2 + cc];
      T Jx = Jp[0 * P2 + cc], Jy = Jp[1 * P2 + cc], Jz = Jp[2 * P2 + cc];
      T t;
      if (d == 0) t = Jz * By - Jy * Bz;
      else if (d == 1) t = Jx * Bz - Jz * Bx;
      else t = Jy * Bx - Jx * By;
      q[sg] = eta * t;
    }
    re += (q[1] - q[0]) / dx2[d];
  }
  s[BX] += rx;
  s[BY] += ry;
  s[BZ] += rz;
  s[EN] += re;
}

// ---- MMC pieces ------------------------------------------------------------------------
// h_{i+1/2} = f+_i + f-_{i+1} with the face speed alpha = max(alpha_i, alpha_{i+1}).
template <typename T, int D>
__device__ __forceinline__ void mmc_h(const T* wl, const T* wr, const Phys<T>& P, T* h) {
  T fl[NV], fr[NV];
  T pl = pressure<T>(wl, P), pr = pressure<T>(wr, P);
  flux_p<T, D>(wl, pl, P, fl);
  flux_p<T, D>(wr, pr, P, fr);
  T al = alpha_p<T, D>(wl, pl, P), ar = alpha_p<T, D>(wr, pr, P);
  T a = al > ar ? al : ar;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T s = glm_pair<D>(v) ? P.ch : a;
    h[v] = T(0.5) * (fl[v] + s * wl[v]) + T(0.5) * (fr[v] - s * wr[v]);
  }
}

// MMC face flux between cells i (w1) and i+1 (w2): u at i-1..i+2 (w0..w3), u~ at i, i+1
// (t0, t1).  Every split term of this face uses this face's speeds (alpha from u_i,
// u_{i+1}; alpha~ from u~_i, u~_{i+1}).
template <typename T, int D, int LIM>
__device__ __forceinline__ void mmc_face(const T* w0, const T* w1, const T* w2, const T* w3,
                                         const T* t0, const T* t1, const Phys<T>& P, T* fh) {
  T p1 = pressure<T>(w1, P), p2 = pressure<T>(w2, P);
  T q0 = pressure<T>(t0, P), q1 = pressure<T>(t1, P);
  T a1 = alpha_p<T, D>(w1, p1, P), a2 = alpha_p<T, D>(w2, p2, P);
  T alpha = a1 > a2 ? a1 : a2;
  T b1 = alpha_p<T, D>(t0, q0, P), b2 = alpha_p<T, D>(t1, q1, P);
  T alphat = b1 > b2 ? b1 : b2;
  T f[NV];
  T h[NV], gpl[NV], gpc[NV], gmc[NV], gmr[NV];
  // u_{i-1}: f+ for g+_{i-1/2}
  flux_p<T, D>(w0, pressure<T>(w0, P), P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alpha;
    gpl[v] = -(T(0.5) * (f[v] + a * w0[v]));
  }
  // u_i: f+ for h and g+_{i+1/2}
  flux_p<T, D>(w1, p1, P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alpha;
    T fp = T(0.5) * (f[v] + a * w1[v]);
    h[v] = fp;
    gpc[v] = fp;
  }
  // u_{i+1}: f- for h and g-_{i+1/2}
  flux_p<T, D>(w2, p2, P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alpha;
    T fm = T(0.5) * (f[v] - a * w2[v]);
    h[v] = h[v] + fm;
    gmc[v] = fm;
  }
  // u_{i+2}: f- for g-_{i+3/2}
  flux_p<T, D>(w3, pressure<T>(w3, P), P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alpha;
    gmr[v] = T(0.5) * (f[v] - a * w3[v]);
  }
  // u~_i: f~+ (g+_{i-1/2}) and f~- (g-_{i+1/2})
  flux_p<T, D>(t0, q0, P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alphat;
    gpl[v] = T(0.5) * (f[v] + a * t0[v]) + gpl[v];
    gmc[v] = gmc[v] - T(0.5) * (f[v] - a * t0[v]);
  }
  // u~_{i+1}: f~+ (g+_{i+1/2}) and f~- (g-_{i+3/2})
  flux_p<T, D>(t1, q1, P, f);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T a = glm_pair<D>(v) ? P.ch : alphat;
    gpc[v] = T(0.5) * (f[v] + a * t1[v]) - gpc[v];
    gmr[v] = gmr[v] - T(0.5) * (f[v] - a * t1[v]);
    fh[v] = h[v] + T(0.5) * (limiter<T, LIM>(gpl[v], gpc[v]) - limiter<T, LIM>(gmr[v], gmc[v]));
  }
}

// ---- the kernel --------------------------------------------------------------------------

template <typename T, int NDIM, int NB, int SCHEME, int LIM, int STAGE>
__global__ void __launch_bounds__(NB * NB, (sizeof(T) == 4 && NDIM == 3 && NB == 16) ? 2 : 1)
step_kernel(StepArgsT<T> A) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, NZ = G::NZ, S = G::S, NT = G::NT;
  constexpr int UPL = G::UPL, WPL = G::WPL;
  constexpr bool HAS_T = SCHEME != SCH_WENO;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sut = su + (size_t)UPL * NV * P2;
  T* sf = sut + (HAS_T ? (size_t)WPL * NV * P2 : 0);
  T* sj = sf + (size_t)NV * G::NFACE;

  const int tid = threadIdx.x;
  const int tx = tid % NB, ty = tid / NB;
  const int cown = (ty + NG) * NP + (tx + NG);

  double alpha_max = 0.0;
  double csum[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) csum[v] = 0.0;
  unsigned errbits = 0;

  for (int bi = blockIdx.x; bi < A.nblocks; bi += gridDim.x) {
    const int blk = A.blocks[bi];
    const BlockGeo gg = A.geo[blk];
    const ProbDyn dy = A.dyn[gg.problem];
    Phys<T> P;
    P.gamma = A.gamma;
    P.gm1 = A.gm1;
    P.ch = (T)dy.ch;
    P.tau = A.tau;
    const double dtd = dy.dt;
    const T dt = (T)dtd;
    T lam[3], lamh[3], dx2[3], dxT[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lam[d] = (T)(dtd / gg.dx[d]);
      lamh[d] = (T)((0.5 * dtd) / gg.dx[d]);
      dx2[d] = (T)(2.0 * gg.dx[d]);
      dxT[d] = (T)gg.dx[d];
    }
    const T damp = (T)dy.damp;
    const T eta = (T)A.eta;
    const T* ub = A.u_in + (size_t)blk * NV * S;
    T* ob = A.u_out + (size_t)blk * NV * S;
    const T* bb = (STAGE == 2) ? A.u_base + (size_t)blk * NV * S : nullptr;
    const bool RES = A.resistive != 0;

    auto uslot = [&](int z) -> T* { return su + (size_t)(NDIM == 3 ? (z & 3) : 0) * NV * P2; };
    auto tslot = [&](int z) -> T* { return sut + (size_t)(NDIM == 3 ? (z % 3) : 0) * NV * P2; };
    auto jslot = [&](int z) -> T* { return sj + (size_t)(NDIM == 3 ? (z % 3) : 0) * 3 * P2; };

    auto load_plane = [&](int z) {
      T* dst = uslot(z);
      const T* src = ub + (size_t)z * P2;
#pragma unroll 1
      for (int v = 0; v < NV; ++v) {
        const T* s = src + (size_t)v * NZ * P2;
        T* d = dst + v * P2;
        for (int c = tid; c < P2; c += NT) d[c] = s[c];
      }
    };

    // u~ (MMC/LF) and J (resistive) on the ring of plane z (needs u planes z-1..z+1)
    auto predict_plane = [&](int z) {
      const T* ul[3] = {uslot(z - 1), uslot(z), uslot(z + 1)};
      T* tp = tslot(z);
      for (int r = tid; r < G::RING; r += NT) {
        const int x = 1 + r % (NB + 2), y = 1 + r / (NB + 2);
        const int c = y * NP + x;
        if (HAS_T) {
          T w[NV], acc[NV];
          ldw<T, P2>(ul[1], c, w);
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] = w[v];
          if (SCHEME == SCH_MMC) {
            T wm[NV], wp[NV], hp[NV], hm[NV];
            // x
            ldw<T, P2>(ul[1], c - 1, wm);
            ldw<T, P2>(ul[1], c + 1, wp);
            mmc_h<T, 0>(w, wp, P, hp);
            mmc_h<T, 0>(wm, w, P, hm);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] -= lam[0] * (hp[v] - hm[v]);
            // y
            ldw<T, P2>(ul[1], c - NP, wm);
            ldw<T, P2>(ul[1], c + NP, wp);
            mmc_h<T, 1>(w, wp, P, hp);
            mmc_h<T, 1>(wm, w, P, hm);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] -= lam[1] * (hp[v] - hm[v]);
            if (NDIM == 3) {
              ldw<T, P2>(ul[0], c, wm);
              ldw<T, P2>(ul[2], c, wp);
              mmc_h<T, 2>(w, wp, P, hp);
              mmc_h<T, 2>(wm, w, P, hm);
#pragma unroll
              for (int v = 0; v < NV; ++v) acc[v] -= lam[2] * (hp[v] - hm[v]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) tp[v * P2 + c] = acc[v];
          } else {
            // LF: MUSCL-Hancock half step
            T a[NV], b[NV], fa[NV], fb[NV];
            auto half = [&](auto Dc, const T* plm, int cm, const T* plp, int cp) {
              constexpr int D = decltype(Dc)::value;
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T ph = limiter<T, LIM>(w[v] - plm[v * P2 + cm], plp[v * P2 + cp] - w[v]);
                a[v] = w[v] + T(0.5) * ph;
                b[v] = w[v] - T(0.5) * ph;
              }
              flux_p<T, D>(a, pressure<T>(a, P), P, fa);
              flux_p<T, D>(b, pressure<T>(b, P), P, fb);
#pragma unroll
              for (int v = 0; v < NV; ++v) acc[v] -= lamh[D] * (fa[v] - fb[v]);
            };
            half(std::integral_constant<int, 0>(), ul[1], c - 1, ul[1], c + 1);
            half(std::integral_constant<int, 1>(), ul[1], c - NP, ul[1], c + NP);
            if (NDIM == 3) half(std::integral_constant<int, 2>(), ul[0], c, ul[2], c);
            T s[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) s[v] = T(0);
            if (A.eglm) eglm_src<T, NDIM, NP>(ul, c, dx2, s);
            const T hdt = (T)(0.5 * dtd);
#pragma unroll
            for (int v = 0; v < NV; ++v) tp[v * P2 + c] = acc[v] + hdt * s[v];
          }
        }
        if (RES) {
          T J[3];
          current<T, NDIM, NP>(ul, c, dx2, J);
          T* jp = jslot(z);
          jp[0 * P2 + c] = J[0];
          jp[1 * P2 + c] = J[1];
          jp[2 * P2 + c] = J[2];
        }
      }
    };

    // face flux between cell cl (planes/offsets given) and its + neighbour in direction D
    auto face_flux = [&](auto Dc, const T* const* up, const T* const* tp, int c0, int st, T* F) {
      // up[k], tp[k]: plane pointers of cells i-1, i, i+1, i+2 (k = 0..3) along D;
      // cell index in its plane = c0 + (k-1)*st (st = 0 for D = 2)
      constexpr int D = decltype(Dc)::value;
      const int cm = c0 - st, c1 = c0, c2 = c0 + st, c3 = c0 + 2 * st;
      if (SCHEME == SCH_MMC) {
        T w0[NV], w1[NV], w2[NV], w3[NV], t0[NV], t1[NV];
        ldw<T, P2>(up[0], cm, w0);
        ldw<T, P2>(up[1], c1, w1);
        ldw<T, P2>(up[2], c2, w2);
        ldw<T, P2>(up[3], c3, w3);
        ldw<T, P2>(tp[1], c1, t0);
        ldw<T, P2>(tp[2], c2, t1);
        mmc_face<T, D, LIM>(w0, w1, w2, w3, t0, t1, P, F);
      } else if (SCHEME == SCH_LF) {
        T a[NV], b[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T um = up[0][v * P2 + cm], u1 = up[1][v * P2 + c1];
          const T u2 = up[2][v * P2 + c2], u3 = up[3][v * P2 + c3];
          T phl = limiter<T, LIM>(u1 - um, u2 - u1);
          T phr = limiter<T, LIM>(u2 - u1, u3 - u2);
          a[v] = tp[1][v * P2 + c1] + T(0.5) * phl;
          b[v] = tp[2][v * P2 + c2] - T(0.5) * phr;
        }
        lf_flux<T, D>(a, b, P, F);
      } else {
        T a[NV], b[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T um = up[0][v * P2 + cm], u1 = up[1][v * P2 + c1];
          const T u2 = up[2][v * P2 + c2], u3 = up[3][v * P2 + c3];
          a[v] = weno_minus_right<T>(um, u1, u2);
          b[v] = weno_plus_left<T>(u1, u2, u3);
        }
        lf_flux<T, D>(a, b, P, F);
      }
    };

    // z-face flux of the own column between planes z and z+1
    auto zface = [&](int z, T* F) {
      const T* up[4] = {uslot(z - 1), uslot(z), uslot(z + 1), uslot(z + 2)};
      const T* tp[4] = {nullptr, HAS_T ? tslot(z) : nullptr, HAS_T ? tslot(z + 1) : nullptr, nullptr};
      face_flux(std::integral_constant<int, 2>(), up, tp, cown, 0, F);
    };

    T Fzlo[NV];
    int zbeg = 0, zend = 1;
    if (NDIM == 3) {
      for (int z = 0; z < 4; ++z) load_plane(z);
      __syncthreads();
      if (HAS_T || RES) {
        predict_plane(1);
        predict_plane(2);
      }
      __syncthreads();
      zface(1, Fzlo);
      __syncthreads();
      zbeg = NG;
      zend = NB + NG;
    } else {
      load_plane(0);
      __syncthreads();
      if (HAS_T || RES) predict_plane(0);
      __syncthreads();
    }

    for (int z = zbeg; z < zend; ++z) {
      if (NDIM == 3) {
        // window: u planes z-1..z+2, u~ and J planes z-1..z+1
        load_plane(z + 2);
        __syncthreads();
        if (HAS_T || RES) predict_plane(z + 1);
        __syncthreads();
      }
      const T* P0 = uslot(z);
      T acc[NV];
      if (SCHEME == SCH_WENO) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = T(0);
      } else {
        ldw<T, P2>(P0, cown, acc);
      }
      // x faces of the plane
      {
        const T* up[4] = {P0, P0, P0, P0};
        const T* tq = HAS_T ? tslot(z) : nullptr;
        const T* tp[4] = {tq, tq, tq, tq};
        for (int f = tid; f < G::NFACE; f += NT) {
          const int row = f / (NB + 1), fx = f % (NB + 1);
          const int cl = (row + NG) * NP + fx + 1;
          T F[NV];
          face_flux(std::integral_constant<int, 0>(), up, tp, cl, 1, F);
#pragma unroll
          for (int v = 0; v < NV; ++v) sf[v * G::NFACE + f] = F[v];
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T fr = sf[v * G::NFACE + ty * (NB + 1) + tx + 1];
          T fl = sf[v * G::NFACE + ty * (NB + 1) + tx];
          if (SCHEME == SCH_WENO) acc[v] -= (fr - fl) / dxT[0];
          else acc[v] -= lam[0] * (fr - fl);
        }
        __syncthreads();
      }
      // y faces
      {
        const T* up[4] = {P0, P0, P0, P0};
        const T* tq = HAS_T ? tslot(z) : nullptr;
        const T* tp[4] = {tq, tq, tq, tq};
        for (int f = tid; f < G::NFACE; f += NT) {
          const int fy = f / NB, col = f % NB;
          const int cl = (fy + 1) * NP + col + NG;
          T F[NV];
          face_flux(std::integral_constant<int, 1>(), up, tp, cl, NP, F);
#pragma unroll
          for (int v = 0; v < NV; ++v) sf[v * G::NFACE + f] = F[v];
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T fr = sf[v * G::NFACE + (ty + 1) * NB + tx];
          T fl = sf[v * G::NFACE + ty * NB + tx];
          if (SCHEME == SCH_WENO) acc[v] -= (fr - fl) / dxT[1];
          else acc[v] -= lam[1] * (fr - fl);
        }
      }
      // z faces
      if (NDIM == 3) {
        T Fzhi[NV];
        zface(z, Fzhi);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (SCHEME == SCH_WENO) acc[v] -= (Fzhi[v] - Fzlo[v]) / dxT[2];
          else acc[v] -= lam[2] * (Fzhi[v] - Fzlo[v]);
          Fzlo[v] = Fzhi[v];
        }
      }
      // sources
      T s[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] = T(0);
      if (A.eglm) {
        if (SCHEME == SCH_LF) {
          const T* tl[3] = {tslot(z - 1), tslot(z), tslot(z + 1)};
          eglm_src<T, NDIM, NP>(tl, cown, dx2, s);
        } else {
          const T* ul[3] = {uslot(z - 1), uslot(z), uslot(z + 1)};
          eglm_src<T, NDIM, NP>(ul, cown, dx2, s);
        }
      }
      if (RES) {
        const T* jl[3] = {jslot(z - 1), jslot(z), jslot(z + 1)};
        const T* ul[3] = {uslot(z - 1), uslot(z), uslot(z + 1)};
        resist_src<T, NDIM, NP>(jl, ul, cown, dx2, eta, s);
      }
      // update and write
      T out[NV];
      const size_t gofs = (size_t)z * P2 + cown;
      if (SCHEME == SCH_WENO) {
        if (STAGE == 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) out[v] = P0[v * P2 + cown] + dt * (acc[v] + s[v]);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T un = bb[(size_t)v * S + gofs];
            out[v] = T(0.5) * ((un + P0[v * P2 + cown]) + dt * (acc[v] + s[v]));
          }
          out[PSI] = out[PSI] * damp;
        }
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = acc[v] + dt * s[v];
        out[PSI] = out[PSI] * damp;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) ob[(size_t)v * S + gofs] = out[v];
      if (STAGE != 1) {
        bool fin = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) fin = fin && isfinite((double)out[v]);
        if (!fin) errbits |= 1u;
        else {
          T pr = pressure<T>(out, P);
          if (!(out[RHO] > T(0)) || pr < T(0)) errbits |= 2u;
          if (A.dyn_next) {
            double am = 0.0;
            am = fmax(am, (double)alpha_p<T, 0>(out, pr, P));
            am = fmax(am, (double)alpha_p<T, 1>(out, pr, P));
            if (NDIM == 3) am = fmax(am, (double)alpha_p<T, 2>(out, pr, P));
            alpha_max = fmax(alpha_max, am);
          }
        }
        if (A.sums) {
          double vol = gg.dx[0] * gg.dx[1] * (NDIM == 3 ? gg.dx[2] : 1.0);
#pragma unroll
          for (int v = 0; v < NV; ++v) csum[v] += (double)out[v] * vol;
        }
      }
      __syncthreads();
    }
    // per-block reductions of the fused diagnostics (block problem is uniform per block)
    if (A.dyn_next || A.sums) {
      __shared__ double red[NV + 1][32];
      const int lane = tid & 31, wid = tid >> 5;
      double am = alpha_max;
      for (int o = 16; o > 0; o >>= 1) am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
      double cs[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        cs[v] = csum[v];
        for (int o = 16; o > 0; o >>= 1) cs[v] += __shfl_xor_sync(0xffffffffu, cs[v], o);
      }
      if (lane == 0) {
        red[NV][wid] = am;
#pragma unroll
        for (int v = 0; v < NV; ++v) red[v][wid] = cs[v];
      }
      __syncthreads();
      if (tid == 0) {
        const int nw = (NT + 31) / 32;
        double a2 = 0.0;
        for (int q = 0; q < nw; ++q) a2 = fmax(a2, red[NV][q]);
        if (A.dyn_next) {
          // alpha >= 0: its IEEE bit pattern orders like the value (NaN above everything)
          atomicMax(&A.dyn_next[gg.problem].alpha_bits, (unsigned long long)__double_as_longlong(a2));
        }
        if (A.sums) {
          for (int v = 0; v < NV; ++v) {
            double t = 0.0;
            for (int q = 0; q < nw; ++q) t += red[v][q];
            atomicAdd(&A.sums[gg.problem * NV + v], t);
          }
        }
      }
      __syncthreads();
      alpha_max = 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) csum[v] = 0.0;
    }
  }
  // error word
  unsigned e = errbits;
  for (int o = 16; o > 0; o >>= 1) e |= __shfl_xor_sync(0xffffffffu, e, o);
  if ((tid & 31) == 0 && e) atomicOr(A.err_word, e);
}

}  // namespace mapgb
