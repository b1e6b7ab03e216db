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
// has NB*NB threads, thread (tx,ty) owning interior column (tx+2, ty+2) -- except the 2D
// 16^2 FP32 kernels, whose 128 threads own two columns each (step_threads).  In 3D the CTA
// marches in z keeping a rolling window in shared memory: four u planes (z..z+3, one in
// flight), the u~ planes and, with resistivity, the J planes (z-1..z+1 for 16^3 blocks; z,
// z+1 for 8^3, whose update carries its own column's plane z-1 values in registers); x- and
// y-face fluxes of the current plane go through one shared buffer, the z-face flux of the
// column is carried in registers from one plane to the next.  In 2D the window is the single
// plane.
#pragma once
#include <type_traits>

#include "map_internal.hpp"
#include "physics.cuh"

namespace mapgb {

enum { SCH_MMC = 0, SCH_LF = 1, SCH_WENO = 2 };
static_assert(SCH_MMC == MAP_MMC && SCH_LF == MAP_LF && SCH_WENO == MAP_WENO, "scheme codes follow map.h");
enum { FLX_LF = 0, FLX_HLLC = 1, FLX_HLLD = 2 };   // interface flux of LF and WENO: f_m, HLLC or HLLD

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
  const PushEntry* pushes;
  T* freg;
  const RefluxLeaf* refl;
  unsigned char sched[8][16];   // warp schedule of the per-plane work list (build_schedule)
  int fail_waits;               // test hook: 1 = the plane waits give up at once
};

template <int NDIM, int NB>
struct Geo {
  static constexpr int NP = NB + 4;
  static constexpr int P2 = NP * NP;
  static constexpr int NZ = NDIM == 3 ? NP : 1;
  static constexpr int S = NZ * P2;
  static constexpr int NCOL = NB * NB;                 // interior columns (threads: step_threads)
  static constexpr int UPL = NDIM == 3 ? 4 : 1;   // u planes z..z+2 and one in flight
  // u~ and J ring planes.  3D 8^3: planes z and z+1 -- the update of plane z reads plane
  // z-1 only at its own column, and only u~ B_z, psi and J, which are carried in registers
  // from the previous plane; the smaller window lets 6 CTAs reside instead of 5.  3D 16^3:
  // planes z-1..z+1 (two CTAs reside either way, and carried values would only add
  // registers at the 128-register cap).
  static constexpr int WPL = NDIM == 3 ? (NB == 8 ? 2 : 3) : 1;
  static constexpr bool CARRY = NDIM == 3 && WPL == 2;
  static constexpr int RW = NB + 2;               // ring row width (padded 1..NB+2)
  static constexpr int RING = RW * RW;
  // ring cells the predictor fills: all but the four corners, which no stencil reads (the
  // faces read u~ across one axis; the sources read u~ and J along the axes)
  static constexpr int NPC = RING - 4;
  static constexpr int NFACE = NB * (NB + 1);
};

template <typename T, int NDIM, int NB, int SCHEME>
__host__ __device__ constexpr size_t step_smem_bytes(bool resistive) {
  using G = Geo<NDIM, NB>;
  size_t n = (size_t)G::UPL * NV * G::P2;                          // u window (full planes)
  if (SCHEME != SCH_WENO) n += (size_t)G::WPL * NV * G::RING;      // u~ window (ring)
  size_t nf = (size_t)2 * NV * G::NFACE;                            // x and y face fluxes
  if (nf < (size_t)(NV + 1) * 32 * 2) nf = (size_t)(NV + 1) * 32 * 2;  // reused for reductions
  n += nf;
  if (resistive) n += (size_t)G::WPL * 3 * G::RING;                 // J window (ring)
  return 256 + n * sizeof(T);                                       // 256 B: mbarriers, block constants
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
  divb += qdiv<T>((p0[BX * P2 + c + 1] - p0[BX * P2 + c - 1]), dx2[0]);
  divb += qdiv<T>((p0[BY * P2 + c + NP] - p0[BY * P2 + c - NP]), dx2[1]);
  if (NDIM == 3) divb += qdiv<T>((pl[2][BZ * P2 + c] - pl[0][BZ * P2 + c]), dx2[2]);
  T bg = T(0);
  bg += p0[BX * P2 + c] * (qdiv<T>((p0[PSI * P2 + c + 1] - p0[PSI * P2 + c - 1]), dx2[0]));
  bg += p0[BY * P2 + c] * (qdiv<T>((p0[PSI * P2 + c + NP] - p0[PSI * P2 + c - NP]), dx2[1]));
  if (NDIM == 3) bg += p0[BZ * P2 + c] * (qdiv<T>((pl[2][PSI * P2 + c] - pl[0][PSI * P2 + c]), dx2[2]));
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
  T dBz_dy = qdiv<T>((p0[BZ * P2 + c + NP] - p0[BZ * P2 + c - NP]), dx2[1]);
  T dBz_dx = qdiv<T>((p0[BZ * P2 + c + 1] - p0[BZ * P2 + c - 1]), dx2[0]);
  T dBy_dx = qdiv<T>((p0[BY * P2 + c + 1] - p0[BY * P2 + c - 1]), dx2[0]);
  T dBx_dy = qdiv<T>((p0[BX * P2 + c + NP] - p0[BX * P2 + c - NP]), dx2[1]);
  T dBy_dz = T(0), dBx_dz = T(0);
  if (NDIM == 3) {
    dBy_dz = qdiv<T>((pl[2][BY * P2 + c] - pl[0][BY * P2 + c]), dx2[2]);
    dBx_dz = qdiv<T>((pl[2][BX * P2 + c] - pl[0][BX * P2 + c]), dx2[2]);
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
    if (d == 0) return qdiv<T>((L[1][comp * P2 + c + 1] - L[1][comp * P2 + c - 1]), dx2[0]);
    if (d == 1) return qdiv<T>((L[1][comp * P2 + c + NP] - L[1][comp * P2 + c - NP]), dx2[1]);
    return qdiv<T>((L[2][comp * P2 + c] - L[0][comp * P2 + c]), dx2[2]);
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
    re += qdiv<T>((q[1] - q[0]), dx2[d]);
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

// ---- bulk-copy (TMA) helpers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Bounded wait on an mbarrier phase: gives up after ~2^31 clock cycles (about a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// EGLM sources at cell c of a centre plane given with its variable stride PS and row stride
// RS; the z-neighbours of the same column come as states zm (z-1) and zp (z+1).
template <typename T, int NDIM>
__device__ __forceinline__ void eglm_src_col(const T* pc, int PS, int RS, int c, const T* zm, const T* zp,
                                             const T* dx2, T* s) {
  T divb = T(0);
  divb += qdiv<T>((pc[BX * PS + c + 1] - pc[BX * PS + c - 1]), dx2[0]);
  divb += qdiv<T>((pc[BY * PS + c + RS] - pc[BY * PS + c - RS]), dx2[1]);
  if (NDIM == 3) divb += qdiv<T>((zp[BZ] - zm[BZ]), dx2[2]);
  T bg = T(0);
  bg += pc[BX * PS + c] * (qdiv<T>((pc[PSI * PS + c + 1] - pc[PSI * PS + c - 1]), dx2[0]));
  bg += pc[BY * PS + c] * (qdiv<T>((pc[PSI * PS + c + RS] - pc[PSI * PS + c - RS]), dx2[1]));
  if (NDIM == 3) bg += pc[BZ * PS + c] * (qdiv<T>((zp[PSI] - zm[PSI]), dx2[2]));
  s[MX] += -divb * pc[BX * PS + c];
  s[MY] += -divb * pc[BY * PS + c];
  s[MZ] += -divb * pc[BZ * PS + c];
  s[EN] += -bg;
}

// Resistive sources at the own column (Sec. 3.5).  J: centre plane jc (ring layout, index
// cj) and the column's J at z-1 / z+1 (jzm, jzp); B: centre plane uc (full layout, index
// cu) and the column's states at z-1 / z+1 (bzm, bzp).
template <typename T, int NDIM, int NP, int RW>
__device__ __forceinline__ void resist_src_col(const T* jc, int cj, const T* jzm, const T* jzp, const T* uc, int cu,
                                               const T* bzm, const T* bzp, const T* dx2, T eta, T* s) {
  constexpr int PJ = RW * RW, PU = NP * NP;
  auto cdJ = [&](int comp, int d) -> T {
    if (d >= NDIM) return T(0);
    if (d == 0) return qdiv<T>((jc[comp * PJ + cj + 1] - jc[comp * PJ + cj - 1]), dx2[0]);
    if (d == 1) return qdiv<T>((jc[comp * PJ + cj + RW] - jc[comp * PJ + cj - RW]), dx2[1]);
    return qdiv<T>((jzp[comp] - jzm[comp]), dx2[2]);
  };
  T rx = eta * cdJ(1, 2) - eta * cdJ(2, 1);
  T ry = eta * cdJ(2, 0) - eta * cdJ(0, 2);
  T rz = eta * cdJ(0, 1) - eta * cdJ(1, 0);
  T re = T(0);
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    T q[2];
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      T Bx, By, Bz, Jx, Jy, Jz;
      if (d < 2) {
        const int oj = d == 0 ? (sg ? 1 : -1) : (sg ? RW : -RW);
        const int ou = d == 0 ? (sg ? 1 : -1) : (sg ? NP : -NP);
        Bx = uc[BX * PU + cu + ou]; By = uc[BY * PU + cu + ou]; Bz = uc[BZ * PU + cu + ou];
        Jx = jc[0 * PJ + cj + oj]; Jy = jc[1 * PJ + cj + oj]; Jz = jc[2 * PJ + cj + oj];
      } else {
        const T* bb = sg ? bzp : bzm;
        const T* jj = sg ? jzp : jzm;
        Bx = bb[BX]; By = bb[BY]; Bz = bb[BZ];
        Jx = jj[0]; Jy = jj[1]; Jz = jj[2];
      }
      T t;
      if (d == 0) t = Jz * By - Jy * Bz;
      else if (d == 1) t = Jx * Bz - Jz * Bx;
      else t = Jy * Bx - Jx * By;
      q[sg] = eta * t;
    }
    re += qdiv<T>((q[1] - q[0]), dx2[d]);
  }
  s[BX] += rx;
  s[BY] += ry;
  s[BZ] += rz;
  s[EN] += re;
}

// Exchange of the x and y components of m and B when yd (the map P with F_y(U) = P F_x(P U)).
template <typename V>
__device__ __forceinline__ void exch_xy(bool yd, V* w) {
  const V mx = w[MX], my = w[MY], bx = w[BX], by = w[BY];
  w[MX] = yd ? my : mx;
  w[MY] = yd ? mx : my;
  w[BX] = yd ? by : bx;
  w[BY] = yd ? bx : by;
}

// ---- the kernel --------------------------------------------------------------------------
//
// 3D z-march with a window of three resident u planes (z..z+2) plus one plane in flight:
// plane z+3 is fetched by bulk copies (cp.async.bulk, completion on an mbarrier) while
// plane z is computed.  Every z-direction stencil (z faces, z derivatives of the sources)
// runs along a thread's own column, so the column's state at z-1 is carried in registers
// and no fourth resident plane is needed.  u~ and J live in ring layout (padded 1..NB+2); for
// 8^3 blocks two planes each, the few values of plane z-1 that the update of plane z needs
// (its own column's u~ B_z and psi, and J) being read while plane z-1 is current and carried.
// Per plane, the predictor of plane z+1 and the x and y faces of plane z form one
// warp-aligned work list (they touch different slots), so a plane costs three barriers.

template <int N>
struct Pad32 { static constexpr int value = (N + 31) / 32 * 32; };

// Threads per CTA of the step kernel: one per interior column, except in the 2D 16^2 FP32
// kernels, whose 128 threads take two columns each in the update.  Their predictor and face
// phases (10 and 17 warp units in separate barrier intervals) then leave fewer warps idle at
// each barrier, and four CTAs reside per SM instead of two, at the same 128 registers.
template <typename T, int NDIM, int NB>
__host__ __device__ constexpr int step_threads() {
  return (sizeof(T) == 4 && NDIM == 2 && NB == 16) ? 128 : NB * NB;
}

// The per-plane work list of the step kernel: warp-sized units of predictor ring cells (NPU,
// corners left out),
// then the x faces and y faces in one numbering (NFU), over the NW warps of NT threads.
template <int NDIM, int NB, int NT>
struct WorkList {
  using G = Geo<NDIM, NB>;
  static constexpr int NW = NT / 32;
  static constexpr int NPU = Pad32<G::NPC>::value / 32;
  static constexpr int NFU = Pad32<2 * G::NFACE>::value / 32;   // x faces, then y faces
  static constexpr int NU = NPU + NFU;
  static_assert(NW <= 8 && NU <= 15 * NW, "work list exceeds the schedule table");
};

// Warp schedule, built on the host once per launch: each unit goes, in order, to the
// least-loaded warp that has room (ties to the lowest warp), a predictor unit weighing w_pred
// and a face unit w_face (their relative cost; default_schedule_weights unless tuned).  s[w][15] holds the
// number of units of warp w, s[w][0..] the units.  Without a predictor (WENO without
// resistivity) its units are left out, so they do not displace face units.
template <int NDIM, int NB, int NT>
inline void build_schedule(int w_pred, int w_face, bool pred, unsigned char (&s)[8][16]) {
  using W = WorkList<NDIM, NB, NT>;
  int load[8] = {0}, cnt[8] = {0};
  for (int q = 0; q < 8; ++q)
    for (int k = 0; k < 16; ++k) s[q][k] = 0;
  for (int u = pred ? 0 : W::NPU; u < W::NU; ++u) {
    int best = -1;
    for (int q = 0; q < W::NW; ++q)
      if (cnt[q] < 15 && (best < 0 || load[q] < load[best])) best = q;
    s[best][cnt[best]++] = (unsigned char)u;
    load[best] += u < W::NPU ? w_pred : w_face;
  }
  for (int q = 0; q < W::NW; ++q) s[q][15] = (unsigned char)cnt[q];
}

// a + b as an unevaluated pair (hi, lo) (TwoSum, Knuth)
template <typename T>
__device__ __forceinline__ void two_sum_acc(T& hi, T& lo, T h2, T l2) {
  const T s = hi + h2;
  const T bp = s - hi;
  const T err = (hi - (s - bp)) + (h2 - bp);
  lo = lo + l2 + err;
  hi = s;
}

// RFX: the mesh has coarse/fine faces with reflux on -- the kernel then records its boundary
// face fluxes and leaves the cells the reflux pass corrects out of the fused reductions.
// Without it none of that code exists in the kernel.
// Resident CTAs per SM the register budget is sized for: the 3D 8^3 window (at most 36 KB of
// shared memory) lets 6 CTAs reside, so asking for 8 would only cap the registers at 128 and
// spill the column state; four 128-thread 2D 16^2 CTAs take the 128 registers two 256-thread
// ones did.
template <typename T, int NDIM, int NB>
constexpr int step_min_ctas() {
  return sizeof(T) != 4 ? 1 : NB == 16 ? (NDIM == 2 ? 4 : 2) : NDIM == 3 ? 6 : 8;
}

template <typename T, int NDIM, int NB, int SCHEME, int LIM, int STAGE, int FLX, bool RFX>
__global__ void __launch_bounds__(step_threads<T, NDIM, NB>(), step_min_ctas<T, NDIM, NB>())
step_kernel(StepArgsT<T> A) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, NZ = G::NZ, S = G::S;
  constexpr int NT = step_threads<T, NDIM, NB>(), CPT = NB * NB / NT;   // columns per thread
  constexpr int UPL = G::UPL, WPL = G::WPL, RW = G::RW, RING = G::RING, NFACE = G::NFACE;
  constexpr bool HAS_T = SCHEME != SCH_WENO;
  // PREF: the FP32 LF faces carry their normal-momentum flux less a per-block reference total
  // pressure (kc[16]); the offset cancels in every flux difference of the update
  constexpr bool PREF = std::is_same<T, float>::value && SCHEME == SCH_LF && FLX == FLX_LF;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);           // UPL mbarriers
  volatile int* status = reinterpret_cast<volatile int*>(smem_raw + 48);
  T* kc = reinterpret_cast<T*>(smem_raw + 64);                       // block constants
  T* su = reinterpret_cast<T*>(smem_raw + 256);
  T* sut = su + (size_t)UPL * NV * P2;
  T* sf = sut + (HAS_T ? (size_t)WPL * NV * RING : 0);
  size_t nf = (size_t)2 * NV * NFACE;
  if (nf < (size_t)(NV + 1) * 32 * 2) nf = (size_t)(NV + 1) * 32 * 2;
  T* sj = sf + nf;
  __shared__ PushEntry spush[27];

  const int tid = threadIdx.x;
  // the thread's column (CPT > 1: the current one of its columns in the update)
  int tx = tid % NB, ty = tid / NB;
  int cown = (ty + NG) * NP + (tx + NG);                // own column, full plane layout
  int rown = (ty + 1) * RW + (tx + 1);                  // own column, ring layout

  // warp schedule of the per-plane work list (WorkList, build_schedule), the same on every
  // block; thread 0 copies it from the arguments with constant indices
  constexpr int NW = WorkList<NDIM, NB, NT>::NW;
  constexpr int NPU = WorkList<NDIM, NB, NT>::NPU;
  __shared__ int sched[NW][16];
  __shared__ RefluxLeaf srl;               // the block's face-register slot and coarse-side mask
  if (tid == 0) {
    for (int q = 0; q < UPL; ++q) mbar_init(&bars[q], 1);
    *status = 0;
    fence_mbar_init();
#pragma unroll
    for (int q = 0; q < NW; ++q)
#pragma unroll
      for (int k = 0; k < 16; ++k) sched[q][k] = A.sched[q][k];
  }
  __syncthreads();
  unsigned phase = 0;                                   // parity bit per u slot
  unsigned inflight = 0;                                // thread 0: slots with copies in flight

  // fused diagnostics: the running alpha maximum is exact in T; the sums of a thread's
  // column are Kahan-compensated in T and promoted to FP64 once per block
  T alpha_max = T(0);
  T csum[NV], ccmp[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { csum[v] = T(0); ccmp[v] = T(0); }
  unsigned errbits = 0;

  for (int bi = blockIdx.x; bi < A.nblocks; bi += gridDim.x) {
    const int blk = A.blocks[bi];
    const BlockGeo gg = A.geo[blk];
    if (A.pushes && tid < 27) spush[tid] = A.pushes[(size_t)blk * 27 + tid];   // read after the first barrier
    if (RFX && tid == 0) srl = A.refl[blk];             // read after the first barrier
    const T* ub = A.u_in + (size_t)blk * NV * S;
    T* ob = A.u_out + (size_t)blk * NV * S;
    const T* bb = (STAGE == 2) ? A.u_base + (size_t)blk * NV * S : nullptr;
    const bool RES = A.resistive != 0;
    const T eta = (T)A.eta;

    auto uslot = [&](int z) -> T* { return su + (size_t)(NDIM == 3 ? (z & 3) : 0) * NV * P2; };
    auto tslot = [&](int z) -> T* { return sut + (size_t)(NDIM == 3 ? (z % WPL) : 0) * NV * RING; };
    auto jslot = [&](int z) -> T* { return sj + (size_t)(NDIM == 3 ? (z % WPL) : 0) * 3 * RING; };

    // issue the bulk copies of u plane z into its slot (thread 0 only)
    auto issue_plane = [&](int z) {
      const int q = NDIM == 3 ? (z & 3) : 0;
      fence_async_smem();
      inflight |= 1u << q;
      mbar_expect_tx(&bars[q], (unsigned)(NV * P2 * sizeof(T)));
#pragma unroll 1
      for (int v = 0; v < NV; ++v)
        bulk_g2s(uslot(z) + v * P2, ub + ((size_t)v * NZ + z) * P2, (unsigned)(P2 * sizeof(T)), &bars[q]);
    };
    // wait for u plane z (thread 0 waits with a bound, the CTA follows via the barrier);
    // returns false on timeout
    auto wait_plane = [&](int z) -> bool {
      const int q = NDIM == 3 ? (z & 3) : 0;
      if (tid == 0) {
        // (the test hook gives up without waiting; the copies are still drained below)
        if (!A.fail_waits && mbar_wait_bounded(&bars[q], (phase >> q) & 1u)) inflight &= ~(1u << q);
        else *status = 1;
      }
      __syncthreads();
      const bool good = *status == 0;
      if (good) phase ^= 1u << q;
      return good;
    };

    // p + B^2/2 at cell c of a full plane (the faces' reference, any value would cancel)
    auto total_pressure = [&](const T* pl, int c) -> T {
      auto q = [&](int v) { return pl[v * P2 + c]; };
      const T b2 = q(BX) * q(BX) + q(BY) * q(BY) + q(BZ) * q(BZ);
      const T m2 = q(MX) * q(MX) + q(MY) * q(MY) + q(MZ) * q(MZ);
      return A.gm1 * (q(EN) - T(0.5) * m2 / q(RHO) - T(0.5) * b2) + T(0.5) * b2;
    };
    // the block constants are valid after the first barrier of the block
    Phys<T> P;
    T lam[3], lamh[3], dx2[3], dxT[3], dt, hdt, damp;
    auto read_constants = [&]() {
      P.gamma = A.gamma;
      P.gm1 = A.gm1;
      P.tau = A.tau;
      P.ch = kc[15];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lam[d] = kc[d];
        lamh[d] = kc[3 + d];
        dx2[d] = kc[6 + d];
        dxT[d] = kc[9 + d];
      }
      dt = kc[12];
      hdt = kc[13];
      damp = kc[14];
    };

    // u~ (MMC/LF) and J (resistive) at ring cell r of plane z (needs u planes z-1..z+1)
    auto predict_cell = [&](int z, int r) {
      const T* ul[3] = {uslot(z - 1), uslot(z), uslot(z + 1)};
      const int x = 1 + r % RW, y = 1 + r / RW;
      const int c = y * NP + x;
      if (HAS_T) {
        T w[NV], acc[NV];
        ldw<T, P2>(ul[1], c, w);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = w[v];
        T* tp = tslot(z);
        if (SCHEME == SCH_MMC) {
          T wm[NV], wp[NV], hp[NV], hm[NV];
          ldw<T, P2>(ul[1], c - 1, wm);
          ldw<T, P2>(ul[1], c + 1, wp);
          mmc_h<T, 0>(w, wp, P, hp);
          mmc_h<T, 0>(wm, w, P, hm);
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] -= lam[0] * (hp[v] - hm[v]);
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
          for (int v = 0; v < NV; ++v) tp[v * RING + r] = acc[v];
        } else {
          auto half = [&](auto Dc, const T* plm, int cm, const T* plp, int cp) {
            constexpr int D = decltype(Dc)::value;
            if constexpr (std::is_same<T, float>::value) {
              // the two half-states u +- phi/2 in the lanes of a float2
              float2 ab[NV], fab[NV];
              // the limited slopes of two variables at a time
#pragma unroll
              for (int v = 0; v + 1 < NV; v += 2) {
                const float2 wv = make_float2(w[v], w[v + 1]);
                const float2 lo = make_float2(plm[v * P2 + cm], plm[(v + 1) * P2 + cm]);
                const float2 hi = make_float2(plp[v * P2 + cp], plp[(v + 1) * P2 + cp]);
                const float2 ph = pair::limiter2<LIM>(pair::sub(wv, lo), pair::sub(hi, wv));
                ab[v] = pair::fma(pair::splat(ph.x), make_float2(0.5f, -0.5f), pair::splat(w[v]));
                ab[v + 1] = pair::fma(pair::splat(ph.y), make_float2(0.5f, -0.5f), pair::splat(w[v + 1]));
              }
              {
                const T ph = limiter<T, LIM>(w[NV - 1] - plm[(NV - 1) * P2 + cm], plp[(NV - 1) * P2 + cp] - w[NV - 1]);
                ab[NV - 1] = pair::fma(pair::splat(ph), make_float2(0.5f, -0.5f), pair::splat(w[NV - 1]));
              }
              pair::flux2<D, !(NDIM == 3 && NB == 16)>(ab, P, fab, nullptr);
#pragma unroll
              for (int v = 0; v < NV; ++v) acc[v] -= lamh[D] * (fab[v].x - fab[v].y);
            } else {
              T a[NV], b[NV], fa[NV], fb[NV];
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
            }
          };
          half(std::integral_constant<int, 0>(), ul[1], c - 1, ul[1], c + 1);
          half(std::integral_constant<int, 1>(), ul[1], c - NP, ul[1], c + NP);
          if (NDIM == 3) half(std::integral_constant<int, 2>(), ul[0], c, ul[2], c);
          T s[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) s[v] = T(0);
          if (A.eglm) eglm_src<T, NDIM, NP>(ul, c, dx2, s);
#pragma unroll
          for (int v = 0; v < NV; ++v) tp[v * RING + r] = acc[v] + hdt * s[v];
        }
      }
      if (RES) {
        T J[3];
        current<T, NDIM, NP>(ul, c, dx2, J);
        T* jp = jslot(z);
        jp[0 * RING + r] = J[0];
        jp[1 * RING + r] = J[1];
        jp[2 * RING + r] = J[2];
      }
    };

    // x (D=0) or y (D=1) face flux between in-plane cells cl and cl+st (full layout), with
    // the u~ ring cells rl and rl+rs
    // x face (yd false) or y face (yd true) flux between in-plane cells cl and cl+st (full
    // layout), with the u~ ring cells rl and rl+rs.  A y face is the x-face flux of the states
    // with the x and y components of m and B exchanged, exchanged back: F_y(U) = P F_x(P U)
    // with the same operations on the same operands, so both directions share one instance
    // of the flux code (and a warp may hold faces of both)
    auto face_xy = [&](bool yd, const T* up, const T* tp, int cl, int st, int rl, int rs, T* F) {
      if (SCHEME == SCH_MMC) {
        T w0[NV], w1[NV], w2[NV], w3[NV], t0[NV], t1[NV];
        ldw<T, P2>(up, cl - st, w0);
        ldw<T, P2>(up, cl, w1);
        ldw<T, P2>(up, cl + st, w2);
        ldw<T, P2>(up, cl + 2 * st, w3);
        ldw<T, RING>(tp, rl, t0);
        ldw<T, RING>(tp, rl + rs, t1);
        exch_xy(yd, w0);
        exch_xy(yd, w1);
        exch_xy(yd, w2);
        exch_xy(yd, w3);
        exch_xy(yd, t0);
        exch_xy(yd, t1);
        mmc_face<T, 0, LIM>(w0, w1, w2, w3, t0, t1, P, F);
      } else if (std::is_same<T, float>::value && SCHEME == SCH_LF && FLX == FLX_LF) {
        float2 ab[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float2 ulo = make_float2(up[v * P2 + cl - st], up[v * P2 + cl]);      // (u_i-1, u_i)
          const float2 umid = make_float2(up[v * P2 + cl], up[v * P2 + cl + st]);    // (u_i, u_i+1)
          const float2 uhi = make_float2(up[v * P2 + cl + st], up[v * P2 + cl + 2 * st]);
          const float2 ph = pair::limiter2<LIM>(pair::sub(umid, ulo), pair::sub(uhi, umid));
          const float2 tt = make_float2(tp[v * RING + rl], tp[v * RING + rl + rs]);
          ab[v] = pair::fma(ph, make_float2(0.5f, -0.5f), tt);
        }
        exch_xy(yd, ab);
        pair::lf_flux2<0, !(NDIM == 3 && NB == 16)>(ab, *reinterpret_cast<const Phys<float>*>(&P), reinterpret_cast<float*>(F), (float)kc[16]);
      } else {
        T a[NV], b[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T um = up[v * P2 + cl - st], u1 = up[v * P2 + cl];
          const T u2 = up[v * P2 + cl + st], u3 = up[v * P2 + cl + 2 * st];
          if (SCHEME == SCH_LF) {
            T phl = limiter<T, LIM>(u1 - um, u2 - u1);
            T phr = limiter<T, LIM>(u2 - u1, u3 - u2);
            a[v] = tp[v * RING + rl] + T(0.5) * phl;
            b[v] = tp[v * RING + rl + rs] - T(0.5) * phr;
          } else {
            a[v] = weno_minus_right<T>(um, u1, u2);
            b[v] = weno_plus_left<T>(u1, u2, u3);
          }
        }
        exch_xy(yd, a);
        exch_xy(yd, b);
        if (FLX == FLX_HLLC) hllc_flux<T, 0>(a, b, P, F);
        else if (FLX == FLX_HLLD) hlld_flux<T, 0>(a, b, P, F);
        else lf_flux<T, 0>(a, b, P, F);
      }
      exch_xy(yd, F);
    };

    // face register (reflux, Sec. 4.2): the flux through a boundary face cell of this block
    // (side 2d or 2d+1, face cell t0 + NB t1), written where the flux is computed; a WENO
    // step holds half of each stage's flux
    auto put_face = [&](int side, int t0, int t1, const T* F) {
      T* r = A.freg + (size_t)srl.slot * (2 * NDIM * NV * NB * NB) + (size_t)side * NV * NB * NB + t1 * NB + t0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T* rv = r + (size_t)v * NB * NB;
        // the full flux: the normal-momentum component gets the faces' reference back
        const bool vn = (v == MX && side < 2) || (v == MY && (side == 2 || side == 3)) || (v == MZ && side >= 4);
        const T fv = (PREF && vn) ? F[v] + kc[16] : F[v];
        *rv = STAGE == 0 ? fv : (STAGE == 1 ? T(0.5) * fv : *rv + T(0.5) * fv);
      }
    };

    // x face f (fx = f % (NB+1), row = f / (NB+1)) or y face f (col = f % NB, fy = f / NB)
    // of plane z into the face buffer (x faces first, then y faces)
    T* sfx = sf;
    T* sfy = sf + (size_t)NV * NFACE;
    // face k of plane z: x faces k < NFACE (f = row (NB+1) + fx), then y faces (f = fy NB + col)
    auto do_face = [&](int z, int k) {
      const bool yd = k >= NFACE;
      const int f = yd ? k - NFACE : k;
      const int row = f / (NB + 1), fx = f % (NB + 1);       // x face
      const int fy = f / NB, col = f % NB;                   // y face
      T F[NV];
      face_xy(yd, uslot(z), HAS_T ? tslot(z) : nullptr, yd ? (fy + 1) * NP + col + NG : (row + NG) * NP + fx + 1,
              yd ? NP : 1, yd ? fy * RW + col + 1 : (row + 1) * RW + fx, yd ? RW : 1, F);
      T* dst = (yd ? sfy : sfx) + f;
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * NFACE] = F[v];
      if (RFX && SCHEME == SCH_LF && srl.slot >= 0) {
        const int pos = yd ? fy : fx, t0 = yd ? col : row;
        if (pos == 0 || pos == NB) put_face((yd ? 2 : 0) + (pos ? 1 : 0), t0, NDIM == 3 ? z - NG : 0, F);
      }
    };

    // z face of the own column between planes z and z+1; um1 = the column's state at z-1
    auto face_z = [&](int z, const T* um1, T* F) {
      const T* p0 = uslot(z);
      const T* p1 = uslot(z + 1);
      const T* p2 = uslot(z + 2);
      if (SCHEME == SCH_MMC) {
        T w1[NV], w2[NV], w3[NV], t0[NV], t1[NV];
        ldw<T, P2>(p0, cown, w1);
        ldw<T, P2>(p1, cown, w2);
        ldw<T, P2>(p2, cown, w3);
        ldw<T, RING>(tslot(z), rown, t0);
        ldw<T, RING>(tslot(z + 1), rown, t1);
        mmc_face<T, 2, LIM>(um1, w1, w2, w3, t0, t1, P, F);
      } else if (std::is_same<T, float>::value && SCHEME == SCH_LF && FLX == FLX_LF) {
        float2 ab[NV];
        const T* t0p = tslot(z);
        const T* t1p = tslot(z + 1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float2 ulo = make_float2(um1[v], p0[v * P2 + cown]);
          const float2 umid = make_float2(p0[v * P2 + cown], p1[v * P2 + cown]);
          const float2 uhi = make_float2(p1[v * P2 + cown], p2[v * P2 + cown]);
          const float2 ph = pair::limiter2<LIM>(pair::sub(umid, ulo), pair::sub(uhi, umid));
          const float2 tt = make_float2(t0p[v * RING + rown], t1p[v * RING + rown]);
          ab[v] = pair::fma(ph, make_float2(0.5f, -0.5f), tt);
        }
        pair::lf_flux2<2, !(NDIM == 3 && NB == 16)>(ab, *reinterpret_cast<const Phys<float>*>(&P), reinterpret_cast<float*>(F), (float)kc[16]);
      } else {
        T a[NV], b[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T um = um1[v], u1 = p0[v * P2 + cown], u2 = p1[v * P2 + cown], u3 = p2[v * P2 + cown];
          if (SCHEME == SCH_LF) {
            T phl = limiter<T, LIM>(u1 - um, u2 - u1);
            T phr = limiter<T, LIM>(u2 - u1, u3 - u2);
            a[v] = tslot(z)[v * RING + rown] + T(0.5) * phl;
            b[v] = tslot(z + 1)[v * RING + rown] - T(0.5) * phr;
          } else {
            a[v] = weno_minus_right<T>(um, u1, u2);
            b[v] = weno_plus_left<T>(u1, u2, u3);
          }
        }
        if (FLX == FLX_HLLC) hllc_flux<T, 2>(a, b, P, F);
        else if (FLX == FLX_HLLD) hlld_flux<T, 2>(a, b, P, F);
        else lf_flux<T, 2>(a, b, P, F);
      }
    };

    // work list of one barrier interval: [predictor ring cells of plane zp (if any)] then
    // [x faces, then y faces, of plane zf], each kind padded to whole warps
    // each warp walks its own list of warp-sized units (see the schedule above); units of a
    // kind that this interval does not run are skipped
    auto work = [&](int zp, bool do_pred, int zf, bool do_faces) {
      const int wq = tid >> 5, lane = tid & 31;
      const int cnt = sched[wq][15];
      for (int k = 0; k < cnt; ++k) {
        const int u = sched[wq][k];
        if (u < NPU) {
          // q-th ring cell in row order, the corners 0, RW-1, RING-RW and RING-1 skipped
          const int q = u * 32 + lane;
          const int r = q + 1 + (q >= RW - 2) + (q >= RING - RW - 2);
          if (do_pred && q < G::NPC) predict_cell(zp, r);
        } else {
          const int k = (u - NPU) * 32 + lane;
          if (do_faces && k < 2 * NFACE) do_face(zf, k);
        }
      }
    };

    T Fzlo[NV], uprev[NV];
    // the own column's u~ B_z, psi and J of the previous plane (its ring slot is reused)
    T car_bz = T(0), car_psi = T(0), car_j[3] = {T(0), T(0), T(0)};
    bool ok = true;
    const bool PRED = HAS_T || RES;
    if (tid == 0) {
      issue_plane(0);
      if (NDIM == 3) {
        issue_plane(1);
        issue_plane(2);
        issue_plane(3);
      }
      // per-block constants, rounded to T while the first planes are in flight.  dt/dx at
      // level L is 2^L dt/dx0 exactly, and rounding to T commutes with scaling by powers of
      // two, so these equal the FP64 dt/dx, (dt/2)/dx, 2 dx, dx, dt, dt/2 rounded to T
      // without an FP64 division per block (the FP64 pipe runs at 1/64 of the FP32 rate)
      const ProbDyn dy = A.dyn[gg.problem];
      const T scale = (T)(1 << gg.level);
      for (int d = 0; d < 3; ++d) {
        const T lam_d = (T)dy.lam0[d] * (d < NDIM ? scale : T(1));
        const T dx_d = (T)gg.dx[d];
        kc[d] = lam_d;
        kc[3 + d] = T(0.5) * lam_d;
        kc[6 + d] = T(2) * dx_d;
        kc[9 + d] = dx_d;
      }
      const T dt_T = (T)dy.dt;
      kc[12] = dt_T;
      kc[13] = T(0.5) * dt_T;
      kc[14] = (T)dy.damp;
      kc[15] = (T)dy.ch;
    }
    // 3D: iteration z predicts plane z+1 and updates plane z (z >= NG); one call site per
    // work-item kind keeps the kernel's code small.  2D: a single plane.
    const int zlast = NDIM == 3 ? NB + NG - 1 : 0;
    for (int z = 0; z <= zlast; ++z) {
      if (NDIM == 3) {
        if (z == 0) {
          ok = wait_plane(0);
          if (ok) ok = wait_plane(1);
          if (ok) ok = wait_plane(2);
        } else {
          ok = wait_plane(z + 2);                               // in flight since z-1
        }
        if (!ok) break;
        if (z == 0) read_constants();
        if (PREF && z == 0 && tid == 0) kc[16] = total_pressure(uslot(NG), cown);   // read after the next barrier
        if (tid == 0 && z >= 1 && z + 3 <= NP - 1) issue_plane(z + 3);   // slot of z-1
        work(z + 1, PRED, z, z >= NG);                           // predictor z+1, faces of z
      } else {
        ok = wait_plane(0);
        if (!ok) break;
        read_constants();
        if (PREF && tid == 0) kc[16] = total_pressure(uslot(0), cown);           // read after the next barrier
        if (PRED) {
          work(0, true, 0, false);
          __syncthreads();
        }
        work(0, false, 0, true);
      }
      __syncthreads();
      // plane z-1's values for this plane's sources; plane z's are kept for the next, as the
      // predictor of plane z+2 overwrites plane z's ring slot in the next interval
      const T zm_bz = car_bz, zm_psi = car_psi;
      const T zm_j[3] = {car_j[0], car_j[1], car_j[2]};
      if (G::CARRY) {
        if (HAS_T) {
          car_bz = tslot(z)[BZ * RING + rown];
          car_psi = tslot(z)[PSI * RING + rown];
        }
        if (RES) {
#pragma unroll
          for (int q = 0; q < 3; ++q) car_j[q] = jslot(z)[q * RING + rown];
        }
      }
      T Fzhi[NV];
      if (NDIM == 3) {
        if (z >= 1) face_z(z, uprev, Fzhi);                     // face between planes z, z+1
        if (RFX && (z == NG - 1 || z == NB + NG - 1) && srl.slot >= 0) put_face(z == NG - 1 ? 4 : 5, tx, ty, Fzhi);
        if (z < NG) {
#pragma unroll
          for (int v = 0; v < NV; ++v) Fzlo[v] = Fzhi[v];
          ldw<T, P2>(uslot(z), cown, uprev);
          __syncthreads();
          continue;
        }
      }
      const T* P0 = uslot(z);
      const T* T0 = HAS_T ? tslot(z) : nullptr;
#pragma unroll 1
      for (int cc = 0; cc < CPT; ++cc) {
        if (CPT > 1) {
          const int col = tid + cc * NT;
          tx = col % NB;
          ty = col / NB;
          cown = (ty + NG) * NP + (tx + NG);
          rown = (ty + 1) * RW + (tx + 1);
        }
        T acc[NV];
        if (SCHEME == SCH_WENO) {
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] = T(0);
        } else {
          ldw<T, P2>(P0, cown, acc);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T fr = sfx[v * NFACE + ty * (NB + 1) + tx + 1];
          const T fl = sfx[v * NFACE + ty * (NB + 1) + tx];
          if (SCHEME == SCH_WENO) acc[v] -= (fr - fl) / dxT[0];
          else acc[v] -= lam[0] * (fr - fl);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T fr = sfy[v * NFACE + (ty + 1) * NB + tx];
          const T fl = sfy[v * NFACE + ty * NB + tx];
          if (SCHEME == SCH_WENO) acc[v] -= (fr - fl) / dxT[1];
          else acc[v] -= lam[1] * (fr - fl);
        }
        // z faces
        if (NDIM == 3) {
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
        T unext[NV];
        if (NDIM == 3) ldw<T, P2>(uslot(z + 1), cown, unext);
        if (A.eglm) {
          if (SCHEME == SCH_LF) {
            T tm[NV], tq[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) tm[v] = T(0);
            if (NDIM == 3) {
              if (G::CARRY) {
                tm[BZ] = zm_bz;                                   // the z-1 values the sources read
                tm[PSI] = zm_psi;
              } else {
                ldw<T, RING>(tslot(z - 1), rown, tm);
              }
              ldw<T, RING>(tslot(z + 1), rown, tq);
            }
            eglm_src_col<T, NDIM>(T0, RING, RW, rown, tm, tq, dx2, s);
          } else {
            eglm_src_col<T, NDIM>(P0, P2, NP, cown, uprev, unext, dx2, s);
          }
        }
        if (RES) {
          T jm[3] = {T(0), T(0), T(0)}, jq[3] = {T(0), T(0), T(0)};
          if (NDIM == 3) {
            const T* j2 = jslot(z + 1);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              jm[q] = G::CARRY ? zm_j[q] : jslot(z - 1)[q * RING + rown];
              jq[q] = j2[q * RING + rown];
            }
          }
          resist_src_col<T, NDIM, NP, RW>(jslot(z), rown, jm, jq, P0, cown, uprev, unext, dx2, eta, s);
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
        if (A.pushes) {
          // the two interior layers next to a face/edge/corner go into the facing ghost
          // region of the same-level neighbour there (padded 2,3 -> low side, NB,NB+1 -> high)
          const int x = tx + NG, y = ty + NG;
          const int fx = x < 2 * NG ? -1 : (x >= NB ? 1 : 0);
          const int fy = y < 2 * NG ? -1 : (y >= NB ? 1 : 0);
          const int fz = NDIM == 3 ? (z < 2 * NG ? -1 : (z >= NB ? 1 : 0)) : 0;
          if (fx | fy | fz) {
            for (int kz = 0; kz < (fz ? 2 : 1); ++kz)
              for (int ky = 0; ky < (fy ? 2 : 1); ++ky)
                for (int kx = 0; kx < (fx ? 2 : 1); ++kx) {
                  const int ex = kx ? fx : 0, ey = ky ? fy : 0, ez = kz ? fz : 0;
                  if (!(ex | ey | ez)) continue;
                  const PushEntry pe = spush[(ex + 1) + 3 * (ey + 1) + 9 * (ez + 1)];
                  if (pe.dst < 0) continue;
                  T* db = A.u_out + (size_t)pe.dst * NV * S;
                  const size_t dc = ((size_t)(z + pe.off[2]) * NP + (y + pe.off[1])) * NP + (x + pe.off[0]);
#pragma unroll
                  for (int v = 0; v < NV; ++v) db[(size_t)v * S + dc] = out[v];
                }
          }
        }
        // cells next to a face where this block is the coarse side change again in the reflux
        // pass, which checks them and adds them to the fused diagnostics itself
        const int cm = RFX ? srl.coarse_mask : 0;
        const bool refluxed = RFX && cm != 0 && (((cm & 1) && tx == 0) || ((cm & 2) && tx == NB - 1) ||
                                          ((cm & 4) && ty == 0) || ((cm & 8) && ty == NB - 1) ||
                                          (NDIM == 3 && (((cm & 16) && z == NG) || ((cm & 32) && z == NB + NG - 1))));
        if (STAGE != 1 && !refluxed) {
          bool fin = true;
#pragma unroll
          for (int v = 0; v < NV; ++v) fin = fin && isfinite(out[v]);
          if (!fin) errbits |= 1u;
          else {
            T pr = pressure<T>(out, P);
            if (!(out[RHO] > T(0)) || pr < T(0)) errbits |= 2u;
            if (A.dyn_next) {
              T am = alpha_p<T, 0>(out, pr, P);
              am = dmax<T>(am, alpha_p<T, 1>(out, pr, P));
              if (NDIM == 3) am = dmax<T>(am, alpha_p<T, 2>(out, pr, P));
              alpha_max = dmax<T>(alpha_max, am);
            }
          }
          if (!fin) alpha_max = (T)NAN;
          if (A.sums) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              // Kahan: csum - ccmp carries the column sum
              const T y = out[v] - ccmp[v];
              const T t = csum[v] + y;
              ccmp[v] = (t - csum[v]) - y;
              csum[v] = t;
            }
          }
        }
        if (NDIM == 3) ldw<T, P2>(P0, cown, uprev);
      }  // the thread's columns
      if (RFX && SCHEME != SCH_LF && srl.slot >= 0 && tid < 4 * NB) {
        // this plane's x and y boundary faces (still in the face buffer) into the face
        // register (LF writes them where it computes them: either place suits one scheme's
        // register allocation better)
        const int side = tid / NB, t0 = tid % NB;
        const T* src = side < 2 ? sfx + t0 * (NB + 1) + (side ? NB : 0) : sfy + (side == 3 ? NB * NB : 0) + t0;
        T F[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = src[v * NFACE];
        put_face(side, t0, NDIM == 3 ? z - NG : 0, F);
      }
      __syncthreads();
    }
    if (!ok) break;
    // reductions of the fused diagnostics, in T within each warp (TwoSum pairs for the sums),
    // then FP64 across warps.  The per-thread maxima and compensated sums keep accumulating
    // over the CTA's consecutive blocks of one problem and level (equal cell volumes) and are
    // reduced once that run ends -- a persistent grid given contiguous block ranges reduces
    // once per run instead of once per block (the decision is the same on every thread)
    bool flush = true;
    if (bi + (int)gridDim.x < A.nblocks) {
      const BlockGeo gn = A.geo[A.blocks[bi + gridDim.x]];
      flush = gn.problem != gg.problem || gn.level != gg.level;
    }
    if ((A.dyn_next || A.sums) && flush) {
      double* red = reinterpret_cast<double*>(sf);     // (NV+1) x 32 doubles
      const int lane = tid & 31, wid = tid >> 5;
      T am = alpha_max;
      for (int o = 16; o > 0; o >>= 1) {
        const T t = __shfl_xor_sync(0xffffffffu, am, o);
        am = (t != t || am != am) ? (T)NAN : dmax<T>(am, t);
      }
      // after the butterflies every lane holds the warp's (hi, lo) of variable v; lane v
      // keeps variable v's pair and widens it to one FP64 value (one conversion per warp:
      // the FP64 pipe runs at 1/64 of the FP32 rate), lane NV the alpha maximum
      T hsel = am, lsel = T(0);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T hi = csum[v], lo = -ccmp[v];
        for (int o = 16; o > 0; o >>= 1) {
          const T h2 = __shfl_xor_sync(0xffffffffu, hi, o);
          const T l2 = __shfl_xor_sync(0xffffffffu, lo, o);
          two_sum_acc<T>(hi, lo, h2, l2);
        }
        if (lane == v) { hsel = hi; lsel = lo; }
      }
      if (lane < NV) red[lane * 32 + wid] = (double)hsel + (double)lsel;
      if (lane == NV) red[NV * 32 + wid] = (double)hsel;
      __syncthreads();
      if (tid <= NV) {
        // warp 0: lane v adds variable v over the warps (in warp order), lane NV takes the
        // alpha maximum
        const int nw = (NT + 31) / 32;
        if (tid == NV) {
          double a2 = 0.0;
          for (int q = 0; q < nw; ++q) {
            const double t = red[NV * 32 + q];
            a2 = (t != t || a2 != a2) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(a2, t);
          }
          // alpha >= 0: its IEEE bit pattern orders like the value (NaN above everything)
          if (A.dyn_next) atomicMax(&A.dyn_next[gg.problem].alpha_bits, (unsigned long long)__double_as_longlong(a2));
        } else if (A.sums) {
          const double vol = gg.dx[0] * gg.dx[1] * (NDIM == 3 ? gg.dx[2] : 1.0);
          double t = 0.0;
          for (int q = 0; q < nw; ++q) t += red[tid * 32 + q];
          atomicAdd(&A.sums[gg.problem * NV + tid], t * vol);
        }
      }
      __syncthreads();
      alpha_max = T(0);
#pragma unroll
      for (int v = 0; v < NV; ++v) { csum[v] = T(0); ccmp[v] = T(0); }
    }
  }
  if (*status != 0) {
    errbits |= 4u;
    // a copy never completed: wait (bounded again) for the copies still in flight so none
    // lands after the block has left
    if (tid == 0)
      for (int q = 0; q < UPL; ++q)
        if ((inflight >> q) & 1u) mbar_wait_bounded(&bars[q], (phase >> q) & 1u);
  }
  unsigned e = errbits;
  for (int o = 16; o > 0; o >>= 1) e |= __shfl_xor_sync(0xffffffffu, e, o);
  if ((tid & 31) == 0 && e) atomicOr(A.err_word, e);
}

}  // namespace mapgb
