// aux.cuh -- ghost fill, restriction, CFL reduction, refinement flags, conservation sums,
// host-layout packing and regrid kernels.
#pragma once
#include "map_internal.hpp"
#include "physics.cuh"
#include "step.cuh"

namespace mapgb {

// Ghost fill of the leaves of one level (Sec. 4.3): every ghost cell gathers from the
// block its region resolves to -- a copy from a same-level block, or the conservative
// minmod prolongation of the covering coarser leaf (whose ghosts an earlier level pass
// filled).  Region tables come from the host tree.
template <int NDIM, int NB>
struct Shell {
  static constexpr int NP = NB + 4;
  static constexpr int P2 = NP * NP;
  static constexpr int PLANE_GHOSTS = P2 - NB * NB;                  // ghost cells of an interior plane
  static constexpr int COUNT = NDIM == 3 ? 2 * NG * P2 + NB * PLANE_GHOSTS : PLANE_GHOSTS;
  // g-th ghost cell of a block -> padded (i, j, k): the 2*NG full ghost planes first (3D),
  // then per interior plane its NG ghost rows on each side and NG ghost columns on each side
  static __device__ __forceinline__ void cell(int g, int& i, int& j, int& k) {
    if (NDIM == 3) {
      if (g < 2 * NG * P2) {
        const int pl = g / P2, c = g % P2;
        k = pl < NG ? pl : NB + pl;
        j = c / NP;
        i = c % NP;
        return;
      }
      g -= 2 * NG * P2;
      k = NG + g / PLANE_GHOSTS;
      g %= PLANE_GHOSTS;
    } else {
      k = 0;
    }
    constexpr int ROWS = 2 * NG * NP;          // full ghost rows of the plane
    if (g < ROWS) {
      const int r = g / NP;
      j = r < NG ? r : NB + r;
      i = g % NP;
    } else {
      g -= ROWS;                                // NB interior rows x 2*NG ghost columns
      j = NG + g / (2 * NG);
      const int q = g % (2 * NG);
      i = q < NG ? q : NB + q;
    }
  }
};

template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) fill_kernel(T* __restrict__ u, const int* __restrict__ blocks,
                                                   int n, const GhostRegion* __restrict__ regions, int skip_pushed,
                                                   int v0, int v1) {
  using G = Geo<NDIM, NB>;
  using SH = Shell<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, S = G::S;
  __shared__ GhostRegion reg[27];
  for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
    const int blk = blocks[bi];
    __syncthreads();
    for (int r = threadIdx.x; r < 27; r += blockDim.x) reg[r] = regions[(size_t)blk * 27 + r];
    __syncthreads();
    T* ub = u + (size_t)blk * NV * S;
    for (int g = threadIdx.x; g < SH::COUNT; g += blockDim.x) {
      int i, j, k;
      SH::cell(g, i, j, k);
      const int c = (k * NP + j) * NP + i;
      const int rx = i < NG ? 0 : (i >= NG + NB ? 2 : 1);
      const int ry = j < NG ? 0 : (j >= NG + NB ? 2 : 1);
      const int rz = NDIM == 3 ? (k < NG ? 0 : (k >= NG + NB ? 2 : 1)) : 1;
      const GhostRegion& gr = reg[rx + 3 * ry + 9 * rz];
      if (skip_pushed && gr.pushed) continue;      // written by the source's step kernel
      const T* sb = u + (size_t)gr.src * NV * S;
      if (gr.kind == 0) {
        const int si = gr.m[0] * i + gr.a[0], sj = gr.m[1] * j + gr.a[1];
        const int sk = NDIM == 3 ? gr.m[2] * k + gr.a[2] : 0;
        const int sc = (sk * NP + sj) * NP + si;
        T val[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v >= v0 && v < v1) val[v] = sb[(size_t)v * S + sc];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v >= v0 && v < v1) ub[(size_t)v * S + c] = val[v];
      } else {
        const int gi = gr.m[0] * i + gr.a[0], gj = gr.m[1] * j + gr.a[1];
        const int gk = NDIM == 3 ? gr.m[2] * k + gr.a[2] : 0;
        const int ci = (gi >> 1) - gr.corg[0] + NG, cj = (gj >> 1) - gr.corg[1] + NG;
        const int ck = NDIM == 3 ? (gk >> 1) - gr.corg[2] + NG : 0;
        const int cc = (ck * NP + cj) * NP + ci;
        const T ox = (gi & 1) ? T(0.25) : T(-0.25);
        const T oy = (gj & 1) ? T(0.25) : T(-0.25);
        const T oz = (gk & 1) ? T(0.25) : T(-0.25);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (v < v0 || v >= v1) continue;
          const T* f = sb + (size_t)v * S;
          T val = f[cc];
          val += minmod<T>(f[cc + 1] - f[cc], f[cc] - f[cc - 1]) * ox;
          val += minmod<T>(f[cc + NP] - f[cc], f[cc] - f[cc - NP]) * oy;
          if (NDIM == 3) val += minmod<T>(f[cc + P2] - f[cc], f[cc] - f[cc - P2]) * oz;
          ub[(size_t)v * S + c] = val;
        }
      }
    }
  }
}

// Parents of one level become the mean of their 2^ndim children (Sec. 4.3 step (1)).
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) restrict_kernel(T* __restrict__ u, const int* __restrict__ parents,
                                                       int n, const int* __restrict__ children) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
    const int par = parents[bi];
    int ch[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ch[q] = children[(size_t)par * 8 + q];
    T* pb = u + (size_t)par * NV * S;
    for (int c = threadIdx.x; c < NI; c += blockDim.x) {
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int dst = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
#pragma unroll 1
      for (int v = 0; v < NV; ++v) {
        T sum = T(0);
        for (int dz = 0; dz < (NDIM == 3 ? 2 : 1); ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              const int fi = 2 * i + dx, fj = 2 * j + dy, fk = 2 * k + dz;
              const int cb = (fi / NB) | ((fj / NB) << 1) | ((NDIM == 3 ? fk / NB : 0) << 2);
              const int lc = ((NDIM == 3 ? fk % NB + NG : 0) * NP + fj % NB + NG) * NP + fi % NB + NG;
              sum += u[(size_t)ch[cb] * NV * S + (size_t)v * S + lc];
            }
        pb[(size_t)v * S + dst] = sum / T(1 << NDIM);
      }
    }
  }
}

// Maximum that keeps a NaN from either side (fmax drops it): a NaN cell anywhere makes the
// reduced signal speed NaN, so the time step built from it is rejected.
template <typename T>
__device__ __forceinline__ T nan_max(T a, T b) {
  return (a != a) ? a : ((b != b) ? b : fmax(a, b));
}

template <typename T>
__device__ __forceinline__ void load_global(const T* b, size_t S, int c, T* w) {
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v] = b[(size_t)v * S + c];
}

// alpha_g: max over leaf interior cells and directions of |v_d| + c_f,d (Sec. 3.7).
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) cfl_kernel(const T* __restrict__ u, const int* __restrict__ blocks, int n,
                                                  const BlockGeo* __restrict__ geo, ProbDyn* dyn, T gamma, T gm1,
                                                  double kappa0) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  __shared__ double red[32], redk[32];
  Phys<T> P;
  P.gamma = gamma;
  P.gm1 = gm1;
  P.ch = T(0);
  P.tau = T(0);
  for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
    const int blk = blocks[bi];
    const T* ub = u + (size_t)blk * NV * S;
    // maxima in T within each warp (a maximum is exact in any precision, and widening to
    // FP64 is exact and monotone), then FP64 across warps
    const bool cond = kappa0 > 0.0;
    const T kap0 = (T)kappa0;
    T am = T(0), km = T(0);
    for (int c = threadIdx.x; c < NI; c += blockDim.x) {
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int cc = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
      T w[NV];
      load_global<T>(ub, S, cc, w);
      const T p = pressure<T>(w, P);
      T a = alpha_p<T, 0>(w, p, P);
      a = nan_max<T>(a, alpha_p<T, 1>(w, p, P));
      if (NDIM == 3) a = nan_max<T>(a, alpha_p<T, 2>(w, p, P));
      am = nan_max<T>(am, a);
      if (cond) {
        // kappa T / p read as kappa / rho, kappa = kappa0 T^(5/2), T = max(p, 0) / rho
        const T tt = (p < T(0) ? T(0) : p) / w[RHO];
        const T kr = kap0 * (tt * tt * sqrt(tt)) / w[RHO];
        km = nan_max<T>(km, kr);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      am = nan_max<T>(am, __shfl_xor_sync(0xffffffffu, am, o));
      km = nan_max<T>(km, __shfl_xor_sync(0xffffffffu, km, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = (double)am;
      redk[threadIdx.x >> 5] = (double)km;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, kk = 0.0;
      for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) {
        a = nan_max<double>(a, red[q]);
        kk = nan_max<double>(kk, redk[q]);
      }
      atomicMax(&dyn[geo[blk].problem].alpha_bits, (unsigned long long)__double_as_longlong(a));
      if (kappa0 > 0.0) atomicMax(&dyn[geo[blk].problem].kmax_bits, (unsigned long long)__double_as_longlong(kk));
    }
    __syncthreads();
  }
}

// Per-block maxima of alpha (the allocation-free CFL variant): partial[b] = max over the
// interior cells of block b and the directions of |v_d| + c_f,d.
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) cfl_partial_kernel(const T* __restrict__ u, int nblocks, T gamma, T gm1,
                                                          double* __restrict__ partial) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  __shared__ double red[32];
  Phys<T> P;
  P.gamma = gamma;
  P.gm1 = gm1;
  P.ch = T(0);
  P.tau = T(0);
  for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const T* ub = u + (size_t)blk * NV * S;
    T am = T(0);                     // in T within each warp, as in cfl_kernel
    for (int c = threadIdx.x; c < NI; c += blockDim.x) {
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int cc = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
      T w[NV];
      load_global<T>(ub, S, cc, w);
      const T p = pressure<T>(w, P);
      T a = alpha_p<T, 0>(w, p, P);
      a = nan_max<T>(a, alpha_p<T, 1>(w, p, P));
      if (NDIM == 3) a = nan_max<T>(a, alpha_p<T, 2>(w, p, P));
      am = nan_max<T>(am, a);
    }
    for (int o = 16; o > 0; o >>= 1) am = nan_max<T>(am, __shfl_xor_sync(0xffffffffu, am, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = am;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) a = nan_max<double>(a, red[q]);
      partial[blk] = a;     // every slot < nblocks is written before it is read
    }
    __syncthreads();
  }
}

// Refinement estimator (Sec. 4.5), computed in FP64 from the pool values, over the
// interior and the first ghost ring; block maximum -> flag.
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) flags_kernel(FlagLaunch L) {
  // the estimator runs in the pool's precision: FP64 pools bitwise as the FP64 formula, FP32
  // pools in FP32 (decisions then differ from FP64 only within float rounding of a threshold)
  using R = T;
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, S = G::S;
  constexpr int NR = NDIM == 3 ? (NB + 2) * (NB + 2) * (NB + 2) : (NB + 2) * (NB + 2);
  __shared__ double red[32];
  const T* u = (const T*)L.u;
  const R gm1 = (R)(L.gamma - 1.0);
  const R bias = (R)L.r.bias, filt = (R)L.r.filter;
  const R half_sqrt3 = (R)(1.7320508075688772 / 2.0);
  // the pool's pressure recovery (FP32 pools: with its FP64 fallback at low e_int / e)
  Phys<T> PP;
  PP.gamma = (T)L.gamma;
  PP.gm1 = (T)gm1;
  PP.ch = T(0);
  PP.tau = (T)L.tau;
  auto pres = [&](const T* ub, int c) -> R {
    R w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = (R)ub[(size_t)v * S + c];
    return pressure<T>(w, PP);
  };
  const int offs[3] = {1, NP, P2};
  for (int bi = blockIdx.x; bi < L.nblocks; bi += gridDim.x) {
    const int blk = L.blocks[bi];
    const BlockGeo gg = L.geo[blk];
    const T* ub = u + (size_t)blk * NV * S;
    double mindx = gg.dx[0];
    for (int d = 1; d < NDIM; ++d) mindx = fmin(mindx, gg.dx[d]);
    const R lvf = (R)L.level_factor[gg.level < 16 ? gg.level : 15];
    const R two_dx[3] = {(R)(2.0 * gg.dx[0]), (R)(2.0 * gg.dx[1]), (R)(NDIM == 3 ? 2.0 * gg.dx[2] : 1.0)};
    R emax = R(0);
    for (int q = threadIdx.x; q < NR; q += blockDim.x) {
      const int i = 1 + q % (NB + 2), j = 1 + (q / (NB + 2)) % (NB + 2);
      const int k = NDIM == 3 ? 1 + q / ((NB + 2) * (NB + 2)) : 0;
      const int c = (k * NP + j) * NP + i;
      auto est = [&](auto field, R eps) -> R {
        R s1 = R(0), s2 = R(0);
        const R f0 = field(c);
        for (int d = 0; d < NDIM; ++d) {
          const R fp = field(c + offs[d]), fm = field(c - offs[d]);
          const R d1 = fp - fm;
          const R d2 = fp - R(2) * f0 + fm;
          s1 += d1 * d1;
          s2 += d2 * d2;
        }
        const R du = half_sqrt3 * sqrt(s1);
        const R d2u = sqrt(s2);
        const R au = fabs(f0) + eps;
        const R e = bias * du / au + (R(1) - bias) * d2u / (du + filt * au);
        return e * lvf;
      };
      if (L.r.var_mask & 1) emax = fmax(emax, est([&](int cc) { return (R)ub[RHO * (size_t)S + cc]; }, (R)L.r.eps_rho));
      if (L.r.var_mask & 2) emax = fmax(emax, est([&](int cc) { return pres(ub, cc); }, (R)L.r.eps_p));
      if (L.r.var_mask & 4) {
        auto cd = [&](int comp, int d) -> R {
          if (d >= NDIM) return R(0);
          return ((R)ub[(size_t)comp * S + c + offs[d]] - (R)ub[(size_t)comp * S + c - offs[d]]) / two_dx[d];
        };
        const R jx = cd(BZ, 1) - cd(BY, 2);
        const R jy = cd(BX, 2) - cd(BZ, 0);
        const R jz = cd(BY, 0) - cd(BX, 1);
        const R bx = ub[(size_t)BX * S + c], by = ub[(size_t)BY * S + c], bz = ub[(size_t)BZ * S + c];
        const R e = sqrt(jx * jx + jy * jy + jz * jz) * (R)mindx / (sqrt(bx * bx + by * by + bz * bz) + (R)L.r.eps_b);
        emax = fmax(emax, e);
      }
    }
    double em = (double)emax;
    for (int o = 16; o > 0; o >>= 1) em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = em;
    __syncthreads();
    if (threadIdx.x == 0) {
      double e = 0.0;
      for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) e = fmax(e, red[q]);
      int8_t f = 0;
      if (e > L.r.thr && gg.level < L.r.max_level) f = 1;
      else if (e < L.r.coarsen_thr && gg.level > 0) f = -1;
      L.flags[bi] = f;
      if (L.est) L.est[bi] = e;
    }
    __syncthreads();
  }
}

// FP64 conservation sums of the leaf interiors: sum U * cell volume per problem.
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) sums_kernel(SumLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  __shared__ double red[NV][32];
  const T* u = (const T*)L.u;
  for (int bi = blockIdx.x; bi < L.nblocks; bi += gridDim.x) {
    const int blk = L.blocks[bi];
    const BlockGeo gg = L.geo[blk];
    const T* ub = u + (size_t)blk * NV * S;
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
    for (int c = threadIdx.x; c < NI; c += blockDim.x) {
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int cc = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] += (double)ub[(size_t)v * S + cc];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      for (int o = 16; o > 0; o >>= 1) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
      if ((threadIdx.x & 31) == 0) red[v][threadIdx.x >> 5] = s[v];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) t += red[threadIdx.x][q];
      const double vol = gg.dx[0] * gg.dx[1] * (NDIM == 3 ? gg.dx[2] : 1.0);
      atomicAdd(&L.sums[gg.problem * NV + threadIdx.x], t * vol);
    }
    __syncthreads();
  }
}

// Host layout [n][9][nz][nb][nb] (FP64) <-> pool interiors.
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) pack_kernel(PackLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  T* u = (T*)L.u;
  for (int bi = blockIdx.x; bi < L.nblocks; bi += gridDim.x) {
    const int blk = L.blocks[bi];
    T* ub = u + (size_t)blk * NV * S;
    double* hb = L.host_layout + (size_t)bi * NV * NI;
    float* hf = reinterpret_cast<float*>(L.host_layout) + (size_t)bi * NV * NI;
    for (int q = threadIdx.x; q < NV * NI; q += blockDim.x) {
      const int v = q / NI, c = q % NI;
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int cc = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
      if (L.to_pool) ub[(size_t)v * S + cc] = L.staging_f32 ? (T)hf[q] : (T)hb[q];
      else if (L.staging_f32) hf[q] = (float)ub[(size_t)v * S + cc];
      else hb[q] = (double)ub[(size_t)v * S + cc];
    }
  }
}

// Regrid: copy kept / coarsened leaves, prolong new children from their old parent leaf
// (Sec. 4.3 formula applied to interior cells; the old parent's ghosts are filled).
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) regrid_kernel(RegridLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, P2 = G::P2, S = G::S;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  const T* uo = (const T*)L.u_old;
  T* un = (T*)L.u_new;
  for (int ti = blockIdx.x; ti < L.ntasks; ti += gridDim.x) {
    const RegridTask tk = L.tasks[ti];
    const T* sb = uo + (size_t)tk.src * NV * S;
    T* db = un + (size_t)tk.dst * NV * S;
    const int bx = tk.cb & 1, by = (tk.cb >> 1) & 1, bz = (tk.cb >> 2) & 1;
    for (int c = threadIdx.x; c < NI; c += blockDim.x) {
      const int i = c % NB, j = (c / NB) % NB, k = NDIM == 3 ? c / (NB * NB) : 0;
      const int dc = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
      if (tk.kind == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) db[(size_t)v * S + dc] = sb[(size_t)v * S + dc];
      } else {
        const int gi = bx * NB + i, gj = by * NB + j, gk = bz * NB + k;
        const int cc = ((NDIM == 3 ? (gk >> 1) + NG : 0) * NP + (gj >> 1) + NG) * NP + (gi >> 1) + NG;
        const T ox = (gi & 1) ? T(0.25) : T(-0.25);
        const T oy = (gj & 1) ? T(0.25) : T(-0.25);
        const T oz = (gk & 1) ? T(0.25) : T(-0.25);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T* f = sb + (size_t)v * S;
          T val = f[cc];
          val += minmod<T>(f[cc + 1] - f[cc], f[cc] - f[cc - 1]) * ox;
          val += minmod<T>(f[cc + NP] - f[cc], f[cc] - f[cc - NP]) * oy;
          if (NDIM == 3) val += minmod<T>(f[cc + P2] - f[cc], f[cc] - f[cc - P2]) * oz;
          db[(size_t)v * S + dc] = val;
        }
      }
    }
  }
}


// Reflux (Sec. 4.2, boundary step (2), after Berger and Colella): one CTA per coarse leaf
// with coarse/fine faces.  For every face cell of such a face the coarse flux recorded by the
// step kernel is replaced by the mean of the fine fluxes covering the cell:
//   u_c += lam (F_fine - F_coarse) on a low face, u_c -= lam (F_fine - F_coarse) on a high one
// (lam = dt / dx_d of the coarse leaf; psi's correction carries the damping factor the step
// already applied).  Faces go in the order (d, low then high) with a barrier between them, so a
// cell on two such faces is corrected in a fixed order.  Then every corrected cell is checked
// and stored again into the ghost regions of the same-level leaves that copy it, and, in the
// fused form, added to alpha_g and the FP64 sums (the step kernel left these cells out).
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) reflux_kernel(RefluxLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int NF = NDIM == 3 ? NB * NB : NB;          // face cells per face
  constexpr int H = NB / 2;
  constexpr size_t NB2 = (size_t)NB * NB;
  constexpr size_t PER = (size_t)2 * NDIM * NV * NB2;   // one register slot
  __shared__ double red[NV + 1][32];
  const RefluxTask& tk = L.tasks[blockIdx.x];
  const int q = tk.coarse;
  const BlockGeo gg = L.geo[q];
  const ProbDyn dy = L.dyn[gg.problem];
  T* ub = (T*)L.u + (size_t)q * NV * S;
  const T* freg = (const T*)L.freg;
  const T damp = (T)dy.damp;
  int mask = 0;
  for (int f = 0; f < 2 * NDIM; ++f)
    if (tk.fslot[f][0] >= 0) mask |= 1 << f;
  // padded offset of the coarse cell on face (d, side) at face cell (t0, t1)
  auto cell_of = [&](int d, int side, int t0, int t1, int* ci) {
    const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
    ci[0] = ci[1] = ci[2] = 0;
    ci[d] = side ? NB - 1 : 0;
    ci[da] = t0;
    if (NDIM == 3) ci[db] = t1;
    return ((NDIM == 3 ? ci[2] + NG : 0) * NP + ci[1] + NG) * NP + ci[0] + NG;
  };
  if (L.nsub && L.it >= L.nsub[gg.problem]) return;        // no substep for this problem
  const double dtp = L.hsub ? L.hsub[gg.problem] : dy.dt;
  for (int d = 0; d < NDIM; ++d)
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      if (!((mask >> f) & 1)) continue;
      const T lam = (T)(dtp / gg.dx[d]);
      const T* rc = freg + (size_t)tk.cslot * PER + (size_t)f * NV * NB2;
      for (int idx = threadIdx.x; idx < NF; idx += blockDim.x) {
        const int t0 = idx % NB, t1 = NDIM == 3 ? idx / NB : 0;
        const int k = t0 / H + (NDIM == 3 ? 2 * (t1 / H) : 0);
        const T* rf = freg + (size_t)tk.fslot[f][k] * PER + (size_t)(2 * d + 1 - side) * NV * NB2;
        const int f0 = 2 * (t0 - (t0 / H) * H), f1 = NDIM == 3 ? 2 * (t1 - (t1 / H) * H) : 0;
        int ci[3];
        const int c = cell_of(d, side, t0, t1, ci);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (v < L.v0 || v >= L.v1) continue;
          const T* fv = rf + (size_t)v * NB2;
          T ff;
          if (NDIM == 2) ff = T(0.5) * (fv[f0] + fv[f0 + 1]);
          else ff = T(0.25) * ((fv[f1 * NB + f0] + fv[f1 * NB + f0 + 1]) +
                               (fv[(f1 + 1) * NB + f0] + fv[(f1 + 1) * NB + f0 + 1]));
          T corr = lam * (ff - rc[(size_t)v * NB2 + t1 * NB + t0]);
          if (v == PSI) corr = corr * damp;
          T* cell = ub + (size_t)v * S + c;
          *cell = side ? *cell - corr : *cell + corr;
        }
      }
      __syncthreads();
    }
  // checks, pushes and fused diagnostics, once per corrected cell (a cell on several such
  // faces is taken with the first of them)
  Phys<T> P;
  P.gamma = (T)L.gamma;
  P.gm1 = (T)(L.gamma - 1.0);
  P.ch = T(0);
  P.tau = (T)L.tau;
  unsigned errbits = 0;
  T am = T(0);
  double sum[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) sum[v] = 0.0;
  for (int d = 0; d < NDIM; ++d)
    for (int side = 0; side < 2; ++side) {
      const int f = 2 * d + side;
      if (!((mask >> f) & 1)) continue;
      for (int idx = threadIdx.x; idx < NF; idx += blockDim.x) {
        const int t0 = idx % NB, t1 = NDIM == 3 ? idx / NB : 0;
        int ci[3];
        const int c = cell_of(d, side, t0, t1, ci);
        bool first = true;
        for (int f2 = 0; f2 < f; ++f2)
          if (((mask >> f2) & 1) && ci[f2 >> 1] == ((f2 & 1) ? NB - 1 : 0)) first = false;
        if (!first) continue;
        T w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = ub[(size_t)v * S + c];
        bool fin = true;
#pragma unroll
        for (int v = 0; v < NV; ++v) fin = fin && isfinite(w[v]);
        if (!fin) {
          errbits |= 1u;
          am = (T)NAN;
        } else {
          const T pr = pressure<T>(w, P);
          if (!(w[RHO] > T(0)) || pr < T(0)) errbits |= 2u;
          T a = alpha_p<T, 0>(w, pr, P);
          a = dmax<T>(a, alpha_p<T, 1>(w, pr, P));
          if (NDIM == 3) a = dmax<T>(a, alpha_p<T, 2>(w, pr, P));
          if (!(am != am)) am = dmax<T>(am, a);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) sum[v] += (double)w[v];
        // the same-level leaves that copy this cell into their ghosts
        const int x = ci[0] + NG, y = ci[1] + NG, z = NDIM == 3 ? ci[2] + NG : 0;
        const int fx = x < 2 * NG ? -1 : (x >= NB ? 1 : 0);
        const int fy = y < 2 * NG ? -1 : (y >= NB ? 1 : 0);
        const int fz = NDIM == 3 ? (z < 2 * NG ? -1 : (z >= NB ? 1 : 0)) : 0;
        for (int kz = 0; kz < (fz ? 2 : 1); ++kz)
          for (int ky = 0; ky < (fy ? 2 : 1); ++ky)
            for (int kx = 0; kx < (fx ? 2 : 1); ++kx) {
              const int ex = kx ? fx : 0, ey = ky ? fy : 0, ez = kz ? fz : 0;
              if (!(ex | ey | ez)) continue;
              const PushEntry pe = L.pushes[(size_t)q * 27 + (ex + 1) + 3 * (ey + 1) + 9 * (ez + 1)];
              if (pe.dst < 0) continue;
              T* db = (T*)L.u + (size_t)pe.dst * NV * S;
              const size_t dc = ((size_t)(z + pe.off[2]) * NP + (y + pe.off[1])) * NP + (x + pe.off[0]);
#pragma unroll
              for (int v = 0; v < NV; ++v) db[(size_t)v * S + dc] = w[v];
            }
      }
    }
  unsigned e = errbits;
  for (int o = 16; o > 0; o >>= 1) e |= __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0 && e) atomicOr(L.err_word, e);
  if (!L.dyn_next && !L.sums) return;
  double a2 = (double)am;
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, a2, o);
    a2 = (t != t || a2 != a2) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(a2, t);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
    for (int o = 16; o > 0; o >>= 1) sum[v] += __shfl_xor_sync(0xffffffffu, sum[v], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[NV][wid] = a2;
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v][wid] = sum[v];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) / 32;
    double a = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) {
      const double t = red[NV][w2];
      a = (t != t || a != a) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(a, t);
    }
    if (L.dyn_next) atomicMax(&L.dyn_next[gg.problem].alpha_bits, (unsigned long long)__double_as_longlong(a));
    if (L.sums) {
      const double vol = gg.dx[0] * gg.dx[1] * (NDIM == 3 ? gg.dx[2] : 1.0);
      for (int v = 0; v < NV; ++v) {
        double t = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) t += red[v][w2];
        atomicAdd(&L.sums[gg.problem * NV + v], t * vol);
      }
    }
  }
}


// Thermal conduction (Sec. 3.6), one substep on one leaf per CTA, in place on the energy:
//   e_i += h sum_d (F_d,i+1/2 - F_d,i-1/2) / dx_d,  kappa = kappa0 T^(5/2), T = max(p,0)/rho,
//   isotropic:     F = sqrt(kappa_l kappa_r) (T_r - T_l) / dx_d,
//   along B:       F = sqrt(kappa_l kappa_r) b_d (b . grad T), b = B_f / |B_f| with B_f the
//                  mean of the two cells' B, transverse derivatives the mean of the two
//                  cells' central differences (no flux where B_f = 0),
// face gradients clipped to +-grad_t_max when it is > 0.  T and kappa of the interior and its
// one-cell ring are staged in shared memory first; other leaves read this leaf's energy only
// through their own ghost copies, so the in-place write is safe.  Boundary face fluxes go to
// the face register's energy slot as fluxes of e along +d (-F) for reflux.

// T and kappa of one cell from its state
template <typename T>
__device__ __forceinline__ void cond_tk(const T* w, const Phys<T>& P, T k0, T& tt, T& kk) {
  T p = pressure<T>(w, P);
  if (p < T(0)) p = T(0);
  tt = p / w[RHO];
  kk = k0 * (tt * tt * sqrt(tt));
}

// The energy rate of one interior cell: r its ring-region index (strides ro), sT / sK the
// ring's T and kappa, bmean(j, d, side) the face mean of B_j on face side of direction d,
// face(d, F) sees the two face fluxes of direction d (the reflux registers take them).  Both
// conduction kernels call it, so their arithmetic is the same.
template <typename T, int NDIM, typename BM, typename FF>
__device__ __forceinline__ T cond_rate(const T* sT, const T* sK, int r, const int* ro, const BlockGeo& gg,
                                       T gmax, int mode, BM bmean, FF face) {
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    T F[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int rl = side ? r : r - ro[d], rr = rl + ro[d];
      T gn = (sT[rr] - sT[rl]) / (T)gg.dx[d];
      if (gmax > T(0)) gn = fmax(-gmax, fmin(gmax, gn));
      const T kf = sqrt(sK[rl] * sK[rr]);
      if (mode == 1) {
        F[side] = kf * gn;
      } else {
        T bf[3], b2 = T(0);
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) {
          bf[j2] = bmean(j2, d, side);
          b2 += bf[j2] * bf[j2];
        }
        if (!(b2 > T(0))) {
          F[side] = T(0);
        } else {
          T bg = bf[d] * gn;
#pragma unroll
          for (int t = 0; t < NDIM; ++t) {
            if (t == d) continue;
            const T dxt = (T)gg.dx[t];
            T gt = T(0.5) * ((sT[rl + ro[t]] - sT[rl - ro[t]]) / (T(2) * dxt) +
                             (sT[rr + ro[t]] - sT[rr - ro[t]]) / (T(2) * dxt));
            if (gmax > T(0)) gt = fmax(-gmax, fmin(gmax, gt));
            bg += bf[t] * gt;
          }
          F[side] = kf * bf[d] * bg / b2;
        }
      }
    }
    face(d, F);
    acc += (F[1] - F[0]) / (T)gg.dx[d];
  }
  return acc;
}

template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(256) conduction_kernel(CondLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int R = NB + 2;
  constexpr int NR = NDIM == 3 ? R * R * R : R * R;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  constexpr size_t NB2 = (size_t)NB * NB;
  extern __shared__ __align__(16) unsigned char csm[];
  T* sT = reinterpret_cast<T*>(csm);
  T* sK = sT + NR;
  const int blk = L.blocks[blockIdx.x];
  const BlockGeo gg = L.geo[blk];
  if (L.it >= L.nsub[gg.problem]) return;
  const T h = (T)L.hsub[gg.problem];
  T* ub = (T*)L.u + (size_t)blk * NV * S;
  Phys<T> P;
  P.gamma = (T)L.gamma;
  P.gm1 = (T)(L.gamma - 1.0);
  P.ch = T(0);
  P.tau = (T)L.tau;
  const T k0 = (T)L.kappa0, gmax = (T)L.grad_t_max;
  // region cell r = (ri, rj, rk) is padded cell (ri+1, rj+1, rk+1)
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    const int ri = r % R, rj = (r / R) % R, rk = NDIM == 3 ? r / (R * R) : 0;
    const int c = ((NDIM == 3 ? rk + 1 : 0) * NP + rj + 1) * NP + ri + 1;
    T w[NV];
    load_global<T>(ub, S, c, w);
    cond_tk<T>(w, P, k0, sT[r], sK[r]);
  }
  __syncthreads();
  const int slot = L.freg ? L.refl[blk].slot : -1;
  T* R0 = slot >= 0 ? (T*)L.freg + (size_t)slot * (2 * NDIM * NV * NB2) : nullptr;
  const int ro[3] = {1, R, R * R};
  const int po[3] = {1, NP, NP * NP};
  for (int q = threadIdx.x; q < NI; q += blockDim.x) {
    const int i = q % NB, j = (q / NB) % NB, k = NDIM == 3 ? q / (NB * NB) : 0;
    const int r = ((NDIM == 3 ? k + 1 : 0) * R + j + 1) * R + i + 1;
    const int c = ((NDIM == 3 ? k + NG : 0) * NP + j + NG) * NP + i + NG;
    const int ic[3] = {i, j, k};
    auto bmean = [&](int j2, int d, int side) -> T {
      const int cl = side ? c : c - po[d], cr = cl + po[d];
      return T(0.5) * (ub[(size_t)(BX + j2) * S + cl] + ub[(size_t)(BX + j2) * S + cr]);
    };
    auto face = [&](int d, const T* F) {
      if (R0) {
        const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
        const int t0 = ic[da], t1 = NDIM == 3 ? ic[db] : 0;
        if (ic[d] == 0) R0[(size_t)(2 * d) * NV * NB2 + (size_t)EN * NB2 + t1 * NB + t0] = -F[0];
        if (ic[d] == NB - 1) R0[(size_t)(2 * d + 1) * NV * NB2 + (size_t)EN * NB2 + t1 * NB + t0] = -F[1];
      }
    };
    const T acc = cond_rate<T, NDIM>(sT, sK, r, ro, gg, gmax, L.mode, bmean, face);
    ub[(size_t)EN * S + c] = ub[(size_t)EN * S + c] + h * acc;
  }
}

// Grid-wide barrier number k of a cooperative launch (the barrier words zeroed before it):
// thread 0 of each CTA arrives on bar[0]; the last arrival resets it and opens the barrier by
// storing k + 1 in bar[1]; the others wait for that value, giving up after ~2^31 clock cycles
// (about a second).  Returns false when this CTA gave up (give_up: the test hook, at once).
// Ordering: the CTA barrier orders the CTA's stores before thread 0's device-scope fence and
// release (cumulative), and thread 0's acquire before the CTA's later loads; only thread 0
// fences.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned* bar, unsigned nblocks, unsigned k, int give_up) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int ok = 1;
    if (give_up) {
      ok = 0;
    } else {
      const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
      if (arrived == nblocks) {
        atomicExch(&bar[0], 0u);
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(k + 1u) : "memory");
      } else {
        const long long t0 = clock64();
        for (;;) {
          unsigned g;
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
          if (g == k + 1u) break;
          if (clock64() - t0 > (1ll << 31)) { ok = 0; break; }
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The substep loop of cond_loop (CondLoopLaunch), one leaf per CTA of a cooperative launch.
// The leaf's ring region (interior and one ghost layer) of every variable but psi stays in
// shared memory over the loop.  Per substep: T and kappa on the ring, the interior energy
// update (cond_rate, as conduction_kernel), the new interior energy into e_pp[it & 1], the
// grid barrier, then the ring's ghost energy from the leaves it copies (all regions are
// copies here, whose first ghost layer reads interior cells).  Leaves of problems with fewer
// substeps take part in the barriers only.  After the loop the interior energy goes back to u;
// its ghosts are stale, as after the per-substep path.  512 threads: a 16^2 leaf's ring region
// (324 cells) and interior take one pass each (256 threads: 7.0 us per substep, 512: 6.6).
template <typename T, int NDIM, int NB>
__global__ void __launch_bounds__(512) cond_loop_kernel(CondLoopLaunch L) {
  using G = Geo<NDIM, NB>;
  constexpr int NP = G::NP, S = G::S;
  constexpr int R = NB + 2;
  constexpr int NR = NDIM == 3 ? R * R * R : R * R;
  constexpr int NI = NDIM == 3 ? NB * NB * NB : NB * NB;
  constexpr int NW = NV - 1;                        // rho, m, B, e (psi enters no T)
  extern __shared__ __align__(16) unsigned char csm[];
  T* sW = reinterpret_cast<T*>(csm);                // [NW][NR]
  T* sT = sW + (size_t)NW * NR;
  T* sK = sT + NR;
  __shared__ GhostRegion reg[27];
  const int blk = L.blocks[blockIdx.x];
  const BlockGeo gg = L.geo[blk];
  for (int q = threadIdx.x; q < 27; q += blockDim.x) reg[q] = L.regions[(size_t)blk * 27 + q];
  const int ns = L.nsub[gg.problem];
  const T h = (T)L.hsub[gg.problem];
  T* ub = (T*)L.u + (size_t)blk * NV * S;
  Phys<T> P;
  P.gamma = (T)L.gamma;
  P.gm1 = (T)(L.gamma - 1.0);
  P.ch = T(0);
  P.tau = (T)L.tau;
  const T k0 = (T)L.kappa0, gmax = (T)L.grad_t_max;
  auto padded = [&](int r) {                        // ring cell -> padded cell
    const int ri = r % R, rj = (r / R) % R, rk = NDIM == 3 ? r / (R * R) : 0;
    return ((NDIM == 3 ? rk + 1 : 0) * NP + rj + 1) * NP + ri + 1;
  };
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    const int c = padded(r);
#pragma unroll
    for (int v = 0; v < NW; ++v) sW[(size_t)v * NR + r] = ub[(size_t)v * S + c];
  }
  const int ro[3] = {1, R, R * R};
  unsigned fail = 0;
  for (int it = 0; it < L.nmax; ++it) {
    __syncthreads();
    const bool active = it < ns;
    if (active) {
      for (int r = threadIdx.x; r < NR; r += blockDim.x) {
        T w[NV];
#pragma unroll
        for (int v = 0; v < NW; ++v) w[v] = sW[(size_t)v * NR + r];
        w[PSI] = T(0);
        cond_tk<T>(w, P, k0, sT[r], sK[r]);
      }
      __syncthreads();
      T* eb = (T*)L.e_pp[it & 1] + (size_t)blk * NV * S + (size_t)EN * S;
      for (int q = threadIdx.x; q < NI; q += blockDim.x) {
        const int i = q % NB, j = (q / NB) % NB, k = NDIM == 3 ? q / (NB * NB) : 0;
        const int r = ((NDIM == 3 ? k + 1 : 0) * R + j + 1) * R + i + 1;
        auto bmean = [&](int j2, int d, int side) -> T {
          const int rl = side ? r : r - ro[d], rr = rl + ro[d];
          return T(0.5) * (sW[(size_t)(BX + j2) * NR + rl] + sW[(size_t)(BX + j2) * NR + rr]);
        };
        auto face = [](int, const T*) {};
        const T acc = cond_rate<T, NDIM>(sT, sK, r, ro, gg, gmax, L.mode, bmean, face);
        // only this thread reads or writes cell r's energy in this phase (the rates read T,
        // kappa and B)
        const T en = sW[(size_t)EN * NR + r] + h * acc;
        sW[(size_t)EN * NR + r] = en;
        eb[padded(r)] = en;
      }
    }
    if (!grid_barrier_bounded(L.bar, (unsigned)L.nblocks, (unsigned)it, L.fail_waits)) {
      fail = 4u;
      break;
    }
    if (active && it + 1 < ns) {
      // the ring's ghost energy: region (rx, ry, rz) maps padded index i to m i + a of its
      // source leaf, an interior cell of that leaf for the first ghost layer
      const T* ebase = (const T*)L.e_pp[it & 1];
      for (int r = threadIdx.x; r < NR; r += blockDim.x) {
        const int ri = r % R, rj = (r / R) % R, rk = NDIM == 3 ? r / (R * R) : 1;
        const int rx = ri == 0 ? 0 : (ri == R - 1 ? 2 : 1), ry = rj == 0 ? 0 : (rj == R - 1 ? 2 : 1);
        const int rz = NDIM == 3 ? (rk == 0 ? 0 : (rk == R - 1 ? 2 : 1)) : 1;
        if (rx == 1 && ry == 1 && rz == 1) continue;
        const GhostRegion& g = reg[rx + 3 * ry + 9 * rz];
        const int si = g.m[0] * (ri + 1) + g.a[0], sj = g.m[1] * (rj + 1) + g.a[1];
        const int sk = NDIM == 3 ? g.m[2] * (rk + 1) + g.a[2] : 0;
        const size_t sc = (size_t)g.src * NV * S + (size_t)EN * S + ((size_t)sk * NP + sj) * NP + si;
        sW[(size_t)EN * NR + r] = __ldcg(ebase + sc);
      }
    }
  }
  __syncthreads();
  if (fail) {
    if (threadIdx.x == 0) atomicOr(L.err_word, fail);
    return;
  }
  if (ns > 0)
    for (int q = threadIdx.x; q < NI; q += blockDim.x) {
      const int i = q % NB, j = (q / NB) % NB, k = NDIM == 3 ? q / (NB * NB) : 0;
      const int r = ((NDIM == 3 ? k + 1 : 0) * R + j + 1) * R + i + 1;
      ub[(size_t)EN * S + padded(r)] = sW[(size_t)EN * NR + r];
    }
}

}  // namespace mapgb
