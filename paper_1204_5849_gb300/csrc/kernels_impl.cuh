// kernels_impl.cuh -- launch dispatch over (ndim, block size, scheme, limiter, stage).
// Included once per precision by kernels_f64.cu and kernels_f32.cu.
#pragma once
#include "aux.cuh"
#include "step.cuh"

namespace mapgb {

template <typename T, int NDIM, int NB, int SCHEME, int LIM, int STAGE, int FLX, bool RFX>
cudaError_t launch_step_one(const StepLaunch& L, cudaStream_t s) {
  const bool res = L.eta > 0.0;
  const size_t smem = step_smem_bytes<T, NDIM, NB, SCHEME>(res);
  auto kern = step_kernel<T, NDIM, NB, SCHEME, LIM, STAGE, FLX, RFX>;
  static bool attr_done[2] = {false, false};
  if (!attr_done[res]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done[res] = true;
  }
  StepArgsT<T> A;
  A.u_in = (const T*)L.u_in;
  A.u_out = (T*)L.u_out;
  A.u_base = (const T*)L.u_base;
  A.blocks = L.blocks;
  A.nblocks = L.nblocks;
  A.geo = L.geo;
  A.dyn = L.dyn;
  A.gamma = (T)L.gamma;
  A.gm1 = (T)(L.gamma - 1.0);
  A.tau = (T)L.tau;
  A.eta = L.eta;
  A.eglm = L.eglm;
  A.resistive = res ? 1 : 0;
  A.err_word = L.err_word;
  A.sums = L.sums;
  A.dyn_next = L.dyn_next;
  A.pushes = L.pushes;
  A.freg = RFX ? (T*)L.freg : nullptr;
  A.refl = RFX ? L.refl : nullptr;
  int wp = L.w_pred, wf = L.w_face;
  if (wp <= 0 || wf <= 0) default_schedule_weights(NDIM, NB, SCHEME, &wp, &wf);
  build_schedule<NDIM, NB, step_threads<T, NDIM, NB>()>(wp, wf, SCHEME != SCH_WENO || res, A.sched);
  A.fail_waits = L.fail_waits;
  const int grid = L.grid > 0 ? (L.grid < L.nblocks ? L.grid : L.nblocks) : L.nblocks;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, step_threads<T, NDIM, NB>(), smem, s>>>(A);
  return cudaGetLastError();
}

// Each (FLX, RFX) pair is instantiated in its own translation unit (kernels_<prec>.cu,
// _hllc.cu, _hlld.cu, _rfx.cu, _hllc_rfx.cu, _hlld_rfx.cu).  FLX = FLX_HLLC and FLX_HLLD
// cover LF and WENO only (MMC has no interface Riemann problem).
template <typename T, int NDIM, int NB, int FLX, bool RFX>
cudaError_t launch_step_geo(const StepLaunch& L, cudaStream_t s) {
  const int lim = L.limiter ? 1 : 0;
  if (L.scheme == SCH_MMC) {
    if constexpr (FLX == FLX_LF)
      return lim ? launch_step_one<T, NDIM, NB, SCH_MMC, 1, 0, 0, RFX>(L, s)
                 : launch_step_one<T, NDIM, NB, SCH_MMC, 0, 0, 0, RFX>(L, s);
    else
      return cudaErrorInvalidValue;
  }
  if (L.scheme == SCH_LF)
    return lim ? launch_step_one<T, NDIM, NB, SCH_LF, 1, 0, FLX, RFX>(L, s)
               : launch_step_one<T, NDIM, NB, SCH_LF, 0, 0, FLX, RFX>(L, s);
  if (L.stage == 1) return launch_step_one<T, NDIM, NB, SCH_WENO, 0, 1, FLX, RFX>(L, s);
  return launch_step_one<T, NDIM, NB, SCH_WENO, 0, 2, FLX, RFX>(L, s);
}

#define MAPGB_GEO_DISPATCH_INT(KC, CALL)                          \
  do {                                                            \
    if ((KC).ndim == 2 && (KC).nb == 16) { CALL(2, 16); }         \
    if ((KC).ndim == 3 && (KC).nb == 16) { CALL(3, 16); }         \
    if ((KC).ndim == 3 && (KC).nb == 8) { CALL(3, 8); }           \
    if ((KC).ndim == 2 && (KC).nb == 8) { CALL(2, 8); }           \
    return 0;                                                     \
  } while (0)

#define MAPGB_GEO_DISPATCH(KC, CALL)                              \
  do {                                                            \
    if ((KC).ndim == 2 && (KC).nb == 16) { CALL(2, 16); }         \
    if ((KC).ndim == 3 && (KC).nb == 16) { CALL(3, 16); }         \
    if ((KC).ndim == 3 && (KC).nb == 8) { CALL(3, 8); }           \
    if ((KC).ndim == 2 && (KC).nb == 8) { CALL(2, 8); }           \
    return cudaErrorInvalidValue;                                 \
  } while (0)

inline int grid_for(int n) { return n < 1 ? 0 : n; }

template <typename T, int FLX, bool RFX>
cudaError_t launch_step_T(const KernelConfig& kc, const StepLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_STEP(ND, NBV) return launch_step_geo<T, ND, NBV, FLX, RFX>(L, s)
  MAPGB_GEO_DISPATCH(kc, CALL_STEP);
#undef CALL_STEP
}

template <typename T>
size_t step_smem_T(const KernelConfig& kc, int scheme, int res) {
#define SM(ND, NBV)                                                                        \
  return scheme == SCH_MMC ? step_smem_bytes<T, ND, NBV, SCH_MMC>(res)                     \
                           : (scheme == SCH_LF ? step_smem_bytes<T, ND, NBV, SCH_LF>(res)  \
                                               : step_smem_bytes<T, ND, NBV, SCH_WENO>(res))
  if (kc.ndim == 2 && kc.nb == 16) { SM(2, 16); }
  if (kc.ndim == 3 && kc.nb == 16) { SM(3, 16); }
  if (kc.ndim == 3 && kc.nb == 8) { SM(3, 8); }
  if (kc.ndim == 2 && kc.nb == 8) { SM(2, 8); }
#undef SM
  return 0;
}

template <typename T>
cudaError_t launch_fill_T(const KernelConfig& kc, const FillLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_FILL(ND, NBV)                                                                   \
  fill_kernel<T, ND, NBV><<<grid_for(L.nblocks), 256, 0, s>>>((T*)L.u, L.blocks, L.nblocks, L.regions, L.skip_pushed, \
                                                              L.v0, L.v1);                                \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_FILL);
#undef CALL_FILL
}

template <typename T>
cudaError_t launch_restrict_T(const KernelConfig& kc, const RestrictLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nparents <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_RES(ND, NBV)                                                                          \
  restrict_kernel<T, ND, NBV><<<grid_for(L.nparents), 256, 0, s>>>((T*)L.u, L.parents, L.nparents, L.children); \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_RES);
#undef CALL_RES
}

template <typename T>
cudaError_t launch_cfl_T(const KernelConfig& kc, const CflLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_CFL(ND, NBV)                                                                     \
  cfl_kernel<T, ND, NBV><<<grid_for(L.nblocks), 256, 0, s>>>((const T*)L.u, L.blocks, L.nblocks, L.geo, L.dyn, \
                                                             (T)L.gamma, (T)(L.gamma - 1.0), L.kappa0); \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_CFL);
#undef CALL_CFL
}

template <typename T>
cudaError_t launch_flags_T(const KernelConfig& kc, const FlagLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_FLAGS(ND, NBV)                                              \
  flags_kernel<T, ND, NBV><<<grid_for(L.nblocks), 256, 0, s>>>(L);       \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_FLAGS);
#undef CALL_FLAGS
}

template <typename T>
cudaError_t launch_sums_T(const KernelConfig& kc, const SumLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_SUMS(ND, NBV)                                             \
  sums_kernel<T, ND, NBV><<<grid_for(L.nblocks), 256, 0, s>>>(L);      \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_SUMS);
#undef CALL_SUMS
}

template <typename T>
cudaError_t launch_pack_T(const KernelConfig& kc, const PackLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_PACK(ND, NBV)                                             \
  pack_kernel<T, ND, NBV><<<grid_for(L.nblocks), 256, 0, s>>>(L);      \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_PACK);
#undef CALL_PACK
}

template <typename T>
cudaError_t launch_regrid_T(const KernelConfig& kc, const RegridLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.ntasks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_REGRID(ND, NBV)                                            \
  regrid_kernel<T, ND, NBV><<<grid_for(L.ntasks), 256, 0, s>>>(L);      \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_REGRID);
#undef CALL_REGRID
}

template <typename T>
cudaError_t launch_reflux_T(const KernelConfig& kc, const RefluxLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.ntasks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_REFLUX(ND, NBV)                                              \
  reflux_kernel<T, ND, NBV><<<L.ntasks, 256, 0, s>>>(L);                  \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_REFLUX);
#undef CALL_REFLUX
}

template <typename T, int NDIM, int NB>
cudaError_t launch_conduction_one(const CondLaunch& L, cudaStream_t s) {
  constexpr int R = NB + 2;
  constexpr size_t smem = (size_t)2 * (NDIM == 3 ? R * R * R : R * R) * sizeof(T);
  auto kern = conduction_kernel<T, NDIM, NB>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  kern<<<L.nblocks, 256, smem, s>>>(L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_conduction_T(const KernelConfig& kc, const CondLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_COND(ND, NBV) return launch_conduction_one<T, ND, NBV>(L, s)
  MAPGB_GEO_DISPATCH(kc, CALL_COND);
#undef CALL_COND
}

// the conduction loop (cond_loop_kernel): the ring region of every variable but psi, T and
// kappa in shared memory; 3D 16^3 leaves would need 233 KB and are left to the per-substep
// kernels
template <typename T, int NDIM, int NB>
constexpr size_t cond_loop_smem() {
  constexpr int R = NB + 2;
  return (size_t)(NV + 1) * (NDIM == 3 ? R * R * R : R * R) * sizeof(T);
}

template <typename T, int NDIM, int NB>
int cond_loop_capacity_one(int nsm) {
  if constexpr (NDIM == 3 && NB == 16) {
    (void)nsm;
    return 0;
  } else {
    constexpr size_t smem = cond_loop_smem<T, NDIM, NB>();
    auto kern = cond_loop_kernel<T, NDIM, NB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per_sm * nsm;
  }
}

template <typename T, int NDIM, int NB>
cudaError_t launch_cond_loop_one(const CondLoopLaunch& L, cudaStream_t s) {
  if constexpr (NDIM == 3 && NB == 16) {
    (void)L;
    (void)s;
    return cudaErrorInvalidValue;
  } else {
    CondLoopLaunch A = L;
    void* args[] = {&A};
    return cudaLaunchCooperativeKernel((const void*)cond_loop_kernel<T, NDIM, NB>, dim3(L.nblocks), dim3(512), args,
                                       cond_loop_smem<T, NDIM, NB>(), s);
  }
}

template <typename T>
int cond_loop_capacity_T(const KernelConfig& kc, int nsm) {
#define CALL_CAP(ND, NBV) return cond_loop_capacity_one<T, ND, NBV>(nsm)
  MAPGB_GEO_DISPATCH_INT(kc, CALL_CAP);
#undef CALL_CAP
}

template <typename T>
cudaError_t launch_cond_loop_T(const KernelConfig& kc, const CondLoopLaunch& L, cudaStream_t s, long long* cnt) {
  if (L.nblocks <= 0) return cudaSuccess;
  if (cnt) ++*cnt;
#define CALL_LOOP(ND, NBV) return launch_cond_loop_one<T, ND, NBV>(L, s)
  MAPGB_GEO_DISPATCH(kc, CALL_LOOP);
#undef CALL_LOOP
}

template <typename T>
cudaError_t launch_cfl_partial_T(const KernelConfig& kc, const void* u, int nblocks, double gamma, double* partial,
                                 cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
#define CALL_PART(ND, NBV)                                                                          \
  cfl_partial_kernel<T, ND, NBV><<<nblocks, 256, 0, s>>>((const T*)u, nblocks, (T)gamma, (T)(gamma - 1.0), \
                                                        partial);                                   \
  return cudaGetLastError()
  MAPGB_GEO_DISPATCH(kc, CALL_PART);
#undef CALL_PART
}

}  // namespace mapgb

#define MAPGB_DEFINE_LAUNCHERS(T, SUFFIX)                                                          \
  namespace mapgb {                                                                                \
  cudaError_t launch_step_##SUFFIX(const KernelConfig& k, const StepLaunch& l, cudaStream_t s, long long* c) { \
    const bool rfx = l.freg != nullptr;                                                          \
    if (l.riemann == 2) return rfx ? launch_step_hlld_rfx_##SUFFIX(k, l, s, c) : launch_step_hlld_##SUFFIX(k, l, s, c); \
    if (l.riemann) return rfx ? launch_step_hllc_rfx_##SUFFIX(k, l, s, c) : launch_step_hllc_##SUFFIX(k, l, s, c); \
    return rfx ? launch_step_rfx_##SUFFIX(k, l, s, c) : launch_step_T<T, FLX_LF, false>(k, l, s, c); } \
  cudaError_t launch_fill_##SUFFIX(const KernelConfig& k, const FillLaunch& l, cudaStream_t s, long long* c) { return launch_fill_T<T>(k, l, s, c); } \
  cudaError_t launch_restrict_##SUFFIX(const KernelConfig& k, const RestrictLaunch& l, cudaStream_t s, long long* c) { return launch_restrict_T<T>(k, l, s, c); } \
  cudaError_t launch_cfl_##SUFFIX(const KernelConfig& k, const CflLaunch& l, cudaStream_t s, long long* c) { return launch_cfl_T<T>(k, l, s, c); } \
  cudaError_t launch_flags_##SUFFIX(const KernelConfig& k, const FlagLaunch& l, cudaStream_t s, long long* c) { return launch_flags_T<T>(k, l, s, c); } \
  cudaError_t launch_sums_##SUFFIX(const KernelConfig& k, const SumLaunch& l, cudaStream_t s, long long* c) { return launch_sums_T<T>(k, l, s, c); } \
  cudaError_t launch_pack_##SUFFIX(const KernelConfig& k, const PackLaunch& l, cudaStream_t s, long long* c) { return launch_pack_T<T>(k, l, s, c); } \
  cudaError_t launch_regrid_##SUFFIX(const KernelConfig& k, const RegridLaunch& l, cudaStream_t s, long long* c) { return launch_regrid_T<T>(k, l, s, c); } \
  cudaError_t launch_reflux_##SUFFIX(const KernelConfig& k, const RefluxLaunch& l, cudaStream_t s, long long* c) { return launch_reflux_T<T>(k, l, s, c); } \
  cudaError_t launch_conduction_##SUFFIX(const KernelConfig& k, const CondLaunch& l, cudaStream_t s, long long* c) { return launch_conduction_T<T>(k, l, s, c); } \
  int cond_loop_capacity_##SUFFIX(const KernelConfig& k, int nsm) { return cond_loop_capacity_T<T>(k, nsm); } \
  cudaError_t launch_cond_loop_##SUFFIX(const KernelConfig& k, const CondLoopLaunch& l, cudaStream_t s, long long* c) { return launch_cond_loop_T<T>(k, l, s, c); } \
  size_t step_smem_##SUFFIX(const KernelConfig& k, int scheme, int res) { return step_smem_T<T>(k, scheme, res); } \
  cudaError_t launch_cfl_partial_##SUFFIX(const KernelConfig& k, const void* u, int n, double g, double* part, cudaStream_t s) { return launch_cfl_partial_T<T>(k, u, n, g, part, s); } \
  }

// The step kernels of one (flux, reflux) variant, for their own translation unit.
#define MAPGB_DEFINE_STEP_VARIANT(T, NAME, FLXV, RFXV)                                             \
  namespace mapgb {                                                                                \
  cudaError_t NAME(const KernelConfig& k, const StepLaunch& l, cudaStream_t s, long long* c) {     \
    return launch_step_T<T, FLXV, RFXV>(k, l, s, c); }                                             \
  }
