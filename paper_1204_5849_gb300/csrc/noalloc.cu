// noalloc.cu -- an allocation-free variant of the CFL reduction.
//
// Some callers cannot allocate device memory: embedders whose memory is owned by another
// allocator (a framework's caching allocator or a fixed arena) and who forbid
// cudaMalloc/cudaFree, and real-time loops that must not synchronise the device the way
// cudaMalloc/cudaFree may.  map_cfl_dt_noalloc serves them: the caller passes the state
// (already in device memory) and receives dt; the kernel's scratch (one partial maximum
// per block) lives in a file-scope static device array of fixed size, so no call
// allocates.  The array is resident on every GPU that loads the library until the process
// exits, and all calls share it.  The call is blocking: it copies the five results to the
// caller's host memory and synchronises its stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <atomic>

#include "map_internal.hpp"
#include "physics.cuh"

namespace mapgb {
void set_global_error(const char* msg);
}

using namespace mapgb;

// Scratch: partial maxima of alpha, one per block, then the result record.
static constexpr int kNoAllocMaxBlocks = MAP_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 8];

// Device address of g_noalloc_scratch per device, looked up once per device with that
// device current (host code may not use the symbol itself as an address).  Atomic because
// host threads may make their first calls concurrently; each stores the same address.  A
// device reset invalidates the kept address (documented at the declaration).
static std::atomic<double*> g_scratch_addr[64];

// Reduces the partial maxima and computes dt, c_h, c_p and the damping factor exactly as
// the pool's finalisation does; result[0..4] = dt, c_h, c_p, damping, alpha_g.
__global__ void __launch_bounds__(256) cfl_final_kernel(const double* __restrict__ partial, int nblocks,
                                                        FinalizeLaunch L, double mindx, double* __restrict__ result) {
  __shared__ double red[32];
  double am = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double t = partial[b];
    am = (t != t || am != am) ? (am != am ? am : t) : fmax(am, t);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, am, o);
    am = (t != t || am != am) ? (am != am ? am : t) : fmax(am, t);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = am;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double ag = 0.0;
  for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q)
    ag = (red[q] != red[q] || ag != ag) ? (ag != ag ? ag : red[q]) : fmax(ag, red[q]);
  double sig = ag;
  if (L.ch_mode == MAP_CH_FIXED && L.ch_fixed > sig) sig = L.ch_fixed;
  double dt = L.c_cfl * mindx / ((double)L.ndim * sig);
  if (L.eta > 0.0) {
    const double dtr = L.c_cfl * mindx * mindx / (2.0 * (double)L.ndim * L.eta);
    if (dtr < dt) dt = dtr;
  }
  if (L.dt_override > 0.0) dt = L.dt_override;
  double ch;
  if (L.ch_mode == MAP_CH_AUTO) ch = ag;
  else if (L.ch_mode == MAP_CH_PAPER) ch = L.c_cfl * mindx / dt;
  else ch = L.ch_fixed;
  const double cp = L.cp_mode == MAP_CP_FROM_CD ? sqrt(-dt * ch * ch / log(L.c_d)) : L.cp_fixed;
  const double damp = cp > 0.0 ? exp(-dt * ch * ch / (cp * cp)) : 1.0;
  result[0] = dt;
  result[1] = ch;
  result[2] = cp;
  result[3] = damp;
  result[4] = ag;
}

extern "C" int map_cfl_dt_noalloc(const void* u_dev, int precision, int ndim, int nb, int nblocks,
                                  const double* dx, const map_params* p, void* stream, double* out) {
  char msg[200];
  if (!u_dev || !dx || !p || !out) {
    set_global_error("map_cfl_dt_noalloc: null argument");
    return MAP_EINVAL;
  }
  if ((ndim != 2 && ndim != 3) || (nb != 8 && nb != 16) || (precision != MAP_FP64 && precision != MAP_FP32_FIX64)) {
    set_global_error("map_cfl_dt_noalloc: ndim must be 2 or 3, nb 8 or 16, precision MAP_FP64 or MAP_FP32_FIX64");
    return MAP_EINVAL;
  }
  if (nblocks < 1 || nblocks > kNoAllocMaxBlocks) {
    snprintf(msg, sizeof msg, "map_cfl_dt_noalloc: nblocks = %d outside 1..%d (MAP_NOALLOC_MAX_BLOCKS)", nblocks,
             kNoAllocMaxBlocks);
    set_global_error(msg);
    return MAP_EINVAL;
  }
  if (const char* why = params_problem(p)) {
    snprintf(msg, sizeof msg, "map_cfl_dt_noalloc: %s", why);
    set_global_error(msg);
    return MAP_EINVAL;
  }
  if (p->conduction != MAP_COND_OFF) {
    set_global_error("map_cfl_dt_noalloc: thermal conduction is not covered (its dt bound needs a second reduction)");
    return MAP_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_global_error("map_cfl_dt_noalloc: no usable current CUDA device");
    return MAP_ECUDA;
  }
  double* partial = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!partial) {
    // set-up, once per device, with that device current (first call on the device)
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
      snprintf(msg, sizeof msg, "map_cfl_dt_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      set_global_error(msg);
      return MAP_ECUDA;
    }
    partial = (double*)addr;
    g_scratch_addr[dev].store(partial, std::memory_order_release);
  }
  double* result = partial + kNoAllocMaxBlocks;
  cudaStream_t s = (cudaStream_t)stream;
  double mindx = dx[0];
  for (int d = 1; d < ndim; ++d) mindx = dx[d] < mindx ? dx[d] : mindx;
  // the per-block kernel is compiled with the pool kernels of the same precision, so its
  // alpha values round exactly like map_cfl_dt's
  const KernelConfig kc{ndim, nb};
  e = precision == MAP_FP64 ? launch_cfl_partial_f64(kc, u_dev, nblocks, p->gamma, partial, s)
                            : launch_cfl_partial_f32(kc, u_dev, nblocks, p->gamma, partial, s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "map_cfl_dt_noalloc: launch failed: %s", cudaGetErrorString(e));
    set_global_error(msg);
    return MAP_ECUDA;
  }
  FinalizeLaunch F{};
  F.nprob = 1;
  F.ndim = ndim;
  F.c_cfl = p->c_cfl;
  F.eta = p->eta;
  F.ch_fixed = p->ch;
  F.cp_fixed = p->cp;
  F.c_d = p->c_d;
  F.dt_override = p->dt_override;
  F.ch_mode = p->ch_mode;
  F.cp_mode = p->cp_mode;
  cfl_final_kernel<<<1, 256, 0, s>>>(partial, nblocks, F, mindx, result);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, result, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "map_cfl_dt_noalloc: %s", cudaGetErrorString(e));
    set_global_error(msg);
    return MAP_ECUDA;
  }
  if (!(isfinite(out[0]) && out[0] > 0.0)) {
    set_global_error("map_cfl_dt_noalloc: time step is not finite and positive");
    return MAP_ENONFINITE;
  }
  return MAP_OK;
}
