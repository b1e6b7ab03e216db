// common.cu -- per-problem time-step finalisation (precision independent).
#include <math.h>

#include "map_internal.hpp"

namespace mapgb {

// dt, c_h, c_p and the psi damping factor of each problem from its alpha_g (Sec. 3.7
// time step; Sec. 2 c_h and c_p; eq. MHD-5 damping exp(-dt c_h^2/c_p^2)).  Resets the
// running alpha maximum for the next reduction.
__global__ void finalize_kernel(FinalizeLaunch L) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.nprob) return;
  ProbDyn d = L.dyn[p];
  const double ag = __longlong_as_double((long long)d.alpha_bits);
  double sig = ag;
  if (L.ch_mode == MAP_CH_FIXED && L.ch_fixed > sig) sig = L.ch_fixed;
  double dt = L.c_cfl * d.mindx / ((double)L.ndim * sig);
  if (L.eta > 0.0) {
    const double dtr = L.c_cfl * d.mindx * d.mindx / (2.0 * (double)L.ndim * L.eta);
    if (dtr < dt) dt = dtr;
  }
  // thermal conduction (Sec. 3.6): dt_c = c_cfl min(dx)^2 / (n_dim max(kappa T / p)), the
  // rate read as kappa / rho; without the subcycle it bounds dt
  double dtc = __longlong_as_double(0x7ff0000000000000ll);
  const double kmax = __longlong_as_double((long long)d.kmax_bits);
  if (L.conduction && kmax > 0.0) dtc = L.c_cfl * d.mindx * d.mindx / ((double)L.ndim * kmax);
  if (L.conduction && !L.subcycle && dtc < dt) dt = dtc;
  if (L.dt_override > 0.0) dt = L.dt_override;
  double ch;
  if (L.ch_mode == MAP_CH_AUTO) ch = ag;
  else if (L.ch_mode == MAP_CH_PAPER) ch = L.c_cfl * d.mindx / dt;
  else ch = L.ch_fixed;
  const double cp = L.cp_mode == MAP_CP_FROM_CD ? sqrt(-dt * ch * ch / log(L.c_d)) : L.cp_fixed;
  const double damp = cp > 0.0 ? exp(-dt * ch * ch / (cp * cp)) : 1.0;
  d.dt = dt;
  d.ch = ch;
  d.cp = cp;
  d.damp = damp;
  d.alpha_g = ag;
  d.alpha_bits = 0ull;
  d.kmax_bits = 0ull;
  d.dtc = dtc;
  // per-dimension dt/dx at level 0; a level-L block takes 2^L of it, which is dt/dx_L
  // exactly (dx_L = dx0 / 2^L as the host computes it), so blocks divide nothing
  for (int k = 0; k < 3; ++k) d.lam0[k] = dt / d.dx0[k];
  L.dyn[p] = d;
}

__global__ void zero_alpha_kernel(ProbDyn* dyn, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) {
    dyn[p].alpha_bits = 0ull;
    dyn[p].kmax_bits = 0ull;
  }
}

// dt, c_h, c_p, damping and alpha_g of every problem, stored by the GPU itself into host
// memory it can address (page-locked and mapped): no copy engine takes part, so the store does
// not queue behind the large state copies that the copy engines may be running.
__global__ void speeds_out_kernel(const ProbDyn* __restrict__ dyn, int n, double* __restrict__ out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double* o = out + 5 * (size_t)p;
    o[0] = dyn[p].dt;
    o[1] = dyn[p].ch;
    o[2] = dyn[p].cp;
    o[3] = dyn[p].damp;
    o[4] = dyn[p].alpha_g;
  }
}

cudaError_t launch_speeds_out(const ProbDyn* dyn, int n, double* out, cudaStream_t s, long long* cnt) {
  if (cnt) ++*cnt;
  speeds_out_kernel<<<1, 128, 0, s>>>(dyn, n, out);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeLaunch& L, cudaStream_t s, long long* cnt) {
  if (cnt) ++*cnt;
  finalize_kernel<<<(L.nprob + 127) / 128, 128, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_zero_alpha(ProbDyn* dyn, int n, cudaStream_t s, long long* cnt) {
  if (cnt) ++*cnt;
  zero_alpha_kernel<<<(n + 127) / 128, 128, 0, s>>>(dyn, n);
  return cudaGetLastError();
}

}  // namespace mapgb
