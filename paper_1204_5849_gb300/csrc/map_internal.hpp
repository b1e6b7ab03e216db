// map_internal.hpp -- internal types shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/map.h"

namespace mapgb {

constexpr int kNV = 9;
constexpr int kNG = 2;
constexpr int kEN = 7;      // index of the energy density among the 9 variables

// Per pool block: geometry of one block (leaf or parent).
struct BlockGeo {
  double dx[3];
  int problem;
  int level;
  int leaf;        // caller leaf index or -1 for a parent
  int pad;
};

// Per problem, device-resident step constants (written by the CFL reduction).
struct ProbDyn {
  double dt, ch, cp, damp, alpha_g, mindx;
  unsigned long long alpha_bits;   // running max of alpha (as ordered bits, alpha >= 0)
  unsigned long long kmax_bits;    // running max of kappa / rho (thermal conduction), as bits
  double dtc;                      // thermal-conduction time step (Sec. 3.6), +inf if none
  double dx0[3];                   // the problem's level-0 cell spacing (host, per tree)
  double lam0[3];                  // dt / dx0 (finalisation); dt/dx at level L = 2^L dt/dx0
};

// One ghost region of a leaf (3^ndim regions, region id = rx + 3 ry + 9 rz with
// r = 0 low ghosts, 1 interior range, 2 high ghosts).  Per dimension the source index is
// m*i + a (i = padded index in the destination block).
//   kind 0 COPY:    src block interior/any cell at padded index (m*i + a)
//   kind 1 PROLONG: fine global cell g = m*i + a; coarse padded = (g >> 1) - corg + NG,
//                   offset sign from g & 1 (minmod-linear, Sec. 4.3)
struct GhostRegion {
  int kind;
  int src;
  int m[3];
  int a[3];
  int corg[3];
  int pushed;      // 1: a same-level leaf copy that the source's step kernel writes itself
};

// Per leaf and direction (dx+1) + 3(dy+1) + 9(dz+1): the same-level neighbour whose ghost
// region facing this block copies from it, and the index shift from this block's padded
// cell to that ghost cell (dst = -1: none).  The source cells are the two interior layers
// next to the shared face, edge or corner.
struct PushEntry {
  int dst;
  int off[3];
};

// Reflux (Sec. 4.2, boundary step (2)).  Leaves on either side of a coarse/fine face own a
// face register: the flux through each of their boundary face cells over the step, laid
// out [side 2d+s][var][t1][t0] (nb*nb per side and variable; t0, t1 the face cell's
// interior coordinates in the other two dimensions, increasing order).
struct RefluxLeaf {
  int slot;          // face-register slot, -1: none
  int coarse_mask;   // bit 2d+s: this leaf is the coarse side of a coarse/fine face there
};

// One coarse leaf with at least one coarse/fine face: the register slots of the fine leaves
// covering each such face, indexed by their tangential child bits (t0 half + 2 * t1 half).
struct RefluxTask {
  int coarse;        // pool id
  int cslot;         // its register slot
  int fslot[6][4];   // per side 2d+s; fslot[side][0] < 0: not a coarse/fine face
};

// Regrid task for one new leaf (Sec. 4.3 interpolation on the interior).
//   kind 0 copy interior of old block src
//   kind 1 prolong from old leaf src; child bits in cb (x | y<<1 | z<<2)
struct RegridTask {
  int kind;
  int src;
  int dst;
  int cb;
};

// Host-side tree built from the caller's leaves.
struct HostTree {
  int ndim = 0, nb = 0;
  int nblocks = 0, nleaves = 0, maxlev = 0;
  std::vector<int> leaf_to_block;           // caller leaf index -> pool block id
  std::vector<BlockGeo> geo;                // per pool block
  std::vector<int> blk_problem, blk_level, blk_ijk;  // ijk: 3 per block
  std::vector<int> children;                // 8 per block (-1 if leaf)
  std::vector<GhostRegion> regions;         // 27 per block (valid for leaves)
  std::vector<PushEntry> pushes;            // 27 per block (valid for leaves)
  std::vector<char> level_has_residual;     // per level: a ghost region the fill must do
  std::vector<RefluxLeaf> refl;             // per block
  std::vector<RefluxTask> reflux_tasks;     // per coarse leaf at a coarse/fine face
  int nslots = 0;                           // face-register slots
  std::vector<std::vector<int>> leaves_by_level;   // pool ids
  std::vector<std::vector<int>> parents_by_level;  // pool ids
  std::vector<std::vector<int>> residual_by_level; // leaves with a ghost region no step pushes
  std::vector<int> all_leaves;              // pool ids, Morton order
  std::vector<double> mindx;                // per problem
  std::vector<int> leaves_per_problem;
  // lookup (problem, level, i, j, k) -> pool id
  int find(int p, int L, int i, int j, int k) const;
  std::vector<std::pair<unsigned long long, int>> keys;  // sorted packed keys -> id
  // open-addressing hash index over the same keys (linear probing, power-of-two table)
  std::vector<unsigned long long> hkeys;
  std::vector<int> hvals;
  unsigned long long hmask = 0;
  void build_index();
  // empty the tree but keep the vectors' storage for the next build_tree into it
  void reset();
};

// The checks of map_params that need no pool (capi.cpp): nullptr when p is acceptable,
// else the reason.
const char* params_problem(const map_params* p);

// Build the tree; returns an empty string on success, else the reason.
std::string build_tree(int ndim, int nb, const std::vector<map_problem_desc>& probs,
                       const map_block_desc* leaves, int n, HostTree& t);

// Regrid decision from per-leaf flags (+1 refine, 0 keep, -1 may coarsen); the new leaf
// list in the documented order.  Empty string on success.
std::string plan_regrid(const HostTree& t, const std::vector<map_problem_desc>& probs, const int8_t* flags,
                        int max_level, std::vector<map_block_desc>& out);

// Partition of the leaves over nranks (Morton ranges of equal count, Sec. 4.2) and, per
// rank, the leaves whose interiors its ghost fill reads (own ones included):
// owner[caller leaf] = rank, need[r * n + caller leaf] = 1 where rank r needs that leaf.
void plan_partition(const HostTree& t, int nranks, std::vector<int>& owner, std::vector<unsigned char>& need);

// Regrid tasks from an old tree to a new one; empty string on success.
std::string build_regrid(const HostTree& old_t, const HostTree& new_t,
                         std::vector<RegridTask>& tasks);

// ---------------------------------------------------------------------------------------
// Kernel launchers (kernels_f64.cu / kernels_f32.cu).

// Default warp-schedule weights (predictor unit : face unit) of the step kernel's per-plane
// work list, from step times measured on GB300 over the weight ratio (map_autotune searches
// around them): 3:1 for 3D LF on 16^3 blocks, 4:1 on 8^3 (the resistive Harris-sheet octree:
// 2.5 % on its step launches), 3:2 for 3D MMC, 7:4 for 2D LF and MMC (the predictor and the
// faces run in separate barrier intervals there), 1:1 for WENO, whose only predictor work is
// the resistive current.
inline void default_schedule_weights(int ndim, int nb, int scheme, int* w_pred, int* w_face) {
  *w_pred = 1;
  *w_face = 1;
  if (scheme == MAP_WENO) return;
  if (ndim == 2) {
    *w_pred = 7;
    *w_face = 4;
  } else if (scheme == MAP_LF) {
    *w_pred = nb == 8 ? 4 : 3;
    *w_face = 1;
  } else {
    *w_pred = 3;
    *w_face = 2;
  }
}

struct StepLaunch {
  const void* u_in;        // state with ghosts
  void* u_out;             // output state (interior written)
  const void* u_base;      // WENO stage 2: u^n (interior read)
  const int* blocks;       // pool ids to update
  int nblocks;
  const BlockGeo* geo;
  const ProbDyn* dyn;
  double gamma, eta, tau;
  int eglm, scheme, limiter, stage;   // stage: 0 single (MMC/LF), 1 WENO stage 1, 2 WENO stage 2
  unsigned* err_word;
  double* sums;            // optional FP64 conservation sums [nprob][9] of the output
  ProbDyn* dyn_next;       // optional: max alpha of the output into dyn_next[p].alpha_bits
  int grid;                // CTAs (0 = one per block)
  int riemann;             // interface flux of LF and WENO: 0 f_m, 1 HLLC, 2 HLLD
  int w_pred = 0, w_face = 0;  // warp-schedule weights (0: default_schedule_weights)
  int fail_waits = 0;          // test hook (map_test_fail_waits)
  const PushEntry* pushes; // optional: write boundary layers into same-level neighbours' ghosts
  void* freg;              // optional: face registers (reflux); with refl
  const RefluxLeaf* refl;  // per block slot and coarse-side mask
};

struct RefluxLaunch {
  void* u;                 // output state of the step (corrected in place)
  const RefluxTask* tasks;
  int ntasks;
  const void* freg;
  const BlockGeo* geo;
  const ProbDyn* dyn;      // dt, damping
  const PushEntry* pushes; // re-push corrected cells to same-level neighbours' ghosts
  double gamma, tau;
  unsigned* err_word;
  double* sums;            // optional: FP64 sums of the corrected cells (fused form)
  ProbDyn* dyn_next;       // optional: alpha max of the corrected cells (fused form)
  int v0 = 0, v1 = kNV;    // variables corrected: [v0, v1)
  const double* hsub = nullptr;  // conduction substeps: lam = hsub[p] / dx (else dyn dt)
  const int* nsub = nullptr;     // with hsub: problems with it >= nsub[p] are skipped
  int it = 0;
};

// Thermal conduction (Sec. 3.6): one substep of the energy update over hsub[p] on every
// leaf of a problem with it < nsub[p], in place (ghosts filled).
struct CondLaunch {
  void* u;
  const int* blocks;       // leaves
  int nblocks;
  const BlockGeo* geo;
  double gamma, tau, kappa0, grad_t_max;
  int mode;                // 1 isotropic, 2 along B
  const double* hsub;
  const int* nsub;
  int it;
  void* freg;              // optional face registers (energy slot, as a flux of e along +d)
  const RefluxLeaf* refl;
};

// The whole conduction substep loop of one step in one cooperative launch (single-level
// meshes whose ghost regions are all copies): each CTA keeps its leaf's ring region in
// shared memory and exchanges the energy of its interior through e_pp[it & 1] (the energy
// slices of two spare state buffers), one bounded grid barrier per substep.
struct CondLoopLaunch {
  void* u;                 // the state: the ring region is read, the interior energy written
  void* e_pp[2];           // two state buffers whose energy slices carry the exchange
  const int* blocks;       // leaves, one CTA each
  int nblocks;
  const BlockGeo* geo;
  const GhostRegion* regions;
  double gamma, tau, kappa0, grad_t_max;
  int mode;                // 1 isotropic, 2 along B
  const double* hsub;
  const int* nsub;
  int nmax;                // substeps of the problem with the most
  unsigned* bar;           // grid barrier words (zeroed before the launch)
  unsigned* err_word;
  int fail_waits;          // test hook: the barrier gives up at once
};

struct FillLaunch {
  void* u;
  const int* blocks;
  int nblocks;
  const GhostRegion* regions;
  int skip_pushed;         // 1: leave regions the previous step kernel wrote
  int v0 = 0, v1 = kNV;    // variables filled: [v0, v1)
};

struct RestrictLaunch {
  void* u;
  const int* parents;
  int nparents;
  const int* children;     // 8 per pool block
};

struct CflLaunch {
  const void* u;
  const int* blocks;
  int nblocks;
  const BlockGeo* geo;
  ProbDyn* dyn;
  double gamma;
  double kappa0 = 0.0;     // > 0: also reduce max kappa / rho into dyn.kmax_bits
};

struct FinalizeLaunch {
  ProbDyn* dyn;
  int nprob;
  int ndim;
  double c_cfl, eta, ch_fixed, cp_fixed, c_d, dt_override;
  int ch_mode, cp_mode;
  int conduction = 0, subcycle = 1;   // conduction on: dt_c; without the subcycle dt <= dt_c
};

struct FlagLaunch {
  const void* u;
  const int* blocks;       // leaves in caller order
  int nblocks;
  const BlockGeo* geo;
  double gamma;
  double tau = 0.0;          // FP32 pools: threshold of the pressure recovery's FP64 fallback
  map_refine_params r;
  int8_t* flags;
  double* est;
  double level_factor[16];   // R^(xi (L+1-1)) for levels L = 0..15, computed on the host
};

struct SumLaunch {
  const void* u;
  const int* blocks;
  int nblocks;
  const BlockGeo* geo;
  double* sums;            // [nprob][9], accumulated
};

struct PackLaunch {
  void* u;                 // pool
  double* host_layout;     // staging [n][9][nz][nb][nb]
  const int* blocks;       // pool ids in caller leaf order
  int nblocks;
  int to_pool;             // 1: staging -> pool, 0: pool -> staging
  int staging_f32 = 0;     // 1: the staging holds floats (FP32 host layout)
};

struct RegridLaunch {
  const void* u_old;
  void* u_new;
  const RegridTask* tasks;
  int ntasks;
};

struct KernelConfig {
  int ndim, nb;
};

// Returns cudaSuccess or the launch error; each adds the number of kernels launched.
#define MAPGB_DECLARE_LAUNCHERS(SUFFIX)                                                  \
  cudaError_t launch_step_##SUFFIX(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_fill_##SUFFIX(const KernelConfig&, const FillLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_restrict_##SUFFIX(const KernelConfig&, const RestrictLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_cfl_##SUFFIX(const KernelConfig&, const CflLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_flags_##SUFFIX(const KernelConfig&, const FlagLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_sums_##SUFFIX(const KernelConfig&, const SumLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_pack_##SUFFIX(const KernelConfig&, const PackLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_regrid_##SUFFIX(const KernelConfig&, const RegridLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_reflux_##SUFFIX(const KernelConfig&, const RefluxLaunch&, cudaStream_t, long long*); \
  cudaError_t launch_conduction_##SUFFIX(const KernelConfig&, const CondLaunch&, cudaStream_t, long long*); \
  int cond_loop_capacity_##SUFFIX(const KernelConfig&, int nsm); \
  cudaError_t launch_cond_loop_##SUFFIX(const KernelConfig&, const CondLoopLaunch&, cudaStream_t, long long*); \
  size_t step_smem_##SUFFIX(const KernelConfig&, int scheme, int resistive); \
  cudaError_t launch_cfl_partial_##SUFFIX(const KernelConfig&, const void* u, int nblocks, double gamma, \
                                          double* partial, cudaStream_t);

MAPGB_DECLARE_LAUNCHERS(f64)
MAPGB_DECLARE_LAUNCHERS(f32)
// step-kernel variants in their own translation units: HLLC flux, reflux bookkeeping, both
cudaError_t launch_step_hllc_f64(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hllc_f32(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_rfx_f64(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_rfx_f32(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hllc_rfx_f64(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hllc_rfx_f32(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hlld_f64(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hlld_f32(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hlld_rfx_f64(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);
cudaError_t launch_step_hlld_rfx_f32(const KernelConfig&, const StepLaunch&, cudaStream_t, long long*);

cudaError_t launch_finalize(const FinalizeLaunch&, cudaStream_t, long long*);
cudaError_t launch_zero_alpha(ProbDyn* dyn, int nprob, cudaStream_t, long long*);
// out: device address of host memory (n x 5 doubles) that the GPU can store to
cudaError_t launch_speeds_out(const ProbDyn* dyn, int nprob, double* out, cudaStream_t, long long*);

}  // namespace mapgb
