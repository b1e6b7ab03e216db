/*
 * map.h -- C ABI of the GB300 EGLM-MHD block-pool step.
 *
 * The library advances the EGLM-MHD equations (Jiang, Fang & Chen, arXiv:1204.5849,
 * Sec. 2, eqs. MHD-1..MHD-5) on a pool of equal-shape blocks (Sec. 4.1) on one GPU:
 * ghost fill (Sec. 4.3), the MMC / TVD-LF / WENO-RK2 update (Sec. 3.1-3.3, Sec. 3.7),
 * resistivity (Sec. 3.5), the GLM psi source and damping (Sec. 2), the global CFL
 * reduction (Sec. 3.7), the refinement estimator (Sec. 4.5) and regrid.
 *
 * Conventions
 *  - Every call returns a map_status (0 = MAP_OK, negative = error); no call aborts or
 *    throws.  map_last_error() gives a one-line description of the last failure.
 *  - A pool is not thread-safe: calls on one pool must be serialised by the caller.
 *  - Asynchronous calls are ordered on the pool's stream (map_create_pool's stream, or
 *    map_set_stream's).  Calls that hand results to the host synchronise that stream.
 *  - Host arrays are caller-owned and only read or written during the call.
 *  - Variables are always the 9 conserved quantities in this order:
 *      rho, rho*vx, rho*vy, rho*vz, Bx, By, Bz, e, psi
 *    (three vector components in 2D as well; psi is the GLM potential, Sec. 2).
 *  - Block interior data crosses the ABI as FP64 [9][nz][nb][nb] (x fastest), nz = nb in
 *    3D and 1 in 2D, whatever the pool precision.
 */
#ifndef MAP_GB300_H
#define MAP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MAP_OK = 0,
  MAP_EINVAL = -1,        /* bad argument, bad tree (unbalanced, overlapping, incomplete) */
  MAP_ENOMEM = -2,        /* device or host allocation failed / capacity exceeded */
  MAP_ECUDA = -3,         /* a CUDA runtime call failed (text in map_last_error) */
  MAP_ENONFINITE = -4,    /* device error word: a non-finite value in a leaf cell */
  MAP_ENEGPRES = -5,      /* device error word: rho <= 0 or p < 0 in a leaf cell */
  MAP_ETIMEOUT = -6,      /* device error word: a bounded device wait gave up */
  MAP_EUNSUPPORTED = -7,  /* combination not built (e.g. block size) */
  MAP_ESTATE = -8         /* call out of order (no tree, no dt yet, ...) */
} map_status;

enum { MAP_FP64 = 0, MAP_FP32_FIX64 = 1 };   /* pool precision */
enum { MAP_MMC = 0, MAP_LF = 1, MAP_WENO = 2 };
enum { MAP_MINMOD = 0, MAP_VANLEER = 1 };
/* Interface flux of LF and WENO (Sec. 3.2-3.3): the Lax-Friedrichs f_m (Equ:LFFlux), the
 * HLLC approximate Riemann solver for MHD the paper uses in 2D and 3D, or the HLLD solver
 * (Miyoshi & Kusano) it also names and compares on the Brio-Wu tube (Sec. 5). */
enum { MAP_RIEMANN_LF = 0, MAP_RIEMANN_HLLC = 1, MAP_RIEMANN_HLLD = 2 };
/* Thermal conduction (Sec. 3.6): off, isotropic, or along the field (the form of the paper's
 * conduction test, Sec. 5), kappa = kappa0 T^(5/2) with T = p / rho. */
enum { MAP_COND_OFF = 0, MAP_COND_ISOTROPIC = 1, MAP_COND_ALIGNED = 2 };
enum { MAP_BC_PERIODIC = 0, MAP_BC_OUTFLOW = 1 };
enum { MAP_CH_AUTO = 0, MAP_CH_PAPER = 1, MAP_CH_FIXED = 2 };
enum { MAP_CP_FROM_CD = 0, MAP_CP_FIXED = 1 };

/* One independent domain (problem): base tiling in blocks, physical box, boundary kind
 * of the low/high face per dimension.  At level L the domain is tiled by nbase*2^L
 * blocks per dimension. */
typedef struct {
  int nbase[3];
  double lo[3], hi[3];
  int bc[3][2];
} map_problem_desc;

typedef struct {
  int ndim;           /* 2 or 3 */
  int nb;             /* cells per block edge: 8 or 16 */
  int n_ghost;        /* must be 2 */
  int precision;      /* MAP_FP64 or MAP_FP32_FIX64 */
  int max_blocks;     /* capacity: leaves + their parents over the pool's life */
  int n_problems;
  const map_problem_desc* problems;  /* n_problems entries, copied */
  void* ext_buffer;   /* optional device buffer for the three state buffers (e.g. a torch
                         tensor's data_ptr), caller-owned, 256-byte aligned, at least
                         3 * max_blocks * 9 * (nb+4)^ndim * element size bytes; NULL =
                         the library allocates */
  size_t ext_bytes;
} map_pool_desc;

/* A leaf block: problem index, level and integer block coordinates at that level. */
typedef struct {
  int problem, level;
  int ijk[3];
} map_block_desc;

/* Method parameters (Sec. 2, Sec. 3). */
typedef struct {
  double gamma;       /* adiabatic index */
  double c_cfl;       /* CFL safety coefficient (Sec. 3.7) */
  int ch_mode;        /* MAP_CH_AUTO: c_h = alpha_g; MAP_CH_PAPER: c_h = c_cfl min dx / dt
                         (Sec. 2, c_h formula); MAP_CH_FIXED: c_h = ch */
  double ch;
  int cp_mode;        /* MAP_CP_FROM_CD: c_p = sqrt(-dt c_h^2 / ln c_d) (Sec. 2); else cp */
  double c_d, cp;
  double eta;         /* uniform resistivity (Sec. 3.5); 0 = ideal */
  int eglm;           /* 1: EGLM non-conservative sources; 0: GLM */
  int scheme;         /* MAP_MMC, MAP_LF, MAP_WENO */
  int limiter;        /* MAP_MINMOD, MAP_VANLEER */
  double dt_override; /* > 0: use this dt instead of the CFL dt */
  double fp64_fix_tau;/* FP32 pools: recompute p in FP64 where e_int < tau * e; <= 0: off
                         (every p recovered in FP32, negative ones included) */
  int reflux;         /* 1: at every coarse/fine face the coarse leaf's flux is replaced by
                         the mean of the fine fluxes covering it (Sec. 4.2, boundary step
                         (2)), so the face carries one flux on both sides; 0: off */
  int riemann;        /* MAP_RIEMANN_LF, _HLLC or _HLLD (LF and WENO; MMC takes only
                         MAP_RIEMANN_LF, else MAP_EINVAL).  HLLC and HLLD: the (B_d, psi)
                         pair keeps the exact upwind flux of its linear system, which also
                         fixes the interface normal field; the other seven components come
                         from the solver's intermediate states with Davis speed bounds (HLLD
                         adds the two Alfven waves to HLLC's contact) */
  int conduction;     /* MAP_COND_*: after each step the energy takes the conduction update
                         e += h sum_d dF_d/dx_d, F = sqrt(kappa_l kappa_r)(T_r - T_l)/dx (along
                         B: times b_d (b . grad T)/|grad_d T| with b from the face-mean B) */
  double kappa0;      /* conduction coefficient (> 0 when conduction is on) */
  int subcycle;       /* 1: n = ceil(dt/dt_c) conduction substeps of dt/n inside each step,
                         dt_c = c_cfl min(dx)^2 / (n_dim max(kappa/rho)); 0: dt <= dt_c and
                         one update.  With conduction, map_advance reads dt back every step
                         to size the loop and is not graph-replayed */
  double grad_t_max;  /* > 0: face temperature gradients clipped to +-grad_t_max (Sec. 3.6
                         threshold); 0: none */
} map_params;

/* Refinement estimator parameters (Sec. 4.5). */
typedef struct {
  int var_mask;       /* 1 rho, 2 p, 4 |J| dx / (|B| + eps_b) */
  double thr;         /* refine if the block maximum exceeds thr */
  double coarsen_thr; /* may coarsen if the block maximum is below coarsen_thr */
  double bias;        /* B = 0.6 */
  double filter;      /* F = 0.05 */
  double eps_rho, eps_p, eps_b;
  double ratio, xi;   /* R^(xi (L-1)) level factor */
  int max_level;
} map_refine_params;

typedef struct map_pool map_pool;

/* Create a pool.  stream: a cudaStream_t the library uses but does not own; NULL makes
 * the library create (and later destroy) a non-blocking stream of its own.  The pool's
 * three state buffers (two ping-pong states and a Runge-Kutta stage) hold max_blocks
 * blocks each.  *out receives the pool.  Errors: MAP_EINVAL (bad desc),
 * MAP_EUNSUPPORTED (nb/ndim not built), MAP_ENOMEM, MAP_ECUDA. */
int map_create_pool(const map_pool_desc* d, void* stream, map_pool** out);

/* Free library-owned device memory and the pool.  NULL is accepted. */
int map_destroy_pool(map_pool* pool);

/* Replace the stream used by later calls (NULL = a stream owned by the library).
 * Synchronises the old stream first. */
int map_set_stream(map_pool* pool, void* stream);

/* Set the block tree from its leaves (Sec. 4.1).  The library adds every parent, orders
 * blocks along the Morton curve, validates the tree (coordinates in range, no leaf inside
 * another, every parent complete, 2:1 balance across faces, edges and corners) and builds
 * the neighbour / ghost-fill tables on the host.  Leaf data is undefined until written.
 * Leaf index l of later calls is the position in this array.  Errors: MAP_EINVAL,
 * MAP_ENOMEM (more blocks than max_blocks). */
int map_set_tree(map_pool* pool, const map_block_desc* leaves, int n);

/* Copy one leaf's interior from / to the host (FP64 [9][nz][nb][nb]).  read synchronises. */
int map_write_block(map_pool* pool, int leaf, const double* u);
int map_read_block(map_pool* pool, int leaf, double* u_out);

/* All leaves at once, in leaf order: n_leaves x [9][nz][nb][nb] FP64 host arrays.
 * Use pinned host memory for full copy bandwidth.  read synchronises. */
int map_write_leaves(map_pool* pool, const double* u);
int map_read_leaves(map_pool* pool, double* u_out);

/* Ghost fill (Sec. 4.3), asynchronous: parents become the mean of their children
 * (bottom-up), then level by level from the coarsest: same-level copy from the
 * neighbour block holding the cell (edges and corners included), periodic wrap or
 * zero-gradient outflow at the domain boundary, conservative minmod prolongation from
 * the coarser leaf where the neighbour level does not exist. */
int map_fill_ghosts(map_pool* pool);

/* Global CFL reduction (Sec. 3.7): alpha_g per problem (max over leaf cells and
 * directions of |v_d| + c_f,d), dt = c_cfl min dx / (ndim alpha_g) (and the diffusive
 * limit c_cfl dx^2 / (2 ndim eta) when eta > 0), c_h, c_p, and the psi damping factor,
 * all kept on the device.  Copies dt to dt_out[n_problems] and synchronises.  Errors:
 * MAP_ENONFINITE if a dt is not finite and positive. */
int map_cfl_dt(map_pool* pool, const map_params* p, double* dt_out);

/* One step (asynchronous, no host synchronisation, no allocation): the scheme update
 * of every leaf with the device-resident dt of the last map_cfl_dt (or
 * p->dt_override), sources, psi damping; WENO refills ghosts between its stages.  Ghosts
 * must be filled before the call. */
int map_step(map_pool* pool, const map_params* p);

/* nsteps x (ghost fill, dt on the device, step), asynchronous: the batched form.  The
 * step kernel also reduces alpha_g of the new state (the next dt) and the FP64
 * conservation sums of the new state, so a separate CFL pass runs only before the first
 * step after the state changed outside this call.  The step sequence is captured once per
 * starting buffer into a CUDA graph and replayed.  map_get_speeds reads the last dt. */
int map_advance(map_pool* pool, const map_params* p, int nsteps);

/* Device error word accumulated by the steps since the last check (rho <= 0, p < 0,
 * non-finite, a bounded wait for a plane copy that gave up), read and cleared;
 * synchronises the pool stream and the pool's copy streams (so the asynchronous host
 * copies are complete on return).  MAP_OK, MAP_ETIMEOUT, MAP_ENONFINITE or MAP_ENEGPRES. */
int map_check(map_pool* pool);

/* Refinement flags (Sec. 4.5): per leaf +1 refine, 0 keep, -1 may coarsen, from the
 * block maximum of the estimator over the interior and the first ghost ring.  Ghosts
 * must be filled.  flags_out[n_leaves]; est_out[n_leaves] may be NULL.  Synchronises. */
int map_flag_refine(map_pool* pool, const map_params* p, const map_refine_params* r,
                    int8_t* flags_out, double* est_out);

/* Replace the tree by a new leaf set (each new leaf: unchanged, a child of an old leaf,
 * or a parent of old leaves).  Kept leaves copy, new children are prolonged from their
 * old parent (Sec. 4.3 formula on the interior), new parents take the restriction of
 * their old children.  Ghosts of the old tree must be filled.  Leaf indices follow the
 * new array.  Errors: MAP_EINVAL. */
int map_regrid(map_pool* pool, const map_block_desc* new_leaves, int n);

/* Regrid decision on the host (Sec. 4.5 "refine if the error exceeds the threshold"):
 * from per-leaf flags (+1 refine, 0 keep, -1 may coarsen, in leaf order) build the new leaf
 * list: refine leaves flagged +1 below max_level; refine further leaves until every new
 * leaf's face, edge and corner neighbours are at most one level coarser (2:1); coarsen a
 * parent whose 2^ndim children are all leaves flagged -1 and none refined, when the
 * coarsened parent keeps 2:1.  Order: old leaf order, a kept leaf in place, a refined leaf
 * as its children (child bits x | y<<1 | z<<2 ascending), a coarsened parent at the place
 * of its first child.  out[cap] receives the list, *n_out its length (also when cap is too
 * small: MAP_ENOMEM).  No device work. */
int map_plan_regrid(map_pool* pool, const int8_t* flags, int max_level, map_block_desc* out,
                    int cap, int* n_out);

/* One adaptation cycle: ghost fill, refinement flags, map_plan_regrid with r->max_level,
 * and map_regrid when the leaf set changes.  *n_out = number of leaves afterwards (read
 * them with map_get_leaves).  Synchronises. */
int map_adapt(map_pool* pool, const map_params* p, const map_refine_params* r, int* n_out);

/* The current leaf list (leaf order of the last map_set_tree / map_regrid / map_adapt). */
int map_get_leaves(map_pool* pool, map_block_desc* out, int cap, int* n_out);

/* FP64 conservation sums: sums_out[n_problems][9] = sum over leaf cells of U * cell
 * volume.  Synchronises. */
int map_conservation(map_pool* pool, double* sums_out);

/* (No counterpart in the paper.)  The FP64 conservation sums (same layout as
 * map_conservation) that the last map_advance step reduced inside its kernels for the state it produced, without another pass over
 * the pool.  MAP_ESTATE when the state changed otherwise since (a write, map_step, a
 * regrid).  Synchronises. */
int map_last_sums(map_pool* pool, double* sums_out);

/* Launch shape chosen by map_autotune. */
typedef struct {
  int grid;           /* step-kernel CTAs: 0 = the default (one per block in 3D; for FP32
                         pools in 2D a persistent grid of four per SM), a value >= the
                         block count = one per block, else a persistent grid */
  int w_pred, w_face; /* warp-schedule cost of a predictor unit and of a face unit */
  double ms_default;  /* step launches with the default shape (grid 0, default
                         weights: 3:1 for 3D LF on 16^3, 4:1 on 8^3, 3:2 for 3D MMC, 7:4 in
                         2D, 1:1 for WENO) */
  double ms_best;     /* with the chosen shape */
  int trials;
} map_tune_result;

/* Autotuner (no counterpart in the paper): times this pool's step launches on its current
 * tree and state under candidate launch shapes -- the default, one CTA per block, or a
 * persistent grid of 1-16 x the SM count, then warp-schedule weight ratios from 1:1 to 6:1 for the per-plane
 * work list -- and keeps the
 * fastest for later map_step / map_advance calls (results are bitwise the same under every
 * shape; the fused FP64 sums may differ in rounding).  The state is not changed: trials
 * write only the other buffers, and the step constants and sums are restored.  Ghosts are
 * refilled first.  reps: timed repetitions per candidate (>= 1).  Synchronises. */
int map_autotune(map_pool* pool, const map_params* p, int reps, map_tune_result* out);

/* (No counterpart in the paper.)  Test hook for the bounded-wait path: with on = 1 every
 * wait of the step kernel for a plane copy gives up at once, as a wait that ran out of its
 * bound (about a second) would: the kernel records the timeout, still waits (bounded) for
 * the copies in flight so none lands after the block has left, and leaves; map_check then
 * returns MAP_ETIMEOUT.  The step's output is not valid afterwards: write the state again.
 * The grid barrier of the conduction loop (map_set_conduction_loop) gives up at once as well;
 * with on = 2 only that barrier does.  0 restores normal waits. */
int map_test_fail_waits(map_pool* pool, int on);

/* (No counterpart in the paper.)  How the thermal-conduction substeps of a step run (Sec.
 * 3.6).  on = 1 (the default): where the pool allows it -- a single-level tree over the
 * whole pool, every ghost region a copy (same-level neighbours, periodic or outflow
 * boundaries), leaves of 2D 16^2, 2D 8^2 or 3D 8^3 cells, and every leaf's CTA resident on
 * the device at once -- one cooperative launch runs all substeps.  Each CTA keeps its leaf's
 * state on chip and exchanges the interior energy with the leaves it borders through the
 * energy slices of the two spare state buffers, with one bounded grid barrier per substep.
 * A barrier that waits about a second without completing sets the timeout bit, and
 * map_check then returns MAP_ETIMEOUT.  Elsewhere, and while the pool's stream is being
 * captured: one ghost fill and one kernel per substep, graph-replayed.  on = 0 always takes
 * that path.  The arithmetic is the same either way.  Returns MAP_OK or MAP_EINVAL (NULL
 * pool). */
int map_set_conduction_loop(map_pool* pool, int on);

/* (No counterpart in the paper.)  Sets the launch shape directly (grid 0 and weights 0
 * restore the defaults).  A persistent grid of the FP32 form gives each CTA a contiguous
 * Morton range of blocks, over whose runs of one problem and level the kernel reduces its
 * fused alpha_g and sums once. */
int map_set_launch(map_pool* pool, int grid, int w_pred, int w_face);

/* (No counterpart in the paper.)  Thermal conduction of the last step, per problem: the
 * conduction time step dt_c of the
 * reduction before it (+inf without conduction) and the number of conduction substeps it
 * ran (1 without the subcycle).  Synchronises. */
int map_last_conduction(map_pool* pool, double* dtc_out, int* nsub_out);

/* Asynchronous form of map_write_leaves (no counterpart in the paper): the copy runs on the
 * pool's own copy stream into one of two device staging buffers, so it overlaps steps still
 * running on the pool stream; the pool stream waits for it before unpacking.  The host
 * buffer (pinned, for a truly asynchronous copy) must stay unchanged until the pool stream
 * has passed this call (map_check, or any synchronising call).  Allocates the two buffers
 * (n_leaves * 9 * nb^ndim doubles each) on first use. */
int map_write_leaves_async(map_pool* pool, const double* u);

/* (No counterpart in the paper.)  map_write_leaves_async with an FP32 host layout (same
 * shape): half the bytes to copy.  An
 * MAP_FP32_FIX64 pool ends up bitwise as with the FP64 call on the same values rounded to
 * nearest; an FP64 pool takes the FP32 values exactly. */
int map_write_leaves_async_f32(map_pool* pool, const float* u);

/* (No counterpart in the paper.)  Asynchronous form of map_read_leaves: the current state's
 * leaf interiors, in the layout of map_read_leaves, are packed on the pool stream (after
 * everything enqueued before the call) into one of two device staging buffers and copied to
 * u_out on the pool's read copy stream, so the copy overlaps the steps enqueued after it and
 * runs in the other direction of the link from map_write_leaves_async.  u_out (pinned, for
 * a truly asynchronous copy) holds the state once map_check has returned (it synchronises
 * the pool's copy streams) or the device has been synchronised; it must not be read or
 * reused before.  A third call waits on the device for the copy of the first to finish
 * before reusing its staging buffer.  Allocates the two buffers (n_leaves * 9 * nb^ndim
 * values of the host layout's type each) on first use.  Errors: MAP_EINVAL, MAP_ESTATE,
 * MAP_ECUDA. */
int map_read_leaves_async(map_pool* pool, double* u_out);

/* (No counterpart in the paper.)  map_read_leaves_async into an FP32 host layout (same
 * shape): half the bytes.  An MAP_FP32_FIX64 pool's values are copied exactly; an FP64
 * pool's are rounded to nearest. */
int map_read_leaves_async_f32(map_pool* pool, float* u_out);

/* (No counterpart in the paper.)  Asynchronous map_get_speeds: out[n_problems][5] is
 * written when the pool stream reaches this point; no synchronisation.  Page-locked host
 * memory that CUDA maps into the device (cudaHostAlloc, cudaHostRegister, a framework's
 * pinned tensors) is stored to by a one-warp kernel on the pool stream, so the values do not
 * wait behind a large copy on a copy engine (an overlapped map_read_leaves_async); other host
 * memory receives a copy on the pool stream. */
int map_get_speeds_async(map_pool* pool, double* out);

/* Per problem: dt, c_h, c_p, psi damping factor, alpha_g of the last CFL reduction
 * (out[n_problems][5]).  Synchronises. */
int map_get_speeds(map_pool* pool, double* out);

/* (No counterpart in the paper.)  Number of kernels the library launched since the pool
 * was created (graph replays count each kernel in the graph). */
long long map_kernel_launches(const map_pool* pool);

/* Last error text of the pool (or of the last failed create when pool is NULL). */
const char* map_last_error(const map_pool* pool);

/* (No counterpart in the paper.)  Host-only forms of the block-tree logic, without a pool
 * or a GPU, for checking a leaf list before it reaches one.  ndim, nb and problems[n_problems]
 * as in map_pool_desc; leaves[n] as in map_set_tree; msg[msg_cap] receives the reason of a
 * rejection (empty on success; NULL allowed).
 * map_check_leaves: the validation map_set_tree performs (leaves inside their domains, no
 *   duplicates or nested leaves, every domain covered, complete parents, 2:1 over faces,
 *   edges and corners; Sec. 4.1).  MAP_OK or MAP_EINVAL.
 * map_plan_leaves: the regrid decision of map_plan_regrid (Sec. 4.5) for flags[n] on that
 *   leaf list.  out[cap] receives the new list, *n_out its length (MAP_ENOMEM when cap is too
 *   small); MAP_EINVAL if the list itself is invalid. */
int map_check_leaves(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                     const map_block_desc* leaves, int n, char* msg, int msg_cap);
int map_plan_leaves(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                    const map_block_desc* leaves, int n, const int8_t* flags, int max_level,
                    map_block_desc* out, int cap, int* n_out, char* msg, int msg_cap);

/* ---- Partition over processes: Sec. 4.2 (load balance: the blocks in curve order are cut
 * into ranges of equal block count, one per process) and Sec. 4.3 (boundary conditions
 * between processes: each process receives the blocks its ghost cells are built from).
 * Every process holds the whole tree and a pool sized for it (the paper replicates the
 * block list on every process too); it steps, reduces and sums only its own leaves.  One
 * step of a partitioned pool, per process:
 *   1. map_pack_leaves of the leaves each peer needs from it, the transfer (the caller's:
 *      NCCL or any other), map_unpack_leaves of the leaves it needs from each peer;
 *   2. map_fill_ghosts (the own leaves' ghosts are then those of the whole pool);
 *   3. map_local_alpha, the maximum over processes (the caller's all-reduce), map_set_alpha:
 *      dt, c_h, c_p exactly as map_cfl_dt on the whole pool gives them;
 *   4. map_step (own leaves only); map_conservation gives the own leaves' sums.
 * A partitioned pool steps MMC and LF without thermal conduction, and with reflux off where
 * coarse/fine faces exist (map_step returns MAP_EUNSUPPORTED otherwise): WENO's second stage,
 * conduction substeps and reflux would each need another exchange inside the step.
 * map_advance is refused (MAP_ESTATE) while a subset is active.  map_flag_refine flags every
 * leaf of the pool, but only the own leaves' flags rest on current values: gather them from
 * the processes (the paper's all-gather of refinement flags) before planning a regrid, which
 * every process then applies to its whole tree (map_regrid restores all leaves as active).
 *
 * map_plan_partition (host only, no pool, no GPU): for a leaf list as map_set_tree takes it,
 *   owner_out[n] = the process (0..nranks-1) stepping each leaf -- Morton-order ranges of
 *   equal count, the first n % nranks one leaf longer -- and need_out[nranks * n]:
 *   need_out[r * n + i] = 1 where process r needs leaf i's interior for its own leaves'
 *   ghost fill (its own leaves included): same-level and restriction sources, the leaves
 *   under a restricted parent, prolongation sources, and, where a source's own ghosts are
 *   read (prolongation stencils), that source's sources in turn.  Process r receives leaf i
 *   from owner_out[i] where need_out[r * n + i] = 1 and owner_out[i] != r.  MAP_EINVAL (text
 *   in msg) if the list is not a valid tree.
 * map_set_active: the leaves (caller indices, n of them) this pool steps, reduces (map_cfl_dt,
 *   map_local_alpha) and sums (map_conservation); leaves = NULL or n < 0 restores all.  A new
 *   tree (map_set_tree, map_regrid) restores all.  MAP_EINVAL for a bad or repeated index.
 * map_pack_leaves / map_unpack_leaves: the interiors of the n listed leaves (caller indices)
 *   to / from dev_buf, a device buffer of n * 9 * nb^ndim values in the pool's precision
 *   (double for MAP_FP64, float for MAP_FP32_FIX64; leaf-major, then [9][nz][nb][nb]),
 *   caller-owned, on the pool stream.  Unpacking is a host write: the next fill rebuilds
 *   every ghost region.
 * map_local_alpha: the maximum signal speed alpha_g (Sec. 3.7) over the active leaves, per
 *   problem, into alpha_out[n_problems] (host); synchronises.
 * map_set_alpha: finalises dt, c_h, c_p and the damping factor from the given alpha_g per
 *   problem (>= 0) as map_cfl_dt does after its own reduction; map_step then uses them.
 *   MAP_ENONFINITE if a dt is not finite and positive. */
int map_plan_partition(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                       const map_block_desc* leaves, int n, int nranks, int* owner_out,
                       unsigned char* need_out, char* msg, int msg_cap);
int map_set_active(map_pool* pool, const int* leaves, int n);
int map_pack_leaves(map_pool* pool, const int* leaves, int n, void* dev_buf);
int map_unpack_leaves(map_pool* pool, const int* leaves, int n, const void* dev_buf);
int map_local_alpha(map_pool* pool, const map_params* p, double* alpha_out);
int map_set_alpha(map_pool* pool, const map_params* p, const double* alpha);

/* Allocation-free CFL reduction (no counterpart in the paper; an interface addition).
 *
 * For callers that cannot allocate device memory: embedders whose device memory belongs to
 * another allocator (a framework's caching allocator, a fixed arena) and who forbid
 * cudaMalloc/cudaFree, and real-time loops that cannot afford the device synchronisation
 * cudaMalloc/cudaFree may cause.  Unlike map_cfl_dt it needs no pool: the caller passes
 * the state and receives the result, and nothing is allocated by this call.
 *
 * u_dev: device pointer to nblocks blocks of one problem with uniform spacing dx[ndim],
 *   in the pool layout [block][9][nz+4][nb+4][nb+4] (nz = nb in 3D, the z extent is 1 in
 *   2D), FP64 (precision MAP_FP64) or FP32 (MAP_FP32_FIX64); ghost cells are not read.
 * p: checked as map_cfl_dt checks it (MAP_EINVAL on the same bad values).  Thermal
 *   conduction is not covered: p->conduction other than MAP_COND_OFF is rejected with
 *   MAP_EINVAL, because its time-step bound (Sec. 3.6) needs a second reduction.
 * out (host): dt, c_h, c_p, psi damping factor, alpha_g -- the same quantities, from the
 *   same formulas, as map_cfl_dt and map_get_speeds for one problem without conduction.  A
 *   NaN anywhere in the interior makes alpha_g NaN and the call return MAP_ENONFINITE, as
 *   map_cfl_dt does.
 * The per-block partial maxima live in one file-scope static device array sized for
 *   MAP_NOALLOC_MAX_BLOCKS blocks (512 KB); every GPU that loads the library holds it until
 *   the process exits.  nblocks above that maximum is rejected with MAP_EINVAL (text in
 *   map_last_error(NULL)).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current and keeps it for the process; make that first call before any
 *   stream capture.  A device reset (cudaDeviceReset) invalidates the kept address: do not
 *   call this entry point on a device after resetting it.  Host threads may call it
 *   concurrently (the kept addresses are atomic), subject to the race below.
 * All calls share the array: calls whose kernels overlap on the GPU (different streams,
 *   no ordering between them) race and give wrong results.  Runs on `stream` (a
 *   cudaStream_t, NULL = legacy default stream), copies the five results to `out` and
 *   synchronises the stream before it returns.
 * Errors: MAP_EINVAL, MAP_ECUDA, MAP_ENONFINITE (dt not finite and positive). */
#define MAP_NOALLOC_MAX_BLOCKS 65536
int map_cfl_dt_noalloc(const void* u_dev, int precision, int ndim, int nb, int nblocks,
                       const double* dx, const map_params* p, void* stream, double* out);

#ifdef __cplusplus
}
#endif
#endif
