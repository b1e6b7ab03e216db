// capi.cpp -- the extern "C" ABI declared in include/map.h: pool memory, tree tables,
// the step sequence and its CUDA-graph replay.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "map_internal.hpp"

using namespace mapgb;

struct DevTree {
  BlockGeo* geo = nullptr;
  GhostRegion* regions = nullptr;
  int* children = nullptr;
  int* leaf_ids = nullptr;     // caller leaf order -> pool id
  int* all_leaves = nullptr;   // pool ids 0..n-1 (Morton order)
  int* level_leaves = nullptr; // concatenated by level
  int* level_parents = nullptr;
  int* level_residual = nullptr;  // per level: leaves with ghost regions the pushes leave over
  PushEntry* pushes = nullptr;
  RefluxLeaf* refl = nullptr;
  RefluxTask* rtasks = nullptr;
  int nrtasks = 0;
  void* freg = nullptr;        // face registers, tree.nslots slots
  std::vector<int> leaf_off, parent_off, residual_off;  // offsets per level (host)
  // partitioned pools (map_set_active): the leaves this pool steps, reduces and sums
  int* act_all = nullptr;      // pool ids, Morton order
  int* act_level = nullptr;    // pool ids, concatenated by level
  std::vector<int> act_off;    // offsets per level (host)
  int n_act = 0;
  int* xfer_ids = nullptr;     // pool ids of the leaves of one map_pack_leaves / map_unpack_leaves
  // the FP32 single launch's block list for a persistent grid of chunk_grid CTAs: CTA c's
  // grid-stride positions c, c + G, ... hold a contiguous Morton range of the leaves
  int* chunk_ids = nullptr;
  int chunk_grid = 0;
  bool chunk_partial = false;
};

struct map_pool {
  int ndim = 0, nb = 0, precision = 0, max_blocks = 0, nprob = 0;
  bool partial = false;        // map_set_active chose a subset of the leaves
  std::vector<map_problem_desc> probs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t block_elems = 0, elem = 0;
  void* buf[3] = {nullptr, nullptr, nullptr};
  bool ext = false;
  int cur = 0;
  HostTree tree;
  HostTree spare;              // the next tree is built here; the two swap on install
  bool have_tree = false;
  DevTree dt;
  ProbDyn* dyn = nullptr;
  unsigned* err_word = nullptr;
  double* sums = nullptr;
  double* hsub = nullptr;    // conduction substep per problem (device)
  int* nsub = nullptr;       // conduction substeps per problem (device)
  std::vector<double> hsub_h;
  std::vector<int> nsub_h;
  double* staging = nullptr;
  // asynchronous host writes: two staging buffers filled on their own copy stream, so the
  // copy of the next state overlaps the steps running on the pool stream
  double* astaging[2] = {nullptr, nullptr};
  size_t astaging_elems = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  int wslot = 0;
  // asynchronous host reads: the pack into one of two read staging buffers runs on the pool
  // stream, the copy out on a second copy stream (the other direction of the link)
  void* rstaging[2] = {nullptr, nullptr};
  size_t rstaging_bytes = 0;
  cudaStream_t rcopy_stream = nullptr;
  cudaEvent_t rpacked[2] = {nullptr, nullptr}, rcopied[2] = {nullptr, nullptr};
  int rslot = 0;
  size_t staging_elems = 0;
  int8_t* flags = nullptr;
  double* est = nullptr;
  int flags_cap = 0;
  RegridTask* tasks = nullptr;
  int tasks_cap = 0;
  bool have_dt = false;
  bool alpha_ready = false;   // dyn.alpha_bits holds alpha_g of the current state
  bool pushed[3] = {false, false, false};  // buffer q: same-level ghosts written by the last step
  bool sums_valid = false;   // sums holds the conservation sums of the current state
  // launch shape of the step kernel (map_autotune / map_set_launch): CTAs (0 = one per
  // block) and warp-schedule weights (0 = defaults)
  int tune_grid = 0, tune_wp = 0, tune_wf = 0;
  int nsm = 0;                 // SM count of the pool's device
  int fail_waits = 0;        // test hook: 1 every bounded wait gives up at once, 2 only the conduction loop's
  // conduction substep loop in one cooperative launch (map_set_conduction_loop): the switch,
  // the grid barrier words, the CTAs that can be resident at once (-1: not asked yet) and
  // whether every ghost region of the tree is a copy (-1: not checked for this tree)
  int cond_loop = 1;
  unsigned* gbar = nullptr;
  int cond_cap = -1;
  int cond_copies = -1;
  long long launches = 0;
  std::string err;
  // graph cache, one per starting buffer parity q and fill kind (2q + 1: residual fill)
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  long long graph_kernels[4] = {0, 0, 0, 0};
  map_params graph_params{};
  // conduction substep loops captured as graphs, keyed by substep count, buffer, the pushed
  // state of the first fill and reflux (cond_params: the parameters they were captured for)
  struct CondGraph {
    int nmax = 0, cur = 0;
    bool pushed = false, rf = false, seen = false;
    cudaGraphExec_t ex = nullptr;
    long long kernels = 0;
  };
  CondGraph cond_graph[8];
  int cond_next = 0;
  map_params cond_params{};
  bool graph_valid[4] = {false, false, false, false};
};

static std::string g_create_error;

namespace mapgb {
// error text for calls without a pool (returned by map_last_error(NULL))
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace mapgb

static int fail(map_pool* p, int code, const std::string& msg) {
  if (p) p->err = msg;
  else g_create_error = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(pool, MAP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static KernelConfig kcfg(const map_pool* p) { return KernelConfig{p->ndim, p->nb}; }
static bool is64(const map_pool* p) { return p->precision == MAP_FP64; }

// dispatch helpers ----------------------------------------------------------------------
#define DISPATCH(pool, name, L) \
  (is64(pool) ? launch_##name##_f64(kcfg(pool), L, pool->stream, &pool->launches) \
              : launch_##name##_f32(kcfg(pool), L, pool->stream, &pool->launches))

static void free_tree(map_pool* pool) {
  cudaFree(pool->dt.geo);
  cudaFree(pool->dt.regions);
  cudaFree(pool->dt.children);
  cudaFree(pool->dt.leaf_ids);
  cudaFree(pool->dt.all_leaves);
  cudaFree(pool->dt.level_leaves);
  cudaFree(pool->dt.level_parents);
  cudaFree(pool->dt.level_residual);
  cudaFree(pool->dt.pushes);
  cudaFree(pool->dt.refl);
  cudaFree(pool->dt.rtasks);
  cudaFree(pool->dt.freg);
  cudaFree(pool->dt.act_all);
  cudaFree(pool->dt.act_level);
  cudaFree(pool->dt.xfer_ids);
  cudaFree(pool->dt.chunk_ids);
  pool->dt = DevTree();
  pool->partial = false;
}

static void drop_graphs(map_pool* pool) {
  for (auto& c : pool->cond_graph) {
    if (c.ex) cudaGraphExecDestroy(c.ex);
    c = map_pool::CondGraph();
  }
  for (int q = 0; q < 4; ++q) {
    if (pool->graph[q]) cudaGraphExecDestroy(pool->graph[q]);
    pool->graph[q] = nullptr;
    pool->graph_valid[q] = false;
  }
}

template <typename X>
static cudaError_t upload(X** dst, const std::vector<X>& src, cudaStream_t s) {
  size_t n = src.size() ? src.size() : 1;
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(X));
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(X), cudaMemcpyHostToDevice, s);
  return e;
}

extern "C" {

int map_create_pool(const map_pool_desc* d, void* stream, map_pool** out) {
  map_pool* pool = nullptr;
  if (!d || !out) return fail(nullptr, MAP_EINVAL, "null argument");
  *out = nullptr;
  if (d->ndim != 2 && d->ndim != 3) return fail(nullptr, MAP_EINVAL, "ndim must be 2 or 3");
  if (d->nb != 8 && d->nb != 16) return fail(nullptr, MAP_EUNSUPPORTED, "nb must be 8 or 16");
  if (d->n_ghost != 2) return fail(nullptr, MAP_EINVAL, "n_ghost must be 2");
  if (d->precision != MAP_FP64 && d->precision != MAP_FP32_FIX64) return fail(nullptr, MAP_EINVAL, "bad precision");
  if (d->max_blocks < 1 || d->n_problems < 1 || !d->problems) return fail(nullptr, MAP_EINVAL, "bad capacity or problems");
  pool = new map_pool();
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&pool->nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  pool->ndim = d->ndim;
  pool->nb = d->nb;
  pool->precision = d->precision;
  pool->max_blocks = d->max_blocks;
  pool->nprob = d->n_problems;
  pool->probs.assign(d->problems, d->problems + d->n_problems);
  const int NP = d->nb + 4;
  const size_t S = (size_t)NP * NP * (d->ndim == 3 ? NP : 1);
  pool->block_elems = (size_t)kNV * S;
  pool->elem = d->precision == MAP_FP64 ? 8 : 4;
  const size_t buf_bytes = pool->block_elems * pool->elem * (size_t)d->max_blocks;
  auto cleanup = [&](int code, const std::string& m) {
    g_create_error = m;
    map_destroy_pool(pool);
    return code;
  };
  if (stream) {
    pool->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&pool->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(MAP_ECUDA, "cudaStreamCreate failed");
    pool->own_stream = true;
  }
  if (d->ext_buffer) {
    if (d->ext_bytes < 3 * buf_bytes) return cleanup(MAP_ENOMEM, "external buffer smaller than 3 state buffers");
    if (((uintptr_t)d->ext_buffer) % 256) return cleanup(MAP_EINVAL, "external buffer must be 256-byte aligned");
    pool->ext = true;
    for (int q = 0; q < 3; ++q) pool->buf[q] = (char*)d->ext_buffer + q * buf_bytes;
  } else {
    for (int q = 0; q < 3; ++q)
      if (cudaMalloc(&pool->buf[q], buf_bytes) != cudaSuccess) return cleanup(MAP_ENOMEM, "cudaMalloc of the block pool failed");
  }
  // zero the state buffers so never-written ghost or parent cells are finite
  for (int q = 0; q < 3; ++q)
    if (cudaMemsetAsync(pool->buf[q], 0, buf_bytes, pool->stream) != cudaSuccess) return cleanup(MAP_ECUDA, "memset failed");
  if (cudaMalloc(&pool->dyn, sizeof(ProbDyn) * pool->nprob) != cudaSuccess ||
      cudaMalloc(&pool->err_word, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&pool->sums, sizeof(double) * kNV * pool->nprob) != cudaSuccess ||
      cudaMalloc(&pool->hsub, sizeof(double) * pool->nprob) != cudaSuccess ||
      cudaMalloc(&pool->nsub, sizeof(int) * pool->nprob) != cudaSuccess ||
      cudaMalloc(&pool->gbar, 2 * sizeof(unsigned)) != cudaSuccess)
    return cleanup(MAP_ENOMEM, "cudaMalloc of the step constants failed");
  cudaMemsetAsync(pool->dyn, 0, sizeof(ProbDyn) * pool->nprob, pool->stream);
  cudaMemsetAsync(pool->err_word, 0, sizeof(unsigned), pool->stream);
  if (cudaStreamSynchronize(pool->stream) != cudaSuccess) return cleanup(MAP_ECUDA, "stream synchronize failed");
  *out = pool;
  return MAP_OK;
}

int map_destroy_pool(map_pool* pool) {
  if (!pool) return MAP_OK;
  if (pool->stream) cudaStreamSynchronize(pool->stream);
  drop_graphs(pool);
  free_tree(pool);
  if (!pool->ext)
    for (int q = 0; q < 3; ++q) cudaFree(pool->buf[q]);
  cudaFree(pool->dyn);
  cudaFree(pool->hsub);
  cudaFree(pool->nsub);
  cudaFree(pool->gbar);
  cudaFree(pool->err_word);
  cudaFree(pool->sums);
  cudaFree(pool->staging);
  if (pool->copy_stream) {
    cudaStreamSynchronize(pool->copy_stream);
    for (int k = 0; k < 2; ++k) {
      cudaFree(pool->astaging[k]);
      cudaEventDestroy(pool->copied[k]);
      cudaEventDestroy(pool->consumed[k]);
    }
    cudaStreamDestroy(pool->copy_stream);
  }
  if (pool->rcopy_stream) {
    cudaStreamSynchronize(pool->rcopy_stream);
    for (int k = 0; k < 2; ++k) {
      cudaFree(pool->rstaging[k]);
      cudaEventDestroy(pool->rpacked[k]);
      cudaEventDestroy(pool->rcopied[k]);
    }
    cudaStreamDestroy(pool->rcopy_stream);
  }
  cudaFree(pool->flags);
  cudaFree(pool->est);
  cudaFree(pool->tasks);
  if (pool->own_stream) cudaStreamDestroy(pool->stream);
  delete pool;
  return MAP_OK;
}

int map_set_stream(map_pool* pool, void* stream) {
  if (!pool) return MAP_EINVAL;
  cudaStreamSynchronize(pool->stream);
  if (pool->own_stream) cudaStreamDestroy(pool->stream);
  pool->own_stream = false;
  if (stream) pool->stream = (cudaStream_t)stream;
  else {
    CK(cudaStreamCreateWithFlags(&pool->stream, cudaStreamNonBlocking));
    pool->own_stream = true;
  }
  drop_graphs(pool);
  return MAP_OK;
}

static int install_tree(map_pool* pool, HostTree& t) {
  free_tree(pool);
  drop_graphs(pool);
  pool->cond_copies = -1;
  DevTree& D = pool->dt;
  CK(upload(&D.geo, t.geo, pool->stream));
  CK(upload(&D.regions, t.regions, pool->stream));
  CK(upload(&D.children, t.children, pool->stream));
  CK(upload(&D.leaf_ids, t.leaf_to_block, pool->stream));
  CK(upload(&D.all_leaves, t.all_leaves, pool->stream));
  CK(upload(&D.pushes, t.pushes, pool->stream));
  CK(upload(&D.refl, t.refl, pool->stream));
  if (!t.reflux_tasks.empty()) {
    CK(upload(&D.rtasks, t.reflux_tasks, pool->stream));
    D.nrtasks = (int)t.reflux_tasks.size();
    CK(cudaMalloc(&D.freg, (size_t)t.nslots * 2 * pool->ndim * kNV * pool->nb * pool->nb * pool->elem));
  }
  std::vector<int> ll, pl, rl;
  D.leaf_off.assign(t.maxlev + 2, 0);
  D.parent_off.assign(t.maxlev + 2, 0);
  D.residual_off.assign(t.maxlev + 2, 0);
  for (int L = 0; L <= t.maxlev; ++L) {
    D.leaf_off[L] = (int)ll.size();
    ll.insert(ll.end(), t.leaves_by_level[L].begin(), t.leaves_by_level[L].end());
    D.parent_off[L] = (int)pl.size();
    pl.insert(pl.end(), t.parents_by_level[L].begin(), t.parents_by_level[L].end());
    D.residual_off[L] = (int)rl.size();
    rl.insert(rl.end(), t.residual_by_level[L].begin(), t.residual_by_level[L].end());
  }
  D.leaf_off[t.maxlev + 1] = (int)ll.size();
  D.parent_off[t.maxlev + 1] = (int)pl.size();
  D.residual_off[t.maxlev + 1] = (int)rl.size();
  CK(upload(&D.level_leaves, ll, pool->stream));
  CK(upload(&D.level_parents, pl, pool->stream));
  CK(upload(&D.level_residual, rl, pool->stream));
  // per-problem minimum spacing (dt uses the finest leaf, Sec. 4.5 / Sec. 3.7)
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  for (int p = 0; p < pool->nprob; ++p) {
    dyn[p].mindx = t.mindx[p];
    dyn[p].alpha_bits = 0ull;
    // level-0 spacing, the same expression as the tree's per-block spacing at level 0
    for (int d = 0; d < 3; ++d) {
      const int ncell = d < pool->ndim ? pool->probs[p].nbase[d] * pool->nb : 1;
      dyn[p].dx0[d] = (pool->probs[p].hi[d] - pool->probs[p].lo[d]) / (double)ncell;
    }
  }
  CK(cudaMemcpyAsync(pool->dyn, dyn.data(), sizeof(ProbDyn) * pool->nprob, cudaMemcpyHostToDevice, pool->stream));
  // staging for host-layout copies
  const size_t ni = (size_t)pool->nb * pool->nb * (pool->ndim == 3 ? pool->nb : 1);
  const size_t need = (size_t)t.nleaves * kNV * ni;
  if (need > pool->staging_elems) {
    cudaFree(pool->staging);
    pool->staging = nullptr;
    CK(cudaMalloc(&pool->staging, need * sizeof(double)));
    pool->staging_elems = need;
  }
  if (t.nleaves > pool->flags_cap) {
    cudaFree(pool->flags);
    cudaFree(pool->est);
    CK(cudaMalloc(&pool->flags, t.nleaves));
    CK(cudaMalloc(&pool->est, t.nleaves * sizeof(double)));
    pool->flags_cap = t.nleaves;
  }
  CK(cudaStreamSynchronize(pool->stream));
  std::swap(pool->tree, t);    // t (the spare) keeps the old tree's storage for reuse
  pool->have_tree = true;
  pool->have_dt = false;
  pool->alpha_ready = false;
  for (int q = 0; q < 3; ++q) pool->pushed[q] = false;
  pool->sums_valid = false;
  return MAP_OK;
}

int map_set_tree(map_pool* pool, const map_block_desc* leaves, int n) {
  if (!pool || !leaves || n <= 0) return fail(pool, MAP_EINVAL, "null or empty leaf list");
  HostTree& t = pool->spare;
  std::string why = build_tree(pool->ndim, pool->nb, pool->probs, leaves, n, t);
  if (!why.empty()) return fail(pool, MAP_EINVAL, why);
  if (t.nblocks > pool->max_blocks) return fail(pool, MAP_ENOMEM, "tree has more blocks than max_blocks");
  return install_tree(pool, t);
}

static size_t interior_elems(const map_pool* p) {
  return (size_t)p->nb * p->nb * (p->ndim == 3 ? p->nb : 1) * kNV;
}

static int pack(map_pool* pool, const int* dev_ids, int n, int to_pool, double* staging = nullptr, int f32 = 0) {
  PackLaunch L;
  L.u = pool->buf[pool->cur];
  L.host_layout = staging ? staging : pool->staging;
  L.staging_f32 = f32;
  L.blocks = dev_ids;
  L.nblocks = n;
  L.to_pool = to_pool;
  CK(DISPATCH(pool, pack, L));
  return MAP_OK;
}

int map_write_block(map_pool* pool, int leaf, const double* u) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  if (leaf < 0 || leaf >= pool->tree.nleaves) return fail(pool, MAP_EINVAL, "leaf index out of range");
  CK(cudaMemcpyAsync(pool->staging, u, interior_elems(pool) * sizeof(double), cudaMemcpyHostToDevice, pool->stream));
  pool->have_dt = false;
  pool->alpha_ready = false;
  pool->pushed[pool->cur] = false;
  pool->sums_valid = false;
  return pack(pool, pool->dt.leaf_ids + leaf, 1, 1);
}

int map_read_block(map_pool* pool, int leaf, double* u) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  if (leaf < 0 || leaf >= pool->tree.nleaves) return fail(pool, MAP_EINVAL, "leaf index out of range");
  int rc = pack(pool, pool->dt.leaf_ids + leaf, 1, 0);
  if (rc) return rc;
  CK(cudaMemcpyAsync(u, pool->staging, interior_elems(pool) * sizeof(double), cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  return MAP_OK;
}

int map_write_leaves(map_pool* pool, const double* u) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const int n = pool->tree.nleaves;
  CK(cudaMemcpyAsync(pool->staging, u, (size_t)n * interior_elems(pool) * sizeof(double), cudaMemcpyHostToDevice,
                     pool->stream));
  pool->have_dt = false;
  pool->alpha_ready = false;
  pool->pushed[pool->cur] = false;
  pool->sums_valid = false;
  return pack(pool, pool->dt.leaf_ids, n, 1);
}

static int write_leaves_async(map_pool* pool, const void* u, int f32) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const int n = pool->tree.nleaves;
  const size_t need = (size_t)n * interior_elems(pool);
  if (!pool->copy_stream) {
    CK(cudaStreamCreateWithFlags(&pool->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventCreateWithFlags(&pool->copied[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&pool->consumed[k], cudaEventDisableTiming));
      CK(cudaEventRecord(pool->consumed[k], pool->stream));
    }
  }
  if (need > pool->astaging_elems) {
    CK(cudaStreamSynchronize(pool->copy_stream));
    CK(cudaStreamSynchronize(pool->stream));
    for (int k = 0; k < 2; ++k) {
      cudaFree(pool->astaging[k]);
      pool->astaging[k] = nullptr;
      CK(cudaMalloc(&pool->astaging[k], need * sizeof(double)));
    }
    pool->astaging_elems = need;
  }
  const int k = pool->wslot;
  pool->wslot ^= 1;
  // the copy into buffer k waits for the pack that last read it; the pack waits for the copy
  CK(cudaStreamWaitEvent(pool->copy_stream, pool->consumed[k], 0));
  CK(cudaMemcpyAsync(pool->astaging[k], u, need * (f32 ? sizeof(float) : sizeof(double)), cudaMemcpyHostToDevice,
                     pool->copy_stream));
  CK(cudaEventRecord(pool->copied[k], pool->copy_stream));
  CK(cudaStreamWaitEvent(pool->stream, pool->copied[k], 0));
  pool->have_dt = false;
  pool->alpha_ready = false;
  pool->pushed[pool->cur] = false;
  pool->sums_valid = false;
  int rc = pack(pool, pool->dt.leaf_ids, n, 1, pool->astaging[k], f32);
  if (rc) return rc;
  CK(cudaEventRecord(pool->consumed[k], pool->stream));
  return MAP_OK;
}

int map_write_leaves_async(map_pool* pool, const double* u) { return write_leaves_async(pool, u, 0); }

int map_write_leaves_async_f32(map_pool* pool, const float* u) { return write_leaves_async(pool, u, 1); }

// pack the current state into read staging buffer k (pool stream), then copy it to the host
// on the read copy stream; the next pack into buffer k waits for that copy
static int read_leaves_async(map_pool* pool, void* u, int f32) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const int n = pool->tree.nleaves;
  const size_t bytes = (size_t)n * interior_elems(pool) * (f32 ? sizeof(float) : sizeof(double));
  if (!pool->rcopy_stream) {
    CK(cudaStreamCreateWithFlags(&pool->rcopy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventCreateWithFlags(&pool->rpacked[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&pool->rcopied[k], cudaEventDisableTiming));
      CK(cudaEventRecord(pool->rcopied[k], pool->rcopy_stream));
    }
  }
  if (bytes > pool->rstaging_bytes) {
    CK(cudaStreamSynchronize(pool->rcopy_stream));
    CK(cudaStreamSynchronize(pool->stream));
    for (int k = 0; k < 2; ++k) {
      cudaFree(pool->rstaging[k]);
      pool->rstaging[k] = nullptr;
      CK(cudaMalloc(&pool->rstaging[k], bytes));
    }
    pool->rstaging_bytes = bytes;
  }
  const int k = pool->rslot;
  pool->rslot ^= 1;
  CK(cudaStreamWaitEvent(pool->stream, pool->rcopied[k], 0));
  int rc = pack(pool, pool->dt.leaf_ids, n, 0, (double*)pool->rstaging[k], f32);
  if (rc) return rc;
  CK(cudaEventRecord(pool->rpacked[k], pool->stream));
  CK(cudaStreamWaitEvent(pool->rcopy_stream, pool->rpacked[k], 0));
  CK(cudaMemcpyAsync(u, pool->rstaging[k], bytes, cudaMemcpyDeviceToHost, pool->rcopy_stream));
  CK(cudaEventRecord(pool->rcopied[k], pool->rcopy_stream));
  return MAP_OK;
}

int map_read_leaves_async(map_pool* pool, double* u) { return read_leaves_async(pool, u, 0); }

int map_read_leaves_async_f32(map_pool* pool, float* u) { return read_leaves_async(pool, u, 1); }

int map_read_leaves(map_pool* pool, double* u) {
  if (!pool || !u) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const int n = pool->tree.nleaves;
  int rc = pack(pool, pool->dt.leaf_ids, n, 0);
  if (rc) return rc;
  CK(cudaMemcpyAsync(u, pool->staging, (size_t)n * interior_elems(pool) * sizeof(double), cudaMemcpyDeviceToHost,
                     pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  return MAP_OK;
}

// ghost fill on state buffer q: restriction bottom-up, then level passes top-down.  When
// the last step kernel writing buffer q already wrote the same-level copies, only the rest
// is filled (and levels without any such region are skipped).
static int fill_on(map_pool* pool, int q) {
  const HostTree& t = pool->tree;
  const DevTree& D = pool->dt;
  // a partitioned pool's ghosts may come from leaves another process steps: every region
  const bool residual = pool->pushed[q] && !pool->partial;
  for (int L = t.maxlev - 1; L >= 0; --L) {
    RestrictLaunch R;
    R.u = pool->buf[q];
    R.parents = D.level_parents + D.parent_off[L];
    R.nparents = D.parent_off[L + 1] - D.parent_off[L];
    R.children = D.children;
    CK(DISPATCH(pool, restrict, R));
  }
  for (int L = 0; L <= t.maxlev; ++L) {
    if (residual && !t.level_has_residual[L]) continue;
    FillLaunch F;
    F.u = pool->buf[q];
    // after a step only the leaves with regions that no push wrote take part
    F.blocks = residual ? D.level_residual + D.residual_off[L] : D.level_leaves + D.leaf_off[L];
    F.nblocks = residual ? D.residual_off[L + 1] - D.residual_off[L] : D.leaf_off[L + 1] - D.leaf_off[L];
    F.regions = D.regions;
    F.skip_pushed = residual ? 1 : 0;
    CK(DISPATCH(pool, fill, F));
  }
  return MAP_OK;
}

// ghosts of the energy alone on buffer q, every region (between conduction substeps)
static int fill_energy_on(map_pool* pool, int q) {
  const HostTree& t = pool->tree;
  const DevTree& D = pool->dt;
  for (int L = t.maxlev - 1; L >= 0; --L) {
    RestrictLaunch R;
    R.u = pool->buf[q];
    R.parents = D.level_parents + D.parent_off[L];
    R.nparents = D.parent_off[L + 1] - D.parent_off[L];
    R.children = D.children;
    CK(DISPATCH(pool, restrict, R));
  }
  for (int L = 0; L <= t.maxlev; ++L) {
    FillLaunch F;
    F.u = pool->buf[q];
    F.blocks = D.level_leaves + D.leaf_off[L];
    F.nblocks = D.leaf_off[L + 1] - D.leaf_off[L];
    F.regions = D.regions;
    F.skip_pushed = 0;
    F.v0 = kEN;
    F.v1 = kEN + 1;
    CK(DISPATCH(pool, fill, F));
  }
  return MAP_OK;
}

int map_fill_ghosts(map_pool* pool) {
  if (!pool) return MAP_EINVAL;
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  return fill_on(pool, pool->cur);
}

static FinalizeLaunch make_finalize(const map_pool* pool, const map_params* p) {
  FinalizeLaunch F;
  F.dyn = pool->dyn;
  F.nprob = pool->nprob;
  F.ndim = pool->ndim;
  F.c_cfl = p->c_cfl;
  F.eta = p->eta;
  F.ch_fixed = p->ch;
  F.cp_fixed = p->cp;
  F.c_d = p->c_d;
  F.dt_override = p->dt_override;
  F.ch_mode = p->ch_mode;
  F.cp_mode = p->cp_mode;
  F.conduction = p->conduction;
  F.subcycle = p->subcycle;
  return F;
}

// alpha_g of the current state into dyn.alpha_bits (max over leaf cells, Sec. 3.7)
static int alpha_device(map_pool* pool, const map_params* p) {
  CK(launch_zero_alpha(pool->dyn, pool->nprob, pool->stream, &pool->launches));
  CflLaunch C;
  C.u = pool->buf[pool->cur];
  C.blocks = pool->partial ? pool->dt.act_all : pool->dt.all_leaves;
  C.nblocks = pool->partial ? pool->dt.n_act : pool->tree.nleaves;
  C.geo = pool->dt.geo;
  C.dyn = pool->dyn;
  C.gamma = p->gamma;
  C.kappa0 = p->conduction ? p->kappa0 : 0.0;
  if (C.nblocks > 0) CK(DISPATCH(pool, cfl, C));
  return MAP_OK;
}

static int cfl_device(map_pool* pool, const map_params* p) {
  int rc = alpha_device(pool, p);
  if (rc) return rc;
  CK(launch_finalize(make_finalize(pool, p), pool->stream, &pool->launches));
  pool->alpha_ready = false;  // finalize consumed and reset the running maximum
  return MAP_OK;
}

static bool params_equal(const map_params& a, const map_params& b) {
  return a.gamma == b.gamma && a.c_cfl == b.c_cfl && a.ch_mode == b.ch_mode && a.ch == b.ch &&
         a.cp_mode == b.cp_mode && a.c_d == b.c_d && a.cp == b.cp && a.eta == b.eta && a.eglm == b.eglm &&
         a.scheme == b.scheme && a.limiter == b.limiter && a.dt_override == b.dt_override &&
         a.fp64_fix_tau == b.fp64_fix_tau && a.reflux == b.reflux && a.riemann == b.riemann &&
         a.conduction == b.conduction && a.kappa0 == b.kappa0 && a.subcycle == b.subcycle &&
         a.grad_t_max == b.grad_t_max;
}

// Threshold of the FP32 pressure recovery's FP64 fallback: tau > 0 recomputes p in FP64
// where e_int < tau e; tau <= 0 turns the fallback off (-inf: the comparison never holds for
// e >= 0), so the FP32 form then recovers every pressure in FP32.  FP64 pools ignore it.
static double fix_tau(const map_pool* pool, const map_params* p) {
  if (is64(pool)) return 0.0;
  return p->fp64_fix_tau > 0.0 ? p->fp64_fix_tau : -INFINITY;
}

}  // extern "C"

// The parameter checks that need no pool: nullptr when p is acceptable, else the reason.
const char* mapgb::params_problem(const map_params* p) {
  if (!p) return "null params";
  if (!(p->gamma > 1.0) || !(p->c_cfl > 0.0)) return "gamma must exceed 1 and c_cfl be positive";
  if (p->scheme < 0 || p->scheme > 2 || p->limiter < 0 || p->limiter > 1) return "bad scheme or limiter";
  if (p->ch_mode < 0 || p->ch_mode > 2 || p->cp_mode < 0 || p->cp_mode > 1) return "bad c_h / c_p mode";
  if (p->cp_mode == MAP_CP_FROM_CD && !(p->c_d > 0.0 && p->c_d < 1.0)) return "c_d must lie in (0,1)";
  if (!(p->eta >= 0.0)) return "eta must be >= 0";
  if (p->riemann != MAP_RIEMANN_LF && p->riemann != MAP_RIEMANN_HLLC && p->riemann != MAP_RIEMANN_HLLD)
    return "bad riemann";
  if (p->conduction < MAP_COND_OFF || p->conduction > MAP_COND_ALIGNED) return "bad conduction mode";
  if (p->conduction && !(p->kappa0 > 0.0)) return "conduction needs kappa0 > 0";
  if (!(p->grad_t_max >= 0.0)) return "grad_t_max must be >= 0";
  if (p->riemann != MAP_RIEMANN_LF && p->scheme == MAP_MMC)
    return "HLLC and HLLD are interface fluxes of LF and WENO; MMC takes MAP_RIEMANN_LF";
  return nullptr;
}

extern "C" {

static int check_params(map_pool* pool, const map_params* p) {
  if (const char* why = params_problem(p)) return fail(pool, MAP_EINVAL, why);
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  size_t smem = is64(pool) ? step_smem_f64(kcfg(pool), p->scheme, p->eta > 0.0)
                           : step_smem_f32(kcfg(pool), p->scheme, p->eta > 0.0);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem == 0 || (optin > 0 && smem > (size_t)optin))
    return fail(pool, MAP_EUNSUPPORTED, "this block size / precision / scheme / resistivity needs more shared memory than a block has");
  return MAP_OK;
}

// What a partitioned pool cannot do inside one map_step: the WENO stage state and the
// conduction substeps need their halo leaves exchanged between the stages, and reflux at a
// coarse/fine face needs the face fluxes of leaves another process may step.
static int check_partial(map_pool* pool, const map_params* p) {
  if (!pool->partial) return MAP_OK;
  if (p->scheme == MAP_WENO)
    return fail(pool, MAP_EUNSUPPORTED, "a partitioned pool steps MMC and LF only (WENO's second stage needs an exchange)");
  if (p->conduction)
    return fail(pool, MAP_EUNSUPPORTED, "a partitioned pool steps without thermal conduction (its substeps need exchanges)");
  if (p->reflux && pool->dt.nrtasks > 0)
    return fail(pool, MAP_EUNSUPPORTED, "a partitioned pool with coarse/fine faces steps with reflux off");
  return MAP_OK;
}

int map_cfl_dt(map_pool* pool, const map_params* p, double* dt_out) {
  if (!pool) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  rc = cfl_device(pool, p);
  if (rc) return rc;
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  pool->have_dt = true;
  int status = MAP_OK;
  for (int q = 0; q < pool->nprob; ++q) {
    if (dt_out) dt_out[q] = dyn[q].dt;
    if (!(isfinite(dyn[q].dt) && dyn[q].dt > 0.0)) status = MAP_ENONFINITE;
  }
  if (status) return fail(pool, status, "time step is not finite and positive (non-finite or zero signal speed)");
  return MAP_OK;
}

// Grid of the FP32 single step launch: the tuned one, else one CTA per block in 3D and, in
// 2D (256-cell blocks, whose per-block reductions weigh), a persistent grid of four CTAs per
// SM (the residency of the 128-thread 2D FP32 kernels).
static int step_grid(const map_pool* pool) {
  if (pool->tune_grid > 0) return pool->tune_grid;
  if (!is64(pool) && pool->ndim == 2 && pool->nsm > 0) return 4 * pool->nsm;
  return 0;
}

// The block list of the FP32 single launch with grid G: for a persistent grid, the leaves
// (or the active ones) reordered so that each CTA's grid-stride positions hold one contiguous
// Morton range (its blocks then share problem and level in long runs, over which the kernel
// reduces its fused diagnostics once).  Built outside stream capture; during a capture
// without it the plain order is used.
static int step_block_list(map_pool* pool, int G, const int** list) {
  DevTree& D = pool->dt;
  const HostTree& t = pool->tree;
  const int n = pool->partial ? D.n_act : t.nleaves;
  *list = pool->partial ? D.act_all : D.all_leaves;
  if (G <= 0 || G >= n) return MAP_OK;
  if (D.chunk_ids && D.chunk_grid == G && D.chunk_partial == pool->partial) {
    *list = D.chunk_ids;
    return MAP_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(pool->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return MAP_OK;
  std::vector<int> src(n), perm(n);
  CK(cudaMemcpyAsync(src.data(), *list, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  int start = 0;
  for (int c = 0; c < G; ++c) {
    const int len = c < n ? (n - 1 - c) / G + 1 : 0;   // positions c, c + G, ... below n
    for (int k = 0; k < len; ++k) perm[c + (size_t)k * G] = src[start + k];
    start += len;
  }
  if (!D.chunk_ids) CK(cudaMalloc(&D.chunk_ids, (size_t)t.nleaves * sizeof(int)));
  CK(cudaMemcpyAsync(D.chunk_ids, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  D.chunk_grid = G;
  D.chunk_partial = pool->partial;
  *list = D.chunk_ids;
  return MAP_OK;
}

// launches of one step on buffer pool->cur; flips cur.  fused: also reduce alpha of the
// new state into dyn (next dt) and the FP64 sums.
static int step_launches(map_pool* pool, const map_params* p, bool fused) {
  const HostTree& t = pool->tree;
  StepLaunch S{};
  S.geo = pool->dt.geo;
  S.dyn = pool->dyn;
  S.gamma = p->gamma;
  S.eta = p->eta;
  S.tau = fix_tau(pool, p);
  S.eglm = p->eglm;
  S.scheme = p->scheme;
  S.limiter = p->limiter;
  S.riemann = p->riemann;
  S.w_pred = pool->tune_wp;
  S.w_face = pool->tune_wf;
  S.fail_waits = pool->fail_waits == 1;
  S.err_word = pool->err_word;
  S.sums = fused ? pool->sums : nullptr;
  S.dyn_next = fused ? pool->dyn : nullptr;
  S.pushes = pool->dt.pushes;
  const bool reflux = p->reflux != 0 && pool->dt.nrtasks > 0;
  S.freg = reflux ? pool->dt.freg : nullptr;
  S.refl = reflux ? pool->dt.refl : nullptr;
  const int in = pool->cur, out = 1 - pool->cur;
  // the plain FP64 form launches once per level; the FP32 form once over all leaves
  auto run = [&](const void* uin, void* uout, const void* ubase, int stage, bool with_fused) -> int {
    S.u_in = uin;
    S.u_out = uout;
    S.u_base = ubase;
    S.stage = stage;
    S.sums = with_fused ? pool->sums : nullptr;
    S.dyn_next = with_fused ? pool->dyn : nullptr;
    const DevTree& D = pool->dt;
    if (is64(pool)) {
      for (int L = 0; L <= t.maxlev; ++L) {
        const std::vector<int>& off = pool->partial ? D.act_off : D.leaf_off;
        S.blocks = (pool->partial ? D.act_level : D.level_leaves) + off[L];
        S.nblocks = off[L + 1] - off[L];
        if (S.nblocks == 0) continue;
        S.grid = pool->tune_grid;
        CK(DISPATCH(pool, step, S));
      }
    } else {
      S.nblocks = pool->partial ? D.n_act : t.nleaves;
      S.grid = step_grid(pool);
      const int rcl = step_block_list(pool, S.grid, &S.blocks);
      if (rcl) return rcl;
      if (S.nblocks > 0) CK(DISPATCH(pool, step, S));
    }
    return MAP_OK;
  };
  int rc;
  if (fused) {
    CK(cudaMemsetAsync(pool->sums, 0, sizeof(double) * kNV * pool->nprob, pool->stream));
  }
  if (p->scheme == MAP_WENO) {
    rc = run(pool->buf[in], pool->buf[2], nullptr, 1, false);
    if (rc) return rc;
    pool->pushed[2] = true;
    rc = fill_on(pool, 2);
    if (rc) return rc;
    rc = run(pool->buf[2], pool->buf[out], pool->buf[in], 2, fused);
    if (rc) return rc;
  } else {
    rc = run(pool->buf[in], pool->buf[out], nullptr, 0, fused);
    if (rc) return rc;
  }
  if (reflux) {
    RefluxLaunch R;
    R.u = pool->buf[out];
    R.tasks = pool->dt.rtasks;
    R.ntasks = pool->dt.nrtasks;
    R.freg = pool->dt.freg;
    R.geo = pool->dt.geo;
    R.dyn = pool->dyn;
    R.pushes = pool->dt.pushes;
    R.gamma = p->gamma;
    R.tau = S.tau;
    R.err_word = pool->err_word;
    R.sums = fused ? pool->sums : nullptr;
    R.dyn_next = fused ? pool->dyn : nullptr;
    CK(DISPATCH(pool, reflux, R));
  }
  pool->cur = out;
  pool->pushed[out] = true;
  return MAP_OK;
}

// Thermal conduction over the step just taken (Sec. 3.6): n = ceil(dt / dt_c) substeps of
// dt / n per problem with the subcycle (dt and dt_c of the reduction before the step), else
// one; each refills the ghosts (the first all variables, then the energy alone), updates the
// energy in place and refluxes it at coarse/fine faces.  Reads dt back to size the loop.
static int conduction_substep(map_pool* pool, const map_params* p, int it, bool rf);

// Whether this step's conduction substeps can run as one cooperative launch: switched on, a
// single-level tree of the whole pool whose ghost regions are all copies (their first ghost
// layer then reads interior cells of the source leaf), no energy reflux, leaf shapes the loop
// kernel holds on chip, every leaf's CTA resident at once, and no stream capture under way.
static bool cond_loop_usable(map_pool* pool, bool rf) {
  if (!pool->cond_loop || rf || pool->partial || pool->tree.maxlev != 0) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(pool->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  if (pool->cond_cap < 0)
    pool->cond_cap = is64(pool) ? cond_loop_capacity_f64(kcfg(pool), pool->nsm) : cond_loop_capacity_f32(kcfg(pool), pool->nsm);
  if (pool->tree.nleaves > pool->cond_cap) return false;
  if (pool->cond_copies < 0) {
    int ok = 1;
    const HostTree& t = pool->tree;
    for (int l = 0; l < t.nleaves && ok; ++l) {
      const int id = t.leaf_to_block[l];
      for (int r = 0; r < 27 && ok; ++r)
        if (t.regions[(size_t)id * 27 + r].kind != 0) ok = 0;
    }
    pool->cond_copies = ok;
  }
  return pool->cond_copies == 1;
}

static int conduction_launches(map_pool* pool, const map_params* p) {
  const int np = pool->nprob;
  std::vector<ProbDyn> dyn(np);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * np, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  pool->hsub_h.assign(np, 0.0);
  pool->nsub_h.assign(np, 1);
  int nmax = 1;
  for (int q = 0; q < np; ++q) {
    double n = 1.0;
    if (p->subcycle && dyn[q].dtc < dyn[q].dt) n = ceil(dyn[q].dt / dyn[q].dtc);
    if (!(n <= 1048576.0)) return fail(pool, MAP_EUNSUPPORTED, "thermal conduction would need more than 2^20 substeps");
    pool->nsub_h[q] = (int)n;
    pool->hsub_h[q] = dyn[q].dt / (double)(int)n;
    if ((int)n > nmax) nmax = (int)n;
  }
  CK(cudaMemcpyAsync(pool->hsub, pool->hsub_h.data(), sizeof(double) * np, cudaMemcpyHostToDevice, pool->stream));
  CK(cudaMemcpyAsync(pool->nsub, pool->nsub_h.data(), sizeof(int) * np, cudaMemcpyHostToDevice, pool->stream));
  const bool rf = p->reflux != 0 && pool->dt.nrtasks > 0;
  if (cond_loop_usable(pool, rf)) {
    // the whole loop in one cooperative launch: a full fill first (as the first substep of
    // the per-substep path does), then every substep on the ring regions kept on chip
    int rc = fill_on(pool, pool->cur);
    if (rc) return rc;
    CK(cudaMemsetAsync(pool->gbar, 0, 2 * sizeof(unsigned), pool->stream));
    CondLoopLaunch C;
    C.u = pool->buf[pool->cur];
    C.e_pp[0] = pool->buf[1 - pool->cur];
    C.e_pp[1] = pool->buf[2];
    C.blocks = pool->dt.all_leaves;
    C.nblocks = pool->tree.nleaves;
    C.geo = pool->dt.geo;
    C.regions = pool->dt.regions;
    C.gamma = p->gamma;
    C.tau = fix_tau(pool, p);
    C.kappa0 = p->kappa0;
    C.grad_t_max = p->grad_t_max;
    C.mode = p->conduction;
    C.hsub = pool->hsub;
    C.nsub = pool->nsub;
    C.nmax = nmax;
    C.bar = pool->gbar;
    C.err_word = pool->err_word;
    C.fail_waits = pool->fail_waits != 0;
    if (DISPATCH(pool, cond_loop, C) == cudaSuccess) {
      pool->pushed[pool->cur] = false;     // the energy ghosts are stale now
      return MAP_OK;
    }
    // the device refused the cooperative launch: the per-substep path from now on
    cudaGetLastError();
    pool->cond_cap = 0;
  }
  // The substep loop is launch-bound on small meshes (a fill and a conduction launch per
  // substep): the second time a (substep count, buffer, fill kind) recurs it is captured into
  // a graph, and later steps replay it.  Substep sizes and counts are read from device memory
  // by the kernels, so a replay covers any dt with the same count.
  if (!params_equal(pool->cond_params, *p)) {
    drop_graphs(pool);
    pool->cond_params = *p;
  }
  const bool pushed0 = pool->pushed[pool->cur];
  map_pool::CondGraph* hit = nullptr;
  for (auto& c : pool->cond_graph)
    if (c.seen && c.nmax == nmax && c.cur == pool->cur && c.pushed == pushed0 && c.rf == rf) hit = &c;
  if (hit && hit->ex) {
    CK(cudaGraphLaunch(hit->ex, pool->stream));
    pool->launches += hit->kernels;
    pool->pushed[pool->cur] = false;
    return MAP_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(pool->stream, &cs));
  const bool capture = hit && cs == cudaStreamCaptureStatusNone;
  if (!hit) {
    map_pool::CondGraph& c = pool->cond_graph[pool->cond_next];
    pool->cond_next = (pool->cond_next + 1) % 8;
    if (c.ex) cudaGraphExecDestroy(c.ex);
    c = map_pool::CondGraph();
    c.nmax = nmax;
    c.cur = pool->cur;
    c.pushed = pushed0;
    c.rf = rf;
    c.seen = true;                 // first time: run eagerly (this also sets kernel attributes)
  }
  const long long before = pool->launches;
  if (capture) CK(cudaStreamBeginCapture(pool->stream, cudaStreamCaptureModeThreadLocal));
  int lrc = MAP_OK;
  for (int it = 0; it < nmax && lrc == MAP_OK; ++it) lrc = conduction_substep(pool, p, it, rf);
  if (capture) {
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(pool->stream, &g);
    if (lrc == MAP_OK && ce == cudaSuccess && g) {
      cudaGraphExec_t ex = nullptr;
      if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
        hit->ex = ex;
        hit->kernels = pool->launches - before;
      }
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (lrc) return lrc;
    if (!hit->ex) return fail(pool, MAP_ECUDA, "capture of the conduction substeps failed");
    CK(cudaGraphLaunch(hit->ex, pool->stream));
  }
  if (lrc) return lrc;
  pool->pushed[pool->cur] = false;       // the energy ghosts are stale now
  return MAP_OK;
}

// one conduction substep (fill, energy update, energy reflux) on the current buffer
static int conduction_substep(map_pool* pool, const map_params* p, int it, bool rf) {
  {
    int rc = it == 0 ? fill_on(pool, pool->cur) : fill_energy_on(pool, pool->cur);
    if (rc) return rc;
    CondLaunch C;
    C.u = pool->buf[pool->cur];
    C.blocks = pool->dt.all_leaves;
    C.nblocks = pool->tree.nleaves;
    C.geo = pool->dt.geo;
    C.gamma = p->gamma;
    C.tau = fix_tau(pool, p);
    C.kappa0 = p->kappa0;
    C.grad_t_max = p->grad_t_max;
    C.mode = p->conduction;
    C.hsub = pool->hsub;
    C.nsub = pool->nsub;
    C.it = it;
    C.freg = rf ? pool->dt.freg : nullptr;
    C.refl = rf ? pool->dt.refl : nullptr;
    CK(DISPATCH(pool, conduction, C));
    if (rf) {
      RefluxLaunch R;
      R.u = pool->buf[pool->cur];
      R.tasks = pool->dt.rtasks;
      R.ntasks = pool->dt.nrtasks;
      R.freg = pool->dt.freg;
      R.geo = pool->dt.geo;
      R.dyn = pool->dyn;
      R.pushes = pool->dt.pushes;
      R.gamma = p->gamma;
      R.tau = C.tau;
      R.err_word = pool->err_word;
      R.sums = nullptr;
      R.dyn_next = nullptr;
      R.v0 = kEN;
      R.v1 = kEN + 1;
      R.hsub = pool->hsub;
      R.nsub = pool->nsub;
      R.it = it;
      CK(DISPATCH(pool, reflux, R));
    }
  }
  return MAP_OK;
}

int map_step(map_pool* pool, const map_params* p) {
  if (!pool) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  if (!pool->have_dt && !(p->dt_override > 0.0)) return fail(pool, MAP_ESTATE, "no time step: call map_cfl_dt first");
  rc = check_partial(pool, p);
  if (rc) return rc;
  if (p->dt_override > 0.0 && !pool->have_dt) {
    rc = cfl_device(pool, p);
    if (rc) return rc;
  }
  rc = step_launches(pool, p, false);
  if (rc == MAP_OK && p->conduction) rc = conduction_launches(pool, p);
  pool->have_dt = false;
  pool->alpha_ready = false;
  pool->sums_valid = false;
  return rc;
}

// one full step on the current buffer: ghost fill, dt from the alpha_g that the previous
// fused step (or the initial reduction) left in dyn, update with the alpha_g of the new
// state and the conservation sums reduced in the same kernel
static int advance_once(map_pool* pool, const map_params* p) {
  int rc = fill_on(pool, pool->cur);
  if (rc) return rc;
  CK(launch_finalize(make_finalize(pool, p), pool->stream, &pool->launches));
  return step_launches(pool, p, true);
}

int map_advance(map_pool* pool, const map_params* p, int nsteps) {
  if (!pool) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  if (pool->partial)
    return fail(pool, MAP_ESTATE, "a partitioned pool steps with map_step, between the exchanges of its halo leaves");
  if (nsteps <= 0) return MAP_OK;
  if (p->conduction) {
    // the substep count depends on dt: each step runs eagerly (fill, dt, update, conduction)
    for (int s = 0; s < nsteps; ++s) {
      rc = fill_on(pool, pool->cur);
      if (rc) return rc;
      rc = cfl_device(pool, p);
      if (rc) return rc;
      rc = step_launches(pool, p, false);
      if (rc) return rc;
      rc = conduction_launches(pool, p);
      if (rc) return rc;
    }
    pool->have_dt = false;
    pool->alpha_ready = false;
    pool->sums_valid = false;
    return MAP_OK;
  }
  if (!params_equal(pool->graph_params, *p)) {
    drop_graphs(pool);
    pool->graph_params = *p;
  }
  if (!pool->alpha_ready) {
    rc = alpha_device(pool, p);
    if (rc) return rc;
    pool->alpha_ready = true;
  }
  for (int s = 0; s < nsteps; ++s) {
    const int q = pool->cur;
    const int gi = 2 * q + (pool->pushed[q] ? 1 : 0);
    if (!pool->graph_valid[gi]) {
      // first step from this buffer: run eagerly (this also sets kernel attributes), then
      // capture the same sequence starting from buffer q for later replays
      rc = advance_once(pool, p);
      if (rc) return rc;
      const int after = pool->cur;
      const long long before = pool->launches;
      pool->cur = q;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(pool->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        rc = advance_once(pool, p);
        cudaError_t ce = cudaStreamEndCapture(pool->stream, &g);
        if (rc == MAP_OK && ce == cudaSuccess && g) {
          size_t nnodes = 0;
          cudaGraphGetNodes(g, nullptr, &nnodes);
          cudaGraphExec_t ex = nullptr;
          if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
            pool->graph[gi] = ex;
            pool->graph_valid[gi] = true;
            pool->graph_kernels[gi] = pool->launches - before;
            (void)nnodes;
          }
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
      }
      pool->cur = after;
      pool->launches = before;
      if (rc) return rc;
      continue;
    }
    CK(cudaGraphLaunch(pool->graph[gi], pool->stream));
    pool->launches += pool->graph_kernels[gi];
    pool->cur = 1 - q;
    pool->pushed[1 - q] = true;
  }
  pool->have_dt = false;
  pool->sums_valid = true;
  return MAP_OK;
}

int map_check(map_pool* pool) {
  if (!pool) return MAP_EINVAL;
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, pool->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaMemsetAsync(pool->err_word, 0, sizeof(unsigned), pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  // the asynchronous host copies are complete too once map_check returns
  if (pool->copy_stream) CK(cudaStreamSynchronize(pool->copy_stream));
  if (pool->rcopy_stream) CK(cudaStreamSynchronize(pool->rcopy_stream));
  if (e & 4u) return fail(pool, MAP_ETIMEOUT, "a bounded device wait for a plane copy gave up");
  if (e & 1u) return fail(pool, MAP_ENONFINITE, "a leaf cell became non-finite");
  if (e & 2u) return fail(pool, MAP_ENEGPRES, "a leaf cell has rho <= 0 or p < 0");
  return MAP_OK;
}

int map_flag_refine(map_pool* pool, const map_params* p, const map_refine_params* r, int8_t* flags_out,
                    double* est_out) {
  if (!pool || !p || !r || !flags_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  FlagLaunch F;
  F.u = pool->buf[pool->cur];
  F.blocks = pool->dt.leaf_ids;
  F.nblocks = pool->tree.nleaves;
  F.geo = pool->dt.geo;
  F.gamma = p->gamma;
  F.tau = fix_tau(pool, p);
  F.r = *r;
  F.flags = pool->flags;
  F.est = pool->est;
  for (int L = 0; L < 16; ++L) F.level_factor[L] = pow(r->ratio, r->xi * (double)(L + 1 - 1));
  CK(DISPATCH(pool, flags, F));
  CK(cudaMemcpyAsync(flags_out, pool->flags, pool->tree.nleaves, cudaMemcpyDeviceToHost, pool->stream));
  if (est_out)
    CK(cudaMemcpyAsync(est_out, pool->est, pool->tree.nleaves * sizeof(double), cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  return MAP_OK;
}

int map_regrid(map_pool* pool, const map_block_desc* leaves, int n) {
  if (!pool || !leaves || n <= 0) return fail(pool, MAP_EINVAL, "null or empty leaf list");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  HostTree& t = pool->spare;
  std::string why = build_tree(pool->ndim, pool->nb, pool->probs, leaves, n, t);
  if (!why.empty()) return fail(pool, MAP_EINVAL, why);
  if (t.nblocks > pool->max_blocks) return fail(pool, MAP_ENOMEM, "tree has more blocks than max_blocks");
  std::vector<RegridTask> tasks;
  why = build_regrid(pool->tree, t, tasks);
  if (!why.empty()) return fail(pool, MAP_EINVAL, why);
  if ((int)tasks.size() > pool->tasks_cap) {
    cudaFree(pool->tasks);
    pool->tasks = nullptr;
    CK(cudaMalloc(&pool->tasks, tasks.size() * sizeof(RegridTask)));
    pool->tasks_cap = (int)tasks.size();
  }
  CK(cudaMemcpyAsync(pool->tasks, tasks.data(), tasks.size() * sizeof(RegridTask), cudaMemcpyHostToDevice, pool->stream));
  RegridLaunch R;
  R.u_old = pool->buf[pool->cur];
  R.u_new = pool->buf[1 - pool->cur];
  R.tasks = pool->tasks;
  R.ntasks = (int)tasks.size();
  CK(DISPATCH(pool, regrid, R));
  CK(cudaStreamSynchronize(pool->stream));
  pool->cur = 1 - pool->cur;
  return install_tree(pool, t);   // also clears alpha_ready and the pushed-ghost flags
}

int map_plan_regrid(map_pool* pool, const int8_t* flags, int max_level, map_block_desc* out, int cap,
                    int* n_out) {
  if (!pool || !flags || !n_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  std::vector<map_block_desc> plan;
  std::string why = plan_regrid(pool->tree, pool->probs, flags, max_level, plan);
  if (!why.empty()) return fail(pool, MAP_EINVAL, why);
  *n_out = (int)plan.size();
  if ((int)plan.size() > cap || !out) return fail(pool, MAP_ENOMEM, "output array too small for the new leaf list");
  memcpy(out, plan.data(), plan.size() * sizeof(map_block_desc));
  return MAP_OK;
}

int map_get_leaves(map_pool* pool, map_block_desc* out, int cap, int* n_out) {
  if (!pool || !n_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const HostTree& t = pool->tree;
  *n_out = t.nleaves;
  if (t.nleaves > cap || !out) return fail(pool, MAP_ENOMEM, "output array too small");
  for (int l = 0; l < t.nleaves; ++l) {
    const int id = t.leaf_to_block[l];
    out[l].problem = t.blk_problem[id];
    out[l].level = t.blk_level[id];
    for (int d = 0; d < 3; ++d) out[l].ijk[d] = t.blk_ijk[3 * id + d];
  }
  return MAP_OK;
}

int map_adapt(map_pool* pool, const map_params* p, const map_refine_params* r, int* n_out) {
  if (!pool || !p || !r || !n_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  int rc = fill_on(pool, pool->cur);
  if (rc) return rc;
  std::vector<int8_t> flags(pool->tree.nleaves);
  rc = map_flag_refine(pool, p, r, flags.data(), nullptr);
  if (rc) return rc;
  std::vector<map_block_desc> plan;
  std::string why = plan_regrid(pool->tree, pool->probs, flags.data(), r->max_level, plan);
  if (!why.empty()) return fail(pool, MAP_EINVAL, why);
  bool same = (int)plan.size() == pool->tree.nleaves;
  for (int l = 0; same && l < pool->tree.nleaves; ++l) {
    const int id = pool->tree.leaf_to_block[l];
    same = plan[l].level == pool->tree.blk_level[id] && plan[l].problem == pool->tree.blk_problem[id] &&
           plan[l].ijk[0] == pool->tree.blk_ijk[3 * id] && plan[l].ijk[1] == pool->tree.blk_ijk[3 * id + 1] &&
           plan[l].ijk[2] == pool->tree.blk_ijk[3 * id + 2];
  }
  *n_out = (int)plan.size();
  if (same) return MAP_OK;                       // nothing to do: tree, tables and graphs stay
  return map_regrid(pool, plan.data(), (int)plan.size());
}

int map_conservation(map_pool* pool, double* sums_out) {
  if (!pool || !sums_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  CK(cudaMemsetAsync(pool->sums, 0, sizeof(double) * kNV * pool->nprob, pool->stream));
  SumLaunch L;
  L.u = pool->buf[pool->cur];
  L.blocks = pool->partial ? pool->dt.act_all : pool->dt.all_leaves;
  L.nblocks = pool->partial ? pool->dt.n_act : pool->tree.nleaves;
  L.geo = pool->dt.geo;
  L.sums = pool->sums;
  if (L.nblocks > 0) CK(DISPATCH(pool, sums, L));
  CK(cudaMemcpyAsync(sums_out, pool->sums, sizeof(double) * kNV * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  pool->sums_valid = true;
  return MAP_OK;
}

int map_test_fail_waits(map_pool* pool, int on) {
  if (!pool) return MAP_EINVAL;
  pool->fail_waits = on == 2 ? 2 : (on ? 1 : 0);
  drop_graphs(pool);
  return MAP_OK;
}

int map_set_conduction_loop(map_pool* pool, int on) {
  if (!pool) return MAP_EINVAL;
  pool->cond_loop = on ? 1 : 0;
  return MAP_OK;
}

int map_set_launch(map_pool* pool, int grid, int w_pred, int w_face) {
  if (!pool) return MAP_EINVAL;
  if (grid < 0 || w_pred < 0 || w_face < 0 || w_pred > 64 || w_face > 64)
    return fail(pool, MAP_EINVAL, "grid, w_pred and w_face must be >= 0 (weights <= 64)");
  pool->tune_grid = grid;
  pool->tune_wp = w_pred;
  pool->tune_wf = w_face;
  drop_graphs(pool);
  return MAP_OK;
}

// Times the step launches (scheme update with its fused reductions, WENO's mid-step fill,
// reflux) from the current buffer under candidate launch shapes and keeps the fastest: first
// the grid (the default, one CTA per block, or k = 1, 2, 3, 4, 6, 8, 12, 16 times the SM count
// as a persistent grid, below the block count) with the
// default weights, then the warp-schedule weights with that grid.  The trials write only the
// other buffers; ghosts are refilled and dt recomputed first, and the step constants and sums
// are restored afterwards, so the state and what later calls see are unchanged.
int map_autotune(map_pool* pool, const map_params* p, int reps, map_tune_result* out) {
  if (!pool || !out) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  if (reps < 1) reps = 1;
  const int np = pool->nprob;
  std::vector<ProbDyn> dyn0(np);
  std::vector<double> sums0((size_t)kNV * np);
  CK(cudaMemcpyAsync(dyn0.data(), pool->dyn, sizeof(ProbDyn) * np, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaMemcpyAsync(sums0.data(), pool->sums, sizeof(double) * kNV * np, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  rc = fill_on(pool, pool->cur);
  if (rc) return rc;
  rc = cfl_device(pool, p);
  if (rc) return rc;
  const int cur0 = pool->cur;
  const bool pushed0[3] = {pool->pushed[0], pool->pushed[1], pool->pushed[2]};
  const int g0 = pool->tune_grid, wp0 = pool->tune_wp, wf0 = pool->tune_wf;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int trials = 0;
  auto trial = [&](int grid, int wp, int wf, float* ms) -> int {
    pool->tune_grid = grid;
    pool->tune_wp = wp;
    pool->tune_wf = wf;
    for (int r = 0; r <= reps; ++r) {
      if (r == 1) CK(cudaEventRecord(e0, pool->stream));
      int rc2 = step_launches(pool, p, true);
      pool->cur = cur0;
      for (int q = 0; q < 3; ++q) pool->pushed[q] = pushed0[q];
      if (rc2) return rc2;
    }
    CK(cudaEventRecord(e1, pool->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= (float)reps;
    ++trials;
    return MAP_OK;
  };
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  float best = 0.f, t = 0.f;
  int dwp = 1, dwf = 1;
  default_schedule_weights(pool->ndim, pool->nb, p->scheme, &dwp, &dwf);
  int bg = 0, bwp = dwp, bwf = dwf;
  rc = trial(0, dwp, dwf, &best);
  const float base = best;
  if (rc == MAP_OK && step_grid(pool) > 0) {
    // the default is persistent here: try one CTA per block as well
    rc = trial(pool->tree.nleaves, dwp, dwf, &t);
    if (rc == MAP_OK && t < best) { best = t; bg = pool->tree.nleaves; }
  }
  const int K[] = {1, 2, 3, 4, 6, 8, 12, 16};
  for (int k : K) {
    if (rc) break;
    const int grid = k * nsm;
    if (grid >= pool->tree.nleaves) break;
    rc = trial(grid, dwp, dwf, &t);
    if (rc == MAP_OK && t < best) { best = t; bg = grid; }
  }
  // weight ratios from 1:1 to 6:1 (only the ratio shapes the schedule); the default's is skipped
  const int W[][2] = {{1, 1}, {5, 4}, {3, 2}, {2, 1}, {9, 4}, {3, 1}, {4, 1}, {6, 1}};
  for (const auto& wgt : W) {
    if (rc) break;
    if (wgt[0] * dwf == wgt[1] * dwp) continue;
    rc = trial(bg, wgt[0], wgt[1], &t);
    if (rc == MAP_OK && t < best) { best = t; bwp = wgt[0]; bwf = wgt[1]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pool->cur = cur0;
  for (int q = 0; q < 3; ++q) pool->pushed[q] = pushed0[q];
  CK(cudaMemcpyAsync(pool->dyn, dyn0.data(), sizeof(ProbDyn) * np, cudaMemcpyHostToDevice, pool->stream));
  CK(cudaMemcpyAsync(pool->sums, sums0.data(), sizeof(double) * kNV * np, cudaMemcpyHostToDevice, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  if (rc) {
    pool->tune_grid = g0;
    pool->tune_wp = wp0;
    pool->tune_wf = wf0;
    return rc;
  }
  pool->tune_grid = bg;
  pool->tune_wp = bwp;
  pool->tune_wf = bwf;
  drop_graphs(pool);
  out->grid = bg;
  out->w_pred = bwp;
  out->w_face = bwf;
  out->ms_default = base;
  out->ms_best = best;
  out->trials = trials;
  return MAP_OK;
}

int map_last_conduction(map_pool* pool, double* dtc_out, int* nsub_out) {
  if (!pool || !dtc_out || !nsub_out) return fail(pool, MAP_EINVAL, "null argument");
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  for (int q = 0; q < pool->nprob; ++q) {
    dtc_out[q] = dyn[q].dtc;
    nsub_out[q] = q < (int)pool->nsub_h.size() ? pool->nsub_h[q] : 0;
  }
  return MAP_OK;
}

int map_last_sums(map_pool* pool, double* sums_out) {
  if (!pool || !sums_out) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->sums_valid) return fail(pool, MAP_ESTATE, "the state changed since the last map_advance step");
  CK(cudaMemcpyAsync(sums_out, pool->sums, sizeof(double) * kNV * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  return MAP_OK;
}

int map_get_speeds_async(map_pool* pool, double* out) {
  if (!pool || !out) return fail(pool, MAP_EINVAL, "null argument");
  static_assert(offsetof(ProbDyn, dt) == 0 && offsetof(ProbDyn, ch) == 8 && offsetof(ProbDyn, cp) == 16 &&
                offsetof(ProbDyn, damp) == 24 && offsetof(ProbDyn, alpha_g) == 32,
                "dt, c_h, c_p, damping, alpha_g lead ProbDyn");
  // page-locked host memory mapped into the device's address space: a one-warp kernel stores
  // the values there.  A small device-to-host copy on the pool stream would instead wait
  // behind a large state copy running on the copy engine of that direction (an overlapped
  // map_read_leaves_async), and hold the next step's launches back with it.
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, out) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
    CK(launch_speeds_out(pool->dyn, pool->nprob, (double*)a.devicePointer, pool->stream, &pool->launches));
    return MAP_OK;
  }
  cudaGetLastError();   // an unregistered pointer is not an error
  CK(cudaMemcpy2DAsync(out, 5 * sizeof(double), pool->dyn, sizeof(ProbDyn), 5 * sizeof(double), pool->nprob,
                       cudaMemcpyDeviceToHost, pool->stream));
  return MAP_OK;
}

int map_get_speeds(map_pool* pool, double* out) {
  if (!pool || !out) return fail(pool, MAP_EINVAL, "null argument");
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  for (int q = 0; q < pool->nprob; ++q) {
    out[5 * q + 0] = dyn[q].dt;
    out[5 * q + 1] = dyn[q].ch;
    out[5 * q + 2] = dyn[q].cp;
    out[5 * q + 3] = dyn[q].damp;
    out[5 * q + 4] = dyn[q].alpha_g;
  }
  return MAP_OK;
}

static void put_msg(char* msg, int cap, const std::string& why) {
  if (!msg || cap <= 0) return;
  const size_t k = why.size() < (size_t)(cap - 1) ? why.size() : (size_t)(cap - 1);
  memcpy(msg, why.data(), k);
  msg[k] = 0;
}

static std::string host_tree(int ndim, int nb, const map_problem_desc* problems, int np,
                             const map_block_desc* leaves, int n, HostTree& t, std::vector<map_problem_desc>& probs) {
  if (ndim != 2 && ndim != 3) return "ndim must be 2 or 3";
  if (nb != 8 && nb != 16) return "nb must be 8 or 16";
  if (!problems || np <= 0) return "no problems";
  if (!leaves || n <= 0) return "null or empty leaf list";
  probs.assign(problems, problems + np);
  return build_tree(ndim, nb, probs, leaves, n, t);
}

int map_check_leaves(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                     const map_block_desc* leaves, int n, char* msg, int msg_cap) {
  HostTree t;
  std::vector<map_problem_desc> probs;
  const std::string why = host_tree(ndim, nb, problems, n_problems, leaves, n, t, probs);
  put_msg(msg, msg_cap, why);
  return why.empty() ? MAP_OK : MAP_EINVAL;
}

int map_plan_leaves(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                    const map_block_desc* leaves, int n, const int8_t* flags, int max_level,
                    map_block_desc* out, int cap, int* n_out, char* msg, int msg_cap) {
  if (!flags || !n_out) {
    put_msg(msg, msg_cap, "null argument");
    return MAP_EINVAL;
  }
  HostTree t;
  std::vector<map_problem_desc> probs;
  std::string why = host_tree(ndim, nb, problems, n_problems, leaves, n, t, probs);
  std::vector<map_block_desc> plan;
  if (why.empty()) why = plan_regrid(t, probs, flags, max_level, plan);
  if (!why.empty()) {
    put_msg(msg, msg_cap, why);
    return MAP_EINVAL;
  }
  *n_out = (int)plan.size();
  if ((int)plan.size() > cap || !out) {
    put_msg(msg, msg_cap, "output array too small for the new leaf list");
    return MAP_ENOMEM;
  }
  memcpy(out, plan.data(), plan.size() * sizeof(map_block_desc));
  put_msg(msg, msg_cap, "");
  return MAP_OK;
}

// ---- partition over processes (Sec. 4.2 load balance; Sec. 4.3 inter-processor boundaries)

int map_plan_partition(int ndim, int nb, const map_problem_desc* problems, int n_problems,
                       const map_block_desc* leaves, int n, int nranks, int* owner_out,
                       unsigned char* need_out, char* msg, int msg_cap) {
  if (!owner_out || !need_out || nranks < 1) {
    put_msg(msg, msg_cap, "null argument or nranks < 1");
    return MAP_EINVAL;
  }
  HostTree t;
  std::vector<map_problem_desc> probs;
  const std::string why = host_tree(ndim, nb, problems, n_problems, leaves, n, t, probs);
  if (!why.empty()) {
    put_msg(msg, msg_cap, why);
    return MAP_EINVAL;
  }
  std::vector<int> owner;
  std::vector<unsigned char> need;
  plan_partition(t, nranks, owner, need);
  memcpy(owner_out, owner.data(), owner.size() * sizeof(int));
  memcpy(need_out, need.data(), need.size());
  put_msg(msg, msg_cap, "");
  return MAP_OK;
}

int map_set_active(map_pool* pool, const int* leaves, int n) {
  if (!pool) return MAP_EINVAL;
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const HostTree& t = pool->tree;
  DevTree& D = pool->dt;
  cudaFree(D.act_all);
  cudaFree(D.act_level);
  D.act_all = D.act_level = nullptr;
  D.n_act = 0;
  D.chunk_grid = 0;
  pool->partial = false;
  drop_graphs(pool);
  pool->have_dt = false;
  pool->alpha_ready = false;
  pool->sums_valid = false;
  if (!leaves || n < 0) return MAP_OK;
  std::vector<char> on(t.nleaves, 0);
  for (int q = 0; q < n; ++q) {
    if (leaves[q] < 0 || leaves[q] >= t.nleaves) return fail(pool, MAP_EINVAL, "active leaf index out of range");
    if (on[leaves[q]]) return fail(pool, MAP_EINVAL, "active leaf listed twice");
    on[leaves[q]] = 1;
  }
  std::vector<int> all, lev;
  for (int blk : t.all_leaves)
    if (on[t.geo[blk].leaf]) all.push_back(blk);
  D.act_off.assign(t.maxlev + 2, 0);
  for (int L = 0; L <= t.maxlev; ++L) {
    D.act_off[L] = (int)lev.size();
    for (int blk : t.leaves_by_level[L])
      if (on[t.geo[blk].leaf]) lev.push_back(blk);
  }
  D.act_off[t.maxlev + 1] = (int)lev.size();
  if (!all.empty()) {
    CK(upload(&D.act_all, all, pool->stream));
    CK(upload(&D.act_level, lev, pool->stream));
  }
  CK(cudaStreamSynchronize(pool->stream));
  D.n_act = (int)all.size();
  pool->partial = true;
  return MAP_OK;
}

static int transfer_leaves(map_pool* pool, const int* leaves, int n, void* dev_buf, int to_pool) {
  if (!pool || (n > 0 && (!leaves || !dev_buf)) || n < 0) return fail(pool, MAP_EINVAL, "null argument");
  if (!pool->have_tree) return fail(pool, MAP_ESTATE, "no tree");
  const HostTree& t = pool->tree;
  if (n > t.nleaves) return fail(pool, MAP_EINVAL, "more leaves than the tree has");
  if (n == 0) return MAP_OK;
  std::vector<int> ids(n);
  for (int q = 0; q < n; ++q) {
    if (leaves[q] < 0 || leaves[q] >= t.nleaves) return fail(pool, MAP_EINVAL, "leaf index out of range");
    ids[q] = t.leaf_to_block[leaves[q]];
  }
  DevTree& D = pool->dt;
  if (!D.xfer_ids) CK(cudaMalloc(&D.xfer_ids, (size_t)t.nleaves * sizeof(int)));
  // stream-ordered behind the previous transfer's kernel, which read the same id array
  CK(cudaMemcpyAsync(D.xfer_ids, ids.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));   // the host id array goes out of scope
  if (to_pool) {
    pool->have_dt = false;
    pool->alpha_ready = false;
    pool->pushed[pool->cur] = false;
    pool->sums_valid = false;
  }
  return pack(pool, D.xfer_ids, n, to_pool, (double*)dev_buf, is64(pool) ? 0 : 1);
}

int map_pack_leaves(map_pool* pool, const int* leaves, int n, void* dev_buf) {
  return transfer_leaves(pool, leaves, n, dev_buf, 0);
}

int map_unpack_leaves(map_pool* pool, const int* leaves, int n, const void* dev_buf) {
  return transfer_leaves(pool, leaves, n, const_cast<void*>(dev_buf), 1);
}

int map_local_alpha(map_pool* pool, const map_params* p, double* alpha_out) {
  if (!pool || !alpha_out) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  rc = alpha_device(pool, p);
  if (rc) return rc;
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  for (int q = 0; q < pool->nprob; ++q) {
    const unsigned long long b = dyn[q].alpha_bits;
    double a;
    memcpy(&a, &b, sizeof a);
    alpha_out[q] = a;
  }
  pool->alpha_ready = false;
  return MAP_OK;
}

int map_set_alpha(map_pool* pool, const map_params* p, const double* alpha) {
  if (!pool || !alpha) return MAP_EINVAL;
  int rc = check_params(pool, p);
  if (rc) return rc;
  for (int q = 0; q < pool->nprob; ++q)
    if (!(alpha[q] >= 0.0)) return fail(pool, MAP_EINVAL, "alpha_g must be >= 0 (and not NaN)");
  static_assert(sizeof(unsigned long long) == sizeof(double), "alpha bits");
  CK(cudaMemcpy2DAsync((char*)pool->dyn + offsetof(ProbDyn, alpha_bits), sizeof(ProbDyn), alpha, sizeof(double),
                       sizeof(double), pool->nprob, cudaMemcpyHostToDevice, pool->stream));
  CK(launch_finalize(make_finalize(pool, p), pool->stream, &pool->launches));
  std::vector<ProbDyn> dyn(pool->nprob);
  CK(cudaMemcpyAsync(dyn.data(), pool->dyn, sizeof(ProbDyn) * pool->nprob, cudaMemcpyDeviceToHost, pool->stream));
  CK(cudaStreamSynchronize(pool->stream));
  pool->have_dt = true;
  pool->alpha_ready = false;
  for (int q = 0; q < pool->nprob; ++q)
    if (!(isfinite(dyn[q].dt) && dyn[q].dt > 0.0))
      return fail(pool, MAP_ENONFINITE, "time step is not finite and positive (non-finite or zero signal speed)");
  return MAP_OK;
}

long long map_kernel_launches(const map_pool* pool) { return pool ? pool->launches : 0; }

const char* map_last_error(const map_pool* pool) {
  return pool ? pool->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
