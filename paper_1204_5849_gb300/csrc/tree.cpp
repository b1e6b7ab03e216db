// tree.cpp -- host-side block tree: Morton ordering, validation, ghost-fill and regrid
// tables (Sec. 4.1 hierarchical structure; Sec. 4.3 boundary conditions).
//
// The paper keeps a replicated linked list of blocks in Hilbert order with parent/child/
// neighbour pointers (Table 1).  Here the tree lives on the host as flat arrays indexed by
// pool block id: leaves first in Morton order (problem, then interleaved coordinates at the
// finest level), then parents.  For each leaf the 3^ndim ghost regions are resolved once
// into a source block and an affine index map, so the device fill is a pure gather.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "map_internal.hpp"

namespace mapgb {

namespace {

unsigned long long pack_key(int p, int L, int i, int j, int k) {
  return ((unsigned long long)p << 50) | ((unsigned long long)L << 45) |
         ((unsigned long long)k << 30) | ((unsigned long long)j << 15) | (unsigned long long)i;
}

unsigned long long spread3(unsigned long long x) {
  // bit q of x -> bit 3q
  unsigned long long r = 0;
  for (int q = 0; q < 21; ++q) r |= ((x >> q) & 1ull) << (3 * q);
  return r;
}

unsigned long long morton(int ndim, int i, int j, int k) {
  if (ndim == 2) {
    unsigned long long r = 0;
    for (int q = 0; q < 31; ++q) {
      r |= ((unsigned long long)((i >> q) & 1) << (2 * q));
      r |= ((unsigned long long)((j >> q) & 1) << (2 * q + 1));
    }
    return r;
  }
  return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2);
}

struct Node {
  int p, L, ijk[3];
  bool leaf;
  int caller;  // caller leaf index
};

std::string fmt(const char* what, int p, int L, const int* ijk) {
  char buf[160];
  snprintf(buf, sizeof buf, "%s: problem %d level %d block (%d,%d,%d)", what, p, L, ijk[0], ijk[1], ijk[2]);
  return buf;
}

// Runs body(id) for id in [0, n): on up to 16 host threads when n is large, each over a
// contiguous range in increasing id.  body only reads the tree and writes slots of its own
// id.  Returns the message of the lowest id whose body failed (what a serial loop returns
// first), else an empty string.
template <typename F>
std::string for_each_leaf(int n, const F& body) {
  auto serial = [&](int lo, int hi, int* at) -> std::string {
    for (int id = lo; id < hi; ++id) {
      std::string e = body(id);
      if (!e.empty()) {
        *at = id;
        return e;
      }
    }
    return std::string();
  };
  int nt = 1;
  if (n >= 2048) {
    const unsigned hw = std::thread::hardware_concurrency();
    nt = std::min(std::min((int)(hw ? hw : 1u), 16), n / 512);
  }
  int at = INT_MAX;
  if (nt <= 1) return serial(0, n, &at);
  std::vector<std::string> err(nt);
  std::vector<int> err_at(nt, INT_MAX);
  std::vector<std::thread> th;
  bool spawned = true;
  try {
    for (int k = 1; k < nt; ++k)
      th.emplace_back([&, k] {
        err[k] = serial((int)((long long)n * k / nt), (int)((long long)n * (k + 1) / nt), &err_at[k]);
      });
  } catch (...) {
    spawned = false;
  }
  if (spawned) err[0] = serial(0, (int)((long long)n / nt), &err_at[0]);
  for (auto& x : th) x.join();
  if (!spawned) return serial(0, n, &at);     // no threads to be had: the plain loop
  for (int k = 0; k < nt; ++k)
    if (!err[k].empty()) return err[k];      // ranges ascend with k
  return std::string();
}

}  // namespace

namespace {
constexpr unsigned long long kEmpty = ~0ull;   // no packed key reaches all ones (p <= 4000)

// SplitMix64's output mix, as the hash of a packed key
unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}
}  // namespace

void HostTree::reset() {
  ndim = nb = nblocks = nleaves = maxlev = nslots = 0;
  hmask = 0;
  for (auto* v : {&leaf_to_block, &blk_problem, &blk_level, &blk_ijk, &children, &all_leaves, &leaves_per_problem,
                  &hvals})
    v->clear();
  geo.clear();
  regions.clear();
  pushes.clear();
  level_has_residual.clear();
  refl.clear();
  reflux_tasks.clear();
  leaves_by_level.clear();
  parents_by_level.clear();
  residual_by_level.clear();
  mindx.clear();
  keys.clear();
  hkeys.clear();
}

void HostTree::build_index() {
  size_t cap = 16;
  while (cap < 2 * keys.size()) cap <<= 1;
  hkeys.assign(cap, kEmpty);
  hvals.assign(cap, -1);
  hmask = cap - 1;
  for (const auto& kv : keys) {
    unsigned long long h = mix64(kv.first) & hmask;
    while (hkeys[h] != kEmpty) h = (h + 1) & hmask;
    hkeys[h] = kv.first;
    hvals[h] = kv.second;
  }
}

int HostTree::find(int p, int L, int i, int j, int k) const {
  if (i < 0 || j < 0 || k < 0 || i >= (1 << 15) || j >= (1 << 15) || k >= (1 << 15)) return -1;
  const unsigned long long key = pack_key(p, L, i, j, k);
  if (hkeys.empty()) {
    auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(key, -1));
    return (it != keys.end() && it->first == key) ? it->second : -1;
  }
  unsigned long long h = mix64(key) & hmask;
  while (hkeys[h] != kEmpty) {
    if (hkeys[h] == key) return hvals[h];
    h = (h + 1) & hmask;
  }
  return -1;
}

std::string build_tree(int ndim, int nb, const std::vector<map_problem_desc>& probs,
                       const map_block_desc* leaves, int n, HostTree& t) {
  t.reset();
  t.ndim = ndim;
  t.nb = nb;
  const int np = (int)probs.size();
  if (n <= 0) return "empty leaf list";
  if (np > 4000) return "too many problems";
  for (int p = 0; p < np; ++p)
    for (int d = 0; d < 3; ++d) {
      if (d < ndim && (probs[p].nbase[d] < 1 || !(probs[p].hi[d] > probs[p].lo[d])))
        return "bad problem box";
      if (d < ndim && (probs[p].bc[d][0] < 0 || probs[p].bc[d][0] > 1 || probs[p].bc[d][1] < 0 ||
                       probs[p].bc[d][1] > 1))
        return "bad boundary kind";
      if (d < ndim && ((probs[p].bc[d][0] == MAP_BC_PERIODIC) != (probs[p].bc[d][1] == MAP_BC_PERIODIC)))
        return "periodic boundaries must pair";
    }

  std::vector<Node> nodes;
  std::vector<std::pair<unsigned long long, int>> keys;
  nodes.reserve((size_t)n * 2);
  for (int l = 0; l < n; ++l) {
    Node nd;
    nd.p = leaves[l].problem;
    nd.L = leaves[l].level;
    for (int d = 0; d < 3; ++d) nd.ijk[d] = d < ndim ? leaves[l].ijk[d] : 0;
    nd.leaf = true;
    nd.caller = l;
    if (nd.p < 0 || nd.p >= np || nd.L < 0 || nd.L > 12) return fmt("bad leaf", nd.p, nd.L, nd.ijk);
    for (int d = 0; d < ndim; ++d) {
      int nblk = probs[nd.p].nbase[d] << nd.L;
      if (nd.ijk[d] < 0 || nd.ijk[d] >= nblk || nblk > (1 << 15)) return fmt("leaf out of range", nd.p, nd.L, nd.ijk);
    }
    if (nd.L > t.maxlev) t.maxlev = nd.L;
    keys.push_back({pack_key(nd.p, nd.L, nd.ijk[0], nd.ijk[1], nd.ijk[2]), (int)nodes.size()});
    nodes.push_back(nd);
  }
  std::sort(keys.begin(), keys.end());
  for (size_t q = 1; q < keys.size(); ++q)
    if (keys[q].first == keys[q - 1].first) return fmt("duplicate leaf", nodes[keys[q].second].p,
                                                       nodes[keys[q].second].L, nodes[keys[q].second].ijk);
  // ancestors
  std::vector<std::pair<unsigned long long, int>> anc;
  for (int l = 0; l < n; ++l) {
    Node c = nodes[l];
    while (c.L > 0) {
      c.L -= 1;
      for (int d = 0; d < 3; ++d) c.ijk[d] >>= 1;
      anc.push_back({pack_key(c.p, c.L, c.ijk[0], c.ijk[1], c.ijk[2]), l});
    }
  }
  std::sort(anc.begin(), anc.end());
  for (size_t q = 0; q < anc.size(); ++q) {
    if (q > 0 && anc[q].first == anc[q - 1].first) continue;
    auto it = std::lower_bound(keys.begin(), keys.end(), std::make_pair(anc[q].first, -1));
    if (it != keys.end() && it->first == anc[q].first) {
      const Node& lf = nodes[it->second];
      return fmt("leaf contains another leaf", lf.p, lf.L, lf.ijk);
    }
    Node c;
    unsigned long long k = anc[q].first;
    c.p = (int)(k >> 50);
    c.L = (int)((k >> 45) & 31);
    c.ijk[2] = (int)((k >> 30) & 32767);
    c.ijk[1] = (int)((k >> 15) & 32767);
    c.ijk[0] = (int)(k & 32767);
    c.leaf = false;
    c.caller = -1;
    nodes.push_back(c);
  }
  // pool order: leaves by (problem, Morton at the finest level), then parents by level
  std::vector<int> order(nodes.size());
  for (size_t q = 0; q < nodes.size(); ++q) order[q] = (int)q;
  const int ML = t.maxlev;
  std::vector<unsigned long long> mk(nodes.size());      // Morton key at the finest level
  for (size_t q = 0; q < nodes.size(); ++q) {
    const Node& a = nodes[q];
    const int s = ML - a.L;
    mk[q] = morton(ndim, a.ijk[0] << s, a.ijk[1] << s, a.ijk[2] << s);
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const Node& a = nodes[x];
    const Node& b = nodes[y];
    if (a.leaf != b.leaf) return a.leaf;
    if (a.p != b.p) return a.p < b.p;
    if (!a.leaf && a.L != b.L) return a.L > b.L;
    if (mk[x] != mk[y]) return mk[x] < mk[y];
    return a.L < b.L;
  });
  const int NB = (int)nodes.size();
  t.nblocks = NB;
  t.nleaves = n;
  t.leaf_to_block.assign(n, -1);
  t.geo.resize(NB);
  t.blk_problem.resize(NB);
  t.blk_level.resize(NB);
  t.blk_ijk.resize((size_t)NB * 3);
  t.children.assign((size_t)NB * 8, -1);
  t.keys.clear();
  t.keys.reserve(NB);
  for (int id = 0; id < NB; ++id) {
    const Node& a = nodes[order[id]];
    t.blk_problem[id] = a.p;
    t.blk_level[id] = a.L;
    for (int d = 0; d < 3; ++d) t.blk_ijk[3 * id + d] = a.ijk[d];
    BlockGeo g;
    for (int d = 0; d < 3; ++d) {
      int ncell = d < ndim ? (probs[a.p].nbase[d] << a.L) * nb : 1;
      g.dx[d] = (probs[a.p].hi[d] - probs[a.p].lo[d]) / (double)ncell;
    }
    g.problem = a.p;
    g.level = a.L;
    g.leaf = a.leaf ? a.caller : -1;
    g.pad = 0;
    t.geo[id] = g;
    if (a.leaf) t.leaf_to_block[a.caller] = id;
    t.keys.push_back({pack_key(a.p, a.L, a.ijk[0], a.ijk[1], a.ijk[2]), id});
  }
  std::sort(t.keys.begin(), t.keys.end());
  t.build_index();
  // parent/child links and completeness
  for (int id = 0; id < NB; ++id) {
    int L = t.blk_level[id];
    if (L == 0) continue;
    const int* c = &t.blk_ijk[3 * id];
    int par = t.find(t.blk_problem[id], L - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1);
    if (par < 0) return "internal error: missing parent";
    int cb = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
    t.children[(size_t)par * 8 + cb] = id;
  }
  for (int id = n; id < NB; ++id)
    for (int cb = 0; cb < (1 << ndim); ++cb)
      if (t.children[(size_t)id * 8 + cb] < 0)
        return fmt("incomplete parent (a child is missing)", t.blk_problem[id], t.blk_level[id], &t.blk_ijk[3 * id]);
  for (int p = 0; p < np; ++p) {
    int nz = ndim == 3 ? probs[p].nbase[2] : 1;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < probs[p].nbase[1]; ++j)
        for (int i = 0; i < probs[p].nbase[0]; ++i)
          if (t.find(p, 0, i, j, k) < 0) {
            int ijk[3] = {i, j, k};
            return fmt("domain not covered", p, 0, ijk);
          }
  }
  // 2:1 balance over faces, edges and corners
  std::string err = for_each_leaf(n, [&](int id) -> std::string {
    int p = t.blk_problem[id], L = t.blk_level[id];
    const int* c = &t.blk_ijk[3 * id];
    for (int oz = (ndim == 3 ? -1 : 0); oz <= (ndim == 3 ? 1 : 0); ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (!ox && !oy && !oz) continue;
          int off[3] = {ox, oy, oz}, q[3] = {0, 0, 0};
          bool outside = false;
          for (int d = 0; d < ndim; ++d) {
            int nblk = probs[p].nbase[d] << L;
            q[d] = c[d] + off[d];
            if (q[d] < 0 || q[d] >= nblk) {
              if (probs[p].bc[d][q[d] < 0 ? 0 : 1] == MAP_BC_PERIODIC) q[d] = (q[d] + nblk) % nblk;
              else outside = true;
            }
          }
          if (outside) continue;
          int nbid = t.find(p, L, q[0], q[1], q[2]);
          if (nbid >= 0) {
            if (nbid < n) continue;
            for (int cb = 0; cb < (1 << ndim); ++cb) {
              bool touch = true;
              for (int d = 0; d < ndim; ++d) {
                int bit = (cb >> d) & 1;
                if (off[d] == 1 && bit != 0) touch = false;
                if (off[d] == -1 && bit != 1) touch = false;
              }
              if (touch && t.children[(size_t)nbid * 8 + cb] >= n)
                return fmt("2:1 balance violated (finer by two levels)", p, L, c);
            }
          } else {
            int cq = L > 0 ? t.find(p, L - 1, q[0] >> 1, q[1] >> 1, q[2] >> 1) : -1;
            if (cq < 0 || cq >= n) return fmt("2:1 balance violated (coarser by two levels)", p, L, c);
          }
        }
    return std::string();
  });
  if (!err.empty()) return err;
  // ghost regions of every leaf
  t.regions.assign((size_t)NB * 27, GhostRegion{});
  err = for_each_leaf(n, [&](int id) -> std::string {
    int p = t.blk_problem[id], L = t.blk_level[id];
    const int* c = &t.blk_ijk[3 * id];
    for (int rz = 0; rz < 3; ++rz)
      for (int ry = 0; ry < 3; ++ry)
        for (int rx = 0; rx < 3; ++rx) {
          if (ndim == 2 && rz != 1) continue;
          int r[3] = {rx, ry, rz};
          int m[3] = {1, 1, 1}, A[3] = {0, 0, 0}, T[3] = {0, 0, 0}, rep[3] = {0, 0, 0};
          for (int d = 0; d < ndim; ++d) {
            int N = (probs[p].nbase[d] << L) * nb;
            int nblk = probs[p].nbase[d] << L;
            int O = c[d] * nb;
            int irep = r[d] == 0 ? 0 : (r[d] == 1 ? kNG : kNG + nb);
            if (r[d] == 1) {
              m[d] = 1; A[d] = O - kNG; T[d] = c[d];
            } else {
              int nbk = c[d] + (r[d] == 0 ? -1 : 1);
              if (nbk >= 0 && nbk < nblk) {
                m[d] = 1; A[d] = O - kNG; T[d] = nbk;
              } else if (probs[p].bc[d][r[d] == 0 ? 0 : 1] == MAP_BC_PERIODIC) {
                m[d] = 1; A[d] = O - kNG + (r[d] == 0 ? N : -N); T[d] = (nbk + nblk) % nblk;
              } else {
                m[d] = 0; A[d] = r[d] == 0 ? 0 : N - 1; T[d] = c[d];
              }
            }
            rep[d] = m[d] * irep + A[d];
          }
          GhostRegion g{};
          int src = t.find(p, L, T[0], T[1], T[2]);
          if (src >= 0) {
            g.kind = 0;
            g.src = src;
            for (int d = 0; d < 3; ++d) {
              g.m[d] = d < ndim ? m[d] : 1;
              g.a[d] = d < ndim ? A[d] - T[d] * nb + kNG : 0;
              g.corg[d] = 0;
            }
          } else {
            int Tc[3] = {0, 0, 0};
            for (int d = 0; d < ndim; ++d) Tc[d] = (rep[d] >> 1) / nb;
            int cs = L > 0 ? t.find(p, L - 1, Tc[0], Tc[1], Tc[2]) : -1;
            if (cs < 0 || cs >= n) return fmt("no coarse source for a ghost region", p, L, c);
            g.kind = 1;
            g.src = cs;
            for (int d = 0; d < 3; ++d) {
              g.m[d] = d < ndim ? m[d] : 1;
              g.a[d] = d < ndim ? A[d] : 0;
              g.corg[d] = d < ndim ? Tc[d] * nb : 0;
            }
          }
          t.regions[(size_t)id * 27 + rx + 3 * ry + 9 * rz] = g;
        }
    return std::string();
  });
  if (!err.empty()) return err;
  // pushes: a same-level leaf copy with an affine map in every dimension is written by the
  // source block's step kernel into the destination's ghost region
  // For a fixed region, the same-level neighbour is a translation (with periodic wrap), a
  // bijection: each (source, direction) slot belongs to one (destination, region), so the
  // leaves fill their slots independently, on host threads.
  t.pushes.assign((size_t)NB * 27, PushEntry{-1, {0, 0, 0}});
  t.level_has_residual.assign(t.maxlev + 1, 0);
  t.residual_by_level.assign(t.maxlev + 1, {});
  std::vector<char> has_residual(n, 0);
  err = for_each_leaf(n, [&](int id) -> std::string {
    bool residual = false;
    for (int rz = 0; rz < 3; ++rz)
      for (int ry = 0; ry < 3; ++ry)
        for (int rx = 0; rx < 3; ++rx) {
          if (ndim == 2 && rz != 1) continue;
          if (rx == 1 && ry == 1 && rz == 1) continue;
          GhostRegion& g = t.regions[(size_t)id * 27 + rx + 3 * ry + 9 * rz];
          g.pushed = 0;
          bool affine = true;
          for (int d = 0; d < ndim; ++d) affine = affine && g.m[d] == 1;
          if (g.kind == 0 && affine && g.src < n && t.blk_level[g.src] == t.blk_level[id]) {
            // seen from the source, this block lies in direction -(r - 1)
            const int dir = (1 - (rx - 1)) + 3 * (1 - (ry - 1)) + 9 * (ndim == 3 ? 1 - (rz - 1) : 1);
            PushEntry& pe = t.pushes[(size_t)g.src * 27 + dir];
            if (pe.dst >= 0) return fmt("internal error: two ghost regions push from one slot", t.blk_problem[id],
                                        t.blk_level[id], &t.blk_ijk[3 * id]);
            pe.dst = id;
            for (int d = 0; d < 3; ++d) pe.off[d] = d < ndim ? -g.a[d] : 0;
            g.pushed = 1;
          }
          if (!g.pushed) residual = true;
        }
    has_residual[id] = residual ? 1 : 0;
    return std::string();
  });
  if (!err.empty()) return err;
  for (int id = 0; id < n; ++id)
    if (has_residual[id]) {
      t.level_has_residual[t.blk_level[id]] = 1;
      t.residual_by_level[t.blk_level[id]].push_back(id);
    }
  // reflux: the coarse leaf of every coarse/fine face gets a task naming the fine leaves
  // covering that face; both sides get a face-register slot
  t.refl.assign((size_t)NB, RefluxLeaf{-1, 0});
  t.reflux_tasks.clear();
  {
    std::vector<char> need(n, 0);
    for (int id = 0; id < n; ++id) {
      const int p = t.blk_problem[id], L = t.blk_level[id];
      const int* c = &t.blk_ijk[3 * id];
      RefluxTask tk;
      tk.coarse = id;
      tk.cslot = -1;
      for (int s6 = 0; s6 < 6; ++s6)
        for (int k = 0; k < 4; ++k) tk.fslot[s6][k] = -1;
      bool coarse_side = false;
      for (int d = 0; d < ndim; ++d)
        for (int side = 0; side < 2; ++side) {
          int q[3] = {c[0], c[1], c[2]};
          const int nblk = probs[p].nbase[d] << L;
          q[d] += side ? 1 : -1;
          if (q[d] < 0 || q[d] >= nblk) {
            if (probs[p].bc[d][side] != MAP_BC_PERIODIC) continue;
            q[d] = (q[d] + nblk) % nblk;
          }
          const int nbid = t.find(p, L, q[0], q[1], q[2]);
          if (nbid >= n) {                        // refined neighbour: this leaf is coarse
            coarse_side = true;
            t.refl[id].coarse_mask |= 1 << (2 * d + side);
            const int da = d == 0 ? 1 : 0, db = d == 2 ? 1 : 2;
            for (int k = 0; k < (1 << (ndim - 1)); ++k) {
              int bits[3] = {0, 0, 0};
              bits[d] = side ? 0 : 1;
              bits[da] = k & 1;
              if (ndim == 3) bits[db] = (k >> 1) & 1;
              const int ch = t.children[(size_t)nbid * 8 + (bits[0] | (bits[1] << 1) | (bits[2] << 2))];
              if (ch < 0 || ch >= n) return fmt("coarse/fine face without fine leaves", p, L, c);
              tk.fslot[2 * d + side][k] = ch;     // pool id for now
              need[ch] = 1;
            }
          } else if (nbid < 0) {
            need[id] = 1;                         // coarser neighbour: this leaf is fine
          }
        }
      if (coarse_side) {
        need[id] = 1;
        t.reflux_tasks.push_back(tk);
      }
    }
    t.nslots = 0;
    for (int id = 0; id < n; ++id)
      if (need[id]) t.refl[id].slot = t.nslots++;
    for (RefluxTask& tk : t.reflux_tasks) {
      tk.cslot = t.refl[tk.coarse].slot;
      for (int s6 = 0; s6 < 6; ++s6)
        for (int k = 0; k < 4; ++k)
          if (tk.fslot[s6][k] >= 0) tk.fslot[s6][k] = t.refl[tk.fslot[s6][k]].slot;
    }
  }
  // level lists, per-problem minimum spacing
  t.leaves_by_level.assign(t.maxlev + 1, {});
  t.parents_by_level.assign(t.maxlev + 1, {});
  t.all_leaves.resize(n);
  t.mindx.assign(np, 1e300);
  t.leaves_per_problem.assign(np, 0);
  for (int id = 0; id < NB; ++id) {
    int L = t.blk_level[id];
    if (id < n) {
      t.leaves_by_level[L].push_back(id);
      t.all_leaves[id] = id;
      int p = t.blk_problem[id];
      t.leaves_per_problem[p]++;
      for (int d = 0; d < ndim; ++d) t.mindx[p] = std::min(t.mindx[p], t.geo[id].dx[d]);
    } else {
      t.parents_by_level[L].push_back(id);
    }
  }
  for (int p = 0; p < np; ++p)
    if (t.leaves_per_problem[p] == 0) return "a problem has no leaves";
  return "";
}

std::string build_regrid(const HostTree& o, const HostTree& nw, std::vector<RegridTask>& tasks) {
  tasks.clear();
  for (int id = 0; id < nw.nleaves; ++id) {
    int p = nw.blk_problem[id], L = nw.blk_level[id];
    const int* c = &nw.blk_ijk[3 * id];
    RegridTask tk{};
    tk.dst = id;
    int same = o.find(p, L, c[0], c[1], c[2]);
    if (same >= 0) {
      tk.kind = 0;
      tk.src = same;
      tk.cb = 0;
    } else {
      int par = L > 0 ? o.find(p, L - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1) : -1;
      if (par < 0 || par >= o.nleaves)
        return fmt("regrid: a new leaf is neither old, nor a child of an old leaf", p, L, c);
      tk.kind = 1;
      tk.src = par;
      tk.cb = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
    }
    tasks.push_back(tk);
  }
  return "";
}

}  // namespace mapgb

namespace mapgb {

namespace {

// leaf index (pool id < nleaves) covering block (p, L, c) of the current tree: the block
// itself, or the leaf at a coarser level that contains it; -1 if the block region is
// refined below L (then no single leaf covers it) or outside the domain.
int covering_leaf(const HostTree& t, int p, int L, const int* c) {
  int ijk[3] = {c[0], c[1], c[2]};
  for (int l = L; l >= 0; --l) {
    const int id = t.find(p, l, ijk[0], ijk[1], ijk[2]);
    if (id >= 0) return id < t.nleaves ? id : -1;
    for (int d = 0; d < 3; ++d) ijk[d] >>= 1;
  }
  return -1;
}

// neighbour block coordinates of (p, L, c) in direction off, periodic wrap; false if the
// neighbour lies outside a non-periodic boundary
bool neighbour(const std::vector<map_problem_desc>& probs, int ndim, int p, int L, const int* c, const int* off,
               int* q) {
  for (int d = 0; d < 3; ++d) q[d] = c[d];
  for (int d = 0; d < ndim; ++d) {
    const int n = probs[p].nbase[d] << L;
    q[d] = c[d] + off[d];
    if (q[d] < 0 || q[d] >= n) {
      if (probs[p].bc[d][q[d] < 0 ? 0 : 1] != MAP_BC_PERIODIC) return false;
      q[d] = (q[d] + n) % n;
    }
  }
  return true;
}

template <typename F>
void for_each_offset(int ndim, F&& f) {
  for (int oz = (ndim == 3 ? -1 : 0); oz <= (ndim == 3 ? 1 : 0); ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        if (!ox && !oy && !oz) continue;
        const int off[3] = {ox, oy, oz};
        f(off);
      }
}

}  // namespace

// Regrid decision (Sec. 4.5): refine leaves flagged +1 (below max_level), refine further
// leaves until every new leaf's neighbours (faces, edges, corners) are at most one level
// coarser, and coarsen a parent whose children are all leaves flagged -1, none refined,
// when the coarsened parent keeps the 2:1 rule.  New leaves are listed in the order of the
// old leaves: a kept leaf in place, a refined leaf as its 2^ndim children (child bits
// x | y<<1 | z<<2 ascending), a coarsened parent at the place of its first child.
std::string plan_regrid(const HostTree& t, const std::vector<map_problem_desc>& probs, const int8_t* flags,
                        int max_level, std::vector<map_block_desc>& out) {
  const int n = t.nleaves, nd = t.ndim;
  out.clear();
  std::vector<char> refine(n, 0);
  std::vector<int> work;
  for (int l = 0; l < n; ++l) {
    const int id = t.leaf_to_block[l];
    if (flags[l] > 0 && t.blk_level[id] < max_level) {
      refine[id] = 1;
      work.push_back(id);
    }
  }
  // balance: children of a refined leaf at level L+1 need neighbours at level >= L
  while (!work.empty()) {
    const int id = work.back();
    work.pop_back();
    const int p = t.blk_problem[id], L = t.blk_level[id];
    const int* c = &t.blk_ijk[3 * id];
    for_each_offset(nd, [&](const int* off) {
      int q[3];
      if (!neighbour(probs, nd, p, L, c, off, q)) return;
      const int cov = covering_leaf(t, p, L, q);
      if (cov < 0 || refine[cov]) return;
      if (t.blk_level[cov] < L) {
        if (t.blk_level[cov] >= max_level) return;  // cannot happen in a balanced tree
        refine[cov] = 1;
        work.push_back(cov);
      }
    });
  }
  // coarsening candidates: parents whose children are all leaves flagged -1, none refined
  std::vector<char> coarsen(t.nblocks, 0);
  std::vector<int> flag_of(n, 0);
  for (int l = 0; l < n; ++l) flag_of[t.leaf_to_block[l]] = flags[l];
  for (int par = n; par < t.nblocks; ++par) {
    bool ok = true;
    for (int cb = 0; cb < (1 << nd) && ok; ++cb) {
      const int ch = t.children[(size_t)par * 8 + cb];
      if (ch < 0 || ch >= n || flag_of[ch] >= 0 || refine[ch]) ok = false;
    }
    if (ok) coarsen[par] = 1;
  }
  // a coarsened parent at level L-1 may not touch a block that stays refined below L or a
  // leaf at level L that is being refined; drop such candidates until none is left
  bool changed = true;
  while (changed) {
    changed = false;
    for (int par = n; par < t.nblocks; ++par) {
      if (!coarsen[par]) continue;
      const int p = t.blk_problem[par], L = t.blk_level[par] + 1;   // children level
      const int* c = &t.blk_ijk[3 * par];
      bool bad = false;
      for_each_offset(nd, [&](const int* off) {
        if (bad) return;
        int q[3];
        if (!neighbour(probs, nd, p, L - 1, c, off, q)) return;
        const int nb = t.find(p, L - 1, q[0], q[1], q[2]);
        if (nb < 0 || nb < n) return;                 // coarser or a leaf at L-1: fine
        // neighbour parent at L-1: its children touching us must end at level <= L
        if (coarsen[nb]) return;
        for (int cb = 0; cb < (1 << nd); ++cb) {
          bool touch = true;
          for (int d = 0; d < nd; ++d) {
            const int bit = (cb >> d) & 1;
            if (off[d] == 1 && bit != 0) touch = false;
            if (off[d] == -1 && bit != 1) touch = false;
          }
          if (!touch) continue;
          const int ch = t.children[(size_t)nb * 8 + cb];
          if (ch >= n || refine[ch]) bad = true;
        }
      });
      if (bad) {
        coarsen[par] = 0;
        changed = true;
      }
    }
  }
  std::vector<char> emitted(t.nblocks, 0);
  for (int l = 0; l < n; ++l) {
    const int id = t.leaf_to_block[l];
    const int p = t.blk_problem[id], L = t.blk_level[id];
    const int* c = &t.blk_ijk[3 * id];
    int par = -1;
    if (L > 0) par = t.find(p, L - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1);
    if (par >= 0 && coarsen[par]) {
      if (!emitted[par]) {
        emitted[par] = 1;
        map_block_desc b;
        b.problem = p;
        b.level = L - 1;
        for (int d = 0; d < 3; ++d) b.ijk[d] = t.blk_ijk[3 * par + d];
        out.push_back(b);
      }
    } else if (refine[id]) {
      for (int cb = 0; cb < (1 << nd); ++cb) {
        map_block_desc b;
        b.problem = p;
        b.level = L + 1;
        b.ijk[0] = 2 * c[0] + (cb & 1);
        b.ijk[1] = 2 * c[1] + ((cb >> 1) & 1);
        b.ijk[2] = nd == 3 ? 2 * c[2] + ((cb >> 2) & 1) : 0;
        out.push_back(b);
      }
    } else {
      map_block_desc b;
      b.problem = p;
      b.level = L;
      for (int d = 0; d < 3; ++d) b.ijk[d] = c[d];
      out.push_back(b);
    }
  }
  return "";
}

// ---------------------------------------------------------------------------------------
// Partition over ranks (Sec. 4.2 load balance): the leaves in Morton order are cut into
// nranks contiguous ranges of equal count (the first n % nranks ranges one longer).  A rank
// then needs, besides its own leaves, the interiors of every leaf its ghost fill reads: the
// dependency closure of the fill of its own leaves.
//   - a region copying from a leaf reads that leaf's cells; where the index map reaches its
//     ghost cells, that leaf's own regions are needed too;
//   - a region prolonging from a coarser leaf reads the coarse cell and its neighbours, which
//     may be ghosts: that leaf's regions are needed too;
//   - a region copying from a parent reads the restriction of all its leaf descendants.
namespace {

// does a copy region (rx, ry, rz) of a destination block read ghost cells of its source?
bool copy_reads_ghosts(const GhostRegion& g, int ndim, int nb, const int r[3]) {
  for (int d = 0; d < ndim; ++d) {
    const int lo = r[d] == 0 ? 0 : (r[d] == 1 ? kNG : kNG + nb);
    const int hi = r[d] == 0 ? kNG : (r[d] == 1 ? kNG + nb : nb + 2 * kNG);   // exclusive
    const int s0 = g.m[d] * lo + g.a[d], s1 = g.m[d] * (hi - 1) + g.a[d];
    const int smin = s0 < s1 ? s0 : s1, smax = s0 < s1 ? s1 : s0;
    if (smin < kNG || smax >= kNG + nb) return true;
  }
  return false;
}

void add_descendant_leaves(const HostTree& t, int blk, std::vector<unsigned char>& need_int) {
  if (t.geo[blk].leaf >= 0) {
    need_int[blk] = 1;
    return;
  }
  for (int q = 0; q < (t.ndim == 3 ? 8 : 4); ++q) {
    const int c = t.children[(size_t)blk * 8 + q];
    if (c >= 0) add_descendant_leaves(t, c, need_int);
  }
}

}  // namespace

void plan_partition(const HostTree& t, int nranks, std::vector<int>& owner, std::vector<unsigned char>& need) {
  const int n = t.nleaves;
  owner.assign(n, 0);
  need.assign((size_t)nranks * n, 0);
  // Morton order = pool ids 0..n-1 (t.all_leaves); caller index = geo[id].leaf
  std::vector<int> rank_of_block(t.nblocks, -1);
  for (int r = 0; r < nranks; ++r) {
    const long long b0 = (long long)n * r / nranks, b1 = (long long)n * (r + 1) / nranks;
    for (long long q = b0; q < b1; ++q) {
      const int blk = t.all_leaves[q];
      rank_of_block[blk] = r;
      owner[t.geo[blk].leaf] = r;
    }
  }
  std::vector<unsigned char> need_int(t.nblocks), need_gh(t.nblocks);
  std::vector<int> work;
  for (int r = 0; r < nranks; ++r) {
    std::fill(need_int.begin(), need_int.end(), 0);
    std::fill(need_gh.begin(), need_gh.end(), 0);
    work.clear();
    for (int q = 0; q < n; ++q) {
      const int blk = t.all_leaves[q];
      if (rank_of_block[blk] == r) {
        need_int[blk] = 1;
        need_gh[blk] = 1;
        work.push_back(blk);
      }
    }
    while (!work.empty()) {
      const int blk = work.back();
      work.pop_back();
      for (int id = 0; id < 27; ++id) {
        const int rr[3] = {id % 3, (id / 3) % 3, id / 9};
        if (id == 13 || (t.ndim == 2 && rr[2] != 1)) continue;
        const GhostRegion& g = t.regions[(size_t)blk * 27 + id];
        const int src = g.src;
        if (src < 0) continue;
        if (t.geo[src].leaf < 0) {
          add_descendant_leaves(t, src, need_int);
          continue;
        }
        need_int[src] = 1;
        const bool ghosts = g.kind == 1 || copy_reads_ghosts(g, t.ndim, t.nb, rr);
        if (ghosts && !need_gh[src]) {
          need_gh[src] = 1;
          work.push_back(src);
        }
      }
    }
    for (int blk = 0; blk < t.nblocks; ++blk)
      if (need_int[blk] && t.geo[blk].leaf >= 0) need[(size_t)r * n + t.geo[blk].leaf] = 1;
  }
}

}  // namespace mapgb
