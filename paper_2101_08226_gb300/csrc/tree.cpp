// Host-side tree construction for the CUDA solver.
//
// Subgrid sets are kept as hash sets of packed positions per level and refinement is propagated
// with a work list: refining a subgrid makes its flagged children refine in turn, and every
// refined subgrid at level l >= 1 demands that each of its 26 in-domain neighbours exists, i.e.
// that the neighbour's parent is refined (proper nesting, Sec. 2.4).  The result is the least
// refined tree that contains every flagged subgrid that exists and is properly nested.
#include "tree.hpp"

#include <algorithm>
#include <cmath>
#include <deque>
#include <unordered_map>
#include <unordered_set>

namespace octofmm {

namespace {

inline uint64_t pos_key(int64_t i, int64_t j, int64_t k) {
  return (uint64_t(i) << 42) | (uint64_t(j) << 21) | uint64_t(k);
}
inline void pos_unkey(uint64_t p, int64_t& i, int64_t& j, int64_t& k) {
  i = int64_t(p >> 42);
  j = int64_t((p >> 21) & ((1u << 21) - 1));
  k = int64_t(p & ((1u << 21) - 1));
}
// Morton interleave: x bit above y bit above z bit in each triple.
inline uint64_t morton(int lev, int64_t i, int64_t j, int64_t k) {
  uint64_t m = 0;
  for (int b = lev - 1; b >= 0; --b)
    m = (m << 3) | (uint64_t((i >> b) & 1) << 2) | (uint64_t((j >> b) & 1) << 1) |
        uint64_t((k >> b) & 1);
  return m;
}

}  // namespace

bool well_separated(int dx, int dy, int dz, double theta) {
  int d2 = dx * dx + dy * dy + dz * dz;
  if (d2 == 0) return false;
  return 1.0 / std::sqrt(double(d2)) < theta;
}

std::string build_host_tree(int max_level, const uint8_t* flags, int64_t n_flags, HostTree& t) {
  if (max_level < 0 || max_level > kMaxLevel) return "max_level out of range";
  std::vector<int64_t> foff(max_level + 1, 0);
  for (int l = 1; l <= max_level; ++l) foff[l] = foff[l - 1] + (int64_t(1) << (3 * (l - 1)));
  if (n_flags != foff[max_level]) return "n_flags does not match max_level";
  if (n_flags > 0 && !flags) return "refine_flags is null";

  auto flagged = [&](int l, int64_t i, int64_t j, int64_t k) -> bool {
    if (l >= max_level) return false;
    int64_t n = int64_t(1) << l;
    return flags[foff[l] + (i * n + j) * n + k] != 0;
  };

  std::vector<std::unordered_set<uint64_t>> refined(max_level + 1);
  std::deque<std::pair<int, uint64_t>> work;
  // Refine (l, p): its parent must be refined for it to exist; flagged children follow.
  struct Refiner {
    std::vector<std::unordered_set<uint64_t>>& refined;
    std::deque<std::pair<int, uint64_t>>& work;
    decltype(flagged)& is_flagged;
    int max_level;
    void operator()(int l, uint64_t p) {
      if (l >= max_level || refined[l].count(p)) return;
      int64_t i, j, k;
      pos_unkey(p, i, j, k);
      if (l > 0) (*this)(l - 1, pos_key(i / 2, j / 2, k / 2));
      if (!refined[l].insert(p).second) return;
      work.emplace_back(l, p);
      for (int o = 0; o < 8; ++o) {
        int64_t a = 2 * i + ((o >> 2) & 1), b = 2 * j + ((o >> 1) & 1), c = 2 * k + (o & 1);
        if (is_flagged(l + 1, a, b, c)) (*this)(l + 1, pos_key(a, b, c));
      }
    }
  } refine{refined, work, flagged, max_level};

  if (flagged(0, 0, 0, 0)) refine(0, pos_key(0, 0, 0));
  while (!work.empty()) {
    auto [l, p] = work.front();
    work.pop_front();
    if (l == 0) continue;
    int64_t i, j, k, n = int64_t(1) << l;
    pos_unkey(p, i, j, k);
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int64_t a = i + dx, b = j + dy, c = k + dz;
          if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) continue;
          refine(l - 1, pos_key(a / 2, b / 2, c / 2));
        }
  }

  // Existing subgrids per level: the root, and the children of refined subgrids.
  struct Node { uint64_t key; int64_t i, j, k; };
  std::vector<std::vector<Node>> levels;
  levels.push_back({Node{0, 0, 0, 0}});
  for (int l = 0; l < max_level && !refined[l].empty(); ++l) {
    std::vector<Node> next;
    next.reserve(refined[l].size() * 8);
    for (uint64_t p : refined[l]) {
      int64_t i, j, k;
      pos_unkey(p, i, j, k);
      for (int o = 0; o < 8; ++o) {
        int64_t a = 2 * i + ((o >> 2) & 1), b = 2 * j + ((o >> 1) & 1), c = 2 * k + (o & 1);
        next.push_back(Node{morton(l + 1, a, b, c), a, b, c});
      }
    }
    levels.push_back(std::move(next));
  }
  t = HostTree();
  t.depth = int(levels.size()) - 1;
  t.lev_off.assign(t.depth + 2, 0);
  for (int l = 0; l <= t.depth; ++l) {
    std::sort(levels[l].begin(), levels[l].end(),
              [](const Node& x, const Node& y) { return x.key < y.key; });
    t.lev_off[l + 1] = t.lev_off[l] + int64_t(levels[l].size());
  }
  t.n_sub = t.lev_off[t.depth + 1];
  t.level.resize(t.n_sub);
  t.ijk.resize(3 * t.n_sub);
  t.leaf.resize(t.n_sub);
  t.parent.assign(t.n_sub, -1);
  t.child.assign(8 * t.n_sub, -1);
  t.nbr.assign(27 * t.n_sub, -1);
  t.leaf_ord.assign(t.n_sub, -1);
  t.refined_at.assign(t.depth + 1, {});
  t.leaves_at.assign(t.depth + 1, {});
  std::vector<std::unordered_map<uint64_t, int32_t>> index(t.depth + 1);
  for (int l = 0; l <= t.depth; ++l) {
    index[l].reserve(levels[l].size() * 2);
    for (size_t q = 0; q < levels[l].size(); ++q) {
      const Node& nd = levels[l][q];
      int32_t s = int32_t(t.lev_off[l] + int64_t(q));
      t.level[s] = l;
      t.ijk[3 * s] = int32_t(nd.i);
      t.ijk[3 * s + 1] = int32_t(nd.j);
      t.ijk[3 * s + 2] = int32_t(nd.k);
      bool is_ref = l < max_level && refined[l].count(pos_key(nd.i, nd.j, nd.k));
      t.leaf[s] = is_ref ? 0 : 1;
      index[l][pos_key(nd.i, nd.j, nd.k)] = s;
    }
  }
  for (int l = 0; l <= t.depth; ++l) {
    int64_t n = int64_t(1) << l;
    for (int64_t s = t.lev_off[l]; s < t.lev_off[l + 1]; ++s) {
      int64_t i = t.ijk[3 * s], j = t.ijk[3 * s + 1], k = t.ijk[3 * s + 2];
      if (l > 0) {
        auto it = index[l - 1].find(pos_key(i / 2, j / 2, k / 2));
        if (it == index[l - 1].end()) return "internal: parent missing";
        t.parent[s] = it->second;
        int o = int((i & 1) << 2 | (j & 1) << 1 | (k & 1));
        t.child[8 * it->second + o] = int32_t(s);
      }
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            int64_t a = i + dx, b = j + dy, c = k + dz;
            if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) continue;
            auto it = index[l].find(pos_key(a, b, c));
            if (it != index[l].end()) t.nbr[27 * s + (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)] = it->second;
          }
      if (t.leaf[s]) {
        t.leaf_ord[s] = int32_t(t.leaf_sub.size());
        t.leaf_sub.push_back(int32_t(s));
        t.leaves_at[l].push_back(int32_t(s));
      } else {
        t.refined_at[l].push_back(int32_t(s));
        for (int o = 0; o < 8; ++o)
          if (!index[l + 1].count(pos_key(2 * i + ((o >> 2) & 1), 2 * j + ((o >> 1) & 1),
                                          2 * k + (o & 1))))
            return "internal: child missing";
        for (int slot = 0; slot < 27; ++slot)
          if (slot != 13) {
            int dx = slot / 9 - 1, dy = (slot / 3) % 3 - 1, dz = slot % 3 - 1;
            int64_t a = i + dx, b = j + dy, c = k + dz;
            if (a >= 0 && b >= 0 && c >= 0 && a < n && b < n && c < n && t.nbr[27 * s + slot] < 0)
              return "internal: nesting violated";
          }
      }
    }
  }
  t.n_leaf_sub = int64_t(t.leaf_sub.size());
  t.n_trees = 1;
  t.tree_leaf_off = {0, t.n_leaf_sub};
  return "";
}

std::string merge_trees(const std::vector<const HostTree*>& parts, HostTree& out) {
  if (parts.empty()) return "no trees";
  HostTree f;
  f.depth = 0;
  f.n_trees = 0;
  for (const HostTree* p : parts) {
    f.depth = std::max(f.depth, p->depth);
    f.n_trees += p->n_trees;
  }
  // new index of every part's subgrids: level-major, part order within a level
  std::vector<std::vector<int32_t>> remap(parts.size());
  f.lev_off.assign(f.depth + 2, 0);
  int64_t next = 0;
  for (int l = 0; l <= f.depth; ++l) {
    f.lev_off[l] = next;
    for (size_t q = 0; q < parts.size(); ++q) {
      const HostTree* p = parts[q];
      if (remap[q].empty()) remap[q].assign(p->n_sub, -1);
      if (l > p->depth) continue;
      for (int64_t s = p->lev_off[l]; s < p->lev_off[l + 1]; ++s) remap[q][s] = int32_t(next++);
    }
  }
  f.lev_off[f.depth + 1] = next;
  f.n_sub = next;
  if (f.n_sub >= (int64_t(1) << 27)) return "forest too large";
  f.level.assign(f.n_sub, 0);
  f.ijk.assign(3 * f.n_sub, 0);
  f.leaf.assign(f.n_sub, 0);
  f.parent.assign(f.n_sub, -1);
  f.child.assign(8 * f.n_sub, -1);
  f.nbr.assign(27 * f.n_sub, -1);
  f.leaf_ord.assign(f.n_sub, -1);
  f.refined_at.assign(f.depth + 1, {});
  f.leaves_at.assign(f.depth + 1, {});
  auto map = [](const std::vector<int32_t>& m, int32_t s) { return s < 0 ? -1 : m[s]; };
  for (size_t q = 0; q < parts.size(); ++q) {
    const HostTree* p = parts[q];
    for (int64_t s = 0; s < p->n_sub; ++s) {
      int32_t n = remap[q][s];
      f.level[n] = p->level[s];
      for (int k = 0; k < 3; ++k) f.ijk[3 * n + k] = p->ijk[3 * s + k];
      f.leaf[n] = p->leaf[s];
      f.parent[n] = map(remap[q], p->parent[s]);
      for (int k = 0; k < 8; ++k) f.child[8 * n + k] = map(remap[q], p->child[8 * s + k]);
      for (int k = 0; k < 27; ++k) f.nbr[27 * n + k] = map(remap[q], p->nbr[27 * s + k]);
    }
  }
  // leaves tree-major, each part's leaves in its own order
  f.tree_leaf_off.assign(1, 0);
  for (size_t q = 0; q < parts.size(); ++q) {
    const HostTree* p = parts[q];
    for (int k = 0; k < p->n_trees; ++k) {
      for (int64_t o = p->tree_leaf_off[k]; o < p->tree_leaf_off[k + 1]; ++o) {
        int32_t n = remap[q][p->leaf_sub[o]];
        f.leaf_ord[n] = int32_t(f.leaf_sub.size());
        f.leaf_sub.push_back(n);
      }
      f.tree_leaf_off.push_back(int64_t(f.leaf_sub.size()));
    }
  }
  f.n_leaf_sub = int64_t(f.leaf_sub.size());
  for (int64_t s = 0; s < f.n_sub; ++s) {
    if (f.leaf[s]) f.leaves_at[f.level[s]].push_back(int32_t(s));
    else f.refined_at[f.level[s]].push_back(int32_t(s));
  }
  out = std::move(f);
  return "";
}

Stencil make_stencil(double theta) {
  Stencil st;
  st.theta = theta;
  for (int par = 0; par < 8; ++par) {
    int a[3] = {(par >> 2) & 1, (par >> 1) & 1, par & 1};
    for (int dx = -kMaxReach; dx <= kMaxReach; ++dx)
      for (int dy = -kMaxReach; dy <= kMaxReach; ++dy)
        for (int dz = -kMaxReach; dz <= kMaxReach; ++dz) {
          if (!well_separated(dx, dy, dz, theta)) continue;
          // parents' offset: floor((a + d) / 2) - floor(a / 2), with a in {0, 1}
          int px = (a[0] + dx) >> 1, py = (a[1] + dy) >> 1, pz = (a[2] + dz) >> 1;
          if (well_separated(px, py, pz, theta)) continue;
          st.offs[par].push_back(pack_offset(dx, dy, dz));
        }
  }
  for (int dx = -2; dx <= 2; ++dx)
    for (int dy = -2; dy <= 2; ++dy)
      for (int dz = -2; dz <= 2; ++dz)
        if ((dx || dy || dz) && !well_separated(dx, dy, dz, theta))
          st.near.push_back(pack_offset(dx, dy, dz));
  return st;
}

void interaction_counts_by_type(const HostTree& t, const Stencil& st, int64_t out[6]) {
  // Per neighbour slot: how many (target cell, offset) pairs of one subgrid land in that slot.
  int64_t m2l_slot[27] = {0}, near_slot[27] = {0};
  for (int c = 0; c < kCells; ++c) {
    int a = c / 64, b = (c / 8) % 8, z = c % 8;
    int par = (a & 1) << 2 | (b & 1) << 1 | (z & 1);
    auto add = [&](const std::vector<int32_t>& list, int64_t* slots) {
      for (int32_t code : list) {
        int dx, dy, dz;
        unpack_offset(code, dx, dy, dz);
        int sx = ((a + dx) >> 3) + 1, sy = ((b + dy) >> 3) + 1, sz = ((z + dz) >> 3) + 1;
        slots[sx * 9 + sy * 3 + sz]++;
      }
    };
    add(st.offs[par], m2l_slot);
    add(st.near, near_slot);
  }
  int64_t root_ws = 0, root_near = 0;
  for (int c = 0; c < kCells; ++c)
    for (int e = 0; e < kCells; ++e) {
      if (c == e) continue;
      if (well_separated(c / 64 - e / 64, (c / 8) % 8 - (e / 8) % 8, c % 8 - e % 8, st.theta))
        root_ws++;
      else
        root_near++;
    }
  for (int k = 0; k < 6; ++k) out[k] = 0;
  for (int64_t s = 0; s < t.lev_off[1]; ++s) {  // the roots: every well-separated pair
    if (t.leaf[s]) {
      out[0] += root_ws;
      out[4] += root_near;
    } else {
      out[3] += root_ws;
    }
  }
  for (int64_t s = t.lev_off[1]; s < t.n_sub; ++s)
    for (int slot = 0; slot < 27; ++slot) {
      int32_t nb = t.nbr[27 * s + slot];
      if (nb < 0) continue;
      out[(t.leaf[s] ? 0 : 2) + (t.leaf[nb] ? 0 : 1)] += m2l_slot[slot];
      if (t.leaf[s]) {
        if (t.leaf[nb]) out[4] += near_slot[slot];
        else out[5] += 16 * near_slot[slot];  // i <- 8 children and 8 children <- i
      }
    }
}

void interaction_counts(const HostTree& t, const Stencil& st, int64_t out[3]) {
  int64_t c[6];
  interaction_counts_by_type(t, st, c);
  out[0] = c[0] + c[1] + c[2] + c[3];
  out[1] = c[4];
  out[2] = c[5];
}

}  // namespace octofmm

namespace octofmm {

// Spatial decomposition of one tree (the multi-node runs of Sec. 5 split one tree over nodes).
// Units in Morton order at the cut level: every subgrid of the cut level (with its whole
// subtree) and every leaf subgrid coarser than the cut (a leaf at level l < c stands at the cut
// level's key of its first corner, (i, j, k) << (c - l)).  The ordered units are split into
// n_ranks contiguous runs of about equal leaf-cell count; a subgrid finer than the cut belongs to
// the rank of its cut-level ancestor.  Refined subgrids coarser than the cut are every rank's
// (owner -1): each rank forms their moments from its share of the leaves, the shares are summed
// over the ranks, and each rank evaluates their interactions itself.
std::string partition_tree(const HostTree& t, int n_ranks, int cut, std::vector<int32_t>& owner) {
  if (t.n_trees != 1) return "the decomposition takes a single tree";
  if (n_ranks < 1) return "n_ranks must be >= 1";
  if (cut < 0 || cut > t.depth) return "cut level outside the tree";
  owner.assign(size_t(t.n_sub), -1);
  struct Unit {
    uint64_t key;
    int32_t s;
    int64_t weight;
  };
  std::vector<Unit> units;
  std::vector<int64_t> leaves_below(size_t(t.n_sub), 0);
  for (int l = t.depth; l >= 0; --l)
    for (int64_t s = t.lev_off[l]; s < t.lev_off[l + 1]; ++s) {
      if (t.leaf[s]) {
        leaves_below[s] = 1;
      } else {
        for (int o = 0; o < 8; ++o) leaves_below[s] += leaves_below[t.child[8 * s + o]];
      }
    }
  for (int l = 0; l <= cut; ++l)
    for (int64_t s = t.lev_off[l]; s < t.lev_off[l + 1]; ++s) {
      if (l < cut && !t.leaf[s]) continue;
      const int sh = cut - l;
      units.push_back(Unit{morton(cut, int64_t(t.ijk[3 * s]) << sh, int64_t(t.ijk[3 * s + 1]) << sh,
                                  int64_t(t.ijk[3 * s + 2]) << sh),
                           int32_t(s), leaves_below[s] * kCells});
    }
  std::stable_sort(units.begin(), units.end(), [](const Unit& a, const Unit& b) { return a.key < b.key; });
  int64_t total = 0;
  for (const Unit& u : units) total += u.weight;
  // rank r takes the units whose cumulative weight midpoint falls in [r, r + 1) total / n_ranks
  int64_t acc = 0;
  std::vector<int32_t> unit_rank(units.size());
  for (size_t k = 0; k < units.size(); ++k) {
    const double mid = double(acc) + 0.5 * double(units[k].weight);
    int r = int(mid * n_ranks / double(total > 0 ? total : 1));
    unit_rank[k] = std::min(r, n_ranks - 1);
    acc += units[k].weight;
  }
  for (size_t k = 0; k < units.size(); ++k) owner[size_t(units[k].s)] = unit_rank[k];
  for (int l = cut + 1; l <= t.depth; ++l)
    for (int64_t s = t.lev_off[l]; s < t.lev_off[l + 1]; ++s) owner[s] = owner[size_t(t.parent[s])];
  return "";
}

// The subgrids whose data rank `rank` reads but another rank owns (ghosts): for every subgrid the
// rank owns or shares (owner -1), its 26 same-level neighbours (multipole partners lie within one
// subgrid for theta >= 0.34); for every leaf it owns, also the leaf children of its refined
// neighbours (direct partners across the level jump) and the leaf neighbours of each of its
// ancestors (direct partners at coarser levels).  A leaf ghost is read as its densities, a refined
// ghost as its cells' moments.  Sorted, without repeats.
std::string ghost_subgrids(const HostTree& t, const std::vector<int32_t>& owner, int rank,
                           std::vector<int32_t>& out) {
  if (owner.size() != size_t(t.n_sub)) return "owner array of the wrong size";
  std::vector<uint8_t> need(size_t(t.n_sub), 0);
  auto mark = [&](int32_t q) {
    if (q >= 0 && owner[size_t(q)] >= 0 && owner[size_t(q)] != rank) need[size_t(q)] = 1;
  };
  for (int64_t s = 0; s < t.n_sub; ++s) {
    const int32_t o = owner[size_t(s)];
    if (o != rank && o != -1) continue;
    for (int k = 0; k < 27; ++k) mark(t.nbr[27 * s + k]);
    if (o != rank || !t.leaf[s]) continue;
    for (int k = 0; k < 27; ++k) {
      const int32_t q = t.nbr[27 * s + k];
      if (q < 0 || t.leaf[q]) continue;
      for (int c = 0; c < 8; ++c)
        if (t.leaf[t.child[8 * q + c]]) mark(t.child[8 * q + c]);
    }
    for (int32_t a = t.parent[s]; a >= 0; a = t.parent[a])
      for (int k = 0; k < 27; ++k) {
        const int32_t q = t.nbr[27 * a + k];
        if (q >= 0 && t.leaf[q]) mark(q);
      }
  }
  out.clear();
  for (int64_t s = 0; s < t.n_sub; ++s)
    if (need[size_t(s)]) out.push_back(int32_t(s));
  return "";
}

}  // namespace octofmm
