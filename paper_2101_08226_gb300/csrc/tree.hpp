// Host-side octree of 8^3-cell subgrids for the CUDA solver: construction with proper nesting
// (Sec. 2.4), same-level stencils from the opening criterion (Sec. 2.2) and interaction counts.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#ifdef __CUDACC__
#define OCTO_HD __host__ __device__
#else
#define OCTO_HD
#endif

namespace octofmm {

constexpr int kSub = 8;        // cells per subgrid edge
constexpr int kCells = 512;    // cells per subgrid
constexpr int kMaxLevel = 9;   // deepest level accepted
constexpr int kMaxReach = 5;   // stencil reach in cells for theta >= 0.34
constexpr double kThetaMin = 0.34;

// A tree, or a forest of independent trees: subgrids are numbered level-major across the trees
// (tree order within a level), so the roots of the n_trees trees are subgrids 0 .. n_trees-1; leaf
// subgrids are ordered tree-major, each tree's in its own canonical (level, Morton) order.
struct HostTree {
  int depth = 0;                       // deepest level that has subgrids
  int n_trees = 1;
  std::vector<int64_t> tree_leaf_off;  // [n_trees + 1]: first leaf-subgrid ordinal of each tree
  int64_t n_sub = 0, n_leaf_sub = 0;
  std::vector<int64_t> lev_off;        // [depth + 2]: first global subgrid index of each level
  std::vector<int32_t> level;          // [n_sub]
  std::vector<int32_t> ijk;            // [3 n_sub]
  std::vector<uint8_t> leaf;           // [n_sub]
  std::vector<int32_t> parent;         // [n_sub], -1 at the root
  std::vector<int32_t> child;          // [8 n_sub], octant (x<<2|y<<1|z); -1 for leaves
  std::vector<int32_t> nbr;            // [27 n_sub], slot (dx+1)*9+(dy+1)*3+(dz+1); -1 if absent
  std::vector<int32_t> leaf_ord;       // [n_sub]: ordinal among leaf subgrids, or -1
  std::vector<int32_t> leaf_sub;       // [n_leaf_sub]: global index of each leaf subgrid
  std::vector<std::vector<int32_t>> refined_at;  // per level: refined subgrids
  std::vector<std::vector<int32_t>> leaves_at;   // per level: leaf subgrids
};

// Returns an empty string on success, otherwise an error message.
std::string build_host_tree(int max_level, const uint8_t* flags, int64_t n_flags, HostTree& t);
// Disjoint union of trees (each may itself be a forest).
std::string merge_trees(const std::vector<const HostTree*>& parts, HostTree& out);

struct Stencil {
  double theta = 0;
  std::vector<int32_t> offs[8];   // per target parity: packed offsets (dx, dy, dz)
  std::vector<int32_t> near;      // offsets d != 0 with cells not well separated
  std::vector<int32_t> root_pairs;  // count per root cell of well-separated cells (levels 0)
};

// theta' = dx / |x_A - x_B| < theta for a same-level offset d (in cells).
bool well_separated(int dx, int dy, int dz, double theta);
Stencil make_stencil(double theta);
void interaction_counts(const HostTree& t, const Stencil& s, int64_t out[3]);
// out[6]: M2L leaf<-leaf, leaf<-refined, refined<-leaf, refined<-refined, direct same, mixed.
void interaction_counts_by_type(const HostTree& t, const Stencil& s, int64_t out[6]);

// Spatial decomposition of a single tree over n_ranks (Morton-contiguous below the cut level,
// refined subgrids above it shared) and the ghost subgrids a rank reads from other ranks.
std::string partition_tree(const HostTree& t, int n_ranks, int cut, std::vector<int32_t>& owner);
std::string ghost_subgrids(const HostTree& t, const std::vector<int32_t>& owner, int rank,
                           std::vector<int32_t>& out);

OCTO_HD inline int32_t pack_offset(int dx, int dy, int dz) {
  return ((dx + 16) << 10) | ((dy + 16) << 5) | (dz + 16);
}
OCTO_HD inline void unpack_offset(int32_t c, int& dx, int& dy, int& dz) {
  dx = ((c >> 10) & 31) - 16;
  dy = ((c >> 5) & 31) - 16;
  dz = (c & 31) - 16;
}

}  // namespace octofmm
