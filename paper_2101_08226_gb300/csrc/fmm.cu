// GB300 (sm_103a) octree FMM gravity solve behind the C ABI of octo_fmm.h.
//
// One solve (Sec. 2.2 of Marcello et al. 2021) is a fixed sequence of kernels on the caller's
// stream:
//   p2m        leaf cells become point masses at their centres
//   m2m        level by level from the finest: exact shift of the 8 children's moments
//   m2l        every cell of every level at once: same-level multipole interactions over the
//              opening-criterion stencil with the angular-momentum correction, plus, for leaf
//              cells, the direct sums with non-separated leaves of the same level and of the
//              adjacent level (proper nesting bounds level jumps to one)
//   l2l        level by level from the root: exact Taylor shift of the parent's expansion, added
//              to the cell's own; leaf cells write phi and g
//   reduce     net force, net torque and their normalisation in FP64, fixed order
// The FP64 path runs everything in double precision.  The mixed path keeps moments, shifts,
// correction sums and reductions in FP64 and runs the pairwise interaction arithmetic in FP32 on
// FP32 copies of the moments, with separations formed from exact cell offsets plus FP32
// centre-of-mass displacements.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/octo_fmm.h"
#include "fmm_kernels.cuh"
#include "scf.cuh"
#include "tree.hpp"

using namespace octofmm;

// ----------------------------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int fmm_record_error(int code, const char* msg) { return fail(code, msg); }

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return fail(FMM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));    \
  } while (0)

// Index checks of the bounds-checked build (-DFMM_BOUNDS_CHECK, libocto_fmm_bc.so): before an
// access through an index read from a table (neighbours, children, leaf ordinals, work lists,
// pair lists, stencil tables), the index is tested against its array; a failed test records
// status bit 8 (FMM_ERR_BOUNDS) and the access is skipped (FMM_SKIP: the thread leaves the kernel
// or the loop iteration; FMM_CLAMP: the index is replaced by a safe one where the thread must
// stay for a barrier or a warp shuffle).  Nothing traps.  The normal build compiles none of it.
#ifdef FMM_BOUNDS_CHECK
#define FMM_BAD(A, cond) (!(cond) ? (atomicOr((A).status, 8), true) : false)
#else
#define FMM_BAD(A, cond) false
#endif

// ----------------------------------------------------------------------------------------------
// device-side tree and workspace
// ----------------------------------------------------------------------------------------------
// The caller's arrays of one tree: rho and phi hold its leaf cells in leaf order (512 per leaf
// subgrid, x-major inside a subgrid), g three numbers per cell.  The solve reads these pointers
// from a small device table written at the start of every call, so that a captured graph does not
// depend on the buffers a call passes.
struct TreeIo {
  const double* rho;
  double* phi;
  double* g;
  const double* src;  // d rho / dt (time-derivative solve), or null
  double* phidot;     // d phi / dt out, or null
};

struct DevArgs {
  int64_t n_cell;          // n_sub * 512
  int64_t n_leaf_cells;
  int depth;
  int n_roots;             // trees in the forest; their roots are subgrids 0 .. n_roots-1
  const int64_t* tree_leaf_off;  // [n_roots + 1] first leaf-subgrid ordinal of each tree
  const int32_t* level;    // [n_sub]
  const int32_t* ijk;      // [3 n_sub]
  const uint8_t* leaf;     // [n_sub]
  const int32_t* parent;   // [n_sub]
  const int32_t* child;    // [8 n_sub]
  const int32_t* nbr;      // [27 n_sub]
  const int32_t* leaf_sub; // [n_leaf_sub]
  const int32_t* leaf_ord; // [n_sub]
  const int32_t* stencil;  // [8][kStencilCap] packed offsets
  const int32_t* near;     // packed near offsets
  int n_stencil;           // per parity (the same for every parity)
  int n_near;
  int ws_d2;               // same-level cells are well separated iff |d|^2 > ws_d2
  const int32_t* ltab_off; // [8][kLeafCap] halo offsets of stencil + near entries
  const int32_t* ltab_code;// [8][kLeafCap] packed offsets
  const double* ltab_k64;  // [8][kLeafCap][4]: 1/|d|, d/|d|^3
  const float* ltab_k32;   // same in FP32
  const double* ltab_d64;  // [8][kLeafCap][4]: d (dx, dy, dz, 0) as floating-point numbers
  const float* ltab_d32;
  const dfloat* ltab_kff;  // the 1/|d|, d/|d|^3 table as double-float pairs
  const dfloat* ltab_dff;  // offsets d as double-float
  double* mom;             // [20][n_cell] raw moments (shifted by m2m)
  double* mtl;             // [20][n_cell] same with detraced M2, M3 (read by the interactions)
  float* mom32;            // [n_cell][20] FP32 copy of mtl (mixed path), cell-major: a partner's
                           // 20 moments are 80 contiguous bytes, five 16-byte loads
  float* m32;              // [n_cell] FP32 masses (the leaf kernel's halo)
  dfloat* momff;           // [n_cell][20] double-float copy of mtl (df64 path), cell-major
  dfloat* massff;          // [n_cell] double-float masses
  double* loc;             // [20][n_cell] own, then total expansion
  float* loc32;            // [20][n_cell] own expansion (mixed path)
  double* ac;              // [3][n_cell] correction acceleration, own then total
  // time-derivative solve (Sec. 2.1): source moments about rho's centres of mass
  // (S0, S1 dipole, S2, S3), raw and with detraced S2, S3, and source expansions
  double* smom;            // [20][n_cell]
  double* smtl;            // [20][n_cell]
  float* smom32;           // [20][n_cell] FP32 copy of smtl (mixed path)
  float* src32;            // [n_cell][28] the same, cell-major, then rho's centre-of-mass offset
                           // (3) and 5 zeros: the staged kernel's records (mixed path)
  double* sloc;            // [20][n_cell]
  float* sloc32;           // [20][n_cell]
  double* root_part;       // [n_roots][kRootChunks][23][512] root partial sums (FP64 path)
  float* root_part32;      // [n_roots][kRootChunks][20][512] (mixed path)
  double* root_part_ac;    // [n_roots][kRootChunks][3][512] (mixed path)
  int* status;
  // refined targets with staged partners (mixed path): per target parity, the stencil entries
  // grouped by the parity class of their partner cell
  const float4* stage_tab;    // [8][kLeafCap] {dx, dy, dz, lattice offset (int bits)}
  const int32_t* stage_seg;   // [8][9] class c of parity p: entries [seg[9p + c], seg[9p + c + 1])
  long long wait_cycles;      // limit of its first wait for each class's copies (SM clock cycles)
  // boundary pair lists (per theta): leaf target cells at a refinement boundary, sorted by work
  int64_t n_bt;
  int64_t n_bt_long;       // k_m2l_split: the targets [0, n_bt_long) with four lanes each
  const int32_t* bt_cell;  // [n_bt] internal cell index of each target
  const int32_t* bm_off;   // [n_bt + 1] its multipole partners: bm_e [bm_off[k], ..)
  const uint16_t* bm_e;    // a partner in 16 bits: the neighbour slot of the target's subgrid that
                           // holds it (bits 9-13) and its internal cell index there (bits 0-8)
  const int32_t* bp_off;   // [n_bt + 1] its point-mass partner entries: bp_e [bp_off[k], ..)
  const uint16_t* bp_e;    // an entry in 16 bits: kind (bit 15), neighbour slot (bits 9-13) and
                           // internal cell index (bits 0-8); see point_partner
  const int32_t* leaf_tree;  // [n_leaf_sub] tree of each leaf subgrid
  const TreeIo* io;          // [n_roots] the caller's arrays of each tree
  double* const* io_net;     // the caller's net array (7 numbers per tree), or null
};

constexpr int kStencilCap = 1024;
constexpr int kLeafCap = 1024;       // stencil + near entries per parity
constexpr int kHalo = 18;            // subgrid plus 5 cells on each side
// The halo is stored split by cell parity: cell (x, y, z) of the 18^3 halo at
// ((x & 1) << 2 | (y & 1) << 1 | (z & 1)) * kHaloPar + (x >> 1) * kHaloSX + (y >> 1) * kHaloSY + (z >> 1),
// each parity class a 9 x 9 x 9 lattice padded to strides 120 / 10 / 1.  A warp's lanes read one
// parity class at lattice offsets 120 i + 10 j + k (i, j < 4, k < 2 or k >= 2), which fall on 32
// distinct 4-byte banks, and on 16 distinct 8-byte banks per half warp.
constexpr int kHaloSY = 10;
constexpr int kHaloSX = 120;
constexpr int kHaloPar = 9 * kHaloSX;
constexpr int kHaloWords = 8 * kHaloPar;
constexpr int kLeafThreads = 256;    // one block = one leaf subgrid, two target cells per thread
constexpr int kRootChunks = 8;       // root sources split into 8 chunks of 64 cells
constexpr int kM2LThreads = 64;      // one block = the 64 cells of one parity of one subgrid
constexpr int kSplitLanes = 4;       // lanes per target in k_m2l_split's long-list blocks
// mixed path launch variants: refined kernel (4) x leaf kernel (3) x leaf kernel placement (2)
// x split threshold of the boundary lists (4)
constexpr int kMixedVariants = 96;
constexpr int kSplitChoices = 4;
constexpr int kReduceThreads = 256;
constexpr int kReduceBlocks = 1216;  // 8 per SM

// Cell width 1 / (8 2^lev), a power of two, assembled from its exponent bits (exact; no divide or
// conversion, which run on the FP64 pipe).
__device__ __forceinline__ double cell_dx(int lev) {
  return __longlong_as_double(int64_t(1023 - 3 - lev) << 52);
}
__device__ __forceinline__ float cell_dx32(int lev) { return __int_as_float((127 - 3 - lev) << 23); }
__device__ __forceinline__ double cell_vol(int lev) {
  return __longlong_as_double(int64_t(1023 - 3 * (3 + lev)) << 52);
}
// The double n 2^-k of a nonzero integer |n| < 2^31, assembled from integer operations (an
// int-to-double conversion runs on the FP64 pipe): sign, exponent of the leading bit, mantissa.
__device__ __forceinline__ double dyadic(int n, int k) {
  const uint32_t a = uint32_t(n < 0 ? -n : n);
  const int e = 31 - __clz(int(a));
  const uint64_t mant = (uint64_t(a) << (52 - e)) & ((1ull << 52) - 1);
  const uint64_t bits = (uint64_t(n < 0) << 63) | (uint64_t(1023 + e - k) << 52) | mant;
  return __longlong_as_double(int64_t(bits));
}
// A value as a double: exact either way; a float is widened with
// integer operations (a float-to-double conversion runs on the FP64 pipe).
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return df_f2d(x); }

template <typename T>
__device__ __forceinline__ T cell_h(int lev);
template <>
__device__ __forceinline__ double cell_h<double>(int lev) { return cell_dx(lev); }
template <>
__device__ __forceinline__ float cell_h<float>(int lev) { return cell_dx32(lev); }
template <>
__device__ __forceinline__ dfloat cell_h<dfloat>(int lev) { return dfloat(cell_dx32(lev), 0.0f); }

// Internal order of the 512 cells of a subgrid (the solver's own arrays; user arrays keep
// (a*8 + b)*8 + c): parity-major, cell (a, b, c) = (2 ia + pa, 2 ib + pb, 2 ic + pc) at
// ((pa<<2 | pb<<1 | pc) << 6) | ia << 4 | ib << 2 | ic.  The 64 cells of one parity are then
// contiguous, and the cells a warp of one parity reads at one stencil offset form contiguous runs.
__device__ __forceinline__ int cidx(int a, int b, int c) {
  return ((((a & 1) << 2) | ((b & 1) << 1) | (c & 1)) << 6) | ((a >> 1) << 4) | ((b >> 1) << 2) |
         (c >> 1);
}
__device__ __forceinline__ void cdecode(int i, int& a, int& b, int& c) {
  const int p = i >> 6;
  a = (((i >> 4) & 3) << 1) | ((p >> 2) & 1);
  b = (((i >> 2) & 3) << 1) | ((p >> 1) & 1);
  c = ((i & 3) << 1) | (p & 1);
}

// ----------------------------------------------------------------------------------------------
// p2m: leaf cells are point masses rho dx^3 at their centres
// ----------------------------------------------------------------------------------------------
__global__ void k_p2m(DevArgs A, int mixed) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= A.n_leaf_cells) return;
  int32_t s = A.leaf_sub[i >> 9];
  const int k = A.leaf_tree[i >> 9];
  if (FMM_BAD(A, s >= 0 && int64_t(s) * kCells < A.n_cell && k >= 0 && k < A.n_roots)) return;
  int lev = A.level[s];
  const int u = int(i & 511);
  int64_t cell = int64_t(s) * kCells + cidx(u >> 6, (u >> 3) & 7, u & 7);
  double r = A.io[k].rho[i - A.tree_leaf_off[k] * kCells];
  // finite and >= 0, tested on the bit pattern (a double compare runs on the FP64 pipe): +0 up to
  // the largest finite value lie below the exponent mask, and -0 is the sign bit alone
  const uint64_t bits = uint64_t(__double_as_longlong(r));
  if (!(bits < 0x7ff0000000000000ull || bits == 0x8000000000000000ull)) {
    atomicOr(A.status, 1);
    r = 0.0;
  }
  // the other 19 moments of a leaf cell stay zero from the workspace initialisation
  const double m = r * cell_vol(lev);
  A.mom[cell] = m;
  if (mixed == 0) A.mtl[cell] = m;  // the FP64 detraced set is read by the FP64 path only
  if (mixed == 1) {
    A.mom32[cell * 20] = float(m);
    A.m32[cell] = float(m);
  } else if (mixed == 2) {
    A.momff[cell * 20] = df_from_double(m);
    A.massff[cell] = df_from_double(m);
  }
}

// ----------------------------------------------------------------------------------------------
// m2m: moments of a refined cell from its 8 children (exact shift to the parent's centre of mass)
// ----------------------------------------------------------------------------------------------
// Writes the moments of one refined cell: raw (m, delta, M2, M3) in FP64, and the detraced set
// its path's interactions read: FP64 (mtl), the FP32 copy (mixed path: detraced in FP32 from the
// FP64 moments; its pair arithmetic is FP32) or the double-float copy (df64 path).
__device__ __forceinline__ void store_moments(const DevArgs& A, int64_t cell, double mt, double dx,
                                              double dy, double dz, const double* M2,
                                              const double* M3, int mixed) {
  const int64_t N = A.n_cell;
  A.mom[cell] = mt;
  A.mom[N + cell] = dx;
  A.mom[2 * N + cell] = dy;
  A.mom[3 * N + cell] = dz;
#pragma unroll
  for (int k = 0; k < 6; ++k) A.mom[(4 + k) * N + cell] = M2[k];
#pragma unroll
  for (int k = 0; k < 10; ++k) A.mom[(10 + k) * N + cell] = M3[k];
  if (mixed == 1) {
    float q[6], p[10];
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = float(M2[k]);
#pragma unroll
    for (int k = 0; k < 10; ++k) p[k] = float(M3[k]);
    const float tr3 = (q[0] + q[3] + q[5]) * (1.0f / 3.0f);
    const float tx = (p[0] + p[3] + p[5]) * 0.2f, ty = (p[1] + p[6] + p[8]) * 0.2f,
                tz = (p[2] + p[7] + p[9]) * 0.2f;
    float4* o = reinterpret_cast<float4*>(A.mom32 + cell * 20);
    o[0] = make_float4(float(mt), float(dx), float(dy), float(dz));
    o[1] = make_float4(q[0] - tr3, q[1], q[2], q[3] - tr3);
    o[2] = make_float4(q[4], q[5] - tr3, p[0] - 3.0f * tx, p[1] - ty);
    o[3] = make_float4(p[2] - tz, p[3] - tx, p[4], p[5] - tx);
    o[4] = make_float4(p[6] - 3.0f * ty, p[7] - tz, p[8] - ty, p[9] - 3.0f * tz);
    A.m32[cell] = float(mt);
    return;
  }
  const double tr3 = (M2[0] + M2[3] + M2[5]) * (1.0 / 3.0);
  const double tx = (M3[0] + M3[3] + M3[5]) * 0.2, ty = (M3[1] + M3[6] + M3[8]) * 0.2,
               tz = (M3[2] + M3[7] + M3[9]) * 0.2;
  const double T[20] = {mt, dx, dy, dz, M2[0] - tr3, M2[1], M2[2], M2[3] - tr3, M2[4],
                        M2[5] - tr3, M3[0] - 3 * tx, M3[1] - ty, M3[2] - tz, M3[3] - tx, M3[4],
                        M3[5] - tx, M3[6] - 3 * ty, M3[7] - tz, M3[8] - ty, M3[9] - 3 * tz};
  if (mixed == 0) {
#pragma unroll
    for (int k = 0; k < 20; ++k) A.mtl[k * N + cell] = T[k];
  } else {
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const dfloat u = df_from_double(T[2 * q]), v = df_from_double(T[2 * q + 1]);
      reinterpret_cast<float4*>(A.momff + cell * 20)[q] = make_float4(u.hi, u.lo, v.hi, v.lo);
    }
    A.massff[cell] = df_from_double(mt);
  }
}

// Parent cells go by child octant: thread u of octant o of subgrid s takes parent cell
// (4 o_a + u_a, 4 o_b + u_b, 4 o_c + u_c), whose 8 children are cells (2 u + e) of child subgrid
// child[s][o], internal index (e << 6) | u: a warp reads one child subgrid, coalesced.  The host
// lists each level's octants twice, by the kind of their child subgrid; each kind has its own
// kernel, and a cell's arithmetic depends only on its children, not on what else is solved.
__device__ __forceinline__ void octant_cell(int o, int u, int& a, int& b, int& c) {
  a = 4 * (o >> 2) + (u >> 4);
  b = 4 * ((o >> 1) & 1) + ((u >> 2) & 3);
  c = 4 * (o & 1) + (u & 3);
}

// Octants whose children are leaves, one thread per parent cell.  The children are point masses
// m_e at offsets s_e w (s_e = +-1 per axis, w = dx_(l+1) / 2) from the parent cell's centre, so
// their moments about that centre are sign sums: the 8-point Walsh-Hadamard transform of the
// masses gives M = sum m, D_a = sum s_a m, Q_ab = sum s_a s_b m, W = sum s_x s_y s_z m, with
// sum m u_a u_b = w^2 (M or Q_ab) and sum m u_a u_b u_c = w^3 (D_a if a = b = c, D_c if a = b != c,
// W for x y z).  Shifted to the centre of mass delta = w D / M (parallel axes, sum m (u - delta)
// = 0), with G_ab = M (a = b) or Q_ab:
//   M2_ab = w^2 G_ab - w D_a delta_b,
//   M3_abc = w^3 H_abc - w^2 (delta_a G_bc + delta_b G_ac + delta_c G_ab) + 2 w D_a delta_b delta_c.
__device__ __forceinline__ void m2m_walsh(const DevArgs& A, const int32_t* __restrict__ octs, int blk,
                                          int mixed) {
  const int32_t code = octs[blk];
  const int32_t s = code >> 3;
  const int o = code & 7, u = int(threadIdx.x);
  int a, b, c;
  octant_cell(o, u, a, b, c);
  if (FMM_BAD(A, s >= 0 && int64_t(s) * kCells < A.n_cell && A.child[8 * s + o] >= 0 &&
                    int64_t(A.child[8 * s + o]) * kCells < A.n_cell))
    return;
  const int64_t c0 = int64_t(A.child[8 * s + o]) * kCells + u;  // child e at c0 + (e << 6)
  double v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = A.mom[c0 + (e << 6)];
  // in-place transform over the bits of e (z, y, x): afterwards v[k] = sum_e prod_(bit in k) s_bit m_e
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (!(e & bit)) {
        const double lo = v[e], hi = v[e | bit];
        v[e] = hi + lo;
        v[e | bit] = hi - lo;
      }
  // v[0] = M, v[4] = D_x, v[2] = D_y, v[1] = D_z, v[6] = Q_xy, v[5] = Q_xz, v[3] = Q_yz, v[7] = W
  const double mt = v[0];
  const double w = 0.5 * cell_dx(A.level[s] + 1), w2 = w * w, w3 = w2 * w;
  const double Dx = v[4], Dy = v[2], Dz = v[1], Qxy = v[6], Qxz = v[5], Qyz = v[3], W = v[7];
  double dx = 0, dy = 0, dz = 0;
  if (mt > 0) {
    const double f = w / mt;
    dx = f * Dx;
    dy = f * Dy;
    dz = f * Dz;
  }
  const double ex = w * Dx, ey = w * Dy, ez = w * Dz;  // = M delta
  double M2[6], M3[10];
  M2[0] = w2 * mt - ex * dx;
  M2[1] = w2 * Qxy - ex * dy;
  M2[2] = w2 * Qxz - ex * dz;
  M2[3] = w2 * mt - ey * dy;
  M2[4] = w2 * Qyz - ey * dz;
  M2[5] = w2 * mt - ez * dz;
  // M3: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
  const double gx = w2 * dx, gy = w2 * dy, gz = w2 * dz;  // w^2 delta
  M3[0] = w3 * Dx - 3 * gx * mt + 2 * ex * dx * dx;
  M3[1] = w3 * Dy - (2 * gx * Qxy + gy * mt) + 2 * ex * dx * dy;
  M3[2] = w3 * Dz - (2 * gx * Qxz + gz * mt) + 2 * ex * dx * dz;
  M3[3] = w3 * Dx - (gx * mt + 2 * gy * Qxy) + 2 * ex * dy * dy;
  M3[4] = w3 * W - (gx * Qyz + gy * Qxz + gz * Qxy) + 2 * ex * dy * dz;
  M3[5] = w3 * Dx - (gx * mt + 2 * gz * Qxz) + 2 * ex * dz * dz;
  M3[6] = w3 * Dy - 3 * gy * mt + 2 * ey * dy * dy;
  M3[7] = w3 * Dz - (2 * gy * Qyz + gz * mt) + 2 * ey * dy * dz;
  M3[8] = w3 * Dy - (gy * mt + 2 * gz * Qyz) + 2 * ey * dz * dz;
  M3[9] = w3 * Dz - 3 * gz * mt + 2 * ez * dz * dz;
  store_moments(A, int64_t(s) * kCells + cidx(a, b, c), mt, dx, dy, dz, M2, M3, mixed);
}

// Octants whose children are refined: eight lanes per parent cell, one per child, 64 threads per
// block.  Each lane shifts its child's moments exactly from the child's centre of mass to the
// parent's.  The centre of mass is a butterfly sum (every lane gets the same totals: IEEE
// addition is commutative); the 16 shifted moments are reduced by recursive halving (each stage
// keeps half the values and adds the partner's copy of them), then gathered into the group's
// first lane.  The grid covers 512 threads per octant, so every warp is complete for the shuffles.
constexpr int kM2MThreads = 64;
__device__ __forceinline__ void m2m_lanes(const DevArgs& A, const int32_t* __restrict__ octs, int blk,
                                          int mixed) {
  const int32_t code = octs[blk >> 3];
  const int32_t s = code >> 3;
  const int o = code & 7;
  const int e = int(threadIdx.x & 7);
  const int lead = int(threadIdx.x & 31) & ~7;
  const int u = (blk & 7) * 8 + int(threadIdx.x >> 3);
  int a, b, c;
  octant_cell(o, u, a, b, c);
  const int64_t N = A.n_cell;
  const double hc = cell_dx(A.level[s] + 1);
  int64_t ci = int64_t(A.child[8 * s + o]) * kCells + u + (e << 6);
  const bool bad = FMM_BAD(A, A.child[8 * s + o] >= 0 && ci < N);
  if (bad) ci = 0;  // stays for the shuffles; nothing is stored
  // this child's centre of mass relative to the parent cell's geometric centre
  const double m = A.mom[ci];
  const double ux = (((e >> 2) & 1) ? 0.5 : -0.5) * hc + A.mom[N + ci],
               uy = (((e >> 1) & 1) ? 0.5 : -0.5) * hc + A.mom[2 * N + ci],
               uz = ((e & 1) ? 0.5 : -0.5) * hc + A.mom[3 * N + ci];
  double mt = m, sx = m * ux, sy = m * uy, sz = m * uz;
#pragma unroll
  for (int w = 4; w >= 1; w >>= 1) {
    mt += __shfl_xor_sync(0xffffffffu, mt, w);
    sx += __shfl_xor_sync(0xffffffffu, sx, w);
    sy += __shfl_xor_sync(0xffffffffu, sy, w);
    sz += __shfl_xor_sync(0xffffffffu, sz, w);
  }
  double dx = 0, dy = 0, dz = 0;
  if (mt > 0) {
    const double inv = 1.0 / mt;
    dx = sx * inv;
    dy = sy * inv;
    dz = sz * inv;
  }
  const double rx = ux - dx, ry = uy - dy, rz = uz - dz;
  double q[6], p[10];
#pragma unroll
  for (int k = 0; k < 6; ++k) q[k] = A.mom[(4 + k) * N + ci];
#pragma unroll
  for (int k = 0; k < 10; ++k) p[k] = A.mom[(10 + k) * N + ci];
  // this child's share: M2c + m r r, M3c + r_a M2c_bc + r_b M2c_ac + r_c M2c_ab + m r r r
  // q: xx0 xy1 xz2 yy3 yz4 zz5; X = M2 (6) then M3 (10)
  double X[16];
  X[0] = q[0] + m * rx * rx;
  X[1] = q[1] + m * rx * ry;
  X[2] = q[2] + m * rx * rz;
  X[3] = q[3] + m * ry * ry;
  X[4] = q[4] + m * ry * rz;
  X[5] = q[5] + m * rz * rz;
  X[6] = p[0] + 3 * rx * q[0] + m * rx * rx * rx;
  X[7] = p[1] + 2 * rx * q[1] + ry * q[0] + m * rx * rx * ry;
  X[8] = p[2] + 2 * rx * q[2] + rz * q[0] + m * rx * rx * rz;
  X[9] = p[3] + rx * q[3] + 2 * ry * q[1] + m * rx * ry * ry;
  X[10] = p[4] + rx * q[4] + ry * q[2] + rz * q[1] + m * rx * ry * rz;
  X[11] = p[5] + rx * q[5] + 2 * rz * q[2] + m * rx * rz * rz;
  X[12] = p[6] + 3 * ry * q[3] + m * ry * ry * ry;
  X[13] = p[7] + 2 * ry * q[4] + rz * q[3] + m * ry * ry * rz;
  X[14] = p[8] + ry * q[5] + 2 * rz * q[4] + m * ry * rz * rz;
  X[15] = p[9] + 3 * rz * q[5] + m * rz * rz * rz;
  // recursive halving: after the stage of lane bit w the lane keeps the half selected by that bit
  double Y[8], Z[4], F[2];
  {
    const bool hi = (e & 4) != 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double keep = hi ? X[k + 8] : X[k], give = hi ? X[k] : X[k + 8];
      Y[k] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
  }
  {
    const bool hi = (e & 2) != 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double keep = hi ? Y[k + 4] : Y[k], give = hi ? Y[k] : Y[k + 4];
      Z[k] = keep + __shfl_xor_sync(0xffffffffu, give, 2);
    }
  }
  {
    const bool hi = (e & 1) != 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double keep = hi ? Z[k + 2] : Z[k], give = hi ? Z[k] : Z[k + 2];
      F[k] = keep + __shfl_xor_sync(0xffffffffu, give, 1);
    }
  }
  // lane e holds entries 8 (e >> 2 & 1) + 4 (e >> 1 & 1) + 2 (e & 1) + {0, 1}
  double R[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int owner = ((j >> 3) & 1) << 2 | ((j >> 2) & 1) << 1 | ((j >> 1) & 1);
    R[j] = __shfl_sync(0xffffffffu, F[j & 1], lead + owner);
  }
  if (e != 0 || bad) return;
  store_moments(A, int64_t(s) * kCells + cidx(a, b, c), mt, dx, dy, dz, R, R + 6, mixed);
}

// Upward pass: blocks [0, n_walsh) take octants whose children are leaves (m2m_walsh), the
// others eight blocks per octant whose children are refined (m2m_lanes).
__global__ void __launch_bounds__(kM2MThreads) k_m2m(DevArgs A, const int32_t* __restrict__ walsh_octs,
                                                    int n_walsh, const int32_t* __restrict__ lanes_octs,
                                                    int mixed) {
  if (int(blockIdx.x) < n_walsh) m2m_walsh(A, walsh_octs, int(blockIdx.x), mixed);
  else m2m_lanes(A, lanes_octs, int(blockIdx.x) - n_walsh, mixed);
}

// ----------------------------------------------------------------------------------------------
// m2l: own expansion of every cell
// ----------------------------------------------------------------------------------------------
template <typename T>
struct LeafOffsets;
template <>
struct LeafOffsets<double> {
  static __device__ __forceinline__ const double* get(const DevArgs& A) { return A.ltab_d64; }
};
template <>
struct LeafOffsets<float> {
  static __device__ __forceinline__ const float* get(const DevArgs& A) { return A.ltab_d32; }
};
template <>
struct LeafOffsets<dfloat> {
  static __device__ __forceinline__ const dfloat* get(const DevArgs& A) { return A.ltab_dff; }
};

template <typename T>
struct MomView;
template <>
struct MomView<double> {
  static __device__ __forceinline__ const double* get(const DevArgs& A) { return A.mtl; }
};
template <>
struct MomView<float> {
  static __device__ __forceinline__ const float* get(const DevArgs& A) { return A.mom32; }
};
template <>
struct MomView<dfloat> {
  static __device__ __forceinline__ const dfloat* get(const DevArgs& A) { return A.momff; }
};

// Read-only loads of table values of any of the arithmetic types.
__device__ __forceinline__ double ldg_t(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg_t(const float* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ldg_t(const dfloat* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(v.x, v.y);
}

// Component k of cell i in a moment array: component-major in FP64, cell-major in FP32.
template <typename T>
struct MomAt;
template <>
struct MomAt<double> {
  static __device__ __forceinline__ int64_t at(int64_t N, int64_t i, int k) { return k * N + i; }
};
template <>
struct MomAt<float> {
  static __device__ __forceinline__ int64_t at(int64_t, int64_t i, int k) { return i * 20 + k; }
};
template <>
struct MomAt<dfloat> {
  static __device__ __forceinline__ int64_t at(int64_t, int64_t i, int k) { return i * 20 + k; }
};
template <typename T>
__device__ __forceinline__ T mom_get(const T* __restrict__ M, int64_t N, int64_t i, int k) {
  return M[MomAt<T>::at(N, i, k)];
}
// All 20 moments of cell i.
__device__ __forceinline__ void mom_load20(const double* __restrict__ M, int64_t N, int64_t i,
                                           double* out) {
#pragma unroll
  for (int k = 0; k < 20; ++k) out[k] = M[k * N + i];
}
__device__ __forceinline__ void mom_load20(const float* __restrict__ M, int64_t, int64_t i, float* out) {
  const float4* p = reinterpret_cast<const float4*>(M + i * 20);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const float4 v = __ldg(p + q);
    out[4 * q] = v.x;
    out[4 * q + 1] = v.y;
    out[4 * q + 2] = v.z;
    out[4 * q + 3] = v.w;
  }
}

__device__ __forceinline__ void mom_load20(const dfloat* __restrict__ M, int64_t, int64_t i, dfloat* out) {
  const float4* p = reinterpret_cast<const float4*>(M + i * 20);
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const float4 v = __ldg(p + q);
    out[2 * q] = dfloat(v.x, v.y);
    out[2 * q + 1] = dfloat(v.z, v.w);
  }
}

// Source moments of the time-derivative solve, as read by the interactions.
template <typename T>
struct SrcView;
template <>
struct SrcView<double> {
  static __device__ __forceinline__ const double* get(const DevArgs& A) { return A.smtl; }
};
template <>
struct SrcView<float> {
  static __device__ __forceinline__ const float* get(const DevArgs& A) { return A.smom32; }
};

// Target state.
template <typename T, bool AREF>
struct Target {
  T L[AREF ? 20 : 4];
  T sa1, sa2x, sa2y, sa2z;  // refined targets: running sums of m g1 and m g2 R (interact_rr)
  double ax, ay, az;     // correction acceleration, FP64 sums
  T px, py, pz;          // FP32-or-FP64 partial sums flushed into ax.. by flush()
  T dAx, dAy, dAz;   // target centre-of-mass displacement
  T mA_inv;          // 1 / m_A (0 when m_A = 0)
  T M3A[AREF ? 10 : 1];
  bool amc;
};

// Interaction of target A with one source cell B (same level) at separation
// R = X_A - X_B = (delta_A - delta_B) + o, with o = (o_x, o_y, o_z) the exact offset of A's cell
// centre from B's (an integer multiple of the cell width); BREF: B is refined (full moments),
// else a point mass.
template <typename T, bool AREF, bool BREF>
__device__ __forceinline__ void interact(Target<T, AREF>& S, const T* __restrict__ M, int64_t N,
                                         int64_t iB, T ox, T oy, T oz) {
  T mB;
  Radial<T> g;
  if constexpr (BREF) {
    T Mv[20];
    mom_load20(M, N, iB, Mv);
    mB = Mv[0];
    const T x = (S.dAx - Mv[1]) + ox, y = (S.dAy - Mv[2]) + oy, z = (S.dAz - Mv[3]) + oz;
    const T* M2 = Mv + 4;
    const T* M3 = Mv + 10;
    g.set(x, y, z, 4);
    T qx, qy, qz, rrr;
    m2l_far<T>(x, y, z, g, mB, M2, M3, S.L, qx, qy, qz, rrr);
    if constexpr (AREF) m2l_high<T>(x, y, z, g, mB, S.L);
    if (S.amc) {
      // Q(R,R) = w M3'_A(R,R) - M3'_B(R,R), w = m_B / m_A
      if constexpr (AREF) {
        const T w = mB * S.mA_inv;
        T px, py, pz;
        sym3_rr(S.M3A, x, y, z, px, py, pz);
        const T prrr = x * px + y * py + z * pz;
        qx = w * px - qx;
        qy = w * py - qy;
        qz = w * pz - qz;
        rrr = w * prrr - rrr;
      } else {
        qx = -qx;
        qy = -qy;
        qz = -qz;
        rrr = -rrr;
      }
      T cx, cy, cz;
      amc_from<T>(x, y, z, g, qx, qy, qz, rrr, cx, cy, cz);
      S.px += cx;
      S.py += cy;
      S.pz += cz;
    }
  } else {
    mB = mom_get(M, N, iB, 0);
    const T x = S.dAx + ox, y = S.dAy + oy, z = S.dAz + oz;
    g.set(x, y, z, AREF ? 4 : 1);
    m2l_mono<T>(x, y, z, g, mB, S.L);
    if constexpr (AREF) {
      m2l_high<T>(x, y, z, g, mB, S.L);
      if (S.amc) {
        const T w = mB * S.mA_inv;
        T px, py, pz;
        sym3_rr(S.M3A, x, y, z, px, py, pz);
        const T prrr = x * px + y * py + z * pz;
        T cx, cy, cz;
        amc_from<T>(x, y, z, g, w * px, w * py, w * pz, w * prrr, cx, cy, cz);
        S.px += cx;
        S.py += cy;
        S.pz += cz;
      }
    }
  }
}

// The dominant pair kind -- a refined target and a refined (or leaf, with zero offset and higher
// moments) partner -- written as explicit multiply-add chains, which the compiler cannot form from
// "L -= a b + c d" on its own: the same expansion and correction as interact<T, true, true>.
// M3'(R,R) uses the tracelessness of the stored M3' (T_xzz = -T_xxx - T_xyy, ...) on the shared
// monomials xx - zz, yy - zz, 2xy, 2xz, 2yz; the correction's Q(R,R,R) is contracted directly.
// The partner lies at offset d (in cells, ex ey ez) from the target, cell width h:
// R = X_A - X_B = (delta_A - delta_B) - d h.  The centre-of-mass offsets' difference is rounded
// once and d h is exact, so R of the pair (B, A) is exactly -R in any precision: both halves of
// a pair see the same |R| and opposite directions, and FP32 rounding of R leaves no systematic
// net force.
template <typename T>
__device__ __forceinline__ void interact_rr_v(Target<T, true>& S, const T* Mv, T ex, T ey, T ez, T h) {
  const T mB = Mv[0];
  const T x = (S.dAx - Mv[1]) - ex * h, y = (S.dAy - Mv[2]) - ey * h, z = (S.dAz - Mv[3]) - ez * h;
  const T* M2 = Mv + 4;
  const T* M3 = Mv + 10;  // zzz is not needed
  Radial<T> g;
  g.set(x, y, z, 4);
  const T xx = x * x, yy = y * y, zz = z * z;
  const T dx2 = xx - zz, dy2 = yy - zz;
  const T x2 = x + x, y2 = y + y;
  const T xy2 = x2 * y, xz2 = x2 * z, yz2 = y2 * z;
  // q = M3'_B(R,R) (M3: xxx0 xxy1 xxz2 xyy3 xyz4 xzz5 yyy6 yyz7 yzz8)
  const T qx = fma(M3[0], dx2, fma(M3[3], dy2, fma(M3[1], xy2, fma(M3[2], xz2, M3[4] * yz2))));
  const T qy = fma(M3[1], dx2, fma(M3[6], dy2, fma(M3[3], xy2, fma(M3[4], xz2, M3[7] * yz2))));
  const T qz = fma(M3[2], dx2, fma(M3[7], dy2, fma(M3[4], xy2, fma(M3[5], xz2, M3[8] * yz2))));
  const T rrr = fma(x, qx, fma(y, qy, z * qz));
  // M2' R and R.M2'.R (M2: xx0 xy1 xz2 yy3 yz4 zz5)
  const T m2rx = fma(M2[0], x, fma(M2[1], y, M2[2] * z));
  const T m2ry = fma(M2[1], x, fma(M2[3], y, M2[4] * z));
  const T m2rz = fma(M2[2], x, fma(M2[4], y, M2[5] * z));
  const T rm2r = fma(x, m2rx, fma(y, m2ry, z * m2rz));
  T* L = S.L;
  // L0 -= m g0 + 1/2 g2 R.M2.R - 1/6 g3 M3(R,R,R)
  const T h2 = T(0.5) * g.g2, h3 = g.g3 * T(1.0 / 6.0), k3 = T(0.5) * g.g3;
  L[0] = fma(h3, rrr, fma(-h2, rm2r, fma(-mB, g.g0, L[0])));
  // L1 -= (m g1 + 1/2 g3 R.M2.R) R + g2 M2 R
  const T a1 = mB * g.g1;
  const T c1 = fma(k3, rm2r, a1);
  L[1] = fma(-g.g2, m2rx, fma(-c1, x, L[1]));
  L[2] = fma(-g.g2, m2ry, fma(-c1, y, L[2]));
  L[3] = fma(-g.g2, m2rz, fma(-c1, z, L[3]));
  // L2 -= m (g2 R R + g1 I), L3 -= m (g3 R R R + g2 sym(R I)): the 12 independent components
  const T a2 = mB * g.g2, a3 = mB * g.g3;
  const T a2x = a2 * x, a2y = a2 * y, a2z = a2 * z;
  // the m g1 I and m g2 sym(R I) parts are the same few sums for every component that has them:
  // kept as running sums and applied once by finish_rr
  S.sa1 += a1;
  S.sa2x += a2x;
  S.sa2y += a2y;
  S.sa2z += a2z;
  L[4] = fma(-a2x, x, L[4]);
  L[5] = fma(-a2x, y, L[5]);
  L[6] = fma(-a2x, z, L[6]);
  L[7] = fma(-a2y, y, L[7]);
  L[8] = fma(-a2y, z, L[8]);
  const T a3x = a3 * x, a3y = a3 * y;
  const T a3xx = a3x * x, a3yy = a3y * y;
  L[10] = fma(-a3xx, x, L[10]);
  L[11] = fma(-a3xx, y, L[11]);
  L[12] = fma(-a3xx, z, L[12]);
  L[13] = fma(-a3yy, x, L[13]);
  L[14] = fma(-(a3x * y), z, L[14]);
  L[16] = fma(-a3yy, y, L[16]);
  L[17] = fma(-a3yy, z, L[17]);
  if (S.amc) {
    // Q = (m_B / m_A) M3'_A - M3'_B;  a += 1/6 g4 R Q(R,R,R) + 1/2 g3 Q(R,R)
    const T w = mB * S.mA_inv;
    const T* A3 = S.M3A;
    const T Qx = fma(w, fma(A3[0], dx2, fma(A3[3], dy2, fma(A3[1], xy2, fma(A3[2], xz2, A3[4] * yz2)))), -qx);
    const T Qy = fma(w, fma(A3[1], dx2, fma(A3[6], dy2, fma(A3[3], xy2, fma(A3[4], xz2, A3[7] * yz2)))), -qy);
    const T Qz = fma(w, fma(A3[2], dx2, fma(A3[7], dy2, fma(A3[4], xy2, fma(A3[5], xz2, A3[8] * yz2)))), -qz);
    const T c4 = (g.g4 * T(1.0 / 6.0)) * fma(x, Qx, fma(y, Qy, z * Qz));
    S.px = fma(k3, Qx, fma(c4, x, S.px));
    S.py = fma(k3, Qy, fma(c4, y, S.py));
    S.pz = fma(k3, Qz, fma(c4, z, S.pz));
  }
}

template <typename T>
__device__ __forceinline__ void interact_rr(Target<T, true>& S, const T* __restrict__ M, int64_t N,
                                            int64_t iB, T ex, T ey, T ez, T h) {
  T Mv[20];
  mom_load20(M, N, iB, Mv);
  interact_rr_v<T>(S, Mv, ex, ey, ez, h);
}

// A leaf target (a point mass at its centre: only L0, L1; no M3 of its own, so the correction
// takes Q = -M3'_B) and a refined partner, in the same multiply-add form as interact_rr.
template <typename T>
__device__ __forceinline__ void interact_lr(Target<T, false>& S, const T* __restrict__ M, int64_t N,
                                            int64_t iB, T x, T y, T z) {
  T Mv[20];
  mom_load20(M, N, iB, Mv);
  const T mB = Mv[0];
  x -= Mv[1];
  y -= Mv[2];
  z -= Mv[3];
  const T* M2 = Mv + 4;
  const T* M3 = Mv + 10;
  Radial<T> g;
  g.set(x, y, z, 4);
  const T xx = x * x, yy = y * y, zz = z * z;
  const T dx2 = xx - zz, dy2 = yy - zz;
  const T x2 = x + x, y2 = y + y;
  const T xy2 = x2 * y, xz2 = x2 * z, yz2 = y2 * z;
  const T qx = fma(M3[0], dx2, fma(M3[3], dy2, fma(M3[1], xy2, fma(M3[2], xz2, M3[4] * yz2))));
  const T qy = fma(M3[1], dx2, fma(M3[6], dy2, fma(M3[3], xy2, fma(M3[4], xz2, M3[7] * yz2))));
  const T qz = fma(M3[2], dx2, fma(M3[7], dy2, fma(M3[4], xy2, fma(M3[5], xz2, M3[8] * yz2))));
  const T rrr = fma(x, qx, fma(y, qy, z * qz));
  const T m2rx = fma(M2[0], x, fma(M2[1], y, M2[2] * z));
  const T m2ry = fma(M2[1], x, fma(M2[3], y, M2[4] * z));
  const T m2rz = fma(M2[2], x, fma(M2[4], y, M2[5] * z));
  const T rm2r = fma(x, m2rx, fma(y, m2ry, z * m2rz));
  T* L = S.L;
  const T h2 = T(0.5) * g.g2, h3 = g.g3 * T(1.0 / 6.0), k3 = T(0.5) * g.g3;
  L[0] = fma(h3, rrr, fma(-h2, rm2r, fma(-mB, g.g0, L[0])));
  const T c1 = fma(k3, rm2r, mB * g.g1);
  L[1] = fma(-g.g2, m2rx, fma(-c1, x, L[1]));
  L[2] = fma(-g.g2, m2ry, fma(-c1, y, L[2]));
  L[3] = fma(-g.g2, m2rz, fma(-c1, z, L[3]));
  if (S.amc) {
    // Q = -M3'_B: a += 1/6 g4 R Q(R,R,R) + 1/2 g3 Q(R,R)
    const T c4 = (g.g4 * T(1.0 / 6.0)) * rrr;
    S.px = fma(-k3, qx, fma(-c4, x, S.px));
    S.py = fma(-k3, qy, fma(-c4, y, S.py));
    S.pz = fma(-k3, qz, fma(-c4, z, S.pz));
  }
}

// The running sums of interact_rr into the L2, L3 components: L2 -= sum m g1 I,
// L3 -= sum m g2 sym(R I) (xxx: 3 x, xxy: y, xxz: z, xyy: x, yyy: 3 y, yyz: z).
template <typename T>
__device__ __forceinline__ void finish_rr(Target<T, true>& S) {
  T* L = S.L;
  L[4] -= S.sa1;
  L[7] -= S.sa1;
  L[10] -= T(3) * S.sa2x;
  L[11] -= S.sa2y;
  L[12] -= S.sa2z;
  L[13] -= S.sa2x;
  L[16] -= T(3) * S.sa2y;
  L[17] -= S.sa2z;
  S.sa1 = S.sa2x = S.sa2y = S.sa2z = T(0);
}

// Adds the partial correction sums to the FP64 accumulators (the mixed path sums at most 64
// pair terms in FP32 before each flush).
template <typename T, bool AREF>
__device__ __forceinline__ void flush(Target<T, AREF>& S) {
  if constexpr (std::is_same<T, float>::value) {
    S.ax += to_f64(S.px);
    S.ay += to_f64(S.py);
    S.az += to_f64(S.pz);
  } else {
    S.ax += double(S.px);
    S.ay += double(S.py);
    S.az += double(S.pz);
  }
  S.px = S.py = S.pz = T(0);
}

// Point-mass source at separation R (exact positions).
template <typename T, bool AREF>
__device__ __forceinline__ void interact_point(Target<T, AREF>& S, T mB, T x, T y, T z) {
  Radial<T> g;
  g.set(x, y, z, 1);
  m2l_mono<T>(x, y, z, g, mB, S.L);
}

template <typename T, bool AREF>
__device__ __forceinline__ void load_target(Target<T, AREF>& S, const DevArgs& A,
                                            const T* __restrict__ M, int64_t iA, bool amc) {
#pragma unroll
  for (int k = 0; k < (AREF ? 20 : 4); ++k) S.L[k] = T(0);
  S.ax = S.ay = S.az = 0.0;
  S.px = S.py = S.pz = T(0);
  S.sa1 = S.sa2x = S.sa2y = S.sa2z = T(0);
  const int64_t N = A.n_cell;
  S.amc = amc;
  if constexpr (AREF) {
    T Mv[20];
    mom_load20(M, N, iA, Mv);
    S.dAx = Mv[1];
    S.dAy = Mv[2];
    S.dAz = Mv[3];
    const T mA = Mv[0];
    S.mA_inv = mA > T(0) ? T(1) / mA : T(0);
    if (!(mA > T(0))) S.amc = false;
#pragma unroll
    for (int k = 0; k < 10; ++k) S.M3A[k] = Mv[10 + k];
  } else {
    S.dAx = S.dAy = S.dAz = T(0);
    S.mA_inv = T(0);
    if (!(mom_get(M, N, iA, 0) > T(0))) S.amc = false;
  }
}

template <typename T, bool AREF>
__device__ __forceinline__ void store_own(const DevArgs& A, const Target<T, AREF>& S, int64_t iA);

template <>
__device__ __forceinline__ void store_own<double, true>(const DevArgs& A,
                                                        const Target<double, true>& S, int64_t iA) {
  const int64_t N = A.n_cell;
  double L[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) L[k] = S.L[k];
  complete_traceless(L);
#pragma unroll
  for (int k = 0; k < 20; ++k) A.loc[k * N + iA] = L[k];
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}
template <>
__device__ __forceinline__ void store_own<double, false>(const DevArgs& A,
                                                         const Target<double, false>& S, int64_t iA) {
  const int64_t N = A.n_cell;
#pragma unroll
  for (int k = 0; k < 4; ++k) A.loc[k * N + iA] = S.L[k];
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}
template <>
__device__ __forceinline__ void store_own<dfloat, true>(const DevArgs& A,
                                                        const Target<dfloat, true>& S, int64_t iA) {
  const int64_t N = A.n_cell;
  dfloat L[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) L[k] = S.L[k];
  complete_traceless(L);
#pragma unroll
  for (int k = 0; k < 20; ++k) A.loc[k * N + iA] = double(L[k]);
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}
template <>
__device__ __forceinline__ void store_own<dfloat, false>(const DevArgs& A,
                                                         const Target<dfloat, false>& S, int64_t iA) {
  const int64_t N = A.n_cell;
#pragma unroll
  for (int k = 0; k < 4; ++k) A.loc[k * N + iA] = double(S.L[k]);
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}
template <>
__device__ __forceinline__ void store_own<float, true>(const DevArgs& A,
                                                       const Target<float, true>& S, int64_t iA) {
  const int64_t N = A.n_cell;
  float L[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) L[k] = S.L[k];
  complete_traceless(L);
#pragma unroll
  for (int k = 0; k < 20; ++k) A.loc32[k * N + iA] = L[k];
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}
template <>
__device__ __forceinline__ void store_own<float, false>(const DevArgs& A,
                                                        const Target<float, false>& S, int64_t iA) {
  const int64_t N = A.n_cell;
#pragma unroll
  for (int k = 0; k < 4; ++k) A.loc32[k * N + iA] = S.L[k];
  A.ac[iA] = S.ax;
  A.ac[N + iA] = S.ay;
  A.ac[2 * N + iA] = S.az;
}

// Target cell of a block: 64 threads = the 64 cells of one parity of one subgrid.
__device__ __forceinline__ void block_cell(int parity, int t, int& a, int& b, int& c) {
  int px = (parity >> 2) & 1, py = (parity >> 1) & 1, pz = parity & 1;
  a = 2 * (t >> 4) + px;
  b = 2 * ((t >> 2) & 3) + py;
  c = 2 * (t & 3) + pz;
}

// Refined target subgrid s of a level >= 1, parity p: multipole interactions with every stencil
// partner.  Under proper nesting a refined subgrid has all 26 same-level neighbours, and a leaf
// partner is a point mass whose centre-of-mass offset and higher moments are stored as zeros, so
// every pair takes the full multipole formula and a warp never splits on the partner's kind.
// The correction partial sums are flushed after each chunk of kFlush stencil entries, outside the
// pair loop: FP64 work under a predicate inside the loop would occupy the FP64 pipe on every pass.
constexpr int kFlush = 64;

template <typename T>
__device__ void m2l_level(const DevArgs& A, int32_t s, int parity, int t, bool amc) {
  __shared__ int32_t nb[27];
  if (threadIdx.x < 27) nb[threadIdx.x] = A.nbr[27 * s + threadIdx.x];
  __syncthreads();
  const int lev = A.level[s];
  const T* __restrict__ M = MomView<T>::get(A);
  const int64_t N = A.n_cell;
  int a, b, c;
  block_cell(parity, t, a, b, c);
  const int64_t iA = int64_t(s) * kCells + cidx(a, b, c);
  Target<T, true> S;
  load_target<T, true>(S, A, M, iA, amc);
  const T h = cell_h<T>(lev);
  const int32_t* __restrict__ st = A.ltab_code + parity * kLeafCap;
  const T* __restrict__ td = LeafOffsets<T>::get(A) + int64_t(parity) * kLeafCap * 4;
  for (int q0 = 0; q0 < A.n_stencil; q0 += kFlush) {
    const int q1 = min(q0 + kFlush, A.n_stencil);
    for (int q = q0; q < q1; ++q) {
      int dx, dy, dz;
      unpack_offset(__ldg(st + q), dx, dy, dz);
      int px = a + dx, py = b + dy, pz = c + dz;
      int slot = ((px >> 3) + 1) * 9 + ((py >> 3) + 1) * 3 + ((pz >> 3) + 1);
      int32_t sB = nb[slot];
      if (sB < 0) continue;  // only without proper nesting
      int64_t iB = int64_t(sB) * kCells + cidx(px & 7, py & 7, pz & 7);
      if (FMM_BAD(A, iB < N && slot >= 0 && slot < 27)) continue;
      interact_rr<T>(S, M, N, iB, ldg_t(td + 4 * q), ldg_t(td + 4 * q + 1), ldg_t(td + 4 * q + 2), h);
    }
    flush(S);
  }
  finish_rr(S);
  store_own<T, true>(A, S, iA);
}

// Root level: every well-separated pair inside the single root subgrid (no parent criterion);
// when the root is a leaf, every other root cell interacts directly.  Sources are split into
// kRootChunks chunks whose partial sums are added in a fixed order by the downward pass.
// Sums a target's partial state over the LANES consecutive lanes that share it (LANES = 1, 2, 4
// or 8); every lane of the warp calls it.  The correction partials must have been flushed.
template <int LANES, typename T, bool AREF>
__device__ __forceinline__ void lane_reduce(Target<T, AREF>& S) {
#pragma unroll
  for (int m = 1; m < LANES; m <<= 1) {
#pragma unroll
    for (int k = 0; k < (AREF ? 20 : 4); ++k) S.L[k] += __shfl_xor_sync(0xffffffffu, S.L[k], m);
    S.ax += __shfl_xor_sync(0xffffffffu, S.ax, m);
    S.ay += __shfl_xor_sync(0xffffffffu, S.ay, m);
    S.az += __shfl_xor_sync(0xffffffffu, S.az, m);
  }
}

// LANES lanes per target: lane r takes the source rows jy in [r 8 / LANES, (r + 1) 8 / LANES),
// and lane 0 stores the sum.
template <typename T, bool AREF, int LANES = 1>
__device__ void m2l_root(const DevArgs& A, int root, int parity, int t, int chunk, bool amc,
                         int r = 0) {
  static_assert(LANES == 1 || LANES == 2 || LANES == 4 || LANES == 8, "LANES divides 8");
  const T* __restrict__ M = MomView<T>::get(A);
  const int64_t N = A.n_cell;
  int a, b, c;
  block_cell(parity, t, a, b, c);
  const int iloc = cidx(a, b, c);
  const int64_t base = int64_t(root) * kCells;
  Target<T, AREF> S;
  load_target<T, AREF>(S, A, M, base + iloc, amc);
  const T h = cell_h<T>(0);
  const bool root_leaf = A.leaf[root] != 0;
  // chunk = source x index; the exact offsets of the target's cell centre from the source's,
  // kept as floating-point counters (no conversions; small multiples of h, so exact)
  const int dx = chunk - a;
  const T ox = -T(dx) * h;
  constexpr int kRows = 8 / LANES;
  const int jy0 = r * kRows;
  // for a source at y = jy0, z = 0
  T oy = T(b - jy0) * h;
  const T oz0 = T(c) * h;
  for (int jy = jy0; jy < jy0 + kRows; ++jy, oy -= h) {
    T oz = oz0;
    for (int jz = 0; jz < 8; ++jz, oz -= h) {
      const int j = cidx(chunk, jy, jz);
      if (j == iloc) continue;
      const int dy = jy - b, dz = jz - c;
      const bool ws = dx * dx + dy * dy + dz * dz > A.ws_d2;
      if (!ws && !root_leaf) continue;
      interact<T, AREF, AREF>(S, M, N, base + j, ox, oy, oz);  // AREF: the root is refined
    }
    if (jy & 1) flush(S);
  }
  flush(S);
  if constexpr (LANES > 1) {
    lane_reduce<LANES>(S);
    if (r != 0) return;
  }
  // partials: [chunk][component][cell]
  if constexpr (AREF) complete_traceless(S.L);
  if (sizeof(T) == 8) {
    double* P = A.root_part + (int64_t(root) * kRootChunks + chunk) * 23 * kCells;
    for (int k = 0; k < (AREF ? 20 : 4); ++k) P[k * kCells + iloc] = double(S.L[k]);
    for (int k = (AREF ? 20 : 4); k < 20; ++k) P[k * kCells + iloc] = 0.0;
    P[20 * kCells + iloc] = S.ax;
    P[21 * kCells + iloc] = S.ay;
    P[22 * kCells + iloc] = S.az;
  } else {
    float* P = A.root_part32 + (int64_t(root) * kRootChunks + chunk) * 20 * kCells;
    for (int k = 0; k < (AREF ? 20 : 4); ++k) P[k * kCells + iloc] = float(S.L[k]);
    for (int k = (AREF ? 20 : 4); k < 20; ++k) P[k * kCells + iloc] = 0.0f;
    double* Q = A.root_part_ac + (int64_t(root) * kRootChunks + chunk) * 3 * kCells;
    Q[iloc] = S.ax;
    Q[kCells + iloc] = S.ay;
    Q[2 * kCells + iloc] = S.az;
  }
}

// Masses of cells as point sources, in each precision's array.
template <typename T>
struct LeafMass;
template <>
struct LeafMass<double> {
  static __device__ __forceinline__ const double* get(const DevArgs& A) { return A.mtl; }
};
template <>
struct LeafMass<float> {
  static __device__ __forceinline__ const float* get(const DevArgs& A) { return A.m32; }
};
template <>
struct LeafMass<dfloat> {
  static __device__ __forceinline__ const dfloat* get(const DevArgs& A) { return A.massff; }
};

// A multipole partner of a boundary target from its 16-bit list entry: the neighbour slot of the
// target's subgrid s (slot = (sx * 3 + sy) * 3 + sz, s itself at 13) and the partner's internal
// cell index there; also the partner's offset from the target cell (a, b, c) in cells.
__device__ __forceinline__ int64_t boundary_partner(const DevArgs& A, int32_t s, int a, int b, int c,
                                                    uint32_t e, int& dx, int& dy, int& dz) {
  const int slot = int(e >> 9), loc = int(e & 511);
  int la, lb, lc;
  cdecode(loc, la, lb, lc);
  dx = (slot / 9 - 1) * kSub + la - a;
  dy = ((slot / 3) % 3 - 1) * kSub + lb - b;
  dz = (slot % 3 - 1) * kSub + lc - c;
  const int32_t q = A.nbr[27 * s + slot];
  return int64_t(q) * kCells + loc;
}
// A point-mass partner entry of a boundary target (kind << 15 | slot << 9 | internal cell index).
// Kind 0: a near cell (offset d in cells from the target cell (a, b, c)) in the refined
// same-level neighbour at `slot` of the target's subgrid s.  It stands for the near cell's 8
// leaf children, which the parity-major order puts 64 apart: child o = ox << 2 | oy << 1 | oz
// is cell first + 64 o, and x_A - x_child = (1 - 2 o_x - 4 d_x, ...) dx / 4.
// Kind 1: a leaf cell one level coarser, in the neighbour at `slot` of the parent subgrid, at
// offset d in coarse cells from the target's parent cell: one partner at first, with
// x_A - x_i = (4 (a & 1) - 2 - 8 d_x, ...) dx / 4.
// Returns the number of point masses (8 or 1) and q = x_A - x_first in units of dx / 4; -1 when
// a bounds check fails (the bounds-checked build).
__device__ __forceinline__ int point_partner(const DevArgs& A, int32_t s, int a, int b, int c,
                                             uint32_t e, int64_t& first, int& qx, int& qy, int& qz) {
  const int slot = int((e >> 9) & 31), loc = int(e & 511);
  int la, lb, lc;
  cdecode(loc, la, lb, lc);
  const int px = (slot / 9 - 1) * kSub + la, py = ((slot / 3) % 3 - 1) * kSub + lb,
            pz = (slot % 3 - 1) * kSub + lc;
  if (!(e >> 15)) {
    const int32_t q = A.nbr[27 * s + slot];
    if (FMM_BAD(A, slot < 27 && q >= 0 && int64_t(q) * kCells < A.n_cell)) return -1;
    const int32_t cs = A.child[8 * q + ((la >> 2) << 2 | (lb >> 2) << 1 | (lc >> 2))];
    if (FMM_BAD(A, cs >= 0 && int64_t(cs) * kCells < A.n_cell)) return -1;
    first = int64_t(cs) * kCells + ((la & 3) << 4 | (lb & 3) << 2 | (lc & 3));
    qx = 1 - 4 * (px - a);
    qy = 1 - 4 * (py - b);
    qz = 1 - 4 * (pz - c);
    return 8;
  }
  const int32_t P = A.parent[s];
  if (FMM_BAD(A, slot < 27 && P >= 0 && int64_t(P) * kCells < A.n_cell)) return -1;
  const int32_t q = A.nbr[27 * P + slot];
  if (FMM_BAD(A, q >= 0 && int64_t(q) * kCells < A.n_cell)) return -1;
  first = int64_t(q) * kCells + loc;
  // the target's parent cell in the parent subgrid: (a >> 1) + 4 (the subgrid's octant bit)
  qx = 4 * (a & 1) - 2 - 8 * (px - ((A.ijk[3 * s] & 1) << 2) - (a >> 1));
  qy = 4 * (b & 1) - 2 - 8 * (py - ((A.ijk[3 * s + 1] & 1) << 2) - (b >> 1));
  qz = 4 * (c & 1) - 2 - 8 * (pz - ((A.ijk[3 * s + 2] & 1) << 2) - (c >> 1));
  return 1;
}
// -d h for an integer offset d and a cell width h = 2^-(lev + 3), exact and without FP64-pipe
// arithmetic in the FP64 path (the double is assembled from integer bits).
template <typename T>
__device__ __forceinline__ T neg_offset(int d, int lev);
template <>
__device__ __forceinline__ double neg_offset<double>(int d, int lev) {
  return __longlong_as_double(d == 0 ? 0ll : __double_as_longlong(dyadic(-d, lev + 3)));
}
template <>
__device__ __forceinline__ float neg_offset<float>(int d, int lev) { return float(-d) * cell_dx32(lev); }
template <>
__device__ __forceinline__ dfloat neg_offset<dfloat>(int d, int lev) {
  return dfloat(float(-d) * cell_dx32(lev), 0.0f);
}

// Leaf targets at a refinement boundary, 64 per block, from the pair lists built on the host:
// multipole interactions with the cells of refined same-level neighbours, then direct sums with
// point masses (the leaf children of refined near cells, and leaves one level coarser near the
// parent cell).  The targets are sorted by work, so the lanes of a warp run lists of similar
// length and no lane scans entries that do not apply to it.  Adds onto the leaf kernel's output.
constexpr int kCodeMax = 64;  // |point-pair offset| in units of dx / 4

// LANES lanes per target: lane r takes the list entries r, r + LANES, ..., and lane 0 stores
// the sum (every lane of the block calls this, also past the last target).
// The block's targets are first + 64 chunk + t, those below end.
template <typename T, int LANES = 1>
__device__ void m2l_boundary(const DevArgs& A, int64_t first, int64_t end, int chunk, int t, bool amc,
                             int r = 0) {
  __shared__ T quarter[2 * kCodeMax + 1];  // quarter[i] = (i - kCodeMax) / 4, exact
  for (int i = threadIdx.x; i <= 2 * kCodeMax; i += blockDim.x) quarter[i] = T(i - kCodeMax) * T(0.25);
  __syncthreads();
  const int64_t k = first + int64_t(chunk) * 64 + t;
  const bool valid = k < end && !FMM_BAD(A, A.bt_cell[k] >= 0 && A.bt_cell[k] < A.n_cell);
  if (LANES == 1 && !valid) return;
  const int64_t iA = valid ? A.bt_cell[k] : 0;
  const T* __restrict__ M = MomView<T>::get(A);
  const int64_t N = A.n_cell;
  Target<T, false> S;
  load_target<T, false>(S, A, M, iA, amc);
  const int32_t sA = int32_t(iA >> 9);
  const int lev = A.level[sA];
  const T h = cell_h<T>(lev);
  int a, b, c;
  cdecode(int(iA & 511), a, b, c);
  // each list entry is loaded and decoded one entry ahead, so that a pair waits for its
  // partner's moments only, not for the index that locates them first; point partners' masses
  // come from the contiguous mass array (the same values as component 0 of the moments)
  const T* __restrict__ Mass = LeafMass<T>::get(A);
  const int32_t m0 = (valid ? A.bm_off[k] : 0) + r, m1 = valid ? A.bm_off[k + 1] : 0;
  int dx_next = 0, dy_next = 0, dz_next = 0;
  int64_t src_next = 0;
  if (m0 < m1) src_next = boundary_partner(A, sA, a, b, c, __ldg(A.bm_e + m0), dx_next, dy_next, dz_next);
  for (int32_t j0 = m0; j0 < m1; j0 += LANES * kFlush) {
    const int32_t j1 = min(j0 + LANES * kFlush, m1);
    for (int32_t j = j0; j < j1; j += LANES) {
      const int64_t src = src_next;
      const int dx = dx_next, dy = dy_next, dz = dz_next;
      if (j + LANES < m1)
        src_next = boundary_partner(A, sA, a, b, c, __ldg(A.bm_e + j + LANES), dx_next, dy_next, dz_next);
      if (FMM_BAD(A, src >= 0 && src < N)) continue;
      interact_lr<T>(S, M, N, src, neg_offset<T>(dx, lev), neg_offset<T>(dy, lev), neg_offset<T>(dz, lev));
    }
    flush(S);
  }
  const int32_t p0 = (valid ? A.bp_off[k] : 0) + r, p1 = valid ? A.bp_off[k + 1] : 0;
  int64_t first_next = 0;
  int n_next = 0, qx_next = 0, qy_next = 0, qz_next = 0;
  if (p0 < p1) n_next = point_partner(A, sA, a, b, c, __ldg(A.bp_e + p0), first_next, qx_next, qy_next, qz_next);
  for (int32_t j = p0; j < p1; j += LANES) {
    const int64_t first = first_next;
    const int n = n_next, qx = qx_next, qy = qy_next, qz = qz_next;
    if (j + LANES < p1)
      n_next = point_partner(A, sA, a, b, c, __ldg(A.bp_e + j + LANES), first_next, qx_next, qy_next, qz_next);
    if (FMM_BAD(A, n > 0 && first + 64 * (n - 1) < N && unsigned(qx + kCodeMax - 2) <= 2u * kCodeMax - 2 &&
                       unsigned(qy + kCodeMax - 2) <= 2u * kCodeMax - 2 &&
                       unsigned(qz + kCodeMax - 2) <= 2u * kCodeMax - 2))
      continue;
    if (n == 8) {
#pragma unroll
      for (int o = 0; o < 8; ++o)
        interact_point<T, false>(S, Mass[first + 64 * o], quarter[qx - 2 * (o >> 2) + kCodeMax] * h,
                                 quarter[qy - 2 * ((o >> 1) & 1) + kCodeMax] * h,
                                 quarter[qz - 2 * (o & 1) + kCodeMax] * h);
    } else {
      interact_point<T, false>(S, Mass[first], quarter[qx + kCodeMax] * h, quarter[qy + kCodeMax] * h,
                               quarter[qz + kCodeMax] * h);
    }
  }
  if constexpr (LANES > 1) {
    lane_reduce<LANES>(S);  // the correction partials were flushed after the multipole pairs
    if (r != 0 || !valid) return;
  }
  if (sizeof(T) == 8) {
    for (int c = 0; c < 4; ++c) A.loc[c * N + iA] += double(S.L[c]);
  } else {
    for (int c = 0; c < 4; ++c) A.loc32[c * N + iA] += float(S.L[c]);
  }
  A.ac[iA] += S.ax;
  A.ac[N + iA] += S.ay;
  A.ac[2 * N + iA] += S.az;
}

// One block per entry of `blocks`, sorted by estimated cost (largest first): code
// (kind << 30) | (parity << 27) | index, kind 0 = source chunk index & 7 of root index >> 3,
// 1 = refined subgrid `index`, 2 = chunk `index` of 64 boundary leaf targets (parity unused).  With NT = 64 a block serves the 64
// cells of one parity; with NT = 512 it serves all 8 parities of the subgrid (or all 512 root
// cells), so that every source the subgrid's cells read is fetched into one SM's L1 once.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_m2l_ref(DevArgs A, const int32_t* __restrict__ blocks,
                                                int amc) {
  const int32_t code = blocks[blockIdx.x];
  const int kind = (code >> 30) & 3, idx = code & ((1 << 27) - 1);
  const int parity = NT == 64 ? (code >> 27) & 7 : int(threadIdx.x >> 6);
  const int t = int(threadIdx.x & 63);
  if (kind == 0) {
    const int root = idx >> 3, chunk = idx & 7;
    if (A.leaf[root]) m2l_root<T, false>(A, root, parity, t, chunk, amc != 0);
    else m2l_root<T, true>(A, root, parity, t, chunk, amc != 0);
  } else if (kind == 1) {
    m2l_level<T>(A, idx, parity, t, amc != 0);
  } else {
    m2l_boundary<T>(A, 0, A.n_bt, idx, t, amc != 0);
  }
}

// The root and boundary work of k_m2l_ref for the mixed path (refined subgrids go to
// k_m2l_stage), 256 threads per block.  Kinds 0 (root chunk) and 2 (64 boundary targets of
// [0, n_bt_long)): 4 lanes per target -- these threads would run long serial lists of partners
// read from L2, so each list is split four ways and the partial sums are added with warp
// shuffles.  Kind 3: the targets n_bt_long + 64 (idx .. idx + 3) + t, one lane each.
// (at most 64 registers, four blocks per SM: this kernel waits on scattered gathers, and the
// extra warps hide more of that latency than the few spilled registers cost -- measured 1.5-2.5 %
// off the mixed solve on the 5- and 7-level binaries and the 64-tree forest)
template <typename T>
__global__ void __launch_bounds__(64 * kSplitLanes, 4) k_m2l_split(DevArgs A, const int32_t* __restrict__ blocks,
                                                                 int amc) {
  const int32_t code = blocks[blockIdx.x];
  const int kind = (code >> 30) & 3, idx = code & ((1 << 27) - 1);
  const int parity = (code >> 27) & 7;
  const int t = int(threadIdx.x) / kSplitLanes, r = int(threadIdx.x) % kSplitLanes;
  if (kind == 0) {
    const int root = idx >> 3, chunk = idx & 7;
    if (A.leaf[root]) m2l_root<T, false, kSplitLanes>(A, root, parity, t, chunk, amc != 0, r);
    else m2l_root<T, true, kSplitLanes>(A, root, parity, t, chunk, amc != 0, r);
  } else if (kind == 2) {
    m2l_boundary<T, kSplitLanes>(A, 0, A.n_bt_long, idx, t, amc != 0, r);
  } else {
    m2l_boundary<T, 1>(A, A.n_bt_long, A.n_bt, idx + int(threadIdx.x) / 64, int(threadIdx.x) % 64,
                       amc != 0);
  }
}

// ----------------------------------------------------------------------------------------------
// Refined targets with their partners' moments staged in shared memory (mixed path)
// ----------------------------------------------------------------------------------------------
// A refined subgrid's 512 targets read the FP32 moments of the 18^3 cells of the subgrid and its
// 5-cell rim, each about 20 times.  The block stages them one parity class at a time (a 9^3
// lattice of 80-byte cells, 57 KB) with bulk asynchronous copies (TMA, cp.async.bulk) completing
// on an mbarrier, double-buffered so that class c + 1 arrives while class c is evaluated, and
// every target then walks the stencil entries whose partner lies in class c.
//
// Halo cell (x, y, z) in [-5, 12]^3, h = x + 5: class ((hx & 1) << 2 | (hy & 1) << 1 | (hz & 1)),
// lattice cell (hx >> 1, hy >> 1, hz >> 1) at lattice strides (kStageSX, kStageSY, 1) cells.
// A warp holds the 32 targets (ia, ib, ic) = (2 half + (lane >> 2 & 1), lane >> 3, lane & 3) of
// one parity, so the 8 lanes of each quarter warp (ic = 0..3, ia even and odd) read 16-byte
// words at 5 (ic + kStageSX ia) mod 8 = {0, 5, 2, 7} + {0, 4}: 8 distinct bank groups.
constexpr int kStageThreads = 512;
constexpr int kStageSY = 9;
constexpr int kStageSX = 84;  // = 4 (mod 8), see above; 84 >= 9 * 9
constexpr int kStageCells = 8 * kStageSX + 8 * kStageSY + 9;
constexpr int kStageSmem = 2 * kStageCells * 80;  // two buffers of 20-float cells
constexpr int kStageRuns = 243;  // per class: 9 x 9 lattice columns, each 3 runs along z
constexpr long long kStageWaitCycles = 1ll << 31;  // about a second: then report and give up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// (the arrive operations return the barrier state, which the callers do not need)
__device__ __forceinline__ uint64_t mbar_arrive(uint64_t* bar) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_u32(bar)) : "memory");
  return state;
}
__device__ __forceinline__ uint64_t mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  return state;
}
// Non-blocking test of the phase of the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase of the given parity to complete, for at most `limit` SM clock cycles;
// false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// Waits like mbar_wait_bounded, but in try_wait (the thread may be suspended in the barrier until
// the phase completes, for the hardware's own time limit) rather than in a test loop, so a
// waiting warp takes few issue slots from the warps still computing.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_sleep_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completing
// `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(uint64_t(__cvta_generic_to_global(src))), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Thread j < kStageRuns copies run j of class c into buf: lattice column (lx, ly) = (j / 27,
// j / 3 % 9), z run j % 3 (halo z < 0, 0 <= z < 8, z >= 8), from the neighbour subgrid that
// holds it; an absent neighbour (only without proper nesting) gives zeros.  W floats per cell.
template <int W>
__device__ __forceinline__ void stage_issue(const DevArgs& A, const float* __restrict__ arr, const int32_t* nb,
                                            int c, float* buf, uint64_t* bar, int j) {
  if (j >= kStageRuns) return;
  const int rx = (c >> 2) & 1, ry = (c >> 1) & 1, rz = c & 1;
  const int lx = j / 27, ly = (j / 3) % 9, run = j % 3;
  const int x = 2 * lx + rx - 5, y = 2 * ly + ry - 5;
  // lattice z range of the run: z = 2 lz + rz - 5 in [-5, 0), [0, 8), [8, 13)
  const int z1 = rz ? 2 : 3, z2 = rz ? 6 : 7;
  const int lz0 = run == 0 ? 0 : (run == 1 ? z1 : z2);
  const int lz1 = run == 0 ? z1 : (run == 1 ? z2 : 9);
  const int z = 2 * lz0 + rz - 5;
  const int32_t sB = nb[((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)];
  float* dst = buf + (lx * kStageSX + ly * kStageSY + lz0) * W;
  const uint32_t bytes = uint32_t(lz1 - lz0) * uint32_t(W * 4);
  if (sB >= 0 && !FMM_BAD(A, int64_t(sB) * kCells < A.n_cell)) {
    // the run's cells are consecutive in the neighbour's parity-major order (cidx)
    const int64_t row = int64_t(sB) * kCells + cidx(x & 7, y & 7, z & 7);
    mbar_arrive_tx(bar, bytes);
    bulk_g2s(dst, arr + row * W, bytes, bar);
  } else {
    for (int k = 0; k < int(bytes / 4); ++k) dst[k] = 0.0f;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(bar);
  }
}

template <typename T, bool AREF>
__device__ __forceinline__ void src_far(T* L, T s0, T s1x, T s1y, T s1z, const T* S2, const T* S3,
                                        T x, T y, T z);
__device__ __forceinline__ void store_src_expansion(const DevArgs& A, int64_t i, const float* L, int n);

// Record width per cell of the staged arrays: the FP32 moments (20 floats) or, for the
// time-derivative solve, the source moments S0, S1, S2', S3' followed by rho's centre-of-mass
// offset (28 floats, padded so that 7 w mod 8 over a quarter warp's cells stays distinct:
// 7 (ic + 84 ia) mod 8 = {0, 7, 6, 5} + {0, 4}).
template <bool SRC>
struct StageW {
  static constexpr int W = SRC ? 28 : 20;
  static constexpr int kBufBytes = kStageCells * W * 4;
};
constexpr int kStageSmemSrc = 2 * StageW<true>::kBufBytes;

// One block per refined subgrid of a level >= 1 (the list `subs`): the same pairs and
// correction as m2l_level<float>, with the partners read from shared memory.  SRC: the
// time-derivative solve's source expansions of the same targets (as m2l_level_src<float>).
template <bool SRC>
__global__ void __launch_bounds__(kStageThreads, 1) k_m2l_stage(DevArgs A, const int32_t* __restrict__ subs,
                                                                 int amc) {
  constexpr int W = StageW<SRC>::W;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  float* buf0 = reinterpret_cast<float*>(stage_smem);
  float* buf1 = reinterpret_cast<float*>(stage_smem + StageW<SRC>::kBufBytes);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int32_t nb[27];
  const float* __restrict__ arr = SRC ? A.src32 : A.mom32;
  const int32_t s = subs[blockIdx.x];
  const int t = threadIdx.x;
  if (t < 27) nb[t] = A.nbr[27 * s + t];
  if (t == 0) {
    mbar_init(&bar[0], kStageRuns);
    mbar_init(&bar[1], kStageRuns);
    mbar_fence_init();
  }
  const int w = t >> 5, lane = t & 31;
  const int parity = w >> 1;
  const int ia = ((w & 1) << 1) | ((lane >> 2) & 1), ib = lane >> 3, ic = lane & 3;
  const int a = 2 * ia + ((parity >> 2) & 1), b = 2 * ib + ((parity >> 1) & 1), c = 2 * ic + (parity & 1);
  const int64_t iA = int64_t(s) * kCells + cidx(a, b, c);
  Target<float, true> S;
  float Ls[SRC ? 20 : 1];
  if constexpr (SRC) {
#pragma unroll
    for (int k = 0; k < 20; ++k) Ls[k] = 0.0f;
    S.dAx = A.mom32[iA * 20 + 1];
    S.dAy = A.mom32[iA * 20 + 2];
    S.dAz = A.mom32[iA * 20 + 3];
  } else {
    load_target<float, true>(S, A, A.mom32, iA, amc != 0);
  }
  const float h = cell_h<float>(A.level[s]);
  const int base = (ia * kStageSX + ib * kStageSY + ic) * W;
  const float4* __restrict__ tab = A.stage_tab + parity * kLeafCap;
  const int32_t* __restrict__ seg = A.stage_seg + parity * 9;
  __syncthreads();
  stage_issue<W>(A, arr, nb, 0, buf0, &bar[0], t);
  for (int cl = 0; cl < 8; ++cl) {
    const bool ok = mbar_wait_bounded(&bar[cl & 1], uint32_t((cl >> 1) & 1), A.wait_cycles);
    // block-uniform decision; also makes the zero fills of class cl visible and frees the other
    // buffer (every thread has finished class cl - 1)
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(A.status, 4);
      // the copies in flight are class cl's (class cl + 1 is issued after this wait): give them
      // time to land before the block's shared memory is released
      mbar_wait_bounded(&bar[cl & 1], uint32_t((cl >> 1) & 1), kStageWaitCycles);
      return;
    }
    if (cl < 7) stage_issue<W>(A, arr, nb, cl + 1, (cl & 1) ? buf0 : buf1, &bar[(cl + 1) & 1], t);
    const float* __restrict__ B = ((cl & 1) ? buf1 : buf0) + base;
    const int q1 = __ldg(seg + cl + 1);
    const int qb = __ldg(seg + cl);
    float4 e_next = __ldg(tab + min(qb, kLeafCap - 1));  // loaded while the previous is evaluated
    for (int q0 = qb; q0 < q1; q0 += kFlush) {
      const int qe = min(q0 + kFlush, q1);
      for (int q = q0; q < qe; ++q) {
        const float4 e = e_next;
        e_next = __ldg(tab + min(q + 1, q1 - 1));
        if (FMM_BAD(A, unsigned(base / W + __float_as_int(e.w)) < unsigned(kStageCells))) continue;
        const float4* m = reinterpret_cast<const float4*>(B + __float_as_int(e.w) * W);
        float Mv[W];
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
          const float4 v = m[k];
          Mv[4 * k] = v.x;
          Mv[4 * k + 1] = v.y;
          Mv[4 * k + 2] = v.z;
          Mv[4 * k + 3] = v.w;
        }
        if constexpr (SRC) {
          const float x = fmaf(-e.x, h, S.dAx), y = fmaf(-e.y, h, S.dAy), z = fmaf(-e.z, h, S.dAz);
          src_far<float, true>(Ls, Mv[0], Mv[1], Mv[2], Mv[3], Mv + 4, Mv + 10, x - Mv[20], y - Mv[21],
                               z - Mv[22]);
        } else {
          interact_rr_v<float>(S, Mv, e.x, e.y, e.z, h);
        }
      }
      if constexpr (!SRC) flush(S);
    }
  }
  if constexpr (SRC) {
    complete_traceless(Ls);
    store_src_expansion(A, iA, Ls, 20);
  } else {
    finish_rr(S);
    store_own<float, true>(A, S, iA);
  }
}

// The same work as k_m2l_stage with the staging decoupled from the evaluation: a 17th warp only
// issues the copies, and each of the two buffers has a "full" barrier (the class's copies have
// landed) and an "empty" barrier (all 16 evaluating warps are done with it).  The producer issues
// class c + 2 into a buffer as soon as every warp has finished class c, so a warp that is done
// with a class moves on to the next one at once; it waits only when it gets a whole class ahead
// of the slowest warp.  (k_m2l_stage makes all warps meet at the end of every class, and the
// uneven split of a parity's stencil over the 8 partner classes makes them wait for each other.)
// Every wait is bounded: a wait that runs out records FMM_ERR_TIMEOUT; the producer then waits
// (bounded) for the copies it issued before it leaves, so no copy lands after the block is gone.
constexpr int kStagePipeThreads = kStageThreads + 32;

template <int W>
__device__ __forceinline__ void stage_issue_warp(const DevArgs& A, const float* __restrict__ arr,
                                                 const int32_t* nb, int c, float* buf, uint64_t* bar,
                                                 int lane) {
  // lane takes runs lane, lane + 32, ...; it zero-fills its runs in absent neighbours, then
  // announces the bytes of its bulk copies with one arrive, then issues them
  uint32_t bytes = 0;
  for (int j = lane; j < kStageRuns; j += 32) {
    const int rx = (c >> 2) & 1, ry = (c >> 1) & 1, rz = c & 1;
    const int lx = j / 27, ly = (j / 3) % 9, run = j % 3;
    const int x = 2 * lx + rx - 5, y = 2 * ly + ry - 5;
    const int z1 = rz ? 2 : 3, z2 = rz ? 6 : 7;
    const int lz0 = run == 0 ? 0 : (run == 1 ? z1 : z2);
    const int lz1 = run == 0 ? z1 : (run == 1 ? z2 : 9);
    const int z = 2 * lz0 + rz - 5;
    const int32_t sB = nb[((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)];
    const uint32_t n = uint32_t(lz1 - lz0) * uint32_t(W * 4);
    if (sB >= 0 && !FMM_BAD(A, int64_t(sB) * kCells < A.n_cell)) {
      bytes += n;
    } else {
      float* dst = buf + (lx * kStageSX + ly * kStageSY + lz0) * W;
      for (int k = 0; k < int(n / 4); ++k) dst[k] = 0.0f;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_tx(bar, bytes);
  for (int j = lane; j < kStageRuns; j += 32) {
    const int rx = (c >> 2) & 1, ry = (c >> 1) & 1, rz = c & 1;
    const int lx = j / 27, ly = (j / 3) % 9, run = j % 3;
    const int x = 2 * lx + rx - 5, y = 2 * ly + ry - 5;
    const int z1 = rz ? 2 : 3, z2 = rz ? 6 : 7;
    const int lz0 = run == 0 ? 0 : (run == 1 ? z1 : z2);
    const int lz1 = run == 0 ? z1 : (run == 1 ? z2 : 9);
    const int z = 2 * lz0 + rz - 5;
    const int32_t sB = nb[((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)];
    if (sB < 0 || int64_t(sB) * kCells >= A.n_cell) continue;  // (the first pass zero-filled it)
    const int64_t row = int64_t(sB) * kCells + cidx(x & 7, y & 7, z & 7);
    bulk_g2s(buf + (lx * kStageSX + ly * kStageSY + lz0) * W, arr + row * W,
             uint32_t(lz1 - lz0) * uint32_t(W * 4), bar);
  }
}

__global__ void __launch_bounds__(kStagePipeThreads, 1) k_m2l_stage_pipe(DevArgs A, const int32_t* __restrict__ subs,
                                                                         int amc) {
  constexpr int W = 20;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  float* const buf0 = reinterpret_cast<float*>(stage_smem);
  constexpr int kBufFloats = StageW<false>::kBufBytes / 4;  // buffer b starts at buf0 + b kBufFloats
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ int32_t nb[27];
  const int32_t s = subs[blockIdx.x];
  const int t = threadIdx.x;
  if (t < 27) nb[t] = A.nbr[27 * s + t];
  if (t == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], 32);                      // one arrival per producer lane
      mbar_init(&empty[b], kStageThreads / 32);     // one arrival per evaluating warp
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int w = t >> 5, lane = t & 31;
  if (w == kStageThreads / 32) {
    // producer: classes 0 and 1 at once, class c >= 2 once class c - 2 is done with
    int last = -1;  // the last class issued
    for (int cl = 0; cl < 8; ++cl) {
      const int b = cl & 1;
      if (cl >= 2 && !mbar_sleep_bounded(&empty[b], uint32_t(((cl - 2) >> 1) & 1), A.wait_cycles)) {
        if (lane == 0) atomicOr(A.status, 4);
        break;
      }
      stage_issue_warp<W>(A, A.mom32, nb, cl, buf0 + b * kBufFloats, &full[b], lane);
      last = cl;
    }
    // every copy this warp issued has landed before the block's shared memory is released: the
    // last class issued into each buffer (earlier ones were waited for before it was reissued)
    for (int cl = last; cl >= 0 && cl >= last - 1; --cl)
      mbar_sleep_bounded(&full[cl & 1], uint32_t((cl >> 1) & 1), kStageWaitCycles);
    return;
  }
  const int parity = w >> 1;
  const int ia = ((w & 1) << 1) | ((lane >> 2) & 1), ib = lane >> 3, ic = lane & 3;
  const int a = 2 * ia + ((parity >> 2) & 1), b_ = 2 * ib + ((parity >> 1) & 1), c = 2 * ic + (parity & 1);
  const int64_t iA = int64_t(s) * kCells + cidx(a, b_, c);
  Target<float, true> S;
  load_target<float, true>(S, A, A.mom32, iA, amc != 0);
  const float h = cell_h<float>(A.level[s]);
  const int base = (ia * kStageSX + ib * kStageSY + ic) * W;
  const float4* __restrict__ tab = A.stage_tab + parity * kLeafCap;
  const int32_t* __restrict__ seg = A.stage_seg + parity * 9;
  for (int cl = 0; cl < 8; ++cl) {
    const int bi = cl & 1;
    // every lane waits (the wait is also what makes the producer's zero fills visible)
    if (!mbar_sleep_bounded(&full[bi], uint32_t((cl >> 1) & 1), A.wait_cycles)) {
      atomicOr(A.status, 4);
      return;  // the producer waits for its own copies before the block ends
    }
    const float* __restrict__ B = buf0 + bi * kBufFloats + base;
    const int q1 = __ldg(seg + cl + 1);
    const int qb = __ldg(seg + cl);
    float4 e_next = __ldg(tab + min(qb, kLeafCap - 1));
    for (int q0 = qb; q0 < q1; q0 += kFlush) {
      const int qe = min(q0 + kFlush, q1);
      for (int q = q0; q < qe; ++q) {
        const float4 e = e_next;
        e_next = __ldg(tab + min(q + 1, q1 - 1));
        if (FMM_BAD(A, unsigned(base / W + __float_as_int(e.w)) < unsigned(kStageCells))) continue;
        const float4* m = reinterpret_cast<const float4*>(B + __float_as_int(e.w) * W);
        float Mv[W];
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
          const float4 v = m[k];
          Mv[4 * k] = v.x;
          Mv[4 * k + 1] = v.y;
          Mv[4 * k + 2] = v.z;
          Mv[4 * k + 3] = v.w;
        }
        interact_rr_v<float>(S, Mv, e.x, e.y, e.z, h);
      }
      flush(S);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[bi]);
  }
  finish_rr(S);
  store_own<float, true>(A, S, iA);
}

// Four consecutive table values (16-byte aligned) in vector loads.
__device__ __forceinline__ void load4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  a = v.x;
  b = v.y;
  c = v.z;
  d = v.w;
}
__device__ __forceinline__ void load4(const dfloat* p, dfloat& a, dfloat& b, dfloat& c, dfloat& d) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  const float4 w = __ldg(reinterpret_cast<const float4*>(p) + 1);
  a = dfloat(v.x, v.y);
  b = dfloat(v.z, v.w);
  c = dfloat(w.x, w.y);
  d = dfloat(w.z, w.w);
}
__device__ __forceinline__ void load4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  const double2 w = __ldg(reinterpret_cast<const double2*>(p) + 1);
  a = v.x;
  b = v.y;
  c = w.x;
  d = w.y;
}

template <typename T>
struct LeafTab;
template <>
struct LeafTab<double> {
  static __device__ __forceinline__ const double* get(const DevArgs& A) { return A.ltab_k64; }
};
template <>
struct LeafTab<float> {
  static __device__ __forceinline__ const float* get(const DevArgs& A) { return A.ltab_k32; }
};
template <>
struct LeafTab<dfloat> {
  static __device__ __forceinline__ const dfloat* get(const DevArgs& A) { return A.ltab_kff; }
};

// Leaf subgrids at levels >= 1.  A leaf cell and a leaf partner at the same level are two point
// masses at their geometric centres, R = -d dx exactly, so their interaction (multipole or direct,
// the same monopole formula) is 1/|d| and d/|d|^3 from a per-offset table times the partner's
// mass: L0 -= m / (|d| dx), L1 -= m d / (|d|^3 dx^2).  The masses of the subgrid and of the 5-cell
// rim of its neighbours are staged in shared memory (0 for cells of refined or absent
// neighbours, whose partners the boundary pass of k_m2l_ref adds afterwards).
// SRC: the time-derivative solve -- the halo holds the source values and only L0 is formed.
template <typename T, bool SRC>
__global__ void __launch_bounds__(kLeafThreads) k_m2l_leaf(DevArgs A, const int32_t* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char leaf_smem[];
  T* hm = reinterpret_cast<T*>(leaf_smem);  // kHaloWords
  __shared__ int32_t nb[27];
  const int32_t s = work[blockIdx.x];
  const int t = threadIdx.x;
  if (t < 27) {
    int32_t q = A.nbr[27 * s + t];
    nb[t] = (q >= 0 && A.leaf[q]) ? q : -1;
  }
  __syncthreads();
  // masses: component 0 of the (component-major) FP64 or source arrays, or the FP32 mass array
  const T* __restrict__ M;
  if constexpr (SRC) M = SrcView<T>::get(A);
  else M = LeafMass<T>::get(A);
  const int64_t N = A.n_cell;
  constexpr int kH3 = kHalo * kHalo * kHalo, kFill = 8;  // halo loads in flight per thread
  for (int i0 = t; i0 < kH3; i0 += kFill * kLeafThreads) {
    T v[kFill];
    int dst[kFill];
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int i = i0 + u * kLeafThreads;
      const int hx = i / (kHalo * kHalo), r = i - hx * (kHalo * kHalo), hy = r / kHalo, hz = r - hy * kHalo;
      const int x = hx - 5, y = hy - 5, z = hz - 5;
      const int32_t q = i < kH3 ? nb[((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)] : -1;
      dst[u] = i < kH3 ? ((hx & 1) << 2 | (hy & 1) << 1 | (hz & 1)) * kHaloPar + (hx >> 1) * kHaloSX +
                             (hy >> 1) * kHaloSY + (hz >> 1)
                       : -1;
      v[u] = q >= 0 && !FMM_BAD(A, int64_t(q) * kCells < N) ? M[int64_t(q) * kCells + cidx(x & 7, y & 7, z & 7)] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kFill; ++u)
      if (dst[u] >= 0) hm[dst[u]] = v[u];
  }
  __syncthreads();
  const T h = cell_h<T>(A.level[s]);
  // warp = parity class; lane = lattice cell (i, j, k), k < 2; second target k + 2
  const int parity = t >> 5, lane = t & 31;
  const int px = (parity >> 2) & 1, py = (parity >> 1) & 1, pz = parity & 1;
  const int li = lane >> 3, lj = (lane >> 1) & 3, lk = lane & 1;
  const int a = 2 * li + px, b = 2 * lj + py, c0 = 2 * lk + pz;  // second target: c0 + 4
  const int base0 = li * kHaloSX + lj * kHaloSY + lk;
  const int base1 = base0 + 2;
  const int32_t* __restrict__ toff = A.ltab_off + parity * kLeafCap;
  const T* __restrict__ tk = LeafTab<T>::get(A) + int64_t(parity) * kLeafCap * 4;
  const int n_tab = A.n_stencil + A.n_near;
  T s0 = 0, sx = 0, sy = 0, sz = 0, u0 = 0, ux = 0, uy = 0, uz = 0;
#pragma unroll 4
  for (int q = 0; q < n_tab; ++q) {
    const int off = __ldg(toff + q);
    if (FMM_BAD(A, off >= 0 && base1 + off < kHaloWords)) continue;
    T k0, kx, ky, kz;
    load4(tk + 4 * q, k0, kx, ky, kz);
    const T m0 = hm[base0 + off], m1 = hm[base1 + off];
    s0 = fma(m0, k0, s0);
    u0 = fma(m1, k0, u0);
    if (!SRC) {
      sx = fma(m0, kx, sx);
      sy = fma(m0, ky, sy);
      sz = fma(m0, kz, sz);
      ux = fma(m1, kx, ux);
      uy = fma(m1, ky, uy);
      uz = fma(m1, kz, uz);
    }
  }
  const T ih = T(1) / h, ih2 = ih * ih;
  const int64_t i0 = int64_t(s) * kCells + cidx(a, b, c0);
  const int64_t i1 = int64_t(s) * kCells + cidx(a, b, c0 + 4);
  if (SRC) {
    if (sizeof(T) == 8) {
      A.sloc[i0] = -double(s0 * ih);
      A.sloc[i1] = -double(u0 * ih);
    } else {
      A.sloc32[i0] = -float(s0 * ih);
      A.sloc32[i1] = -float(u0 * ih);
    }
    return;
  }
  if (sizeof(T) == 8) {
    double* L = reinterpret_cast<double*>(A.loc);
    L[i0] = -double(s0 * ih);
    L[N + i0] = -double(sx * ih2);
    L[2 * N + i0] = -double(sy * ih2);
    L[3 * N + i0] = -double(sz * ih2);
    L[i1] = -double(u0 * ih);
    L[N + i1] = -double(ux * ih2);
    L[2 * N + i1] = -double(uy * ih2);
    L[3 * N + i1] = -double(uz * ih2);
  } else {
    float* L = A.loc32;
    L[i0] = -float(s0 * ih);
    L[N + i0] = -float(sx * ih2);
    L[2 * N + i0] = -float(sy * ih2);
    L[3 * N + i0] = -float(sz * ih2);
    L[i1] = -float(u0 * ih);
    L[N + i1] = -float(ux * ih2);
    L[2 * N + i1] = -float(uy * ih2);
    L[3 * N + i1] = -float(uz * ih2);
  }
  A.ac[i0] = A.ac[N + i0] = A.ac[2 * N + i0] = 0.0;
  A.ac[i1] = A.ac[N + i1] = A.ac[2 * N + i1] = 0.0;
}

// FP32 form of k_m2l_leaf: the same pairs, with the shared-memory and table traffic per
// multiply-add cut (the FP32 kernel is bound by L1 / shared-memory wavefronts, not by its
// arithmetic).  A block holds two leaf subgrids (two halos); warp w = parity class w of both,
// lanes 0-15 the first subgrid's and 16-31 the second's lattice cells (i, j) = (lane >> 2 & 3,
// lane & 3), each lane the four targets k = 0..3 along z.  Every lane of a warp reads the same
// table entry; the offsets come four to a 16-byte load (the tables are zero-padded, so the loop
// runs to a multiple of four).  The second halo starts one word past the first, so the two half
// warps fall on the even and the odd banks: lattice offsets 120 i + 10 j are the 16 even banks.
// NSUB leaf subgrids per block (2 or 4, a tile parameter of the autotuner): warp w takes parity
// class w % 8 of the pair of subgrids 2 (w / 8), 2 (w / 8) + 1, one per half warp.
constexpr int kLeaf4Threads = 256;  // per pair of subgrids
template <int NSUB>
constexpr int leaf4_smem() { return (NSUB * kHaloWords + NSUB - 1) * 4; }
constexpr int kLeaf4Smem = leaf4_smem<2>();
template <bool SRC, int NSUB = 2>
__global__ void __launch_bounds__(kLeaf4Threads * NSUB / 2) k_m2l_leaf4(DevArgs A, const int32_t* __restrict__ work,
                                                                       int64_t n_work) {
  constexpr int NT = kLeaf4Threads * NSUB / 2;
  extern __shared__ __align__(16) float leaf4_smem[];
  __shared__ int32_t nb[NSUB][27];
  __shared__ int32_t sub[NSUB];
  const int t = threadIdx.x;
  if (t < NSUB) {
    const int64_t w = NSUB * int64_t(blockIdx.x) + t;
    sub[t] = w < n_work ? work[w] : -1;
  }
  __syncthreads();
  if (t < 27 * NSUB) {
    const int h = t / 27, k = t % 27;
    int32_t q = sub[h] >= 0 ? A.nbr[27 * sub[h] + k] : -1;
    nb[h][k] = (q >= 0 && A.leaf[q]) ? q : -1;
  }
  __syncthreads();
  const float* __restrict__ M = SRC ? A.smom32 : A.m32;
  constexpr int kH3 = kHalo * kHalo * kHalo;
  constexpr int kFill = 8;  // halo loads in flight per thread
  for (int i0 = t; i0 < NSUB * kH3; i0 += kFill * NT) {
    float v[kFill];
    int dst[kFill];
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int i = i0 + u * NT;
      const int h = i / kH3, j = i - h * kH3;
      const int hx = j / (kHalo * kHalo), r = j - hx * (kHalo * kHalo), hy = r / kHalo, hz = r - hy * kHalo;
      const int x = hx - 5, y = hy - 5, z = hz - 5;
      const int32_t q = i < NSUB * kH3 ? nb[h][((x >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((z >> 3) + 1)] : -1;
      dst[u] = i < NSUB * kH3 ? h * (kHaloWords + 1) + ((hx & 1) << 2 | (hy & 1) << 1 | (hz & 1)) * kHaloPar +
                                    (hx >> 1) * kHaloSX + (hy >> 1) * kHaloSY + (hz >> 1)
                              : -1;
      v[u] = q >= 0 && !FMM_BAD(A, int64_t(q) * kCells < A.n_cell)
                 ? __ldg(M + int64_t(q) * kCells + cidx(x & 7, y & 7, z & 7))
                 : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kFill; ++u)
      if (dst[u] >= 0) leaf4_smem[dst[u]] = v[u];
  }
  __syncthreads();
  const int warp = t >> 5, parity = warp & 7, lane = t & 31;
  const int hsub = 2 * (warp >> 3) + (lane >> 4);
  const int32_t s = sub[hsub];
  const int px = (parity >> 2) & 1, py = (parity >> 1) & 1, pz = parity & 1;
  const int li = (lane >> 2) & 3, lj = lane & 3;
  const float* __restrict__ hm = leaf4_smem + hsub * (kHaloWords + 1) + li * kHaloSX + lj * kHaloSY;
  const int4* __restrict__ toff = reinterpret_cast<const int4*>(A.ltab_off + parity * kLeafCap);
  const float4* __restrict__ tk = reinterpret_cast<const float4*>(A.ltab_k32 + int64_t(parity) * kLeafCap * 4);
  const int n4 = (A.n_stencil + A.n_near + 3) >> 2;
  float s0[4] = {0, 0, 0, 0}, sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0}, sz[4] = {0, 0, 0, 0};
  // the next group's table entries are loaded while this group's are used
  int4 o = __ldg(toff);
  float4 kv[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) kv[u] = __ldg(tk + u);
  for (int q4 = 0; q4 < n4; ++q4) {
    const int qn = min(q4 + 1, n4 - 1);
    const int4 on = __ldg(toff + qn);
    float4 kn[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) kn[u] = __ldg(tk + 4 * qn + u);
    int off[4] = {o.x, o.y, o.z, o.w};
#ifdef FMM_BOUNDS_CHECK
    for (int u = 0; u < 4; ++u)
      if (FMM_BAD(A, off[u] >= 0 && li * kHaloSX + lj * kHaloSY + off[u] + 3 < kHaloWords)) off[u] = 0;
#endif
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float m = hm[off[u] + k];
        s0[k] = fmaf(m, kv[u].x, s0[k]);
        if (!SRC) {
          sx[k] = fmaf(m, kv[u].y, sx[k]);
          sy[k] = fmaf(m, kv[u].z, sy[k]);
          sz[k] = fmaf(m, kv[u].w, sz[k]);
        }
      }
    }
    o = on;
#pragma unroll
    for (int u = 0; u < 4; ++u) kv[u] = kn[u];
  }
  if (s < 0) return;
  const float h = cell_dx32(A.level[s]);
  const float ih = 1.0f / h, ih2 = ih * ih;
  const int64_t N = A.n_cell;
  const int a = 2 * li + px, b = 2 * lj + py;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = int64_t(s) * kCells + cidx(a, b, 2 * k + pz);
    if (SRC) {
      A.sloc32[i] = -s0[k] * ih;
      continue;
    }
    A.loc32[i] = -s0[k] * ih;
    A.loc32[N + i] = -sx[k] * ih2;
    A.loc32[2 * N + i] = -sy[k] * ih2;
    A.loc32[3 * N + i] = -sz[k] * ih2;
    A.ac[i] = A.ac[N + i] = A.ac[2 * N + i] = 0.0;
  }
}

// Exact Taylor shift of a 3rd-order expansion P about X to the point X + r, added onto L:
//   L0 += P0 + P1.r + 1/2 r.P2.r + 1/6 P3(r,r,r),  L1 += P1 + P2 r + 1/2 P3(r,r),
//   L2 += P2 + P3 r,  L3 += P3.
template <typename T>
__device__ __forceinline__ void shift_add(const T* P, T rx, T ry, T rz, T* L) {
  T qx, qy, qz;
  sym3_rr<T>(P + 10, rx, ry, rz, qx, qy, qz);
  // L2 r
  T l2x = P[4] * rx + P[5] * ry + P[6] * rz;
  T l2y = P[5] * rx + P[7] * ry + P[8] * rz;
  T l2z = P[6] * rx + P[8] * ry + P[9] * rz;
  L[0] += P[0] + P[1] * rx + P[2] * ry + P[3] * rz + T(0.5) * (rx * l2x + ry * l2y + rz * l2z) +
          (rx * qx + ry * qy + rz * qz) * T(1.0 / 6.0);
  L[1] += P[1] + l2x + T(0.5) * qx;
  L[2] += P[2] + l2y + T(0.5) * qy;
  L[3] += P[3] + l2z + T(0.5) * qz;
  // (L3 r)_ab, L3: xxx0 xxy1 xxz2 xyy3 xyz4 xzz5 yyy6 yyz7 yzz8 zzz9
  const T* Q = P + 10;
  L[4] += P[4] + Q[0] * rx + Q[1] * ry + Q[2] * rz;
  L[5] += P[5] + Q[1] * rx + Q[3] * ry + Q[4] * rz;
  L[6] += P[6] + Q[2] * rx + Q[4] * ry + Q[5] * rz;
  L[7] += P[7] + Q[3] * rx + Q[6] * ry + Q[7] * rz;
  L[8] += P[8] + Q[4] * rx + Q[7] * ry + Q[8] * rz;
  L[9] += P[9] + Q[5] * rx + Q[8] * ry + Q[9] * rz;
#pragma unroll
  for (int k = 10; k < 20; ++k) L[k] += P[k];
}

// Downward pass.  Expansions: FP64 in the FP64 path; in the mixed path every expansion is FP32
// (own, shifted and total), while the correction accelerations stay FP64 sums.
// SRC: the time-derivative solve's source expansions (same centres, no correction term).
template <bool MIXED, bool SRC = false>
struct Down {
  using T = typename std::conditional<MIXED, float, double>::type;
  static __device__ __forceinline__ T ld(const DevArgs& A, int k, int64_t i) {
    if constexpr (MIXED) return (SRC ? A.sloc32 : A.loc32)[k * A.n_cell + i];
    else return (SRC ? A.sloc : A.loc)[k * A.n_cell + i];
  }
  static __device__ __forceinline__ void st(const DevArgs& A, int k, int64_t i, T v) {
    if constexpr (MIXED) (SRC ? A.sloc32 : A.loc32)[k * A.n_cell + i] = v;
    else (SRC ? A.sloc : A.loc)[k * A.n_cell + i] = v;
  }
  static __device__ __forceinline__ T com(const DevArgs& A, int k, int64_t i) {
    if constexpr (MIXED) return A.mom32[i * 20 + k];
    else return A.mom[k * A.n_cell + i];
  }
};

// Writes phi and g of leaf cell (subgrid s, cell (a, b, c)) in the caller's arrays.
__device__ __forceinline__ void store_leaf(const DevArgs& A, int32_t s, int a, int b, int c,
                                           double phi_v, double gx, double gy, double gz) {
  const int32_t ls = A.leaf_ord[s];
  if (FMM_BAD(A, ls >= 0 && int64_t(ls) * kCells < A.n_leaf_cells)) return;
  const int k = A.leaf_tree[ls];
  if (FMM_BAD(A, k >= 0 && k < A.n_roots)) return;
  const int64_t o = (int64_t(ls) - A.tree_leaf_off[k]) * kCells + (a * 8 + b) * 8 + c;
  double* __restrict__ phi = A.io[k].phi;
  double* __restrict__ g = A.io[k].g;
  phi[o] = phi_v;
  g[3 * o] = gx;
  g[3 * o + 1] = gy;
  g[3 * o + 2] = gz;
}

// dphi/dt of leaf cell (subgrid s, cell (a, b, c)) in the caller's array.
__device__ __forceinline__ void store_leaf_dt(const DevArgs& A, int32_t s, int a, int b, int c, double v) {
  const int32_t ls = A.leaf_ord[s];
  const int k = A.leaf_tree[ls];
  A.io[k].phidot[(int64_t(ls) - A.tree_leaf_off[k]) * kCells + (a * 8 + b) * 8 + c] = v;
}

// Level 0: each root cell's expansion is the fixed-order sum of its kRootChunks partial sums.
// A refined root keeps it as its total, one thread per (root, component, cell) -- 20 expansion
// and 3 correction components; a leaf root is evaluated by the component-0 thread of each cell
// (phi = L0, g = -L1 + a_c).
constexpr int kRootComps = 23;
template <bool MIXED, bool SRC>
__global__ void k_root_total(DevArgs A) {
  using T = typename Down<MIXED>::T;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(A.n_roots) * kRootComps * kCells) return;
  const int loc = int(t & 511);
  const int comp = int((t >> 9) % kRootComps);
  const int32_t s = int32_t((t >> 9) / kRootComps);  // roots are subgrids 0 .. n_roots - 1
  const int64_t i = int64_t(s) * kCells + loc;
  // partial sum of component k (0..22) of chunk ch
  auto part = [&](int ch, int k) -> double {
    const int64_t pc = int64_t(s) * kRootChunks + ch;
    if (!MIXED) return A.root_part[(pc * 23 + k) * kCells + loc];
    if (k < 20) return double(A.root_part32[(pc * 20 + k) * kCells + loc]);
    return A.root_part_ac[(pc * 3 + (k - 20)) * kCells + loc];
  };
  if (A.leaf[s]) {
    if (comp != 0) return;
    double L[4] = {0.0, 0.0, 0.0, 0.0}, ax = 0.0, ay = 0.0, az = 0.0;
    for (int ch = 0; ch < kRootChunks; ++ch) {
      for (int k = 0; k < 4; ++k) L[k] += part(ch, k);
      if (!SRC) {
        ax += part(ch, 20);
        ay += part(ch, 21);
        az += part(ch, 22);
      }
    }
    int a, b, c;
    cdecode(loc, a, b, c);
    if (SRC) store_leaf_dt(A, s, a, b, c, L[0]);
    else store_leaf(A, s, a, b, c, L[0], -L[1] + ax, -L[2] + ay, -L[3] + az);
    return;
  }
  if (SRC && comp >= 20) return;
  double v = 0.0;
  for (int ch = 0; ch < kRootChunks; ++ch) v += part(ch, comp);
  if (comp < 20) Down<MIXED, SRC>::st(A, comp, i, T(v));
  else A.ac[(comp - 20) * A.n_cell + i] = v;
}

// Levels >= 1, 64 threads per block.  Blocks [0, n_ref_blocks): 8 per refined subgrid of level
// lev, one thread per cell: total = own + the parent's total shifted from the parent's centre of
// mass to the cell's (r = X_A - X_P).  The other blocks: one per (refined parent subgrid,
// octant) whose child subgrid is a leaf (of any level: lev is then the child's), one thread per
// parent cell and its 8 leaf children.  The parent's total is shifted once to the parent cell's
// geometric centre; there the children sit at s w (s = +-1 per axis, w = dx_l / 2), and the
// expansion's value and gradient at the 8 children are sums of the 8 Walsh functions
// prod_(a in k) s_a.  With L2, L3 traceless up to rounding (t_a = L3_abb, kept for exactness):
//   phi(s w) = [L0 + w^2/2 tr L2] + w sum_a s_a [L1_a + w^2 (t_a / 2 - L3_aaa / 3)]
//              + w^2 sum_(a<b) s_a s_b L2_ab + w^3 s_x s_y s_z L3_xyz,
//   dphi/dr_a (s w) = [L1_a + w^2 t_a / 2] + w sum_b s_b L2_ab + w^2 sum_(b<c) s_b s_c L3_abc,
// each evaluated at all 8 children by an inverse 8-point Walsh-Hadamard transform.
// One 64-thread work item of the downward pass (blk: the item's index, blockIdx.x of k_down).
template <bool MIXED, bool SRC>
__device__ __forceinline__ void down_item(const DevArgs& A, int lev, const int32_t* __restrict__ ref,
                                          int n_ref_blocks, const int32_t* __restrict__ octs, int blk) {
  using T = typename Down<MIXED>::T;
  using D = Down<MIXED, SRC>;
  const int64_t N = A.n_cell;
  if (blk < n_ref_blocks) {
    const int32_t s = ref[blk >> 3];
    if (FMM_BAD(A, s >= 0 && int64_t(s) * kCells < N && A.parent[s] >= 0)) return;
    const int loc = (blk & 7) * 64 + int(threadIdx.x);
    const int64_t i = int64_t(s) * kCells + loc;
    const int32_t Pn = A.parent[s];
    int a, b, c;
    cdecode(loc, a, b, c);
    const int ga = A.ijk[3 * s] * 8 + a, gb = A.ijk[3 * s + 1] * 8 + b, gc = A.ijk[3 * s + 2] * 8 + c;
    const int64_t ip = int64_t(Pn) * kCells + cidx((ga >> 1) - A.ijk[3 * Pn] * 8,
                                                   (gb >> 1) - A.ijk[3 * Pn + 1] * 8,
                                                   (gc >> 1) - A.ijk[3 * Pn + 2] * 8);
    T P[20], L[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) {
      P[k] = D::ld(A, k, ip);
      L[k] = D::ld(A, k, i);
    }
    const T h = cell_h<T>(lev), hh = T(0.5) * h;
    // r = X_A - X_P = ((g & 1) - 1/2) dx_l + delta_A - delta_P
    const T rx = ((ga & 1) ? hh : -hh) + Down<MIXED>::com(A, 1, i) - Down<MIXED>::com(A, 1, ip);
    const T ry = ((gb & 1) ? hh : -hh) + Down<MIXED>::com(A, 2, i) - Down<MIXED>::com(A, 2, ip);
    const T rz = ((gc & 1) ? hh : -hh) + Down<MIXED>::com(A, 3, i) - Down<MIXED>::com(A, 3, ip);
    shift_add<T>(P, rx, ry, rz, L);
#pragma unroll
    for (int k = 0; k < 20; ++k) D::st(A, k, i, L[k]);
    if (SRC) return;
    A.ac[i] += A.ac[ip];
    A.ac[N + i] += A.ac[N + ip];
    A.ac[2 * N + i] += A.ac[2 * N + ip];
    return;
  }
  const int32_t code = octs[blk - n_ref_blocks];
  const int32_t Pn = code >> 3;
  const int o = code & 7, u = int(threadIdx.x);
  if (FMM_BAD(A, Pn >= 0 && int64_t(Pn) * kCells < N && A.child[8 * Pn + o] >= 0 &&
                     int64_t(A.child[8 * Pn + o]) * kCells < N))
    return;
  int pa, pb, pc;
  octant_cell(o, u, pa, pb, pc);
  const int64_t ip = int64_t(Pn) * kCells + cidx(pa, pb, pc);
  const int32_t s = A.child[8 * Pn + o];
  lev = A.level[s];  // the leaf octants of every level share one launch
  T L[20], P[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) {
    P[k] = D::ld(A, k, ip);
    L[k] = T(0);
  }
  // to the parent cell's geometric centre: r = -delta_P
  shift_add<T>(P, -Down<MIXED>::com(A, 1, ip), -Down<MIXED>::com(A, 2, ip),
               -Down<MIXED>::com(A, 3, ip), L);
  const T w = T(0.5) * cell_h<T>(lev), w2 = w * w, w3 = w2 * w;
  const T tr2 = L[4] + L[7] + L[9];
  const T tx = L[10] + L[13] + L[15], ty = L[11] + L[16] + L[18], tz = L[12] + L[17] + L[19];
  // Walsh coefficients, index (x << 2) | (y << 1) | z
  T f[8], gxv[8], gyv[8], gzv[8];
  f[0] = L[0] + T(0.5) * w2 * tr2;
  f[4] = w * (L[1] + w2 * (T(0.5) * tx - L[10] * (T(1) / T(3))));
  f[2] = w * (L[2] + w2 * (T(0.5) * ty - L[16] * (T(1) / T(3))));
  f[1] = w * (L[3] + w2 * (T(0.5) * tz - L[19] * (T(1) / T(3))));
  f[6] = w2 * L[5];
  f[5] = w2 * L[6];
  f[3] = w2 * L[8];
  f[7] = w3 * L[14];
  if (SRC) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (!(e & bit)) {
          const T lo = f[e], hi = f[e | bit];
          f[e] = lo - hi;
          f[e | bit] = lo + hi;
        }
    const int64_t c0 = int64_t(s) * kCells + u;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      store_leaf_dt(A, s, 2 * (pa & 3) + ((e >> 2) & 1), 2 * (pb & 3) + ((e >> 1) & 1),
                    2 * (pc & 3) + (e & 1), to_f64(D::ld(A, 0, c0 + (e << 6)) + f[e]));
    return;
  }
  gxv[0] = L[1] + T(0.5) * w2 * tx;
  gxv[4] = w * L[4];
  gxv[2] = w * L[5];
  gxv[1] = w * L[6];
  gxv[6] = w2 * L[11];
  gxv[5] = w2 * L[12];
  gxv[3] = w2 * L[14];
  gxv[7] = T(0);
  gyv[0] = L[2] + T(0.5) * w2 * ty;
  gyv[4] = w * L[5];
  gyv[2] = w * L[7];
  gyv[1] = w * L[8];
  gyv[6] = w2 * L[13];
  gyv[5] = w2 * L[14];
  gyv[3] = w2 * L[17];
  gyv[7] = T(0);
  gzv[0] = L[3] + T(0.5) * w2 * tz;
  gzv[4] = w * L[6];
  gzv[2] = w * L[8];
  gzv[1] = w * L[9];
  gzv[6] = w2 * L[14];
  gzv[5] = w2 * L[15];
  gzv[3] = w2 * L[18];
  gzv[7] = T(0);
  // inverse transforms: value at child e (bit set = upper half, s = +1)
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (!(e & bit)) {
        T lo, hi;
        lo = f[e], hi = f[e | bit], f[e] = lo - hi, f[e | bit] = lo + hi;
        lo = gxv[e], hi = gxv[e | bit], gxv[e] = lo - hi, gxv[e | bit] = lo + hi;
        lo = gyv[e], hi = gyv[e | bit], gyv[e] = lo - hi, gyv[e | bit] = lo + hi;
        lo = gzv[e], hi = gzv[e | bit], gzv[e] = lo - hi, gzv[e | bit] = lo + hi;
      }
  const double apx = A.ac[ip], apy = A.ac[N + ip], apz = A.ac[2 * N + ip];
  const int64_t c0 = int64_t(s) * kCells + u;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t i = c0 + (e << 6);
    const T phi = D::ld(A, 0, i) + f[e];
    const T l1x = D::ld(A, 1, i) + gxv[e], l1y = D::ld(A, 2, i) + gyv[e],
            l1z = D::ld(A, 3, i) + gzv[e];
    const double ax = A.ac[i] + apx, ay = A.ac[N + i] + apy, az = A.ac[2 * N + i] + apz;
    store_leaf(A, s, 2 * (pa & 3) + ((e >> 2) & 1), 2 * (pb & 3) + ((e >> 1) & 1), 2 * (pc & 3) + (e & 1),
               to_f64(phi), ax - to_f64(l1x), ay - to_f64(l1y), az - to_f64(l1z));
  }
}
template <bool MIXED, bool SRC>
__global__ void __launch_bounds__(64) k_down(DevArgs A, int lev, const int32_t* __restrict__ ref,
                                             int n_ref_blocks, const int32_t* __restrict__ octs) {
  down_item<MIXED, SRC>(A, lev, ref, n_ref_blocks, octs, int(blockIdx.x));
}

// ----------------------------------------------------------------------------------------------
// the level passes as one persistent launch per direction
// ----------------------------------------------------------------------------------------------
// The upward pass after P2M (the octants with leaf children, then the octants with refined
// children level by level, finest first) and the downward pass below the root (the refined
// subgrids level by level, then every leaf octant) are sequences of phases, each of which needs
// the one before it complete on the whole tree.  Instead of one launch per phase, k_levels runs
// a whole sequence in one cooperative launch whose blocks stay resident: block b takes the
// phase's 64-thread work items b, b + gridDim.x, ..., and the blocks meet at a grid-wide barrier
// between phases.  The items are the same device functions as those of k_m2m and k_down, so the
// results are the same bit for bit.
constexpr int kMaxPhases = 40;
struct LevelPlan {
  int n;                               // phases
  int kind[kMaxPhases];                // 0 m2m_walsh, 1 m2m_lanes, 2 down (refined), 3 down (leaf octants)
  int lev[kMaxPhases];                 // kind 2: the level
  int items[kMaxPhases];               // 64-thread work items of the phase
  const int32_t* list[kMaxPhases];     // its octant or subgrid list
};

// Grid-wide barrier of a cooperative launch (all blocks resident): every block arrives with one
// atomic add on bar[0]; the last to arrive resets it and starts the next generation (bar[1]); the
// others wait for that for at most `limit` SM cycles.  The fences around the arrival make each
// block's writes before the barrier visible to every block after it.  False on time-out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;  // read before arriving: the generation cannot move until we have
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
      ok = 1;
    } else {
      const long long t0 = clock64();
      bool done = false;
      while (!(done = *gen != g) && clock64() - t0 <= limit) __nanosleep(32);
      ok = done ? 1 : 0;
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <bool MIXED>
__global__ void __launch_bounds__(64) k_levels(DevArgs A, LevelPlan P, int mode, unsigned* bar) {
  for (int p = 0; p < P.n; ++p) {
    if (p > 0 && !grid_barrier(bar, A.wait_cycles)) {
      if (threadIdx.x == 0) atomicOr(A.status, 16);  // FMM_ERR_TIMEOUT; the other blocks time out too
      return;
    }
    const int n = P.items[p], kind = P.kind[p];
    const int32_t* list = P.list[p];
    for (int b = int(blockIdx.x); b < n; b += int(gridDim.x)) {
      if (kind == 0) m2m_walsh(A, list, b, mode);
      else if (kind == 1) m2m_lanes(A, list, b, mode);
      else if (kind == 2) down_item<MIXED, false>(A, P.lev[p], list, n, nullptr, b);
      else down_item<MIXED, false>(A, 0, nullptr, 0, list, b);
    }
  }
}

// ----------------------------------------------------------------------------------------------
// time derivative of the potential (Sec. 2.1): the same operator applied to s = (d rho/dt) dx^3
// ----------------------------------------------------------------------------------------------
// The expansion centres stay rho's centres of mass, so about them a source cell has a dipole:
// S0 = sum s, S1 = sum s r, S2 = sum s r r, S3 = sum s r r r (r = x - X), stored in the order of
// the moments (S1 where rho's cells keep delta).  Expanding -s / |R + t - u| to total order 3:
//   L_k = -sum_(n <= 3 - k) (-1)^n / n! D^(k+n) : S_n.
// Only the potential is needed at the leaves; there is no correction term.

// index of (a, b) in the 6 stored components of a symmetric 2-tensor (xx xy xz yy yz zz)
__host__ __device__ constexpr int sym2_index(int a, int b) {
  return (a < b ? a : b) == 0 ? (a < b ? b : a) : ((a < b ? a : b) == 1 ? 2 + (a < b ? b : a) : 5);
}
// axis j (0..2) of the (a <= b <= c) triple of stored component k (0..9) of a symmetric
// 3-tensor (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz); a function rather than a device table, so
// that in unrolled loops the indices are compile-time constants and the operands stay in
// registers
__host__ __device__ constexpr int sym3_axis(int k, int j) {
  // component k's triple as the base-3 number 9 a + 3 b + c, six bits per component
  return int((0x69138d205102040ull >> (6 * k)) & 63u) / (j == 0 ? 9 : (j == 1 ? 3 : 1)) % 3;
}

// Exact shift of raw source moments c about X_c to the point X_c - r (r = X_c - X_new), added
// onto S:  S0 += c0,  S1 += c1 + c0 r,  S2 += c2 + r c1 + c1 r + c0 r r,
//          S3 += c3 + 3 sym(r c2) + 3 sym(r r c1) + c0 r r r.
__device__ __forceinline__ void src_shift_add(const double* c, const double* r, double* S) {
  S[0] += c[0];
#pragma unroll
  for (int a = 0; a < 3; ++a) S[1 + a] += c[1 + a] + c[0] * r[a];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b)
      S[4 + sym2_index(a, b)] += c[4 + sym2_index(a, b)] + r[a] * c[1 + b] + r[b] * c[1 + a] +
                                 c[0] * r[a] * r[b];
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const int a = sym3_axis(k, 0), b = sym3_axis(k, 1), cc = sym3_axis(k, 2);
    S[10 + k] += c[10 + k] + r[a] * c[4 + sym2_index(b, cc)] + r[b] * c[4 + sym2_index(a, cc)] +
                 r[cc] * c[4 + sym2_index(a, b)] + r[a] * r[b] * c[1 + cc] + r[a] * r[cc] * c[1 + b] +
                 r[b] * r[cc] * c[1 + a] + c[0] * r[a] * r[b] * r[cc];
  }
}

// Raw source moments of one refined cell, their detraced copy, and its FP32 copy (mixed path).
__device__ __forceinline__ void store_src_moments(const DevArgs& A, int64_t cell, const double* S,
                                                  int mixed) {
  const int64_t N = A.n_cell;
#pragma unroll
  for (int k = 0; k < 20; ++k) A.smom[k * N + cell] = S[k];
  const double tr3 = (S[4] + S[7] + S[9]) * (1.0 / 3.0);
  const double tx = (S[10] + S[13] + S[15]) * 0.2, ty = (S[11] + S[16] + S[18]) * 0.2,
               tz = (S[12] + S[17] + S[19]) * 0.2;
  const double T[20] = {S[0], S[1], S[2], S[3], S[4] - tr3, S[5], S[6], S[7] - tr3, S[8],
                        S[9] - tr3, S[10] - 3 * tx, S[11] - ty, S[12] - tz, S[13] - tx, S[14],
                        S[15] - tx, S[16] - 3 * ty, S[17] - tz, S[18] - ty, S[19] - 3 * tz};
#pragma unroll
  for (int k = 0; k < 20; ++k) A.smtl[k * N + cell] = T[k];
  if (mixed) {
#pragma unroll
    for (int k = 0; k < 20; ++k) A.smom32[k * N + cell] = float(T[k]);
    float4* r = reinterpret_cast<float4*>(A.src32 + cell * 28);
#pragma unroll
    for (int q = 0; q < 5; ++q)
      r[q] = make_float4(float(T[4 * q]), float(T[4 * q + 1]), float(T[4 * q + 2]), float(T[4 * q + 3]));
    r[5] = make_float4(float(A.mom[N + cell]), float(A.mom[2 * N + cell]), float(A.mom[3 * N + cell]), 0.0f);
  }
}

// Leaf cells: s = (d rho/dt) dx^3 at the centre (a leaf's centre of mass), no higher moments.
__global__ void k_p2m_src(DevArgs A, int mixed) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= A.n_leaf_cells) return;
  const int32_t s = A.leaf_sub[i >> 9];
  const int u = int(i & 511);
  const int64_t cell = int64_t(s) * kCells + cidx(u >> 6, (u >> 3) & 7, u & 7);
  const int k = A.leaf_tree[i >> 9];
  double v = A.io[k].src[i - A.tree_leaf_off[k] * kCells];
  // finite (any sign), on the bit pattern
  if ((uint64_t(__double_as_longlong(v)) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull) {
    atomicOr(A.status, 2);
    v = 0.0;
  }
  const double m = v * cell_vol(A.level[s]);
  A.smom[cell] = m;
  A.smtl[cell] = m;
  if (mixed) {
    A.smom32[cell] = float(m);
    A.src32[cell * 28] = float(m);  // a leaf's centre of mass is its centre: offset zero
  }
}

// Source moments of the refined cells of one level, one thread per parent cell, 64 per block
// (one octant, as for rho).  Blocks [0, n_walsh) take octants with leaf children: the children
// are point sources at s_e w about the parent cell's centre, whose raw moments there are the
// sign sums of the Walsh-Hadamard transform (P1 = w D, P2 = w^2 G, P3 = w^3 H as for rho), then
// shifted to the parent's centre of mass.  The other blocks take octants with refined children:
// each child's moments are shifted exactly from the child's centre of mass.
__global__ void __launch_bounds__(64) k_m2m_src(DevArgs A, const int32_t* __restrict__ oct_leaf,
                                                int n_walsh, const int32_t* __restrict__ oct_ref,
                                                int mixed) {
  const bool walsh = int(blockIdx.x) < n_walsh;
  const int32_t code = walsh ? oct_leaf[blockIdx.x] : oct_ref[blockIdx.x - n_walsh];
  const int32_t s = code >> 3;
  const int o = code & 7, u = int(threadIdx.x);
  int a, b, c;
  octant_cell(o, u, a, b, c);
  const int64_t N = A.n_cell;
  const int64_t cell = int64_t(s) * kCells + cidx(a, b, c);
  const int64_t c0 = int64_t(A.child[8 * s + o]) * kCells + u;  // child e at c0 + (e << 6)
  const double hc = cell_dx(A.level[s] + 1);
  const double d[3] = {A.mom[N + cell], A.mom[2 * N + cell], A.mom[3 * N + cell]};  // parent delta
  double S[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) S[k] = 0.0;
  if (walsh) {
    double v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = A.smom[c0 + (e << 6)];
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (!(e & bit)) {
          const double lo = v[e], hi = v[e | bit];
          v[e] = hi + lo;
          v[e | bit] = hi - lo;
        }
    const double w = 0.5 * hc, w2 = w * w, w3 = w2 * w;
    const double S0 = v[0];
    const double P1[3] = {w * v[4], w * v[2], w * v[1]};
    // P2 (xx xy xz yy yz zz) and P3 (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz) about the centre
    const double P2[6] = {w2 * S0, w2 * v[6], w2 * v[5], w2 * S0, w2 * v[3], w2 * S0};
    const double D[3] = {v[4], v[2], v[1]};
    const double P3[10] = {w3 * D[0], w3 * D[1], w3 * D[2], w3 * D[0], w3 * v[7],
                           w3 * D[0], w3 * D[1], w3 * D[2], w3 * D[1], w3 * D[2]};
    // the same points about the parent's centre of mass: r = u - delta
    S[0] = S0;
#pragma unroll
    for (int k = 0; k < 3; ++k) S[1 + k] = P1[k] - S0 * d[k];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = p; q < 3; ++q)
        S[4 + sym2_index(p, q)] = P2[sym2_index(p, q)] - d[p] * P1[q] - d[q] * P1[p] + S0 * d[p] * d[q];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int p = sym3_axis(k, 0), q = sym3_axis(k, 1), r = sym3_axis(k, 2);
      S[10 + k] = P3[k] - (d[p] * P2[sym2_index(q, r)] + d[q] * P2[sym2_index(p, r)] +
                           d[r] * P2[sym2_index(p, q)]) +
                  (d[p] * d[q] * P1[r] + d[p] * d[r] * P1[q] + d[q] * d[r] * P1[p]) -
                  S0 * d[p] * d[q] * d[r];
    }
  } else {
#pragma unroll 1
    for (int e = 0; e < 8; ++e) {
      const int64_t ci = c0 + (e << 6);
      double ch[20];
#pragma unroll
      for (int k = 0; k < 20; ++k) ch[k] = A.smom[k * N + ci];
      // r = X_child - X_parent
      const double r[3] = {(((e >> 2) & 1) ? 0.5 : -0.5) * hc + A.mom[N + ci] - d[0],
                           (((e >> 1) & 1) ? 0.5 : -0.5) * hc + A.mom[2 * N + ci] - d[1],
                           ((e & 1) ? 0.5 : -0.5) * hc + A.mom[3 * N + ci] - d[2]};
      src_shift_add(ch, r, S);
    }
  }
  store_src_moments(A, cell, S, mixed);
}

// Expansion of a target due to a source cell at separation R = X_A - X_B (truncation k + n <= 3),
// with detraced S2', S3' (every D^(n) is traceless) and rs1 = R.S1, rs2r = R.S2'.R, q = S3'(R,R):
//   L0 -= S0 g0 - g1 rs1 + 1/2 g2 rs2r - 1/6 g3 R.q
//   L1 -= (S0 g1 - g2 rs1 + 1/2 g3 rs2r) R - g1 S1 + g2 S2' R
//   L2 -= (S0 g2 - g3 rs1) R R + (S0 g1 - g2 rs1) I - g2 (R S1 + S1 R)
//   L3 -= S0 (g3 R R R + g2 sym(R I)).
// AREF: all 20 components (targets with children; L2, L3 as 12 independent components); else
// L0 only.  BREF: the source has children (full moments); else a point source.
// A source cell with children (S0, dipole S1, detraced S2, S3) at separation R = (x, y, z) from
// the target's expansion centre.
template <typename T, bool AREF>
__device__ __forceinline__ void src_far(T* L, T s0, T s1x, T s1y, T s1z, const T* S2, const T* S3,
                                        T x, T y, T z) {
  Radial<T> g;
  g.set(x, y, z, 3);
  const T q2x = S2[0] * x + S2[1] * y + S2[2] * z;
  const T q2y = S2[1] * x + S2[3] * y + S2[4] * z;
  const T q2z = S2[2] * x + S2[4] * y + S2[5] * z;
  const T rs2r = x * q2x + y * q2y + z * q2z;
  const T rs1 = x * s1x + y * s1y + z * s1z;
  T qx, qy, qz;
  sym3_rr(S3, x, y, z, qx, qy, qz);
  const T rrr = x * qx + y * qy + z * qz;
  L[0] -= s0 * g.g0 - g.g1 * rs1 + T(0.5) * g.g2 * rs2r - T(1.0 / 6.0) * g.g3 * rrr;
  if constexpr (AREF) {
    const T c1 = s0 * g.g1 - g.g2 * rs1 + T(0.5) * g.g3 * rs2r;
    L[1] -= c1 * x - g.g1 * s1x + g.g2 * q2x;
    L[2] -= c1 * y - g.g1 * s1y + g.g2 * q2y;
    L[3] -= c1 * z - g.g1 * s1z + g.g2 * q2z;
    const T c2 = s0 * g.g2 - g.g3 * rs1, c0 = s0 * g.g1 - g.g2 * rs1, e = g.g2;
    L[4] -= c2 * x * x + c0 - T(2) * e * x * s1x;
    L[5] -= c2 * x * y - e * (x * s1y + s1x * y);
    L[6] -= c2 * x * z - e * (x * s1z + s1x * z);
    L[7] -= c2 * y * y + c0 - T(2) * e * y * s1y;
    L[8] -= c2 * y * z - e * (y * s1z + s1y * z);
    // L3 from S0 alone: the L3 part of m2l_high
    const T a2 = s0 * g.g2, a3 = s0 * g.g3;
    const T a2x = a2 * x, a2y = a2 * y, a2z = a2 * z, a3xx = a3 * x * x, a3yy = a3 * y * y;
    L[10] -= a3xx * x + T(3) * a2x;
    L[11] -= a3xx * y + a2y;
    L[12] -= a3xx * z + a2z;
    L[13] -= a3yy * x + a2x;
    L[14] -= a3 * x * y * z;
    L[16] -= a3yy * y + T(3) * a2y;
    L[17] -= a3yy * z + a2z;
  }
}

template <typename T, bool AREF, bool BREF>
__device__ __forceinline__ void interact_src(T* L, const T* __restrict__ Sm, const T* __restrict__ G,
                                             int64_t N, int64_t iB, T x, T y, T z) {
  const T s0 = Sm[iB];
  if constexpr (BREF) {
    x -= mom_get(G, N, iB, 1);
    y -= mom_get(G, N, iB, 2);
    z -= mom_get(G, N, iB, 3);
    T S2[6], S3[10];
#pragma unroll
    for (int k = 0; k < 6; ++k) S2[k] = Sm[(4 + k) * N + iB];
#pragma unroll
    for (int k = 0; k < 10; ++k) S3[k] = Sm[(10 + k) * N + iB];
    src_far<T, AREF>(L, s0, Sm[N + iB], Sm[2 * N + iB], Sm[3 * N + iB], S2, S3, x, y, z);
  } else {
    Radial<T> g;
    g.set(x, y, z, AREF ? 3 : 0);
    L[0] -= s0 * g.g0;
    if constexpr (AREF) {
      const T c = s0 * g.g1;
      L[1] -= c * x;
      L[2] -= c * y;
      L[3] -= c * z;
      m2l_high<T>(x, y, z, g, s0, L);
    }
  }
}


__device__ __forceinline__ void store_src_expansion(const DevArgs& A, int64_t i, const double* L, int n) {
  for (int k = 0; k < n; ++k) A.sloc[k * A.n_cell + i] = L[k];
}
__device__ __forceinline__ void store_src_expansion(const DevArgs& A, int64_t i, const float* L, int n) {
  for (int k = 0; k < n; ++k) A.sloc32[k * A.n_cell + i] = L[k];
}

// Refined targets of a level >= 1, one parity per block (as m2l_level): every stencil partner
// through the full source formula (a leaf partner's dipole and higher moments are zeros).
template <typename T>
__device__ void m2l_level_src(const DevArgs& A, int32_t s, int parity, int t) {
  __shared__ int32_t nb[27];
  if (threadIdx.x < 27) nb[threadIdx.x] = A.nbr[27 * s + threadIdx.x];
  __syncthreads();
  const T* __restrict__ G = MomView<T>::get(A);
  const T* __restrict__ Sm = SrcView<T>::get(A);
  const int64_t N = A.n_cell;
  int a, b, c;
  block_cell(parity, t, a, b, c);
  const int64_t iA = int64_t(s) * kCells + cidx(a, b, c);
  const T dAx = mom_get(G, N, iA, 1), dAy = mom_get(G, N, iA, 2), dAz = mom_get(G, N, iA, 3);
  T L[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) L[k] = T(0);
  const T h = cell_h<T>(A.level[s]);
  const int32_t* __restrict__ st = A.ltab_code + parity * kLeafCap;
  const T* __restrict__ td = LeafOffsets<T>::get(A) + int64_t(parity) * kLeafCap * 4;
  for (int q = 0; q < A.n_stencil; ++q) {
    int dx, dy, dz;
    unpack_offset(__ldg(st + q), dx, dy, dz);
    const int px = a + dx, py = b + dy, pz = c + dz;
    const int slot = ((px >> 3) + 1) * 9 + ((py >> 3) + 1) * 3 + ((pz >> 3) + 1);
    const int32_t sB = nb[slot];
    if (sB < 0) continue;  // only without proper nesting
    interact_src<T, true, true>(L, Sm, G, N, int64_t(sB) * kCells + cidx(px & 7, py & 7, pz & 7),
                                dAx - ldg_t(td + 4 * q) * h, dAy - ldg_t(td + 4 * q + 1) * h,
                                dAz - ldg_t(td + 4 * q + 2) * h);
  }
  complete_traceless(L);
  store_src_expansion(A, iA, L, 20);
}

// Root level: every well-separated root pair (all pairs, directly, when the root is a leaf),
// sources in kRootChunks chunks whose partial sums the downward pass adds in a fixed order.
// LANES lanes per target (as m2l_root): lane r takes rows jy in [r 8 / LANES, (r + 1) 8 / LANES).
template <typename T, bool AREF, int LANES = 1>
__device__ void m2l_root_src(const DevArgs& A, int root, int parity, int t, int chunk, int r = 0) {
  const T* __restrict__ G = MomView<T>::get(A);
  const T* __restrict__ Sm = SrcView<T>::get(A);
  const int64_t N = A.n_cell;
  int a, b, c;
  block_cell(parity, t, a, b, c);
  const int iloc = cidx(a, b, c);
  const int64_t base = int64_t(root) * kCells;
  const T dAx = mom_get(G, N, base + iloc, 1), dAy = mom_get(G, N, base + iloc, 2),
          dAz = mom_get(G, N, base + iloc, 3);
  T L[20];
#pragma unroll
  for (int k = 0; k < 20; ++k) L[k] = T(0);
  const T h = cell_h<T>(0);
  const int dx = chunk - a;
  const T rx0 = dAx - T(dx) * h;
  constexpr int kRows = 8 / LANES;
  const int jy0 = r * kRows;
  T ry = dAy + T(b - jy0) * h;
  const T rz0 = dAz + T(c) * h;
  for (int jy = jy0; jy < jy0 + kRows; ++jy, ry -= h) {
    T rz = rz0;
    for (int jz = 0; jz < 8; ++jz, rz -= h) {
      const int j = cidx(chunk, jy, jz);
      if (j == iloc) continue;
      const int dy = jy - b, dz = jz - c;
      if (AREF && !(dx * dx + dy * dy + dz * dz > A.ws_d2)) continue;
      interact_src<T, AREF, AREF>(L, Sm, G, N, base + j, rx0, ry, rz);
    }
  }
  if constexpr (LANES > 1) {
#pragma unroll
    for (int m = 1; m < LANES; m <<= 1)
#pragma unroll
      for (int k = 0; k < (AREF ? 20 : 1); ++k) L[k] += __shfl_xor_sync(0xffffffffu, L[k], m);
    if (r != 0) return;
  }
  if constexpr (AREF) complete_traceless(L);
  // partials: [chunk][component][cell]
  if (sizeof(T) == 8) {
    double* P = A.root_part + (int64_t(root) * kRootChunks + chunk) * 23 * kCells;
    for (int k = 0; k < 20; ++k) P[k * kCells + iloc] = (AREF || k == 0) ? double(L[k]) : 0.0;
  } else {
    float* P = A.root_part32 + (int64_t(root) * kRootChunks + chunk) * 20 * kCells;
    for (int k = 0; k < 20; ++k) P[k * kCells + iloc] = (AREF || k == 0) ? float(L[k]) : 0.0f;
  }
}

// Leaf targets at refinement boundaries from the pair lists: multipole partners (refined) and
// point partners; adds L0 onto the source leaf kernel's output.
// The block's targets are first + 64 chunk + t, those below end; LANES lanes per target (as
// m2l_boundary), every lane of the block calls this.
template <typename T, int LANES = 1>
__device__ void m2l_boundary_src(const DevArgs& A, int64_t first, int64_t end, int chunk, int t, int r = 0) {
  __shared__ T quarter[2 * kCodeMax + 1];
  for (int i = threadIdx.x; i <= 2 * kCodeMax; i += blockDim.x) quarter[i] = T(i - kCodeMax) * T(0.25);
  __syncthreads();
  const int64_t k = first + int64_t(chunk) * 64 + t;
  const bool valid = k < end;
  if (LANES == 1 && !valid) return;
  const int64_t iA = valid ? A.bt_cell[k] : 0;
  const T* __restrict__ G = MomView<T>::get(A);
  const T* __restrict__ Sm = SrcView<T>::get(A);
  const int64_t N = A.n_cell;
  const int32_t sA = int32_t(iA >> 9);
  const int lev = A.level[sA];
  const T h = cell_h<T>(lev);
  int a, b, c;
  cdecode(int(iA & 511), a, b, c);
  T L[1] = {T(0)};
  const int32_t m1 = valid ? A.bm_off[k + 1] : 0;
  for (int32_t j = (valid ? A.bm_off[k] : 0) + r; j < m1; j += LANES) {
    int dx, dy, dz;
    const int64_t src = boundary_partner(A, sA, a, b, c, __ldg(A.bm_e + j), dx, dy, dz);
    interact_src<T, false, true>(L, Sm, G, N, src, neg_offset<T>(dx, lev), neg_offset<T>(dy, lev),
                                 neg_offset<T>(dz, lev));
  }
  const int32_t p1 = valid ? A.bp_off[k + 1] : 0;
  for (int32_t j = (valid ? A.bp_off[k] : 0) + r; j < p1; j += LANES) {
    int64_t first;
    int qx, qy, qz;
    const int n = point_partner(A, sA, a, b, c, __ldg(A.bp_e + j), first, qx, qy, qz);
    if (FMM_BAD(A, n > 0 && first + 64 * (n - 1) < N && unsigned(qx + kCodeMax - 2) <= 2u * kCodeMax - 2 &&
                       unsigned(qy + kCodeMax - 2) <= 2u * kCodeMax - 2 &&
                       unsigned(qz + kCodeMax - 2) <= 2u * kCodeMax - 2))
      continue;
    for (int o = 0; o < n; ++o)
      interact_src<T, false, false>(L, Sm, G, N, first + 64 * o,
                                    quarter[qx - (n == 8 ? 2 * (o >> 2) : 0) + kCodeMax] * h,
                                    quarter[qy - (n == 8 ? 2 * ((o >> 1) & 1) : 0) + kCodeMax] * h,
                                    quarter[qz - (n == 8 ? 2 * (o & 1) : 0) + kCodeMax] * h);
  }
  if constexpr (LANES > 1) {
#pragma unroll
    for (int m = 1; m < LANES; m <<= 1) L[0] += __shfl_xor_sync(0xffffffffu, L[0], m);
    if (r != 0 || !valid) return;
  }
  if (sizeof(T) == 8) A.sloc[iA] += double(L[0]);
  else A.sloc32[iA] += float(L[0]);
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_m2l_ref_src(DevArgs A, const int32_t* __restrict__ blocks) {
  const int32_t code = blocks[blockIdx.x];
  const int kind = (code >> 30) & 3, idx = code & ((1 << 27) - 1);
  const int parity = (code >> 27) & 7;
  const int t = int(threadIdx.x & 63);
  if (kind == 0) {
    const int root = idx >> 3, chunk = idx & 7;
    if (A.leaf[root]) m2l_root_src<T, false>(A, root, parity, t, chunk);
    else m2l_root_src<T, true>(A, root, parity, t, chunk);
  } else if (kind == 1) {
    m2l_level_src<T>(A, idx, parity, t);
  } else {
    m2l_boundary_src<T>(A, 0, A.n_bt, idx, t);
  }
}

// The time-derivative solve's root and boundary work for the mixed path (its refined subgrids
// go to k_m2l_stage<true>), with k_m2l_split's block list and lanes.
template <typename T>
__global__ void __launch_bounds__(64 * kSplitLanes) k_m2l_split_src(DevArgs A, const int32_t* __restrict__ blocks) {
  const int32_t code = blocks[blockIdx.x];
  const int kind = (code >> 30) & 3, idx = code & ((1 << 27) - 1);
  const int parity = (code >> 27) & 7;
  const int t = int(threadIdx.x) / kSplitLanes, r = int(threadIdx.x) % kSplitLanes;
  if (kind == 0) {
    const int root = idx >> 3, chunk = idx & 7;
    if (A.leaf[root]) m2l_root_src<T, false, kSplitLanes>(A, root, parity, t, chunk, r);
    else m2l_root_src<T, true, kSplitLanes>(A, root, parity, t, chunk, r);
  } else if (kind == 2) {
    m2l_boundary_src<T, kSplitLanes>(A, 0, A.n_bt_long, idx, t, r);
  } else {
    m2l_boundary_src<T, 1>(A, A.n_bt_long, A.n_bt, idx + int(threadIdx.x) / 64, int(threadIdx.x) % 64);
  }
}

// ----------------------------------------------------------------------------------------------
// net force and torque: F = sum m g, T = sum x cross m g, S = sum |x| |m g|; fixed order
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ void block_sum7(double* v, double (*sh)[kReduceThreads]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 7; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
    if (t < w)
#pragma unroll
      for (int k = 0; k < 7; ++k) sh[k][t] += sh[k][t + w];
    __syncthreads();
  }
}

// Block b reduces chunk plan[2 b + 1] of tree k = plan[2 b]: tree k's leaf cells are shared by
// its nb = tree_plan[2 k] blocks in a fixed order (each tree's share of the blocks is in
// proportion to its leaf cells, so that the trees of a forest finish together), and the last of
// them to finish (a counter per tree, reset by that block) adds the nb partial sums, stored from
// partials[7 tree_plan[2 k + 1]] on, in block order into the tree's 7 numbers.  The FP64 work per cell is m, m g, F and the
// torque (13 operations); the normalisation S, a scale, is formed in FP32 from values converted
// with integer operations.
__global__ void __launch_bounds__(kReduceThreads)
    k_net_partial(DevArgs A, double* __restrict__ partials, unsigned* __restrict__ counters,
                  const int32_t* __restrict__ plan, const int32_t* __restrict__ tree_plan) {
  __shared__ double sh[7][kReduceThreads];
  double v[6] = {0, 0, 0, 0, 0, 0};
  float sn = 0.0f;  // this thread's share of the normalisation S, formed and summed in FP32
  const int tree = plan[2 * blockIdx.x], chunk = plan[2 * blockIdx.x + 1];
  if (FMM_BAD(A, tree >= 0 && tree < A.n_roots)) return;  // (no block waits for another)
  const int nb = tree_plan[2 * tree];
  const int64_t stride = int64_t(nb) * kReduceThreads;
  const int64_t base = A.tree_leaf_off[tree] * kCells;
  const int64_t end = A.tree_leaf_off[tree + 1] * kCells;
  const double* __restrict__ rho = A.io[tree].rho;
  const double* __restrict__ g = A.io[tree].g;
#pragma unroll 4
  for (int64_t i = base + int64_t(chunk) * kReduceThreads + threadIdx.x; i < end; i += stride) {
    const int32_t s = A.leaf_sub[i >> 9];
    const int lev = A.level[s];
    const int loc = int(i & 511);
    // cell centre x = -1/2 + (g + 1/2) dx = (2 g + 1 - 2^(lev + 3)) 2^-(lev + 4), an odd multiple
    const int full = 1 << (lev + 3);
    const int nx = 2 * (A.ijk[3 * s] * 8 + (loc >> 6)) + 1 - full;
    const int ny = 2 * (A.ijk[3 * s + 1] * 8 + ((loc >> 3) & 7)) + 1 - full;
    const int nz = 2 * (A.ijk[3 * s + 2] * 8 + (loc & 7)) + 1 - full;
    const double x = dyadic(nx, lev + 4), y = dyadic(ny, lev + 4), z = dyadic(nz, lev + 4);
    const int64_t o = i - base;
    const double m = rho[o] * cell_vol(lev);
    const double fx = m * g[3 * o], fy = m * g[3 * o + 1], fz = m * g[3 * o + 2];
    v[0] += fx;
    v[1] += fy;
    v[2] += fz;
    v[3] = fma(y, fz, fma(-z, fy, v[3]));
    v[4] = fma(z, fx, fma(-x, fz, v[4]));
    v[5] = fma(x, fy, fma(-y, fx, v[5]));
    const float sc = __int_as_float((127 - lev - 4) << 23);
    const float xf = float(nx) * sc, yf = float(ny) * sc, zf = float(nz) * sc;
    const float ffx = df_d2f_trunc(fx), ffy = df_d2f_trunc(fy), ffz = df_d2f_trunc(fz);
    sn += sqrtf(xf * xf + yf * yf + zf * zf) * sqrtf(ffx * ffx + ffy * ffy + ffz * ffz);
  }
  double w[7] = {v[0], v[1], v[2], v[3], v[4], v[5], df_f2d(sn)};
  block_sum7(w, sh);
  double* P = partials + int64_t(tree_plan[2 * tree + 1]) * 7;
  if (threadIdx.x < 7) P[int64_t(chunk) * 7 + threadIdx.x] = sh[threadIdx.x][0];
  __shared__ bool last;
  __threadfence();  // this block's partial sums are visible before it is counted
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&counters[tree], 1u) == unsigned(nb) - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double u[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nb; b += kReduceThreads)
#pragma unroll
    for (int k = 0; k < 7; ++k) u[k] += P[int64_t(b) * 7 + k];
  block_sum7(u, sh);
  if (threadIdx.x < 7) (*A.io_net)[int64_t(tree) * 7 + threadIdx.x] = sh[threadIdx.x][0];
  if (threadIdx.x == 0) counters[tree] = 0u;  // ready for the next solve
}

// blockIdx.x = tree (or set of partials): sums n_blocks partials in a fixed order into out[7 x];
// out is read from *out_slot when that is given.
__global__ void __launch_bounds__(kReduceThreads)
    k_net_final(const double* __restrict__ partials, int n_blocks, double* out,
                double* const* out_slot) {
  if (out_slot) out = *out_slot;
  __shared__ double sh[7][kReduceThreads];
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const double* P = partials + int64_t(blockIdx.x) * n_blocks * 7;
  for (int b = threadIdx.x; b < n_blocks; b += kReduceThreads)
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] += P[int64_t(b) * 7 + k];
  block_sum7(v, sh);
  if (threadIdx.x < 7) out[int64_t(blockIdx.x) * 7 + threadIdx.x] = sh[threadIdx.x][0];
}

// ----------------------------------------------------------------------------------------------
// binary diagnostics (Sec. 4): star membership by the effective acceleration, per-star sums
// ----------------------------------------------------------------------------------------------
// g_eff = g + Omega^2 (x, y, 0);  q_s = g_eff . (x - x_s) / |x - x_s| (0 at x_s itself).  A cell
// belongs to the accretor (1) if min(q_1, 0) < min(q_2, 0), to the donor (2) if greater, else to
// neither; within rc_s of x_s it belongs to star s whatever q says (the accretor tested last, so
// it wins).  The decision is taken with single correctly rounded FP64 operations in a fixed order
// (no fused multiply-add), so it is reproducible operation for operation.  Per star, with
// m = rho dx^3: M, sum m x, F = sum m g, T = sum (x - x_s) x m g, and the number of cells.
struct BinaryParams {
  double w2;          // Omega^2
  double c[2][3];     // x_1, x_2
  double rc2[2];      // squared critical radii
};
constexpr int kDiagVals = 22;   // 2 stars x (M, m x[3], F[3], T[3], count)
constexpr int kDiagThreads = 128;

__device__ __forceinline__ double q_of(double gex, double gey, double gez, double dx, double dy,
                                       double dz, double& d2) {
  d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double dot = __dadd_rn(__dadd_rn(__dmul_rn(gex, dx), __dmul_rn(gey, dy)), __dmul_rn(gez, dz));
  return d2 > 0.0 ? __ddiv_rn(dot, __dsqrt_rn(d2)) : 0.0;
}

__global__ void __launch_bounds__(kDiagThreads)
    k_binary_partial(DevArgs A, const BinaryParams* __restrict__ Pdev, double* __restrict__ partials,
                     int8_t* member) {
  __shared__ double sh[kDiagVals][kDiagThreads];
  const BinaryParams P = *Pdev;
  double v[kDiagVals];
#pragma unroll
  for (int k = 0; k < kDiagVals; ++k) v[k] = 0.0;
  const int64_t stride = int64_t(gridDim.x) * kDiagThreads;
  const double* __restrict__ rho = A.io[0].rho;
  const double* __restrict__ g = A.io[0].g;
  for (int64_t i = int64_t(blockIdx.x) * kDiagThreads + threadIdx.x; i < A.n_leaf_cells; i += stride) {
    const int32_t s = A.leaf_sub[i >> 9];
    const int lev = A.level[s];
    const int loc = int(i & 511);
    const int full = 1 << (lev + 3);
    const double x = dyadic(2 * (A.ijk[3 * s] * 8 + (loc >> 6)) + 1 - full, lev + 4);
    const double y = dyadic(2 * (A.ijk[3 * s + 1] * 8 + ((loc >> 3) & 7)) + 1 - full, lev + 4);
    const double z = dyadic(2 * (A.ijk[3 * s + 2] * 8 + (loc & 7)) + 1 - full, lev + 4);
    const double gx = g[3 * i], gy = g[3 * i + 1], gz = g[3 * i + 2];
    const double gex = __dadd_rn(gx, __dmul_rn(P.w2, x)), gey = __dadd_rn(gy, __dmul_rn(P.w2, y));
    double d2a, d2b;
    const double q1 = q_of(gex, gey, gz, __dsub_rn(x, P.c[0][0]), __dsub_rn(y, P.c[0][1]),
                           __dsub_rn(z, P.c[0][2]), d2a);
    const double q2 = q_of(gex, gey, gz, __dsub_rn(x, P.c[1][0]), __dsub_rn(y, P.c[1][1]),
                           __dsub_rn(z, P.c[1][2]), d2b);
    const double m1 = fmin(q1, 0.0), m2 = fmin(q2, 0.0);
    int who = m1 < m2 ? 1 : (m1 > m2 ? 2 : 0);
    if (d2b < P.rc2[1]) who = 2;
    if (d2a < P.rc2[0]) who = 1;
    if (member) member[i] = int8_t(who);
    if (who == 0) continue;
    const int b = who == 1 ? 0 : 11;
    const double m = rho[i] * cell_vol(lev);
    const double fx = m * gx, fy = m * gy, fz = m * gz;
    const double rx = x - P.c[who - 1][0], ry = y - P.c[who - 1][1], rz = z - P.c[who - 1][2];
    v[b] += m;
    v[b + 1] += m * x;
    v[b + 2] += m * y;
    v[b + 3] += m * z;
    v[b + 4] += fx;
    v[b + 5] += fy;
    v[b + 6] += fz;
    v[b + 7] += ry * fz - rz * fy;
    v[b + 8] += rz * fx - rx * fz;
    v[b + 9] += rx * fy - ry * fx;
    v[b + 10] += 1.0;
  }
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < kDiagVals; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if (t < w)
#pragma unroll
      for (int k = 0; k < kDiagVals; ++k) sh[k][t] += sh[k][t + w];
    __syncthreads();
  }
  if (t < kDiagVals) partials[int64_t(blockIdx.x) * kDiagVals + t] = sh[t][0];
}

// Eggleton's (1983) volume-equivalent Roche-lobe radius of a star of mass ratio
// q = M_star / M_other at separation a (within 1 % of the exact lobe volume for all q).
__device__ __forceinline__ double roche_lobe(double q, double a) {
  const double q23 = pow(q, 2.0 / 3.0);
  return a * 0.49 * q23 / (0.6 * q23 + log(1.0 + pow(q, 1.0 / 3.0)));
}

// Sets the parameters of the first pass.
__global__ void k_binary_init(BinaryParams P, BinaryParams* __restrict__ state) { *state = P; }

// One block: the partials of all blocks in a fixed order.  With `update`, thread 0 then takes
// one step of the diagnostics' fixed-point iteration on the parameters of the next pass: the
// centres used by this pass and the orbital torque x_1 x F_1 + x_2 x F_2 go to centres_out (6)
// and torque_out (3); each star's centre moves to its centre of mass, and the critical radii
// become a quarter of the Roche-lobe radii of the two masses at the new separation.  A star that
// received no mass keeps its centre, and both radii stay as they were until both stars have mass.
__global__ void __launch_bounds__(kDiagThreads)
    k_binary_final(const double* __restrict__ partials, int n_blocks, double* __restrict__ out,
                   BinaryParams* __restrict__ state, double* __restrict__ centres_out,
                   double* __restrict__ torque_out, int update) {
  __shared__ double sums[kDiagVals];
  const int t = threadIdx.x;
  if (t < kDiagVals) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += partials[int64_t(b) * kDiagVals + t];
    out[t] = v;
    sums[t] = v;
  }
  __syncthreads();
  if (!update || t != 0) return;
  BinaryParams& P = *state;
  const double* F1 = sums + 4;
  const double* F2 = sums + 15;
  const double* c1 = P.c[0];
  const double* c2 = P.c[1];
  for (int k = 0; k < 3; ++k) {
    centres_out[k] = c1[k];
    centres_out[3 + k] = c2[k];
  }
  torque_out[0] = (c1[1] * F1[2] - c1[2] * F1[1]) + (c2[1] * F2[2] - c2[2] * F2[1]);
  torque_out[1] = (c1[2] * F1[0] - c1[0] * F1[2]) + (c2[2] * F2[0] - c2[0] * F2[2]);
  torque_out[2] = (c1[0] * F1[1] - c1[1] * F1[0]) + (c2[0] * F2[1] - c2[1] * F2[0]);
  const double M1 = sums[0], M2 = sums[11];
  for (int k = 0; k < 3; ++k) {
    if (M1 > 0.0) P.c[0][k] = sums[1 + k] / M1;
    if (M2 > 0.0) P.c[1][k] = sums[12 + k] / M2;
  }
  if (M1 > 0.0 && M2 > 0.0) {
    const double dx = P.c[0][0] - P.c[1][0], dy = P.c[0][1] - P.c[1][1], dz = P.c[0][2] - P.c[1][2];
    const double a = sqrt(dx * dx + dy * dy + dz * dz);
    const double r1 = 0.25 * roche_lobe(M1 / M2, a), r2 = 0.25 * roche_lobe(M2 / M1, a);
    P.rc2[0] = r1 * r1;
    P.rc2[1] = r2 * r2;
  }
}

// ----------------------------------------------------------------------------------------------
// the caller's pointers of one call, passed by value as kernel parameters
// ----------------------------------------------------------------------------------------------
constexpr int kIoChunk = 96;  // trees per launch: the parameter block stays under 4 KB
struct IoChunk {
  double* net;
  int32_t first, count;
  TreeIo e[kIoChunk];
};
static_assert(sizeof(IoChunk) <= 4000, "kernel parameter block too large");

__global__ void k_set_io(IoChunk c, TreeIo* __restrict__ table, double** net_slot) {
  const int j = threadIdx.x;
  if (j < c.count) table[c.first + j] = c.e[j];
  if (j == 0) *net_slot = c.net;
}

// ----------------------------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------------------------
struct StencilDev {
  int32_t* d_stencil = nullptr;  // [8][kStencilCap]
  int32_t* d_near = nullptr;
  int32_t* d_ltab_off = nullptr;   // [8][kLeafCap]
  int32_t* d_ltab_code = nullptr;  // [8][kLeafCap]
  double* d_ltab_k64 = nullptr;    // [8][kLeafCap][4]
  float* d_ltab_k32 = nullptr;
  double* d_ltab_d64 = nullptr;    // [8][kLeafCap][4]
  float* d_ltab_d32 = nullptr;
  dfloat* d_ltab_kff = nullptr;    // [8][kLeafCap][4] double-float copies
  dfloat* d_ltab_dff = nullptr;
  int32_t* d_blocks = nullptr;     // general-kernel blocks (one parity each) for this tree, theta
  int64_t n_blocks = 0;
  int mixed_variant = 0;              // mixed path launch variant (fmm_set_variant, fmm_autotune)
  // mixed path: k_m2l_split's blocks (root, boundary) for each choice of the threshold above which
  // a boundary target's lists are split over four lanes (built when first used)
  int32_t* d_blocks_split[kSplitChoices] = {};
  int64_t n_blocks_split[kSplitChoices] = {};
  int64_t n_bt_long[kSplitChoices] = {};  // boundary targets [0, n_bt_long) take four lanes
  std::vector<double> bnd_cost;           // estimated cost of each boundary target (sorted)
  float* d_stage_tab = nullptr;    // [8][kLeafCap][4] (DevArgs::stage_tab)
  int32_t* d_stage_seg = nullptr;  // [8][9]
  // boundary pair lists (see DevArgs)
  int64_t n_bt = 0;
  uint16_t* d_bm_e = nullptr;
  int32_t *d_bt_cell = nullptr, *d_bm_off = nullptr,
          *d_bp_off = nullptr;
  uint16_t* d_bp_e = nullptr;

  int n_stencil = 0, n_near = 0;
  int ws_d2 = 0;
};

struct fmm_tree {
  HostTree h;
  int device = -1;
  int n_sms = 1;
  bool dev_ready = false, mixed_ready = false;
  int32_t *d_level = nullptr, *d_ijk = nullptr, *d_parent = nullptr, *d_child = nullptr,
          *d_nbr = nullptr, *d_leaf_sub = nullptr, *d_leaf_ord = nullptr, *d_work = nullptr,
          *d_work_leaf = nullptr;
  int64_t n_work_leaf = 0, n_work_bnd = 0;
  uint8_t* d_leaf = nullptr;
  // upward pass: (refined subgrid << 3 | octant) of each level, by the kind of the child subgrid
  int32_t *d_oct_leaf = nullptr, *d_oct_ref = nullptr;
  std::vector<int64_t> oct_leaf_off, oct_ref_off;
  // downward pass: refined subgrids of each level
  int32_t* d_ref_sub = nullptr;
  std::vector<int64_t> ref_off;
  int64_t n_work = 0;
  double *d_mom = nullptr, *d_mtl = nullptr, *d_loc = nullptr, *d_ac = nullptr, *d_root_part = nullptr,
         *d_root_part_ac = nullptr, *d_partials = nullptr;
  unsigned* d_net_count = nullptr;  // k_net_partial's finished-block counters, one per tree
  int32_t *d_net_plan = nullptr, *d_net_tree_plan = nullptr;  // its blocks' trees and chunks
  int64_t net_blocks = 0;
  unsigned* d_bar = nullptr;        // k_levels' grid barrier: arrivals, generation
  int persistent = 0;               // level passes as persistent launches (fmm_set_persistent)
  int levels_cap[2] = {0, 0};       // co-resident blocks of k_levels<false>, k_levels<true>
  float *d_mom32 = nullptr, *d_m32 = nullptr, *d_loc32 = nullptr, *d_root_part32 = nullptr;
  int* d_status = nullptr;
  int64_t* d_tree_leaf_off = nullptr;
  double *d_rho = nullptr, *d_phi = nullptr, *d_g = nullptr, *d_net = nullptr;
  // pipelined host solves (fmm_solve_host_async): two device slots, a stream for the copies in, one
  // for the solves, one for the copies out, and per slot the events that order them
  struct HostPipe {
    double *rho[2] = {}, *phi[2] = {}, *g[2] = {}, *net[2] = {};
    cudaStream_t in = nullptr, solve = nullptr, out = nullptr;
    cudaEvent_t copied_in[2] = {}, solved[2] = {}, copied_out[2] = {}, caller = nullptr;
    int slot = 0;
  } hp;
  // time-derivative solve workspace (allocated on first use)
  bool src_ready = false, src32_ready = false;
  double* d_diag_partials = nullptr;  // binary diagnostics: [blocks][kDiagVals]
  BinaryParams* d_diag_state = nullptr;  // the parameters of the next diagnostics pass
  // self-consistent-field iteration (allocated on first use)
  int64_t* d_scf_axis = nullptr;           // leaf cells touching the x axis
  int64_t n_scf_axis = 0;
  ScfState* d_scf_state = nullptr;
  ScfPartial* d_scf_part = nullptr;
  ScfAxisPartial* d_scf_apart = nullptr;
  bool scf_started = false;               // fmm_scf_init has enqueued an initial state
  int prio_high = 0;                      // the device's highest stream priority
  bool df_ready = false;
  dfloat *d_momff = nullptr, *d_massff = nullptr;
  double *d_smom = nullptr, *d_smtl = nullptr, *d_sloc = nullptr;
  float *d_smom32 = nullptr, *d_sloc32 = nullptr, *d_src32 = nullptr;
  std::map<double, StencilDev> stencils;
  bool profiling = false;
  cudaEvent_t ev[10] = {nullptr, nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr, nullptr};
  // a second stream, forked from and joined back to the tree's stream inside a solve: the leaf
  // kernel beside the upward pass, and the mixed path's root and boundary kernel
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_m2m = nullptr;
  bool ev_recorded = false;
  bool ev_stage = false;  // the recorded solve ran k_m2l_stage between ev[6] and ev[7]
  int32_t launches = 0;
  std::vector<void*> allocs;
  std::vector<int32_t> work, work_bnd;  // refined and boundary leaf subgrids of levels >= 1
  int32_t* d_leaf_tree = nullptr;
  TreeIo* d_io = nullptr;         // [n_trees] the caller's arrays of the current call
  double** d_io_net = nullptr;    // the caller's net array of the current call
  // Every call of a tree runs on the tree's own stream, ordered after the caller's stream by
  // ev_in and before its later work by ev_out, so that calls of one tree never overlap.
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool use_graphs = true;
  long long wait_cycles = 0;  // first-wait limit of the staging kernel (0: kStageWaitCycles)
  bool capturing = false;
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int32_t launches = 0;
  };
  // one instantiated graph per (theta, precision, correction, net output, profiling, dphi/dt)
  std::map<std::tuple<double, int, int, int, int, int, long long, int, int>, Graph> graphs;
};

// The net reduction's blocks: about kReduceBlocks in all, each tree's share in proportion to its
// leaf cells (at least one).  plan: (tree, chunk) per block; tree_plan: (blocks, first partial)
// per tree.  Returns the number of blocks.
static int64_t net_plan(const std::vector<int64_t>& tree_leaf_off, std::vector<int32_t>& plan,
                        std::vector<int32_t>& tree_plan) {
  const int64_t nr = int64_t(tree_leaf_off.size()) - 1;
  const int64_t total = tree_leaf_off[size_t(nr)] - tree_leaf_off[0];
  plan.clear();
  tree_plan.assign(size_t(2 * nr), 0);
  int64_t first = 0;
  for (int64_t k = 0; k < nr; ++k) {
    const int64_t cells = tree_leaf_off[size_t(k + 1)] - tree_leaf_off[size_t(k)];
    const int64_t nb = std::max<int64_t>(1, total > 0 ? (kReduceBlocks * cells) / total : 1);
    tree_plan[size_t(2 * k)] = int32_t(nb);
    tree_plan[size_t(2 * k + 1)] = int32_t(first);
    for (int64_t c = 0; c < nb; ++c) {
      plan.push_back(int32_t(k));
      plan.push_back(int32_t(c));
    }
    first += nb;
  }
  return first;
}

template <typename P>
static cudaError_t dalloc(fmm_tree* t, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    t->allocs.push_back(q);
    *p = static_cast<P*>(q);
  }
  return e;
}

template <typename V>
static cudaError_t upload(fmm_tree* t, typename V::value_type** p, const V& v) {
  cudaError_t e = dalloc(t, p, sizeof(typename V::value_type) * v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*p, v.data(), sizeof(typename V::value_type) * v.size(),
                    cudaMemcpyHostToDevice);
}

static int ensure_device(fmm_tree* t) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (t->dev_ready) {
    if (dev != t->device) return fail(FMM_ERR_STATE, "tree workspace lives on another device");
    return FMM_OK;
  }
  t->device = dev;
  CUDA_TRY(cudaDeviceGetAttribute(&t->n_sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kHaloWords * sizeof(double))));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kHaloWords * sizeof(float))));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf<dfloat, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kHaloWords * sizeof(dfloat))));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kHaloWords * sizeof(double))));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kHaloWords * sizeof(float))));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf4<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeaf4Smem));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf4<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeaf4Smem));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_leaf4<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                leaf4_smem<4>()));
  const HostTree& h = t->h;
  const int64_t nc = h.n_sub * kCells;
  CUDA_TRY(upload(t, &t->d_level, h.level));
  CUDA_TRY(upload(t, &t->d_ijk, h.ijk));
  CUDA_TRY(upload(t, &t->d_leaf, h.leaf));
  CUDA_TRY(upload(t, &t->d_parent, h.parent));
  CUDA_TRY(upload(t, &t->d_child, h.child));
  CUDA_TRY(upload(t, &t->d_nbr, h.nbr));
  CUDA_TRY(upload(t, &t->d_leaf_sub, h.leaf_sub));
  CUDA_TRY(upload(t, &t->d_leaf_ord, h.leaf_ord));
  // interaction work at levels >= 1: refined subgrids (coarse to fine) and leaf subgrids
  std::vector<int32_t> work, work_leaf;
  for (int l = 1; l <= h.depth; ++l) work.insert(work.end(), h.refined_at[l].begin(), h.refined_at[l].end());
  for (int l = 1; l <= h.depth; ++l) work_leaf.insert(work_leaf.end(), h.leaves_at[l].begin(), h.leaves_at[l].end());
  // leaf subgrids at a refinement boundary: a refined same-level neighbour, or a leaf neighbour
  // of the parent (leaves one level coarser)
  std::vector<int32_t> work_bnd;
  for (int32_t s : work_leaf) {
    bool bnd = false;
    for (int k = 0; k < 27; ++k) {
      int32_t q = h.nbr[27 * s + k];
      if (q >= 0 && !h.leaf[q]) bnd = true;
      int32_t pq = h.nbr[27 * h.parent[s] + k];
      if (pq >= 0 && h.leaf[pq]) bnd = true;
    }
    if (bnd) work_bnd.push_back(s);
  }
  t->n_work = int64_t(work.size());
  t->n_work_leaf = int64_t(work_leaf.size());
  t->n_work_bnd = int64_t(work_bnd.size());
  t->work = work;
  t->work_bnd = work_bnd;
  CUDA_TRY(upload(t, &t->d_work, work));
  CUDA_TRY(upload(t, &t->d_work_leaf, work_leaf));
  std::vector<int32_t> ref_sub;
  t->ref_off.assign(h.depth + 2, 0);
  for (int l = 0; l <= h.depth; ++l) {
    ref_sub.insert(ref_sub.end(), h.refined_at[l].begin(), h.refined_at[l].end());
    t->ref_off[l + 1] = int64_t(ref_sub.size());
  }
  CUDA_TRY(upload(t, &t->d_ref_sub, ref_sub));
  std::vector<int32_t> oct_leaf, oct_ref;
  t->oct_leaf_off.assign(h.depth + 2, 0);
  t->oct_ref_off.assign(h.depth + 2, 0);
  for (int l = 0; l <= h.depth; ++l) {
    for (int32_t s : h.refined_at[l])
      for (int o = 0; o < 8; ++o) (h.leaf[h.child[8 * s + o]] ? oct_leaf : oct_ref).push_back(s * 8 + o);
    t->oct_leaf_off[l + 1] = int64_t(oct_leaf.size());
    t->oct_ref_off[l + 1] = int64_t(oct_ref.size());
  }
  if (int64_t(h.n_sub) * 8 > INT32_MAX) return fail(FMM_ERR_ARG, "too many subgrids");
  CUDA_TRY(upload(t, &t->d_oct_leaf, oct_leaf));
  CUDA_TRY(upload(t, &t->d_oct_ref, oct_ref));
  CUDA_TRY(dalloc(t, &t->d_mom, sizeof(double) * kNMom * nc));
  CUDA_TRY(cudaMemset(t->d_mom, 0, sizeof(double) * kNMom * nc));  // leaf cells keep zeros
  CUDA_TRY(dalloc(t, &t->d_mtl, sizeof(double) * kNMom * nc));
  CUDA_TRY(cudaMemset(t->d_mtl, 0, sizeof(double) * kNMom * nc));
  CUDA_TRY(dalloc(t, &t->d_loc, sizeof(double) * 20 * nc));
  CUDA_TRY(dalloc(t, &t->d_ac, sizeof(double) * 3 * nc));
  const int64_t nr = h.n_trees;
  CUDA_TRY(dalloc(t, &t->d_root_part, sizeof(double) * nr * kRootChunks * 23 * kCells));
  {
    std::vector<int32_t> plan, tree_plan;
    t->net_blocks = net_plan(h.tree_leaf_off, plan, tree_plan);
    CUDA_TRY(dalloc(t, &t->d_partials, sizeof(double) * 7 * size_t(t->net_blocks)));
    CUDA_TRY(upload(t, &t->d_net_plan, plan));
    CUDA_TRY(upload(t, &t->d_net_tree_plan, tree_plan));
  }
  CUDA_TRY(dalloc(t, &t->d_net_count, sizeof(unsigned) * size_t(nr)));
  CUDA_TRY(dalloc(t, &t->d_bar, sizeof(unsigned) * 2));
  CUDA_TRY(cudaMemset(t->d_net_count, 0, sizeof(unsigned) * size_t(nr)));
  CUDA_TRY(upload(t, &t->d_tree_leaf_off, h.tree_leaf_off));
  CUDA_TRY(dalloc(t, &t->d_status, sizeof(int)));
  CUDA_TRY(cudaMemset(t->d_status, 0, sizeof(int)));
  std::vector<int32_t> leaf_tree(size_t(h.n_leaf_sub));
  for (int k = 0; k < h.n_trees; ++k)
    for (int64_t l = h.tree_leaf_off[k]; l < h.tree_leaf_off[k + 1]; ++l) leaf_tree[size_t(l)] = k;
  CUDA_TRY(upload(t, &t->d_leaf_tree, leaf_tree));
  CUDA_TRY(dalloc(t, &t->d_io, sizeof(TreeIo) * size_t(nr)));
  CUDA_TRY(dalloc(t, &t->d_io_net, sizeof(double*)));
  // The tree's stream carries the level-by-level passes, short launches on the critical path;
  // the second stream carries the leaf and boundary kernels, which only need to finish before the
  // downward pass.  With the first at the higher priority, the blocks of a pass are scheduled
  // ahead of the waiting blocks of the long kernel beside it.
  int prio_low = 0, prio_high = 0;
  CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  t->prio_high = prio_high;
  CUDA_TRY(cudaStreamCreateWithPriority(&t->stream, cudaStreamNonBlocking, prio_high));
  CUDA_TRY(cudaStreamCreateWithPriority(&t->stream2, cudaStreamNonBlocking, prio_low));
  CUDA_TRY(cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&t->ev_m2m, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&t->ev_in, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&t->ev_out, cudaEventDisableTiming));
  for (auto& e : t->ev) CUDA_TRY(cudaEventCreate(&e));
  t->dev_ready = true;
  return FMM_OK;
}

static int ensure_mixed(fmm_tree* t) {
  if (t->mixed_ready) return FMM_OK;
  const int64_t nc = t->h.n_sub * kCells;
  CUDA_TRY(dalloc(t, &t->d_mom32, sizeof(float) * kNMom * nc));
  CUDA_TRY(cudaMemset(t->d_mom32, 0, sizeof(float) * kNMom * nc));  // leaf cells keep zeros
  CUDA_TRY(dalloc(t, &t->d_m32, sizeof(float) * nc));
  CUDA_TRY(dalloc(t, &t->d_loc32, sizeof(float) * 20 * nc));
  const int64_t nr = t->h.n_trees;
  CUDA_TRY(dalloc(t, &t->d_root_part32, sizeof(float) * nr * kRootChunks * 20 * kCells));
  CUDA_TRY(dalloc(t, &t->d_root_part_ac, sizeof(double) * nr * kRootChunks * 3 * kCells));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_stage<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageSmem));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_stage<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageSmemSrc));
  CUDA_TRY(cudaFuncSetAttribute(k_m2l_stage_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageSmem));
  t->mixed_ready = true;
  return FMM_OK;
}

static int ensure_df(fmm_tree* t) {
  if (t->df_ready) return FMM_OK;
  const int64_t nc = t->h.n_sub * kCells;
  CUDA_TRY(dalloc(t, &t->d_momff, sizeof(dfloat) * kNMom * nc));
  CUDA_TRY(cudaMemset(t->d_momff, 0, sizeof(dfloat) * kNMom * nc));  // leaf cells keep zeros
  CUDA_TRY(dalloc(t, &t->d_massff, sizeof(dfloat) * nc));
  t->df_ready = true;
  return FMM_OK;
}

static int ensure_src(fmm_tree* t, bool mixed) {
  const int64_t nc = t->h.n_sub * kCells;
  if (!t->src_ready) {
    CUDA_TRY(dalloc(t, &t->d_smom, sizeof(double) * kNMom * nc));
    CUDA_TRY(cudaMemset(t->d_smom, 0, sizeof(double) * kNMom * nc));  // leaf cells keep zeros
    CUDA_TRY(dalloc(t, &t->d_smtl, sizeof(double) * kNMom * nc));
    CUDA_TRY(cudaMemset(t->d_smtl, 0, sizeof(double) * kNMom * nc));
    CUDA_TRY(dalloc(t, &t->d_sloc, sizeof(double) * 20 * nc));
    t->src_ready = true;
  }
  if (mixed && !t->src32_ready) {
    CUDA_TRY(dalloc(t, &t->d_smom32, sizeof(float) * kNMom * nc));
    CUDA_TRY(cudaMemset(t->d_smom32, 0, sizeof(float) * kNMom * nc));
    CUDA_TRY(dalloc(t, &t->d_sloc32, sizeof(float) * 20 * nc));
    CUDA_TRY(dalloc(t, &t->d_src32, sizeof(float) * 28 * nc));
    CUDA_TRY(cudaMemset(t->d_src32, 0, sizeof(float) * 28 * nc));  // leaf cells keep zeros
    t->src32_ready = true;
  }
  return FMM_OK;
}

static int32_t block_code(uint32_t kind, uint32_t parity, uint32_t index) {
  return int32_t((kind << 30) | (parity << 27) | index);
}

// Host copy of the internal cell order (parity-major inside a subgrid).
static inline int host_cidx(int a, int b, int c) {
  return (((a & 1) << 2 | (b & 1) << 1 | (c & 1)) << 6) | (a >> 1) << 4 | (b >> 1) << 2 | (c >> 1);
}
static inline int slot_of(int p) { return p < 0 ? 0 : (p < 8 ? 1 : 2); }

// Pair lists of the leaf targets at refinement boundaries (Sec. 2.2 same-level interactions,
// with the mixed-level pairs read as direct sums): for every cell of every boundary leaf subgrid,
//   - multipole partners: stencil entries that land in a refined same-level neighbour;
//   - point-mass partners: the 8 leaf children of each near entry in a refined same-level
//     neighbour, and the near entries of the parent cell that land in a leaf one level coarser.
// Targets without partners are dropped; the rest are sorted by estimated work, largest first.
struct BoundaryLists {
  std::vector<int32_t> cell, m_off, p_off;
  std::vector<uint16_t> m_e;  // multipole partners: neighbour slot << 9 | internal cell index
  std::vector<uint16_t> p_e;  // point-mass partners: kind << 15 | neighbour slot << 9 | cell index
  std::vector<double> cost;  // per target, in the order of `cell`
};

static std::string boundary_lists(const HostTree& h, const Stencil& st,
                                  const std::vector<int32_t>& work_bnd, BoundaryLists& out) {
  const double c_m = 150, c_p = 20;
  // an entry's offsets x_A - x_first in units of dx / 4 (the kernel forms the same numbers, and
  // kind 0 lowers each by up to 2 for the children): all must index the kernel's table
  bool code_ok = true;
  auto check = [&](int qx, int qy, int qz) {
    for (int v : {qx, qy, qz}) code_ok = code_ok && v <= kCodeMax && v - 2 >= -kCodeMax;
  };
  // first pass: every target's lists in subgrid order, flat
  std::vector<int32_t> cell;
  std::vector<int64_t> moff{0}, poff{0};
  std::vector<uint16_t> ms, ps;
  std::vector<int64_t> npt{0};  // point masses per target, running
  int64_t n_points = 0;
  for (int32_t s : work_bnd) {
    int32_t nb[27], pnb[27];
    bool nb_ref[27], pnb_leaf[27];
    const int32_t P = h.parent[s];
    for (int k = 0; k < 27; ++k) {
      nb[k] = h.nbr[27 * s + k];
      nb_ref[k] = nb[k] >= 0 && !h.leaf[nb[k]];
      pnb[k] = h.nbr[27 * P + k];
      pnb_leaf[k] = pnb[k] >= 0 && h.leaf[pnb[k]];
    }
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        for (int c = 0; c < 8; ++c) {
          const int par = (a & 1) << 2 | (b & 1) << 1 | (c & 1);
          const size_t m0 = ms.size(), p0 = ps.size();
          const auto& offs = st.offs[par];
          for (size_t q = 0; q < offs.size(); ++q) {
            int dx, dy, dz;
            unpack_offset(offs[q], dx, dy, dz);
            const int px = a + dx, py = b + dy, pz = c + dz;
            const int sl = slot_of(px) * 9 + slot_of(py) * 3 + slot_of(pz);
            if (!nb_ref[sl]) continue;
            ms.push_back(uint16_t((sl << 9) | host_cidx(px & 7, py & 7, pz & 7)));
          }
          for (int32_t code : st.near) {
            int dx, dy, dz;
            unpack_offset(code, dx, dy, dz);
            const int px = a + dx, py = b + dy, pz = c + dz;
            const int sl = slot_of(px) * 9 + slot_of(py) * 3 + slot_of(pz);
            if (!nb_ref[sl]) continue;
            // the 8 leaf children C (o = 0..7) of the near cell: x_A - x_C = (1/2 - o - 2 d) dx_(l+1)
            // = (1 - 2 o - 4 d) dx_l / 4
            ps.push_back(uint16_t((sl << 9) | host_cidx(px & 7, py & 7, pz & 7)));
            check(1 - 4 * dx, 1 - 4 * dy, 1 - 4 * dz);
            n_points += 8;
          }
          const int ga = h.ijk[3 * s] * 8 + a, gb = h.ijk[3 * s + 1] * 8 + b, gc = h.ijk[3 * s + 2] * 8 + c;
          const int ja = (ga >> 1) - h.ijk[3 * P] * 8, jb = (gb >> 1) - h.ijk[3 * P + 1] * 8,
                    jc = (gc >> 1) - h.ijk[3 * P + 2] * 8;
          for (int32_t code : st.near) {
            int dx, dy, dz;
            unpack_offset(code, dx, dy, dz);
            const int px = ja + dx, py = jb + dy, pz = jc + dz;
            const int sl = slot_of(px) * 9 + slot_of(py) * 3 + slot_of(pz);
            if (!pnb_leaf[sl]) continue;
            // a leaf i one level coarser: x_A - x_i = ((g_A & 1) - 1/2 - 2 d) dx_l
            // = (4 (g_A & 1) - 2 - 8 d) dx_l / 4
            ps.push_back(uint16_t(0x8000 | (sl << 9) | host_cidx(px & 7, py & 7, pz & 7)));
            check(4 * (ga & 1) - 2 - 8 * dx, 4 * (gb & 1) - 2 - 8 * dy, 4 * (gc & 1) - 2 - 8 * dz);
            n_points += 1;
          }
          if (ms.size() == m0 && ps.size() == p0) continue;  // no partners
          cell.push_back(int32_t(int64_t(s) * kCells + host_cidx(a, b, c)));
          moff.push_back(int64_t(ms.size()));
          poff.push_back(int64_t(ps.size()));
          npt.push_back(n_points);
        }
  }
  if (!code_ok) return "point-pair offset outside the table";
  if (ms.size() > size_t(INT32_MAX) || ps.size() > size_t(INT32_MAX))
    return "boundary pair lists exceed 2^31 entries";
  // second pass: targets by estimated work, largest first
  const size_t n = cell.size();
  std::vector<double> cost(n);
  std::vector<size_t> order(n);
  for (size_t k = 0; k < n; ++k) {
    cost[k] = c_m * double(moff[k + 1] - moff[k]) + c_p * double(npt[k + 1] - npt[k]);
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  out = BoundaryLists();
  out.cell.resize(n);
  out.cost.resize(n);
  out.m_off.resize(n + 1);
  out.p_off.resize(n + 1);
  out.m_e.resize(ms.size());
  out.p_e.resize(ps.size());
  int64_t mo = 0, po = 0;
  out.m_off[0] = out.p_off[0] = 0;
  for (size_t r = 0; r < n; ++r) {
    const size_t k = order[r];
    out.cell[r] = cell[k];
    out.cost[r] = cost[k];
    std::copy(ms.begin() + moff[k], ms.begin() + moff[k + 1], out.m_e.begin() + mo);
    std::copy(ps.begin() + poff[k], ps.begin() + poff[k + 1], out.p_e.begin() + po);
    mo += moff[k + 1] - moff[k];
    po += poff[k + 1] - poff[k];
    out.m_off[r + 1] = int32_t(mo);
    out.p_off[r + 1] = int32_t(po);
  }
  return "";
}

static std::vector<int32_t> general_blocks(const HostTree& h, const Stencil& st,
                                           const std::vector<int32_t>& work,
                                           const BoundaryLists& bnd, bool whole) {
  const double c_rr = 230, c_pt = 20, c_iter = 4;
  // per target parity: how many (cell, offset) pairs land in each neighbour slot
  double st_slot[8][27] = {};
  for (int c = 0; c < kCells; ++c) {
    int a = c / 64, b = (c / 8) % 8, z = c % 8;
    int par = (a & 1) << 2 | (b & 1) << 1 | (z & 1);
    for (int32_t code : st.offs[par]) {
      int dx, dy, dz;
      unpack_offset(code, dx, dy, dz);
      st_slot[par][((a + dx) >> 3) * 9 + ((b + dy) >> 3) * 3 + ((z + dz) >> 3) + 13]++;
    }
  }
  std::vector<std::pair<double, int32_t>> items;
  for (int r = 0; r < h.n_trees; ++r) {
    const double root_cost = 64.0 * 64.0 * (h.leaf[r] ? c_pt : c_rr);
    for (int ch = 0; ch < kRootChunks; ++ch)
      for (int p = 0; p < 8; ++p) items.push_back({root_cost, block_code(0, p, uint32_t(r * 8 + ch))});
  }
  for (int32_t s : work)
    for (int p = 0; p < 8; ++p) {
      double cost = c_iter * 64 * double(st.offs[p].size());
      for (int k = 0; k < 27; ++k) {
        int32_t q = h.nbr[27 * s + k];
        if (q >= 0) cost += st_slot[p][k] * c_rr;  // leaf partners take the full formula too
      }
      items.push_back({cost, block_code(1, p, s)});
    }
  for (size_t c = 0; c * 64 < bnd.cell.size(); ++c) {
    double cost = 0;
    for (size_t k = c * 64; k < std::min(bnd.cell.size(), c * 64 + 64); ++k) cost += bnd.cost[k];
    items.push_back({cost, block_code(2, 0, uint32_t(c))});
  }
  if (whole) {
    // merge the 8 parity items of each unit into one item (code with parity 0)
    std::map<int32_t, double> unit;
    std::vector<int32_t> order;
    for (auto& it : items) {
      int32_t key = it.second & ~int32_t(7 << 27);
      if (!unit.count(key)) order.push_back(key);
      unit[key] += it.first;
    }
    items.clear();
    for (int32_t key : order) items.push_back({unit[key], key});
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                     return x.first > y.first;
                   });
  std::vector<int32_t> out;
  out.reserve(items.size());
  for (auto& it : items) out.push_back(it.second);
  return out;
}

// Blocks of k_m2l_split (mixed path).  The root chunks, and the boundary targets whose lists
// are long (estimated cost above kSplitCost), get four lanes per target (kinds 0 and 2); the
// other boundary targets go 256 to a block with one lane each (kind 3), where splitting would
// only add per-target overhead.  The choice depends on the target's own lists alone, so a tree
// gives the same results alone and inside a forest.  Largest per-lane work first.
constexpr double kSplitCost = 6000;  // about 40 multipole partners
// the thresholds of the split-lane choices: kSplitCost, a quarter, four times, never split
constexpr double kSplitCosts[kSplitChoices] = {kSplitCost, kSplitCost / 4, kSplitCost * 4, 1e300};
static std::vector<int32_t> split_blocks(const HostTree& h, const std::vector<double>& cost,
                                         double split_cost, int64_t* n_long) {
  const double c_rr = 230, root_lane = 64.0 * c_rr / kSplitLanes;
  std::vector<std::pair<double, int32_t>> items;
  for (int r = 0; r < h.n_trees; ++r)
    for (int ch = 0; ch < kRootChunks; ++ch)
      for (int p = 0; p < 8; ++p) items.push_back({root_lane, block_code(0, p, uint32_t(r * 8 + ch))});
  const int64_t n = int64_t(cost.size());
  int64_t nl = 0;
  while (nl < n && cost[size_t(nl)] > split_cost) ++nl;  // targets are sorted by cost
  *n_long = nl;
  for (int64_t c = 0; c * 64 < nl; ++c)
    items.push_back({cost[size_t(c * 64)] / kSplitLanes, block_code(2, 0, uint32_t(c))});
  for (int64_t c = 0; nl + c * 64 < n; c += 4)
    items.push_back({cost[size_t(nl + c * 64)], block_code(3, 0, uint32_t(c))});
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                     return x.first > y.first;
                   });
  std::vector<int32_t> out;
  out.reserve(items.size());
  for (auto& it : items) out.push_back(it.second);
  return out;
}

// The split-lane choice of a stencil's current mixed launch variant, and its block list.
static inline int split_choice(const StencilDev* sd) { return (sd->mixed_variant / 24) % kSplitChoices; }
static int ensure_split(fmm_tree* t, StencilDev* sd) {
  const int c = split_choice(sd);
  if (sd->d_blocks_split[c]) return FMM_OK;
  std::vector<int32_t> blocks = split_blocks(t->h, sd->bnd_cost, kSplitCosts[c], &sd->n_bt_long[c]);
  sd->n_blocks_split[c] = int64_t(blocks.size());
  CUDA_TRY(upload(t, &sd->d_blocks_split[c], blocks));
  return FMM_OK;
}

static int get_stencil(fmm_tree* t, double theta, StencilDev** out) {
  auto it = t->stencils.find(theta);
  if (it == t->stencils.end()) {
    Stencil st = make_stencil(theta);
    std::vector<int32_t> packed(8 * kStencilCap, 0);
    int n = int(st.offs[0].size());
    for (int p = 0; p < 8; ++p) {
      if (int(st.offs[p].size()) != n || n > kStencilCap)
        return fail(FMM_ERR_THETA, "stencil sizes differ between parities");
      std::copy(st.offs[p].begin(), st.offs[p].end(), packed.begin() + p * kStencilCap);
    }
    StencilDev sd;
    CUDA_TRY(upload(t, &sd.d_stencil, packed));
    CUDA_TRY(upload(t, &sd.d_near, st.near));
    // per parity: stencil entries, then near entries, with their exact 1/|d| and d/|d|^3
    if (n + int(st.near.size()) > kLeafCap) return fail(FMM_ERR_THETA, "stencil too large");
    std::vector<int32_t> loff(8 * kLeafCap, 0), lcode(8 * kLeafCap, 0);
    std::vector<double> lk(8 * kLeafCap * 4, 0.0), ld(8 * kLeafCap * 4, 0.0);
    std::vector<float> lk32(8 * kLeafCap * 4, 0.0f), ld32(8 * kLeafCap * 4, 0.0f);
    std::vector<dfloat> lkff(8 * kLeafCap * 4, dfloat(0)), ldff(8 * kLeafCap * 4, dfloat(0));
    for (int p = 0; p < 8; ++p) {
      std::vector<int32_t> all(st.offs[p]);
      all.insert(all.end(), st.near.begin(), st.near.end());
      for (size_t q = 0; q < all.size(); ++q) {
        int dx, dy, dz;
        unpack_offset(all[q], dx, dy, dz);
        double d2 = double(dx * dx + dy * dy + dz * dz);
        double k0 = 1.0 / std::sqrt(d2), k3 = k0 / d2;
        size_t e = size_t(p) * kLeafCap + q;
        // source halo cell (a + d + 5) of a target of parity p: its parity class and lattice
        // offset from the target's lattice cell
        const int px = (p >> 2) & 1, py = (p >> 1) & 1, pz = p & 1;
        const int hx = px + dx + 5, hy = py + dy + 5, hz = pz + dz + 5;
        loff[e] = ((hx & 1) << 2 | (hy & 1) << 1 | (hz & 1)) * kHaloPar + (hx >> 1) * kHaloSX +
                  (hy >> 1) * kHaloSY + (hz >> 1);
        lcode[e] = all[q];
        double kk[4] = {k0, dx * k3, dy * k3, dz * k3};
        double dd[4] = {double(dx), double(dy), double(dz), 0.0};
        for (int c = 0; c < 4; ++c) {
          lk[4 * e + c] = kk[c];
          lk32[4 * e + c] = float(kk[c]);
          lkff[4 * e + c] = dfloat(kk[c]);
          ldff[4 * e + c] = dfloat(dd[c]);
          ld[4 * e + c] = dd[c];
          ld32[4 * e + c] = float(dd[c]);
        }
      }
    }
    CUDA_TRY(upload(t, &sd.d_ltab_off, loff));
    CUDA_TRY(upload(t, &sd.d_ltab_code, lcode));
    CUDA_TRY(upload(t, &sd.d_ltab_k64, lk));
    CUDA_TRY(upload(t, &sd.d_ltab_k32, lk32));
    CUDA_TRY(upload(t, &sd.d_ltab_d64, ld));
    CUDA_TRY(upload(t, &sd.d_ltab_d32, ld32));
    CUDA_TRY(upload(t, &sd.d_ltab_kff, lkff));
    CUDA_TRY(upload(t, &sd.d_ltab_dff, ldff));
    BoundaryLists bl;
    std::string err = boundary_lists(t->h, st, t->work_bnd, bl);
    if (!err.empty()) return fail(FMM_ERR_ARG, err);
    sd.n_bt = int64_t(bl.cell.size());
    CUDA_TRY(upload(t, &sd.d_bt_cell, bl.cell));
    CUDA_TRY(upload(t, &sd.d_bm_off, bl.m_off));
    CUDA_TRY(upload(t, &sd.d_bm_e, bl.m_e));
    CUDA_TRY(upload(t, &sd.d_bp_off, bl.p_off));
    CUDA_TRY(upload(t, &sd.d_bp_e, bl.p_e));
    std::vector<int32_t> blocks = general_blocks(t->h, st, t->work, bl, false);
    sd.n_blocks = int64_t(blocks.size());
    CUDA_TRY(upload(t, &sd.d_blocks, blocks));
    sd.bnd_cost = bl.cost;
    // staged refined targets: per parity, the stencil entries grouped by partner class, with
    // the partner's lattice offset from a target at lattice cell (0, 0, 0) of that parity
    std::vector<float> stab(8 * kLeafCap * 4, 0.0f);
    std::vector<int32_t> sseg(8 * 9, 0);
    for (int p = 0; p < 8; ++p) {
      const int px = (p >> 2) & 1, py = (p >> 1) & 1, pz = p & 1;
      int e = 0;
      for (int cl = 0; cl < 8; ++cl) {
        sseg[9 * p + cl] = e;
        for (int32_t code : st.offs[p]) {
          int dx, dy, dz;
          unpack_offset(code, dx, dy, dz);
          const int hx = px + dx + 5, hy = py + dy + 5, hz = pz + dz + 5;
          if (hx < 0 || hy < 0 || hz < 0 || hx > 11 || hy > 11 || hz > 11)
            return fail(FMM_ERR_THETA, "stencil reaches beyond the 5-cell rim");
          if (((hx & 1) << 2 | (hy & 1) << 1 | (hz & 1)) != cl) continue;
          const int32_t off = (hx >> 1) * kStageSX + (hy >> 1) * kStageSY + (hz >> 1);
          float* f = &stab[(size_t(p) * kLeafCap + e) * 4];
          f[0] = float(dx);
          f[1] = float(dy);
          f[2] = float(dz);
          std::memcpy(&f[3], &off, sizeof(off));
          ++e;
        }
      }
      sseg[9 * p + 8] = e;
    }
    CUDA_TRY(upload(t, &sd.d_stage_tab, stab));
    CUDA_TRY(upload(t, &sd.d_stage_seg, sseg));

    sd.n_stencil = n;
    sd.n_near = int(st.near.size());
    // the opening test is monotone in |d|^2: find the largest |d|^2 that is not well separated
    // (root cells are at most 7 apart per axis)
    for (int d2 = 1; d2 <= 3 * 49; ++d2) {
      bool ws = 1.0 / std::sqrt(double(d2)) < theta;
      if (!ws) sd.ws_d2 = d2;
    }
    for (int d2 = sd.ws_d2 + 1; d2 <= 3 * 49; ++d2)
      if (!(1.0 / std::sqrt(double(d2)) < theta)) return fail(FMM_ERR_THETA, "opening test not monotone");
    it = t->stencils.emplace(theta, sd).first;
  }
  *out = &it->second;
  return FMM_OK;
}

static DevArgs make_args(fmm_tree* t, const StencilDev* sd) {
  DevArgs A;
  A.n_cell = t->h.n_sub * kCells;
  A.n_leaf_cells = t->h.n_leaf_sub * kCells;
  A.depth = t->h.depth;
  A.n_roots = t->h.n_trees;
  A.tree_leaf_off = t->d_tree_leaf_off;
  A.level = t->d_level;
  A.ijk = t->d_ijk;
  A.leaf = t->d_leaf;
  A.parent = t->d_parent;
  A.child = t->d_child;
  A.nbr = t->d_nbr;
  A.leaf_sub = t->d_leaf_sub;
  A.leaf_ord = t->d_leaf_ord;
  A.stencil = sd ? sd->d_stencil : nullptr;
  A.near = sd ? sd->d_near : nullptr;
  A.n_stencil = sd ? sd->n_stencil : 0;
  A.n_near = sd ? sd->n_near : 0;
  A.ws_d2 = sd ? sd->ws_d2 : 0;
  A.ltab_off = sd ? sd->d_ltab_off : nullptr;
  A.ltab_code = sd ? sd->d_ltab_code : nullptr;
  A.ltab_k64 = sd ? sd->d_ltab_k64 : nullptr;
  A.ltab_k32 = sd ? sd->d_ltab_k32 : nullptr;
  A.ltab_d64 = sd ? sd->d_ltab_d64 : nullptr;
  A.ltab_d32 = sd ? sd->d_ltab_d32 : nullptr;
  A.ltab_kff = sd ? sd->d_ltab_kff : nullptr;
  A.ltab_dff = sd ? sd->d_ltab_dff : nullptr;
  A.mom = t->d_mom;
  A.mtl = t->d_mtl;
  A.mom32 = t->d_mom32;
  A.m32 = t->d_m32;
  A.momff = t->d_momff;
  A.massff = t->d_massff;
  A.loc = t->d_loc;
  A.loc32 = t->d_loc32;
  A.ac = t->d_ac;
  A.root_part = t->d_root_part;
  A.root_part32 = t->d_root_part32;
  A.root_part_ac = t->d_root_part_ac;
  A.status = t->d_status;
  A.stage_tab = sd ? reinterpret_cast<const float4*>(sd->d_stage_tab) : nullptr;
  A.stage_seg = sd ? sd->d_stage_seg : nullptr;
  A.n_bt_long = sd ? sd->n_bt_long[split_choice(sd)] : 0;
  A.wait_cycles = t->wait_cycles > 0 ? t->wait_cycles : kStageWaitCycles;
  A.smom = t->d_smom;
  A.smtl = t->d_smtl;
  A.smom32 = t->d_smom32;
  A.src32 = t->d_src32;
  A.sloc = t->d_sloc;
  A.sloc32 = t->d_sloc32;
  A.n_bt = sd ? sd->n_bt : 0;
  A.bt_cell = sd ? sd->d_bt_cell : nullptr;
  A.bm_off = sd ? sd->d_bm_off : nullptr;
  A.bm_e = sd ? sd->d_bm_e : nullptr;
  A.bp_off = sd ? sd->d_bp_off : nullptr;
  A.bp_e = sd ? sd->d_bp_e : nullptr;
  A.leaf_tree = t->d_leaf_tree;
  A.io = t->d_io;
  A.io_net = t->d_io_net;
  return A;
}

// Launches kernel k on stream st with a scheduling priority given as a launch attribute (captured
// graphs keep it as the kernel node's priority, which a stream's own priority does not reliably
// become).
template <typename... P, typename... Args>
static cudaError_t launch_prio(int prio, void (*k)(P...), dim3 grid, dim3 block, size_t smem,
                               cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

static inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

static int record(fmm_tree* t, int k, cudaStream_t st) {
  if (!t->profiling) return FMM_OK;
  // inside a capture the record becomes an event node of the graph
  CUDA_TRY(cudaEventRecordWithFlags(t->ev[k], st, t->capturing ? cudaEventRecordExternal : 0));
  return FMM_OK;
}

// Writes the caller's pointers of this call into the device table (one launch per kIoChunk trees).
static int set_io(fmm_tree* t, const std::vector<TreeIo>& io, double* net, cudaStream_t st,
                  int32_t* launches) {
  const int n = int(io.size());  // the trees of t: at least one
  const int chunks = (n + kIoChunk - 1) / kIoChunk;
  for (int q = 0; q < chunks; ++q) {
    IoChunk c;
    c.net = net;
    c.first = q * kIoChunk;
    c.count = std::min(kIoChunk, n - c.first);
    for (int j = 0; j < c.count; ++j) c.e[j] = io[size_t(c.first + j)];
    k_set_io<<<1, kIoChunk, 0, st>>>(c, t->d_io, t->d_io_net);
    CUDA_TRY(cudaGetLastError());
  }
  *launches = chunks;
  return FMM_OK;
}

static int launch_net(fmm_tree* t, const DevArgs& A, cudaStream_t st) {
  k_net_partial<<<unsigned(t->net_blocks), kReduceThreads, 0, st>>>(
      A, t->d_partials, t->d_net_count, t->d_net_plan, t->d_net_tree_plan);
  CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

// Downward pass below the root: one launch per level with refined subgrids (their cells'
// totals need the parent level's), then one launch evaluating every leaf octant of every level
// from its parent cell's total.
template <bool SRC>
static int launch_down(fmm_tree* t, const DevArgs& A, bool mixed, cudaStream_t st, int32_t* nl) {
  const HostTree& h = t->h;
  for (int l = 1; l <= h.depth; ++l) {
    const int64_t nr = t->ref_off[l + 1] - t->ref_off[l];
    if (nr == 0) continue;
    const int32_t* ref = t->d_ref_sub + t->ref_off[l];
    if (mixed) k_down<true, SRC><<<unsigned(nr * 8), 64, 0, st>>>(A, l, ref, int(nr * 8), nullptr);
    else k_down<false, SRC><<<unsigned(nr * 8), 64, 0, st>>>(A, l, ref, int(nr * 8), nullptr);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
  }
  const int64_t no = t->oct_leaf_off[h.depth + 1];  // every leaf octant, parents of all levels
  if (no > 0) {
    if (mixed) k_down<true, SRC><<<unsigned(no), 64, 0, st>>>(A, 0, nullptr, 0, t->d_oct_leaf);
    else k_down<false, SRC><<<unsigned(no), 64, 0, st>>>(A, 0, nullptr, 0, t->d_oct_leaf);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
  }
  return FMM_OK;
}

// The level passes of one direction as one cooperative launch of k_levels (fmm_set_persistent):
// a grid of at most the blocks that fit on the device at once, and never more than the largest
// phase has items.  The barrier words are cleared before every launch, so a launch that timed out
// leaves nothing behind.
static int launch_levels(fmm_tree* t, const DevArgs& A, const LevelPlan& P, bool mixed, int mode,
                         int prio, cudaStream_t st, int32_t* nl) {
  if (P.n == 0) return FMM_OK;
  int& cap = t->levels_cap[mixed ? 1 : 0];
  if (cap == 0) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (mixed) CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels<true>, 64, 0));
    else CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels<false>, 64, 0));
    if (!coop || per_sm < 1) return fail(FMM_ERR_CUDA, "persistent level passes: no cooperative launch");
    cap = per_sm * sms;
  }
  int most = 1;
  for (int p = 0; p < P.n; ++p) most = std::max(most, P.items[p]);
  CUDA_TRY(cudaMemsetAsync(t->d_bar, 0, 2 * sizeof(unsigned), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(std::min(cap, most)));
  cfg.blockDim = dim3(64);
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = prio;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  if (mixed) CUDA_TRY(cudaLaunchKernelEx(&cfg, k_levels<true>, A, P, mode, t->d_bar));
  else CUDA_TRY(cudaLaunchKernelEx(&cfg, k_levels<false>, A, P, mode, t->d_bar));
  ++*nl;
  return FMM_OK;
}
static bool add_phase(LevelPlan& P, int kind, int lev, int64_t items, const int32_t* list) {
  if (items <= 0) return true;
  if (P.n == kMaxPhases || items > INT32_MAX) return false;
  P.kind[P.n] = kind;
  P.lev[P.n] = lev;
  P.items[P.n] = int(items);
  P.list[P.n] = list;
  ++P.n;
  return true;
}

// All launches of one solve, in order, on stream st (which may be capturing).
static int enqueue_src(fmm_tree* t, const StencilDev* sd, bool mixed, cudaStream_t st, int32_t* nl);

static int enqueue_solve(fmm_tree* t, const StencilDev* sd, int mode, int amc, bool net,
                         bool src, cudaStream_t st, int32_t* launches) {
  const HostTree& h = t->h;
  DevArgs A = make_args(t, sd);
  const bool mixed = mode == FMM_MIXED, df = mode == FMM_DF64;
  int rc;
  int32_t nl = 0;
  if ((rc = record(t, 0, st))) return rc;
  // upward pass
  k_p2m<<<blocks_for(A.n_leaf_cells, 256), 256, 0, st>>>(A, mode);
  CUDA_TRY(cudaGetLastError());
  ++nl;
  // The same-level leaf pairs need only the leaf masses: their kernel runs on the second stream,
  // forked from here, beside the level-by-level (latency-bound) upward pass, or (mixed launch
  // variants with p = 1) forked after the upward pass, beside the refined targets' kernel.
  const int v_ref = sd->mixed_variant % 4, v_leaf = (sd->mixed_variant / 4) % 3,
            v_place = mixed ? (sd->mixed_variant / 12) % 2 : 0;
  auto launch_leaf = [&]() -> int {
    CUDA_TRY(cudaEventRecord(t->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(t->stream2, t->ev_fork, 0));
    int rc2 = record(t, 8, t->stream2);
    if (rc2) return rc2;
    if (t->n_work_leaf > 0) {
      cudaStream_t s2 = t->stream2;
      if (mixed && v_leaf == 0)
        k_m2l_leaf4<false, 2><<<unsigned((t->n_work_leaf + 1) / 2), kLeaf4Threads, kLeaf4Smem, s2>>>(
            A, t->d_work_leaf, t->n_work_leaf);
      else if (mixed && v_leaf == 2)
        k_m2l_leaf4<false, 4><<<unsigned((t->n_work_leaf + 3) / 4), 2 * kLeaf4Threads, leaf4_smem<4>(), s2>>>(
            A, t->d_work_leaf, t->n_work_leaf);
      else if (mixed)
        k_m2l_leaf<float, false><<<unsigned(t->n_work_leaf), kLeafThreads, kHaloWords * sizeof(float), s2>>>(
            A, t->d_work_leaf);
      else if (df)
        k_m2l_leaf<dfloat, false><<<unsigned(t->n_work_leaf), kLeafThreads, kHaloWords * sizeof(dfloat), s2>>>(
            A, t->d_work_leaf);
      else
        k_m2l_leaf<double, false><<<unsigned(t->n_work_leaf), kLeafThreads, kHaloWords * sizeof(double), s2>>>(
            A, t->d_work_leaf);
      CUDA_TRY(cudaGetLastError());
      ++nl;
    }
    return record(t, 9, t->stream2);
  };
  if (v_place == 0 && (rc = launch_leaf())) return rc;
  // octants whose children are leaves need only the leaf masses: every level's in one launch;
  // then the octants with refined children, finest level first (or all of it in one persistent
  // launch)
  const int64_t n_walsh = t->oct_leaf_off[h.depth + 1];
  LevelPlan up = {}, down = {};
  bool persistent = t->persistent != 0 && add_phase(up, 0, 0, n_walsh, t->d_oct_leaf);
  for (int l = h.depth - 1; persistent && l >= 0; --l)
    persistent = add_phase(up, 1, l, (t->oct_ref_off[l + 1] - t->oct_ref_off[l]) * 8,
                           t->d_oct_ref + t->oct_ref_off[l]);
  for (int l = 1; persistent && l <= h.depth; ++l)
    persistent = add_phase(down, 2, l, (t->ref_off[l + 1] - t->ref_off[l]) * 8, t->d_ref_sub + t->ref_off[l]);
  persistent = persistent && add_phase(down, 3, 0, t->oct_leaf_off[h.depth + 1], t->d_oct_leaf);
  if (persistent) {
    if ((rc = launch_levels(t, A, up, mixed, mode, t->prio_high, st, &nl))) return rc;
  } else if (n_walsh > 0) {
    CUDA_TRY(launch_prio(t->prio_high, k_m2m, dim3(unsigned(n_walsh)), dim3(kM2MThreads), 0, st, A,
                         (const int32_t*)t->d_oct_leaf, int(n_walsh), (const int32_t*)nullptr, mode));
    ++nl;
  }
  for (int l = h.depth - 1; !persistent && l >= 0; --l) {
    const int64_t nr_oct = t->oct_ref_off[l + 1] - t->oct_ref_off[l];
    if (nr_oct > 0) {
      CUDA_TRY(launch_prio(t->prio_high, k_m2m, dim3(unsigned(nr_oct * 8)), dim3(kM2MThreads), 0, st, A,
                           (const int32_t*)nullptr, 0, (const int32_t*)(t->d_oct_ref + t->oct_ref_off[l]),
                           mode));
      ++nl;
    }
  }

  if ((rc = record(t, 1, st))) return rc;
  if (v_place == 1 && (rc = launch_leaf())) return rc;
  // interactions of refined targets, the root level and boundary leaf targets (these add onto
  // the leaf kernel's output, so they follow it).  Mixed path, by the launch variant of this
  // tree and theta (kMixedVariants): refined subgrids by k_m2l_stage on this stream while the
  // root and boundary kernel follows the leaf kernel on the second (one staging block per SM
  // leaves room for theirs), or both on this stream, or by k_m2l_ref's per-parity blocks
  // reading their partners from L2; the leaf pairs by k_m2l_leaf4 or k_m2l_leaf<float>.
  const bool staged = mixed && !t->work.empty() && v_ref != 2;
  const bool split2 = staged && (v_ref == 0 || v_ref == 3);  // root and boundary kernel on the second stream
  if (split2) {
    CUDA_TRY(cudaEventRecord(t->ev_m2m, st));
    CUDA_TRY(cudaStreamWaitEvent(t->stream2, t->ev_m2m, 0));
    const int sc = split_choice(sd);
    if (sd->n_blocks_split[sc] > 0) {
      k_m2l_split<float><<<unsigned(sd->n_blocks_split[sc]), 64 * kSplitLanes, 0, t->stream2>>>(
          A, sd->d_blocks_split[sc], amc);
      CUDA_TRY(cudaGetLastError());
      ++nl;
    }
  }
  CUDA_TRY(cudaEventRecord(t->ev_join, t->stream2));
  if (split2) {
    if ((rc = record(t, 6, st))) return rc;
    if (v_ref == 3)
      CUDA_TRY(launch_prio(t->prio_high, k_m2l_stage_pipe, dim3(unsigned(t->work.size())),
                           dim3(kStagePipeThreads), kStageSmem, st, A, (const int32_t*)t->d_work, amc));
    else
      CUDA_TRY(launch_prio(t->prio_high, k_m2l_stage<false>, dim3(unsigned(t->work.size())),
                           dim3(kStageThreads), kStageSmem, st, A, (const int32_t*)t->d_work, amc));
    CUDA_TRY(cudaGetLastError());
    ++nl;
    if ((rc = record(t, 7, st))) return rc;
    CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
  } else {
    CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
    if (mixed && v_ref == 2) {
      k_m2l_ref<float, kM2LThreads><<<unsigned(sd->n_blocks), kM2LThreads, 0, st>>>(A, sd->d_blocks, amc);
    } else if (mixed) {
      k_m2l_split<float><<<unsigned(sd->n_blocks_split[split_choice(sd)]), 64 * kSplitLanes, 0, st>>>(
          A, sd->d_blocks_split[split_choice(sd)], amc);
      if (staged) {
        CUDA_TRY(cudaGetLastError());
        ++nl;
        if ((rc = record(t, 6, st))) return rc;
        k_m2l_stage<false><<<unsigned(t->work.size()), kStageThreads, kStageSmem, st>>>(A, t->d_work, amc);
        CUDA_TRY(cudaGetLastError());
        if ((rc = record(t, 7, st))) return rc;
      }
    } else if (df) {
      k_m2l_ref<dfloat, kM2LThreads><<<unsigned(sd->n_blocks), kM2LThreads, 0, st>>>(A, sd->d_blocks, amc);
    } else {
      k_m2l_ref<double, kM2LThreads><<<unsigned(sd->n_blocks), kM2LThreads, 0, st>>>(A, sd->d_blocks, amc);
    }
    CUDA_TRY(cudaGetLastError());
    ++nl;  // the last (or only) launch of this branch
  }
  if ((rc = record(t, 2, st))) return rc;
  // downward pass: the roots, then per level the refined cells' totals and the leaf cells
  if (mixed) k_root_total<true, false><<<blocks_for(int64_t(h.n_trees) * kRootComps * kCells, 128), 128, 0, st>>>(A);
  else k_root_total<false, false><<<blocks_for(int64_t(h.n_trees) * kRootComps * kCells, 128), 128, 0, st>>>(A);
  CUDA_TRY(cudaGetLastError());
  ++nl;
  if (persistent) {
    if ((rc = launch_levels(t, A, down, mixed, mode, 0, st, &nl))) return rc;
  } else if ((rc = launch_down<false>(t, A, mixed, st, &nl))) {
    return rc;
  }
  if ((rc = record(t, 3, st))) return rc;
  if (net) {
    if ((rc = launch_net(t, A, st))) return rc;
    nl += 1;
  }
  if ((rc = record(t, 4, st))) return rc;
  // time-derivative solve: rho's centres of mass and lists, the source's moments (it reuses the
  // root partial sums, which the rho downward pass has consumed)
  if (src && (rc = enqueue_src(t, sd, mixed, st, &nl))) return rc;
  *launches = nl;
  return FMM_OK;
}

static int enqueue_src(fmm_tree* t, const StencilDev* sd, bool mixed, cudaStream_t st, int32_t* nl) {
  const HostTree& h = t->h;
  DevArgs A = make_args(t, sd);
  const int mx = mixed ? 1 : 0;
  k_p2m_src<<<blocks_for(A.n_leaf_cells, 256), 256, 0, st>>>(A, mx);
  CUDA_TRY(cudaGetLastError());
  ++*nl;
  // as in the rho solve: the leaf kernel on the second stream beside the upward pass; the root
  // and boundary kernel after it (it adds onto its output) and after the upward pass; the
  // refined subgrids (mixed: the staging kernel) on this stream
  CUDA_TRY(cudaEventRecord(t->ev_fork, st));
  CUDA_TRY(cudaStreamWaitEvent(t->stream2, t->ev_fork, 0));
  if (t->n_work_leaf > 0) {
    if (mixed)
      k_m2l_leaf4<true><<<unsigned((t->n_work_leaf + 1) / 2), kLeaf4Threads, kLeaf4Smem, t->stream2>>>(
          A, t->d_work_leaf, t->n_work_leaf);
    else
      k_m2l_leaf<double, true><<<unsigned(t->n_work_leaf), kLeafThreads, kHaloWords * sizeof(double),
                                 t->stream2>>>(A, t->d_work_leaf);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
  }
  for (int l = h.depth - 1; l >= 0; --l) {
    const int64_t nw = t->oct_leaf_off[l + 1] - t->oct_leaf_off[l];
    const int64_t nr = t->oct_ref_off[l + 1] - t->oct_ref_off[l];
    if (nw + nr == 0) continue;
    k_m2m_src<<<unsigned(nw + nr), 64, 0, st>>>(A, t->d_oct_leaf + t->oct_leaf_off[l], int(nw),
                                                 t->d_oct_ref + t->oct_ref_off[l], mx);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
  }
  if (mixed) {
    CUDA_TRY(cudaEventRecord(t->ev_m2m, st));
    CUDA_TRY(cudaStreamWaitEvent(t->stream2, t->ev_m2m, 0));
    k_m2l_split_src<float><<<unsigned(sd->n_blocks_split[split_choice(sd)]), 64 * kSplitLanes, 0,
                              t->stream2>>>(A, sd->d_blocks_split[split_choice(sd)]);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
    CUDA_TRY(cudaEventRecord(t->ev_join, t->stream2));
    if (!t->work.empty()) {
      k_m2l_stage<true><<<unsigned(t->work.size()), kStageThreads, kStageSmemSrc, st>>>(A, t->d_work, 0);
      CUDA_TRY(cudaGetLastError());
      ++*nl;
    }
    CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
  } else {
    CUDA_TRY(cudaEventRecord(t->ev_join, t->stream2));
    CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
    k_m2l_ref_src<double, kM2LThreads><<<unsigned(sd->n_blocks), kM2LThreads, 0, st>>>(A, sd->d_blocks);
    CUDA_TRY(cudaGetLastError());
    ++*nl;
  }
  if (mixed) k_root_total<true, true><<<blocks_for(int64_t(h.n_trees) * kRootComps * kCells, 128), 128, 0, st>>>(A);
  else k_root_total<false, true><<<blocks_for(int64_t(h.n_trees) * kRootComps * kCells, 128), 128, 0, st>>>(A);
  CUDA_TRY(cudaGetLastError());
  ++*nl;
  int rc = launch_down<true>(t, A, mixed, st, nl);
  if (rc) return rc;
  return FMM_OK;
}

// Captures the launches of one solve configuration into a graph and instantiates it.
static int capture_graph(fmm_tree* t, const StencilDev* sd, int mode, int amc, bool net,
                         bool src, fmm_tree::Graph* out) {
  CUDA_TRY(cudaStreamBeginCapture(t->stream, cudaStreamCaptureModeThreadLocal));
  t->capturing = true;
  int32_t nl = 0;
  int rc = enqueue_solve(t, sd, mode, amc, net, src, t->stream, &nl);
  t->capturing = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(t->stream, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : fail(FMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(FMM_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
  out->exec = x;
  out->launches = nl;
  return FMM_OK;
}

// One solve of every tree of t: io[k] holds the caller's arrays of tree k.
static int solve_impl(fmm_tree* t, const std::vector<TreeIo>& io, double theta, int precision,
                      int amc, double* net, cudaStream_t caller) {
  if (!(theta >= kThetaMin && theta < 1.0))
    return fail(FMM_ERR_THETA, "theta must lie in [0.34, 1)");
  if (precision != FMM_FP64 && precision != FMM_MIXED && precision != FMM_DF64)
    return fail(FMM_ERR_ARG, "bad precision");
  const bool src = !io.empty() && io[0].src != nullptr;
  if (src && precision == FMM_DF64)
    return fail(FMM_ERR_ARG, "the time-derivative solve takes FMM_FP64 or FMM_MIXED");
  for (const TreeIo& e : io)
    if (!e.rho || !e.phi || !e.g || (src && (!e.src || !e.phidot)))
      return fail(FMM_ERR_ARG, "null device pointer");
  int rc = ensure_device(t);
  if (rc) return rc;
  const bool mixed = precision == FMM_MIXED;
  if (mixed && (rc = ensure_mixed(t))) return rc;
  if (precision == FMM_DF64 && (rc = ensure_df(t))) return rc;
  if (src && (rc = ensure_src(t, mixed))) return rc;
  StencilDev* sd = nullptr;
  if ((rc = get_stencil(t, theta, &sd))) return rc;
  if ((rc = ensure_split(t, sd))) return rc;
  amc = amc ? 1 : 0;
  fmm_tree::Graph* gr = nullptr;
  if (t->use_graphs) {
    auto key = std::make_tuple(theta, precision, amc, net ? 1 : 0, t->profiling ? 1 : 0, src ? 1 : 0,
                               t->wait_cycles, precision == FMM_MIXED ? sd->mixed_variant : 0,
                               t->persistent);
    auto it = t->graphs.find(key);
    if (it == t->graphs.end()) {
      fmm_tree::Graph fresh;
      if ((rc = capture_graph(t, sd, precision, amc, net != nullptr, src, &fresh))) return rc;
      it = t->graphs.emplace(key, fresh).first;
    }
    gr = &it->second;
  }
  CUDA_TRY(cudaEventRecord(t->ev_in, caller));
  CUDA_TRY(cudaStreamWaitEvent(t->stream, t->ev_in, 0));
  int32_t n_io = 0, n_solve = 0;
  if ((rc = set_io(t, io, net, t->stream, &n_io))) return rc;
  if (gr) {
    CUDA_TRY(cudaGraphLaunch(gr->exec, t->stream));
    n_solve = gr->launches;
  } else if ((rc = enqueue_solve(t, sd, precision, amc, net != nullptr, src, t->stream, &n_solve))) {
    return rc;
  }
  CUDA_TRY(cudaEventRecord(t->ev_out, t->stream));
  CUDA_TRY(cudaStreamWaitEvent(caller, t->ev_out, 0));
  t->ev_recorded = t->profiling;
  t->ev_stage = t->profiling && mixed && !t->work.empty() && sd->mixed_variant % 4 != 2;  // ev[6], ev[7]
  t->launches = n_io + n_solve;
  return FMM_OK;
}

// io table of a forest whose trees' arrays are consecutive parts of one array each
static std::vector<TreeIo> contiguous_io(const fmm_tree* t, const double* rho, double* phi,
                                         double* g) {
  std::vector<TreeIo> io(size_t(t->h.n_trees));
  for (int k = 0; k < t->h.n_trees; ++k) {
    const int64_t o = t->h.tree_leaf_off[k] * kCells;
    io[size_t(k)] = TreeIo{rho ? rho + o : nullptr, phi ? phi + o : nullptr, g ? g + 3 * o : nullptr};
  }
  return io;
}

// ----------------------------------------------------------------------------------------------
// net force and torque of an explicit point set, with no device allocation
// ----------------------------------------------------------------------------------------------
// Some callers cannot allocate device memory: code that runs inside a framework owning all
// device memory through its own pool, or code on a latency-critical path where cudaMalloc and
// its implicit device synchronisation are not acceptable.  For them this reduction keeps its
// per-block partial sums in a fixed, file-scope device array instead of a workspace.  The array
// is shared by every call on a device and is held by every GPU that loads this library until the
// process exits.  Each block overwrites its own slot, so nothing needs clearing between calls;
// calls that overlap on the GPU (different streams, or threads) race on the slots.
constexpr int kStaticNetPointsPerBlock = 4096;
constexpr int kStaticNetMaxBlocks = 2048;  // 2048 * 7 doubles = 112 KiB
constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_net_static_scratch[kStaticNetMaxBlocks * 7];

__global__ void __launch_bounds__(kReduceThreads)
    k_net_points_partial(int64_t n, const double* __restrict__ x, const double* __restrict__ m,
                         const double* __restrict__ g, double* __restrict__ partials) {
  __shared__ double sh[7][kReduceThreads];
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t begin = int64_t(blockIdx.x) * kStaticNetPointsPerBlock;
  int64_t end = begin + kStaticNetPointsPerBlock;
  if (end > n) end = n;
  for (int64_t i = begin + threadIdx.x; i < end; i += kReduceThreads) {
    double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    double fx = m[i] * g[3 * i], fy = m[i] * g[3 * i + 1], fz = m[i] * g[3 * i + 2];
    v[0] += fx;
    v[1] += fy;
    v[2] += fz;
    v[3] += py * fz - pz * fy;
    v[4] += pz * fx - px * fz;
    v[5] += px * fy - py * fx;
    // the normalisation S is a scale, formed in FP32 and summed in FP64 (as in k_net_partial)
    const float xf = float(px), yf = float(py), zf = float(pz), gf = float(fx), hf = float(fy),
                kf = float(fz);
    v[6] += double(sqrtf(xf * xf + yf * yf + zf * zf) * sqrtf(gf * gf + hf * hf + kf * kf));
  }
  block_sum7(v, sh);
  if (threadIdx.x < 7) partials[int64_t(blockIdx.x) * 7 + threadIdx.x] = sh[threadIdx.x][0];
}

static std::mutex g_static_mu;
static double* g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
static int static_net_scratch(double** out) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(FMM_ERR_STATE, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_net_static_scratch));
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return FMM_OK;
}

// ----------------------------------------------------------------------------------------------
// self-consistent-field iteration (Sec. 4.1): the host side (kernels in scf.cu)
// ----------------------------------------------------------------------------------------------
// The leaf cells whose closure touches the x axis: cells with y and z centres at +-dx / 2, i.e.
// global cell indices n/2 - 1 and n/2 of n = 8 2^l cells per axis.
static int ensure_scf(fmm_tree* t) {
  if (t->d_scf_state) return FMM_OK;
  const HostTree& h = t->h;
  std::vector<int64_t> axis;
  for (int64_t ls = 0; ls < h.n_leaf_sub; ++ls) {
    const int32_t s = h.leaf_sub[size_t(ls)];
    const int lev = h.level[s];
    const int64_t half = int64_t(kSub) << lev >> 1;
    for (int b = 0; b < kSub; ++b)
      for (int c = 0; c < kSub; ++c) {
        const int64_t gy = int64_t(h.ijk[3 * s + 1]) * kSub + b, gz = int64_t(h.ijk[3 * s + 2]) * kSub + c;
        if ((gy != half - 1 && gy != half) || (gz != half - 1 && gz != half)) continue;
        for (int a = 0; a < kSub; ++a) axis.push_back(ls * kCells + (a * kSub + b) * kSub + c);
      }
  }
  std::sort(axis.begin(), axis.end());
  t->n_scf_axis = int64_t(axis.size());
  CUDA_TRY(upload(t, &t->d_scf_axis, axis));
  CUDA_TRY(dalloc(t, &t->d_scf_state, sizeof(ScfState)));
  CUDA_TRY(dalloc(t, &t->d_scf_part, sizeof(ScfPartial) * size_t(scf_blocks(h.n_leaf_sub * kCells))));
  CUDA_TRY(dalloc(t, &t->d_scf_apart, sizeof(ScfAxisPartial) * size_t(scf_blocks(t->n_scf_axis))));
  return FMM_OK;
}

static ScfGeom scf_geom(const fmm_tree* t) {
  ScfGeom G;
  G.n_leaf_cells = t->h.n_leaf_sub * kCells;
  G.leaf_sub = t->d_leaf_sub;
  G.level = t->d_level;
  G.ijk = t->d_ijk;
  G.axis = t->d_scf_axis;
  G.n_axis = t->n_scf_axis;
  return G;
}

static int scf_check(fmm_tree* t, const fmm_scf_params* p, ScfProblem* P) {
  if (!t || !p) return fail(FMM_ERR_ARG, "null argument");
  if (t->h.n_trees != 1) return fail(FMM_ERR_ARG, "the SCF iteration takes a single tree");
  if (!(p->M1 > 0.0) || !(p->M2 > 0.0) || !(p->n > 0.0) || !(p->f > 0.0 && p->f <= 1.0) ||
      !(p->J0 > 0.0) || !(p->rho_floor >= 0.0))
    return fail(FMM_ERR_ARG, "SCF parameters: M1, M2, n, J0 > 0, 0 < f <= 1, rho_floor >= 0");
  *P = ScfProblem{p->M1, p->M2, p->n, p->f, p->J0, p->rho_floor};
  int rc = ensure_device(t);
  if (rc) return rc;
  try {
    return ensure_scf(t);
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

// ----------------------------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------------------------
extern "C" {

int fmm_build_tree(int max_level, const uint8_t* refine_flags, int64_t n_flags, fmm_tree** out) {
  if (!out) return fail(FMM_ERR_ARG, "out is null");
  *out = nullptr;
  try {
    std::unique_ptr<fmm_tree> t(new fmm_tree());
    std::string err = build_host_tree(max_level, refine_flags, n_flags, t->h);
    if (!err.empty()) return fail(FMM_ERR_ARG, err);
    *out = t.release();
    return FMM_OK;
  } catch (const std::bad_alloc&) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  } catch (...) {
    return fail(FMM_ERR_ARG, "tree construction failed");
  }
}

void fmm_destroy(fmm_tree* t) {
  if (!t) return;
  int cur = -1;
  bool switched = false;
  if (t->dev_ready && cudaGetDevice(&cur) == cudaSuccess && cur != t->device) {
    switched = cudaSetDevice(t->device) == cudaSuccess;
  }
  for (auto& kv : t->graphs) cudaGraphExecDestroy(kv.second.exec);
  if (t->stream) {
    cudaStreamSynchronize(t->stream);
    cudaStreamDestroy(t->stream);
  }
  if (t->stream2) {
    cudaStreamSynchronize(t->stream2);
    cudaStreamDestroy(t->stream2);
  }
  if (t->ev_fork) cudaEventDestroy(t->ev_fork);
  if (t->ev_join) cudaEventDestroy(t->ev_join);
  if (t->ev_m2m) cudaEventDestroy(t->ev_m2m);
  for (void* p : t->allocs) cudaFree(p);
  for (auto& e : t->ev)
    if (e) cudaEventDestroy(e);
  if (t->ev_in) cudaEventDestroy(t->ev_in);
  if (t->ev_out) cudaEventDestroy(t->ev_out);
  for (cudaStream_t q : {t->hp.in, t->hp.solve, t->hp.out})
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  for (int k = 0; k < 2; ++k)
    for (cudaEvent_t e : {t->hp.copied_in[k], t->hp.solved[k], t->hp.copied_out[k]})
      if (e) cudaEventDestroy(e);
  if (t->hp.caller) cudaEventDestroy(t->hp.caller);
  if (switched) cudaSetDevice(cur);
  delete t;
}

int fmm_build_forest(const fmm_tree* const* trees, int n, fmm_tree** out) {
  if (!out || !trees || n <= 0) return fail(FMM_ERR_ARG, "bad argument");
  *out = nullptr;
  try {
    std::vector<const HostTree*> parts;
    for (int k = 0; k < n; ++k) {
      if (!trees[k]) return fail(FMM_ERR_ARG, "null tree");
      parts.push_back(&trees[k]->h);
    }
    std::unique_ptr<fmm_tree> f(new fmm_tree());
    std::string err = merge_trees(parts, f->h);
    if (!err.empty()) return fail(FMM_ERR_ARG, err);
    *out = f.release();
    return FMM_OK;
  } catch (const std::bad_alloc&) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_forest_info(const fmm_tree* t, int32_t* n_trees, int64_t* leaf_subgrid_offsets) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (n_trees) *n_trees = t->h.n_trees;
  if (leaf_subgrid_offsets)
    for (int k = 0; k <= t->h.n_trees; ++k) leaf_subgrid_offsets[k] = t->h.tree_leaf_off[k];
  return FMM_OK;
}

int fmm_tree_info(const fmm_tree* t, int64_t* n_subgrids, int64_t* n_leaf_subgrids, int32_t* depth) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (n_subgrids) *n_subgrids = t->h.n_sub;
  if (n_leaf_subgrids) *n_leaf_subgrids = t->h.n_leaf_sub;
  if (depth) *depth = t->h.depth;
  return FMM_OK;
}

int fmm_tree_subgrids(const fmm_tree* t, int32_t* rows) {
  if (!t || !rows) return fail(FMM_ERR_ARG, "null argument");
  for (int64_t s = 0; s < t->h.n_sub; ++s) {
    rows[5 * s] = t->h.level[s];
    rows[5 * s + 1] = t->h.ijk[3 * s];
    rows[5 * s + 2] = t->h.ijk[3 * s + 1];
    rows[5 * s + 3] = t->h.ijk[3 * s + 2];
    rows[5 * s + 4] = t->h.leaf[s];
  }
  return FMM_OK;
}

int fmm_stencil(double theta, int parity, int32_t* offsets, int32_t capacity, int32_t* count) {
  if (!(theta >= kThetaMin && theta < 1.0)) return fail(FMM_ERR_THETA, "theta must lie in [0.34, 1)");
  if (parity < 0 || parity > 7 || !count || capacity < 0 || (capacity > 0 && !offsets))
    return fail(FMM_ERR_ARG, "bad argument");
  Stencil st = make_stencil(theta);
  const auto& v = st.offs[parity];
  *count = int32_t(v.size());
  for (int32_t q = 0; q < int32_t(v.size()) && q < capacity; ++q) {
    int dx, dy, dz;
    unpack_offset(v[q], dx, dy, dz);
    offsets[3 * q] = dx;
    offsets[3 * q + 1] = dy;
    offsets[3 * q + 2] = dz;
  }
  return FMM_OK;
}

int fmm_interaction_counts(const fmm_tree* t, double theta, int64_t counts[3]) {
  if (!t || !counts) return fail(FMM_ERR_ARG, "null argument");
  if (!(theta >= kThetaMin && theta < 1.0)) return fail(FMM_ERR_THETA, "theta must lie in [0.34, 1)");
  interaction_counts(t->h, make_stencil(theta), counts);
  return FMM_OK;
}

int fmm_interaction_counts_by_type(const fmm_tree* t, double theta, int64_t counts[6]) {
  if (!t || !counts) return fail(FMM_ERR_ARG, "null argument");
  if (!(theta >= kThetaMin && theta < 1.0)) return fail(FMM_ERR_THETA, "theta must lie in [0.34, 1)");
  interaction_counts_by_type(t->h, make_stencil(theta), counts);
  return FMM_OK;
}

int fmm_last_launches(const fmm_tree* t, int32_t* n) {
  if (!t || !n) return fail(FMM_ERR_ARG, "null argument");
  *n = t->launches;
  return FMM_OK;
}

int fmm_solve(fmm_tree* t, const double* rho_dev, double theta, int precision, int amc,
              double* phi_dev, double* g_dev, double* net_dev, void* stream) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (!rho_dev || !phi_dev || !g_dev) return fail(FMM_ERR_ARG, "null device pointer");
  try {
    return solve_impl(t, contiguous_io(t, rho_dev, phi_dev, g_dev), theta, precision, amc,
                      net_dev, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_solve_dt(fmm_tree* t, const double* rho_dev, const double* rhodot_dev, double theta,
                 int precision, int amc, double* phi_dev, double* g_dev, double* phidot_dev,
                 double* net_dev, void* stream) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (!rho_dev || !phi_dev || !g_dev || !rhodot_dev || !phidot_dev)
    return fail(FMM_ERR_ARG, "null device pointer");
  try {
    std::vector<TreeIo> io = contiguous_io(t, rho_dev, phi_dev, g_dev);
    for (int k = 0; k < t->h.n_trees; ++k) {
      const int64_t o = t->h.tree_leaf_off[k] * kCells;
      io[size_t(k)].src = rhodot_dev + o;
      io[size_t(k)].phidot = phidot_dev + o;
    }
    return solve_impl(t, io, theta, precision, amc, net_dev, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_solve_batch(fmm_tree* f, const double* const* rho_dev, double theta, int precision,
                    int amc, double* const* phi_dev, double* const* g_dev, double* net_dev,
                    void* stream) {
  if (!f || !rho_dev || !phi_dev || !g_dev) return fail(FMM_ERR_ARG, "null argument");
  try {
    std::vector<TreeIo> io(size_t(f->h.n_trees));
    for (int k = 0; k < f->h.n_trees; ++k) {
      if (!rho_dev[k] || !phi_dev[k] || !g_dev[k]) return fail(FMM_ERR_ARG, "null per-tree pointer");
      io[size_t(k)] = TreeIo{rho_dev[k], phi_dev[k], g_dev[k]};
    }
    return solve_impl(f, io, theta, precision, amc, net_dev, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_sync_status(fmm_tree* t, void* stream) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (!t->dev_ready) return FMM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaStreamSynchronize(st));
  for (cudaStream_t q : {t->hp.in, t->hp.solve, t->hp.out})
    if (q) CUDA_TRY(cudaStreamSynchronize(q));
  int status = 0;
  CUDA_TRY(cudaMemcpy(&status, t->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(t->d_status, 0, sizeof(int)));
  if (status & 1) return fail(FMM_ERR_NONFINITE, "a density was negative, NaN or infinite");
  if (status & 2) return fail(FMM_ERR_NONFINITE, "a density time derivative was NaN or infinite");
  if (status & 4) return fail(FMM_ERR_TIMEOUT, "a shared-memory staging wait timed out");
  if (status & 8) return fail(FMM_ERR_BOUNDS, "an index check of the bounds-checked build failed");
  if (status & 16) return fail(FMM_ERR_TIMEOUT, "a grid barrier of a persistent level pass timed out");
  return FMM_OK;
}

int fmm_solve_host(fmm_tree* t, const double* rho_host, double theta, int precision, int amc,
                   double* phi_host, double* g_host, double* net_host, void* stream) {
  if (!t || !rho_host || !phi_host || !g_host) return fail(FMM_ERR_ARG, "null argument");
  int rc = ensure_device(t);
  if (rc) return rc;
  const int64_t n = t->h.n_leaf_sub * kCells;
  if (!t->d_rho) {
    CUDA_TRY(dalloc(t, &t->d_rho, sizeof(double) * n));
    CUDA_TRY(dalloc(t, &t->d_phi, sizeof(double) * n));
    CUDA_TRY(dalloc(t, &t->d_g, sizeof(double) * 3 * n));
    CUDA_TRY(dalloc(t, &t->d_net, sizeof(double) * 7 * t->h.n_trees));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemcpyAsync(t->d_rho, rho_host, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  rc = fmm_solve(t, t->d_rho, theta, precision, amc, t->d_phi, t->d_g, net_host ? t->d_net : nullptr,
                 stream);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(phi_host, t->d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(g_host, t->d_g, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
  if (net_host)
    CUDA_TRY(cudaMemcpyAsync(net_host, t->d_net, sizeof(double) * 7 * t->h.n_trees,
                             cudaMemcpyDeviceToHost, st));
  return fmm_sync_status(t, stream);
}

int fmm_solve_host_async(fmm_tree* t, const double* rho_host, double theta, int precision, int amc,
                         double* phi_host, double* g_host, double* net_host, void* stream) {
  if (!t || !rho_host || !phi_host || !g_host) return fail(FMM_ERR_ARG, "null argument");
  int rc = ensure_device(t);
  if (rc) return rc;
  fmm_tree::HostPipe& P = t->hp;
  const int64_t n = t->h.n_leaf_sub * kCells;
  if (!P.in) {
    for (int k = 0; k < 2; ++k) {
      CUDA_TRY(dalloc(t, &P.rho[k], sizeof(double) * n));
      CUDA_TRY(dalloc(t, &P.phi[k], sizeof(double) * n));
      CUDA_TRY(dalloc(t, &P.g[k], sizeof(double) * 3 * n));
      CUDA_TRY(dalloc(t, &P.net[k], sizeof(double) * 7 * t->h.n_trees));
      CUDA_TRY(cudaEventCreateWithFlags(&P.copied_in[k], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&P.solved[k], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&P.copied_out[k], cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventCreateWithFlags(&P.caller, cudaEventDisableTiming));
    CUDA_TRY(cudaStreamCreateWithFlags(&P.in, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&P.solve, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&P.out, cudaStreamNonBlocking));
  }
  const int k = P.slot;
  // copy in: after the caller's work so far, and after the solve two calls back read this slot
  CUDA_TRY(cudaEventRecord(P.caller, static_cast<cudaStream_t>(stream)));
  CUDA_TRY(cudaStreamWaitEvent(P.in, P.caller, 0));
  CUDA_TRY(cudaStreamWaitEvent(P.in, P.solved[k], 0));
  CUDA_TRY(cudaMemcpyAsync(P.rho[k], rho_host, sizeof(double) * n, cudaMemcpyHostToDevice, P.in));
  CUDA_TRY(cudaEventRecord(P.copied_in[k], P.in));
  // solve: after the copy in, and after the copies out two calls back emptied this slot
  CUDA_TRY(cudaStreamWaitEvent(P.solve, P.copied_in[k], 0));
  CUDA_TRY(cudaStreamWaitEvent(P.solve, P.copied_out[k], 0));
  rc = fmm_solve(t, P.rho[k], theta, precision, amc, P.phi[k], P.g[k], net_host ? P.net[k] : nullptr,
                 P.solve);
  if (rc) return rc;
  CUDA_TRY(cudaEventRecord(P.solved[k], P.solve));
  // copy out
  CUDA_TRY(cudaStreamWaitEvent(P.out, P.solved[k], 0));
  CUDA_TRY(cudaMemcpyAsync(phi_host, P.phi[k], sizeof(double) * n, cudaMemcpyDeviceToHost, P.out));
  CUDA_TRY(cudaMemcpyAsync(g_host, P.g[k], sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, P.out));
  if (net_host)
    CUDA_TRY(cudaMemcpyAsync(net_host, P.net[k], sizeof(double) * 7 * t->h.n_trees,
                             cudaMemcpyDeviceToHost, P.out));
  CUDA_TRY(cudaEventRecord(P.copied_out[k], P.out));
  P.slot = 1 - k;
  return FMM_OK;
}

int fmm_net_force_torque(fmm_tree* t, const double* rho_dev, const double* g_dev, double* net_dev,
                         void* stream) {
  if (!t || !rho_dev || !g_dev || !net_dev) return fail(FMM_ERR_ARG, "null argument");
  int rc = ensure_device(t);
  if (rc) return rc;
  try {
    // the reduction reads rho and g through the tree's pointer table, on the tree's stream
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    // (the reduction only reads g)
    std::vector<TreeIo> io = contiguous_io(t, rho_dev, nullptr, const_cast<double*>(g_dev));
    CUDA_TRY(cudaEventRecord(t->ev_in, caller));
    CUDA_TRY(cudaStreamWaitEvent(t->stream, t->ev_in, 0));
    int32_t n_io = 0;
    if ((rc = set_io(t, io, net_dev, t->stream, &n_io))) return rc;
    if ((rc = launch_net(t, make_args(t, nullptr), t->stream))) return rc;
    CUDA_TRY(cudaEventRecord(t->ev_out, t->stream));
    CUDA_TRY(cudaStreamWaitEvent(caller, t->ev_out, 0));
    return FMM_OK;
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

// Enqueues n_pass diagnostics passes on the tree's stream, the parameters of the first written
// by a small kernel and, with `iterate`, those of each later pass updated on the device by the
// previous pass's final kernel.
static int enqueue_binary(fmm_tree* t, const double* rho_dev, const double* g_dev, const BinaryParams& P,
                          int n_pass, bool iterate, double* out_dev, double* centres_dev,
                          double* torque_dev, int8_t* member_dev, cudaStream_t caller) {
  const int nb = 2 * t->n_sms;
  if (!t->d_diag_partials) CUDA_TRY(dalloc(t, &t->d_diag_partials, sizeof(double) * nb * kDiagVals));
  if (!t->d_diag_state) CUDA_TRY(dalloc(t, &t->d_diag_state, sizeof(BinaryParams)));
  std::vector<TreeIo> io = contiguous_io(t, rho_dev, nullptr, const_cast<double*>(g_dev));
  CUDA_TRY(cudaEventRecord(t->ev_in, caller));
  CUDA_TRY(cudaStreamWaitEvent(t->stream, t->ev_in, 0));
  int32_t n_io = 0;
  int rc = set_io(t, io, nullptr, t->stream, &n_io);
  if (rc) return rc;
  k_binary_init<<<1, 1, 0, t->stream>>>(P, t->d_diag_state);
  CUDA_TRY(cudaGetLastError());
  DevArgs A = make_args(t, nullptr);
  for (int k = 0; k < n_pass; ++k) {
    k_binary_partial<<<nb, kDiagThreads, 0, t->stream>>>(A, t->d_diag_state, t->d_diag_partials, member_dev);
    CUDA_TRY(cudaGetLastError());
    k_binary_final<<<1, kDiagThreads, 0, t->stream>>>(t->d_diag_partials, nb, out_dev, t->d_diag_state,
                                                      centres_dev, torque_dev, iterate ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaEventRecord(t->ev_out, t->stream));
  CUDA_TRY(cudaStreamWaitEvent(caller, t->ev_out, 0));
  t->launches = n_io + 1 + 2 * n_pass;
  return FMM_OK;
}

int fmm_binary_diagnostics(fmm_tree* t, const double* rho_dev, const double* g_dev, double omega,
                           const double* x1, const double* x2, double rc1, double rc2,
                           double* out_dev, int8_t* member_dev, void* stream) {
  if (!t || !rho_dev || !g_dev || !x1 || !x2 || !out_dev) return fail(FMM_ERR_ARG, "null argument");
  if (t->h.n_trees != 1) return fail(FMM_ERR_ARG, "diagnostics take a single tree");
  if (!(rc1 >= 0.0) || !(rc2 >= 0.0)) return fail(FMM_ERR_ARG, "critical radii must be >= 0");
  int rc = ensure_device(t);
  if (rc) return rc;
  try {
    BinaryParams P;
    P.w2 = omega * omega;
    for (int a = 0; a < 3; ++a) {
      P.c[0][a] = x1[a];
      P.c[1][a] = x2[a];
    }
    P.rc2[0] = rc1 * rc1;
    P.rc2[1] = rc2 * rc2;
    return enqueue_binary(t, rho_dev, g_dev, P, 1, false, out_dev, nullptr, nullptr, member_dev,
                          static_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_binary_iterate(fmm_tree* t, const double* rho_dev, const double* g_dev, double omega,
                       const double* x1, const double* x2, int n_iter, double* out_dev,
                       double* centres_dev, double* torque_dev, int8_t* member_dev, void* stream) {
  if (!t || !rho_dev || !g_dev || !x1 || !x2 || !out_dev || !centres_dev || !torque_dev)
    return fail(FMM_ERR_ARG, "null argument");
  if (n_iter < 1) return fail(FMM_ERR_ARG, "n_iter must be >= 1");
  if (t->h.n_trees != 1) return fail(FMM_ERR_ARG, "diagnostics take a single tree");
  int rc = ensure_device(t);
  if (rc) return rc;
  try {
    BinaryParams P;
    P.w2 = omega * omega;
    for (int a = 0; a < 3; ++a) {
      P.c[0][a] = x1[a];
      P.c[1][a] = x2[a];
    }
    P.rc2[0] = P.rc2[1] = 0.0;  // the first pass uses no critical radius
    return enqueue_binary(t, rho_dev, g_dev, P, n_iter, true, out_dev, centres_dev, torque_dev,
                          member_dev, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_set_variant(fmm_tree* t, double theta, int variant) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  if (variant < 0 || variant >= kMixedVariants) return fail(FMM_ERR_ARG, "variant out of range");
  if (!(theta >= kThetaMin && theta < 1.0)) return fail(FMM_ERR_THETA, "theta must lie in [0.34, 1)");
  int rc = ensure_device(t);
  if (rc) return rc;
  StencilDev* sd = nullptr;
  try {
    if ((rc = get_stencil(t, theta, &sd))) return rc;
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
  sd->mixed_variant = variant;
  return FMM_OK;
}

int fmm_set_persistent(fmm_tree* t, int on) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  t->persistent = on ? 1 : 0;
  return FMM_OK;
}

int fmm_autotune(fmm_tree* t, const double* rho_dev, double theta, int precision, int amc,
                 double* phi_dev, double* g_dev, int reps, float* ms_host, int32_t* variant_out,
                 void* stream) {
  if (!t || !rho_dev || !phi_dev || !g_dev || !variant_out || reps < 1)
    return fail(FMM_ERR_ARG, "null argument or reps < 1");
  if (precision != FMM_FP64 && precision != FMM_MIXED && precision != FMM_DF64)
    return fail(FMM_ERR_ARG, "bad precision");
  try {
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    const std::vector<TreeIo> io = contiguous_io(t, rho_dev, phi_dev, g_dev);
    int rc = solve_impl(t, io, theta, precision, amc, nullptr, caller);  // builds the lists
    if (rc) return rc;
    StencilDev* sd = nullptr;
    if ((rc = get_stencil(t, theta, &sd))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // each timed solve starts with cold caches, as a solve does inside a time step: a buffer of
    // twice the L2's size is overwritten before it (outside the timed interval)
    int l2 = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, t->device));
    const size_t flush_bytes = size_t(2) * size_t(l2 > 0 ? l2 : (64 << 20));
    void* flush = nullptr;
    CUDA_TRY(cudaMalloc(&flush, flush_bytes));
    if (ms_host)
      for (int v = 0; v < (precision == FMM_MIXED ? kMixedVariants : 1); ++v) ms_host[v] = -1.0f;
    // median time of `reps` solves of variant v after a warm-up solve (which captures its graph)
    auto time_variant = [&](int v, float* med) -> int {
      if (precision == FMM_MIXED) sd->mixed_variant = v;
      int r = solve_impl(t, io, theta, precision, amc, nullptr, caller);
      std::vector<float> ms;
      for (int k = 0; k < reps && r == FMM_OK; ++k) {
        float x = 0.0f;
        if (cudaMemsetAsync(flush, k & 0xff, flush_bytes, caller) != cudaSuccess) r = fail(FMM_ERR_CUDA, "L2 flush");
        if (!r && cudaEventRecord(e0, caller) != cudaSuccess) r = fail(FMM_ERR_CUDA, "event record");
        if (!r) r = solve_impl(t, io, theta, precision, amc, nullptr, caller);
        if (!r && (cudaEventRecord(e1, caller) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                   cudaEventElapsedTime(&x, e0, e1) != cudaSuccess))
          r = fail(FMM_ERR_CUDA, "event timing");
        ms.push_back(x);
      }
      if (r) return r;
      std::sort(ms.begin(), ms.end());
      *med = ms[ms.size() / 2];
      if (ms_host) ms_host[v] = *med;
      return FMM_OK;
    };
    // coordinate search: every kernel / leaf layout / placement combination at the default split
    // threshold, then the split thresholds with the best of those.  A variant displaces the one
    // kept so far only when it is at least 1 % faster, so that timing noise does not move the
    // choice away from the default
    int best = 0;
    float best_ms = 0.0f;
    const int n_first = precision == FMM_MIXED ? 24 : 1;
    for (int v = 0; v < n_first && rc == FMM_OK; ++v) {
      float m = 0.0f;
      rc = time_variant(v, &m);
      if (!rc && (v == 0 || m < 0.99f * best_ms)) {
        best = v;
        best_ms = m;
      }
    }
    if (precision == FMM_MIXED) {
      const int base = best;
      for (int c = 1; c < kSplitChoices && rc == FMM_OK; ++c) {
        float m = 0.0f;
        rc = time_variant(base + 24 * c, &m);
        if (!rc && m < 0.99f * best_ms) {
          best = base + 24 * c;
          best_ms = m;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(flush);
    if (rc) return rc;
    if (precision == FMM_MIXED) sd->mixed_variant = best;
    *variant_out = best;
    // leave the outputs of the chosen variant in phi and g
    return solve_impl(t, io, theta, precision, amc, nullptr, caller);
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_set_wait_limit(fmm_tree* t, long long cycles) {
  if (!t || cycles < 0) return fail(FMM_ERR_ARG, "tree is null or limit negative");
  t->wait_cycles = cycles;
  return FMM_OK;
}

int fmm_set_graphs(fmm_tree* t, int on) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  t->use_graphs = on != 0;
  return FMM_OK;
}

int fmm_set_profiling(fmm_tree* t, int on) {
  if (!t) return fail(FMM_ERR_ARG, "tree is null");
  t->profiling = on != 0;
  t->ev_recorded = false;
  return FMM_OK;
}

int fmm_phase_times(fmm_tree* t, float* ms, int n) {
  if (!t || !ms || n < 0) return fail(FMM_ERR_ARG, "null argument");
  if (!t->ev_recorded) return fail(FMM_ERR_STATE, "no profiled solve recorded");
  CUDA_TRY(cudaEventSynchronize(t->ev[4]));
  for (int k = 0; k < n && k < 4; ++k) CUDA_TRY(cudaEventElapsedTime(&ms[k], t->ev[k], t->ev[k + 1]));
  // [4] from the end of the leaf kernel (second stream) to the end of the interactions, [5] the
  // leaf kernel, which starts beside the upward pass
  if (n > 4) CUDA_TRY(cudaEventElapsedTime(&ms[4], t->ev[9], t->ev[2]));
  if (n > 5) CUDA_TRY(cudaEventElapsedTime(&ms[5], t->ev[8], t->ev[9]));
  // [6] the staged refined-target kernel of a mixed solve (0 for the other precisions)
  if (n > 6) {
    ms[6] = 0.0f;
    if (t->ev_stage) CUDA_TRY(cudaEventElapsedTime(&ms[6], t->ev[6], t->ev[7]));
  }
  return FMM_OK;
}

int fmm_net_force_torque_points_static(int64_t n, const double* x_dev, const double* m_dev,
                                       const double* g_dev, double* net_dev, void* stream) {
  if (!x_dev || !m_dev || !g_dev || !net_dev || n < 0) return fail(FMM_ERR_ARG, "bad argument");
  if (n > int64_t(kStaticNetMaxBlocks) * kStaticNetPointsPerBlock)
    return fail(FMM_ERR_ARG, "n exceeds FMM_NET_STATIC_MAX_POINTS (" +
                                 std::to_string(int64_t(kStaticNetMaxBlocks) * kStaticNetPointsPerBlock) +
                                 "), the capacity of the fixed scratch array");
  double* scratch = nullptr;
  int rc = static_net_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int blocks = int((n + kStaticNetPointsPerBlock - 1) / kStaticNetPointsPerBlock);
  if (blocks > 0) {
    k_net_points_partial<<<blocks, kReduceThreads, 0, st>>>(n, x_dev, m_dev, g_dev, scratch);
    CUDA_TRY(cudaGetLastError());
  }
  k_net_final<<<1, kReduceThreads, 0, st>>>(scratch, blocks, net_dev, nullptr);
  CUDA_TRY(cudaGetLastError());
  return FMM_OK;
}

int fmm_partition(const fmm_tree* t, int n_ranks, int cut_level, int32_t* owner_host) {
  if (!t || !owner_host) return fail(FMM_ERR_ARG, "null argument");
  try {
    std::vector<int32_t> owner;
    std::string err = partition_tree(t->h, n_ranks, cut_level, owner);
    if (!err.empty()) return fail(FMM_ERR_ARG, err);
    std::copy(owner.begin(), owner.end(), owner_host);
    return FMM_OK;
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_ghosts(const fmm_tree* t, const int32_t* owner_host, int rank, int32_t* ghosts_host,
               int64_t capacity, int64_t* count) {
  if (!t || !owner_host || !count || capacity < 0 || (capacity > 0 && !ghosts_host))
    return fail(FMM_ERR_ARG, "null argument or negative capacity");
  try {
    std::vector<int32_t> owner(owner_host, owner_host + t->h.n_sub), out;
    std::string err = ghost_subgrids(t->h, owner, rank, out);
    if (!err.empty()) return fail(FMM_ERR_ARG, err);
    *count = int64_t(out.size());
    for (int64_t k = 0; k < int64_t(out.size()) && k < capacity; ++k) ghosts_host[k] = out[size_t(k)];
    return FMM_OK;
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
}

int fmm_scf_init(fmm_tree* t, const fmm_scf_params* p, const double* rho_dev, double K0,
                 double* phi_dev, double* g_dev, void* stream) {
  ScfProblem P;
  int rc = scf_check(t, p, &P);
  if (rc) return rc;
  if (!rho_dev || !phi_dev || !g_dev || !(K0 > 0.0)) return fail(FMM_ERR_ARG, "null pointer or K0 <= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  try {
    // the solve before the iterations
    rc = solve_impl(t, contiguous_io(t, rho_dev, phi_dev, g_dev), p->theta, p->precision, 1, nullptr, st);
    if (rc) return rc;
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
  CUDA_TRY(scf_launch_init(scf_geom(t), P, rho_dev, phi_dev, K0, t->d_scf_state, t->d_scf_part,
                           t->d_scf_apart, st));
  t->scf_started = true;
  return FMM_OK;
}

int fmm_scf_iterate(fmm_tree* t, const fmm_scf_params* p, int n_iter, double* rho_dev,
                    double* phi_dev, double* g_dev, double* state_dev, double* history_dev,
                    void* stream) {
  ScfProblem P;
  int rc = scf_check(t, p, &P);
  if (rc) return rc;
  if (!rho_dev || !phi_dev || !g_dev || n_iter < 0) return fail(FMM_ERR_ARG, "null pointer or n_iter < 0");
  if (!t->scf_started) return fail(FMM_ERR_STATE, "fmm_scf_init has not been called on this tree");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ScfGeom G = scf_geom(t);
  try {
    for (int k = 0; k < n_iter; ++k) {
      CUDA_TRY(scf_launch_scale(G, P, rho_dev, t->d_scf_state, t->d_scf_part, st));
      rc = solve_impl(t, contiguous_io(t, rho_dev, phi_dev, g_dev), p->theta, p->precision, 1, nullptr, st);
      if (rc) return rc;
      CUDA_TRY(scf_launch_update(G, P, rho_dev, phi_dev, t->d_scf_state, t->d_scf_apart,
                                 history_dev ? history_dev + int64_t(k) * kScfState : nullptr, st));
    }
  } catch (...) {
    return fail(FMM_ERR_NOMEM, "host allocation failed");
  }
  if (state_dev)
    CUDA_TRY(cudaMemcpyAsync(state_dev, t->d_scf_state, sizeof(double) * kScfState,
                             cudaMemcpyDeviceToDevice, st));
  return FMM_OK;
}

const char* fmm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
