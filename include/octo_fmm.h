/*
 * octo_fmm.h -- C ABI of the GB300 (sm_103a) octree FMM gravity solver.
 *
 * The solver computes the gravitational potential phi and acceleration g = -grad phi (G = 1) of a
 * density field given on the leaf cells of an octree of 8x8x8-cell subgrids, with the Cartesian
 * fast multipole method and the angular-momentum correction described in Marcello et al. 2021
 * (arXiv 2101.08226), Sec. 2.2; the mesh and its proper nesting follow Sec. 2.4.
 *
 * Geometry.  The domain is the unit box [-1/2, 1/2]^3.  A level-l subgrid at integer position
 * (i, j, k) in [0, 2^l)^3 covers [-1/2 + i/2^l, -1/2 + (i+1)/2^l] x ...; its 512 cells have width
 * dx_l = 1 / (8 * 2^l) and are numbered (a*8 + b)*8 + c within the subgrid (c, the z index,
 * fastest).  Every leaf cell is a point mass m = rho * dx^3 at its centre.
 *
 * Canonical leaf order.  Leaf subgrids are ordered by level, then by the Morton key of (i, j, k)
 * (bits interleaved x, y, z from most to least significant within each triple); a leaf cell's
 * index is (leaf-subgrid ordinal) * 512 + (a*8 + b)*8 + c.  Every per-cell array below (rho, phi,
 * g) uses this order.
 *
 * Ownership.  The caller owns every density / potential / acceleration buffer and the CUDA stream;
 * the library owns the tree, its device-resident tables and its workspace (allocated on the
 * first solve, freed by fmm_destroy).  Pointers named *_dev are device pointers on the current
 * CUDA device; pointers named *_host are host pointers (pinned memory gives faster copies).
 *
 * Errors.  Every int-returning entry point returns FMM_OK (0) or a negative FMM_ERR_* code and
 * never aborts or throws; fmm_last_error() gives a message for the calling thread.  Solves are
 * enqueued asynchronously on `stream`; problems found on the device (a non-finite or negative
 * density, a timed-out wait) are recorded in the tree's status word and reported by
 * fmm_sync_status().
 *
 * Threads.  A tree may be used by one host thread at a time.  Different trees are independent.
 */
#ifndef OCTO_FMM_H
#define OCTO_FMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMM_OK 0
#define FMM_ERR_ARG (-1)       /* invalid argument (null pointer, size mismatch, bad level) */
#define FMM_ERR_THETA (-3)     /* opening criterion outside [0.34, 1) */
#define FMM_ERR_CUDA (-4)      /* a CUDA runtime call failed */
#define FMM_ERR_NONFINITE (-6) /* a density was negative, NaN or infinite (found on the device) */
#define FMM_ERR_NOMEM (-7)     /* host or device allocation failed */
#define FMM_ERR_STATE (-8)     /* tree not usable (destroyed or built on another device) */
#define FMM_ERR_TIMEOUT (-9)   /* a kernel's bounded wait for its shared-memory copies gave up
                                  (found on the device; that block's results are missing) */
#define FMM_ERR_BOUNDS (-10)   /* an index read from the library's tables failed its range check;
                                  only the bounds-checked build of the library
                                  (libocto_fmm_bc.so, compiled with -DFMM_BOUNDS_CHECK) checks,
                                  skipping the access instead of making it */

#define FMM_FP64 0  /* every step in FP64 */
#define FMM_MIXED 1 /* multipole interactions and direct sums in FP32, expansions in FP32;
                       moments, correction sums and reductions in FP64 */
#define FMM_DF64 2  /* FP64 except the pair arithmetic of the interactions and direct sums, which
                       runs in double-float (pairs of floats, about 48 bits, on the FP32 pipes):
                       results within the FP64 path's 1e-12 parity bar, at FP32-pipe speed.  The
                       float exponent range applies inside the pair arithmetic (|values| between
                       about 1e-38 and 3e38).  Not for fmm_solve_dt. */

#define FMM_MAX_LEVEL 9 /* deepest refinement level accepted (levels 0..9) */

typedef struct fmm_tree fmm_tree;

/* Build the octree (Sec. 2.4, refinement as in Sec. 2.7).
 * refine_flags: host array of dense per-level flags for levels 0 .. max_level-1; level l occupies
 *   8^l bytes starting at sum_{k<l} 8^k, indexed (i * 2^l + j) * 2^l + k.  A subgrid that exists
 *   and is flagged is refined; flags of positions that do not exist are ignored.  Further
 *   subgrids are refined until proper nesting holds: every refined subgrid has all 26
 *   same-level neighbours inside the domain, so leaf levels differ by at most one across any
 *   subgrid boundary.
 * n_flags must equal sum_{l<max_level} 8^l; 0 <= max_level <= FMM_MAX_LEVEL.
 * On success *out receives a new tree (destroy with fmm_destroy).  Host-only: needs no GPU. */
int fmm_build_tree(int max_level, const uint8_t* refine_flags, int64_t n_flags, fmm_tree** out);

/* Release a tree (or forest) and its device workspace.  NULL is ignored. */
void fmm_destroy(fmm_tree* tree);

/* A forest: the disjoint union of n independent trees (or forests), solved by one set of
 * launches -- every level of every tree at once, however uneven their depths.  The parts are
 * copied; they stay valid and independent.  In every per-cell array of a forest the trees' leaf
 * cells follow each other in part order, each tree's in its own canonical order; net sums are
 * per tree (7 doubles each, tree order).  Host-only: needs no GPU. */
int fmm_build_forest(const fmm_tree* const* trees, int n, fmm_tree** out);

/* Number of trees (1 for a tree built by fmm_build_tree) and, if leaf_subgrid_offsets is not
 * NULL, n_trees + 1 offsets: tree k's leaf cells are [512 offsets[k], 512 offsets[k+1]). */
int fmm_forest_info(const fmm_tree* tree, int32_t* n_trees, int64_t* leaf_subgrid_offsets);

/* Sizes: total subgrids, leaf subgrids (leaf cells = 512 * n_leaf_subgrids), deepest level.
 * Any output pointer may be NULL. */
int fmm_tree_info(const fmm_tree* tree, int64_t* n_subgrids, int64_t* n_leaf_subgrids,
                  int32_t* depth);

/* Rows (level, i, j, k, is_leaf) of every subgrid, by level then Morton key: host array of
 * 5 * n_subgrids int32. */
int fmm_tree_subgrids(const fmm_tree* tree, int32_t* rows_host);

/* Same-level interaction stencil (Sec. 2.2 opening criterion): the offsets d (in cells) for which
 * cells A and A + d are well separated, dx/|x_A - x_B| < theta, while their parents are not.
 * parity = (a & 1) << 2 | (b & 1) << 1 | (c & 1) of the target cell.  Writes up to `capacity`
 * rows (dx, dy, dz) in lexicographic order into offsets_host and the full count into *count. */
int fmm_stencil(double theta, int parity, int32_t* offsets_host, int32_t capacity,
                int32_t* count);

/* Directed interaction counts of one solve at this theta (host-only):
 *   counts[0] multipole (cell-cell) interactions over all levels,
 *   counts[1] direct leaf-leaf pairs at the same level,
 *   counts[2] direct leaf-leaf pairs across one level jump. */
int fmm_interaction_counts(const fmm_tree* tree, double theta, int64_t counts_host[3]);

/* The same counts split by the kind of arithmetic they need (host-only), 6 entries:
 *   [0] multipole interactions leaf cell <- leaf cell     [1] leaf cell <- refined cell
 *   [2] refined cell <- leaf cell                          [3] refined cell <- refined cell
 *   [4] same-level direct pairs                            [5] direct pairs across a level jump
 * A refined cell has children (it carries 2nd and 3rd moments and needs the 2nd and 3rd
 * derivatives of its expansion); a leaf cell is a point mass. */
int fmm_interaction_counts_by_type(const fmm_tree* tree, double theta, int64_t counts_host[6]);

/* One gravity solve (Sec. 2.2): multipoles up the tree, same-level multipole interactions with
 * the angular-momentum correction (amc != 0), direct near-field sums, expansions down the tree.
 * rho_dev: [n_leaf] leaf-cell densities (>= 0, finite).  phi_dev: [n_leaf] potential.
 * g_dev: [n_leaf][3] acceleration.  net_dev (optional, may be NULL): 7 doubles
 *   (F_x, F_y, F_z, T_x, T_y, T_z, S) with F = sum m g, T = sum x cross m g, S = sum |x| |m g|,
 *   reduced in FP64 in a fixed order (the terms of the normalisation S are formed in FP32).
 * theta in [0.34, 1).  precision FMM_FP64, FMM_MIXED or FMM_DF64.  stream: a cudaStream_t (NULL = legacy
 * default stream).  Asynchronous: returns once the work is enqueued.  On a forest, net_dev holds
 * 7 doubles per tree.
 * Execution: the work runs on a stream the tree owns, after all work enqueued on `stream` before
 * the call and before all work enqueued on `stream` after it, so that the calls of one tree never
 * overlap whatever streams they name.  By default the launches of each configuration (theta,
 * precision, amc, net_dev NULL or not, profiling) are captured once into a CUDA graph, which
 * every later call of that configuration replays after one small kernel that writes this call's
 * pointers into a device table (fmm_set_graphs turns this off).  The first call of a
 * configuration therefore costs extra host time. */
int fmm_solve(fmm_tree* tree, const double* rho_dev, double theta, int precision, int amc,
              double* phi_dev, double* g_dev, double* net_dev, void* stream);

/* fmm_solve plus the time derivative of the potential (Sec. 2.1: the FMM with the computed
 * d(rho)/dt as the source, so that the two parts of the energy equation's gravity term cancel
 * over the grid).  rhodot_dev: [n_leaf] d(rho)/dt (any sign, finite).  phidot_dev: [n_leaf]
 * d(phi)/dt out: the same operator as the rho solve -- same lists, the same expansion centres
 * (rho's centres of mass), the same truncation -- applied to s = rhodot dx^3, whose moments about
 * those centres include a dipole.  With these centres the operator is symmetric:
 * sum_i s_i phi_i = sum_i m_i phidot_i to rounding.  Other arguments, ordering and errors as
 * fmm_solve (FMM_ERR_NONFINITE also for a NaN or infinite rhodot); one graph per configuration. */
int fmm_solve_dt(fmm_tree* tree, const double* rho_dev, const double* rhodot_dev, double theta,
                 int precision, int amc, double* phi_dev, double* g_dev, double* phidot_dev,
                 double* net_dev, void* stream);

/* fmm_solve on a forest with one device buffer per tree: rho_dev[k], phi_dev[k], g_dev[k] are
 * tree k's arrays (its own canonical order), read and written in place by the kernels (the
 * pointer arrays themselves are host arrays, read before the call returns); net_dev (optional)
 * gets 7 doubles per tree.  Asynchronous, ordered on `stream` as fmm_solve. */
int fmm_solve_batch(fmm_tree* forest, const double* const* rho_dev, double theta, int precision,
                    int amc, double* const* phi_dev, double* const* g_dev, double* net_dev,
                    void* stream);

/* Waits for `stream` (and for the tree's pipelined host solves), then returns FMM_OK, or
 * FMM_ERR_NONFINITE if a solve since the last call
 * met an invalid density, FMM_ERR_TIMEOUT if one of its bounded waits gave up, or FMM_ERR_CUDA;
 * clears the recorded status. */
int fmm_sync_status(fmm_tree* tree, void* stream);

/* End-to-end solve with host buffers: copies rho_host to the device, solves, copies phi, g and
 * (if net_host is not NULL) the 7 net sums back, and waits for completion.  The device buffers
 * are owned by the tree.  Returns the solve's status. */
int fmm_solve_host(fmm_tree* tree, const double* rho_host, double theta, int precision, int amc,
                   double* phi_host, double* g_host, double* net_host, void* stream);

/* Pipelined form of fmm_solve_host for a sequence of solves: enqueues, without waiting, the copy
 * of rho_host into one of two device slots owned by the tree, the solve, and the copies of phi, g
 * and (if net_host is not NULL) the 7 net sums into the host buffers, each on a stream of its own,
 * so that one call's copies overlap the neighbouring calls' solves.  The copy in is ordered after
 * the work enqueued on `stream` before the call; `stream` is not made to wait for anything.  The
 * host buffers must stay valid, and rho_host unchanged, until the work is done: call
 * fmm_sync_status (which waits for every pipelined call) before reading the outputs or reusing the
 * buffers.  Pinned host memory is needed for the copies to overlap.  Errors of the solve itself
 * are reported by fmm_sync_status. */
int fmm_solve_host_async(fmm_tree* tree, const double* rho_host, double theta, int precision,
                         int amc, double* phi_host, double* g_host, double* net_host, void* stream);

/* Net force, torque and normalisation (as net_dev above) of an arbitrary acceleration field g_dev
 * for the masses given by rho_dev on this tree's leaf cells.  Uses the tree's workspace. */
int fmm_net_force_torque(fmm_tree* tree, const double* rho_dev, const double* g_dev,
                         double* net_dev, void* stream);

/* Binary diagnostics (Sec. 4, the merger analysis), one pass over the leaf cells of a single
 * tree (a forest is rejected).  In the frame rotating about the z axis at omega, with
 * g_eff = g + omega^2 (x, y, 0) and q_s = g_eff . (x - x_s) / |x - x_s| (0 at x_s), a cell
 * belongs to star 1 (the accretor) if min(q_1, 0) < min(q_2, 0), to star 2 (the donor) if
 * min(q_1, 0) > min(q_2, 0), else to neither; a cell closer to x_s than rc_s (the paper uses a
 * quarter of the star's Roche-lobe radius) belongs to star s regardless (star 1 wins).  The
 * decision uses single correctly rounded FP64 operations in a fixed order.
 * rho_dev [n_leaf], g_dev [n_leaf][3] (e.g. fmm_solve's output); x1, x2: host double[3];
 * out_dev: 22 doubles, per star (1 then 2): M, sum m x (3), F = sum m g (3),
 * T = sum (x - x_s) x m g (3), cell count; m = rho dx^3, sums in FP64 in a fixed order.
 * member_dev (optional): int8 [n_leaf], 0 / 1 / 2.  Asynchronous, ordered on `stream`. */
int fmm_binary_diagnostics(fmm_tree* tree, const double* rho_dev, const double* g_dev,
                           double omega, const double* x1, const double* x2, double rc1,
                           double rc2, double* out_dev, int8_t* member_dev, void* stream);

/* The diagnostics' fixed-point iteration (Sec. 4: the stars' centres are found by repeating the
 * classification), n_iter >= 1 passes of fmm_binary_diagnostics enqueued back to back, each pass's
 * parameters computed on the device from the previous pass's sums: every star's centre moves to
 * its centre of mass (sum m x / M; a star that received no mass keeps its centre), and the
 * critical radii become a quarter of Eggleton's (1983) volume-equivalent Roche-lobe radius of
 * each star, 0.49 q^(2/3) / (0.6 q^(2/3) + ln(1 + q^(1/3))) a with q = M_star / M_other and a the
 * distance of the new centres (once both stars have mass; the first pass uses none).
 * x1, x2: host double[3], the starting centres.  After the last pass: out_dev (22 doubles, as
 * fmm_binary_diagnostics) holds its sums, centres_dev (6 doubles, device) the centres it used
 * (x_1 then x_2), torque_dev (3 doubles, device) the orbital torque x_1 x F_1 + x_2 x F_2 about
 * the origin with those centres, member_dev (optional, int8 [n_leaf]) its membership.  Omega,
 * rho_dev, g_dev as for fmm_binary_diagnostics.  Asynchronous, ordered on `stream`; a forest is
 * rejected (FMM_ERR_ARG), as are null pointers and n_iter < 1. */
int fmm_binary_iterate(fmm_tree* tree, const double* rho_dev, const double* g_dev, double omega,
                       const double* x1, const double* x2, int n_iter, double* out_dev,
                       double* centres_dev, double* torque_dev, int8_t* member_dev, void* stream);

/* Launch variants of the mixed path (FMM_MIXED), per tree and theta: variant = r + 4 l + 12 p + 24 c
 * with
 *   r = 0: refined targets by the shared-memory staging kernel on a second stream, beside the
 *          leaf and boundary kernels (the default);
 *   r = 1: the same kernel after them, on one stream;
 *   r = 2: refined targets by per-parity blocks that read their partners from L2;
 *   r = 3: as r = 0 with the staging pipelined: a separate warp issues the copies and each buffer
 *          has its own full and empty barriers, so the evaluating warps never meet;
 *   l = 0: leaf pairs by the four-targets-per-lane FP32 kernel, two leaf subgrids per block (the
 *          default); l = 1: by the two-targets-per-thread kernel, one subgrid per block;
 *          l = 2: by the four-targets-per-lane kernel with four subgrids per block;
 *   p = 0: the leaf-pair kernel starts beside the upward pass (the default); p = 1: after it,
 *          beside the refined targets' kernel;
 *   c = 0..3: boundary targets whose estimated list cost exceeds 6000, 1500, 24000 or (c = 3)
 *          nothing split their lists over four lanes (the default c = 0).
 * Variants with the same c that differ only in r among 0, 1, 3, in l or in p give the same results
 * bit for bit; r = 2 and other c sum some pairs in another order (results differ at FP32
 * rounding, within the mixed path's tolerance).  FMM_ERR_ARG for a variant outside
 * [0, FMM_MIXED_VARIANTS), FMM_ERR_THETA for a theta outside [0.34, 1).  The FP64 and df64 paths
 * have one launch configuration. */
#define FMM_MIXED_VARIANTS 96
int fmm_set_variant(fmm_tree* tree, double theta, int variant);

/* Autotuner: times launch variants of `precision` on the caller's density, `reps` timed solves
 * each after one warm-up solve (CUDA events on `stream`, the median kept; before every timed
 * solve a scratch buffer of twice the L2's size is overwritten, so that each starts with cold
 * caches as a solve inside a time step does), and keeps the fastest for this tree and theta (part
 * of the graph key); a variant displaces the one kept so far only when it is at least 1 % faster.
 * FMM_MIXED: a coordinate search -- the 24 variants with c = 0 (variant 0 first), then the other
 * three split thresholds c with the best of them; FP64 and df64: their one configuration.  The
 * scratch buffer is allocated and freed by the call.  Writes the chosen variant to *variant_out and, when ms_host is
 * not null, each timed variant's median (ms) to ms_host[variant] (FMM_MIXED_VARIANTS floats; -1
 * for variants not timed), and leaves the chosen variant's phi and g in the output buffers.
 * Blocks the calling thread until done.  rho_dev, phi_dev, g_dev as for fmm_solve.  FMM_ERR_ARG
 * for a null pointer or reps < 1. */
int fmm_autotune(fmm_tree* tree, const double* rho_dev, double theta, int precision, int amc,
                 double* phi_dev, double* g_dev, int reps, float* ms_host, int32_t* variant_out,
                 void* stream);

/* Mixed-precision refined targets stage their partners' moments in shared memory with bulk
 * asynchronous copies; each wait for a parity class's copies gives up after `cycles` SM clock
 * cycles (0, the default: 2^31, about a second), records FMM_ERR_TIMEOUT in the status word and
 * leaves that subgrid's expansions unset.  The same limit bounds each grid-barrier wait of the
 * persistent level passes (fmm_set_persistent).  A small limit exercises this path; the solve's
 * results are then invalid.  FMM_ERR_ARG for a negative limit. */
int fmm_set_wait_limit(fmm_tree* tree, long long cycles);

/* on != 0 (the default): replay one captured CUDA graph per solve configuration; on == 0:
 * enqueue the kernels one by one on every call.  The results are the same bit for bit. */
int fmm_set_graphs(fmm_tree* tree, int on);

/* Level passes of the rho solve (Sec. 2.2's upward M2M after P2M -- the octants with leaf
 * children, then those with refined children level by level -- and the downward pass below the
 * root -- the refined subgrids level by level, then every leaf octant): on == 0 (the default),
 * one launch per phase; on != 0, one persistent, level-ordered cooperative launch per direction,
 * whose resident blocks take each phase's work items in turn and meet at a grid-wide barrier
 * between phases (part of the graph key).  Each barrier wait is bounded by the fmm_set_wait_limit
 * limit; a wait that runs out records FMM_ERR_TIMEOUT (fmm_sync_status) and the launch leaves
 * its remaining phases undone.  The results are the same bit for bit.  The time-derivative
 * solve's source pass keeps its per-phase launches.  FMM_ERR_ARG for a null tree. */
int fmm_set_persistent(fmm_tree* tree, int on);

/* Per-phase device times (ms) of the most recent solve on this tree, measured with CUDA events
 * when profiling is on: [0] upward pass, [1] interactions after the upward pass, [2] downward
 * pass, [3] reductions, [4] from the end of the leaf-cell interaction kernel to the end of the
 * interactions (FP64 and df64: the kernel of refined cells, the root level and boundary leaves;
 * mixed: the root and boundary kernel, and the wait for the refined cells' kernel), [5] the
 * leaf-cell interaction kernel, which runs on a second stream from the end of the first upward
 * step (so it overlaps [0]), [6] mixed only (else 0): the refined cells' kernel.  Writes
 * min(n, 7) values.  fmm_set_profiling(tree, 1) turns it on. */
int fmm_set_profiling(fmm_tree* tree, int on);
int fmm_phase_times(fmm_tree* tree, float* ms_host, int n);

/* Number of kernels the most recent solve on this tree launched (all of them this library's). */
int fmm_last_launches(const fmm_tree* tree, int32_t* n);

/* Net force, torque and normalisation of an explicit point set, allocating no device memory.
 * The paper has no counterpart: this serves callers that cannot call cudaMalloc, such as code
 * inside a framework that owns all device memory through its own pool, or a latency-critical
 * loop where an allocation (and the device synchronisation it can imply) is not acceptable.
 * x_dev: [n][3] positions, m_dev: [n] masses, g_dev: [n][3] accelerations (device pointers);
 * net_dev: 7 doubles (F_x, F_y, F_z, T_x, T_y, T_z, S) as for fmm_solve, with F = sum m g,
 * T = sum x cross m g, S = sum |x| |m g| (FP64 sums; the terms of S formed in FP32).  Partial sums live in a fixed 112 KiB device array of
 * this library, so n may not exceed FMM_NET_STATIC_MAX_POINTS (FMM_ERR_ARG otherwise); n = 0
 * gives seven zeros.  The first call on a device looks up that array's address and caches it for
 * the life of the process; make that first call before any stream capture.  The cached address
 * belongs to the device's primary context (the one the CUDA runtime uses): it is not valid in
 * another context made current on the same device, nor after cudaDeviceReset.  All calls share the array: calls that overlap on the GPU race and must be serialised
 * by the caller (one stream, or events).  Asynchronous on `stream`. */
#define FMM_NET_STATIC_MAX_POINTS (2048LL * 4096LL)
int fmm_net_force_torque_points_static(int64_t n, const double* x_dev, const double* m_dev,
                                       const double* g_dev, double* net_dev, void* stream);

/* Spatial decomposition of one tree over n_ranks GPUs (Sec. 5: the large runs split one tree
 * over many nodes), host-only.  The subgrids of level cut_level (each with its whole subtree) and
 * the leaf subgrids coarser than it are ordered by the Morton key of their first corner at the cut
 * level and split into n_ranks contiguous runs of about equal leaf-cell count; owner_host
 * [n_subgrids] receives each subgrid's rank, or -1 for a refined subgrid coarser than the cut,
 * which every rank keeps: its moments are the sum over the ranks of the moments of each rank's
 * own leaves (an all-reduce), and every rank evaluates its interactions.  FMM_ERR_ARG for a forest,
 * n_ranks < 1 or a cut level outside [0, depth]. */
int fmm_partition(const fmm_tree* tree, int n_ranks, int cut_level, int32_t* owner_host);

/* The ghost subgrids of `rank` under an owner array from fmm_partition: the subgrids owned by
 * other ranks whose data this rank's solve reads -- for each subgrid it owns or keeps, the 26
 * same-level neighbours (every multipole partner lies among them for theta >= 0.34); for each leaf
 * it owns, also the leaf children of its refined neighbours and the leaf neighbours of each of its
 * ancestors (direct partners one level finer and coarser).  A leaf ghost is sent as its 512
 * densities, a refined ghost as its cells' moments.  Writes up to `capacity` subgrid indices,
 * ascending, into ghosts_host and their number into *count.  Host-only. */
int fmm_ghosts(const fmm_tree* tree, const int32_t* owner_host, int rank, int32_t* ghosts_host,
               int64_t capacity, int64_t* count);

/* Self-consistent-field (SCF) construction of a synchronously rotating binary of two polytropes
 * (Sec. 4.1, "The Initial Stellar Model"), every step on the device around this library's gravity
 * solve.  The stars lie on the x axis, the accretor (star 1) at smaller x than the donor (star 2);
 * a star is the material denser than rho_floor on its side of the plane x = x_L1 through the inner
 * Lagrange point.  An iteration: (1) each star's density scaled to its prescribed mass; the solve
 * of the scaled density; (2) the rotation axis through the centre of mass (x_cm, y_cm), parallel
 * to z; (3) Omega = J0 (M1 + M2) / (M1 M2 a^2), a the distance of the stars' centres of mass;
 * (4) with phi_eff = phi - Omega^2 ((x - x_cm)^2 + (y - y_cm)^2) / 2: L1 = the leaf cell touching
 * the x axis between the centres with the largest phi_eff, C2 = (1 - f) phi_C + f phi_L1 (phi_C at
 * the donor's densest cell); (5) K = (C2 - phi_C) / ((n + 1) rho_2^(1/n)) (rho_2 the donor's
 * largest density), C1 = K (1 + n) rho_1^(1/n) + phi_1 (the accretor's largest density and
 * phi_eff there); (6) rho = ((C - phi_eff) / (K (n + 1)))^n inside each star's ball about its
 * centre of mass up to the plane of L1 where positive, rho_floor elsewhere.  Ties (densest cell,
 * L1) go to the first cell in canonical leaf order.  Where the printed equations are garbled this
 * follows a reading: Omega squared in phi_eff, K from C2 - phi_C (the printed product does not
 * balance dimensionally), C - phi_eff in step (6), the axis through the centre of mass instead of
 * advecting the grid, and the solve placed after the mass scaling (the printed order diverges).
 * The gravity solves take theta and precision (FMM_FP64, FMM_MIXED or FMM_DF64) with the
 * correction on.  A single tree only (FMM_ERR_ARG for a forest); the tree stays fixed. */
typedef struct {
  double M1, M2;    /* prescribed masses of the accretor and the donor (> 0) */
  double n;         /* polytropic index (> 0) */
  double f;         /* the donor's Roche filling factor, (phi_edge - phi_C) / (phi_L1 - phi_C), in (0, 1] */
  double J0;        /* orbital angular momentum, held fixed (> 0) */
  double rho_floor; /* atmosphere density (>= 0) */
  double theta;     /* opening criterion of the solves */
  int precision;    /* FMM_FP64, FMM_MIXED or FMM_DF64 */
} fmm_scf_params;

/* The state of the iteration, FMM_SCF_STATE doubles: K, Omega, C1, C2, x_L1, phi_L1 (phi_eff at
 * L1), the accretor's and the donor's centres of mass (3 + 3), the system's centre of mass (3), the
 * separation a, the stars' masses before the last scaling (2), their largest densities after it
 * (rho_1, rho_2), phi_eff at the densest cells (phi_1, phi_C).  K is NaN once a star lost all its
 * material or no axis cell lay between the centres (the iteration then leaves rho alone). */
#define FMM_SCF_STATE 22

/* The solve before the iterations and the initial state: the centres of mass of the material at
 * x < 0 and x >= 0, Omega of the Kepler orbit at their separation, L1 from the solved potential,
 * K = K0 (> 0).  rho_dev [n_leaf]: the initial density (two stars); phi_dev, g_dev: the solve's
 * outputs.  Asynchronous on `stream`.  Must precede fmm_scf_iterate on this tree. */
int fmm_scf_init(fmm_tree* tree, const fmm_scf_params* params, const double* rho_dev, double K0,
                 double* phi_dev, double* g_dev, void* stream);

/* n_iter >= 0 iterations from the state fmm_scf_init or the previous call left: rho_dev [n_leaf]
 * holds the current density on entry and the new density (step (6)) on return; phi_dev, g_dev
 * hold the last solve's potential and acceleration (of the last scaled density).  state_dev
 * (optional, FMM_SCF_STATE doubles, device) receives the final state, history_dev (optional,
 * n_iter x FMM_SCF_STATE doubles, device) the state after every iteration.  Asynchronous on
 * `stream`: no host synchronisation inside; FMM_ERR_STATE without a prior fmm_scf_init. */
int fmm_scf_iterate(fmm_tree* tree, const fmm_scf_params* params, int n_iter, double* rho_dev,
                    double* phi_dev, double* g_dev, double* state_dev, double* history_dev,
                    void* stream);

/* `bits` of fmm_measure_fma_rate for FP32 fused multiply-adds in packed pairs (fma.rn.f32x2, one
 * instruction per two FMAs, sm_100 and later). */
#define FMM_FMA_F32X2 (-32)

/* Measured rate of the FP64 (bits = 64) or FP32 (bits = 32; FMM_FMA_F32X2: packed pairs) fused
 * multiply-add pipes of the current device, the denominator of the roofline of the interaction kernels (they are bound by
 * arithmetic, Sec. 2.2's multipole interactions evaluated pair by pair).  Every thread of a fully
 * occupied grid (8 blocks of 256 threads per SM) runs 8 independent FMA chains; the trip count is
 * calibrated to about 40 ms per launch, and the fastest of `reps` launches, timed with CUDA events
 * on `stream`, gives *tflops = 2 x FMAs / s / 1e12 (and *ms_per_launch, optional).  Allocates and
 * frees a small output buffer; synchronises with the stream.  FMM_ERR_ARG for other bits, reps < 1
 * or a null tflops. */
int fmm_measure_fma_rate(int bits, int reps, double* tflops, double* ms_per_launch, void* stream);

/* Message describing the last error on the calling thread ("" if none). */
const char* fmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OCTO_FMM_H */
