// Self-consistent-field (SCF) iteration of a synchronously rotating binary (Sec. 4.1): the
// device kernels (scf.cu) and their launchers, called by fmm_scf_init / fmm_scf_iterate in fmm.cu,
// which own the tree, its gravity solves and the stream order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace octofmm {

// Leaf geometry of one tree in canonical leaf order (leaf cell i = ordinal * 512 + (a*8+b)*8+c):
// the subgrid of each leaf ordinal, every subgrid's level and (i, j, k), and the leaf cells whose
// closure touches the x axis (the line through both stars).
struct ScfGeom {
  int64_t n_leaf_cells;
  const int32_t* leaf_sub;  // [n_leaf_sub]
  const int32_t* level;     // [n_sub]
  const int32_t* ijk;       // [3 n_sub]
  const int64_t* axis;      // [n_axis] canonical leaf indices
  int64_t n_axis;
};

// The prescribed problem (fmm_scf_params without the solver settings).
struct ScfProblem {
  double M1, M2, n, f, J0, rho_floor;
};

constexpr int kScfState = 22;  // the public state entries (octo_fmm.h, FMM_SCF_STATE)

// Device state: the public entries, then the step's internal values.
struct ScfState {
  double v[kScfState];
  double s1, s2;       // step (1)'s scale factors
  int64_t i1, i2;      // the cells of largest density of the accretor and the donor
  int32_t ok;          // 0 once a star had no material or no axis cell lay between the centres
};

// Per-block partial results of the density pass and of the axis pass.
struct ScfPartial {
  double m[2], mx[2][3];
  double rmax[2];
  int64_t imax[2];
};
struct ScfAxisPartial {
  double v;
  int64_t i;
};

constexpr int kScfThreads = 256;

// State entry indices (the order of the public state).
enum ScfKey {
  kK = 0, kOmega, kC1, kC2, kXL1, kPhiL1, kX1x, kX1y, kX1z, kX2x, kX2y, kX2z, kXcmx, kXcmy, kXcmz,
  kA, kM1raw, kM2raw, kRho1, kRho2, kPhi1, kPhiC
};

int scf_blocks(int64_t n);
// initial state: centres from the density split at x = 0, Kepler Omega, L1 from phi
cudaError_t scf_launch_init(const ScfGeom& G, const ScfProblem& P, const double* rho, const double* phi,
                            double K0, ScfState* st, ScfPartial* part, ScfAxisPartial* apart,
                            cudaStream_t s);
// step (1): masses, centres and densest cells of the stars, then the scaling of rho in place
cudaError_t scf_launch_scale(const ScfGeom& G, const ScfProblem& P, double* rho, ScfState* st,
                             ScfPartial* part, cudaStream_t s);
// steps (2)-(6) after the solve: L1, C1, C2, K, and the new density into rho (in place); the state
// is copied to history (kScfState doubles) when history is not null
cudaError_t scf_launch_update(const ScfGeom& G, const ScfProblem& P, double* rho, const double* phi,
                              ScfState* st, ScfAxisPartial* apart, double* history, cudaStream_t s);

}  // namespace octofmm
