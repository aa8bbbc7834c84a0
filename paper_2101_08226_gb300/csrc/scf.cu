// Self-consistent-field iteration of a synchronously rotating binary (Sec. 4.1) on the device.
//
// One iteration is three kernel groups around the library's gravity solve, all on one stream and
// with every scalar of the iteration kept in a device state (no host round trip):
//   scale   step (1): each star's mass, centre of mass and densest cell (one pass over the leaf
//           cells, fixed-order partial sums), the scale factors and steps (2)-(3) -- the centre
//           of mass of the system and Omega = J0 (M1 + M2) / (M1 M2 a^2) -- then the densities of
//           each star multiplied by its factor;
//   (the solve of the scaled density, step (7) of the previous iteration)
//   update  step (4): phi_eff = phi - Omega^2 r^2 / 2 about the axis through the centre of mass,
//           L1 as the axis cell of largest phi_eff between the centres, C2 = (1 - f) phi_C +
//           f phi_L1; step (5): K = (C2 - phi_C) / ((n + 1) rho_2^(1/n)), then C1 = K (1 + n)
//           rho_1^(1/n) + phi_1; step (6): rho = ((C - phi_eff) / (K (n + 1)))^n inside each
//           star's ball up to the plane of L1, the atmosphere density elsewhere.
// Stars: the accretor is the material (density above the atmosphere) at x < x_L1, the donor at
// x >= x_L1.  Ties of the densest cell and of L1 go to the first cell in canonical leaf order.
#include "scf.cuh"

#include <cmath>

namespace octofmm {

namespace {

// Centre of leaf cell i in canonical leaf order, from integer coordinates: the double
// (2 g + 1 - 2^(l + 3)) 2^-(l + 4) is exact.
__device__ __forceinline__ void leaf_centre(const ScfGeom& G, int64_t i, double x[3]) {
  const int32_t s = G.leaf_sub[i >> 9];
  const int lev = G.level[s];
  const int loc = int(i & 511);
  const int full = 1 << (lev + 3);
  const double sc = ldexp(1.0, -(lev + 4));
  x[0] = double(2 * (G.ijk[3 * s] * 8 + (loc >> 6)) + 1 - full) * sc;
  x[1] = double(2 * (G.ijk[3 * s + 1] * 8 + ((loc >> 3) & 7)) + 1 - full) * sc;
  x[2] = double(2 * (G.ijk[3 * s + 2] * 8 + (loc & 7)) + 1 - full) * sc;
}
__device__ __forceinline__ double leaf_volume(const ScfGeom& G, int64_t i) {
  return ldexp(1.0, -3 * (G.level[G.leaf_sub[i >> 9]] + 3));
}

// (v, i) is the better maximum: larger value, or the same value at a smaller index.
__device__ __forceinline__ bool better(double v, int64_t i, double w, int64_t j) {
  return v > w || (v == w && i < j);
}

__device__ __forceinline__ double phi_eff(const double* st, double phi, const double x[3]) {
  const double dx = x[0] - st[kXcmx], dy = x[1] - st[kXcmy];
  const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return __dsub_rn(phi, __dmul_rn(__dmul_rn(0.5 * st[kOmega], st[kOmega]), r2));
}

// One pass over the leaf cells: per star (split by the plane x = state x_L1) the mass, the first
// moment and the densest cell of the star material.
__global__ void __launch_bounds__(kScfThreads) k_scf_stats(ScfGeom G, ScfProblem P, const double* __restrict__ rho,
                                                           const ScfState* __restrict__ st,
                                                           ScfPartial* __restrict__ part) {
  __shared__ ScfPartial sh[kScfThreads];
  ScfPartial a = {};
  a.rmax[0] = a.rmax[1] = -1.0;
  a.imax[0] = a.imax[1] = INT64_MAX;
  const double xl1 = st->v[kXL1];
  for (int64_t i = int64_t(blockIdx.x) * kScfThreads + threadIdx.x; i < G.n_leaf_cells;
       i += int64_t(gridDim.x) * kScfThreads) {
    const double r = rho[i];
    if (!(r > P.rho_floor)) continue;
    double x[3];
    leaf_centre(G, i, x);
    const int k = x[0] < xl1 ? 0 : 1;
    const double m = r * leaf_volume(G, i);
    a.m[k] += m;
    for (int d = 0; d < 3; ++d) a.mx[k][d] += m * x[d];
    if (better(r, i, a.rmax[k], a.imax[k])) {
      a.rmax[k] = r;
      a.imax[k] = i;
    }
  }
  const int t = threadIdx.x;
  sh[t] = a;
  __syncthreads();
  for (int w = kScfThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      ScfPartial& u = sh[t];
      const ScfPartial& v = sh[t + w];
      for (int k = 0; k < 2; ++k) {
        u.m[k] += v.m[k];
        for (int d = 0; d < 3; ++d) u.mx[k][d] += v.mx[k][d];
        if (better(v.rmax[k], v.imax[k], u.rmax[k], u.imax[k])) {
          u.rmax[k] = v.rmax[k];
          u.imax[k] = v.imax[k];
        }
      }
    }
    __syncthreads();
  }
  if (t == 0) part[blockIdx.x] = sh[0];
}

// One thread: the partials in block order, then the centres, the system's centre of mass, the
// separation and Omega (init: Kepler at the separation; step: from J0), and, in a step, the scale
// factors and the scaled central densities.
__global__ void k_scf_centres(ScfProblem P, const ScfPartial* __restrict__ part, int nb,
                              const double* __restrict__ rho, ScfState* __restrict__ st, int init) {
  double m[2] = {0.0, 0.0}, mx[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  double rmax[2] = {-1.0, -1.0};
  int64_t imax[2] = {INT64_MAX, INT64_MAX};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 2; ++k) {
      m[k] += part[b].m[k];
      for (int d = 0; d < 3; ++d) mx[k][d] += part[b].mx[k][d];
      if (better(part[b].rmax[k], part[b].imax[k], rmax[k], imax[k])) {
        rmax[k] = part[b].rmax[k];
        imax[k] = part[b].imax[k];
      }
    }
  double* v = st->v;
  if (!st->ok || !(m[0] > 0.0) || !(m[1] > 0.0)) {  // a star without material: give up
    st->ok = 0;
    v[kK] = NAN;
    return;
  }
  double X[2][3];
  for (int k = 0; k < 2; ++k)
    for (int d = 0; d < 3; ++d) X[k][d] = mx[k][d] / m[k];
  const double Mt = P.M1 + P.M2;
  for (int d = 0; d < 3; ++d) {
    v[kX1x + d] = X[0][d];
    v[kX2x + d] = X[1][d];
    v[kXcmx + d] = (P.M1 * X[0][d] + P.M2 * X[1][d]) / Mt;
  }
  const double ex = X[0][0] - X[1][0], ey = X[0][1] - X[1][1], ez = X[0][2] - X[1][2];
  const double a = sqrt(ex * ex + ey * ey + ez * ez);
  v[kA] = a;
  if (init) {
    v[kOmega] = sqrt(Mt / (a * a * a));
    return;
  }
  v[kOmega] = P.J0 * Mt / (P.M1 * P.M2 * a * a);
  v[kM1raw] = m[0];
  v[kM2raw] = m[1];
  st->s1 = P.M1 / m[0];
  st->s2 = P.M2 / m[1];
  st->i1 = imax[0];
  st->i2 = imax[1];
  v[kRho1] = rho[imax[0]] * st->s1;
  v[kRho2] = rho[imax[1]] * st->s2;
}

// Step (1): every star cell multiplied by its star's factor (the same split as k_scf_stats).
__global__ void k_scf_scale(ScfGeom G, ScfProblem P, double* __restrict__ rho,
                            const ScfState* __restrict__ st) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= G.n_leaf_cells || !st->ok) return;
  const double r = rho[i];
  if (!(r > P.rho_floor)) return;
  double x[3];
  leaf_centre(G, i, x);
  rho[i] = r * (x[0] < st->v[kXL1] ? st->s1 : st->s2);
}

// The axis cells between the two centres: the largest phi_eff (first index on a tie).
__global__ void __launch_bounds__(kScfThreads) k_scf_axis(ScfGeom G, const double* __restrict__ phi,
                                                          const ScfState* __restrict__ st,
                                                          ScfAxisPartial* __restrict__ part) {
  __shared__ ScfAxisPartial sh[kScfThreads];
  const double* v = st->v;
  const double lo = fmin(v[kX1x], v[kX2x]), hi = fmax(v[kX1x], v[kX2x]);
  ScfAxisPartial a = {-INFINITY, INT64_MAX};
  for (int64_t q = int64_t(blockIdx.x) * kScfThreads + threadIdx.x; q < G.n_axis;
       q += int64_t(gridDim.x) * kScfThreads) {
    const int64_t i = G.axis[q];
    double x[3];
    leaf_centre(G, i, x);
    if (!(x[0] > lo && x[0] < hi)) continue;
    const double pe = phi_eff(v, phi[i], x);
    if (better(pe, i, a.v, a.i)) a = ScfAxisPartial{pe, i};
  }
  const int t = threadIdx.x;
  sh[t] = a;
  __syncthreads();
  for (int w = kScfThreads / 2; w > 0; w >>= 1) {
    if (t < w && better(sh[t + w].v, sh[t + w].i, sh[t].v, sh[t].i)) sh[t] = sh[t + w];
    __syncthreads();
  }
  if (t == 0) part[blockIdx.x] = sh[0];
}

// One thread: L1, then (step) C2, K, C1; the state copied to history.
__global__ void k_scf_consts(ScfGeom G, ScfProblem P, const ScfAxisPartial* __restrict__ part, int nb,
                             const double* __restrict__ phi, ScfState* __restrict__ st, double* history,
                             int init) {
  ScfAxisPartial best = {-INFINITY, INT64_MAX};
  for (int b = 0; b < nb; ++b)
    if (better(part[b].v, part[b].i, best.v, best.i)) best = part[b];
  double* v = st->v;
  if (!st->ok || best.i == INT64_MAX) {  // no axis cell between the centres: give up
    st->ok = 0;
    v[kK] = NAN;
    if (history)
      for (int k = 0; k < kScfState; ++k) history[k] = v[k];
    return;
  }
  double x[3];
  leaf_centre(G, best.i, x);
  v[kXL1] = x[0];
  v[kPhiL1] = best.v;
  if (!init) {
    const double n = P.n;
    leaf_centre(G, st->i1, x);
    const double phi1 = phi_eff(v, phi[st->i1], x);
    leaf_centre(G, st->i2, x);
    const double phiC = phi_eff(v, phi[st->i2], x);
    v[kPhi1] = phi1;
    v[kPhiC] = phiC;
    const double C2 = (1.0 - P.f) * phiC + P.f * best.v;
    const double K = (C2 - phiC) / ((n + 1.0) * pow(v[kRho2], 1.0 / n));
    v[kC2] = C2;
    v[kK] = K;
    v[kC1] = K * (1.0 + n) * pow(v[kRho1], 1.0 / n) + phi1;
  }
  if (history)
    for (int k = 0; k < kScfState; ++k) history[k] = v[k];
}

// Step (6): the new density of every leaf cell.
__global__ void k_scf_density(ScfGeom G, ScfProblem P, const double* __restrict__ phi,
                              const ScfState* __restrict__ st, double* __restrict__ rho) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= G.n_leaf_cells || !st->ok) return;
  const double* v = st->v;
  double x[3];
  leaf_centre(G, i, x);
  const double xl1 = v[kXL1];
  const int k = x[0] < xl1 ? 0 : 1;
  const double* X = v + (k == 0 ? kX1x : kX2x);
  const double d = fabs(xl1 - X[0]);
  const double ex = x[0] - X[0], ey = x[1] - X[1], ez = x[2] - X[2];
  double r = P.rho_floor;
  if (sqrt(ex * ex + ey * ey + ez * ez) < d) {
    const double h = ((k == 0 ? v[kC1] : v[kC2]) - phi_eff(v, phi[i], x)) / (v[kK] * (P.n + 1.0));
    if (h > 0.0) r = fmax(pow(h, P.n), P.rho_floor);
  }
  rho[i] = r;
}

__global__ void k_scf_begin(ScfState* st, double K0) {
  for (int k = 0; k < kScfState; ++k) st->v[k] = 0.0;
  st->v[kK] = K0;
  st->v[kXL1] = 0.0;  // the initial split of the stars
  st->s1 = st->s2 = 1.0;
  st->i1 = st->i2 = 0;
  st->ok = 1;
}

}  // namespace

int scf_blocks(int64_t n) {
  const int64_t b = (n + kScfThreads - 1) / kScfThreads;
  return int(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t scf_launch_init(const ScfGeom& G, const ScfProblem& P, const double* rho, const double* phi,
                            double K0, ScfState* st, ScfPartial* part, ScfAxisPartial* apart,
                            cudaStream_t s) {
  const int nb = scf_blocks(G.n_leaf_cells), na = scf_blocks(G.n_axis);
  k_scf_begin<<<1, 1, 0, s>>>(st, K0);
  k_scf_stats<<<nb, kScfThreads, 0, s>>>(G, P, rho, st, part);
  k_scf_centres<<<1, 1, 0, s>>>(P, part, nb, rho, st, 1);
  k_scf_axis<<<na, kScfThreads, 0, s>>>(G, phi, st, apart);
  k_scf_consts<<<1, 1, 0, s>>>(G, P, apart, na, phi, st, nullptr, 1);
  return cudaGetLastError();
}

cudaError_t scf_launch_scale(const ScfGeom& G, const ScfProblem& P, double* rho, ScfState* st,
                             ScfPartial* part, cudaStream_t s) {
  const int nb = scf_blocks(G.n_leaf_cells);
  k_scf_stats<<<nb, kScfThreads, 0, s>>>(G, P, rho, st, part);
  k_scf_centres<<<1, 1, 0, s>>>(P, part, nb, rho, st, 0);
  k_scf_scale<<<unsigned((G.n_leaf_cells + 255) / 256), 256, 0, s>>>(G, P, rho, st);
  return cudaGetLastError();
}

cudaError_t scf_launch_update(const ScfGeom& G, const ScfProblem& P, double* rho, const double* phi,
                              ScfState* st, ScfAxisPartial* apart, double* history, cudaStream_t s) {
  const int na = scf_blocks(G.n_axis);
  k_scf_axis<<<na, kScfThreads, 0, s>>>(G, phi, st, apart);
  k_scf_consts<<<1, 1, 0, s>>>(G, P, apart, na, phi, st, history, 0);
  k_scf_density<<<unsigned((G.n_leaf_cells + 255) / 256), 256, 0, s>>>(G, P, phi, st, rho);
  return cudaGetLastError();
}

}  // namespace octofmm
