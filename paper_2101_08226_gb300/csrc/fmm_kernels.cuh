// Device arithmetic of the octree FMM (Sec. 2.2): Cartesian expansions about cell centres of
// mass, symmetric truncation at total order 3, and the angular-momentum correction.
//
// Storage of one cell (structure of arrays, component c of cell i at c * n_cell + i):
//   moments   0: m | 1-3: delta = X - geometric centre | 4-9: M2 (xx xy xz yy yz zz)
//             10-19: M3 (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)
//   expansion 0: L0 | 1-3: L1 | 4-9: L2 (as M2) | 10-19: L3 (as M3)
// M2 = sum m r r and M3 = sum m r r r about the centre of mass (the dipole vanishes there).
// The Green's-function derivatives D^(n) = grad^n (1/|R|) are never formed as tensors: with
// g_n = (-1)^n (2n-1)!! / r^(2n+1) they are D^(n) = g_n R^n + g_(n-1) (R^(n-2) I)_sym + ..., and
// every contraction with a symmetric moment reduces to a few vector quantities.  Because
// 1/|R| is harmonic, every D^(n) is traceless in each pair of indices, so a contraction only sees
// the traceless part of a moment: the interaction kernels read detraced copies
//   M2' = M2 - (tr M2 / 3) I,   M3'_abc = M3_abc - (t_a d_bc + t_b d_ac + t_c d_ab) / 5,
// t_a = M3_abb, for which every term carrying a Kronecker delta drops out.
#pragma once
#include <cstdint>

#include "dfloat.cuh"

namespace octofmm {

constexpr int kNMom = 20;

// TRR_a = sum_bc T_abc R_b R_c of a symmetric 3rd-rank tensor T (10 unique entries, order as M3).
template <typename T>
__device__ __forceinline__ void sym3_rr(const T* t3, T x, T y, T z, T& rx, T& ry, T& rz) {
  T xx = x * x, yy = y * y, zz = z * z, xy2 = T(2) * x * y, xz2 = T(2) * x * z,
    yz2 = T(2) * y * z;
  rx = t3[0] * xx + t3[3] * yy + t3[5] * zz + t3[1] * xy2 + t3[2] * xz2 + t3[4] * yz2;
  ry = t3[1] * xx + t3[6] * yy + t3[8] * zz + t3[3] * xy2 + t3[4] * xz2 + t3[7] * yz2;
  rz = t3[2] * xx + t3[7] * yy + t3[9] * zz + t3[4] * xy2 + t3[5] * xz2 + t3[8] * yz2;
}

// Vector quantities of a symmetric 3rd-rank tensor T (10 unique entries, order as M3):
//   t_a = sum_b T_abb (trace vector) and TRR_a = sum_bc T_abc R_b R_c.
template <typename T>
__device__ __forceinline__ void sym3_vectors(const T* t3, T x, T y, T z, T& tx, T& ty, T& tz,
                                             T& rx, T& ry, T& rz) {
  // t3: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
  tx = t3[0] + t3[3] + t3[5];
  ty = t3[1] + t3[6] + t3[8];
  tz = t3[2] + t3[7] + t3[9];
  T xx = x * x, yy = y * y, zz = z * z, xy2 = T(2) * x * y, xz2 = T(2) * x * z,
    yz2 = T(2) * y * z;
  rx = t3[0] * xx + t3[3] * yy + t3[5] * zz + t3[1] * xy2 + t3[2] * xz2 + t3[4] * yz2;
  ry = t3[1] * xx + t3[6] * yy + t3[8] * zz + t3[3] * xy2 + t3[4] * xz2 + t3[7] * yz2;
  rz = t3[2] * xx + t3[7] * yy + t3[9] * zz + t3[4] * xy2 + t3[5] * xz2 + t3[8] * yz2;
}

// Radial factors g0..g4 of the derivatives of 1/r.
template <typename T>
__device__ __forceinline__ T rsqrt_t(T v);
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }
// FP32: the hardware approximation (PTX rsqrt.approx.ftz.f32, relative error below 2^-22.9)
// as one instruction; arguments are squared separations of at least a cell width, never
// subnormal.
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
template <>
__device__ __forceinline__ dfloat rsqrt_t<dfloat>(dfloat v) { return df_rsqrt(v); }

template <typename T>
struct Radial {
  T g0, g1, g2, g3, g4;
  __device__ __forceinline__ void set(T x, T y, T z, int order) {
    T r2 = x * x + y * y + z * z;
    T ri = rsqrt_t<T>(r2);
    T ri2 = ri * ri;
    g0 = ri;
    g1 = -g0 * ri2;
    if (order >= 2) g2 = T(-3) * g1 * ri2;
    if (order >= 3) g3 = T(-5) * g2 * ri2;
    if (order >= 4) g4 = T(-7) * g3 * ri2;
  }
};

// Expansion of a target A due to a source B with R = X_A - X_B (truncation k + n <= 3):
//   L0 -= m D0 + 1/2 D2:M2 - 1/6 D3:M3,   L1 -= m D1 + 1/2 D3:M2,   L2 -= m D2,   L3 -= m D3.
// With detraced moments: D2:M2' = g2 R.M2'.R, D3:M3' = g3 M3'(R,R,R),
// (D3:M2')_a = g3 R_a R.M2'.R + 2 g2 (M2' R)_a.
// Also returns q = M3'(R,R) and rrr = R.q, which the correction reuses.
template <typename T>
__device__ __forceinline__ void m2l_far(T x, T y, T z, const Radial<T>& g, T m, const T* M2,
                                        const T* M3, T* L, T& qx, T& qy, T& qz, T& rrr) {
  // M2: xx xy xz yy yz zz
  T m2rx = M2[0] * x + M2[1] * y + M2[2] * z;
  T m2ry = M2[1] * x + M2[3] * y + M2[4] * z;
  T m2rz = M2[2] * x + M2[4] * y + M2[5] * z;
  T rm2r = x * m2rx + y * m2ry + z * m2rz;
  sym3_rr(M3, x, y, z, qx, qy, qz);
  rrr = x * qx + y * qy + z * qz;
  const T sixth = T(1.0 / 6.0);
  L[0] -= m * g.g0 + T(0.5) * g.g2 * rm2r - sixth * g.g3 * rrr;
  T c1 = m * g.g1 + T(0.5) * g.g3 * rm2r;
  L[1] -= c1 * x + g.g2 * m2rx;
  L[2] -= c1 * y + g.g2 * m2ry;
  L[3] -= c1 * z + g.g2 * m2rz;
}

// Monopole-only part of the expansion (a source with M2 = M3 = 0, e.g. a leaf cell): the
// potential and the field, L0 -= m g0, L1 -= m g1 R.
template <typename T>
__device__ __forceinline__ void m2l_mono(T x, T y, T z, const Radial<T>& g, T m, T* L) {
  L[0] -= m * g.g0;
  T c = m * g.g1;
  L[1] -= c * x;
  L[2] -= c * y;
  L[3] -= c * z;
}

// Second and third derivatives of the expansion (needed only by targets with children):
//   L2_ab -= m (g2 R_a R_b + g1 d_ab),  L3_abc -= m (g3 R_a R_b R_c + g2 (R_a d_bc + ...)).
// Both sums are traceless (every D^(n) is), so only the independent components L2 xx xy xz yy yz
// and L3 xxx xxy xxz xyy xyz yyy yyz are accumulated; complete_traceless() fills in the rest.
template <typename T>
__device__ __forceinline__ void m2l_high(T x, T y, T z, const Radial<T>& g, T m, T* L) {
  T a2 = m * g.g2, a1 = m * g.g1, a3 = m * g.g3;
  T a2x = a2 * x, a2y = a2 * y, a2z = a2 * z;
  L[4] -= a2x * x + a1;
  L[5] -= a2x * y;
  L[6] -= a2x * z;
  L[7] -= a2y * y + a1;
  L[8] -= a2y * z;
  T a3xx = a3 * x * x, a3yy = a3 * y * y;
  L[10] -= a3xx * x + T(3) * a2x;
  L[11] -= a3xx * y + a2y;
  L[12] -= a3xx * z + a2z;
  L[13] -= a3yy * x + a2x;
  L[14] -= a3 * x * y * z;
  L[16] -= a3yy * y + T(3) * a2y;
  L[17] -= a3yy * z + a2z;
}

// L2zz = -(L2xx + L2yy); L3xzz = -(L3xxx + L3xyy), L3yzz = -(L3xxy + L3yyy),
// L3zzz = -(L3xxz + L3yyz).
template <typename T>
__device__ __forceinline__ void complete_traceless(T* L) {
  L[9] = -(L[4] + L[7]);
  L[15] = -(L[10] + L[13]);
  L[18] = -(L[11] + L[16]);
  L[19] = -(L[12] + L[17]);
}

// Angular-momentum correction acceleration of A (Sec. 2.2):
//   a_A += 1/6 D4 : Q,  Q = (m_B / m_A) M3'_A - M3'_B,
//   (D4:Q)_a = g4 R_a Q(R,R,R) + 3 g3 Q(R,R)_a  (Q traceless),
// given the contracted vector Q(R,R) and Q(R,R,R) (linear in Q, so the parts of M3'_A and M3'_B
// are contracted separately and M3'_B(R,R) is shared with the expansion).
template <typename T>
__device__ __forceinline__ void amc_from(T x, T y, T z, const Radial<T>& g, T qx, T qy, T qz,
                                         T qrrr, T& ax, T& ay, T& az) {
  const T sixth = T(1.0 / 6.0);
  T c4 = sixth * g.g4 * qrrr, c3 = T(0.5) * g.g3;
  ax = c4 * x + c3 * qx;
  ay = c4 * y + c3 * qy;
  az = c4 * z + c3 * qz;
}

}  // namespace octofmm
