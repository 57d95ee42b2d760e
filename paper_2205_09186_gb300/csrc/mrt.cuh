// D2Q9 multiple-relaxation-time collision (Eq. 1, 3-5) with exact-difference
// forcing (Eq. 8).
//
// The moments of Eq. 3 are taken with the rows written out (velocity order of
// Eq. 2: rest, +x, +y, -x, -y, (1,1), (-1,1), (-1,-1), (1,-1)).  For the
// second-order equilibrium of Eq. 6 the equilibrium moments have the closed
// forms e = rho (-2 + 3 u^2), epsilon = rho (1 - 3 u^2), q = -rho u,
// p_xx = rho (u_x^2 - u_y^2), p_xy = rho u_x u_y; the conserved moments (rho,
// j) are at equilibrium by construction (u = j / rho).  The rows of M are
// orthogonal, so M^-1 = M^T diag(1 / |row|^2) with |row|^2 = 9, 36, 36, 6, 12,
// 6, 12, 4, 4.
#pragma once
#include "lbm_device.cuh"

namespace lbmd {

struct Mrt {
  double s[9];   // rates s_1..s_9 of Eq. 5 in the row order of Eq. 3
  double sd[9];  // s_k / |row k|^2, the factors of M^-1 S (FP64 kernels)
  float sf[9];   // the same in FP32 (FP32 kernels)
  int on;        // 0: single relaxation with 1/tau
};

// The operator of a case: mrt on/off and the nine rates; all-zero rates select
// the paper's (1, 1.64, 1.54, 1, 1.7, 1, 1.7, 1/tau, 1/tau).
inline Mrt make_mrt(bool on, const double* s9, double tau) {
  Mrt m{};
  m.on = on ? 1 : 0;
  bool zero = true;
  for (int k = 0; k < 9; ++k) zero = zero && s9[k] == 0.0;
  const double paper[9] = {1.0, 1.64, 1.54, 1.0, 1.7, 1.0, 1.7, 1.0 / tau, 1.0 / tau};
  const double norm2[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};
  for (int k = 0; k < 9; ++k) {
    m.s[k] = zero ? paper[k] : s9[k];
    m.sd[k] = m.s[k] / norm2[k];
    m.sf[k] = float(m.sd[k]);
  }
  return m;
}

// Post-collision populations of one node.  Populations are deviations
// f_i - w_i rho_ref (rho_ref = 0 for full values), dsv = rho - rho_ref; v =
// u + F / rho is the velocity of the forcing equilibrium (Eq. 8).
template <typename T>
__device__ __forceinline__ void mrt_post9(const T* fv, T dsv, T rho, T ux, T uy, T vx, T vy, const Mrt& m,
                                          T* out) {
  using L = Lattice<0>;
  const T u2 = ux * ux + uy * uy;
  // non-equilibrium parts of the six non-conserved moments; the reference
  // part w_i rho_ref contributes -2 rho_ref to e and rho_ref to epsilon
  const T s14 = fv[1] + fv[2] + fv[3] + fv[4], s58 = fv[5] + fv[6] + fv[7] + fv[8];
  const T ne = (T(-4) * fv[0] - s14 + T(2) * s58) + T(2) * dsv - T(3) * rho * u2;
  const T np = (T(4) * fv[0] - T(2) * s14 + s58) - dsv + T(3) * rho * u2;
  const T nqx = (T(2) * (fv[3] - fv[1]) + (fv[5] - fv[6] - fv[7] + fv[8])) + rho * ux;
  const T nqy = (T(2) * (fv[4] - fv[2]) + (fv[5] + fv[6] - fv[7] - fv[8])) + rho * uy;
  const T nxx = (fv[1] - fv[2] + fv[3] - fv[4]) - rho * (ux * ux - uy * uy);
  const T nxy = (fv[5] - fv[6] + fv[7] - fv[8]) - rho * ux * uy;
  auto r = [&](int k) { if constexpr (sizeof(T) == 8) return T(m.sd[k]); else return T(m.sf[k]); };
  const T a1 = r(1) * ne, a2 = r(2) * np;
  const T a4 = r(4) * nqx, a6 = r(6) * nqy;
  const T a7 = r(7) * nxx, a8 = r(8) * nxy;
  // M^-1 S (m - m_eq): column i of M weighting the scaled moments
  T c[9];
  c[0] = T(-4) * a1 + T(4) * a2;
  const T ax = -a1 - T(2) * a2;
  c[1] = ax - T(2) * a4 + a7;
  c[2] = ax - T(2) * a6 - a7;
  c[3] = ax + T(2) * a4 + a7;
  c[4] = ax + T(2) * a6 - a7;
  const T ad = T(2) * a1 + a2;
  c[5] = ad + a4 + a6 + a8;
  c[6] = ad - a4 + a6 - a8;
  c[7] = ad - a4 - a6 + a8;
  c[8] = ad + a4 - a6 - a8;
  // forcing: f_eq(rho, v) - f_eq(rho, u)
  const T uu15 = T(1.5) * u2, vv15 = T(1.5) * (vx * vx + vy * vy);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T eu = T(L::ex(i)) * ux + T(L::ey(i)) * uy, ev = T(L::ex(i)) * vx + T(L::ey(i)) * vy;
    const T Au = eu * (T(3) + T(4.5) * eu) - uu15, Av = ev * (T(3) + T(4.5) * ev) - vv15;
    out[i] = fv[i] - c[i] + T(L::w(i)) * rho * (Av - Au);
  }
}

}  // namespace lbmd
