// Device-side building blocks of the chemical-potential multiphase LBM step:
// lattice tables, the Carnahan-Starling chemical potential, the difference
// stencils of Sec. 2.3 and the BGK + exact-difference-method collision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmd {

// ------------------------------------------------------------------ lattices
// D2Q9 in the order of Eq. 2; D3Q19: rest, +-x, +-y, +-z, twelve edges.
template <int LAT>
struct Lattice;

template <>
struct Lattice<0> {
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int ex(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
  __host__ __device__ static constexpr int ey(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
  __host__ __device__ static constexpr int ez(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

template <>
struct Lattice<1> {
  static constexpr int Q = 19, D = 3;
  // rows: rest; +x -x +y -y +z -z; (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
  //       (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
  __host__ __device__ static constexpr int ex(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
  }
  __host__ __device__ static constexpr int ey(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
  }
  __host__ __device__ static constexpr int ez(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

// ------------------------------------------------------------------ precision policies
// FP64: everything double.  FP32DEV: populations stored as f_i - w_i rho_ref and
// the density field as rho - rho_ref, both in float; collision and stencils in
// float; Tm is the type of the chemical potential.  No FP64 instruction is on
// the FP32DEV step path unless Tm is double.
struct PrecF64 {
  using Tr = double;  // stored density field (full density)
  using Tf = double;  // stored population
  using Tc = double;  // collision / force arithmetic
  using Ts = double;  // density stencil operand
  using Tm = double;  // chemical potential
  static constexpr bool DEV = false;
};
struct PrecF32 {
  using Tr = float;  // stored density field: rho - rho_ref
  using Tf = float;
  using Tc = float;
  using Ts = float;
  using Tm = float;
  static constexpr bool DEV = true;
};
struct PrecF32M64 {
  using Tr = float;
  using Tf = float;
  using Tc = float;
  using Ts = float;
  using Tm = double;
  static constexpr bool DEV = true;
};

// ------------------------------------------------------------------ parameters
struct KParams {
  int nx, ny, nz;
  long long n;            // nodes
  double RT, b4, two_a;   // R*T, b/4, 2a of the CS chemical potential
  double k2, kappa;       // k^2 and kappa-hat (Eq. 16)
  double omega;           // 1/tau
  double rho_ref;         // FP32DEV reference density (0 in FP64 mode)
  int eos;                // 0 Carnahan-Starling, 1 Peng-Robinson (Eq. 14-15), 2 van der Waals, 3 Redlich-Kwong-Soave
  double aa, c1;          // PR: a alpha(T), a alpha(T) / (2 sqrt2 b); RKS: a alpha(T), a alpha(T) / b
};

struct StepAux {
  long long t;                     // step index of the state being advanced
  unsigned long long* bad_step;    // atomicMin target: first step with rho <= 0 or NaN
  double* partials;                // observables: per-block partial results
  const void* rho_snap;            // observables: density field (type Tr) at the previous observation
};

__device__ __forceinline__ float lg(float x) { return logf(x); }
__device__ __forceinline__ double lg(double x) { return log(x); }

// Bulk chemical potential psi'(rho) of the Carnahan-Starling fluid, from
// Eq. 10 and Eq. 13:  R T [ln rho + eta (8 - 9 eta + 3 eta^2)/(1 - eta)^3] - 2 a rho.
template <typename T>
__device__ __forceinline__ T cs_mu(T rho, T RT, T b4, T two_a) {
  T eta = b4 * rho;
  T om = T(1) - eta;
  T hs = eta * (T(8) + eta * (T(-9) + T(3) * eta)) / (om * om * om);
  return RT * (lg(rho) + hs) - two_a * rho;
}

// Bulk chemical potential of the Peng-Robinson fluid, Eq. 15 without the
// kappa term: with x = b rho,
//   R T [ln(rho / (1 - x)) + 1 / (1 - x)] - c1 ln((sqrt2 - 1 + x) / (sqrt2 + 1 - x)) - a alpha rho / (1 + 2x - x^2),
// c1 = a alpha / (2 sqrt2 b).
template <typename T>
__device__ __forceinline__ T pr_mu(T rho, T RT, T b, T aa, T c1) {
  const T x = b * rho, om = T(1) - x;
  const T s2 = T(1.4142135623730950488);
  return RT * (lg(rho / om) + T(1) / om) - c1 * lg((s2 - T(1) + x) / (s2 + T(1) - x)) -
         aa * rho / (T(1) + x * (T(2) - x));
}

// van der Waals and Redlich-Kwong-Soave by Eq. 13: with x = b rho the
// repulsive part is R T [ln(rho / (1 - x)) + 1 / (1 - x)]; the attractive part
// is -2 a rho (VDW) or -(a alpha / b) ln(1 + x) - a alpha rho / (1 + x) (RKS).
template <typename T>
__device__ __forceinline__ T vdw_mu(T rho, T RT, T b, T two_a) {
  const T om = T(1) - b * rho;
  return RT * (lg(rho / om) + T(1) / om) - two_a * rho;
}
template <typename T>
__device__ __forceinline__ T rks_mu(T rho, T RT, T b, T aa, T c1) {
  const T x = b * rho, om = T(1) - x;
  return RT * (lg(rho / om) + T(1) / om) - c1 * lg(T(1) + x) - aa * rho / (T(1) + x);
}

// psi'(rho) of the case's EOS (Eq. 10, 13-15), additive constant dropped
template <typename T>
__device__ __forceinline__ T eos_mu(T rho, const KParams& p) {
  if (p.eos == 1) return pr_mu<T>(rho, T(p.RT), T(4.0 * p.b4), T(p.aa), T(p.c1));
  if (p.eos == 2) return vdw_mu<T>(rho, T(p.RT), T(4.0 * p.b4), T(p.two_a));
  if (p.eos == 3) return rks_mu<T>(rho, T(p.RT), T(4.0 * p.b4), T(p.aa), T(p.c1));
  return cs_mu<T>(rho, T(p.RT), T(p.b4), T(p.two_a));
}

// FP32 form with the hardware logarithm and division approximations, for the
// FP32-deviation kernels; the constants converted once per thread
struct EosF {
  int eos;
  float RT, b4, two_a, b, aa, c1;
};
__device__ __forceinline__ EosF eos_f(const KParams& p) {
  return EosF{p.eos, float(p.RT), float(p.b4), float(p.two_a), float(4.0 * p.b4), float(p.aa), float(p.c1)};
}
__device__ __forceinline__ float eos_mu_f(float rho, const EosF& e) {
  if (e.eos >= 2) {
    const float x = e.b * rho, iom = __fdividef(1.f, 1.f - x);
    const float rep = e.RT * (__logf(rho * iom) + iom);
    if (e.eos == 2) return rep - e.two_a * rho;
    return rep - e.c1 * __logf(1.f + x) - __fdividef(e.aa * rho, 1.f + x);
  }
  if (e.eos == 1) {
    const float x = e.b * rho, om = 1.f - x;
    const float iom = __fdividef(1.f, om);
    return e.RT * (__logf(rho * iom) + iom) -
           e.c1 * __logf(__fdividef(0.41421356f + x, 2.41421356f - x)) -
           __fdividef(e.aa * rho, 1.f + x * (2.f - x));
  }
  const float eta = e.b4 * rho, om = 1.f - eta;
  const float hs = __fdividef(eta * (8.f + eta * (-9.f + 3.f * eta)), om * om * om);
  return e.RT * (__logf(rho) + hs) - e.two_a * rho;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// periodic wrap of an index in [-n, inf): also for halo regions wider than a
// small lattice (a 38-wide region on an 8-wide lattice reaches 4 periods out).
// A loop, not i % n: the common case costs two compares, and a select form
// lets the compiler evaluate the division for every index.
__device__ __forceinline__ int wrapn(int i, int n) {
  if (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// ------------------------------------------------------------------ difference stencils
// Line schemes (Eq. 18-20): derivative = sum_m g(m) (phi[+m] - phi[-m]);
// matching-order central second derivative sum_m l(m) (phi[+m] + phi[-m]) + l(0) phi.
// Isotropic schemes (Eq. 25): gradient sum_i w(|e_i|^2) e_i phi(x + e_i),
// Laplacian 2 sum_i w(|e_i|^2) (phi(x + e_i) - phi(x)).
enum { S_EFDS2 = 0, S_EFDS4 = 1, S_EFDS6 = 2, S_CFDS4 = 3, S_CFDS6 = 4, S_CFDS8 = 5, S_OCFDS4 = 6, S_E4 = 7, S_E8 = 8 };

template <int S>
struct Sch;

// GF: gradients are read from precomputed fields (compact schemes, solved by
// line kernels); the fused kernel then needs no stencil halo (R = 0).
template <>
struct Sch<S_EFDS2> {
  static constexpr int R = 1;
  static constexpr bool ISO = false, GF = false;
  __host__ __device__ static constexpr double g(int) { return 0.5; }
  __host__ __device__ static constexpr double l(int m) { return m == 0 ? -2.0 : 1.0; }
};
template <>
struct Sch<S_EFDS4> {
  static constexpr int R = 2;
  static constexpr bool ISO = false, GF = false;
  __host__ __device__ static constexpr double g(int m) { return m == 1 ? 2.0 / 3.0 : -1.0 / 12.0; }
  __host__ __device__ static constexpr double l(int m) { return m == 0 ? -2.5 : (m == 1 ? 4.0 / 3.0 : -1.0 / 12.0); }
};
template <>
struct Sch<S_EFDS6> {
  static constexpr int R = 3;
  static constexpr bool ISO = false, GF = false;
  __host__ __device__ static constexpr double g(int m) { return m == 1 ? 0.75 : (m == 2 ? -0.15 : 1.0 / 60.0); }
  __host__ __device__ static constexpr double l(int m) {
    return m == 0 ? -49.0 / 18.0 : (m == 1 ? 1.5 : (m == 2 ? -0.15 : 1.0 / 90.0));
  }
};
// isotropic: weight of offset (dx, dy, dz); 0 outside the stencil
template <>
struct Sch<S_E4> {
  static constexpr int R = 1;
  static constexpr bool ISO = true, GF = false;
  __host__ __device__ static constexpr double w2d(int dx, int dy) {
    return (dx * dx + dy * dy == 1) ? 1.0 / 3.0 : (dx * dx + dy * dy == 2 ? 1.0 / 12.0 : 0.0);
  }
  __host__ __device__ static constexpr double w3d(int dx, int dy, int dz) {
    return (dx * dx + dy * dy + dz * dz == 1) ? 1.0 / 6.0 : (dx * dx + dy * dy + dz * dz == 2 ? 1.0 / 12.0 : 0.0);
  }
};
template <>
struct Sch<S_E8> {
  static constexpr int R = 2;
  static constexpr bool ISO = true, GF = false;
  __host__ __device__ static constexpr double w2d(int dx, int dy) {
    return (dx * dx + dy * dy == 1) ? 4.0 / 21.0
         : (dx * dx + dy * dy == 2) ? 4.0 / 45.0
         : (dx * dx + dy * dy == 4) ? 1.0 / 60.0
         : (dx * dx + dy * dy == 5) ? 2.0 / 315.0
         : (dx * dx + dy * dy == 8) ? 1.0 / 5040.0 : 0.0;
  }
  __host__ __device__ static constexpr double w3d(int, int, int) { return 0.0; }
};

// compact schemes in the fused kernel: gradients come from fields
template <>
struct Sch<S_CFDS4> {
  static constexpr int R = 0;
  static constexpr bool ISO = false, GF = true;
  __host__ __device__ static constexpr double g(int) { return 0.0; }
  __host__ __device__ static constexpr double l(int) { return 0.0; }
};

// precomputed gradient fields (component-major, D*N) and mu (N) for GF schemes
struct GradIn {
  const void* gmu;
  const void* grho;
  const void* mu;
};

// 2D gradient and Laplacian on a row-major shared array at (cx, cy), row stride W.
template <int S, typename T, typename A>
__device__ __forceinline__ void grad2d(const A* s, int W, int cx, int cy, T& gx, T& gy) {
  using Sc = Sch<S>;
  constexpr int R = Sc::R;
  T ax = 0, ay = 0;
  if constexpr (Sc::ISO) {
#pragma unroll
    for (int dy = -R; dy <= R; ++dy)
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        const double w = Sc::w2d(dx, dy);
        if (w != 0.0) {
          T v = T(s[(cy + dy) * W + cx + dx]);
          if (dx != 0) ax += T(w * dx) * v;
          if (dy != 0) ay += T(w * dy) * v;
        }
      }
  } else {
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      ax += T(Sc::g(m)) * (T(s[cy * W + cx + m]) - T(s[cy * W + cx - m]));
      ay += T(Sc::g(m)) * (T(s[(cy + m) * W + cx]) - T(s[(cy - m) * W + cx]));
    }
  }
  gx = ax;
  gy = ay;
}

template <int S, typename T, typename A>
__device__ __forceinline__ T lap2d(const A* s, int W, int cx, int cy) {
  using Sc = Sch<S>;
  constexpr int R = Sc::R;
  T c = T(s[cy * W + cx]);
  T acc = 0;
  if constexpr (Sc::ISO) {
#pragma unroll
    for (int dy = -R; dy <= R; ++dy)
#pragma unroll
      for (int dx = -R; dx <= R; ++dx) {
        const double w = Sc::w2d(dx, dy);
        if (w != 0.0) acc += T(2.0 * w) * (T(s[(cy + dy) * W + cx + dx]) - c);
      }
  } else {
    acc = T(2.0 * Sc::l(0)) * c;
#pragma unroll
    for (int m = 1; m <= R; ++m)
      acc += T(Sc::l(m)) * ((T(s[cy * W + cx + m]) + T(s[cy * W + cx - m])) + (T(s[(cy + m) * W + cx]) + T(s[(cy - m) * W + cx])));
  }
  return acc;
}

// ------------------------------------------------------------------ collision
// Post-collision population in deviation form (rho_ref = 0 gives the plain form):
//   d*_i = (1 - omega) d_i + omega w_i (rho - rho_ref) + w_i rho [omega A_i(u) + A_i(u + du) - A_i(u)],
//   A_i(U) = 3 e_i.U + 4.5 (e_i.U)^2 - 1.5 U.U,
// which is f_i - (f_i - f_i^eq(rho,u))/tau + [f_i^eq(rho,u+du) - f_i^eq(rho,u)] (Eq. 1, 6, 8)
// with f_i^eq - w_i rho_ref written out.
template <int LAT, typename T>
__device__ __forceinline__ T coll_one(int i, T d, T dr, T rho, T omega, T ux, T uy, T uz, T vx, T vy, T vz) {
  using L = Lattice<LAT>;
  const T ei_u = T(L::ex(i)) * ux + T(L::ey(i)) * uy + T(L::ez(i)) * uz;
  const T ei_v = T(L::ex(i)) * vx + T(L::ey(i)) * vy + T(L::ez(i)) * vz;
  const T uu = ux * ux + uy * uy + uz * uz;
  const T vv = vx * vx + vy * vy + vz * vz;
  const T Au = T(3) * ei_u + T(4.5) * ei_u * ei_u - T(1.5) * uu;
  const T Av = T(3) * ei_v + T(4.5) * ei_v * ei_v - T(1.5) * vv;
  const T w = T(L::w(i));
  return (T(1) - omega) * d + omega * w * dr + w * rho * (omega * Au + Av - Au);
}

// Error-free float summation (TwoSum accumulation) used for densities in
// FP32DEV mode: returns s_hi + s_lo ~= exact sum of the terms.
// asynchronous global -> shared copies (4 bytes, through L1) and their groups
__device__ __forceinline__ void cpa4(void* sdst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// 16 bytes, L2 only; both addresses 16-byte aligned
__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// all but the most recent group complete
__device__ __forceinline__ void cpa_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// all but the N most recent groups complete
template <int N>
__device__ __forceinline__ void cpa_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ int ring(int s, int n) { return s < 0 ? s + n : (s >= n ? s - n : s); }

// e_i . (x, y, z) from the nonzero components of e_i only.  Under IEEE rules
// 0 * x and 0 + x do not fold away (NaN, signed zero), so the plain dot product
// costs three FMA-pipe instructions per population even for an axis direction;
// with i a constant after unrolling this folds to at most two adds.
template <class L>
__device__ __forceinline__ float edot(int i, float x, float y, float z) {
  const int a = L::ex(i), b = L::ey(i), c = L::ez(i);
  const float X = a > 0 ? x : -x, Y = b > 0 ? y : -y, Z = c > 0 ? z : -z;
  if (a != 0 && b != 0 && c != 0) return X + Y + Z;
  if (a != 0 && b != 0) return X + Y;
  if (a != 0 && c != 0) return X + Z;
  if (b != 0 && c != 0) return Y + Z;
  if (a != 0) return X;
  if (b != 0) return Y;
  if (c != 0) return Z;
  return 0.f;
}

struct FSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
  __device__ __forceinline__ float fvalue() const { return s + c; }
};

}  // namespace lbmd
