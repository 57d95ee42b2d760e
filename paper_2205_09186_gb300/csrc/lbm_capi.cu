// C ABI of the GB300 chemical-potential multiphase LBM library (include/lbm.h).
// Host-side handle management, initialisation kernels, the step loop and the
// observables reduction.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "launch.cuh"
#include "walls.cuh"
#include "compact.cuh"

using namespace lbmd;

struct lbm_handle {
  lbm_params p;
  Mrt mrt{};  // D2Q9 collision operator
  int Q = 0, D = 0, prec = 0;
  long long N = 0;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  bool own_alloc = false;
  void* f[2] = {nullptr, nullptr};
  void* rho[2] = {nullptr, nullptr};  // FP64: density; FP32DEV: float rho - rho_ref
  int cur = 0;
  void* rho_snap = nullptr;
  unsigned long long* d_bad = nullptr;
  double* d_partials = nullptr;
  int n_partials = 0;
  double* d_obs = nullptr;   // 8 doubles, then one packed lbm_obs
  long long t = 0, t_snap = 0;
  KParams kp{};
  StepFn fn = nullptr;
  CompactBufs cb{};
  bool compact = false;
  int zc = 0;  // z-chunk of the pipelined D3Q19 kernel (0 = heuristic)
  void* mu = nullptr;  // mu field of the split D3Q19 FP32DEV path
  signed char* layer = nullptr;  // wall layers (Appendix A): 0 fluid, 1..3, 4 deeper; null: no walls
  void* wmu = nullptr;           // mu field of the wall step (N values of the precision's mu type)
  double mu_w = 0.0;             // wall chemical potential
  alignas(64) unsigned char tmap[2][128];  // D3Q19 FP32DEV: tensor maps (CUtensorMap) of f[0], f[1]
  bool has_tmap = false;
  unsigned long long* qc = nullptr;  // D3Q19 FP32DEV: corner accumulators of the collision pass
  long long n_qc = 0;
  float qscale = 0.f;
  int rpt2d = 0;  // D2Q9 FP32DEV split tiles: rows per thread (0 = default)
};

// ------------------------------------------------------------------ allocation
static void* dalloc(lbm_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  return h->alloc.alloc(bytes, h->alloc.ctx);
}
static void dfree(lbm_handle* h, void* p, size_t bytes) {
  if (p) h->alloc.free(p, bytes == 0 ? 256 : bytes, h->alloc.ctx);
}
static void* cuda_alloc_cb(size_t bytes, void*) {
  void* p = nullptr;
  return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
static void cuda_free_cb(void* p, size_t, void*) { cudaFree(p); }

static size_t f_bytes(const lbm_handle* h) {
  return size_t(h->Q) * size_t(h->N) * (h->p.precision == LBM_FP64 ? sizeof(double) : sizeof(float));
}
static size_t r_bytes(const lbm_handle* h) {
  return size_t(h->N) * (h->p.precision == LBM_FP64 ? sizeof(double) : sizeof(float));
}

// ------------------------------------------------------------------ EOS on the host
// Carnahan-Starling: p0 = rho R T C0(eta) - a rho^2 with eta = b rho / 4 and
// C0 = (1 + eta + eta^2 - eta^3)/(1 - eta)^3.  dp0/drho = R T C1(eta) - 2 a rho,
// C1 = d(eta C0)/d eta = (1 + 4eta + 4eta^2 - 4eta^3 + eta^4)/(1 - eta)^4.
static double cs_c1(double e) {
  const double q = 1.0 - e;
  return (1.0 + e * (4.0 + e * (4.0 + e * (-4.0 + e)))) / (q * q * q * q);
}
static double cs_c1p(double e) {  // d C1 / d eta
  const double q = 1.0 - e;
  const double num = 1.0 + e * (4.0 + e * (4.0 + e * (-4.0 + e)));
  const double dnum = 4.0 + e * (8.0 + e * (-12.0 + 4.0 * e));
  return dnum / (q * q * q * q) + 4.0 * num / (q * q * q * q * q);
}

// Peng-Robinson (Eq. 14-15) with x = b rho, D = 1 + 2x - x^2:
//   p0 = rho R T / (1 - x) - a alpha rho^2 / D,   dp0/drho = R T / (1 - x)^2 - 2 a alpha rho (1 + x) / D^2.
// Critical point (alpha = 1): with h(x) = x^2 / D, p0' = p0'' = 0 give
// 2 h'(x) = (1 - x) h''(x) and R T_c = (a / b) (1 - x)^2 h'(x).
static double pr_hp(double x) {  // h'
  const double D = 1.0 + x * (2.0 - x);
  return 2.0 * x * (1.0 + x) / (D * D);
}
static double pr_hpp(double x) {  // h''
  const double D = 1.0 + x * (2.0 - x);
  return (2.0 * (1.0 + 2.0 * x) * D - 8.0 * x * (1.0 + x) * (1.0 - x)) / (D * D * D);
}
static double pr_kappa(double w) { return 0.37464 + w * (1.54226 - 0.26992 * w); }
static double rks_kappa(double w) { return 0.480 + w * (1.574 - 0.176 * w); }

// van der Waals and Redlich-Kwong-Soave share the repulsive term; their
// attractive terms h(x) = x^2 (VDW) and x^2 / (1 + x) (RKS) give the critical
// point the same way as PR: 2 h'(x) = (1 - x) h''(x), R T_c = (a / b) (1 - x)^2 h'(x).
static double cubic_hp(int kind, double x) {
  if (kind == LBM_EOS_VDW) return 2.0 * x;
  if (kind == LBM_EOS_RKS) return x * (2.0 + x) / ((1.0 + x) * (1.0 + x));
  return pr_hp(x);
}
static double cubic_hpp(int kind, double x) {
  if (kind == LBM_EOS_VDW) return 2.0;
  if (kind == LBM_EOS_RKS) return 2.0 / ((1.0 + x) * (1.0 + x) * (1.0 + x));
  return pr_hpp(x);
}

namespace {
struct HostEos {
  int kind = LBM_EOS_CS;
  double a = 0, b = 0, R = 0, T = 0, aa = 0;  // aa = a alpha(T) (PR)
  double rc = 0, Tc = 0, rmax = 0;

  double p(double rho) const {
    if (kind == LBM_EOS_VDW || kind == LBM_EOS_RKS) {
      const double x = b * rho;
      return rho * R * T / (1.0 - x) - aa * rho * rho / (kind == LBM_EOS_RKS ? 1.0 + x : 1.0);
    }
    if (kind == LBM_EOS_PR) {
      const double x = b * rho;
      return rho * R * T / (1.0 - x) - aa * rho * rho / (1.0 + x * (2.0 - x));
    }
    const double e = 0.25 * b * rho, q = 1.0 - e;
    return rho * R * T * (1.0 + e * (1.0 + e * (1.0 - e))) / (q * q * q) - a * rho * rho;
  }
  double dp(double rho) const {
    if (kind == LBM_EOS_VDW) return R * T / ((1.0 - b * rho) * (1.0 - b * rho)) - 2.0 * aa * rho;
    if (kind == LBM_EOS_RKS) {
      const double x = b * rho;
      return R * T / ((1.0 - x) * (1.0 - x)) - aa * rho * (2.0 + x) / ((1.0 + x) * (1.0 + x));
    }
    if (kind == LBM_EOS_PR) {
      const double x = b * rho, D = 1.0 + x * (2.0 - x);
      return R * T / ((1.0 - x) * (1.0 - x)) - 2.0 * aa * rho * (1.0 + x) / (D * D);
    }
    return R * T * cs_c1(0.25 * b * rho) - 2.0 * a * rho;
  }
  double mu(double rho) const {  // psi'(rho), additive constant dropped
    if (kind == LBM_EOS_VDW || kind == LBM_EOS_RKS) {
      const double x = b * rho, rep = R * T * (std::log(rho / (1.0 - x)) + 1.0 / (1.0 - x));
      if (kind == LBM_EOS_VDW) return rep - 2.0 * aa * rho;
      return rep - aa / b * std::log(1.0 + x) - aa * rho / (1.0 + x);
    }
    if (kind == LBM_EOS_PR) {
      const double x = b * rho, s2 = std::sqrt(2.0);
      return R * T * (std::log(rho / (1.0 - x)) + 1.0 / (1.0 - x)) -
             aa / (2.0 * s2 * b) * std::log((s2 - 1.0 + x) / (s2 + 1.0 - x)) - aa * rho / (1.0 + x * (2.0 - x));
    }
    const double e = 0.25 * b * rho, q = 1.0 - e;
    return R * T * (std::log(rho) + e * (8.0 + e * (-9.0 + 3.0 * e)) / (q * q * q)) - 2.0 * a * rho;
  }
};

int eos_critical(int kind, double a, double b, double R, double* rho_c, double* T_c) {
  if (!(a > 0 && b > 0 && R > 0) || !rho_c || !T_c) return LBM_EINVAL;
  if (kind == LBM_EOS_PR || kind == LBM_EOS_VDW || kind == LBM_EOS_RKS) {
    double lo = 1e-8, hi = 0.9;
    for (int it = 0; it < 200; ++it) {
      const double m = 0.5 * (lo + hi);
      if ((1.0 - m) * cubic_hpp(kind, m) - 2.0 * cubic_hp(kind, m) > 0) lo = m; else hi = m;
    }
    const double x = 0.5 * (lo + hi);
    *rho_c = x / b;
    *T_c = (a / b) * (1.0 - x) * (1.0 - x) * cubic_hp(kind, x) / R;
    return LBM_OK;
  }
  if (kind != LBM_EOS_CS) return LBM_EINVAL;
  // dp0/drho = 0 and d2p0/drho2 = 0  <=>  C1(eta) = eta C1'(eta);  R T_c = 8 a / (b C1'(eta_c))
  double lo = 1e-8, hi = 0.5;
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (lo + hi);
    if (cs_c1(m) - m * cs_c1p(m) > 0) lo = m; else hi = m;
  }
  const double e = 0.5 * (lo + hi);
  *rho_c = 4.0 * e / b;
  *T_c = 8.0 * a / (b * R * cs_c1p(e));
  return LBM_OK;
}

int make_eos(const lbm_params* p, HostEos* e) {
  if (!p || p->eos < LBM_EOS_CS || p->eos > LBM_EOS_RKS) return LBM_EINVAL;
  if (eos_critical(p->eos, p->a, p->b, p->R, &e->rc, &e->Tc) != LBM_OK) return LBM_EINVAL;
  e->kind = p->eos; e->a = p->a; e->b = p->b; e->R = p->R; e->T = p->Tr * e->Tc;
  if (p->eos == LBM_EOS_PR || p->eos == LBM_EOS_RKS) {
    const double kap = p->eos == LBM_EOS_PR ? pr_kappa(p->acentric) : rks_kappa(p->acentric);
    const double s = 1.0 + kap * (1.0 - std::sqrt(p->Tr));
    e->aa = p->a * s * s;
    e->rmax = 1.0 / p->b;
  } else if (p->eos == LBM_EOS_VDW) {
    e->aa = p->a;
    e->rmax = 1.0 / p->b;
  } else {
    e->aa = p->a;
    e->rmax = 4.0 / p->b;
  }
  return LBM_OK;
}

// Coexistence by bisection on the common chemical potential m: on the gas
// branch (0, spinodal_g) and the liquid branch (spinodal_l, rho_max) mu is
// increasing in rho, so each branch has one root of mu = m; by Gibbs-Duhem
// (dp = rho dmu) p_gas(m) - p_liq(m) decreases with m, which brackets the
// equal-pressure level.
int maxwell_eos(const HostEos& E, double* rg, double* rl) {
  const double rc = E.rc;
  if (!(E.T > 0 && E.T < E.Tc)) return LBM_EINVAL;
  double lo = std::log(rc) - 800.0, hi = std::log(rc);  // ln rho on the gas side
  for (int it = 0; it < 400; ++it) {
    const double m = 0.5 * (lo + hi);
    if (E.dp(std::exp(m)) > 0) lo = m; else hi = m;
  }
  const double sg = std::exp(lo);
  lo = rc; hi = E.rmax;
  for (int it = 0; it < 400; ++it) {
    const double m = 0.5 * (lo + hi);
    if (E.dp(m) < 0) lo = m; else hi = m;
  }
  const double sl = hi;
  auto gas = [&](double m) {
    double l = std::log(rc) - 800.0, u = std::log(sg);
    for (int it = 0; it < 400; ++it) {
      const double c = 0.5 * (l + u);
      if (E.mu(std::exp(c)) < m) l = c; else u = c;
    }
    return std::exp(0.5 * (l + u));
  };
  auto liq = [&](double m) {
    double l = sl, u = E.rmax;
    for (int it = 0; it < 400; ++it) {
      const double c = 0.5 * (l + u);
      if (E.mu(c) < m) l = c; else u = c;
    }
    return 0.5 * (l + u);
  };
  double mlo = E.mu(sl), mhi = E.mu(sg);
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (mlo + mhi);
    const double g = gas(m), l = liq(m);
    if (E.p(g) - E.p(l) > 0) mlo = m; else mhi = m;
    if (mhi - mlo <= 1e-17 * std::fabs(m)) break;
  }
  const double m = 0.5 * (mlo + mhi);
  *rg = gas(m);
  *rl = liq(m);
  return LBM_OK;
}
}  // namespace

int lbmd::params_to_kp(const lbm_params* p, KParams* kp) {
  HostEos E;
  if (make_eos(p, &E) != LBM_OK) return LBM_EINVAL;
  *kp = KParams{};
  kp->nx = p->nx; kp->ny = p->ny; kp->nz = p->nz;
  kp->n = (long long)p->nx * p->ny * p->nz;
  kp->RT = p->R * E.T; kp->b4 = 0.25 * p->b; kp->two_a = 2.0 * p->a;
  kp->eos = p->eos;  // the device codes equal the LBM_EOS_ values
  kp->aa = E.aa;
  kp->c1 = p->eos == LBM_EOS_PR ? E.aa / (2.0 * std::sqrt(2.0) * p->b) : (p->eos == LBM_EOS_RKS ? E.aa / p->b : 0.0);
  kp->k2 = p->k * p->k; kp->kappa = p->kappa; kp->omega = 1.0 / p->tau;
  kp->rho_ref = 0.0;
  if (p->precision == LBM_FP32DEV) {
    kp->rho_ref = p->rho_ref;
    if (!(kp->rho_ref > 0)) {
      double g, l;
      if (maxwell_eos(E, &g, &l) != LBM_OK) return LBM_EINVAL;
      kp->rho_ref = g;
    }
  }
  return LBM_OK;
}

extern "C" int lbm_critical(double a, double b, double R, double* rho_c, double* T_c) {
  return eos_critical(LBM_EOS_CS, a, b, R, rho_c, T_c);
}

extern "C" int lbm_eos_critical(const lbm_params* p, double* rho_c, double* T_c) {
  if (!p) return LBM_EINVAL;
  return eos_critical(p->eos, p->a, p->b, p->R, rho_c, T_c);
}

extern "C" int lbm_maxwell(const lbm_params* p, double* rho_g, double* rho_l) {
  if (!p || !rho_g || !rho_l) return LBM_EINVAL;
  HostEos E;
  if (make_eos(p, &E) != LBM_OK) return LBM_EINVAL;
  return maxwell_eos(E, rho_g, rho_l);
}

extern "C" int lbm_bulk_mu(const lbm_params* p, double rho, double* mu) {
  if (!p || !mu || !(rho > 0)) return LBM_EINVAL;
  HostEos E;
  if (make_eos(p, &E) != LBM_OK) return LBM_EINVAL;
  if (E.kind != LBM_EOS_CS && !(E.b * rho < 1.0)) return LBM_EINVAL;
  if (E.kind == LBM_EOS_CS && !(0.25 * E.b * rho < 1.0)) return LBM_EINVAL;
  *mu = p->k * p->k * E.mu(rho);
  return LBM_OK;
}

extern "C" int lbm_lattice_q(int lattice) { return lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q19 ? 19 : 0); }

extern "C" const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "device allocation failed";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_EUNSTABLE: return "simulation unstable (non-positive or NaN density)";
    case LBM_ETIMEOUT: return "device-side wait timed out";
    case LBM_ENOTSUP: return "unsupported lattice/scheme combination";
    case LBM_ESCRATCH: return "lattice too large for the fixed scratch array of the non-allocating entry point";
    default: return "unknown error";
  }
}

// ------------------------------------------------------------------ kernels
namespace {

__constant__ double c_w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
__constant__ double c_w19[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

__constant__ float c_w9f[9] = {4.f / 9, 1.f / 9, 1.f / 9, 1.f / 9, 1.f / 9, 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36};
__constant__ float c_w19f[19] = {1.f / 3,  1.f / 18, 1.f / 18, 1.f / 18, 1.f / 18, 1.f / 18, 1.f / 18,
                                 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36,
                                 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36, 1.f / 36};

struct InitSpec {
  int kind;  // 0 droplet, 1 slab, 2 radial profile, 3 density array
  double cx, cy, cz, radius, width, rho_l, rho_g;
  int axis;
  const double* r;
  const double* prof;
  int nprof;
  const double* dens;
};

__device__ double init_density(const InitSpec& s, int x, int y, int z, long long node) {
  if (s.kind == 3) return s.dens[node];
  if (s.kind == 1) {
    const double c = s.axis == 0 ? x - s.cx : (s.axis == 1 ? y - s.cy : z - s.cz);
    return 0.5 * (s.rho_l + s.rho_g) - 0.5 * (s.rho_l - s.rho_g) * tanh(2.0 * (fabs(c) - 0.5 * s.radius) / s.width);
  }
  const double dx = x - s.cx, dy = y - s.cy, dz = z - s.cz;
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  if (s.kind == 0) return 0.5 * (s.rho_l + s.rho_g) - 0.5 * (s.rho_l - s.rho_g) * tanh(2.0 * (r - s.radius) / s.width);
  // radial profile, linear interpolation
  if (r <= s.r[0]) return s.prof[0];
  if (r >= s.r[s.nprof - 1]) return s.prof[s.nprof - 1];
  int lo = 0, hi = s.nprof - 1;
  while (hi - lo > 1) {
    const int m = (lo + hi) / 2;
    if (s.r[m] < r) lo = m; else hi = m;
  }
  const double t = (r - s.r[lo]) / (s.r[hi] - s.r[lo]);
  return s.prof[lo] + t * (s.prof[hi] - s.prof[lo]);
}

// f_i = w_i rho0 (u = 0); the density field is the sum of the stored populations
// (Q a template parameter: the population loop unrolls, its weights and
// population offsets become constants)
template <typename Tf, int Q>
__global__ void k_init(KParams p, InitSpec s, Tf* f, Tf* rho) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  // (a density array needs no coordinates: skip the 64-bit divisions)
  const int x = s.kind == 3 ? 0 : int(n % p.nx), y = s.kind == 3 ? 0 : int((n / p.nx) % p.ny);
  const int z = s.kind == 3 ? 0 : int(n / ((long long)p.nx * p.ny));
  const double r0 = init_density(s, x, y, z, n);
  Tf* fn = f + n;
  if constexpr (sizeof(Tf) == 8) {
    const double* w = Q == 9 ? c_w9 : c_w19;
    double acc = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double fi = w[i] * r0;
      fn[i * p.n] = Tf(fi);
      acc += fi;
    }
    rho[n] = acc;
  } else {
    // the deviation once in FP64, the Q weighted copies in FP32 (FP64 runs at
    // a small fraction of the FP32 rate on this GPU)
    const float dv = float(r0 - p.rho_ref);
    const float* w = Q == 9 ? c_w9f : c_w19f;
    FSum acc;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float d = w[i] * dv;
      fn[i * p.n] = d;
      acc.add(d);
    }
    rho[n] = acc.fvalue();
  }
}

// density field from the stored populations
template <typename Tf>
__global__ void k_density(KParams p, int Q, const Tf* f, Tf* rho) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  if constexpr (sizeof(Tf) == 8) {
    double acc = 0;
    for (int i = 0; i < Q; ++i) acc += double(f[i * p.n + n]);
    rho[n] = acc;
  } else {
    FSum acc;
    for (int i = 0; i < Q; ++i) acc.add(float(f[i * p.n + n]));
    rho[n] = acc.fvalue();
  }
}

// density field (stored form) -> FP64 full density
template <typename Tr>
__global__ void k_export_rho(KParams p, const Tr* r, double* out) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  out[n] = sizeof(Tr) == 8 ? double(r[n]) : p.rho_ref + double(r[n]);
}

// full FP64 populations <-> stored form
template <typename Tf>
__global__ void k_export_f(KParams p, int Q, const Tf* f, double* out) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  const double* w = Q == 9 ? c_w9 : c_w19;
  for (int i = 0; i < Q; ++i) out[i * p.n + n] = double(f[i * p.n + n]) + (sizeof(Tf) == 8 ? 0.0 : w[i] * p.rho_ref);
}
template <typename Tf>
__global__ void k_import_f(KParams p, int Q, const double* in, Tf* f) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  const double* w = Q == 9 ? c_w9 : c_w19;
  for (int i = 0; i < Q; ++i) f[i * p.n + n] = Tf(in[i * p.n + n] - (sizeof(Tf) == 8 ? 0.0 : w[i] * p.rho_ref));
}

// final reduction of per-CTA observables, fixed order (deterministic)
// rec (optional): the same as a complete lbm_obs of the state of step t_obs,
// max |d rho / dt| over dt steps (0: none)
template <typename Tr>
__global__ void k_obs_final(const double* part, int nb, const Tr* rho, double rho_ref, long long center,
                            const unsigned long long* bad, double* out, lbm_obs* rec, long long t_obs, long long dt) {
  __shared__ double red[4][256];
  double a = 0, b = 0, c = 0, d = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a = fmax(a, part[4 * i]);
    b = fmax(b, part[4 * i + 1]);
    c += part[4 * i + 2];
    d = fmax(d, part[4 * i + 3]);
  }
  red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c; red[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0]; out[1] = red[1][0]; out[2] = red[2][0]; out[3] = red[3][0];
    out[4] = sizeof(Tr) == 8 ? double(rho[center]) : rho_ref + double(rho[center]);
    out[5] = sizeof(Tr) == 8 ? double(rho[0]) : rho_ref + double(rho[0]);
    unsigned long long bs = *bad;
    reinterpret_cast<unsigned long long*>(out)[6] = bs;
    if (rec) {
      rec->max_v = out[0];
      rec->max_u = out[1];
      rec->mass = out[2];
      rec->max_drho = dt > 0 ? out[3] / double(dt) : 0.0;
      rec->rho_center = out[4];
      rec->rho_corner = out[5];
      rec->step = bs != ~0ULL ? (long long)bs : t_obs;
      rec->status = bs != ~0ULL ? LBM_EUNSTABLE : LBM_OK;
    }
  }
}

inline unsigned grid1(long long n, int bs) { return unsigned((n + bs - 1) / bs); }

}  // namespace

namespace lbmd {

cudaError_t ensure_smem(const void* fn, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;  // (device, kernel) -> limit set
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({dev, fn});
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) done[{dev, fn}] = bytes;
  return e;
}

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  static std::mutex mu;
  static std::map<int, int> sms;
  std::lock_guard<std::mutex> lock(mu);
  auto it = sms.find(dev);
  if (it != sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  sms[dev] = n;
  return n;
}

}  // namespace lbmd

static int ck(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

// ------------------------------------------------------------------ create/destroy
extern "C" void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  dfree(h, h->f[0], f_bytes(h));
  dfree(h, h->f[1], f_bytes(h));
  dfree(h, h->rho[0], r_bytes(h));
  dfree(h, h->rho[1], r_bytes(h));
  dfree(h, h->rho_snap, r_bytes(h));
  dfree(h, h->d_bad, 8);
  dfree(h, h->d_partials, size_t(h->n_partials) * 4 * 8);
  dfree(h, h->d_obs, 64 + sizeof(lbm_obs));
  dfree(h, h->mu, size_t(h->N) * 4);
  dfree(h, h->qc, size_t(h->n_qc) * 8);
  dfree(h, h->layer, size_t(h->N));
  dfree(h, h->wmu, size_t(h->N) * 8);
  compact_free(h->cb, [&](void* p, size_t b) { dfree(h, p, b); });
  delete h;
}

static int validate(const lbm_params* p) {
  if (!p) return LBM_EINVAL;
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return LBM_EINVAL;
  if (p->nx < 8 || p->ny < 8) return LBM_EINVAL;
  if (p->lattice == LBM_D2Q9 && p->nz != 1) return LBM_EINVAL;
  if (p->lattice == LBM_D3Q19 && p->nz < 8) return LBM_EINVAL;
  if ((long long)p->nx * p->ny * p->nz > (1LL << 31) / 19) return LBM_EINVAL;
  if (p->eos < LBM_EOS_CS || p->eos > LBM_EOS_RKS) return LBM_EINVAL;
  if ((p->eos == LBM_EOS_PR || p->eos == LBM_EOS_RKS) && !(p->Tr < 1.0 && p->acentric > -1.0)) return LBM_EINVAL;
  if (!(p->a > 0 && p->b > 0 && p->R > 0 && p->Tr > 0)) return LBM_EINVAL;
  if (!(p->k > 0) || !(p->kappa >= 0) || !(p->tau > 0.5)) return LBM_EINVAL;
  if (p->scheme < LBM_EFDS2 || p->scheme > LBM_E8) return LBM_EINVAL;
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32DEV) return LBM_EINVAL;
  if (p->scheme == LBM_E8 && p->lattice != LBM_D2Q9) return LBM_ENOTSUP;
  if (p->collision != LBM_BGK && p->collision != LBM_MRT) return LBM_EINVAL;
  if (p->collision == LBM_MRT && p->lattice != LBM_D2Q9) return LBM_ENOTSUP;
  return LBM_OK;
}

extern "C" int lbm_create(const lbm_params* params, void* stream, const lbm_allocator* alloc, lbm_handle** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  int rc = validate(params);
  if (rc != LBM_OK) return rc;
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return LBM_ENOMEM;
  h->p = *params;
  h->Q = lbm_lattice_q(params->lattice);
  h->D = params->lattice == LBM_D2Q9 ? 2 : 3;
  h->N = (long long)params->nx * params->ny * params->nz;
  h->stream = static_cast<cudaStream_t>(stream);
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
  } else {
    h->alloc.alloc = cuda_alloc_cb;
    h->alloc.free = cuda_free_cb;
    h->alloc.ctx = nullptr;
    h->own_alloc = true;
  }
  if (params_to_kp(params, &h->kp) != LBM_OK) { delete h; return LBM_EINVAL; }
  const double rho_ref = h->kp.rho_ref;
  h->prec = params->precision == LBM_FP64 ? 0 : (params->mu_fp64 ? 2 : 1);
  h->mrt = make_mrt(params->collision == LBM_MRT, params->mrt_s, params->tau);
  h->compact = (params->scheme >= LBM_CFDS4 && params->scheme <= LBM_OCFDS4);
  h->p.rho_ref = rho_ref;
  if (h->compact) {
    h->fn = nullptr;
  } else {
    h->fn = h->D == 2 ? step2d_fn(params->scheme, h->prec) : step3d_fn(params->scheme, h->prec);
    if (!h->fn) { delete h; return LBM_ENOTSUP; }
  }
  const size_t fb = f_bytes(h);
  h->f[0] = dalloc(h, fb);
  h->f[1] = dalloc(h, fb);
  h->rho[0] = dalloc(h, r_bytes(h));
  h->rho[1] = dalloc(h, r_bytes(h));
  h->rho_snap = dalloc(h, r_bytes(h));
  h->d_bad = static_cast<unsigned long long*>(dalloc(h, 8));
  h->d_obs = static_cast<double*>(dalloc(h, 64 + sizeof(lbm_obs)));
  // partials: one per CTA of the observation pass (upper bound over tilings used)
  h->n_partials = int((params->nx / 8 + 2) * (params->ny / 8 + 2) * (params->lattice == LBM_D2Q9 ? 1 : (params->nz / 8 + 2)));
  // the node-parallel observation pass of the split D3Q19 path uses up to 8 CTAs per SM
  if (h->n_partials < 8 * 1024) h->n_partials = 8 * 1024;
  h->d_partials = static_cast<double*>(dalloc(h, size_t(h->n_partials) * 4 * 8));
  bool ok = h->f[0] && h->f[1] && h->rho[0] && h->rho[1] && h->rho_snap && h->d_bad && h->d_obs && h->d_partials;
  if (ok && !h->compact &&
      (h->D == 3 ? split3d_scheme(params->scheme, h->prec) : split2d_scheme(params->scheme, h->prec))) {
    h->mu = dalloc(h, size_t(h->N) * 4);
    ok = h->mu != nullptr;
  }
  // tensor maps of both population buffers for the D3Q19 FP32DEV collision
  // pass's copies (split explicit schemes and compact schemes)
  if (ok && h->D == 3 && (h->prec == 1 || h->prec == 2)) {
    h->has_tmap = make_coll3d_tmap(h->f[0], h->kp, h->tmap[0]) && make_coll3d_tmap(h->f[1], h->kp, h->tmap[1]);
    // corner accumulators of the tiled collision pass (zero between passes)
    h->n_qc = coll3d_corner_count(h->kp);
    h->qscale = coll3d_corner_scale(params->eos, params->b);
    h->qc = static_cast<unsigned long long*>(dalloc(h, size_t(h->n_qc) * 8));
    ok = h->qc != nullptr && cudaMemsetAsync(h->qc, 0, size_t(h->n_qc) * 8, h->stream) == cudaSuccess;
  }
  if (ok && h->compact) {
    rc = compact_alloc(h->cb, h->kp, h->D, params->scheme, h->prec, [&](size_t b) { return dalloc(h, b); });
    if (rc != LBM_OK) ok = false;
  }
  if (!ok) {
    lbm_destroy(h);
    return LBM_ENOMEM;
  }
  unsigned long long init = ULLONG_MAX;
  if (cudaMemcpyAsync(h->d_bad, &init, 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    lbm_destroy(h);
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

// ------------------------------------------------------------------ init
static int run_init(lbm_handle* h, const InitSpec& s) {
  const int bs = 256;
  double* fd = static_cast<double*>(h->f[0]);
  double* rd = static_cast<double*>(h->rho[0]);
  float* ff = static_cast<float*>(h->f[0]);
  float* rf = static_cast<float*>(h->rho[0]);
  if (h->p.precision == LBM_FP64) {
    if (h->Q == 9) k_init<double, 9><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, s, fd, rd);
    else k_init<double, 19><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, s, fd, rd);
  } else {
    if (h->Q == 9) k_init<float, 9><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, s, ff, rf);
    else k_init<float, 19><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, s, ff, rf);
  }
  h->cur = 0;
  h->t = 0;
  h->t_snap = 0;
  unsigned long long init = ULLONG_MAX;
  if (cudaMemcpyAsync(h->d_bad, &init, 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return LBM_ECUDA;
  if (cudaMemcpyAsync(h->rho_snap, h->rho[0], r_bytes(h), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return LBM_ECUDA;
  // host arrays referenced by the spec must outlive the kernel: synchronise
  return ck(cudaStreamSynchronize(h->stream));
}

static int default_dens(lbm_handle* h, double& rl, double& rg) {
  if (rl > 0 && rg > 0) return LBM_OK;
  double g, l;
  if (lbm_maxwell(&h->p, &g, &l) != LBM_OK) return LBM_EINVAL;
  rl = l;
  rg = g;
  return LBM_OK;
}

static void set_center(lbm_handle* h, InitSpec& s, const double* c) {
  s.cx = c ? c[0] : double(h->p.nx / 2);
  s.cy = c ? c[1] : double(h->p.ny / 2);
  s.cz = c ? c[2] : double(h->p.nz / 2);
  if (h->D == 2) s.cz = 0;
}

extern "C" int lbm_init_droplet(lbm_handle* h, const double center[3], double radius, double width, double rho_l,
                                double rho_g) {
  if (!h || !(width > 0) || !(radius >= 0)) return LBM_EINVAL;
  if (default_dens(h, rho_l, rho_g) != LBM_OK) return LBM_EINVAL;
  InitSpec s{};
  s.kind = 0;
  set_center(h, s, center);
  s.radius = radius; s.width = width; s.rho_l = rho_l; s.rho_g = rho_g;
  return run_init(h, s);
}

extern "C" int lbm_init_slab(lbm_handle* h, int axis, double thickness, double width, double rho_l, double rho_g) {
  if (!h || axis < 0 || axis >= h->D || !(width > 0) || !(thickness >= 0)) return LBM_EINVAL;
  if (default_dens(h, rho_l, rho_g) != LBM_OK) return LBM_EINVAL;
  InitSpec s{};
  s.kind = 1;
  s.axis = axis;
  set_center(h, s, nullptr);
  s.radius = thickness; s.width = width; s.rho_l = rho_l; s.rho_g = rho_g;
  return run_init(h, s);
}

extern "C" int lbm_init_profile(lbm_handle* h, const double center[3], const double* r, const double* rho, int n) {
  if (!h || !r || !rho || n < 2) return LBM_EINVAL;
  for (int j = 0; j < n; ++j) {
    if (!(rho[j] > 0)) return LBM_EINVAL;
    if (j > 0 && !(r[j] > r[j - 1])) return LBM_EINVAL;
  }
  double* d = static_cast<double*>(dalloc(h, size_t(2 * n) * 8));
  if (!d) return LBM_ENOMEM;
  int rc = ck(cudaMemcpyAsync(d, r, size_t(n) * 8, cudaMemcpyHostToDevice, h->stream));
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(d + n, rho, size_t(n) * 8, cudaMemcpyHostToDevice, h->stream));
  if (rc == LBM_OK) {
    InitSpec s{};
    s.kind = 2;
    set_center(h, s, center);
    s.r = d; s.prof = d + n; s.nprof = n;
    rc = run_init(h, s);
  }
  cudaStreamSynchronize(h->stream);
  dfree(h, d, size_t(2 * n) * 8);
  return rc;
}

extern "C" int lbm_init_density(lbm_handle* h, const double* host_rho) {
  if (!h || !host_rho) return LBM_EINVAL;
  double* tmp = static_cast<double*>(dalloc(h, size_t(h->N) * 8));
  if (!tmp) return LBM_ENOMEM;
  int rc = ck(cudaMemcpyAsync(tmp, host_rho, h->N * 8, cudaMemcpyHostToDevice, h->stream));
  if (rc == LBM_OK) {
    InitSpec s{};
    s.kind = 3;
    s.dens = tmp;
    rc = run_init(h, s);
  }
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, size_t(h->N) * 8);
  return rc;
}

extern "C" int lbm_set_f(lbm_handle* h, const double* host_f) {
  if (!h || !host_f) return LBM_EINVAL;
  const size_t bytes = size_t(h->Q) * h->N * 8;
  double* tmp = static_cast<double*>(dalloc(h, bytes));
  if (!tmp) return LBM_ENOMEM;
  int rc = ck(cudaMemcpyAsync(tmp, host_f, bytes, cudaMemcpyHostToDevice, h->stream));
  const int bs = 256;
  if (rc == LBM_OK) {
    h->cur = 0;
    if (h->p.precision == LBM_FP64) {
      k_import_f<double><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, tmp, static_cast<double*>(h->f[0]));
      k_density<double><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, static_cast<double*>(h->f[0]),
                                                               static_cast<double*>(h->rho[0]));
    } else {
      k_import_f<float><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, tmp, static_cast<float*>(h->f[0]));
      k_density<float><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, static_cast<float*>(h->f[0]),
                                                              static_cast<float*>(h->rho[0]));
    }
    rc = ck(cudaGetLastError());
  }
  h->t = 0;
  h->t_snap = 0;
  unsigned long long init = ULLONG_MAX;
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(h->d_bad, &init, 8, cudaMemcpyHostToDevice, h->stream));
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(h->rho_snap, h->rho[0], r_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, bytes);
  return rc;
}

// ------------------------------------------------------------------ stepping
static Launch make_launch(lbm_handle* h, int out_buf) {
  Launch c{};
  c.kp = h->kp;
  c.fin = h->f[h->cur];
  c.fout = h->f[out_buf];
  c.rin = h->rho[h->cur];
  c.rout = h->rho[out_buf];
  c.aux.t = h->t;
  c.aux.bad_step = h->d_bad;
  c.aux.partials = h->d_partials;
  c.aux.rho_snap = h->rho_snap;
  c.stream = h->stream;
  c.zc = h->zc;
  c.mu = h->mu;
  c.mrt = h->mrt;
  c.tmap = h->has_tmap ? h->tmap[h->cur] : nullptr;
  c.rpt2d = h->rpt2d;
  c.qc = h->qc;
  c.qscale = h->qscale;
  return c;
}

// one pass of the handle's step: walls, compact line schemes or the fused kernels
static cudaError_t run_pass(lbm_handle* h, const Launch& c, int mode, int* nb) {
  if (h->layer) {
    WallLaunch w{c, h->layer, h->mu_w, h->wmu};
    return wall_step(w, h->D == 2 ? 0 : 1, h->p.scheme, h->prec, mode, nb);
  }
  if (h->compact) return compact_step(h->cb, c, h->D, h->p.scheme, h->prec, mode, nb);
  return h->fn(c, mode, nb);
}

// handles whose D3Q19 collision pass marches z-chunks: the explicit FP32DEV
// schemes, and the compact ones with FP32 mu (the tiled pass reading the
// derivative fields)
static bool tunable(const lbm_handle* h) {
  if (h->D != 3 || h->layer) return false;
  if (h->compact) return h->prec == 1 && h->has_tmap;
  return (h->prec == 1 || (h->prec == 2 && h->mu)) &&
         (h->p.scheme == LBM_EFDS2 || h->p.scheme == LBM_EFDS4 || h->p.scheme == LBM_EFDS6 || h->p.scheme == LBM_E4);
}

extern "C" int lbm_set_zchunk(lbm_handle* h, int zc) {
  if (!h || zc < 0) return LBM_EINVAL;
  h->zc = zc > h->p.nz ? h->p.nz : zc;
  return LBM_OK;
}

extern "C" int lbm_set_tile_rows(lbm_handle* h, int rows) {
  if (!h || (rows != 0 && rows != 1 && rows != 2 && rows != 4)) return LBM_EINVAL;
  h->rpt2d = rows;
  return LBM_OK;
}

// the D2Q9 FP32DEV split step runs on tiles of 16 x rows-per-thread rows
static bool tunable2d(const lbm_handle* h) { return h->D == 2 && h->prec == 1 && h->mu && !h->compact && !h->layer; }

extern "C" int lbm_autotune(lbm_handle* h, int* zc_out) {
  if (!h) return LBM_EINVAL;
  if (zc_out) *zc_out = 0;
  if (tunable2d(h)) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LBM_ECUDA; }
    const long long t_saved = h->t;
    // three interleaved rounds, each shape's fastest counting (shapes a few
    // percent apart, and small lattices' short steps, are otherwise ordered by noise)
    const int shapes[3] = {1, 2, 4};
    float shape_ms[3] = {1e30f, 1e30f, 1e30f};
    int rc = LBM_OK;
    for (int round = 0; round < 3 && rc == LBM_OK; ++round) {
      for (int j = 0; j < 3; ++j) {
        h->rpt2d = shapes[j];
        if ((rc = lbm_step(h, 2)) != LBM_OK) break;  // warm up
        cudaEventRecord(e0, h->stream);
        if ((rc = lbm_step(h, 10)) != LBM_OK) break;
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = LBM_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        shape_ms[j] = std::min(shape_ms[j], ms);
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = 0;
    float best_ms = 1e30f;
    for (int j = 0; j < 3; ++j)
      if (shape_ms[j] < best_ms) { best_ms = shape_ms[j]; best = shapes[j]; }
    h->t = t_saved;
    h->rpt2d = best;
    if (zc_out) *zc_out = best;
    return rc != LBM_OK ? rc : (best > 0 ? LBM_OK : LBM_ECUDA);
  }
  if (!tunable(h)) return LBM_OK;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LBM_ECUDA;
  const long long t_saved = h->t;
  int prev = 0, best_zc = 0;
  float best = 1e30f;
  for (int nzc = 1; nzc <= 32 && nzc <= h->p.nz; ++nzc) {
    const int zc = (h->p.nz + nzc - 1) / nzc;
    if (zc == prev || (zc < 4 && nzc > 1)) continue;
    prev = zc;
    h->zc = zc;
    if (lbm_step(h, 1) != LBM_OK) break;
    cudaEventRecord(e0, h->stream);
    if (lbm_step(h, 3) != LBM_OK) break;
    cudaEventRecord(e1, h->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_zc = zc; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->t = t_saved;
  h->zc = best_zc;
  if (zc_out) *zc_out = best_zc;
  return best_zc > 0 ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_step(lbm_handle* h, long long n) {
  if (!h || n < 0) return LBM_EINVAL;
  for (long long s = 0; s < n; ++s) {
    Launch c = make_launch(h, 1 - h->cur);
    if (run_pass(h, c, MODE_STEP, nullptr) != cudaSuccess) return LBM_ECUDA;
    h->cur = 1 - h->cur;
    h->t += 1;
  }
  // wall densities of the state left behind (the next step refreshes them anyway)
  if (h->layer && n > 0 && run_pass(h, make_launch(h, h->cur), MODE_WALL_FILL, nullptr) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}

extern "C" long long lbm_get_step(const lbm_handle* h) { return h ? h->t : -1; }

extern "C" int lbm_step_timed(lbm_handle* h, long long n, double* ms) {
  if (!h || n < 0 || n > 100000 || !ms) return LBM_EINVAL;
  ms[0] = ms[1] = ms[2] = 0.0;
  const bool split = h->mu != nullptr && !h->layer;
  // three events per step, recorded back to back; one synchronisation at the end
  const size_t ne = size_t(3 * n);
  cudaEvent_t* e = new (std::nothrow) cudaEvent_t[ne > 0 ? ne : 1];
  if (!e) return LBM_ENOMEM;
  size_t made = 0;
  int rc = LBM_OK;
  for (; made < ne; ++made)
    if (cudaEventCreate(&e[made]) != cudaSuccess) { rc = LBM_ECUDA; break; }
  for (long long s = 0; s < n && rc == LBM_OK; ++s) {
    Launch c = make_launch(h, 1 - h->cur);
    c.ev_mid = split ? e[3 * s + 1] : nullptr;
    cudaEventRecord(e[3 * s], h->stream);
    cudaError_t err = run_pass(h, c, MODE_STEP, nullptr);
    cudaEventRecord(e[3 * s + 2], h->stream);
    if (err != cudaSuccess) rc = LBM_ECUDA;
    h->cur = 1 - h->cur;
    h->t += 1;
  }
  if (rc == LBM_OK && n > 0 && cudaEventSynchronize(e[3 * n - 1]) != cudaSuccess) rc = LBM_ECUDA;
  for (long long s = 0; s < n && rc == LBM_OK; ++s) {
    float a = 0.f, b = 0.f;
    if (split) {
      cudaEventElapsedTime(&a, e[3 * s], e[3 * s + 1]);
      cudaEventElapsedTime(&b, e[3 * s + 1], e[3 * s + 2]);
    } else {
      cudaEventElapsedTime(&b, e[3 * s], e[3 * s + 2]);
    }
    ms[0] += a;
    ms[1] += b;
    ms[2] += a + b;
  }
  for (size_t k = 0; k < made; ++k) cudaEventDestroy(e[k]);
  delete[] e;
  return rc;
}

// reduce nb per-CTA partials, read the result (and the density at the centre
// and corner nodes of rho_obs) back, fill out for the state of step t_obs.
// async: the record is packed on the device and copied to out by the stream
// (no synchronisation; out valid once the stream has been synchronised).
static int finish_observables(lbm_handle* h, int nb, const void* rho_obs, long long t_obs, lbm_obs* out,
                              bool async = false) {
  if (nb > h->n_partials) return LBM_ECUDA;
  const long long center =
      (long long)(h->p.nz / 2) * h->p.nx * h->p.ny + (long long)(h->p.ny / 2) * h->p.nx + h->p.nx / 2;
  lbm_obs* rec = async ? reinterpret_cast<lbm_obs*>(h->d_obs + 8) : nullptr;
  const long long dt = t_obs > h->t_snap ? t_obs - h->t_snap : 0;
  if (h->p.precision == LBM_FP64)
    k_obs_final<double><<<1, 256, 0, h->stream>>>(h->d_partials, nb, static_cast<const double*>(rho_obs), 0.0, center,
                                                  h->d_bad, h->d_obs, rec, t_obs, dt);
  else
    k_obs_final<float><<<1, 256, 0, h->stream>>>(h->d_partials, nb, static_cast<const float*>(rho_obs),
                                                 h->kp.rho_ref, center, h->d_bad, h->d_obs, rec, t_obs, dt);
  if (async) {
    h->t_snap = t_obs;
    return ck(cudaMemcpyAsync(out, rec, sizeof(lbm_obs), cudaMemcpyDefault, h->stream));
  }
  double host[8];
  if (cudaMemcpyAsync(host, h->d_obs, 64, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return LBM_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
  unsigned long long bad;
  std::memcpy(&bad, &host[6], 8);
  out->max_v = host[0];
  out->max_u = host[1];
  out->mass = host[2];
  out->max_drho = t_obs > h->t_snap ? host[3] / double(t_obs - h->t_snap) : 0.0;
  out->rho_center = host[4];
  out->rho_corner = host[5];
  out->step = t_obs;
  out->status = LBM_OK;
  h->t_snap = t_obs;
  if (bad != ULLONG_MAX) {
    out->status = LBM_EUNSTABLE;
    out->step = (long long)bad;
    return LBM_EUNSTABLE;
  }
  return LBM_OK;
}

static int observe_impl(lbm_handle* h, lbm_obs* out, bool async) {
  Launch c = make_launch(h, h->cur);
  c.fout = nullptr;
  c.rout = nullptr;
  int nb = 0;
  cudaError_t e = run_pass(h, c, MODE_OBS, &nb);
  if (e != cudaSuccess) return LBM_ECUDA;
  if (nb > h->n_partials) return LBM_ECUDA;
  // the snapshot for the next max |d rho / dt|, ordered after the reduction
  if (cudaMemcpyAsync(h->rho_snap, h->rho[h->cur], r_bytes(h), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return LBM_ECUDA;
  return finish_observables(h, nb, h->rho[h->cur], h->t, out, async);
}

extern "C" int lbm_observables(lbm_handle* h, lbm_obs* out) {
  if (!h || !out) return LBM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  return observe_impl(h, out, false);
}

static int step_observe_impl(lbm_handle* h, long long n, lbm_obs* out, bool async) {
  int rc = lbm_step(h, n - 1);
  if (rc != LBM_OK) return rc;
  if (h->D == 3 && h->mu && !h->compact && !h->layer) {
    // the last step reduces the observables of the state it advances and
    // leaves that state's density in the snapshot
    Launch c = make_launch(h, 1 - h->cur);
    int nb = h->n_partials;  // capacity in, CTAs out
    const cudaError_t e = h->fn(c, MODE_STEP_OBS, &nb);
    if (e == cudaSuccess) {
      const void* rho_obs = h->rho[h->cur];  // not overwritten before the next step
      const long long t_obs = h->t;
      h->cur = 1 - h->cur;
      h->t += 1;
      return finish_observables(h, nb, rho_obs, t_obs, out, async);
    }
    if (e != cudaErrorNotSupported) return LBM_ECUDA;
    cudaGetLastError();  // nothing was launched: observe, then step
  }
  rc = observe_impl(h, out, async);
  if (rc != LBM_OK && rc != LBM_EUNSTABLE) return rc;
  const int rs = lbm_step(h, 1);
  return rs != LBM_OK ? rs : rc;
}

extern "C" int lbm_step_observe(lbm_handle* h, long long n, lbm_obs* out) {
  if (!h || !out || n < 1) return LBM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  return step_observe_impl(h, n, out, false);
}

extern "C" int lbm_step_observe_async(lbm_handle* h, long long n, lbm_obs* out) {
  if (!h || !out || n < 1) return LBM_EINVAL;
  return step_observe_impl(h, n, out, true);
}

extern "C" int lbm_get_density(lbm_handle* h, double* host_rho) {
  if (!h || !host_rho) return LBM_EINVAL;
  if (h->p.precision == LBM_FP64) {
    int rc = ck(cudaMemcpyAsync(host_rho, h->rho[h->cur], h->N * 8, cudaMemcpyDeviceToHost, h->stream));
    if (rc == LBM_OK) rc = ck(cudaStreamSynchronize(h->stream));
    return rc;
  }
  double* tmp = static_cast<double*>(dalloc(h, size_t(h->N) * 8));
  if (!tmp) return LBM_ENOMEM;
  const int bs = 256;
  k_export_rho<float><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, static_cast<const float*>(h->rho[h->cur]), tmp);
  int rc = ck(cudaGetLastError());
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(host_rho, tmp, h->N * 8, cudaMemcpyDeviceToHost, h->stream));
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, size_t(h->N) * 8);
  return rc;
}

extern "C" int lbm_get_f(lbm_handle* h, double* host_f) {
  if (!h || !host_f) return LBM_EINVAL;
  const size_t bytes = size_t(h->Q) * h->N * 8;
  double* tmp = static_cast<double*>(dalloc(h, bytes));
  if (!tmp) return LBM_ENOMEM;
  const int bs = 256;
  if (h->p.precision == LBM_FP64)
    k_export_f<double><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, static_cast<double*>(h->f[h->cur]), tmp);
  else
    k_export_f<float><<<grid1(h->N, bs), bs, 0, h->stream>>>(h->kp, h->Q, static_cast<float*>(h->f[h->cur]), tmp);
  int rc = ck(cudaGetLastError());
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(host_f, tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, bytes);
  return rc;
}

extern "C" int lbm_get_force(lbm_handle* h, double* host_F, double* host_mu) {
  if (!h) return LBM_EINVAL;
  const size_t bytes = size_t(h->D + 1) * h->N * 8;
  double* tmp = static_cast<double*>(dalloc(h, bytes));
  if (!tmp) return LBM_ENOMEM;
  Launch c = make_launch(h, h->cur);
  c.fout = nullptr;
  c.rout = nullptr;
  c.fo.F = tmp;
  c.fo.mu = tmp + size_t(h->D) * h->N;
  cudaError_t e = run_pass(h, c, MODE_FIELDS, nullptr);
  int rc = ck(e);
  if (rc == LBM_OK && host_F) rc = ck(cudaMemcpyAsync(host_F, tmp, size_t(h->D) * h->N * 8, cudaMemcpyDeviceToHost, h->stream));
  if (rc == LBM_OK && host_mu) rc = ck(cudaMemcpyAsync(host_mu, c.fo.mu, size_t(h->N) * 8, cudaMemcpyDeviceToHost, h->stream));
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, bytes);
  return rc;
}

extern "C" int lbm_device_state(lbm_handle* h, void** f, void** rho) {
  if (!h) return LBM_EINVAL;
  if (f) *f = h->f[h->cur];
  if (rho) *rho = h->rho[h->cur];
  return LBM_OK;
}

// ------------------------------------------------------------------ walls (Appendix A)
// Wall layers by breadth-first search over the lattice links from the fluid:
// a wall node's layer is its link distance to the nearest fluid node (periodic
// lattice), capped at 4.
extern "C" int lbm_set_solid(lbm_handle* h, const unsigned char* mask, double mu_w) {
  if (!h) return LBM_EINVAL;
  const long long N = h->N;
  if (!mask) {
    cudaStreamSynchronize(h->stream);
    dfree(h, h->layer, size_t(N));
    dfree(h, h->wmu, size_t(N) * 8);
    h->layer = nullptr;
    h->wmu = nullptr;
    return LBM_OK;
  }
  if (!std::isfinite(mu_w)) return LBM_EINVAL;
  if (h->compact || (h->p.scheme != LBM_EFDS2 && h->p.scheme != LBM_EFDS4 && h->p.scheme != LBM_EFDS6))
    return LBM_ENOTSUP;
  const int nx = h->p.nx, ny = h->p.ny, nz = h->D == 3 ? h->p.nz : 1;
  int ex[19], ey[19], ez[19];
  for (int i = 0; i < h->Q; ++i) {
    ex[i] = h->D == 2 ? Lattice<0>::ex(i) : Lattice<1>::ex(i);
    ey[i] = h->D == 2 ? Lattice<0>::ey(i) : Lattice<1>::ey(i);
    ez[i] = h->D == 2 ? 0 : Lattice<1>::ez(i);
  }
  std::vector<signed char> lay(size_t(N), -1);
  std::vector<long long> front, next;
  for (long long n = 0; n < N; ++n)
    if (!mask[n]) {
      lay[size_t(n)] = 0;
      front.push_back(n);
    }
  if (front.empty()) return LBM_EINVAL;
  for (int d = 1; d <= 3 && !front.empty(); ++d) {
    next.clear();
    for (const long long n : front) {
      const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / ((long long)nx * ny));
      for (int i = 1; i < h->Q; ++i) {
        const int tx = (x + ex[i] + nx) % nx, ty = (y + ey[i] + ny) % ny, tz = (z + ez[i] + nz) % nz;
        const long long t = ((long long)tz * ny + ty) * nx + tx;
        if (lay[size_t(t)] < 0) {
          lay[size_t(t)] = static_cast<signed char>(d);
          next.push_back(t);
        }
      }
    }
    front.swap(next);
  }
  for (auto& v : lay)
    if (v < 0) v = 4;
  if (!h->layer) {
    h->layer = static_cast<signed char*>(dalloc(h, size_t(N)));
    h->wmu = dalloc(h, size_t(N) * 8);
    if (!h->layer || !h->wmu) {
      dfree(h, h->layer, size_t(N));
      dfree(h, h->wmu, size_t(N) * 8);
      h->layer = nullptr;
      h->wmu = nullptr;
      return LBM_ENOMEM;
    }
  }
  int rc = ck(cudaMemcpyAsync(h->layer, lay.data(), size_t(N), cudaMemcpyHostToDevice, h->stream));
  if (rc == LBM_OK) rc = ck(cudaStreamSynchronize(h->stream));
  h->mu_w = mu_w;
  return rc;
}

// ------------------------------------------------------------------ Sec. 3.1-3.2 diagnostics
// Flat interface (Eq. 29): uniform mu-hat (Eq. 16) gives the first integral
// (kappa / 2) rho'^2 = k^2 W(rho), W = rho (mu_b(rho) - mu_b(rho_g)) - (p0(rho) -
// p0(rho_g)).  Position as a function of density, y(rho) = int dr / rho', is
// integrated in t = atanh(2 (rho - rho_m) / (rho_l - rho_g)) (finite dy/dt)
// with composite 4-point Gauss-Legendre on a uniform t grid; node densities
// by bracketing on the grid and Newton steps.  Outside |t| <= 8 (densities
// within ~1e-7 of a bulk value) the linearised equation's exponential tails.
extern "C" int lbm_flat_profile(const lbm_params* p, int n, double y0, double* rho, double* drho) {
  if (!p || n < 1 || !rho || !(p->k > 0) || !(p->kappa > 0)) return LBM_EINVAL;
  HostEos E;
  if (make_eos(p, &E) != LBM_OK) return LBM_EINVAL;
  double g, l;
  if (maxwell_eos(E, &g, &l) != LBM_OK) return LBM_EINVAL;
  const double mug = E.mu(g), pg = E.p(g), rm = 0.5 * (g + l), hw = 0.5 * (l - g);
  const double k = p->k, kap = p->kappa;
  auto slope = [&](double r) {
    const double W = r * (E.mu(r) - mug) - (E.p(r) - pg);
    return W > 0 ? k * std::sqrt(2.0 * W / kap) : 0.0;
  };
  auto dens = [&](double t) { return rm + hw * std::tanh(t); };
  auto dydt = [&](double t) {
    const double c = std::cosh(t);
    return hw / (c * c) / slope(dens(t));
  };
  const double gx[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
  const double gw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
  auto integ = [&](double a, double b) {
    const double m = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0;
    for (int q = 0; q < 4; ++q) s += gw[q] * dydt(m + h * gx[q]);
    return h * s;
  };
  const double TMAX = 8.0, DT = 0.005;
  const int M = int(2 * TMAX / DT + 0.5);
  std::vector<double> Y(M + 1);
  Y[M / 2] = 0.0;
  for (int i = M / 2 + 1; i <= M; ++i) Y[i] = Y[i - 1] + integ(-TMAX + (i - 1) * DT, -TMAX + i * DT);
  for (int i = M / 2 - 1; i >= 0; --i) Y[i] = Y[i + 1] - integ(-TMAX + i * DT, -TMAX + (i + 1) * DT);
  const double lg_ = k * std::sqrt(E.dp(g) / g / kap), ll_ = k * std::sqrt(E.dp(l) / l / kap);
  for (int j = 0; j < n; ++j) {
    const double y = double(j) - y0;
    double r, d;
    if (y <= Y[0]) {
      r = g + (dens(-TMAX) - g) * std::exp(lg_ * (y - Y[0]));
      d = lg_ * (r - g);
    } else if (y >= Y[M]) {
      r = l - (l - dens(TMAX)) * std::exp(-ll_ * (y - Y[M]));
      d = ll_ * (l - r);
    } else {
      const int i = int(std::upper_bound(Y.begin(), Y.end(), y) - Y.begin()) - 1;
      const double ta = -TMAX + i * DT;
      double t = ta + DT * (y - Y[i]) / (Y[i + 1] - Y[i]);
      for (int it = 0; it < 5; ++it) t -= (Y[i] + integ(ta, t) - y) / dydt(t);
      r = dens(t);
      d = slope(r);
    }
    rho[j] = r;
    if (drho) drho[j] = d;
  }
  return LBM_OK;
}

namespace {
// Eq. 30 generalised to any dimension: the angle between the force and the
// radial line through the droplet centre, atan2(|F x r|, |F . r|) (atan in
// Eq. 30 defines the direction modulo pi; the atan2 form keeps small angles
// accurate, where acos of a ratio near 1 would not); nodes with |F| >= frac max |F|.
// Pass 1: per-CTA max |F|^2.  Pass 2: per-CTA max angle, sum of |F| angle, sum of |F|, count.
__global__ void k_fmax(const double* F, int D, long long N, double* part) {
  __shared__ double red[256];
  double m = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    double s = 0;
    for (int d = 0; d < D; ++d) s += F[d * N + n] * F[d * N + n];
    m = fmax(m, s);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_fangle(const double* F, int D, int nx, int ny, long long N, double cx, double cy, double cz,
                         const double* fmax_part, int nparts, double frac, double* part) {
  __shared__ double red[4][256];
  __shared__ double s_thr;
  if (threadIdx.x == 0) {
    double m = 0;
    for (int i = 0; i < nparts; ++i) m = fmax(m, fmax_part[i]);
    s_thr = frac * frac * m;  // on |F|^2
  }
  __syncthreads();
  double amax = 0, wsum = 0, fsum = 0, cnt = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const double x = double(n % nx) - cx, y = double((n / nx) % ny) - cy;
    const double z = D == 3 ? double(n / ((long long)nx * ny)) - cz : 0.0;
    const double r2 = x * x + y * y + z * z;
    const double fx = F[n], fy = F[N + n], fz = D == 3 ? F[2 * N + n] : 0.0;
    const double f2 = fx * fx + fy * fy + fz * fz, fr = fx * x + fy * y + fz * z;
    const double c0 = fy * z - fz * y, c1 = fz * x - fx * z, c2 = fx * y - fy * x;
    if (r2 > 0 && f2 > 0 && f2 >= s_thr) {
      const double a = atan2(sqrt(c0 * c0 + c1 * c1 + c2 * c2), fabs(fr)), fm = sqrt(f2);
      amax = fmax(amax, a);
      wsum += fm * a;
      fsum += fm;
      cnt += 1;
    }
  }
  red[0][threadIdx.x] = amax; red[1][threadIdx.x] = wsum; red[2][threadIdx.x] = fsum; red[3][threadIdx.x] = cnt;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      for (int q = 1; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = red[q][0];
}
}  // namespace

extern "C" int lbm_force_angle(lbm_handle* h, const double center[3], double frac, double out[3]) {
  if (!h || !out || !(frac >= 0 && frac <= 1)) return LBM_EINVAL;
  const int nb = 512;
  const size_t fbytes = size_t(h->D + 1) * h->N * 8, pbytes = size_t(nb) * 5 * 8;
  double* tmp = static_cast<double*>(dalloc(h, fbytes + pbytes));
  if (!tmp) return LBM_ENOMEM;
  double* fpart = tmp + size_t(h->D + 1) * h->N;
  double* apart = fpart + nb;
  Launch c = make_launch(h, h->cur);
  c.fout = nullptr;
  c.rout = nullptr;
  c.fo.F = tmp;
  c.fo.mu = tmp + size_t(h->D) * h->N;
  cudaError_t e = run_pass(h, c, MODE_FIELDS, nullptr);
  int rc = ck(e);
  const double cx = center ? center[0] : double(h->p.nx / 2), cy = center ? center[1] : double(h->p.ny / 2);
  const double cz = center ? center[2] : double(h->p.nz / 2);
  if (rc == LBM_OK) {
    k_fmax<<<nb, 256, 0, h->stream>>>(tmp, h->D, h->N, fpart);
    k_fangle<<<nb, 256, 0, h->stream>>>(tmp, h->D, h->p.nx, h->p.ny, h->N, cx, cy, cz, fpart, nb, frac, apart);
    rc = ck(cudaGetLastError());
  }
  std::vector<double> host(size_t(nb) * 4);
  if (rc == LBM_OK) rc = ck(cudaMemcpyAsync(host.data(), apart, host.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  cudaStreamSynchronize(h->stream);
  dfree(h, tmp, fbytes + pbytes);
  if (rc != LBM_OK) return rc;
  double amax = 0, wsum = 0, fsum = 0, cnt = 0;
  for (int b = 0; b < nb; ++b) {
    amax = std::max(amax, host[4 * b]);
    wsum += host[4 * b + 1];
    fsum += host[4 * b + 2];
    cnt += host[4 * b + 3];
  }
  out[0] = amax;
  out[1] = fsum > 0 ? wsum / fsum : 0.0;
  out[2] = cnt;
  return LBM_OK;
}
