// Compact-scheme path: mu field, PCR line solves for the periodic tridiagonal
// systems of Eq. 21 (beta = 0), and the fused collide/stream kernels that read
// the resulting gradient fields.
#include <cmath>

#include <type_traits>

#include "compact.cuh"
#include "compact_dev.cuh"
#include "step2d.cuh"
#include "step3d.cuh"

namespace lbmd {

void compact_coeffs(int scheme, double* alpha, double* a, double* b, double* c) {
  *alpha = *a = *b = *c = 0.0;
  switch (scheme) {
    case S_CFDS4: *alpha = 0.25; *a = 1.5; break;                               // Eq. 22
    case S_CFDS6: *alpha = 1.0 / 3.0; *a = 14.0 / 9.0; *b = 1.0 / 9.0; break;   // Eq. 23
    case S_CFDS8: *alpha = 0.375; *a = 25.0 / 16.0; *b = 0.2; *c = -1.0 / 80.0; break;  // Eq. 24
    case S_OCFDS4: {
      const double al = 0.446776, cc = -0.0541132;
      // a + b + c = 1 + 2 alpha and a + 4 b + 9 c = 6 alpha
      const double bb = ((6.0 * al - 9.0 * cc) - (1.0 + 2.0 * al - cc)) / 3.0;
      *alpha = al; *c = cc; *b = bb; *a = (1.0 + 2.0 * al - cc) - bb;
      break;
    }
    default: break;
  }
}

// PCR on x_i + al (x_{i-s} + x_{i+s}) = d_i: combining rows i-s, i, i+s gives
// x_i + al' (x_{i-2s} + x_{i+2s}) = d'_i with al' = -al^2/(1 - 2 al^2) and
// d'_i = (d_i - al (d_{i-s} + d_{i+s}))/(1 - 2 al^2); exact for circulant
// systems of any length (indices modulo the line length).
LineCoef make_line_coef(int scheme) {
  LineCoef lc{};
  double al, a, b, c;
  compact_coeffs(scheme, &al, &a, &b, &c);
  lc.A1 = 0.5 * a;
  lc.A2 = 0.25 * b;
  lc.A3 = c / 6.0;
  int k = 0;
  while (std::fabs(al) > 1e-17 && k < 16) {
    lc.alpha[k] = al;
    lc.inv[k] = 1.0 / (1.0 - 2.0 * al * al);
    al = -al * al * lc.inv[k];
    ++k;
  }
  lc.nlev = k;
  return lc;
}

namespace {

// mu field of the compact schemes, one node per thread
template <typename Tm, typename Tr, int LO>
__global__ void k_mu_field(KParams p, int D, bool dev, const Tr* __restrict__ rho, Tm* __restrict__ mu) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  mu[n] = mu_field_node<Tm, Tr, LO>(p, D, dev, rho, n);
}

// line solves: one group of LPB lines per CTA
constexpr int LT = 256;  // threads of a line CTA: 8 warps

template <typename Tin, typename T>
__global__ void __launch_bounds__(LT) k_lines(int axis, int nx, int ny, int nz, const Tin* __restrict__ in,
                                              T* __restrict__ out, const LineCoef lc, int LPB, int lpb_shift) {
  extern __shared__ __align__(16) unsigned char smem[];
  lines_block<LT, Tin, T>(axis, nx, ny, nz, in, out, lc, LPB, lpb_shift, blockIdx.x, smem);
}

template <typename Tin, typename T>
cudaError_t run_lines(int axis, const KParams& kp, const Tin* in, double ref, T* out, const LineCoef& lc,
                      cudaStream_t st) {
  (void)ref;
  const int L = axis == 0 ? kp.nx : (axis == 1 ? kp.ny : kp.nz);
  int LPB = 32, sh = 5;
  while (LPB > 1 && size_t(2) * LPB * (L + 1) * sizeof(T) > 200 * 1024) { LPB /= 2; --sh; }
  const size_t smem = size_t(2) * LPB * (L + 1) * sizeof(T);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  if (cudaError_t e = ensure_smem(k_lines<Tin, T>, size_t(220) * 1024); e != cudaSuccess) return e;
  unsigned grid;
  if (axis == 0) {
    grid = unsigned(((long long)kp.ny * kp.nz + LPB - 1) / LPB);
  } else {
    const int gx = (kp.nx + LPB - 1) / LPB;
    grid = unsigned((long long)gx * (axis == 1 ? kp.nz : kp.ny));
  }
  const LineCoef lf = line_coef_for(lc, sizeof(T) == 4);
  k_lines<Tin, T><<<grid, LT, smem, st>>>(axis, kp.nx, kp.ny, kp.nz, in, out, lf, LPB, sh);
  return cudaGetLastError();
}

constexpr int TXc = 32, TYc = 8, ZCc = 32;

template <class P, int MODE>
cudaError_t launch_gf(const Launch& c, int D, int* nblocks) {
  using Tf = typename P::Tf;
  using Tr = typename P::Tr;
  const Tr* rin = static_cast<const Tr*>(c.rin);
  Tr* rout = static_cast<Tr*>(c.rout);
  if (D == 2) {
    using Sh = Step2DShape<S_CFDS4, P, TXc, TYc>;
    auto k = k_step2d<S_CFDS4, P, TXc, TYc, MODE>;
    if (cudaError_t e = ensure_smem(k, Sh::bytes); e != cudaSuccess) return e;
    dim3 grid((c.kp.nx + TXc - 1) / TXc, (c.kp.ny + TYc - 1) / TYc, 1);
    if (nblocks) *nblocks = int(grid.x * grid.y);
    k<<<grid, NT2, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout), rin, rout,
                                          c.aux, c.fo, c.gi, c.mrt);
  } else {
    using Sh = Step3DShape<S_CFDS4, P, TXc, TYc>;
    auto k = k_step3d<S_CFDS4, P, TXc, TYc, ZCc, MODE>;
    if (cudaError_t e = ensure_smem(k, Sh::bytes); e != cudaSuccess) return e;
    dim3 grid((c.kp.nx + TXc - 1) / TXc, (c.kp.ny + TYc - 1) / TYc, (c.kp.nz + ZCc - 1) / ZCc);
    if (nblocks) *nblocks = int(grid.x * grid.y * grid.z);
    k<<<grid, NT3, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout), rin, rout,
                                          c.aux, c.fo, c.gi);
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t step_prec(const CompactBufs& cb, Launch c, int D, int mode, int* nblocks) {
  using Tm = typename P::Tm;
  using Tc = typename P::Tc;
  using Tr = typename P::Tr;
  const Tr* rin = static_cast<const Tr*>(c.rin);
  const KParams& kp = c.kp;
  const int bs = 256;
  const unsigned g = unsigned((kp.n + bs - 1) / bs);
  Tm* mu = static_cast<Tm*>(cb.mu);
  cudaError_t e;
  if (std::is_same<P, PrecF32>::value && D == 3 && (cb.lap_order == 4 || cb.lap_order == 6)) {
    // FP32 mu in 3D: the z-marching mu pass of the split path
    Launch cm = c;
    cm.mu = mu;
    e = mu3d_pass(cm, cb.lap_order);
  } else {
    if (cb.lap_order == 4) k_mu_field<Tm, Tr, 4><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    else if (cb.lap_order == 6) k_mu_field<Tm, Tr, 6><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    else k_mu_field<Tm, Tr, 8><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  Tm* gmu = static_cast<Tm*>(cb.gmu);
  Tc* grho = static_cast<Tc*>(cb.grho);
  for (int ax = 0; ax < D; ++ax) {
    e = run_lines<Tm, Tm>(ax, kp, mu, 0.0, gmu + size_t(ax) * kp.n, cb.lc, c.stream);
    if (e != cudaSuccess) return e;
    e = run_lines<Tr, Tc>(ax, kp, rin, 0.0, grho + size_t(ax) * kp.n, cb.lc, c.stream);
    if (e != cudaSuccess) return e;
  }
  c.gi.gmu = gmu;
  c.gi.grho = grho;
  c.gi.mu = mu;
  if (std::is_same<P, PrecF32>::value && D == 3 && mode == MODE_STEP) {
    e = coll3d_gf_step(c, nblocks);
    if (e != cudaErrorNotSupported) return e;
  }
  if (mode == MODE_STEP) return launch_gf<P, MODE_STEP>(c, D, nblocks);
  if (mode == MODE_OBS) return launch_gf<P, MODE_OBS>(c, D, nblocks);
  return launch_gf<P, MODE_FIELDS>(c, D, nblocks);
}

}  // namespace

cudaError_t compact_step(const CompactBufs& cb, Launch c, int D, int scheme, int prec, int mode, int* nblocks) {
  (void)scheme;
  if (prec == 0) return step_prec<PrecF64>(cb, c, D, mode, nblocks);
  if (prec == 1) return step_prec<PrecF32>(cb, c, D, mode, nblocks);
  return step_prec<PrecF32M64>(cb, c, D, mode, nblocks);
}

}  // namespace lbmd
