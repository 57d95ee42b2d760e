// Compact-scheme path: mu field, PCR line solves for the periodic tridiagonal
// systems of Eq. 21 (beta = 0), and the fused collide/stream kernels that read
// the resulting gradient fields.
#include <cmath>

#include <type_traits>

#include "compact.cuh"
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

__device__ __forceinline__ int lmod(long long a, int n) {
  long long r = a % n;
  return int(r < 0 ? r + n : r);
}

// mu = k^2 psi'(rho) - kappa lap rho with the explicit central second
// derivative of order LO along each axis (the compact scheme's Laplacian).
template <typename Tm, typename Tr, int LO>
__global__ void k_mu_field(KParams p, int D, bool dev, const Tr* __restrict__ rho, Tm* __restrict__ mu) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.n) return;
  constexpr int R = LO / 2;
  const double l0 = LO == 4 ? -2.5 : (LO == 6 ? -49.0 / 18.0 : -205.0 / 72.0);
  const double lc[5] = {l0, LO == 4 ? 4.0 / 3.0 : (LO == 6 ? 1.5 : 1.6), LO == 4 ? -1.0 / 12.0 : (LO == 6 ? -0.15 : -0.2),
                        LO == 6 ? 1.0 / 90.0 : (LO == 8 ? 8.0 / 315.0 : 0.0), LO == 8 ? -1.0 / 560.0 : 0.0};
  const int x = int(n % p.nx), y = int((n / p.nx) % p.ny), z = int(n / ((long long)p.nx * p.ny));
  // rho holds rho - rho_ref when dev: the Laplacian needs no offset
  const Tm c0 = Tm(rho[n]);
  Tm lap = Tm(D * lc[0]) * c0;
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    const long long row = (long long)z * p.nx * p.ny + (long long)y * p.nx;
    Tm s = Tm(rho[row + lmod(x + m, p.nx)]) + Tm(rho[row + lmod(x - m, p.nx)]);
    s += Tm(rho[(long long)z * p.nx * p.ny + (long long)lmod(y + m, p.ny) * p.nx + x]) +
         Tm(rho[(long long)z * p.nx * p.ny + (long long)lmod(y - m, p.ny) * p.nx + x]);
    if (D == 3)
      s += Tm(rho[(long long)lmod(z + m, p.nz) * p.nx * p.ny + (long long)y * p.nx + x]) +
           Tm(rho[(long long)lmod(z - m, p.nz) * p.nx * p.ny + (long long)y * p.nx + x]);
    lap += Tm(lc[m]) * s;
  }
  const Tm rfull = dev ? Tm(p.rho_ref) + Tm(rho[n]) : Tm(rho[n]);
  mu[n] = Tm(p.k2) * eos_mu<Tm>(rfull, p) - Tm(p.kappa) * lap;
}

// Derivative along `axis` of lines of `in`: LPB lines per CTA (a power of
// two, 1..32) held in shared memory, line j owned by warp j % 8.  A warp forms
// the explicit right side of Eq. 21 for its lines and runs the PCR levels on
// them with only warp-level synchronisation (element i of a line on lane
// i % 32); CTA barriers separate the copies in and out only where the global
// layout differs from the warp ownership (lines along y and z are copied
// across x, runs of LPB consecutive lines, for coalescing).
constexpr int LT = 256;  // threads of a line CTA: 8 warps

template <typename Tin, typename T>
__global__ void __launch_bounds__(LT) k_lines(int axis, int nx, int ny, int nz, const Tin* __restrict__ in,
                                              T* __restrict__ out, const LineCoef lc, int LPB, int lpb_shift) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const int LP = L + 1;
  T* A = reinterpret_cast<T*>(smem);
  T* B = A + LPB * LP;
  const long long NXY = (long long)nx * ny;
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : NXY);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int groups_x = (nx + LPB - 1) >> lpb_shift;  // y/z lines: groups of LPB consecutive x
  // global offset of the first element of line j of this CTA (ok: the line exists)
  auto line_base = [&](int j, bool& ok) -> long long {
    if (axis == 0) {
      const long long row = (long long)blockIdx.x * LPB + j;  // (y, z) row
      ok = row < (long long)ny * nz;
      return row * nx;
    }
    const int gx = (blockIdx.x % groups_x) * LPB + j;
    const long long r = blockIdx.x / groups_x;  // z (axis 1) or y (axis 2)
    ok = gx < nx;
    return axis == 1 ? r * NXY + gx : r * nx + gx;
  };
  if (axis == 0) {
    for (int j = warp; j < LPB; j += LT / 32) {
      bool ok;
      const long long b = line_base(j, ok);
      for (int i = lane; i < L; i += 32) A[j * LP + i] = ok ? T(in[b + i]) : T(0);
    }
    __syncwarp();
  } else {
    // thread t copies line t % LPB at positions t / LPB + k LT / LPB
    const int j = threadIdx.x & (LPB - 1), i0 = threadIdx.x >> lpb_shift, di = LT >> lpb_shift;
    bool ok;
    const long long b = line_base(j, ok);
    for (int i = i0; i < L; i += di) A[j * LP + i] = ok ? T(in[b + i * stride]) : T(0);
    __syncthreads();
  }
  // element loops outside, the warp's lines inside: a wrapped position is
  // computed once for all the lines of the warp (index arithmetic, not the
  // few flops, dominated the per-element cost)
  constexpr int NW = LT / 32;
  auto for_lines = [&](auto&& fn) {
    if (LPB == 4 * NW) {
#pragma unroll
      for (int q = 0; q < 4; ++q) fn(warp + q * NW);
    } else {
      for (int j = warp; j < LPB; j += NW) fn(j);
    }
  };
  const T A1 = T(lc.A1), A2 = T(lc.A2), A3 = T(lc.A3);
  const bool has2 = lc.A2 != 0.0, has3 = lc.A3 != 0.0;
  for (int i = lane; i < L; i += 32) {
    // explicit side: a (f[i+1]-f[i-1])/2 + b (f[i+2]-f[i-2])/4 + c (f[i+3]-f[i-3])/6
    auto wr = [&](int k) { return k < 0 ? k + L : (k >= L ? k - L : k); };
    const int p1 = wr(i + 1), m1 = wr(i - 1), p2 = wr(i + 2), m2 = wr(i - 2), p3 = wr(i + 3), m3 = wr(i - 3);
    for_lines([&](int j) {
      const T* f = A + j * LP;
      T r = A1 * (f[p1] - f[m1]);
      if (has2) r += A2 * (f[p2] - f[m2]);
      if (has3) r += A3 * (f[p3] - f[m3]);
      B[j * LP + i] = r;
    });
  }
  __syncwarp();
  T* cur = B;
  T* nxt = A;
  int s = 1 % L;
  for (int k = 0; k < lc.nlev; ++k) {
    const T al = sizeof(T) == 4 ? T(lc.alpha_f[k]) : T(lc.alpha[k]);
    const T iv = sizeof(T) == 4 ? T(lc.inv_f[k]) : T(lc.inv[k]);
    for (int i = lane; i < L; i += 32) {
      int ip = i + s; if (ip >= L) ip -= L;
      int im = i - s; if (im < 0) im += L;
      for_lines([&](int j) {
        const T* d = cur + j * LP;
        nxt[j * LP + i] = (d[i] - al * (d[im] + d[ip])) * iv;
      });
    }
    __syncwarp();
    T* t = cur; cur = nxt; nxt = t;
    s = 2 * s; if (s >= L) s -= L;
  }
  if (axis == 0) {
    for (int j = warp; j < LPB; j += LT / 32) {
      bool ok;
      const long long b = line_base(j, ok);
      if (ok)
        for (int i = lane; i < L; i += 32) out[b + i] = cur[j * LP + i];
    }
  } else {
    __syncthreads();
    const int j = threadIdx.x & (LPB - 1), i0 = threadIdx.x >> lpb_shift, di = LT >> lpb_shift;
    bool ok;
    const long long b = line_base(j, ok);
    if (ok)
      for (int i = i0; i < L; i += di) out[b + i * stride] = cur[j * LP + i];
  }
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
  // FP32 lines: a level whose |alpha| is below 2^-30 moves no value by more
  // than 2^-29 of itself, far below the float rounding: stop before it
  LineCoef lf = lc;
  if (sizeof(T) == 4) {
    int k = 0;
    while (k < lc.nlev && std::fabs(lc.alpha[k]) > 9.3e-10) ++k;
    lf.nlev = k;
  }
  for (int k = 0; k < 16; ++k) {
    lf.alpha_f[k] = float(lf.alpha[k]);
    lf.inv_f[k] = float(lf.inv[k]);
  }
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
