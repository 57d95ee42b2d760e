// Compact-scheme path: mu field, PCR line solves for the periodic tridiagonal
// systems of Eq. 21 (beta = 0), and the fused collide/stream kernels that read
// the resulting gradient fields.
#include <cmath>

#include <type_traits>
#include <utility>

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

// FP32 lines whose length is a multiple of 32, L = 32 LW (LW = 2..16): one
// warp holds a whole line in registers, lane l the block of elements
// l LW .. l LW + LW - 1 (element i in v[i % LW] of lane i / LW).  The value at
// offset o from element l LW + k is element (l + q) LW + r of the periodic
// line, with q and r fixed by k and o: register r of lane (l + q) mod 32, one
// shuffle when q is not a multiple of 32, a register of the lane itself when
// it is.  A PCR level of stride s needs min(LW, s) shuffles per direction (one
// per register that looks past its lane's block), the right side of Eq. 21
// 1 + 2 + 3 per direction; no selects.  The arithmetic is that of k_lines.
// Lines are staged in shared memory to switch between the coalesced global
// layout and the blocked one: x lines one row per warp, y and z lines padded
// tiles of 32 lines of consecutive x.  One launch does both fields of an axis:
// for x lines the first half of the blocks takes mu, the second rho; a block
// of y or z lines takes the same 32 lines of both fields.
constexpr int LRT = 256;  // 8 warps

template <int LW>
struct BlkLine {
  float v[LW];
};

// value at offset O (|O| < L) from each of the lane's elements
template <int LW, int O>
__device__ __forceinline__ void blk_shift(const BlkLine<LW>& f, int lane, float* out) {
  constexpr int L = 32 * LW;
#pragma unroll
  for (int k = 0; k < LW; ++k) {
    const int j = ((k + O) % L + L) % L;  // compile-time: k is unrolled
    const int q = j / LW, r = j % LW;
    if (q % 32 == 0) out[k] = f.v[r];
    else out[k] = __shfl_sync(0xffffffffu, f.v[r], (lane + q) & 31);
  }
}

// stride of PCR level lev on a periodic line of L elements: 2^lev mod L
__host__ __device__ constexpr int pcr_stride(int lev, int L) {
  int s = 1 % L;
  for (int k = 0; k < lev; ++k) {
    s *= 2;
    if (s >= L) s -= L;
  }
  return s;
}

// A PCR level divides every row by 1 - 2 alpha^2, the same number for every
// element of every line: the register kernel leaves those divisions out and
// takes their product into the right side instead (lc.A1..A3 arrive scaled by
// it, see run_lines_pair_f32), two flops per element and level.
template <int LW, int LEV>
__device__ __forceinline__ void pcr_level(BlkLine<LW>& d, int lane, const LineCoef& lc) {
  constexpr int S = pcr_stride(LEV, 32 * LW);
  const float al = lc.alpha_f[LEV];
  float m[LW], p[LW];
  blk_shift<LW, S>(d, lane, p);
  blk_shift<LW, -S>(d, lane, m);
#pragma unroll
  for (int k = 0; k < LW; ++k) d.v[k] = d.v[k] - al * (m[k] + p[k]);
}

template <int LW, int... LEV>
__device__ __forceinline__ void pcr_levels(BlkLine<LW>& d, int lane, const LineCoef& lc,
                                           std::integer_sequence<int, LEV...>) {
  ((LEV < lc.nlev ? pcr_level<LW, LEV>(d, lane, lc) : void()), ...);
}

template <int LW>
__device__ __forceinline__ void solve_line(BlkLine<LW>& f, int lane, const LineCoef& lc) {
  const float A1 = float(lc.A1), A2 = float(lc.A2), A3 = float(lc.A3);
  const bool has2 = lc.A2 != 0.0, has3 = lc.A3 != 0.0;
  float p[LW], m[LW];
  BlkLine<LW> r;
  blk_shift<LW, 1>(f, lane, p);
  blk_shift<LW, -1>(f, lane, m);
#pragma unroll
  for (int k = 0; k < LW; ++k) r.v[k] = A1 * (p[k] - m[k]);
  if (has2) {
    blk_shift<LW, 2>(f, lane, p);
    blk_shift<LW, -2>(f, lane, m);
#pragma unroll
    for (int k = 0; k < LW; ++k) r.v[k] += A2 * (p[k] - m[k]);
  }
  if (has3) {
    blk_shift<LW, 3>(f, lane, p);
    blk_shift<LW, -3>(f, lane, m);
#pragma unroll
    for (int k = 0; k < LW; ++k) r.v[k] += A3 * (p[k] - m[k]);
  }
  pcr_levels<LW>(r, lane, lc, std::make_integer_sequence<int, 16>{});
  f = r;
}

// x lines: 8 lines of one field per block, one line per warp, staged per
// warp in a row of the shared tile (tile: [8][L] floats)
template <int LW>
__device__ __forceinline__ void lines_reg_x(unsigned b, int nx, int ny, int nz, const float* __restrict__ in,
                                            float* __restrict__ out, const LineCoef& lc, float* tile) {
  constexpr int L = 32 * LW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long row = (long long)b * (LRT / 32) + warp;
  if (row >= (long long)ny * nz) return;  // whole warps only: the warp's own row of the tile, no CTA barrier
  float* t = tile + warp * L;
  const float* src = in + row * nx;
  BlkLine<LW> f;
#pragma unroll
  for (int k = 0; k < LW; ++k) t[lane + 32 * k] = src[lane + 32 * k];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LW; ++k) f.v[k] = t[lane * LW + k];
  solve_line<LW>(f, lane, lc);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LW; ++k) t[lane * LW + k] = f.v[k];
  __syncwarp();
  float* dst = out + row * nx;
#pragma unroll
  for (int k = 0; k < LW; ++k) dst[lane + 32 * k] = t[lane + 32 * k];
}

// y (axis 1) or z (axis 2) lines: block bb = (32 consecutive x) x (z or y);
// NF = 2: both fields of the same 32 lines in one block (tile: 2 x [L][33]
// floats), so that twice the row loads are in flight while the block waits for
// them; NF = 1: the first field only (mu, gmu)
template <int LW, int NF = 2>
__device__ __forceinline__ void lines_reg_yz(int axis, unsigned bb, int nx, int ny, const float* __restrict__ mu,
                                             const float* __restrict__ rho, float* __restrict__ gmu,
                                             float* __restrict__ grho, const LineCoef& lc, float* tile) {
  constexpr int L = 32 * LW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long NXY = (long long)nx * ny;
  const int gxs = (nx + 31) / 32;
  const int x0 = int(bb % gxs) * 32;
  const long long r = bb / gxs;  // z (axis 1) or y (axis 2)
  const long long base = axis == 1 ? r * NXY + x0 : r * nx + x0;
  const long long stride = axis == 1 ? nx : NXY;
  const bool xin = x0 + lane < nx;
  float* t0 = tile;
  float* t1 = tile + L * 33;
  BlkLine<LW> f;
  // every row load of the warp in flight before the first is used
#pragma unroll
  for (int i = warp; i < L; i += LRT / 32) {
    t0[i * 33 + lane] = xin ? mu[base + i * stride + lane] : 0.f;
    if (NF == 2) t1[i * 33 + lane] = xin ? rho[base + i * stride + lane] : 0.f;
  }
  __syncthreads();
  for (int j = warp; j < 32 * NF; j += LRT / 32) {
    float* t = j < 32 ? t0 : t1;
    const int jj = j & 31;
#pragma unroll
    for (int k = 0; k < LW; ++k) f.v[k] = t[(lane * LW + k) * 33 + jj];
    solve_line<LW>(f, lane, lc);
#pragma unroll
    for (int k = 0; k < LW; ++k) t[(lane * LW + k) * 33 + jj] = f.v[k];
  }
  __syncthreads();
  if (xin) {
#pragma unroll
    for (int i = warp; i < L; i += LRT / 32) {
      gmu[base + i * stride + lane] = t0[i * 33 + lane];
      if (NF == 2) grho[base + i * stride + lane] = t1[i * 33 + lane];
    }
  }
}

// one axis: axis 0, 2 fields x ceil(lines / 8) blocks (the first `half` take
// mu); axes 1, 2, ceil(nx / 32) x (nz or ny) blocks of both fields
template <int LW>
__global__ void __launch_bounds__(LRT) k_lines_reg(int axis, int nx, int ny, int nz, const float* __restrict__ mu,
                                                   const float* __restrict__ rho, float* __restrict__ gmu,
                                                   float* __restrict__ grho, const LineCoef lc, unsigned half) {
  extern __shared__ __align__(16) float tile[];
  if (axis == 0) {
    const bool second = blockIdx.x >= half;
    lines_reg_x<LW>(second ? blockIdx.x - half : blockIdx.x, nx, ny, nz, second ? rho : mu, second ? grho : gmu, lc,
                    tile);
  } else {
    lines_reg_yz<LW>(axis, blockIdx.x, nx, ny, mu, rho, gmu, grho, lc, tile);
  }
}

// the three axes of a lattice whose edges are all L = 32 LW long, in one
// launch: blocks [0, nyz) the z lines, [nyz, 2 nyz) the y lines, then the x
// lines (NF xh blocks, the first xh taking the first field); the derivative
// fields are component-major (3 x N floats).  NF = 2: both fields (mu, rho);
// NF = 1: one field, passed as mu / gmu.  One launch instead of three: the
// blocks of all axes share the field reads through L2, and the tail of one
// axis overlaps the others.
template <int LW, int NF>
__global__ void __launch_bounds__(LRT) k_lines_reg3(int n, const float* __restrict__ mu,
                                                    const float* __restrict__ rho, float* __restrict__ gmu,
                                                    float* __restrict__ grho, const LineCoef lc, unsigned nyz,
                                                    unsigned xh) {
  extern __shared__ __align__(16) float tile[];
  const long long N = (long long)n * n * n;
  const unsigned b = blockIdx.x;
  if (b < nyz) {
    lines_reg_yz<LW, NF>(2, b, n, n, mu, rho, gmu + 2 * N, grho + 2 * N, lc, tile);
  } else if (b < 2 * nyz) {
    lines_reg_yz<LW, NF>(1, b - nyz, n, n, mu, rho, gmu + N, grho + N, lc, tile);
  } else {
    const unsigned bx = b - 2 * nyz;
    const bool second = bx >= xh;
    lines_reg_x<LW>(second ? bx - xh : bx, n, n, n, second ? rho : mu, second ? grho : gmu, lc, tile);
  }
}

template <int LW>
cudaError_t launch_lines_reg(int axis, const KParams& kp, const float* mu, const float* rho, float* gmu, float* grho,
                             const LineCoef& lf, cudaStream_t st) {
  constexpr int L = 32 * LW;
  unsigned half;
  size_t smem = 0;
  if (axis == 0) {
    half = unsigned(((long long)kp.ny * kp.nz + LRT / 32 - 1) / (LRT / 32));
    smem = size_t(LRT / 32) * L * 4;
  } else {
    half = unsigned((long long)((kp.nx + 31) / 32) * (axis == 1 ? kp.nz : kp.ny));
    smem = size_t(2) * L * 33 * 4;
  }
  if (cudaError_t e = ensure_smem(k_lines_reg<LW>, smem); e != cudaSuccess) return e;
  // axis 0: the first half of the blocks takes mu, the second rho; y and z:
  // every block takes both
  const unsigned blocks = axis == 0 ? 2 * half : half;
  k_lines_reg<LW><<<blocks, LRT, smem, st>>>(axis, kp.nx, kp.ny, kp.nz, mu, rho, gmu, grho, lf, half);
  return cudaGetLastError();
}

// lattices whose three axes the single-launch line kernel solves (a cube of
// edge 32 LW, LW one of the register kernel's block lengths)
static bool lines3_ok(const KParams& kp) {
  const int lw = kp.nx / 32;
  return kp.nx == kp.ny && kp.nx == kp.nz && kp.nx % 32 == 0 &&
         (lw >= 2 && lw <= 8 || lw == 10 || lw == 12 || lw == 16);
}

// coefficients of the register kernels: the levels' row scalings folded into
// the right side
static LineCoef reg_coef(const LineCoef& lc) {
  const LineCoef lf = line_coef_for(lc, true);
  LineCoef lr = lf;
  double scale = 1.0;
  for (int k = 0; k < lf.nlev; ++k) scale *= lf.inv[k];
  lr.A1 = lf.A1 * scale;
  lr.A2 = lf.A2 * scale;
  lr.A3 = lf.A3 * scale;
  return lr;
}

template <int LW>
cudaError_t launch_lines_reg3(const KParams& kp, const float* mu, const float* rho, float* gmu, float* grho,
                              const LineCoef& lr, cudaStream_t st) {
  constexpr int L = 32 * LW;
  const unsigned nyz = unsigned((long long)((L + 31) / 32) * L);
  const unsigned xh = unsigned(((long long)L * L + LRT / 32 - 1) / (LRT / 32));
  if (rho) {
    const size_t smem = size_t(2) * L * 33 * 4;
    if (cudaError_t e = ensure_smem(k_lines_reg3<LW, 2>, smem); e != cudaSuccess) return e;
    k_lines_reg3<LW, 2><<<2 * nyz + 2 * xh, LRT, smem, st>>>(L, mu, rho, gmu, grho, lr, nyz, xh);
  } else {
    const size_t smem = size_t(L) * 33 * 4;
    if (cudaError_t e = ensure_smem(k_lines_reg3<LW, 1>, smem); e != cudaSuccess) return e;
    k_lines_reg3<LW, 1><<<2 * nyz + xh, LRT, smem, st>>>(L, mu, nullptr, gmu, nullptr, lr, nyz, xh);
  }
  return cudaGetLastError();
}

// grad mu and grad rho along all three axes of FP32 fields on a cubic lattice
// (gmu, grho component-major, 3 x N floats) in one launch, when its edge is a
// multiple of 32 (64 .. 512); cudaErrorNotSupported (nothing launched)
// otherwise.  rho == nullptr: the first field only (mu into gmu).
cudaError_t run_lines3_f32(const KParams& kp, const float* mu, const float* rho, float* gmu, float* grho,
                           const LineCoef& lc, cudaStream_t st) {
  if (!lines3_ok(kp)) return cudaErrorNotSupported;
  const LineCoef lr = reg_coef(lc);
  if (lr.nlev > 16) return cudaErrorNotSupported;
  switch (kp.nx / 32) {
    case 2: return launch_lines_reg3<2>(kp, mu, rho, gmu, grho, lr, st);
    case 3: return launch_lines_reg3<3>(kp, mu, rho, gmu, grho, lr, st);
    case 4: return launch_lines_reg3<4>(kp, mu, rho, gmu, grho, lr, st);
    case 5: return launch_lines_reg3<5>(kp, mu, rho, gmu, grho, lr, st);
    case 6: return launch_lines_reg3<6>(kp, mu, rho, gmu, grho, lr, st);
    case 7: return launch_lines_reg3<7>(kp, mu, rho, gmu, grho, lr, st);
    case 8: return launch_lines_reg3<8>(kp, mu, rho, gmu, grho, lr, st);
    case 10: return launch_lines_reg3<10>(kp, mu, rho, gmu, grho, lr, st);
    case 12: return launch_lines_reg3<12>(kp, mu, rho, gmu, grho, lr, st);
    case 16: return launch_lines_reg3<16>(kp, mu, rho, gmu, grho, lr, st);
    default: return cudaErrorNotSupported;
  }
}

// grad mu and grad rho along one axis of FP32 fields: the register kernel
// when the line length is a multiple of 32 (64 .. 512), else k_lines per field
cudaError_t run_lines_pair_f32(int axis, const KParams& kp, const float* mu, const float* rho, float* gmu,
                               float* grho, const LineCoef& lc, cudaStream_t st) {
  const int L = axis == 0 ? kp.nx : (axis == 1 ? kp.ny : kp.nz);
  const LineCoef lr = reg_coef(lc);
  if (L % 32 == 0 && lr.nlev <= 16) {
    switch (L / 32) {
      case 2: return launch_lines_reg<2>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 3: return launch_lines_reg<3>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 4: return launch_lines_reg<4>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 5: return launch_lines_reg<5>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 6: return launch_lines_reg<6>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 7: return launch_lines_reg<7>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 8: return launch_lines_reg<8>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 10: return launch_lines_reg<10>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 12: return launch_lines_reg<12>(axis, kp, mu, rho, gmu, grho, lr, st);
      case 16: return launch_lines_reg<16>(axis, kp, mu, rho, gmu, grho, lr, st);
      default: break;
    }
  }
  cudaError_t e = run_lines<float, float>(axis, kp, mu, 0.0, gmu, lc, st);
  if (e != cudaSuccess) return e;
  return run_lines<float, float>(axis, kp, rho, 0.0, grho, lc, st);
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
  // D3Q19 FP32 steps collide on the tiled z-marching kernel when the lattice
  // allows it; its output density's band edge rows are zeroed first
  const bool gf3 = std::is_same<P, PrecF32>::value && D == 3 && mode == MODE_STEP && coll3d_gf_ok(c);
  Tm* gmu = static_cast<Tm*>(cb.gmu);
  Tc* grho = static_cast<Tc*>(cb.grho);
  // D3Q19 FP32 on a cube of register-kernel lines: the density's line solves
  // (which do not need mu) run on the side stream while this stream computes
  // mu and then its line solves; the collision waits for both
  // (the fork is recorded before the mu pass, whose launch is submitted
  // first; the side stream's launch follows it)
  bool fork_rec = false, forked = false;
  if constexpr (std::is_same<P, PrecF32>::value) {
    if (D == 3 && cb.side && lines3_ok(kp)) {
      if ((e = cudaEventRecord(cb.fork, c.stream)) != cudaSuccess) return e;
      fork_rec = true;
    }
  }
  auto fork_lines = [&]() -> cudaError_t {
    if (!fork_rec) return cudaSuccess;
    cudaError_t ef = cudaStreamWaitEvent(cb.side, cb.fork, 0);
    if (ef != cudaSuccess) return ef;
    ef = run_lines3_f32(kp, reinterpret_cast<const float*>(rin), nullptr, reinterpret_cast<float*>(grho), nullptr,
                        cb.lc, cb.side);
    const cudaError_t ej = cudaEventRecord(cb.join, cb.side);
    if (ef == cudaSuccess && ej != cudaSuccess) ef = ej;
    if (ef != cudaSuccess) {
      cudaStreamWaitEvent(c.stream, cb.join, 0);
      return ef == cudaErrorNotSupported ? cudaSuccess : ef;
    }
    forked = true;
    return cudaSuccess;
  };
  if (std::is_same<P, PrecF32>::value && D == 3 && (cb.lap_order == 4 || cb.lap_order == 6)) {
    // FP32 mu in 3D: the z-marching mu pass of the split path
    Launch cm = c;
    cm.mu = mu;
    e = mu3d_pass(cm, cb.lap_order, gf3);
    if (e == cudaSuccess) e = fork_lines();
  } else {
    if (cb.lap_order == 4) k_mu_field<Tm, Tr, 4><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    else if (cb.lap_order == 6) k_mu_field<Tm, Tr, 6><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    else k_mu_field<Tm, Tr, 8><<<g, bs, 0, c.stream>>>(kp, D, P::DEV, rin, mu);
    e = cudaGetLastError();
    if constexpr (std::is_same<P, PrecF32>::value)
      if (e == cudaSuccess && gf3)
        e = coll3d_zero_edges(kp, rin, static_cast<float*>(c.rout), c.aux.bad_step, c.aux.t, c.stream);
    if (e == cudaSuccess) e = fork_lines();
  }
  if (e != cudaSuccess) {
    if (forked) cudaStreamWaitEvent(c.stream, cb.join, 0);
    return e;
  }
  bool lines_done = false;
  if constexpr (std::is_same<P, PrecF32>::value) {
    if (forked) {
      e = run_lines3_f32(kp, mu, nullptr, gmu, nullptr, cb.lc, c.stream);
      const cudaError_t ej = cudaStreamWaitEvent(c.stream, cb.join, 0);
      if (e == cudaSuccess) e = ej;
      if (e != cudaSuccess) return e;
      lines_done = true;
    } else if (D == 3) {
      e = run_lines3_f32(kp, mu, rin, gmu, grho, cb.lc, c.stream);
      if (e != cudaSuccess && e != cudaErrorNotSupported) return e;
      lines_done = e == cudaSuccess;
    }
  }
  for (int ax = 0; ax < D && !lines_done; ++ax) {
    if constexpr (std::is_same<P, PrecF32>::value) {
      e = run_lines_pair_f32(ax, kp, mu, rin, gmu + size_t(ax) * kp.n, grho + size_t(ax) * kp.n, cb.lc, c.stream);
      if (e != cudaSuccess) return e;
      continue;
    }
    e = run_lines<Tm, Tm>(ax, kp, mu, 0.0, gmu + size_t(ax) * kp.n, cb.lc, c.stream);
    if (e != cudaSuccess) return e;
    e = run_lines<Tr, Tc>(ax, kp, rin, 0.0, grho + size_t(ax) * kp.n, cb.lc, c.stream);
    if (e != cudaSuccess) return e;
  }
  c.gi.gmu = gmu;
  c.gi.grho = grho;
  c.gi.mu = mu;
  if (gf3) return coll3d_gf_step(c, nblocks);
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
