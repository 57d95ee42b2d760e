// Device parts of the compact-scheme path shared by the single-case kernels
// (compact.cu) and the batched persistent kernels (batch.cu): the chemical
// potential of one node with the compact scheme's explicit Laplacian, and one
// CTA's share of the periodic tridiagonal line solves of Eq. 21.
#pragma once
#include "compact.cuh"
#include "lbm_device.cuh"

namespace lbmd {

// a + d wrapped into [0, n) for |d| <= 4 < n (one period at most: a
// compare and an add, not an integer division)
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// mu = k^2 psi'(rho) - kappa lap rho at node n, with the explicit central
// second derivative of order LO along each axis (the compact scheme's
// Laplacian); rho holds rho - rho_ref when dev (the Laplacian needs no offset).
template <typename Tm, typename Tr, int LO>
__device__ __forceinline__ Tm mu_field_node(const KParams& p, int D, bool dev, const Tr* rho, long long n) {
  constexpr int R = LO / 2;
  const double l0 = LO == 4 ? -2.5 : (LO == 6 ? -49.0 / 18.0 : -205.0 / 72.0);
  const double lc[5] = {l0, LO == 4 ? 4.0 / 3.0 : (LO == 6 ? 1.5 : 1.6), LO == 4 ? -1.0 / 12.0 : (LO == 6 ? -0.15 : -0.2),
                        LO == 6 ? 1.0 / 90.0 : (LO == 8 ? 8.0 / 315.0 : 0.0), LO == 8 ? -1.0 / 560.0 : 0.0};
  const long long nxy = (long long)p.nx * p.ny;
  const int z = int(n / nxy);
  const int rem = int(n - z * nxy), y = rem / p.nx, x = rem - y * p.nx;
  const Tm c0 = Tm(rho[n]);
  Tm lap = Tm(D * lc[0]) * c0;
  const long long zo = z * nxy, row = zo + (long long)y * p.nx;
#pragma unroll
  for (int m = 1; m <= R; ++m) {
    Tm s = Tm(rho[row + wrap1(x + m, p.nx)]) + Tm(rho[row + wrap1(x - m, p.nx)]);
    s += Tm(rho[zo + (long long)wrap1(y + m, p.ny) * p.nx + x]) + Tm(rho[zo + (long long)wrap1(y - m, p.ny) * p.nx + x]);
    if (D == 3)
      s += Tm(rho[wrap1(z + m, p.nz) * nxy + (long long)y * p.nx + x]) +
           Tm(rho[wrap1(z - m, p.nz) * nxy + (long long)y * p.nx + x]);
    lap += Tm(lc[m]) * s;
  }
  const Tm rfull = dev ? Tm(p.rho_ref) + Tm(rho[n]) : Tm(rho[n]);
  return Tm(p.k2) * eos_mu<Tm>(rfull, p) - Tm(p.kappa) * lap;
}

template <typename Tm, typename Tr>
__device__ __forceinline__ Tm mu_field_node_order(int lo, const KParams& p, int D, bool dev, const Tr* rho, long long n) {
  if (lo == 4) return mu_field_node<Tm, Tr, 4>(p, D, dev, rho, n);
  if (lo == 6) return mu_field_node<Tm, Tr, 6>(p, D, dev, rho, n);
  return mu_field_node<Tm, Tr, 8>(p, D, dev, rho, n);
}

// Derivative along `axis` of LPB lines (LPB a power of two, 1..32, lpb_shift
// its log2) of `in`, lines group `blk` of the lattice, by a CTA of NTH threads
// (NTH / 32 warps) with 2 LPB (L + 1) values of T of shared memory at smem.
// Line j is owned by warp j % (NTH / 32): the warp forms the explicit right
// side of Eq. 21 for its lines and runs the PCR levels on them with only
// warp-level synchronisation (element i of a line on lane i % 32); CTA
// barriers separate the copies in and out only where the global layout
// differs from the warp ownership (lines along y and z are copied across x,
// runs of LPB consecutive lines, for coalescing).  The caller's CTA must reach
// this function as a whole (it contains CTA barriers).
template <int NTH, typename Tin, typename T>
__device__ __forceinline__ void lines_block(int axis, int nx, int ny, int nz, const Tin* in, T* out,
                                            const LineCoef& lc, int LPB, int lpb_shift, long long blk,
                                            unsigned char* smem) {
  const int L = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const int LP = L + 1;
  T* A = reinterpret_cast<T*>(smem);
  T* B = A + LPB * LP;
  const long long NXY = (long long)nx * ny;
  const long long stride = axis == 0 ? 1 : (axis == 1 ? nx : NXY);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int groups_x = (nx + LPB - 1) >> lpb_shift;  // y/z lines: groups of LPB consecutive x
  // global offset of the first element of line j of this group (ok: the line exists)
  auto line_base = [&](int j, bool& ok) -> long long {
    if (axis == 0) {
      const long long row = blk * LPB + j;  // (y, z) row
      ok = row < (long long)ny * nz;
      return row * nx;
    }
    const int gx = int(blk % groups_x) * LPB + j;
    const long long r = blk / groups_x;  // z (axis 1) or y (axis 2)
    ok = gx < nx;
    return axis == 1 ? r * NXY + gx : r * nx + gx;
  };
  if (axis == 0) {
    for (int j = warp; j < LPB; j += NTH / 32) {
      bool ok;
      const long long b = line_base(j, ok);
      for (int i = lane; i < L; i += 32) A[j * LP + i] = ok ? T(in[b + i]) : T(0);
    }
    __syncwarp();
  } else {
    // thread t copies line t % LPB at positions t / LPB + k NTH / LPB
    const int j = threadIdx.x & (LPB - 1), i0 = threadIdx.x >> lpb_shift, di = NTH >> lpb_shift;
    bool ok;
    const long long b = line_base(j, ok);
    for (int i = i0; i < L; i += di) A[j * LP + i] = ok ? T(in[b + i * stride]) : T(0);
    __syncthreads();
  }
  // element loops outside, the warp's lines inside: a wrapped position is
  // computed once for all the lines of the warp (index arithmetic, not the
  // few flops, dominated the per-element cost)
  constexpr int NW = NTH / 32;
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
    for (int j = warp; j < LPB; j += NTH / 32) {
      bool ok;
      const long long b = line_base(j, ok);
      if (ok)
        for (int i = lane; i < L; i += 32) out[b + i] = cur[j * LP + i];
    }
  } else {
    __syncthreads();
    const int j = threadIdx.x & (LPB - 1), i0 = threadIdx.x >> lpb_shift, di = NTH >> lpb_shift;
    bool ok;
    const long long b = line_base(j, ok);
    if (ok)
      for (int i = i0; i < L; i += di) out[b + i * stride] = cur[j * LP + i];
  }
}

// FP32 lines stop at the first PCR level whose |alpha| is below 2^-30: that
// level moves no value by more than 2^-29 of itself, far below the float
// rounding; the float copies of the coefficients are filled in
inline LineCoef line_coef_for(const LineCoef& lc, bool fp32) {
  LineCoef lf = lc;
  if (fp32) {
    int k = 0;
    while (k < lc.nlev && (lc.alpha[k] > 9.3e-10 || lc.alpha[k] < -9.3e-10)) ++k;
    lf.nlev = k;
  }
  for (int k = 0; k < 16; ++k) {
    lf.alpha_f[k] = float(lf.alpha[k]);
    lf.inv_f[k] = float(lf.inv[k]);
  }
  return lf;
}

}  // namespace lbmd
