// Chemical-potential wall boundary (Appendix A) for the explicit schemes
// EFDS2/4/6 on D2Q9 and D3Q19, FP64 and FP32-deviation storage.
//
// A step with walls runs as node-parallel passes (walls break the tile
// regularity the fused kernels rely on; this path is correctness first):
//   1. wall densities, layer 1, 2, 3 in turn: the w_i-weighted average of the
//      neighbours in the layer before (Eq. A.1; layer 0 = fluid);
//   2. mu: k^2 psi'(rho) - kappa-hat lap rho on fluid nodes (Eq. 16), the wall
//      chemical potential mu_w on wall nodes;
//   3. fluid nodes: moments, grad mu and grad rho (Eq. 17-20), F (Eq. 12),
//      BGK or MRT collision with EDM forcing, push streaming with halfway
//      bounce-back off wall nodes;
//   4. next density of the fluid nodes (sum of the populations).
// Wall layers come from the host (lbm_set_solid): 0 fluid, 1..3 the layers
// that fluid stencils reach, 4 deeper (never read, never written).
// Threads: 32 x 8 per CTA over (x, row), row = y + ny z, both grid-strided;
// indices are 32-bit (the handle caps Q N below 2^31).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/lbm.h"
#include "launch.cuh"
#include "mrt.cuh"
#include "walls.cuh"

namespace lbmd {
namespace {

constexpr int WX = 32, WY = 8, WT = WX * WY;

struct Geo {
  int nx, ny, nz, n;
};

// node of (x + dx, y + dy, z + dz) on the periodic lattice, |d| < n along each axis
__device__ __forceinline__ int at(const Geo& g, int x, int y, int z, int dx, int dy, int dz) {
  x += dx; y += dy; z += dz;
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
  return (z * g.ny + y) * g.nx + x;
}

// calls fn(x, y, z, node) for every node this thread owns
template <class Fn>
__device__ __forceinline__ void for_nodes(const Geo& g, Fn&& fn) {
  const int rows = g.ny * g.nz;
  for (int r = blockIdx.y * WY + threadIdx.y; r < rows; r += gridDim.y * WY) {
    const int y = r % g.ny, z = r / g.ny;
    for (int x = blockIdx.x * WX + threadIdx.x; x < g.nx; x += gridDim.x * WX) fn(x, y, z, r * g.nx + x);
  }
}

template <int LAT, typename Tr>
__global__ void __launch_bounds__(WT) k_wall_fill(Geo g, const signed char* __restrict__ layer, int L, Tr* rho) {
  using Lt = Lattice<LAT>;
  constexpr int Q = LAT == 0 ? 9 : 19;
  for_nodes(g, [&](int x, int y, int z, int n) {
    if (layer[n] != L) return;
    double num = 0, den = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int t = at(g, x, y, z, Lt::ex(i), Lt::ey(i), Lt::ez(i));
      if (layer[t] == L - 1) {
        num += Lt::w(i) * double(rho[t]);
        den += Lt::w(i);
      }
    }
    rho[n] = Tr(num / den);  // deviations average like densities (normalised weights)
  });
}

template <int LAT, int S, class P>
__global__ void __launch_bounds__(WT) k_wall_mu(Geo g, KParams p, const signed char* __restrict__ layer,
                                                const typename P::Tr* __restrict__ rho, double mu_w,
                                                typename P::Tm* mu) {
  using Tm = typename P::Tm;
  constexpr int D = LAT == 0 ? 2 : 3, R = Sch<S>::R;
  for_nodes(g, [&](int x, int y, int z, int n) {
    if (layer[n] != 0) {
      mu[n] = Tm(mu_w);
      return;
    }
    // Laplacian of the stored values (deviations in FP32DEV: the weights sum to zero)
    auto st = [&](int dx, int dy, int dz) { return Tm(rho[at(g, x, y, z, dx, dy, dz)]); };
    const Tm c0 = Tm(rho[n]);
    Tm lap = Tm(D * Sch<S>::l(0)) * c0;
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      Tm s = (st(m, 0, 0) + st(-m, 0, 0)) + (st(0, m, 0) + st(0, -m, 0));
      if (D == 3) s += st(0, 0, m) + st(0, 0, -m);
      lap += Tm(Sch<S>::l(m)) * s;
    }
    const Tm c = P::DEV ? Tm(p.rho_ref) + c0 : c0;
    mu[n] = Tm(p.k2) * eos_mu<Tm>(c, p) - Tm(p.kappa) * lap;
  });
}

// mode 0: collide and stream; mode 1: F (D x N) and mu (N) as FP64 fields
template <int LAT, int S, class P>
__global__ void __launch_bounds__(WT) k_wall_coll(Geo g, KParams p, Mrt mrt, const signed char* __restrict__ layer,
                                                  const typename P::Tf* __restrict__ fin,
                                                  typename P::Tf* __restrict__ fout,
                                                  const typename P::Tr* __restrict__ rho,
                                                  const typename P::Tm* __restrict__ mu, unsigned long long* bad,
                                                  long long t, int mode, double* F, double* muo) {
  using Lt = Lattice<LAT>;
  using Tc = typename P::Tc;
  using Tm = typename P::Tm;
  using Tf = typename P::Tf;
  constexpr int Q = LAT == 0 ? 9 : 19, D = LAT == 0 ? 2 : 3, R = Sch<S>::R;
  const int N = g.n;
  for_nodes(g, [&](int x, int y, int z, int n) {
    if (layer[n] != 0) {
      if (mode == 1) {  // no force on wall nodes; their mu is mu_w
        for (int a = 0; a < D; ++a) F[a * N + n] = 0.0;
        if (muo) muo[n] = double(mu[n]);
      }
      return;
    }
    Tc fv[Q];
    Tc j[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      fv[i] = Tc(fin[i * N + n]);
      if (Lt::ex(i) != 0) j[0] += Tc(Lt::ex(i)) * fv[i];
      if (Lt::ey(i) != 0) j[1] += Tc(Lt::ey(i)) * fv[i];
      if (Lt::ez(i) != 0) j[2] += Tc(Lt::ez(i)) * fv[i];
    }
    const Tc dsv = Tc(rho[n]);
    const Tc rc = P::DEV ? Tc(p.rho_ref) + dsv : dsv;
    Tc Fv[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      Tm gm = 0;
      Tc gr = 0;
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const int pp = at(g, x, y, z, a == 0 ? m : 0, a == 1 ? m : 0, a == 2 ? m : 0);
        const int qq = at(g, x, y, z, a == 0 ? -m : 0, a == 1 ? -m : 0, a == 2 ? -m : 0);
        gm += Tm(Sch<S>::g(m)) * (mu[pp] - mu[qq]);
        gr += Tc(Sch<S>::g(m)) * (Tc(rho[pp]) - Tc(rho[qq]));
      }
      Fv[a] = -rc * Tc(gm) + gr / Tc(3);
    }
    if (mode == 1) {
      for (int a = 0; a < D; ++a) F[a * N + n] = double(Fv[a]);
      if (muo) muo[n] = double(mu[n]);
      return;
    }
    if (!(rc > Tc(0))) atomicMin(bad, (unsigned long long)t);
    const Tc ux = j[0] / rc, uy = j[1] / rc, uz = j[2] / rc;
    const Tc vx = ux + Fv[0] / rc, vy = uy + Fv[1] / rc, vz = uz + Fv[2] / rc;
    Tc post[Q];
    bool done = false;
    if constexpr (LAT == 0) {
      if (mrt.on) {
        mrt_post9<Tc>(fv, dsv, rc, ux, uy, vx, vy, mrt, post);
        done = true;
      }
    }
    if (!done) {
#pragma unroll
      for (int i = 0; i < Q; ++i) post[i] = coll_one<LAT, Tc>(i, fv[i], dsv, rc, Tc(p.omega), ux, uy, uz, vx, vy, vz);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int tg = at(g, x, y, z, Lt::ex(i), Lt::ey(i), Lt::ez(i));
      if (layer[tg] != 0) {
        // halfway bounce-back: the population returns to this node reversed
        int o = 0;
#pragma unroll
        for (int k = 0; k < Q; ++k)
          if (Lt::ex(k) == -Lt::ex(i) && Lt::ey(k) == -Lt::ey(i) && Lt::ez(k) == -Lt::ez(i)) o = k;
        fout[o * N + n] = Tf(post[i]);
      } else {
        fout[i * N + tg] = Tf(post[i]);
      }
    }
  });
}

template <int LAT, class P>
__global__ void __launch_bounds__(WT) k_wall_dens(Geo g, KParams p, const signed char* __restrict__ layer,
                                                  const typename P::Tf* __restrict__ f, typename P::Tr* rho,
                                                  unsigned long long* bad, long long t) {
  constexpr int Q = LAT == 0 ? 9 : 19;
  for_nodes(g, [&](int, int, int, int n) {
    if (layer[n] != 0) return;
    double s = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) s += double(f[i * g.n + n]);
    rho[n] = typename P::Tr(s);
    const double full = P::DEV ? p.rho_ref + s : s;
    if (!(full > 0)) atomicMin(bad, (unsigned long long)t);
  });
}

// observables over fluid nodes, one partial per CTA: max |v| (v = u + F/(2 rho)),
// max |u|, mass, max |rho - snap|
template <int LAT, int S, class P>
__global__ void __launch_bounds__(WT) k_wall_obs(Geo g, KParams p, const signed char* __restrict__ layer,
                                                 const typename P::Tf* __restrict__ f,
                                                 const typename P::Tr* __restrict__ rho,
                                                 const typename P::Tm* __restrict__ mu,
                                                 const typename P::Tr* __restrict__ snap, double* part,
                                                 unsigned long long* bad, long long t) {
  using Lt = Lattice<LAT>;
  constexpr int Q = LAT == 0 ? 9 : 19, D = LAT == 0 ? 2 : 3, R = Sch<S>::R;
  __shared__ double red[4][WT];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const int N = g.n;
  for_nodes(g, [&](int x, int y, int z, int n) {
    if (layer[n] != 0) return;
    double j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      const double fi = double(f[i * N + n]);
      j[0] += Lt::ex(i) * fi;
      j[1] += Lt::ey(i) * fi;
      j[2] += Lt::ez(i) * fi;
    }
    const double rc = P::DEV ? p.rho_ref + double(rho[n]) : double(rho[n]);
    double uu = 0, vv = 0;
    for (int a = 0; a < 3; ++a) {
      double Fa = 0;
      if (a < D) {
        double gm = 0, gr = 0;
        for (int m = 1; m <= R; ++m) {
          const int pp = at(g, x, y, z, a == 0 ? m : 0, a == 1 ? m : 0, a == 2 ? m : 0);
          const int qq = at(g, x, y, z, a == 0 ? -m : 0, a == 1 ? -m : 0, a == 2 ? -m : 0);
          gm += Sch<S>::g(m) * (double(mu[pp]) - double(mu[qq]));
          gr += Sch<S>::g(m) * (double(rho[pp]) - double(rho[qq]));
        }
        Fa = -rc * gm + gr / 3.0;
      }
      const double ua = j[a] / rc, va = ua + Fa / (2.0 * rc);
      uu += ua * ua;
      vv += va * va;
    }
    a0 = fmax(a0, sqrt(vv));
    a1 = fmax(a1, sqrt(uu));
    a2 += rc;
    a3 = fmax(a3, fabs(double(rho[n]) - double(snap[n])));
    if (!(rc > 0.0)) atomicMin(bad, (unsigned long long)t);
  });
  const int tid = threadIdx.y * WX + threadIdx.x;
  red[0][tid] = a0; red[1][tid] = a1; red[2][tid] = a2; red[3][tid] = a3;
  __syncthreads();
  for (int s = WT / 2; s > 0; s >>= 1) {
    if (tid < s) {
      red[0][tid] = fmax(red[0][tid], red[0][tid + s]);
      red[1][tid] = fmax(red[1][tid], red[1][tid + s]);
      red[2][tid] += red[2][tid + s];
      red[3][tid] = fmax(red[3][tid], red[3][tid + s]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    for (int q = 0; q < 4; ++q) part[4 * b + q] = red[q][0];
  }
}

// grid over (x, row) with at most max_ctas CTAs (both axes grid-strided)
dim3 wall_grid(const Geo& g, int max_ctas) {
  const int gx = std::min((g.nx + WX - 1) / WX, max_ctas);
  const int rows = g.ny * g.nz;
  const int gy = std::max(1, std::min({(rows + WY - 1) / WY, max_ctas / gx, 65535}));
  return dim3(unsigned(gx), unsigned(gy));
}

template <int LAT, int S, class P>
cudaError_t wall_run(const WallLaunch& w, int mode, int* nblocks) {
  const Geo g{w.c.kp.nx, w.c.kp.ny, w.c.kp.nz, int(w.c.kp.n)};
  using Tr = typename P::Tr;
  using Tf = typename P::Tf;
  using Tm = typename P::Tm;
  const dim3 blk(WX, WY), grid = wall_grid(g, 1 << 20);
  cudaStream_t st = w.c.stream;
  Tr* rin = static_cast<Tr*>(const_cast<void*>(w.c.rin));  // wall layers are refreshed in place
  for (int L = 1; L <= 3; ++L) k_wall_fill<LAT, Tr><<<grid, blk, 0, st>>>(g, w.layer, L, rin);
  if (mode == MODE_WALL_FILL) return cudaGetLastError();
  k_wall_mu<LAT, S, P><<<grid, blk, 0, st>>>(g, w.c.kp, w.layer, rin, w.mu_w, static_cast<Tm*>(w.mu));
  if (mode == MODE_OBS) {
    const dim3 og = wall_grid(g, 4096);
    if (nblocks) *nblocks = int(og.x * og.y);
    k_wall_obs<LAT, S, P><<<og, blk, 0, st>>>(g, w.c.kp, w.layer, static_cast<const Tf*>(w.c.fin), rin,
                                             static_cast<const Tm*>(w.mu), static_cast<const Tr*>(w.c.aux.rho_snap),
                                             w.c.aux.partials, w.c.aux.bad_step, w.c.aux.t);
    return cudaGetLastError();
  }
  const int cm = mode == MODE_FIELDS ? 1 : 0;
  k_wall_coll<LAT, S, P><<<grid, blk, 0, st>>>(g, w.c.kp, w.c.mrt, w.layer, static_cast<const Tf*>(w.c.fin),
                                              static_cast<Tf*>(w.c.fout), rin, static_cast<const Tm*>(w.mu),
                                              w.c.aux.bad_step, w.c.aux.t, cm, w.c.fo.F, w.c.fo.mu);
  if (mode == MODE_STEP)
    k_wall_dens<LAT, P><<<grid, blk, 0, st>>>(g, w.c.kp, w.layer, static_cast<const Tf*>(w.c.fout),
                                             static_cast<Tr*>(w.c.rout), w.c.aux.bad_step, w.c.aux.t + 1);
  return cudaGetLastError();
}

template <int LAT, class P>
cudaError_t wall_by_scheme(const WallLaunch& w, int scheme, int mode, int* nb) {
  switch (scheme) {
    case S_EFDS2: return wall_run<LAT, S_EFDS2, P>(w, mode, nb);
    case S_EFDS4: return wall_run<LAT, S_EFDS4, P>(w, mode, nb);
    case S_EFDS6: return wall_run<LAT, S_EFDS6, P>(w, mode, nb);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t wall_step(const WallLaunch& w, int lattice, int scheme, int prec, int mode, int* nblocks) {
  if (mode != MODE_STEP && mode != MODE_OBS && mode != MODE_FIELDS && mode != MODE_WALL_FILL)
    return cudaErrorNotSupported;
  if (lattice == 0) {
    if (prec == 0) return wall_by_scheme<0, PrecF64>(w, scheme, mode, nblocks);
    if (prec == 1) return wall_by_scheme<0, PrecF32>(w, scheme, mode, nblocks);
    return wall_by_scheme<0, PrecF32M64>(w, scheme, mode, nblocks);
  }
  if (prec == 0) return wall_by_scheme<1, PrecF64>(w, scheme, mode, nblocks);
  if (prec == 1) return wall_by_scheme<1, PrecF32>(w, scheme, mode, nblocks);
  return wall_by_scheme<1, PrecF32M64>(w, scheme, mode, nblocks);
}

}  // namespace lbmd
