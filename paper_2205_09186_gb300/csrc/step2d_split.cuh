// D2Q9 FP32-deviation step as two passes (the 2D counterpart of
// step3d_split.cuh):
//
//  mu2d_tile    mu = k^2 psi'(rho) - kappa lap rho (Eq. 16) for one
//               32 x 16 RPT tile (halo R staged in shared memory).
//  coll2d_tile  grad mu, grad rho (Eq. 17-25) -> F (Eq. 12) -> BGK + EDM
//               (Eq. 1, 6, 8) -> push streaming and the next density for a
//               30 x (16 RPT - 2) tile; its 32 x 16 RPT tile-plus-ring region
//               maps one warp to RPT rows, w, w + 16, ... (512 threads, RPT
//               collisions per thread: with RPT = 2, the default, the
//               per-tile staging, barriers and bookkeeping are shared by twice
//               the nodes of RPT = 1, and the ring is 6% of the region's rows
//               instead of 12%).
//
// Both are device functions so that the single-case kernels and the
// persistent batch kernel share them.
#pragma once
#include "lbm_device.cuh"
#include "step2d.cuh"

namespace lbmd {

constexpr int NT2S = 512;                   // threads of both passes
constexpr int M2X = 32, C2X = 32;           // mu tile and collision region width
constexpr int T2X = C2X - 2;                // collision tile width
// Tile heights by rows per thread RPT (1, 2 or 4; 2 unless tuned): mu tile
// 32 x 16 RPT, collision region 32 x 16 RPT around a 30 x (16 RPT - 2) tile.
template <int RPT>
struct Tile2 {
  static constexpr int M2Y = 16 * RPT, C2Y = 16 * RPT, T2Y = C2Y - 2, C2N = C2X * C2Y;
};
constexpr int RPT_DEFAULT = 2;

template <int S, int RPT = RPT_DEFAULT>
struct Split2DShape {
  static constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, C2N = Tile2<RPT>::C2N;
  static constexpr int R = Sch<S>::R;
  static constexpr int MW = M2X + 2 * R, MH = M2Y + 2 * R;      // mu pass: density region
  static constexpr int GW = C2X + 2 * R, GH = C2Y + 2 * R;      // collision: field region
  static constexpr size_t mu_bytes = size_t(MW) * MH * 4;
  // compact schemes (GF): per collided node its density deviation (at 0) and
  // its four derivative values d_x mu, d_y mu, d_x rho, d_y rho (at off_mu,
  // component-major) instead of the two halo regions
  static constexpr bool GF = Sch<S>::GF;
  static constexpr size_t off_mu = GF ? size_t(C2N) * 4 : size_t(GW) * GH * 4;
  static constexpr size_t off_f = GF ? size_t(5) * C2N * 4 : (off_mu + size_t(GW) * GH * 4 + 15) / 16 * 16;
  static constexpr size_t coll_bytes = off_f + size_t(9) * C2N * 4;
  static constexpr size_t bytes = coll_bytes > mu_bytes ? coll_bytes : mu_bytes;
};

// Each pass is a load half (asynchronous copies into the tile's shared-memory
// buffer; the caller commits and waits) and a compute half, so that the batch
// kernel can copy its next tile while computing the current one.

template <int S, int RPT>
__device__ __forceinline__ void mu2d_load(const KParams& p, const float* __restrict__ rin, int x0, int y0,
                                          unsigned char* smem) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  using Sh = Split2DShape<S, RPT>;
  constexpr int R = Sh::R, MW = Sh::MW, MH = Sh::MH;
  static_assert(MW <= 64 && MW > 32, "two columns per lane");
  float* s = reinterpret_cast<float*>(smem);
  const int nx = p.nx, ny = p.ny;
  // warp w copies rows w, w + 16, ...; lane l columns l and 32 + l
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool two = lane + 32 < MW;
  const int xa = wrapn(x0 - R + lane, nx), xb = two ? wrapn(x0 - R + 32 + lane, nx) : 0;
  for (int ry = warp; ry < MH; ry += NT2S / 32) {
    const float* src = rin + wrapn(y0 - R + ry, ny) * nx;
    cpa4(s + ry * MW + lane, src + xa);
    if (two) cpa4(s + ry * MW + 32 + lane, src + xb);
  }
}

template <int S, int RPT>
__device__ __forceinline__ void mu2d_compute(const KParams& p, float* __restrict__ mu, int x0, int y0,
                                             const unsigned char* smem) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  using Sh = Split2DShape<S, RPT>;
  constexpr int R = Sh::R, MW = Sh::MW;
  const float* s = reinterpret_cast<const float*>(smem);
  const int nx = p.nx, ny = p.ny;
  const int tx = threadIdx.x % M2X;
  const float k2 = float(p.k2), kap = float(p.kappa);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int ty = threadIdx.x / M2X + r * (NT2S / M2X);
    if (x0 + tx < nx && y0 + ty < ny) {
      const float rho = float(p.rho_ref) + s[(ty + R) * MW + tx + R];
      const float lap = lap2d<S, float>(s, MW, tx + R, ty + R);
      mu[(y0 + ty) * nx + x0 + tx] = k2 * eos_mu_f(rho, eos_f(p)) - kap * lap;
    }
  }
}

// S a compact scheme (GF): gmu and grho are the derivative fields of the line
// solves (component-major, 2 N each); muf is not read.
template <int S, int RPT>
__device__ __forceinline__ void coll2d_load(const KParams& p, const float* __restrict__ fin,
                                            const float* __restrict__ rin, const float* __restrict__ muf, int x0,
                                            int y0, unsigned char* smem, const float* gmu = nullptr,
                                            const float* grho = nullptr) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  using Sh = Split2DShape<S, RPT>;
  constexpr int Q = 9, R = Sh::R, GW = Sh::GW, GH = Sh::GH;
  float* s_ds = reinterpret_cast<float*>(smem);
  float* s_mu = reinterpret_cast<float*>(smem + Sh::off_mu);
  float* s_f = reinterpret_cast<float*>(smem + Sh::off_f);
  const int nx = p.nx, ny = p.ny, N = int(p.n);
  const int VW = min(T2X, nx - x0), VH = min(T2Y, ny - y0);
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int node = tid + r * NT2S;  // region rows w and w + 16 of warp w
    const int cy = node / C2X, cx = node - cy * C2X;
    if (cx - 1 <= VW && cy - 1 <= VH) {  // collided node: stage its populations
      const int g = wrapi(y0 + cy - 1, ny) * nx + wrapi(x0 + cx - 1, nx);
      const float* fs = fin + g;
#pragma unroll
      for (int i = 0; i < Q; ++i) cpa4(s_f + i * C2N + node, fs + i * N);
      if constexpr (Sch<S>::GF) {
        // its density deviation and derivative values
        cpa4(s_ds + node, rin + g);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          cpa4(s_mu + a * C2N + node, gmu + a * N + g);
          cpa4(s_mu + (2 + a) * C2N + node, grho + a * N + g);
        }
      }
    }
  }
  if constexpr (Sch<S>::GF) return;
  // fields: warp w copies rows w, w + 16, ...; lane l columns l and 32 + l
  // (the region of a ragged tile only as far as its collided nodes reach)
  static_assert(Sch<S>::GF || (GW <= 64 && GW > 32), "two columns per lane");
  const int lane = tid & 31, warp = tid >> 5;
  const int xa = wrapi(x0 - 1 - R + lane, nx);
  const bool two = lane + 32 < GW && lane + 32 < VW + 2 + 2 * R;
  const int xb = two ? wrapi(x0 - 1 - R + 32 + lane, nx) : 0;
  const bool one = lane < VW + 2 + 2 * R;
  for (int ry = warp; ry < min(GH, VH + 2 + 2 * R); ry += NT2S / 32) {
    const int g = wrapi(y0 - 1 - R + ry, ny) * nx;
    if (one) {
      cpa4(s_ds + ry * GW + lane, rin + g + xa);
      cpa4(s_mu + ry * GW + lane, muf + g + xa);
    }
    if (two) {
      cpa4(s_ds + ry * GW + 32 + lane, rin + g + xb);
      cpa4(s_mu + ry * GW + 32 + lane, muf + g + xb);
    }
  }
}

template <int S, bool TAU1, int RPT>
__device__ __forceinline__ void coll2d_compute(const KParams& p, float* __restrict__ fout, float* __restrict__ rout,
                                               unsigned long long* bad, long long t, int x0, int y0,
                                               unsigned char* smem, const Mrt& mrt) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  using L = Lattice<0>;
  using Sh = Split2DShape<S, RPT>;
  constexpr int Q = 9, R = Sh::R, GW = Sh::GW;
  const float* s_ds = reinterpret_cast<const float*>(smem);
  const float* s_mu = reinterpret_cast<const float*>(smem + Sh::off_mu);
  float* s_f = reinterpret_cast<float*>(smem + Sh::off_f);
  const int nx = p.nx, ny = p.ny, N = int(p.n);
  const int VW = min(T2X, nx - x0), VH = min(T2Y, ny - y0);
  const float omega = float(p.omega), rref = float(p.rho_ref);
#pragma unroll 1
  for (int r = 0; r < RPT; ++r) {
    const int node = threadIdx.x + r * NT2S;  // region rows w and w + 16 of warp w
    const int cy = node / C2X, cx = node - cy * C2X;
    const int lx = cx - 1, ly = cy - 1;
    if (!(lx <= VW && ly <= VH)) continue;  // not a collided node
    const bool interior = lx >= 0 && lx < VW && ly >= 0 && ly < VH;
    const int gx = wrapi(x0 + lx, nx), gy = wrapi(y0 + ly, ny);
    float fv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fv[i] = s_f[i * C2N + node];
    const int c = (cy + R) * GW + cx + R;
    const float dsv = s_ds[c];
    const float rc = rref + dsv;
    float jx = 0.f, jy = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::ex(i) != 0) jx += float(L::ex(i)) * fv[i];
      if (L::ey(i) != 0) jy += float(L::ey(i)) * fv[i];
    }
    const float irc = __fdividef(1.f, rc);
    const float ux = jx * irc, uy = jy * irc;
    float gmx, gmy, grx, gry;
    if constexpr (Sch<S>::GF) {
      gmx = s_mu[node];
      gmy = s_mu[C2N + node];
      grx = s_mu[2 * C2N + node];
      gry = s_mu[3 * C2N + node];
    } else {
      grad2d<S, float>(s_mu, GW, cx + R, cy + R, gmx, gmy);
      grad2d<S, float>(s_ds, GW, cx + R, cy + R, grx, gry);
    }
    const float Fx = -rc * gmx + grx * (1.f / 3.f), Fy = -rc * gmy + gry * (1.f / 3.f);
    const float vx = ux + Fx * irc, vy = uy + Fy * irc;
    if (interior && !(rc > 0.f)) atomicMin(bad, (unsigned long long)t);
    const int dxp = (gx + 1 < nx) ? 1 : 1 - nx, dxm = (gx > 0) ? -1 : nx - 1;
    const int dyp = (gy + 1 < ny) ? nx : nx - N, dym = (gy > 0) ? -nx : N - nx;
    float* fo = fout + gy * nx + gx;
    if (mrt.on) {
      float post[Q];
      mrt_post9<float>(fv, dsv, rc, ux, uy, vx, vy, mrt, post);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        s_f[i * C2N + node] = post[i];
        if (interior) {
          const int d = (L::ex(i) > 0 ? dxp : (L::ex(i) < 0 ? dxm : 0)) + (L::ey(i) > 0 ? dyp : (L::ey(i) < 0 ? dym : 0));
          fo[i * N + d] = post[i];
        }
      }
    } else {
      const float vv15 = 1.5f * (vx * vx + vy * vy), uu15 = 1.5f * (ux * ux + uy * uy);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float w = float(L::w(i));
        const float ev = edot<L>(i, vx, vy, 0.f);
        const float Av = i == 0 ? -vv15 : ev * (3.f + 4.5f * ev) - vv15;
        float fs;
        if constexpr (TAU1) {
          fs = w * (dsv + rc * Av);
        } else {
          const float eu = edot<L>(i, ux, uy, 0.f);
          const float Au = i == 0 ? -uu15 : eu * (3.f + 4.5f * eu) - uu15;
          fs = (1.f - omega) * fv[i] + w * (omega * dsv + rc * (omega * Au + Av - Au));
        }
        s_f[i * C2N + node] = fs;
        if (interior) {
          const int d = (L::ex(i) > 0 ? dxp : (L::ex(i) < 0 ? dxm : 0)) + (L::ey(i) > 0 ? dyp : (L::ey(i) < 0 ? dym : 0));
          fo[i * N + d] = fs;
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int node = threadIdx.x + r * NT2S;
    const int cy = node / C2X, cx = node - cy * C2X;
    const int lx = cx - 1, ly = cy - 1;
    if (lx >= 0 && lx < VW && ly >= 0 && ly < VH) {
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) acc += s_f[i * C2N + node - L::ey(i) * C2X - L::ex(i)];
      rout[(y0 + ly) * nx + x0 + lx] = acc;
      if (!(rref + acc > 0.f)) atomicMin(bad, (unsigned long long)(t + 1));
    }
  }
}

// mu of 8 rows x 32 columns of a mu tile straight from global memory, for
// one warp (lane l: column x0 + l), every stencil value an L1-cached load.
// The stencil rows come from one table of wrapped row offsets, so a value that
// several of the eight rows use is loaded once, and the results are stored
// after the last load (with the buffers not marked __restrict__, a store
// between them would keep later loads behind it).  No shared memory and no
// barrier: the persistent batch kernel deals these units to warps.  The inputs
// are written earlier in the same persistent launch (by other CTAs, before a
// device-wide barrier with acquire semantics), so they are read with ordinary
// coherent loads, never through the non-coherent read-only path (no __ldg, no
// __restrict__).
constexpr int MU_UNIT_ROWS = 8;

template <int S>
__device__ __forceinline__ void mu2d_rows(const KParams& p, const float* rin, float* mu, int x0, int y0, int lane) {
  using Sc = Sch<S>;
  constexpr int R = Sc::R, U = MU_UNIT_ROWS;
  const int nx = p.nx, ny = p.ny;
  const int gx = x0 + lane;
  if (gx >= nx) return;
  const int nr = min(U, ny - y0);
  int xo[2 * R + 1];  // wrapped x of the stencil columns
#pragma unroll
  for (int d = -R; d <= R; ++d) xo[d + R] = wrapi(gx + d, nx);
  int ro[U + 2 * R];  // wrapped row offsets of rows y0 - R .. y0 + U + R - 1
#pragma unroll
  for (int k = 0; k < U + 2 * R; ++k) ro[k] = wrapn(y0 - R + k, ny) * nx;
  const float k2 = float(p.k2), kap = float(p.kappa), rref = float(p.rho_ref);
  const EosF ef = eos_f(p);
  float res[U];
#pragma unroll
  for (int r = 0; r < U; ++r) {
    auto at = [&](int dx, int dy) { return rin[ro[r + R + dy] + xo[dx + R]]; };
    const float c = at(0, 0);
    float lap;
    if constexpr (Sc::ISO) {
      lap = 0.f;
#pragma unroll
      for (int dy = -R; dy <= R; ++dy)
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
          const double w = Sc::w2d(dx, dy);
          if (w != 0.0) lap += float(2.0 * w) * (at(dx, dy) - c);
        }
    } else {
      lap = float(2.0 * Sc::l(0)) * c;
#pragma unroll
      for (int m = 1; m <= R; ++m) lap += float(Sc::l(m)) * ((at(m, 0) + at(-m, 0)) + (at(0, m) + at(0, -m)));
    }
    res[r] = k2 * eos_mu_f(rref + c, ef) - kap * lap;
  }
#pragma unroll
  for (int r = 0; r < U; ++r)
    if (r < nr) mu[(y0 + r) * nx + gx] = res[r];
}

// y-marching vector mu pass (line schemes EFDS2/4/6, nx % 4 == 0, 16-byte
// aligned fields): thread (tx, ty) of a 256-thread CTA owns four x-adjacent
// nodes (one float4, x = 64 blockIdx.x + 4 tx) through rpt consecutive rows.
// Its y neighbours sit in a register queue fed one row ahead by 16-byte loads;
// its x neighbours are the neighbouring lanes' centre chunks (shuffles within
// the 16-lane group that marches the same rows); a group's edge lanes load the
// chunk beyond it themselves.  No shared memory, no CTA barrier.
constexpr int YMT = 256;

template <int S>
__global__ void __launch_bounds__(YMT) k_mu2d_ym(const KParams p, const float* __restrict__ rin,
                                                 float* __restrict__ mu, const int rpt) {
  static_assert(!Sch<S>::ISO && Sch<S>::R <= 4, "line schemes, stencil within one chunk on each side");
  constexpr int R = Sch<S>::R;
  const int nx = p.nx, ny = p.ny;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int x = blockIdx.x * 64 + 4 * tx;
  const int ya = (blockIdx.y * (YMT / 16) + ty) * rpt;
  if (ya >= ny) return;  // the whole 16-lane group (same ty)
  const int yb = min(ya + rpt, ny);
  const unsigned gmask = 0xffffu << (16 * (ty & 1));  // this group's lanes
  const bool own = x < nx;
  const bool need_lo = tx == 0, need_hi = tx == 15 || x + 4 >= nx;
  auto ld = [&](int xx, int yy) {
    return __ldg(reinterpret_cast<const float4*>(rin + wrapn(yy, ny) * nx + wrapn(xx, nx)));
  };
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 q[2 * R + 1];
#pragma unroll
  for (int d = 1; d <= 2 * R; ++d) q[d] = own ? ld(x, ya - R - 1 + d) : z4;
  float4 pre = own ? ld(x, ya + R) : z4;
  float4 elo_n = own && need_lo ? ld(x - 4, ya) : z4, ehi_n = own && need_hi ? ld(x + 4, ya) : z4;
  const float k2 = float(p.k2), kap = float(p.kappa), rref = float(p.rho_ref);
  const EosF ef = eos_f(p);
  for (int y = ya; y < yb; ++y) {
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
    q[2 * R] = pre;
    const float4 elo = elo_n, ehi = ehi_n;
    if (own && y + 1 < yb) {
      pre = ld(x, y + R + 1);
      if (need_lo) elo_n = ld(x - 4, y + 1);
      if (need_hi) ehi_n = ld(x + 4, y + 1);
    }
    const float4 c4 = q[R];
    float4 lo, hi;
    lo.x = __shfl_up_sync(gmask, c4.x, 1, 16); lo.y = __shfl_up_sync(gmask, c4.y, 1, 16);
    lo.z = __shfl_up_sync(gmask, c4.z, 1, 16); lo.w = __shfl_up_sync(gmask, c4.w, 1, 16);
    hi.x = __shfl_down_sync(gmask, c4.x, 1, 16); hi.y = __shfl_down_sync(gmask, c4.y, 1, 16);
    hi.z = __shfl_down_sync(gmask, c4.z, 1, 16); hi.w = __shfl_down_sync(gmask, c4.w, 1, 16);
    if (need_lo) lo = elo;
    if (need_hi) hi = ehi;
    if (!own) continue;
    const float row[12] = {lo.x, lo.y, lo.z, lo.w, c4.x, c4.y, c4.z, c4.w, hi.x, hi.y, hi.z, hi.w};
    float res[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float cv = row[4 + k];
      float lap = float(2.0 * Sch<S>::l(0)) * cv;
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float4 e = q[R + m], f = q[R - m];
        const float ym = k == 0 ? e.x + f.x : (k == 1 ? e.y + f.y : (k == 2 ? e.z + f.z : e.w + f.w));
        lap += float(Sch<S>::l(m)) * ((row[4 + k + m] + row[4 + k - m]) + ym);
      }
      res[k] = k2 * eos_mu_f(rref + cv, ef) - kap * lap;
    }
    *reinterpret_cast<float4*>(mu + y * nx + x) = make_float4(res[0], res[1], res[2], res[3]);
  }
}

// whole tiles (load, wait, compute) for the single-case kernels
template <int S, int RPT>
__device__ __forceinline__ void mu2d_tile(const KParams& p, const float* __restrict__ rin, float* __restrict__ mu,
                                          int x0, int y0, unsigned char* smem) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  mu2d_load<S, RPT>(p, rin, x0, y0, smem);
  cpa_commit();
  cpa_wait_all();
  __syncthreads();
  mu2d_compute<S, RPT>(p, mu, x0, y0, smem);
}

template <int S, bool TAU1, int RPT>
__device__ __forceinline__ void coll2d_tile(const KParams& p, const float* __restrict__ fin, float* __restrict__ fout,
                                            const float* __restrict__ rin, const float* __restrict__ muf,
                                            float* __restrict__ rout, unsigned long long* bad, long long t, int x0,
                                            int y0, unsigned char* smem, const Mrt& mrt) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  coll2d_load<S, RPT>(p, fin, rin, muf, x0, y0, smem);
  cpa_commit();
  cpa_wait_all();
  __syncthreads();
  coll2d_compute<S, TAU1, RPT>(p, fout, rout, bad, t, x0, y0, smem, mrt);
}

template <int S, int RPT>
__global__ void __launch_bounds__(NT2S) k_mu2d(const KParams p, const float* __restrict__ rin, float* __restrict__ mu) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  extern __shared__ __align__(16) unsigned char smem[];
  mu2d_tile<S, RPT>(p, rin, mu, blockIdx.x * M2X, blockIdx.y * M2Y, smem);
}

template <int S, bool TAU1, int RPT>
__global__ void __launch_bounds__(NT2S) k_coll2d(const KParams p, const float* __restrict__ fin,
                                                 float* __restrict__ fout, const float* __restrict__ rin,
                                                 const float* __restrict__ mu, float* __restrict__ rout,
                                                 const StepAux aux, const Mrt mrt) {
  [[maybe_unused]] constexpr int M2Y = Tile2<RPT>::M2Y, C2Y = Tile2<RPT>::C2Y, T2Y = Tile2<RPT>::T2Y, C2N = Tile2<RPT>::C2N;
  extern __shared__ __align__(16) unsigned char smem[];
  coll2d_tile<S, TAU1, RPT>(p, fin, fout, rin, mu, rout, aux.bad_step, aux.t, blockIdx.x * T2X, blockIdx.y * T2Y, smem,
                       mrt);
}

}  // namespace lbmd
