// The mu pass of the D3Q19 FP32-deviation step (mu = k^2 psi'(rho) - kappa
// lap rho, Eq. 16, once per node) and the node-parallel observation pass that
// reads the mu field.
#pragma once
#include "lbm_device.cuh"
#include "step2d.cuh"
#include "step3d.cuh"
#include "step3d_fast.cuh"

namespace lbmd {

// ------------------------------------------------------------------ row bands
// The collision pass (k_coll3d) cuts the lattice's rows into bands of ry rows
// (the last band may be shorter); band b holds rows [start(b), start(b + 1)).
// A last band of a single row takes one row from the band before it, so that
// every band has two distinct edge rows unless ny = 1.  The next density of a
// band's first and last rows is completed by two atomic additions onto zero:
// one from the band itself and one from the band that streams into the row
// from the other side.  The mu pass that precedes the collision pass in the
// same step zeroes those rows of the output density (EdgeZero below).
struct RowBands {
  int ny, ry, nb, adj;
  __host__ __device__ RowBands(int ny_, int ry_) : ny(ny_), ry(ry_), nb((ny_ + ry_ - 1) / ry_), adj(0) {
    if (nb >= 2 && ny - (nb - 1) * ry == 1) adj = 1;
  }
  __host__ __device__ int start(int b) const { return b >= nb ? ny : b * ry - (b == nb - 1 ? adj : 0); }
  __host__ __device__ int band(int y) const {
    const int b = y / ry < nb - 1 ? y / ry : nb - 1;
    return (adj && b == nb - 2 && y >= start(nb - 1)) ? nb - 1 : b;
  }
  __host__ __device__ bool edge(int y) const {
    const int b = band(y);
    return y == start(b) || y == start(b + 1) - 1;
  }
};

// Column tiles of the collision pass: 32 columns each (one warp lane per
// column), the last one ragged.  A last tile of a single column (nx % 32 == 1,
// odd nx, so never on the 16-byte paths) takes one column from the tile
// before it, so that every tile has two distinct edge columns.
struct ColTiles {
  int nx, nt, adj;
  __host__ __device__ explicit ColTiles(int nx_) : nx(nx_), nt((nx_ + 31) / 32), adj(0) {
    if (nt >= 2 && nx - (nt - 1) * 32 == 1) adj = 1;
  }
  __host__ __device__ int start(int t) const { return t >= nt ? nx : 32 * t - (t == nt - 1 ? adj : 0); }
  __host__ __device__ int tile(int x) const {
    const int t = x / 32 < nt - 1 ? x / 32 : nt - 1;
    return (adj && t == nt - 2 && x >= start(nt - 1)) ? nt - 1 : t;
  }
  __host__ __device__ bool edge(int x) const {
    const int t = tile(x);
    return x == start(t) || x == start(t + 1) - 1;
  }
};

// What the mu pass does for the collision pass that follows it: zero the
// nodes of the collision pass's output density rz that it completes by atomic
// additions (the edge rows of its row bands of ry rows and the edge columns of
// its column tiles), and flag step t in bad when the density of such a node is
// not positive (the collision pass checks the other nodes of the density it
// produces, flagging the same step index).  rz == nullptr: nothing.
struct EdgeZero {
  float* rz;
  int ry;
  unsigned long long* bad;
  long long t;
};

// ------------------------------------------------------------------ mu pass
// One CTA: a 32 x 8 x 8 block of nodes.  The block and its stencil halo are
// copied to shared memory in one asynchronous batch (every copy of the CTA in
// flight at once: no per-plane round trip), then each thread walks its column
// through the 8 planes with the z neighbours in a register queue.
constexpr int MUX = 32, MUY = 8, MUZ = 8, MUT = MUX * MUY;

// M64: the EOS chemical potential k^2 psi'(rho) evaluated in FP64 from
// rho = rho_ref + deviation (FP64 division and logarithm), the Laplacian term
// in FP32 as with M64 off, the sum rounded once to the float mu field.
template <bool M64>
__device__ __forceinline__ float mu_value(const KParams& p, const EosF& ef, float k2, float kap, float rref, float dev,
                                          float lap) {
  if constexpr (M64)
    return float(p.k2 * eos_mu<double>(p.rho_ref + double(dev), p) - p.kappa * double(lap));
  else
    return k2 * eos_mu_f(rref + dev, ef) - kap * lap;
}

// line schemes only (the isotropic 3D Laplacian needs diagonal neighbours)
template <int S, bool M64 = false>
__global__ void __launch_bounds__(MUT) k_mu3d(const KParams p, const float* __restrict__ rin,
                                              float* __restrict__ mu, const EdgeZero ez) {
  static_assert(!Sch<S>::ISO, "line schemes only");
  constexpr int R = Sch<S>::R;
  constexpr int PW = MUX + 2 * R, PH = MUY + 2 * R, PD = MUZ + 2 * R;
  static_assert(MUT / 32 < PH && PH + PD <= MUT, "row walk and offset tables");
  __shared__ float blk[PD][PH][PW];
  __shared__ int s_yo[PH], s_zo[PD];  // wrapped row and plane offsets of the block
  const int nx = p.nx, ny = p.ny, nz = p.nz, NXY = nx * ny;
  const int x0 = blockIdx.x * MUX, y0 = blockIdx.y * MUY, z0 = blockIdx.z * MUZ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < PH) s_yo[threadIdx.x] = wrapn(y0 - R + int(threadIdx.x), ny) * nx;
  else if (threadIdx.x < PH + PD) s_zo[threadIdx.x - PH] = wrapn(z0 - R + int(threadIdx.x) - PH, nz) * NXY;
  // x sources of this lane (lanes < 2R also fill the two columns past 32)
  const int xa = wrapn(x0 - R + lane, nx);
  const int xb = wrapn(x0 - R + 32 + min(lane, 2 * R - 1), nx);
  __syncthreads();
  // rows warp, warp + 8, ...: (rz, ry) advanced incrementally (8 < PH)
  int ry = warp, rz = 0;
  float* dst = &blk[0][warp][lane];
  for (int row = warp; row < PH * PD; row += MUT / 32) {
    const float* src = rin + (s_zo[rz] + s_yo[ry]);
    cpa4(dst, src + xa);
    if (lane < 2 * R) cpa4(dst + 32, src + xb);
    dst += (MUT / 32) * PW;
    ry += MUT / 32;
    if (ry >= PH) { ry -= PH; ++rz; }
  }
  cpa_commit();
  cpa_wait_all();
  __syncthreads();
  const int tx = threadIdx.x % MUX, ty = threadIdx.x / MUX;
  if (x0 + tx >= nx || y0 + ty >= ny) return;
  const float k2 = float(p.k2), kap = float(p.kappa);
  const EosF ef = eos_f(p);
  const float rref = float(p.rho_ref);
  const int cx = tx + R, cy = ty + R;
  float q[2 * R + 1];  // q[R + d]: density deviation at plane z + d of this column
#pragma unroll
  for (int d = 0; d < 2 * R; ++d) q[d + 1] = blk[d][cy][cx];
  const int zend = min(MUZ, nz - z0);
  float* out = mu + z0 * NXY + (y0 + ty) * nx + x0 + tx;
  const bool enode = ez.rz && (RowBands(ny, ez.ry).edge(y0 + ty) || ColTiles(nx).edge(x0 + tx));
#pragma unroll
  for (int dz = 0; dz < MUZ; ++dz) {
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
    q[2 * R] = blk[dz + 2 * R][cy][cx];
    if (dz < zend) {
      const int pz = dz + R;
      const float c = q[R];
      float lap = float(3.0 * Sch<S>::l(0)) * c;
#pragma unroll
      for (int m = 1; m <= R; ++m)
        lap += float(Sch<S>::l(m)) * ((blk[pz][cy][cx + m] + blk[pz][cy][cx - m]) +
                                      (blk[pz][cy + m][cx] + blk[pz][cy - m][cx]) + (q[R + m] + q[R - m]));
      out[dz * NXY] = mu_value<M64>(p, ef, k2, kap, rref, c, lap);
      if (enode) {
        ez.rz[(out - mu) + dz * NXY] = 0.f;
        if (!(rref + c > 0.f)) atomicMin(ez.bad, (unsigned long long)ez.t);
      }
    }
  }
}

// Vector variant (nx % 4 == 0, 16-byte aligned fields), z-marching: a CTA
// owns a 64 x 16 column of nodes (four x-adjacent nodes per thread, one
// float4) through a chunk of zc planes.  Only the current plane, with its x-y
// halo, sits in shared memory, double-buffered (the next plane's 16-byte
// copies are in flight while this one is computed); the z neighbours of a
// thread's nodes come from a register queue fed by one 16-byte load per
// plane, issued one plane ahead.  (Timed against alternatives on a 256^3
// field, L2 flushed between launches: a 64 x 8 x 8 block with its full 3D
// halo, 0.066 ms; this kernel, 0.055 ms; deeper copy or queue pipelines, and
// a queue fed from a ring of staged planes, were slower.)
constexpr int MZX = 64, MZY = 16, MZT = (MZX / 4) * MZY;

template <int S>
struct MuZShape {
  static constexpr int R = Sch<S>::R;
  static constexpr int NCH = MZX / 4 + 2;  // chunks per row: x0 - 4 .. x0 + 67
  static constexpr int PH = MZY + 2 * R;   // rows per plane
  static constexpr int PCH = PH * NCH;     // chunks per plane
  static constexpr size_t bytes = size_t(2) * PCH * 16;
};

template <int S, bool M64 = false>
__global__ void __launch_bounds__(MZT) k_mu3d_zm(const KParams p, const float* __restrict__ rin,
                                                 float* __restrict__ mu, const int zc, const EdgeZero ez) {
  static_assert(!Sch<S>::ISO, "line schemes only");
  using Sh = MuZShape<S>;
  constexpr int R = Sh::R, NCH = Sh::NCH, PH = Sh::PH, PCH = Sh::PCH, KC = (PCH + MZT - 1) / MZT;
  static_assert(R <= 4 && PH <= MZT, "stencil within one chunk on each side; row table");
  extern __shared__ __align__(16) float4 pl4[];  // [2][PH][NCH]
  __shared__ int s_yo[PH];
  const int nx = p.nx, ny = p.ny, nz = p.nz, NXY = nx * ny;
  const int x0 = blockIdx.x * MZX, y0 = blockIdx.y * MZY, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const int tid = threadIdx.x;
  if (tid < PH) s_yo[tid] = wrapn(y0 - R + tid, ny) * nx;
  __syncthreads();
  // x-y source offset of each of this thread's chunks (fixed through the march)
  int cof[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int c = tid + k * MZT;
    const int ry = c / NCH, j = c - ry * NCH;
    cof[k] = c < PCH ? s_yo[ry] + wrapn(x0 - 4 + 4 * j, nx) : 0;
  }
  auto issue = [&](int z, int b) {
    const float* src = rin + wrapi(z, nz) * NXY;
    float4* dst = pl4 + b * PCH;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const int c = tid + k * MZT;
      if (c < PCH) cpa16(dst + c, src + cof[k]);
    }
    cpa_commit();
  };
  const int tx = tid % (MZX / 4), ty = tid / (MZX / 4);
  const bool own = x0 + 4 * tx < nx && y0 + ty < ny;  // nx % 4 == 0: all four nodes or none
  const int col = own ? (y0 + ty) * nx + x0 + 4 * tx : 0;
  // this thread's four nodes hold a node of an edge row or an edge column:
  // all four are zeroed (the others are stored by the collision pass before
  // anything reads them) and checked
  bool erow = ez.rz && own && RowBands(ny, ez.ry).edge(y0 + ty);
  if (ez.rz && own && !erow) {
    const ColTiles ct(nx);
#pragma unroll
    for (int k = 0; k < 4; ++k) erow = erow || ct.edge(x0 + 4 * tx + k);
  }
  bool ebad = false;
  auto ld = [&](int z) { return __ldg(reinterpret_cast<const float4*>(rin + wrapi(z, nz) * NXY + col)); };
  const float k2 = float(p.k2), kap = float(p.kappa);
  const EosF ef = eos_f(p);
  const float rref = float(p.rho_ref);
  issue(z0, 0);
  float4 q[2 * R + 1];  // q[R + d]: the four nodes' deviations at plane z + d
  float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
  if (own) {
#pragma unroll
    for (int d = 1; d <= 2 * R; ++d) q[d] = ld(z0 - R - 1 + d);
    nxt = ld(z0 + R);
  }
  const int cy = ty + R;
  for (int z = z0; z < z1; ++z) {
    const int b = (z - z0) & 1;
    cpa_wait_all();
    __syncthreads();
    if (z + 1 < z1) issue(z + 1, b ^ 1);  // into the buffer read before the barrier
    if (!own) continue;
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
    q[2 * R] = nxt;
    if (z + 1 < z1) nxt = ld(z + R + 1);
    const float4* pb = pl4 + b * PCH;
    const float4 lo = pb[cy * NCH + tx], hi = pb[cy * NCH + tx + 2], c4 = q[R];
    const float row[12] = {lo.x, lo.y, lo.z, lo.w, c4.x, c4.y, c4.z, c4.w, hi.x, hi.y, hi.z, hi.w};
    float yz[4][R];
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      const float4 a = pb[(cy + m) * NCH + 1 + tx], bb = pb[(cy - m) * NCH + 1 + tx], e = q[R + m], f = q[R - m];
      yz[0][m - 1] = (a.x + bb.x) + (e.x + f.x);
      yz[1][m - 1] = (a.y + bb.y) + (e.y + f.y);
      yz[2][m - 1] = (a.z + bb.z) + (e.z + f.z);
      yz[3][m - 1] = (a.w + bb.w) + (e.w + f.w);
    }
    float res[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float cv = row[4 + k];
      float lap = float(3.0 * Sch<S>::l(0)) * cv;
#pragma unroll
      for (int m = 1; m <= R; ++m) lap += float(Sch<S>::l(m)) * ((row[4 + k + m] + row[4 + k - m]) + yz[k][m - 1]);
      res[k] = mu_value<M64>(p, ef, k2, kap, rref, cv, lap);
    }
    *reinterpret_cast<float4*>(mu + z * NXY + col) = make_float4(res[0], res[1], res[2], res[3]);
    if (erow) {
      *reinterpret_cast<float4*>(ez.rz + z * NXY + col) = make_float4(0.f, 0.f, 0.f, 0.f);
      ebad |= !(rref + c4.x > 0.f && rref + c4.y > 0.f && rref + c4.z > 0.f && rref + c4.w > 0.f);
    }
  }
  // one flag per thread through the march, one atomic after it (an atomic
  // inside the march cost it 30 registers)
  if (erow && ebad) atomicMin(ez.bad, (unsigned long long)ez.t);
}

// ------------------------------------------------------------------ observation pass
// max |v| (v = u + F/(2 rho)), max |u|, mass and max |rho - rho_snap| of the
// current state from the populations, the density deviation and the mu field
// (computed by k_mu3d); stencil neighbours are read through L1/L2.  One CTA
// walks x-rows (grid-stride over the ny * nz rows, fixed grid); the node values
// are FP32 like the step, the mass a compensated FP32 sum per thread, the CTA
// partials FP64.
template <int S>
__global__ void __launch_bounds__(256) k_obs3d(const KParams p, const float* __restrict__ f,
                                               const float* __restrict__ rin, const float* __restrict__ muf,
                                               const StepAux aux) {
  using L = Lattice<1>;
  constexpr int R = Sch<S>::R;
  const int nx = p.nx, ny = p.ny, nz = p.nz, N = int(p.n);
  const float rref = float(p.rho_ref);
  float o_vmax = 0.f, o_umax = 0.f, o_dmax = 0.f;
  FSum o_dev;   // sum of the density deviations
  int cnt = 0;  // nodes visited (mass = cnt * rho_ref + deviations)
  const float* snap = static_cast<const float*>(aux.rho_snap);
  bool bad = false;
  for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
    const int z = row / ny, y = row - z * ny;
    int ym[R], yp[R], zm[R], zp[R];
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      ym[m - 1] = (z * ny + wrapi(y - m, ny)) * nx;  // m <= 3 < 8 <= ny, nz: one period
      yp[m - 1] = (z * ny + wrapi(y + m, ny)) * nx;
      zm[m - 1] = (wrapi(z - m, nz) * ny + y) * nx;
      zp[m - 1] = (wrapi(z + m, nz) * ny + y) * nx;
    }
    const int rowb = row * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const int n = rowb + x;
      float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const float fi = f[i * N + n];
        if (L::ex(i) != 0) jx += float(L::ex(i)) * fi;
        if (L::ey(i) != 0) jy += float(L::ey(i)) * fi;
        if (L::ez(i) != 0) jz += float(L::ez(i)) * fi;
      }
      const float dsv = rin[n];
      const float rc = rref + dsv;
      float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, gr0 = 0.f, gr1 = 0.f, gr2 = 0.f;
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float g = float(Sch<S>::g(m));
        const int xp = rowb + wrapi(x + m, nx), xm = rowb + wrapi(x - m, nx);
        const int yq = yp[m - 1] + x, yr = ym[m - 1] + x, zq = zp[m - 1] + x, zr = zm[m - 1] + x;
        gm0 += g * (muf[xp] - muf[xm]); gm1 += g * (muf[yq] - muf[yr]); gm2 += g * (muf[zq] - muf[zr]);
        gr0 += g * (rin[xp] - rin[xm]); gr1 += g * (rin[yq] - rin[yr]); gr2 += g * (rin[zq] - rin[zr]);
      }
      const float irc = __fdividef(1.f, rc);
      const float ux = jx * irc, uy = jy * irc, uz = jz * irc;
      const float h = 0.5f * irc;
      const float vx = ux + (-rc * gm0 + gr0 * (1.f / 3.f)) * h, vy = uy + (-rc * gm1 + gr1 * (1.f / 3.f)) * h,
                  vz = uz + (-rc * gm2 + gr2 * (1.f / 3.f)) * h;
      o_vmax = fmaxf(o_vmax, sqrtf(vx * vx + vy * vy + vz * vz));
      o_umax = fmaxf(o_umax, sqrtf(ux * ux + uy * uy + uz * uz));
      o_dev.add(dsv);
      ++cnt;
      o_dmax = fmaxf(o_dmax, fabsf(dsv - snap[n]));
      bad |= !(rc > 0.f);
    }
  }
  if (bad) atomicMin(aux.bad_step, (unsigned long long)aux.t);
  block_obs_reduce<256>(double(o_vmax), double(o_umax), double(cnt) * p.rho_ref + o_dev.value(), double(o_dmax),
                        aux.partials + 4 * blockIdx.x);
}

}  // namespace lbmd
