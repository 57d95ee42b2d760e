// D3Q19 fused step for FP32 deviation storage (populations f_i - w_i rho_ref
// and density rho - rho_ref in float, FP32 chemical potential): the same
// 2.5D algorithm as k_step3d, arranged for throughput.
//
//  - 16 x 16 tiles, 352 threads: one thread per node of the tile plus its
//    one-node ring (324 nodes), so the collision is a single round.
//  - 32-bit indexing (the library limits 19 N to 2^31); ring-buffer slots are
//    advanced incrementally; no integer division in the plane loop except by
//    compile-time constants.
//  - Software pipeline with cp.async: while plane p is reduced (mu, force,
//    collision, density gather), the density plane and the populations of
//    plane p+1 are already being copied into shared memory.  Each thread
//    copies the 19 populations of its own node, so only the density plane
//    needs the block barrier.
//  - Post-collision populations overwrite the staged inputs in place; the
//    tile's next density is gathered from them (three target planes kept in
//    registers).
//  - tau = 1 (the configurations of the paper's droplet runs) takes a shorter
//    collision: f*_i = f_i^eq(rho, u + F/rho).
//  - The z-chunk length is a launch argument (chosen by the host heuristic or
//    by lbm_autotune).
//  - No FP64 instruction in the loop.
#pragma once
#include "lbm_device.cuh"
#include "step2d.cuh"
#include "step3d.cuh"

namespace lbmd {

constexpr int FT = 16;                 // tile edge
constexpr int FC = FT + 2;             // collision region edge
constexpr int FNC = FC * FC;           // 324 collision nodes
constexpr int FNT = 352;               // threads (11 warps)

template <int S>
struct FastShape {
  static constexpr int R = Sch<S>::R, H = 2 * R + 1;
  static constexpr int RW = FT + 2 * H;                 // density region edge
  static constexpr int MW = FT + 2 * R + 2;             // mu region edge
  static constexpr int NSD = 3 * R + 2;                 // density ring (one slot in flight)
  static constexpr int NSM = 2 * R + 1;                 // mu ring
  static constexpr int NLD = (RW * RW + FNT - 1) / FNT; // density loads per thread
  static constexpr int NLM = (MW * MW + FNT - 1) / FNT; // mu points per thread
  static constexpr int ds_plane = RW * RW;
  static constexpr int mu_plane = MW * MW;
  static constexpr size_t off_mu = size_t(NSD) * ds_plane * 4;
  static constexpr size_t off_f = (off_mu + size_t(NSM) * mu_plane * 4 + 15) / 16 * 16;
  static constexpr int fbuf = 19 * FNC;                 // floats per population buffer
  static constexpr size_t bytes = off_f + size_t(2) * fbuf * 4;
};


template <int S, bool TAU1>
__global__ void __launch_bounds__(FNT, 2) k_step3d_fast(const KParams p, const float* __restrict__ fin,
                                                         float* __restrict__ fout, const float* __restrict__ rin,
                                                         float* __restrict__ rout, const StepAux aux, const int zc) {
  using L = Lattice<1>;
  using Sh = FastShape<S>;
  constexpr int Q = 19, R = Sh::R, H = Sh::H, RW = Sh::RW, MW = Sh::MW, NSD = Sh::NSD, NSM = Sh::NSM;
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_ds = reinterpret_cast<float*>(smem);
  float* s_mu = reinterpret_cast<float*>(smem + Sh::off_mu);
  float* s_f = reinterpret_cast<float*>(smem + Sh::off_f);

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int N = int(p.n), NXY = nx * ny;
  const int x0 = blockIdx.x * FT, y0 = blockIdx.y * FT, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const int VW = min(FT, nx - x0), VH = min(FT, ny - y0);
  const int tid = threadIdx.x;

  // collision node of this thread (tile + one-node ring)
  const int cy = tid / FC, cx = tid - cy * FC;
  const int lx = cx - 1, ly = cy - 1;
  const bool cnode = tid < FNC && lx <= VW && ly <= VH;
  const bool interior = cnode && lx >= 0 && lx < VW && ly >= 0 && ly < VH;
  const int gx = wrapi(x0 + lx, nx), gy = wrapi(y0 + ly, ny);
  // gather target of this thread (tile node)
  const int ty = tid / FT, tx = tid - ty * FT;
  const bool gnode = tid < FT * FT && tx < VW && ty < VH;

  const float k2 = float(p.k2), kap = float(p.kappa);
  const EosF ef = eos_f(p);
  const float omega = float(p.omega), rref = float(p.rho_ref);

  const int pc_first = z0 - 1, pc_last = z1;
  const int ql0 = pc_first - 2 * R, ql1 = pc_last + 2 * R;

  // copies for density plane q into ring slot `slot`, and the populations of
  // plane q - 2R into the staging buffer of its parity
  auto issue = [&](int q, int slot) {
    const float* src = rin + pmod(q, nz) * NXY;
    float* dst = s_ds + slot * Sh::ds_plane;
#pragma unroll
    for (int k = 0; k < Sh::NLD; ++k) {
      const int idx = tid + k * FNT;
      const int ry = idx / RW, rx = idx - ry * RW;
      if (idx < RW * RW && rx < VW + 2 * H && ry < VH + 2 * H)
        cpa4(dst + idx, src + wrapi(y0 - H + ry, ny) * nx + wrapi(x0 - H + rx, nx));
    }
    const int pc = q - 2 * R;
    if (pc >= pc_first && cnode) {
      const float* fs = fin + pmod(pc, nz) * NXY + gy * nx + gx;
      float* fd = s_f + (pc & 1) * Sh::fbuf + tid;
#pragma unroll
      for (int i = 0; i < Q; ++i) cpa4(fd + i * FNC, fs + i * N);
    }
    cpa_commit();
  };

  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;  // next density of target planes pc-1, pc, pc+1
  int sd = pmod(ql0, NSD);                     // density ring slot of plane ql
  int sm = pmod(ql0 - R, NSM);                 // mu ring slot of plane ql - R
  issue(ql0, sd);
  for (int ql = ql0; ql <= ql1; ++ql) {
    cpa_wait_all();
    __syncthreads();
    if (ql < ql1) issue(ql + 1, ring(sd + 1, NSD));
    // ---- mu(qm) = k^2 psi'(rho) - kappa lap rho on the mu region (Eq. 16), qm = ql - R
    if (ql >= pc_first) {
      int base[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; ++d) base[d + R] = ring(sd - R + d, NSD) * Sh::ds_plane;  // planes qm + d
      float* mup = s_mu + sm * Sh::mu_plane;
#pragma unroll
      for (int k = 0; k < Sh::NLM; ++k) {
        const int idx = tid + k * FNT;
        const int my = idx / MW, mx = idx - my * MW;
        if (idx < MW * MW && mx < VW + 2 * R + 2 && my < VH + 2 * R + 2) {
          const int sx = mx + (H - R - 1), sy = my + (H - R - 1);
          const float rho = rref + s_ds[base[R] + sy * RW + sx];
          const float mub = eos_mu_f(rho, ef);
          mup[idx] = k2 * mub - kap * lap3d<S, float>(s_ds, base, RW, sx, sy);
        }
      }
    }
    __syncthreads();
    const int pc = ql - 2 * R;
    if (pc >= pc_first) {
      float* fb = s_f + (pc & 1) * Sh::fbuf;
      // ---- collide plane pc on tile + ring (Eq. 1, 6, 7, 8, 12)
      if (cnode) {
        int bds[2 * R + 1], bmu[2 * R + 1];
#pragma unroll
        for (int d = -R; d <= R; ++d) {
          bds[d + R] = ring(sd - 2 * R + d, NSD) * Sh::ds_plane;
          bmu[d + R] = ring(sm - R + d, NSM) * Sh::mu_plane;
        }
        float fv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = fb[i * FNC + tid];
        const float dsv = s_ds[bds[R] + (ly + H) * RW + lx + H];
        const float rc = rref + dsv;
        float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (L::ex(i) != 0) jx += float(L::ex(i)) * fv[i];
          if (L::ey(i) != 0) jy += float(L::ey(i)) * fv[i];
          if (L::ez(i) != 0) jz += float(L::ez(i)) * fv[i];
        }
        const float irc = __fdividef(1.f, rc);
        const float ux = jx * irc, uy = jy * irc, uz = jz * irc;
        float gmx, gmy, gmz, grx, gry, grz;
        grad3d<S, float>(s_mu, bmu, MW, lx + R + 1, ly + R + 1, gmx, gmy, gmz);
        grad3d<S, float>(s_ds, bds, RW, lx + H, ly + H, grx, gry, grz);
        const float Fx = -rc * gmx + grx * (1.f / 3.f), Fy = -rc * gmy + gry * (1.f / 3.f),
                    Fz = -rc * gmz + grz * (1.f / 3.f);
        const float vx = ux + Fx * irc, vy = uy + Fy * irc, vz = uz + Fz * irc;
        const bool push = interior && pc >= z0 && pc < z1;
        if (push && !(rc > 0.f)) atomicMin(aux.bad_step, (unsigned long long)aux.t);
        const int pz = pmod(pc, nz);
        const int xm = wrapi(gx - 1, nx), xp = wrapi(gx + 1, nx);
        const int rowm = wrapi(gy - 1, ny) * nx, row0 = gy * nx, rowp = wrapi(gy + 1, ny) * nx;
        const int zb = pz * NXY, zbm = wrapi(pz - 1, nz) * NXY, zbp = wrapi(pz + 1, nz) * NXY;
        const float vv15 = 1.5f * (vx * vx + vy * vy + vz * vz);
        const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float w = float(L::w(i));
          const float ev = edot<L>(i, vx, vy, vz);
          const float Av = i == 0 ? -vv15 : ev * (3.f + 4.5f * ev) - vv15;
          float fs;
          if constexpr (TAU1) {
            fs = w * (dsv + rc * Av);
          } else {
            const float eu = edot<L>(i, ux, uy, uz);
            const float Au = i == 0 ? -uu15 : eu * (3.f + 4.5f * eu) - uu15;
            fs = (1.f - omega) * fv[i] + w * (omega * dsv + rc * (omega * Au + Av - Au));
          }
          fb[i * FNC + tid] = fs;
          if (push) {
            const int txx = L::ex(i) > 0 ? xp : (L::ex(i) < 0 ? xm : gx);
            const int tyy = L::ey(i) > 0 ? rowp : (L::ey(i) < 0 ? rowm : row0);
            const int tz = L::ez(i) > 0 ? zbp : (L::ez(i) < 0 ? zbm : zb);
            fout[i * N + tz + tyy + txx] = fs;
          }
        }
      }
      __syncthreads();
      // ---- gather the populations streaming into the tile's nodes
      if (gnode) {
        const int c = (ty + 1) * FC + tx + 1;
        float s_m = 0.f, s_0 = 0.f, s_p = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float v = fb[i * FNC + c - L::ey(i) * FC - L::ex(i)];
          if (L::ez(i) < 0) s_m += v; else if (L::ez(i) == 0) s_0 += v; else s_p += v;
        }
        // sources in plane pc feed target planes pc-1 (ez < 0), pc (ez = 0), pc+1 (ez > 0)
        acc0 += s_m;
        acc1 += s_0;
        acc2 += s_p;
        const int zt = pc - 1;
        if (zt >= z0 && zt < z1) {
          rout[zt * NXY + (y0 + ty) * nx + x0 + tx] = acc0;
          if (!(rref + acc0 > 0.f)) atomicMin(aux.bad_step, (unsigned long long)(aux.t + 1));
        }
        acc0 = acc1;
        acc1 = acc2;
        acc2 = 0.f;
      }
    }
    sd = ring(sd + 1, NSD);
    if (ql >= pc_first) sm = ring(sm + 1, NSM);
  }
}

}  // namespace lbmd
