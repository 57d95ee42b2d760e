// D3Q19 FP32-deviation step as two passes per time step:
//
//  k_mu3d      mu = k^2 psi'(rho) - kappa lap rho (Eq. 16) for every node, once
//              (a 2.5D stencil: x-y neighbours from a shared plane, z
//              neighbours from a per-thread register queue).
//  k_coll3d    grad mu, grad rho (Eq. 17-25) -> F (Eq. 12) -> BGK + EDM
//              (Eq. 1, 6, 8) -> push streaming, plus the next density, for
//              a 30 x 9 tile and its one-node ring marching through z.
//
// Compared with evaluating mu inside the collision kernel (where the halo
// makes each CTA recompute it ~2.3 times per node and the recomputation
// dominates shared-memory traffic), the split costs one extra float read and
// write per node (168 instead of 160 bytes per lattice update) and removes
// the mu phase, one block barrier per plane and most shared-memory loads from
// the collision kernel.  In k_coll3d one warp owns one 32-wide row of the
// collision region, so the stencil reads of a warp are contiguous (free of
// bank conflicts).
#pragma once
#include "lbm_device.cuh"
#include "step3d.cuh"
#include "step3d_fast.cuh"

namespace lbmd {

// ------------------------------------------------------------------ mu pass
constexpr int MUX = 32, MUY = 8, MUT = MUX * MUY;

// line schemes only (the isotropic 3D Laplacian needs diagonal neighbours in
// the planes above and below, which the z queue does not hold)
template <int S>
__global__ void __launch_bounds__(MUT) k_mu3d(const KParams p, const float* __restrict__ rin, float* __restrict__ mu,
                                              const int zc) {
  static_assert(!Sch<S>::ISO, "line schemes only");
  constexpr int R = Sch<S>::R;
  constexpr int PW = MUX + 2 * R, PH = MUY + 2 * R;
  __shared__ float pl[2][PH][PW];
  const int nx = p.nx, ny = p.ny, nz = p.nz, NXY = nx * ny;
  const int x0 = blockIdx.x * MUX, y0 = blockIdx.y * MUY, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const int tx = threadIdx.x % MUX, ty = threadIdx.x / MUX;
  const bool act = x0 + tx < nx && y0 + ty < ny;
  const int gx = min(x0 + tx, nx - 1), gy = min(y0 + ty, ny - 1);
  const float RT = float(p.RT), b4 = float(p.b4), two_a = float(p.two_a), k2 = float(p.k2), kap = float(p.kappa);
  const float rref = float(p.rho_ref);
  // z queue: q[R + d] = rho - rho_ref at (gx, gy, z + d)
  float q[2 * R + 1];
#pragma unroll
  for (int d = -R; d <= R; ++d) q[d + R] = rin[pmod(z0 + d, nz) * NXY + gy * nx + gx];
  auto load_plane = [&](int z, int b) {
    const float* src = rin + pmod(z, nz) * NXY;
    for (int idx = threadIdx.x; idx < PW * PH; idx += MUT) {
      const int ry = idx / PW, rx = idx - ry * PW;
      pl[b][ry][rx] = src[wrapi(y0 - R + ry, ny) * nx + wrapi(x0 - R + rx, nx)];
    }
  };
  load_plane(z0, 0);
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    const int b = (z - z0) & 1;
    if (z + 1 < z1) load_plane(z + 1, b ^ 1);
    const float next = rin[pmod(z + R + 1, nz) * NXY + gy * nx + gx];
    if (act) {
      const int cx = tx + R, cy = ty + R;
      const float c = pl[b][cy][cx];
      float lap = float(3.0 * Sch<S>::l(0)) * c;
#pragma unroll
      for (int m = 1; m <= R; ++m)
        lap += float(Sch<S>::l(m)) * ((pl[b][cy][cx + m] + pl[b][cy][cx - m]) + (pl[b][cy + m][cx] + pl[b][cy - m][cx]) +
                                      (q[R + m] + q[R - m]));
      const float rho = rref + c;
      const float eta = b4 * rho, om = 1.f - eta;
      const float hs = __fdividef(eta * (8.f + eta * (-9.f + 3.f * eta)), om * om * om);
      mu[z * NXY + gy * nx + gx] = k2 * (RT * (__logf(rho) + hs) - two_a * rho) - kap * lap;
    }
#pragma unroll
    for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
    q[2 * R] = next;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ collision pass
constexpr int CX = 32, CY = 11;     // collision region (tile + ring), one warp per row
constexpr int TXC = CX - 2, TYC = CY - 2;  // 30 x 9 tile
constexpr int CNT = CX * CY;        // 352 threads

template <int S>
struct CollShape {
  static constexpr int R = Sch<S>::R;
  static constexpr int GW = CX + 2 * R, GH = CY + 2 * R;  // field region (ring + stencil halo)
  static constexpr int NS = 2 * R + 2;                    // ring of planes (one in flight)
  static constexpr int plane = GW * GH;
  static constexpr int NLD = (plane + CNT - 1) / CNT;
  static constexpr size_t off_mu = size_t(NS) * plane * 4;
  static constexpr size_t off_f = (off_mu + size_t(NS) * plane * 4 + 15) / 16 * 16;
  static constexpr int fbuf = 19 * CNT;
  static constexpr size_t bytes = off_f + size_t(2) * fbuf * 4;
};

template <int S, bool TAU1>
__global__ void __launch_bounds__(CNT, 2) k_coll3d(const KParams p, const float* __restrict__ fin,
                                                    float* __restrict__ fout, const float* __restrict__ rin,
                                                    const float* __restrict__ muf, float* __restrict__ rout,
                                                    const StepAux aux, const int zc) {
  using L = Lattice<1>;
  using Sh = CollShape<S>;
  constexpr int Q = 19, R = Sh::R, GW = Sh::GW, GH = Sh::GH, NS = Sh::NS;
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_ds = reinterpret_cast<float*>(smem);
  float* s_mu = reinterpret_cast<float*>(smem + Sh::off_mu);
  float* s_f = reinterpret_cast<float*>(smem + Sh::off_f);

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const int N = int(p.n), NXY = nx * ny;
  const int x0 = blockIdx.x * TXC, y0 = blockIdx.y * TYC, z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, nz);
  const int VW = min(TXC, nx - x0), VH = min(TYC, ny - y0);
  const int tid = threadIdx.x;
  const int cy = tid / CX, cx = tid - cy * CX;  // one warp per row
  const int lx = cx - 1, ly = cy - 1;
  const bool cnode = lx <= VW && ly <= VH;
  const bool interior = lx >= 0 && lx < VW && ly >= 0 && ly < VH;
  const int gx = wrapi(x0 + lx, nx), gy = wrapi(y0 + ly, ny);
  const float omega = float(p.omega), rref = float(p.rho_ref);
  const int pc_first = z0 - 1, pc_last = z1;

  // field planes q (density deviation and mu, region GW x GH) -> ring slot;
  // populations of plane q - R (if collided) -> staging buffer of its parity
  auto issue = [&](int q, int slot) {
    const int zo = pmod(q, nz) * NXY;
    float* dd = s_ds + slot * Sh::plane;
    float* dm = s_mu + slot * Sh::plane;
#pragma unroll
    for (int k = 0; k < Sh::NLD; ++k) {
      const int idx = tid + k * CNT;
      const int ry = idx / GW, rx = idx - ry * GW;
      if (idx < Sh::plane && rx < VW + 2 + 2 * R && ry < VH + 2 + 2 * R) {
        const int g = zo + wrapi(y0 - 1 - R + ry, ny) * nx + wrapi(x0 - 1 - R + rx, nx);
        cpa4(dd + idx, rin + g);
        cpa4(dm + idx, muf + g);
      }
    }
    const int pc = q - R;
    if (pc >= pc_first && pc <= pc_last && cnode) {
      const float* fs = fin + pmod(pc, nz) * NXY + gy * nx + gx;
      float* fd = s_f + (pc & 1) * Sh::fbuf + tid;
#pragma unroll
      for (int i = 0; i < Q; ++i) cpa4(fd + i * CNT, fs + i * N);
    }
    cpa_commit();
  };

  // prologue: planes pc_first - R .. pc_first + R
  int slot = 0;  // ring slot of plane pc_first - R + (number issued)
  for (int q = pc_first - R; q <= pc_first + R - 1; ++q) {
    issue(q, slot);
    slot = ring(slot + 1, NS);
  }
  int sc = R;  // ring slot of the collision plane
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  issue(pc_first + R, slot);
  slot = ring(slot + 1, NS);
  for (int pc = pc_first; pc <= pc_last; ++pc) {
    cpa_wait_all();
    __syncthreads();
    if (pc < pc_last) {
      issue(pc + R + 1, slot);
      slot = ring(slot + 1, NS);
    }
    float* fb = s_f + (pc & 1) * Sh::fbuf;
    if (cnode) {
      int base[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; ++d) base[d + R] = ring(sc + d, NS) * Sh::plane;
      float fv[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) fv[i] = fb[i * CNT + tid];
      const int c = (cy + R) * GW + cx + R;
      const float dsv = s_ds[base[R] + c];
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
      grad3d<S, float>(s_mu, base, GW, cx + R, cy + R, gmx, gmy, gmz);
      grad3d<S, float>(s_ds, base, GW, cx + R, cy + R, grx, gry, grz);
      const float Fx = -rc * gmx + grx * (1.f / 3.f), Fy = -rc * gmy + gry * (1.f / 3.f),
                  Fz = -rc * gmz + grz * (1.f / 3.f);
      const float vx = ux + Fx * irc, vy = uy + Fy * irc, vz = uz + Fz * irc;
      const bool push = interior && pc >= z0 && pc < z1;
      if (push && !(rc > 0.f)) atomicMin(aux.bad_step, (unsigned long long)aux.t);
      // target of population i = own node + per-axis deltas (periodic wrap folded in)
      const int pz = pmod(pc, nz);
      const int dxp = (gx + 1 < nx) ? 1 : 1 - nx, dxm = (gx > 0) ? -1 : nx - 1;
      const int dyp = (gy + 1 < ny) ? nx : nx - NXY, dym = (gy > 0) ? -nx : NXY - nx;
      const int dzp = (pz + 1 < nz) ? NXY : NXY - N, dzm = (pz > 0) ? -NXY : N - NXY;
      float* fo = fout + pz * NXY + gy * nx + gx;
      const float vv15 = 1.5f * (vx * vx + vy * vy + vz * vz);
      const float uu15 = 1.5f * (ux * ux + uy * uy + uz * uz);
      const float wd0 = float(L::w(0)) * dsv, wd1 = float(L::w(1)) * dsv, wd2 = float(L::w(7)) * dsv;
      const float wr0 = float(L::w(0)) * rc, wr1 = float(L::w(1)) * rc, wr2 = float(L::w(7)) * rc;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float wd = i == 0 ? wd0 : (i < 7 ? wd1 : wd2);
        const float wr = i == 0 ? wr0 : (i < 7 ? wr1 : wr2);
        const float ev = float(L::ex(i)) * vx + float(L::ey(i)) * vy + float(L::ez(i)) * vz;
        const float Av = ev * (3.f + 4.5f * ev) - vv15;
        float fs;
        if constexpr (TAU1) {
          fs = wd + wr * Av;
        } else {
          const float eu = float(L::ex(i)) * ux + float(L::ey(i)) * uy + float(L::ez(i)) * uz;
          const float Au = eu * (3.f + 4.5f * eu) - uu15;
          fs = (1.f - omega) * fv[i] + omega * wd + wr * (omega * Au + Av - Au);
        }
        fb[i * CNT + tid] = fs;
        if (push) {
          const int d = (L::ex(i) > 0 ? dxp : (L::ex(i) < 0 ? dxm : 0)) + (L::ey(i) > 0 ? dyp : (L::ey(i) < 0 ? dym : 0)) +
                        (L::ez(i) > 0 ? dzp : (L::ez(i) < 0 ? dzm : 0));
          fo[i * N + d] = fs;
        }
      }
    }
    __syncthreads();
    // gather for the tile's own node of this thread
    if (interior) {
      float s_m = 0.f, s_0 = 0.f, s_p = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float v = fb[i * CNT + tid - L::ey(i) * CX - L::ex(i)];
        if (L::ez(i) < 0) s_m += v; else if (L::ez(i) == 0) s_0 += v; else s_p += v;
      }
      acc0 += s_m;
      acc1 += s_0;
      acc2 += s_p;
      const int zt = pc - 1;
      if (zt >= z0 && zt < z1) {
        rout[zt * NXY + (y0 + ly) * nx + x0 + lx] = acc0;
        if (!(rref + acc0 > 0.f)) atomicMin(aux.bad_step, (unsigned long long)(aux.t + 1));
      }
      acc0 = acc1;
      acc1 = acc2;
      acc2 = 0.f;
    }
    sc = ring(sc + 1, NS);
  }
}

}  // namespace lbmd
