// Fused D3Q19 time step, 2.5D: each CTA owns a TX x TY column of the x-y
// plane and a chunk of ZC planes, and marches through z.  Shared memory holds
// ring buffers of planes: the density deviation (3R+1 planes, x-y halo 2R+1)
// and the chemical potential (3R+1 planes, x-y halo R+1), so every density
// value is read from global memory once per CTA and mu is evaluated once per
// node of its region.  A plane is collided on its tile plus a one-node x-y
// ring (the ring's populations are L2 re-reads), its post-collision values go
// to a shared plane buffer, and each tile node gathers the populations that
// stream into it; the partial sums of the three target planes p-1, p, p+1
// live in registers, so the next density is produced in the same pass.  The
// chunk's planes z0-1 and z1 are collided as well (not written) to supply the
// populations crossing the chunk faces.
//
// Step per plane (Sec. 2.1-2.3): mu = k^2 psi'(rho) - kappa lap rho (Eq. 16);
// grad mu, grad rho (Eq. 18-20, 25); F = -rho grad mu + grad rho / 3 (Eq. 12);
// BGK + exact-difference forcing (Eq. 1, 6, 8); push streaming.
#pragma once
#include "lbm_device.cuh"
#include "step2d.cuh"

namespace lbmd {

constexpr int NT3 = 256;

template <int S, class P, int TX, int TY>
struct Step3DShape {
  static constexpr int R = Sch<S>::R, H = 2 * R + 1, NS = 3 * R + 1;
  static constexpr int RW = TX + 2 * H, RH = TY + 2 * H;          // density plane region
  static constexpr int MW = TX + 2 * R + 2, MH = TY + 2 * R + 2;  // mu plane region
  static constexpr int CW = TX + 2, CH = TY + 2;                  // collision region
  static constexpr size_t ds_plane = size_t(RH) * RW;
  static constexpr size_t mu_plane = size_t(MH) * MW;
  static constexpr size_t off_mu = (NS * ds_plane * sizeof(typename P::Tr) + 15) / 16 * 16;
  static constexpr size_t off_f = (off_mu + NS * mu_plane * sizeof(typename P::Tm) + 15) / 16 * 16;
  static constexpr size_t bytes = off_f + size_t(19) * CH * CW * sizeof(typename P::Tf);
  static constexpr int K = (TX * TY + NT3 - 1) / NT3;  // interior nodes per thread
};

template <int S, typename T, typename A>
__device__ __forceinline__ void grad3d(const A* s, const int* base, int W, int cx, int cy, T& gx, T& gy, T& gz) {
  using Sc = Sch<S>;
  constexpr int R = Sc::R;
  T ax = 0, ay = 0, az = 0;
  if constexpr (Sc::ISO) {
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const double w = Sc::w3d(dx, dy, dz);
          if (w != 0.0) {
            const T v = T(s[base[dz + R] + (cy + dy) * W + cx + dx]);
            if (dx != 0) ax += T(w * dx) * v;
            if (dy != 0) ay += T(w * dy) * v;
            if (dz != 0) az += T(w * dz) * v;
          }
        }
  } else {
    const int c = cy * W + cx;
#pragma unroll
    for (int m = 1; m <= R; ++m) {
      ax += T(Sc::g(m)) * (T(s[base[R] + c + m]) - T(s[base[R] + c - m]));
      ay += T(Sc::g(m)) * (T(s[base[R] + c + m * W]) - T(s[base[R] + c - m * W]));
      az += T(Sc::g(m)) * (T(s[base[R + m] + c]) - T(s[base[R - m] + c]));
    }
  }
  gx = ax;
  gy = ay;
  gz = az;
}

template <int S, typename T, typename A>
__device__ __forceinline__ T lap3d(const A* s, const int* base, int W, int cx, int cy) {
  using Sc = Sch<S>;
  constexpr int R = Sc::R;
  const int c = cy * W + cx;
  const T v0 = T(s[base[R] + c]);
  T acc = 0;
  if constexpr (Sc::ISO) {
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const double w = Sc::w3d(dx, dy, dz);
          if (w != 0.0) acc += T(2.0 * w) * (T(s[base[dz + R] + (cy + dy) * W + cx + dx]) - v0);
        }
  } else {
    acc = T(3.0 * Sc::l(0)) * v0;
#pragma unroll
    for (int m = 1; m <= R; ++m)
      acc += T(Sc::l(m)) * ((T(s[base[R] + c + m]) + T(s[base[R] + c - m])) +
                            (T(s[base[R] + c + m * W]) + T(s[base[R] + c - m * W])) +
                            (T(s[base[R + m] + c]) + T(s[base[R - m] + c])));
  }
  return acc;
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <int S, class P, int TX, int TY, int ZC, int MODE>
__global__ void __launch_bounds__(NT3) k_step3d(const KParams p, const typename P::Tf* __restrict__ fin,
                                                typename P::Tf* __restrict__ fout, const typename P::Tr* __restrict__ rin,
                                                typename P::Tr* __restrict__ rout, const StepAux aux, const FieldOut fo,
                                                const GradIn gi) {
  using Tr = typename P::Tr;
  using Tf = typename P::Tf;
  using Tc = typename P::Tc;
  using Ts = typename P::Ts;
  using Tm = typename P::Tm;
  using L = Lattice<1>;
  using Sh = Step3DShape<S, P, TX, TY>;
  constexpr int Q = 19, R = Sh::R, H = Sh::H, NS = Sh::NS, RW = Sh::RW, MW = Sh::MW, CW = Sh::CW, CH = Sh::CH;
  constexpr int K = Sh::K;

  extern __shared__ __align__(16) unsigned char smem[];
  Tr* s_ds = reinterpret_cast<Tr*>(smem);  // density (FP64) or rho - rho_ref (FP32DEV)
  Tm* s_mu = reinterpret_cast<Tm*>(smem + Sh::off_mu);
  Tf* s_f = reinterpret_cast<Tf*>(smem + Sh::off_f);

  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const long long N = p.n;
  const long long NXY = (long long)nx * ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
  const int z1 = min(z0 + ZC, nz);
  const int VW = min(TX, nx - x0), VH = min(TY, ny - y0);
  const int tid = threadIdx.x;
  const int rw = VW + 2 * H, rh = VH + 2 * H, mw = VW + 2 * R + 2, mh = VH + 2 * R + 2, cw = VW + 2, ch = VH + 2;
  const Tm k2 = Tm(p.k2), kap = Tm(p.kappa);
  const Tc omega = Tc(p.omega);

  // per-thread accumulators of the next density for target planes p-1, p, p+1
  FSum accD[K][3];
  double accS[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) { accD[k][j] = FSum(); accS[k][j] = 0.0; }
  double o_vmax = 0, o_umax = 0, o_mass = 0, o_dmax = 0;

  // the first plane collided is z0-1 (it feeds plane z0), the last is z1
  const int pc_first = (MODE == MODE_STEP) ? z0 - 1 : z0;
  const int pc_last = (MODE == MODE_STEP) ? z1 : z1 - 1;
  for (int ql = pc_first - 2 * R; ql <= pc_last + 2 * R; ++ql) {
    // ---- load density plane ql (x-y halo H); start mu(ql) = k^2 psi'(rho)
    {
      const int slot = pmod(ql, NS);
      const long long zoff = (long long)pmod(ql, nz) * NXY;
      Tr* dsp = s_ds + slot * Sh::ds_plane;
      Tm* mup = s_mu + slot * Sh::mu_plane;
      for (int idx = tid; idx < rw * rh; idx += NT3) {
        const int ry = idx / rw, rx = idx - ry * rw;
        int gx = (x0 - H + rx) % nx;
        if (gx < 0) gx += nx;
        int gy = (y0 - H + ry) % ny;
        if (gy < 0) gy += ny;
        const Tr v = rin[zoff + (long long)gy * nx + gx];
        dsp[ry * RW + rx] = v;
        const int mx = rx - (H - R - 1), my = ry - (H - R - 1);
        if constexpr (!Sch<S>::GF)
          if (mx >= 0 && mx < mw && my >= 0 && my < mh)
            mup[my * MW + mx] = k2 * eos_mu<Tm>(P::DEV ? Tm(p.rho_ref) + Tm(v) : Tm(v), p);
      }
    }
    __syncthreads();
    // ---- finish mu(ql - R) -= kappa lap(rho)
    const int qm = ql - R;
    if (!Sch<S>::GF && qm >= pc_first - R) {
      int base[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; ++d) base[d + R] = pmod(qm + d, NS) * int(Sh::ds_plane);
      Tm* mup = s_mu + pmod(qm, NS) * Sh::mu_plane;
      for (int idx = tid; idx < mw * mh; idx += NT3) {
        const int my = idx / mw, mx = idx - my * mw;
        const int sx = mx + (H - R - 1), sy = my + (H - R - 1);
        mup[my * MW + mx] -= kap * lap3d<S, Tm>(s_ds, base, RW, sx, sy);
      }
    }
    __syncthreads();
    // ---- collide plane pc = ql - 2R on tile + ring
    const int pc = ql - 2 * R;
    if (pc < pc_first) continue;
    const bool own = (pc >= z0 && pc < z1);
    {
      int bds[2 * R + 1], bmu[2 * R + 1];
#pragma unroll
      for (int d = -R; d <= R; ++d) {
        bds[d + R] = pmod(pc + d, NS) * int(Sh::ds_plane);
        bmu[d + R] = pmod(pc + d, NS) * int(Sh::mu_plane);
      }
      const long long zoff = (long long)pmod(pc, nz) * NXY;
      const int ncol = (MODE == MODE_STEP) ? cw * ch : VW * VH;
      for (int idx = tid; idx < ncol; idx += NT3) {
        int lx, ly, cx, cy;
        if (MODE == MODE_STEP) {
          cy = idx / cw; cx = idx - cy * cw; lx = cx - 1; ly = cy - 1;
        } else {
          ly = idx / VW; lx = idx - ly * VW; cx = lx + 1; cy = ly + 1;
        }
        const bool interior = (lx >= 0 && lx < VW && ly >= 0 && ly < VH);
        const int gx = wrapi(x0 + lx, nx), gy = wrapi(y0 + ly, ny);
        const long long node = zoff + (long long)gy * nx + gx;
        Tf fv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fv[i] = fin[i * N + node];
        const Tr dsv = s_ds[bds[R] + (ly + H) * RW + lx + H];
        Tc jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (L::ex(i) != 0) jx += Tc(L::ex(i)) * Tc(fv[i]);
          if (L::ey(i) != 0) jy += Tc(L::ey(i)) * Tc(fv[i]);
          if (L::ez(i) != 0) jz += Tc(L::ez(i)) * Tc(fv[i]);
        }
        const Tc rc = P::DEV ? Tc(p.rho_ref) + Tc(dsv) : Tc(dsv);
        const Tc ux = jx / rc, uy = jy / rc, uz = jz / rc;
        Tm gmx, gmy, gmz;
        Tc grx, gry, grz;
        if constexpr (Sch<S>::GF) {
          const Tm* gm = static_cast<const Tm*>(gi.gmu);
          const Tc* gr = static_cast<const Tc*>(gi.grho);
          gmx = gm[node]; gmy = gm[N + node]; gmz = gm[2 * N + node];
          grx = gr[node]; gry = gr[N + node]; grz = gr[2 * N + node];
        } else {
          grad3d<S, Tm>(s_mu, bmu, MW, lx + R + 1, ly + R + 1, gmx, gmy, gmz);
          grad3d<S, Tc>(s_ds, bds, RW, lx + H, ly + H, grx, gry, grz);
        }
        const Tc Fx = -rc * Tc(gmx) + grx / Tc(3), Fy = -rc * Tc(gmy) + gry / Tc(3), Fz = -rc * Tc(gmz) + grz / Tc(3);
        if constexpr (MODE == MODE_STEP) {
          if (own && interior && !(rc > Tc(0))) atomicMin(aux.bad_step, (unsigned long long)aux.t);
          const Tc vx = ux + Fx / rc, vy = uy + Fy / rc, vz = uz + Fz / rc;
          const Tc dr = P::DEV ? Tc(dsv) : rc;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const Tc fs = coll_one<1, Tc>(i, Tc(fv[i]), dr, rc, omega, ux, uy, uz, vx, vy, vz);
            s_f[i * CH * CW + cy * CW + cx] = Tf(fs);
            if (own && interior) {
              const int txx = wrapi(gx + L::ex(i), nx), tyy = wrapi(gy + L::ey(i), ny), tzz = wrapi(pmod(pc, nz) + L::ez(i), nz);
              fout[i * N + (long long)tzz * NXY + (long long)tyy * nx + txx] = Tf(fs);
            }
          }
        } else if constexpr (MODE == MODE_OBS) {
          const double rho = P::DEV ? p.rho_ref + double(dsv) : double(dsv);
          const double dux = double(ux), duy = double(uy), duz = double(uz);
          const double vx = dux + double(Fx) / (2.0 * rho), vy = duy + double(Fy) / (2.0 * rho),
                       vz = duz + double(Fz) / (2.0 * rho);
          o_vmax = fmax(o_vmax, sqrt(vx * vx + vy * vy + vz * vz));
          o_umax = fmax(o_umax, sqrt(dux * dux + duy * duy + duz * duz));
          const double rtrue = P::DEV ? p.rho_ref + double(rin[node]) : double(rin[node]);
          o_mass += rtrue;
          o_dmax = fmax(o_dmax, fabs(double(rin[node]) - double(static_cast<const Tr*>(aux.rho_snap)[node])));
          if (!(rtrue > 0.0)) atomicMin(aux.bad_step, (unsigned long long)aux.t);
        } else {
          fo.F[node] = double(Fx);
          fo.F[N + node] = double(Fy);
          fo.F[2 * N + node] = double(Fz);
          if constexpr (Sch<S>::GF) fo.mu[node] = double(static_cast<const Tm*>(gi.mu)[node]);
          else fo.mu[node] = double(s_mu[bmu[R] + (ly + R + 1) * MW + lx + R + 1]);
        }
      }
    }
    // the next iteration's load overwrites the ring slot read by this collision
    __syncthreads();
    if constexpr (MODE == MODE_STEP) {
      // ---- gather: populations of plane pc stream into planes pc-1, pc, pc+1
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int idx = tid + k * NT3;
        if (idx < VW * VH) {
          const int ly = idx / VW, lx = idx - ly * VW;
          const int cx = lx + 1, cy = ly + 1;
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const Tf v = s_f[i * CH * CW + (cy - L::ey(i)) * CW + cx - L::ex(i)];
            const int j = L::ez(i) + 1;  // target plane pc + ez -> slot j (0: pc-1, 1: pc, 2: pc+1)
            if constexpr (P::DEV) accD[k][j].add(float(v)); else accS[k][j] += double(v);
          }
          // plane pc-1 is complete
          const int zt = pc - 1;
          if (zt >= z0 && zt < z1) {
            Tr rn;
            bool okr;
            if constexpr (P::DEV) { rn = accD[k][0].fvalue(); okr = float(p.rho_ref) + rn > 0.f; }
            else { rn = accS[k][0]; okr = rn > 0.0; }
            rout[(long long)zt * NXY + (long long)(y0 + ly) * nx + x0 + lx] = rn;
            if (!okr) atomicMin(aux.bad_step, (unsigned long long)(aux.t + 1));
          }
        }
        accD[k][0] = accD[k][1]; accD[k][1] = accD[k][2]; accD[k][2] = FSum();
        accS[k][0] = accS[k][1]; accS[k][1] = accS[k][2]; accS[k][2] = 0.0;
      }
    }
  }
  if constexpr (MODE == MODE_OBS) {
    block_obs_reduce<NT3>(o_vmax, o_umax, o_mass, o_dmax,
                          aux.partials + 4 * ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x));
  }
}

}  // namespace lbmd
