// Fused D2Q9 time step: mu (Eq. 16) -> grad mu, grad rho (Eq. 18-20, 25) ->
// F (Eq. 12) -> BGK + exact-difference forcing (Eq. 1, 6, 8) -> push streaming,
// plus the density of the next step, in one pass over the populations.
//
// One CTA owns a TX x TY tile.  The density of the tile plus a halo of 2R+1
// nodes (R = stencil radius) is staged in shared memory; mu is evaluated on
// the tile plus a halo of R+1; the tile plus a one-node ring is collided, so
// that every population streaming into the tile is known on chip and the
// tile's next density is a sum over shared memory.  Only the tile's own
// post-collision populations are written.  DRAM traffic per node is one read
// and one write of the Q populations and of the density; the halo re-reads
// are served by L2.
#pragma once
#include "lbm_device.cuh"
#include "mrt.cuh"

namespace lbmd {

// MODE_STEP_OBS: one step that also reduces the observables of the state it
// advances (split D3Q19 FP32DEV path only; other paths report not-supported)
enum { MODE_STEP = 0, MODE_OBS = 1, MODE_FIELDS = 2, MODE_STEP_OBS = 3 };

// fields written in MODE_FIELDS: F (component-major, D*N) and mu (N), FP64
struct FieldOut {
  double* F;
  double* mu;
};

constexpr int NT2 = 256;  // threads per CTA

template <int S, class P, int TX, int TY>
struct Step2DShape {
  static constexpr int R = Sch<S>::R, H = 2 * R + 1;
  static constexpr int RW = TX + 2 * H, RH = TY + 2 * H;          // density region
  static constexpr int MW = TX + 2 * R + 2, MH = TY + 2 * R + 2;  // mu region
  static constexpr int CW = TX + 2, CH = TY + 2;                  // collision region
  static constexpr size_t off_mu = (size_t(RH) * RW * sizeof(typename P::Tr) + 15) / 16 * 16;
  static constexpr size_t off_f = (off_mu + size_t(MH) * MW * sizeof(typename P::Tm) + 15) / 16 * 16;
  static constexpr size_t bytes = off_f + size_t(9) * CH * CW * sizeof(typename P::Tf);
};

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of 4 observables (max, max, sum, max) into partials[block*4..]
template <int NT>
__device__ __forceinline__ void block_obs_reduce(double vmax, double umax, double mass, double dmax, double* out) {
  __shared__ double red[4][NT / 32];
  vmax = warp_max(vmax);
  umax = warp_max(umax);
  mass = warp_sum(mass);
  dmax = warp_max(dmax);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = vmax; red[1][wid] = umax; red[2][wid] = mass; red[3][wid] = dmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0, d = 0;
    for (int w = 0; w < NT / 32; ++w) { a = fmax(a, red[0][w]); b = fmax(b, red[1][w]); c += red[2][w]; d = fmax(d, red[3][w]); }
    out[0] = a; out[1] = b; out[2] = c; out[3] = d;
  }
}

// One TX x TY tile of the fused step (all threads of the CTA take part).
// partial: where MODE_OBS writes this tile's 4 partial observables.
template <int S, class P, int TX, int TY, int MODE>
// (fin and rin without __restrict__: the persistent batch kernel calls this on
// buffers it rewrites every step, so their reads must stay coherent loads,
// never the non-coherent read-only path)
__device__ __forceinline__ void step2d_tile(const KParams& p, const typename P::Tf* fin,
                                            typename P::Tf* __restrict__ fout, const typename P::Tr* rin,
                                            typename P::Tr* __restrict__ rout, const StepAux& aux, const FieldOut& fo,
                                            const GradIn& gi, const Mrt& mrt, const int x0, const int y0,
                                            unsigned char* smem,
                                            double* partial) {
  using Tf = typename P::Tf;
  using Tc = typename P::Tc;
  using Ts = typename P::Ts;
  using Tm = typename P::Tm;
  using L = Lattice<0>;
  using Sh = Step2DShape<S, P, TX, TY>;
  constexpr int Q = 9, R = Sh::R, H = Sh::H, RW = Sh::RW, MW = Sh::MW, CW = Sh::CW, CH = Sh::CH;

  using Tr = typename P::Tr;
  // density (FP64 mode) or density deviation rho - rho_ref (FP32DEV) of the region
  Tr* s_ds = reinterpret_cast<Tr*>(smem);
  Tm* s_mu = reinterpret_cast<Tm*>(smem + Sh::off_mu);
  Tf* s_f = reinterpret_cast<Tf*>(smem + Sh::off_f);

  const int nx = p.nx, ny = p.ny;
  const long long N = p.n;
  const int VW = min(TX, nx - x0), VH = min(TY, ny - y0);
  const int tid = threadIdx.x;

  // 1. density of tile + halo H (periodic)
  {
    const int rw = VW + 2 * H, rh = VH + 2 * H;
    for (int idx = tid; idx < rw * rh; idx += NT2) {
      const int ry = idx / rw, rx = idx - ry * rw;
      int gx = (x0 - H + rx) % nx;
      if (gx < 0) gx += nx;
      int gy = (y0 - H + ry) % ny;
      if (gy < 0) gy += ny;
      s_ds[ry * RW + rx] = rin[(long long)gy * nx + gx];
    }
  }
  __syncthreads();

  // 2. mu = k^2 psi'(rho) - kappa lap(rho) on tile + halo R+1 (Eq. 16)
  if constexpr (!Sch<S>::GF) {
    const int mw = VW + 2 * R + 2, mh = VH + 2 * R + 2;
    const Tm k2 = Tm(p.k2), kap = Tm(p.kappa);
    for (int idx = tid; idx < mw * mh; idx += NT2) {
      const int my = idx / mw, mx = idx - my * mw;
      const int sx = mx + (H - R - 1), sy = my + (H - R - 1);
      const Tm rho = P::DEV ? Tm(p.rho_ref) + Tm(s_ds[sy * RW + sx]) : Tm(s_ds[sy * RW + sx]);
      const Tm lap = lap2d<S, Tm>(s_ds, RW, sx, sy);
      s_mu[my * MW + mx] = k2 * eos_mu<Tm>(rho, p) - kap * lap;
    }
  }
  __syncthreads();

  // 3. collide tile + ring; push the tile's populations
  double o_vmax = 0, o_umax = 0, o_mass = 0, o_dmax = 0;
  {
    const int cw = VW + 2, ch = VH + 2;
    const Tc omega = Tc(p.omega);
    for (int idx = tid; idx < cw * ch; idx += NT2) {
      const int cy = idx / cw, cx = idx - cy * cw;
      const int lx = cx - 1, ly = cy - 1;
      const bool interior = (lx >= 0 && lx < VW && ly >= 0 && ly < VH);
      if (MODE != MODE_STEP && !interior) continue;
      const int gx = wrapi(x0 + lx, nx), gy = wrapi(y0 + ly, ny);
      const long long node = (long long)gy * nx + gx;
      Tf fv[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) fv[i] = fin[i * N + node];
      const Tr dsv = s_ds[(ly + H) * RW + lx + H];
      const double rho = P::DEV ? p.rho_ref + double(dsv) : double(dsv);
      Tc jx = 0, jy = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (L::ex(i) != 0) jx += Tc(L::ex(i)) * Tc(fv[i]);
        if (L::ey(i) != 0) jy += Tc(L::ey(i)) * Tc(fv[i]);
      }
      const Tc rc = P::DEV ? Tc(p.rho_ref) + Tc(dsv) : Tc(dsv);
      const Tc ux = jx / rc, uy = jy / rc;
      Tm gmx, gmy;
      Tc grx, gry;
      if constexpr (Sch<S>::GF) {
        const Tm* gm = static_cast<const Tm*>(gi.gmu);
        const Tc* gr = static_cast<const Tc*>(gi.grho);
        gmx = gm[node]; gmy = gm[N + node];
        grx = gr[node]; gry = gr[N + node];
      } else {
        grad2d<S, Tm>(s_mu, MW, lx + R + 1, ly + R + 1, gmx, gmy);
        grad2d<S, Tc>(s_ds, RW, lx + H, ly + H, grx, gry);
      }
      const Tc Fx = -rc * Tc(gmx) + grx / Tc(3), Fy = -rc * Tc(gmy) + gry / Tc(3);
      if constexpr (MODE == MODE_STEP) {
        if (interior && !(rc > Tc(0))) atomicMin(aux.bad_step, (unsigned long long)aux.t);
        const Tc vx = ux + Fx / rc, vy = uy + Fy / rc;
        const Tc dr = P::DEV ? Tc(dsv) : rc;
        Tc post[Q];
        if (mrt.on) {
          Tc fc[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) fc[i] = Tc(fv[i]);
          mrt_post9<Tc>(fc, dr, rc, ux, uy, vx, vy, mrt, post);
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) post[i] = coll_one<0, Tc>(i, Tc(fv[i]), dr, rc, omega, ux, uy, Tc(0), vx, vy, Tc(0));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const Tc fs = post[i];
          s_f[i * CH * CW + cy * CW + cx] = Tf(fs);
          if (interior) {
            const int tx = wrapi(gx + L::ex(i), nx), ty = wrapi(gy + L::ey(i), ny);
            fout[i * N + (long long)ty * nx + tx] = Tf(fs);
          }
        }
      } else if constexpr (MODE == MODE_OBS) {
        const double dux = double(ux), duy = double(uy);
        const double vx = dux + double(Fx) / (2.0 * rho), vy = duy + double(Fy) / (2.0 * rho);
        o_vmax = fmax(o_vmax, sqrt(vx * vx + vy * vy));
        o_umax = fmax(o_umax, sqrt(dux * dux + duy * duy));
        o_mass += rho;
        o_dmax = fmax(o_dmax, fabs(double(dsv) - double(static_cast<const Tr*>(aux.rho_snap)[node])));
        if (!(rho > 0.0)) atomicMin(aux.bad_step, (unsigned long long)aux.t);
      } else {
        fo.F[node] = double(Fx);
        fo.F[N + node] = double(Fy);
        if constexpr (Sch<S>::GF) fo.mu[node] = double(static_cast<const Tm*>(gi.mu)[node]);
        else fo.mu[node] = double(s_mu[(ly + R + 1) * MW + lx + R + 1]);
      }
    }
  }

  if constexpr (MODE == MODE_OBS) {
    block_obs_reduce<NT2>(o_vmax, o_umax, o_mass, o_dmax, partial);
    return;
  }
  if constexpr (MODE == MODE_STEP) {
    __syncthreads();
    // 4. next density of the tile: sum of the populations streaming in
    for (int idx = tid; idx < VW * VH; idx += NT2) {
      const int ly = idx / VW, lx = idx - ly * VW;
      const int cx = lx + 1, cy = ly + 1;
      Tr rn;
      bool ok;
      if constexpr (P::DEV) {
        FSum acc;
#pragma unroll
        for (int i = 0; i < Q; ++i) acc.add(float(s_f[i * CH * CW + (cy - L::ey(i)) * CW + cx - L::ex(i)]));
        rn = acc.fvalue();
        ok = float(p.rho_ref) + rn > 0.f;
      } else {
        double acc = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) acc += double(s_f[i * CH * CW + (cy - L::ey(i)) * CW + cx - L::ex(i)]);
        rn = acc;
        ok = rn > 0.0;
      }
      const long long node = (long long)(y0 + ly) * nx + x0 + lx;
      rout[node] = rn;
      if (!ok) atomicMin(aux.bad_step, (unsigned long long)(aux.t + 1));
    }
  }
}

template <int S, class P, int TX, int TY, int MODE>
__global__ void __launch_bounds__(NT2) k_step2d(const KParams p, const typename P::Tf* __restrict__ fin,
                                                typename P::Tf* __restrict__ fout, const typename P::Tr* __restrict__ rin,
                                                typename P::Tr* __restrict__ rout, const StepAux aux, const FieldOut fo,
                                                const GradIn gi, const Mrt mrt) {
  extern __shared__ __align__(16) unsigned char smem[];
  step2d_tile<S, P, TX, TY, MODE>(p, fin, fout, rin, rout, aux, fo, gi, mrt, blockIdx.x * TX, blockIdx.y * TY, smem,
                                  aux.partials + 4 * (blockIdx.y * gridDim.x + blockIdx.x));
}

}  // namespace lbmd
