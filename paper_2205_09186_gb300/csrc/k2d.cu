// Instantiations of the fused D2Q9 step for the explicit and isotropic schemes.
#include <type_traits>

#include <cstdint>

#include "launch.cuh"
#include "step2d.cuh"
#include "step2d_split.cuh"

namespace lbmd {

constexpr int TX2 = 32, TY2 = 8;

namespace {

template <int S, class P, int MODE>
cudaError_t launch_mode(const Launch& c, int* nblocks) {
  using Sh = Step2DShape<S, P, TX2, TY2>;
  auto k = k_step2d<S, P, TX2, TY2, MODE>;
  if (cudaError_t e = ensure_smem(k, Sh::bytes); e != cudaSuccess) return e;
  dim3 grid((c.kp.nx + TX2 - 1) / TX2, (c.kp.ny + TY2 - 1) / TY2, 1);
  if (nblocks) *nblocks = int(grid.x * grid.y);
  using Tf = typename P::Tf;
  using Tr = typename P::Tr;
  k<<<grid, NT2, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout),
                                        static_cast<const Tr*>(c.rin), static_cast<Tr*>(c.rout),
                                        c.aux, c.fo, c.gi, c.mrt);
  return cudaGetLastError();
}

// FP32 deviation storage with FP32 mu: mu pass + row-per-warp collision pass,
// tiles of RPT rows per thread
template <int S, bool TAU1, int RPT>
cudaError_t launch_split2d_t(const Launch& c, int* nblocks) {
  using Sh = Split2DShape<S, RPT>;
  constexpr int M2Y = Tile2<RPT>::M2Y, T2Y = Tile2<RPT>::T2Y;
  if (cudaError_t e = ensure_smem(k_mu2d<S, RPT>, Sh::bytes); e != cudaSuccess) return e;
  if (cudaError_t e = ensure_smem(k_coll2d<S, TAU1, RPT>, Sh::bytes); e != cudaSuccess) return e;
  if constexpr (!Sch<S>::ISO) {
    if (c.kp.nx % 4 == 0 && (reinterpret_cast<uintptr_t>(c.rin) & 15) == 0 && (reinterpret_cast<uintptr_t>(c.mu) & 15) == 0) {
      // rows per thread: about four CTAs of 8 warps per SM, 2..32 rows
      const int gx = (c.kp.nx + 63) / 64;
      const int sms = device_sms();
      const int want_gy = (4 * sms + gx - 1) / gx;
      int rows = (c.kp.ny + 16 * want_gy - 1) / (16 * want_gy);
      rows = rows < 2 ? 2 : (rows > 32 ? 32 : rows);
      dim3 gm(gx, (c.kp.ny + 16 * rows - 1) / (16 * rows));
      k_mu2d_ym<S><<<gm, YMT, 0, c.stream>>>(c.kp, static_cast<const float*>(c.rin), static_cast<float*>(c.mu), rows);
    } else {
      dim3 gm((c.kp.nx + M2X - 1) / M2X, (c.kp.ny + M2Y - 1) / M2Y);
      k_mu2d<S, RPT><<<gm, NT2S, Sh::bytes, c.stream>>>(c.kp, static_cast<const float*>(c.rin),
                                                        static_cast<float*>(c.mu));
    }
  } else {
    dim3 gm((c.kp.nx + M2X - 1) / M2X, (c.kp.ny + M2Y - 1) / M2Y);
    k_mu2d<S, RPT><<<gm, NT2S, Sh::bytes, c.stream>>>(c.kp, static_cast<const float*>(c.rin),
                                                      static_cast<float*>(c.mu));
  }
  if (c.ev_mid) cudaEventRecord(c.ev_mid, c.stream);
  dim3 gc((c.kp.nx + T2X - 1) / T2X, (c.kp.ny + T2Y - 1) / T2Y);
  if (nblocks) *nblocks = int(gc.x * gc.y);
  k_coll2d<S, TAU1, RPT><<<gc, NT2S, Sh::bytes, c.stream>>>(c.kp, static_cast<const float*>(c.fin),
                                                       static_cast<float*>(c.fout), static_cast<const float*>(c.rin),
                                                       static_cast<const float*>(c.mu), static_cast<float*>(c.rout),
                                                       c.aux, c.mrt);
  return cudaGetLastError();
}

// tile rows per thread of the handle (Launch::rpt2d: 1, 2 or 4; 0 = default)
template <int S, bool TAU1>
cudaError_t launch_split2d(const Launch& c, int* nblocks) {
  if (c.rpt2d == 1) return launch_split2d_t<S, TAU1, 1>(c, nblocks);
  if (c.rpt2d == 4) return launch_split2d_t<S, TAU1, 4>(c, nblocks);
  return launch_split2d_t<S, TAU1, 2>(c, nblocks);
}

template <int S, class P>
cudaError_t launch(const Launch& c, int mode, int* nblocks) {
  if constexpr (std::is_same<P, PrecF32>::value) {
    if (mode == MODE_STEP && c.mu)
      return c.kp.omega == 1.0 ? launch_split2d<S, true>(c, nblocks) : launch_split2d<S, false>(c, nblocks);
  }
  if (mode == MODE_STEP_OBS) return cudaErrorNotSupported;
  if (mode == MODE_STEP) return launch_mode<S, P, MODE_STEP>(c, nblocks);
  if (mode == MODE_OBS) return launch_mode<S, P, MODE_OBS>(c, nblocks);
  return launch_mode<S, P, MODE_FIELDS>(c, nblocks);
}

template <int S>
StepFn pick(int prec) {
  if (prec == 0) return launch<S, PrecF64>;
  if (prec == 1) return launch<S, PrecF32>;
  return launch<S, PrecF32M64>;
}
}  // namespace

long long step2d_obs_ctas(const KParams& kp) {
  return (long long)((kp.nx + TX2 - 1) / TX2) * ((kp.ny + TY2 - 1) / TY2);
}

bool split2d_scheme(int scheme, int prec) {
  return prec == 1 && (scheme == S_EFDS2 || scheme == S_EFDS4 || scheme == S_EFDS6 || scheme == S_E4 || scheme == S_E8);
}

StepFn step2d_fn(int scheme, int prec) {
  switch (scheme) {
    case S_EFDS2: return pick<S_EFDS2>(prec);
    case S_EFDS4: return pick<S_EFDS4>(prec);
    case S_EFDS6: return pick<S_EFDS6>(prec);
    case S_E4: return pick<S_E4>(prec);
    case S_E8: return pick<S_E8>(prec);
    default: return nullptr;
  }
}

}  // namespace lbmd
