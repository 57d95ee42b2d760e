// Instantiations of the fused D2Q9 step for the explicit and isotropic schemes.
#include "launch.cuh"
#include "step2d.cuh"

namespace lbmd {

constexpr int TX2 = 32, TY2 = 8;

namespace {

template <int S, class P, int MODE>
cudaError_t launch_mode(const Launch& c, int* nblocks) {
  using Sh = Step2DShape<S, P, TX2, TY2>;
  auto k = k_step2d<S, P, TX2, TY2, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::bytes));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((c.kp.nx + TX2 - 1) / TX2, (c.kp.ny + TY2 - 1) / TY2, 1);
  if (nblocks) *nblocks = int(grid.x * grid.y);
  using Tf = typename P::Tf;
  using Tr = typename P::Tr;
  k<<<grid, NT2, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout),
                                        static_cast<const Tr*>(c.rin), static_cast<Tr*>(c.rout),
                                        c.aux, c.fo, c.gi);
  return cudaGetLastError();
}

template <int S, class P>
cudaError_t launch(const Launch& c, int mode, int* nblocks) {
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
