// Instantiations of the fused 2.5D D3Q19 step for the explicit and isotropic schemes.
#include "launch.cuh"
#include "step3d.cuh"

namespace lbmd {

namespace {
constexpr int TX3 = 32, TY3 = 8, ZC3 = 32;

template <int S, class P, int MODE>
cudaError_t launch_mode(const Launch& c, int* nblocks) {
  using Sh = Step3DShape<S, P, TX3, TY3>;
  auto k = k_step3d<S, P, TX3, TY3, ZC3, MODE>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::bytes));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((c.kp.nx + TX3 - 1) / TX3, (c.kp.ny + TY3 - 1) / TY3, (c.kp.nz + ZC3 - 1) / ZC3);
  if (nblocks) *nblocks = int(grid.x * grid.y * grid.z);
  using Tf = typename P::Tf;
  k<<<grid, NT3, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout), c.rin, c.rout,
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

StepFn step3d_fn(int scheme, int prec) {
  switch (scheme) {
    case S_EFDS2: return pick<S_EFDS2>(prec);
    case S_EFDS4: return pick<S_EFDS4>(prec);
    case S_EFDS6: return pick<S_EFDS6>(prec);
    case S_E4: return pick<S_E4>(prec);
    default: return nullptr;
  }
}

}  // namespace lbmd
