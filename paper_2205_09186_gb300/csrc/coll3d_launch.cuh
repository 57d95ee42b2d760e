// Launcher of the D3Q19 FP32-deviation collision pass (k_coll3d) for one tile
// shape: 32-column tiles (ColTiles), bands of RY rows (RowBands) and NB staged
// population planes, followed by k_coll3d_corners.  The pass adds into the
// edge rows and edge columns of its output density: the mu pass of the same
// step (launch_mu with an EdgeZero of the same RY) must have zeroed them.
#pragma once
#include <cuda.h>

#include <algorithm>

#include "launch.cuh"
#include "step3d_split.cuh"

namespace lbmd {

template <int S, bool TAU1, bool VEC, bool OBS, int RY = CY, int NB = 2, int FD = (Sch<S>::GF ? 1 : COLL_FD)>
cudaError_t launch_coll(const Launch& c, int zc) {
  using Sh = CollShape<S, RY, NB, FD>;
  auto kc = k_coll3d<S, TAU1, VEC, OBS, RY, NB, FD>;
  constexpr size_t by = OBS ? Sh::bytes_obs : Sh::bytes;
  static_assert(by <= size_t(227) * 1024, "shared memory of one CTA");
  CUtensorMap tm{};
  if constexpr (VEC) {
    if (!c.tmap) return cudaErrorInvalidValue;
    if constexpr (RY == CY) {
      tm = *static_cast<const CUtensorMap*>(c.tmap);
    } else {
      // the handle keeps maps for the default box height; other shapes
      // encode theirs (a host-side call) for the launch's populations
      if (!make_coll3d_tmap(c.fin, c.kp, &tm, RY)) return cudaErrorInvalidValue;
    }
  }
  if (!c.qc || !(c.qscale > 0.f)) return cudaErrorInvalidValue;
  if (cudaError_t e = ensure_smem(kc, by); e != cudaSuccess) return e;
  const ColTiles tiles(c.kp.nx);
  const RowBands bands(c.kp.ny, RY);
  const dim3 grid(tiles.nt, bands.nb, (c.kp.nz + zc - 1) / zc);
  kc<<<grid, Sh::NT, by, c.stream>>>(c.kp, static_cast<const float*>(c.fin), static_cast<float*>(c.fout),
                                     static_cast<const float*>(c.rin), static_cast<const float*>(c.mu),
                                     static_cast<float*>(c.rout), c.aux, zc,
                                     OBS ? static_cast<float*>(const_cast<void*>(c.aux.rho_snap)) : nullptr, tm,
                                     static_cast<const float*>(c.gi.gmu), static_cast<const float*>(c.gi.grho), c.qc,
                                     c.qscale);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
  const long long ncorner = 4LL * tiles.nt * bands.nb * c.kp.nz;
  const int nblk = int(std::min<long long>((ncorner + 255) / 256, 4096LL));
  k_coll3d_corners<<<nblk, 256, 0, c.stream>>>(c.kp, RY, c.qc, static_cast<float*>(c.rout), 1.f / c.qscale,
                                               c.aux.bad_step, c.aux.t + 1);
  return cudaGetLastError();
}

}  // namespace lbmd
