// Wall (Appendix A) step of a handle: the common launch descriptor plus the
// wall layers (0 fluid, 1..3 wall layers, 4 deeper), the wall chemical
// potential and an N-value mu buffer (of the precision's mu type).
#pragma once
#include "launch.cuh"

namespace lbmd {

struct WallLaunch {
  Launch c;
  const signed char* layer;
  double mu_w;
  void* mu;
};

// wall densities only (layers 1..3 of c.rin, in place)
constexpr int MODE_WALL_FILL = 16;

// mode MODE_STEP, MODE_OBS (partials into c.aux.partials, *nblocks set),
// MODE_FIELDS (F and mu into c.fo; F = 0 and mu = mu_w on wall nodes) or
// MODE_WALL_FILL; explicit line schemes only (else cudaErrorNotSupported)
cudaError_t wall_step(const WallLaunch& w, int lattice, int scheme, int prec, int mode, int* nblocks);

}  // namespace lbmd
