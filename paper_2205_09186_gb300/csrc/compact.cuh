// Compact difference schemes (Eq. 21-24 and the optimal fourth-order scheme of
// Sec. 3.1).  On a periodic lattice each grid line gives a cyclic tridiagonal
// system (alpha, 1, alpha) for the derivative; it is solved on chip by
// parallel cyclic reduction (PCR), one shared-memory line per system.  The
// step then runs as: mu field -> line solves for grad mu and grad rho along
// every axis -> the fused collide/stream kernel reading those fields.
#pragma once
#include <cuda_runtime.h>

#include "launch.cuh"

namespace lbmd {

struct LineCoef {
  double A1, A2, A3;  // a/2, b/4, c/6 of the explicit side of Eq. 21
  int nlev;           // PCR levels until |alpha_k| < 1e-17
  double alpha[16], inv[16];
  float alpha_f[16], inv_f[16];  // the same rounded to float (FP32 lines: no FP64 conversion per level)
};

struct CompactBufs {
  void* mu = nullptr;    // mu field (Tm)
  void* gmu = nullptr;   // grad mu (Tm), component-major
  void* grho = nullptr;  // grad rho (Tc), component-major
  size_t mu_bytes = 0, gmu_bytes = 0, grho_bytes = 0;
  LineCoef lc{};
  int lap_order = 4;
  // D3Q19 FP32: a second stream on which the density's line solves run while
  // the handle's stream computes mu and its line solves (fork and join events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// coefficients (alpha, a, b, c) of the compact schemes; OCFDS4 takes the
// printed alpha and c with a, b from the fourth-order conditions
// a + b + c = 1 + 2 alpha and a + 4 b + 9 c = 6 alpha
void compact_coeffs(int scheme, double* alpha, double* a, double* b, double* c);
LineCoef make_line_coef(int scheme);

template <class AllocF>
int compact_alloc(CompactBufs& cb, const KParams& kp, int D, int scheme, int prec, AllocF alloc) {
  const size_t tm = (prec == 1) ? 4 : 8;  // FP32 mu only in mode 1
  const size_t tc = (prec == 0) ? 8 : 4;
  cb.mu_bytes = size_t(kp.n) * tm;
  cb.gmu_bytes = size_t(D) * kp.n * tm;
  cb.grho_bytes = size_t(D) * kp.n * tc;
  cb.mu = alloc(cb.mu_bytes);
  cb.gmu = alloc(cb.gmu_bytes);
  cb.grho = alloc(cb.grho_bytes);
  cb.lc = make_line_coef(scheme);
  cb.lap_order = (scheme == 4) ? 6 : (scheme == 5 ? 8 : 4);
  if (!(cb.mu && cb.gmu && cb.grho)) return -2;
  if (prec == 1 && D == 3) {
    // the side stream at the lowest priority: the handle's stream carries the
    // critical path (mu, then mu's line solves)
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&cb.side, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&cb.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cb.join, cudaEventDisableTiming) != cudaSuccess)
      return -3;
  }
  return 0;
}

template <class FreeF>
void compact_free(CompactBufs& cb, FreeF fr) {
  if (cb.mu) fr(cb.mu, cb.mu_bytes);
  if (cb.gmu) fr(cb.gmu, cb.gmu_bytes);
  if (cb.grho) fr(cb.grho, cb.grho_bytes);
  cb.mu = cb.gmu = cb.grho = nullptr;
  if (cb.side) cudaStreamDestroy(cb.side);
  if (cb.fork) cudaEventDestroy(cb.fork);
  if (cb.join) cudaEventDestroy(cb.join);
  cb.side = nullptr;
  cb.fork = cb.join = nullptr;
}

cudaError_t compact_step(const CompactBufs& cb, Launch c, int D, int scheme, int prec, int mode, int* nblocks);

}  // namespace lbmd
