// Launch descriptors shared by the kernel translation units and the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "step2d.cuh"

namespace lbmd {

struct Launch {
  KParams kp;
  const void* fin;
  void* fout;
  const void* rin;   // density field, type P::Tr
  void* rout;
  StepAux aux;
  FieldOut fo;
  GradIn gi;
  cudaStream_t stream;
  int zc;       // z-chunk of the pipelined D3Q19 kernel; 0 = heuristic
  void* mu;     // N floats: mu field of the split D3Q19 FP32DEV path (else unused)
  Mrt mrt;      // D2Q9 collision operator (on = 0: single relaxation)
  cudaEvent_t ev_mid;  // if set: recorded between the mu pass and the collision pass
  const void* tmap;    // D3Q19 FP32DEV: tensor map (CUtensorMap) of the populations fin, or null
  int rpt2d;           // D2Q9 FP32DEV split tiles: rows per thread (1, 2, 4; 0 = default 2)
  // D3Q19 FP32DEV collision pass: corner accumulators (coll3d_corner_count
  // 64-bit integers, zero between passes) and their fixed-point scale
  unsigned long long* qc;
  float qscale;
};

// Kernel constants of a case: lattice size, the EOS at T = Tr T_c (either
// kind), k^2, kappa-hat, 1/tau and the FP32DEV reference density (p->rho_ref,
// or the Maxwell gas density when that is <= 0; 0 in FP64 mode).  Returns an
// LBM_ status.
int params_to_kp(const lbm_params* p, KParams* kp);

// the D3Q19 FP32DEV step of this scheme runs as mu pass + collision pass and
// needs an N-float mu buffer in Launch::mu
bool split3d_scheme(int scheme, int prec);
bool split2d_scheme(int scheme, int prec);

// z-chunk length for the pipelined D3Q19 kernel: balances the last wave of
// CTAs against the per-chunk prologue (4R + 2 extra planes, of which only 2
// are collided)
int fast_zchunk_heuristic(const KParams& kp, int R);

// launch one fused step (mode MODE_STEP), an observation pass (MODE_OBS) or a
// field dump (MODE_FIELDS); returns the number of CTAs through *nblocks
using StepFn = cudaError_t (*)(const Launch&, int mode, int* nblocks);

// precision index: 0 = FP64, 1 = FP32DEV with FP32 mu, 2 = FP32DEV with FP64 mu
StepFn step2d_fn(int scheme, int prec);
StepFn step3d_fn(int scheme, int prec);

// Corner accumulators of the D3Q19 FP32-deviation collision pass: four per
// tile and band in every plane.
long long coll3d_corner_count(const KParams& kp);

// Fixed-point scale of those accumulators: 2^s with s as large as keeps any
// partial sum of population deviations (bounded by twice the largest density
// the EOS allows: 4/b for Carnahan-Starling, 1/b for the cubic EOS) inside
// the 64-bit range with a factor eight to spare (four addends, and two).
float coll3d_corner_scale(int eos, double b);

// Tensor map of a D3Q19 FP32-deviation population array f[19][nz][ny][nx]
// for the collision pass's tensor copies (box 32 x rows x 1 x 19; rows = the
// collision region's rows, 11 for the tiles the library launches), written to out (a
// CUtensorMap, 128 bytes, 64-byte aligned).  False when the lattice or the
// pointer does not allow one (nx % 4 != 0, unaligned base) or the driver
// refuses it.
bool make_coll3d_tmap(const void* f, const KParams& kp, void* out, int rows = 11);


// D3Q19 FP32 mu field (Eq. 16) with the explicit central Laplacian of the
// given order (4 or 6) from c.rin into c.mu (N floats): the mu pass of the
// split path, shared with the compact schemes.  zero_edges: also zero the
// nodes of c.rout that the collision pass completes by atomic addition (the
// edge rows of its row bands, the edge columns of its tiles), as
// coll3d_gf_step needs.
cudaError_t mu3d_pass(const Launch& c, int order, bool zero_edges);

// Zero the edge rows and edge columns of the collision pass's bands and tiles
// in rout (N floats) and flag step t in bad where the density rin is not
// positive there: what mu3d_pass does with zero_edges, for a mu field
// computed otherwise.
cudaError_t coll3d_zero_edges(const KParams& kp, const float* rin, float* rout, unsigned long long* bad, long long t,
                              cudaStream_t st);

// D3Q19 FP32DEV collision pass of the compact schemes on the tiled z-marching
// kernel, the derivatives read from c.gi (gmu, grho: 3 x N floats each).
// coll3d_gf_ok tells whether the lattice and buffers allow it; when they do,
// the edge nodes of c.rout must have been zeroed in this step (mu3d_pass with
// zero_edges, or coll3d_zero_edges) before coll3d_gf_step runs.  Otherwise
// cudaErrorNotSupported, nothing launched.
bool coll3d_gf_ok(const Launch& c);
cudaError_t coll3d_gf_step(const Launch& c, int* nblocks);

// Raise kernel fn's dynamic shared-memory limit to at least `bytes` on the
// current device.  The attribute belongs to one device (context): it is set
// once per device and kernel, under a lock, so handles on several GPUs and
// several host threads may launch.  A cudaDeviceReset drops every attribute
// (and every handle's memory) of that device: the library is not usable on it
// again in the same process.
cudaError_t ensure_smem(const void* fn, size_t bytes);
template <class K>
inline cudaError_t ensure_smem(K* fn, size_t bytes) { return ensure_smem(reinterpret_cast<const void*>(fn), bytes); }

// multiprocessor count of the current device (looked up once per device)
int device_sms();

// number of CTAs (hence partial results) of the observation pass
long long step2d_obs_ctas(const KParams& kp);
long long step3d_obs_ctas(const KParams& kp);

}  // namespace lbmd
