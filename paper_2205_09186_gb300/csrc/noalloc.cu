// Observables of a caller-held state without any device allocation.
//
// lbm_observables needs a handle, whose buffers (including the per-CTA
// partial results of the reduction) come from an allocator.  Some callers
// cannot let a library allocate: a solver embedded in a host application that
// owns every device buffer under a fixed memory budget, or code running where
// a new cudaMalloc would stall or fail.  This entry point takes the state as
// plain device pointers and keeps the reduction's partial results in a fixed
// file-scope device array instead.
//
// The array (kMaxCtas x 4 partial values + 16 result words, about 2 MiB) is
// held by every GPU that loads the library until the process exits.  Every
// call shares it and it keeps the previous call's contents: the status word is
// cleared by each call, the partials and results are overwritten.  Calls whose
// work overlaps on the GPU (different streams, or host threads without
// ordering) race on the array; serialise them.  The address cached per device
// belongs to the device's context: after a cudaDeviceReset the library is not
// usable on that device again in the same process.
//
// The observation pass is the periodic one, with no wall mask: a state
// produced with walls (lbm_set_solid) would count its wall nodes in the mass
// and the velocity maxima, so this entry point is for states without walls.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstring>

#include "../../include/lbm.h"
#include "launch.cuh"

using namespace lbmd;

namespace {

constexpr long long kMaxCtas = 65536;            // observation-pass CTAs supported
constexpr long long kResults = kMaxCtas * 4;     // offset of the 16 result words

static __device__ __align__(256) double g_obs_scratch[kMaxCtas * 4 + 16];

constexpr int kMaxDevices = 64;
// device address of the array, per device: looked up by the first call on
// that device; atomic, since host threads may make their first calls together
// (each finds the same address)
std::atomic<double*> g_scratch_addr[kMaxDevices] = {};

// fixed-order reduction of the per-CTA partials (max, max, sum, max)
template <typename Tr>
__global__ void k_noalloc_final(const double* part, int nb, const Tr* rho, double rho_ref, long long center,
                                double* res) {
  __shared__ double red[4][256];
  double a = 0, b = 0, c = 0, d = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a = fmax(a, part[4 * i]);
    b = fmax(b, part[4 * i + 1]);
    c += part[4 * i + 2];
    d = fmax(d, part[4 * i + 3]);
  }
  red[0][threadIdx.x] = a; red[1][threadIdx.x] = b; red[2][threadIdx.x] = c; red[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
      red[2][threadIdx.x] += red[2][threadIdx.x + s];
      red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    res[0] = red[0][0]; res[1] = red[1][0]; res[2] = red[2][0]; res[3] = red[3][0];
    res[4] = sizeof(Tr) == 8 ? double(rho[center]) : rho_ref + double(rho[center]);
    res[5] = sizeof(Tr) == 8 ? double(rho[0]) : rho_ref + double(rho[0]);
  }
}

}  // namespace

extern "C" int lbm_observables_noalloc(const lbm_params* p, const void* d_f, const void* d_rho,
                                       const void* d_rho_prev, long long steps_since_prev, long long step,
                                       void* stream, lbm_obs* out) {
  if (!p || !d_f || !d_rho || !out || steps_since_prev < 0) return LBM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return LBM_EINVAL;
  if (p->nx < 8 || p->ny < 8 || (p->lattice == LBM_D2Q9 ? p->nz != 1 : p->nz < 8)) return LBM_EINVAL;
  if ((long long)p->nx * p->ny * p->nz > (1LL << 31) / 19) return LBM_EINVAL;
  if (!(p->a > 0 && p->b > 0 && p->R > 0 && p->Tr > 0 && p->k > 0 && p->kappa >= 0 && p->tau > 0.5)) return LBM_EINVAL;
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32DEV) return LBM_EINVAL;
  if (p->scheme >= LBM_CFDS4 && p->scheme <= LBM_OCFDS4) return LBM_ENOTSUP;  // needs gradient fields
  const int prec = p->precision == LBM_FP64 ? 0 : (p->mu_fp64 ? 2 : 1);
  const bool d3 = p->lattice == LBM_D3Q19;
  StepFn fn = d3 ? step3d_fn(p->scheme, prec) : step2d_fn(p->scheme, prec);
  if (!fn) return LBM_ENOTSUP;

  KParams kp;
  if (params_to_kp(p, &kp) != LBM_OK) return LBM_EINVAL;
  const long long nctas = d3 ? step3d_obs_ctas(kp) : step2d_obs_ctas(kp);
  if (nctas > kMaxCtas) return LBM_ESCRATCH;

  // once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
  double* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    if (cudaGetSymbolAddress((void**)&scratch, g_obs_scratch) != cudaSuccess || !scratch) return LBM_ECUDA;
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }
  double* res = scratch + kResults;
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(res + 8);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // the status word must start at "no bad step"
  if (cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st) != cudaSuccess) return LBM_ECUDA;
  Launch c{};
  c.kp = kp;
  c.fin = d_f;
  c.fout = nullptr;
  c.rin = d_rho;
  c.rout = nullptr;
  c.aux.t = step;
  c.aux.bad_step = bad;
  c.aux.partials = scratch;
  c.aux.rho_snap = d_rho_prev ? d_rho_prev : d_rho;
  c.stream = st;
  int nb = 0;
  if (fn(c, MODE_OBS, &nb) != cudaSuccess) return LBM_ECUDA;
  const long long center = (long long)(p->nz / 2) * p->nx * p->ny + (long long)(p->ny / 2) * p->nx + p->nx / 2;
  if (prec == 0)
    k_noalloc_final<double><<<1, 256, 0, st>>>(scratch, nb, static_cast<const double*>(d_rho), 0.0, center, res);
  else
    k_noalloc_final<float><<<1, 256, 0, st>>>(scratch, nb, static_cast<const float*>(d_rho), kp.rho_ref, center, res);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  double host[9];
  if (cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBM_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ECUDA;
  unsigned long long b;
  std::memcpy(&b, &host[8], 8);
  out->max_v = host[0];
  out->max_u = host[1];
  out->mass = host[2];
  out->max_drho = (d_rho_prev && steps_since_prev > 0) ? host[3] / double(steps_since_prev) : 0.0;
  out->rho_center = host[4];
  out->rho_corner = host[5];
  out->step = step;
  out->status = LBM_OK;
  if (b != ULLONG_MAX) {
    out->status = LBM_EUNSTABLE;
    return LBM_EUNSTABLE;
  }
  return LBM_OK;
}
