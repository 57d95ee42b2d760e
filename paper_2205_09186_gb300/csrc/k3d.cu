// Instantiations of the fused 2.5D D3Q19 step for the explicit and isotropic schemes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include <cudaTypedefs.h>

#include "launch.cuh"
#include "step3d.cuh"
#include "step3d_fast.cuh"
#include "step3d_split.cuh"
#include "coll3d_launch.cuh"

namespace lbmd {

static int num_sms() { return device_sms(); }

// FP32DEV with the FP32 chemical potential (prec 1) or with the EOS part of
// it evaluated in FP64 (prec 2) in the mu pass; the collision pass is the same
bool split3d_scheme(int scheme, int prec) {
  return (prec == 1 || prec == 2) && (scheme == S_EFDS2 || scheme == S_EFDS4 || scheme == S_EFDS6);
}

// z-chunk for the split collision pass: last-wave balance against the
// prologue (2R planes of field loads and two extra collided planes) for tiles
// of ty rows and per_sm resident CTAs per SM
static int split_zchunk_heuristic(const KParams& kp, int R, int ty, int per_sm) {
  const long long tiles = (long long)ColTiles(kp.nx).nt * RowBands(kp.ny, ty).nb;
  const long long slots = (long long)per_sm * num_sms();
  double best = 1e300;
  int best_zc = kp.nz;
  for (int nzc = 1; nzc <= kp.nz && nzc <= 128; ++nzc) {
    const int zc = (kp.nz + nzc - 1) / nzc;
    if (zc < 4 && nzc > 1) break;
    const long long ctas = tiles * ((kp.nz + zc - 1) / zc);
    const double waves = double((ctas + slots - 1) / slots);
    const double cost = waves * (zc + 2 + 0.2 * 2 * R);
    if (cost < best - 1e-9) { best = cost; best_zc = zc; }
  }
  return best_zc;
}

// CTAs of one collision pass (k_coll3d): 32-column tiles x row bands x z chunks
static long long coll3d_ctas(const KParams& kp, int zc) {
  return (long long)ColTiles(kp.nx).nt * RowBands(kp.ny, CY).nb * ((kp.nz + zc - 1) / zc);
}

long long coll3d_corner_count(const KParams& kp) {
  return 4LL * ColTiles(kp.nx).nt * RowBands(kp.ny, CY).nb * kp.nz;
}

float coll3d_corner_scale(int eos, double b) {
  const double rmax = (eos == LBM_EOS_CS ? 4.0 : 1.0) / (b > 0 ? b : 1.0);
  // |partial| <= 2 rmax <= 2^e; four of them: 4 * 2^e * 2^s <= 2^62
  int e = 0;
  while (std::ldexp(1.0, e) < 2.0 * rmax && e < 40) ++e;
  const int s = std::min(60, 60 - e);
  return float(std::ldexp(1.0, s));
}

int fast_zchunk_heuristic(const KParams& kp, int R) {
  const int sms = num_sms();
  const long long tiles = (long long)((kp.nx + FT - 1) / FT) * ((kp.ny + FT - 1) / FT);
  const long long slots = 2LL * sms;  // two CTAs per SM
  double best = 1e300;
  int best_zc = kp.nz;
  for (int nzc = 1; nzc <= kp.nz && nzc <= 128; ++nzc) {
    const int zc = (kp.nz + nzc - 1) / nzc;
    if (zc < 4 && nzc > 1) break;
    const long long ctas = tiles * ((kp.nz + zc - 1) / zc);
    const double waves = double((ctas + slots - 1) / slots);
    const double cost = waves * (zc + 2 + 0.3 * 4 * R);
    if (cost < best - 1e-9) { best = cost; best_zc = zc; }
  }
  return best_zc;
}

constexpr int TX3 = 32, TY3 = 8, ZC3 = 32;

namespace {

template <int S, class P, int MODE>
cudaError_t launch_mode(const Launch& c, int* nblocks) {
  using Sh = Step3DShape<S, P, TX3, TY3>;
  auto k = k_step3d<S, P, TX3, TY3, ZC3, MODE>;
  if (cudaError_t e = ensure_smem(k, Sh::bytes); e != cudaSuccess) return e;
  dim3 grid((c.kp.nx + TX3 - 1) / TX3, (c.kp.ny + TY3 - 1) / TY3, (c.kp.nz + ZC3 - 1) / ZC3);
  if (nblocks) *nblocks = int(grid.x * grid.y * grid.z);
  using Tf = typename P::Tf;
  using Tr = typename P::Tr;
  k<<<grid, NT3, Sh::bytes, c.stream>>>(c.kp, static_cast<const Tf*>(c.fin), static_cast<Tf*>(c.fout),
                                        static_cast<const Tr*>(c.rin), static_cast<Tr*>(c.rout),
                                        c.aux, c.fo, c.gi);
  return cudaGetLastError();
}

// FP32 deviation storage with FP32 mu: the pipelined kernel (step mode)
template <int S, bool TAU1>
cudaError_t launch_fast(const Launch& c, int* nblocks) {
  using Sh = FastShape<S>;
  auto k = k_step3d_fast<S, TAU1>;
  if (cudaError_t e = ensure_smem(k, Sh::bytes); e != cudaSuccess) return e;
  const int zc = c.zc > 0 ? c.zc : fast_zchunk_heuristic(c.kp, Sh::R);
  dim3 grid((c.kp.nx + FT - 1) / FT, (c.kp.ny + FT - 1) / FT, (c.kp.nz + zc - 1) / zc);
  if (nblocks) *nblocks = int(grid.x * grid.y * grid.z);
  k<<<grid, FNT, Sh::bytes, c.stream>>>(c.kp, static_cast<const float*>(c.fin), static_cast<float*>(c.fout),
                                        static_cast<const float*>(c.rin), static_cast<float*>(c.rout), c.aux, zc);
  return cudaGetLastError();
}


static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }


// the mu pass: the vector kernel when rows are whole 16-byte chunks; with
// zero_edges it also prepares c.rout for the collision pass (EdgeZero)
template <int S, bool M64 = false>
cudaError_t launch_mu(const Launch& c, bool zero_edges = false) {
  const EdgeZero ez{zero_edges ? static_cast<float*>(c.rout) : nullptr, CY, c.aux.bad_step, c.aux.t};
  if (zero_edges && !c.rout) return cudaErrorInvalidValue;
  if (c.kp.nx % 4 == 0 && aligned16(c.rin) && aligned16(c.mu)) {
    // z chunks: enough CTAs for several waves, at least 8 planes per chunk
    const int gx = (c.kp.nx + MZX - 1) / MZX, gy = (c.kp.ny + MZY - 1) / MZY;
    const long long want = 8LL * num_sms();
    const int nzc = int(std::max<long long>(1, std::min<long long>((want + gx * gy - 1) / (gx * gy),
                                                                    (c.kp.nz + 7) / 8)));
    const int zc = (c.kp.nz + nzc - 1) / nzc;
    dim3 g(gx, gy, (c.kp.nz + zc - 1) / zc);
    k_mu3d_zm<S, M64><<<g, MZT, MuZShape<S>::bytes, c.stream>>>(c.kp, static_cast<const float*>(c.rin),
                                                                static_cast<float*>(c.mu), zc, ez);
  } else {
    dim3 g((c.kp.nx + MUX - 1) / MUX, (c.kp.ny + MUY - 1) / MUY, (c.kp.nz + MUZ - 1) / MUZ);
    k_mu3d<S, M64><<<g, MUT, 0, c.stream>>>(c.kp, static_cast<const float*>(c.rin), static_cast<float*>(c.mu), ez);
  }
  return cudaGetLastError();
}

// mu pass + collision pass (line schemes, FP32DEV, FP32 mu); with obs the
// collision pass also reduces the observables of the state it advances
template <int S, bool TAU1, bool M64 = false>
cudaError_t launch_split(const Launch& c, int* nblocks, bool obs) {
  if (!c.mu) return cudaErrorInvalidValue;
  const int zc = c.zc > 0 ? c.zc : split_zchunk_heuristic(c.kp, Sch<S>::R, TYC, CollShape<S, CY, 2, COLL_FD>::MINB);
  const long long ctas = coll3d_ctas(c.kp, zc);
  if (nblocks) {
    // observation: the caller's partials buffer holds *nblocks entries
    if (obs && ctas > *nblocks) return cudaErrorNotSupported;
    *nblocks = int(ctas);
  } else if (obs) {
    return cudaErrorInvalidValue;
  }
  cudaError_t em = launch_mu<S, M64>(c, true);
  if (em != cudaSuccess) return em;
  if (c.ev_mid) cudaEventRecord(c.ev_mid, c.stream);
  // 16-byte copies need rows of whole chunks and aligned bases
  const bool vec = c.kp.nx % 4 == 0 && aligned16(c.fin) && aligned16(c.rin) && aligned16(c.mu) && c.tmap;
  if (obs)
    return vec ? launch_coll<S, TAU1, true, true>(c, zc) : launch_coll<S, TAU1, false, true>(c, zc);
  return vec ? launch_coll<S, TAU1, true, false>(c, zc) : launch_coll<S, TAU1, false, false>(c, zc);
}

// observation pass of the split path: mu field, then the node-parallel reduction
template <int S, bool M64 = false>
cudaError_t launch_obs_split(const Launch& c, int* nblocks) {
  cudaError_t em = launch_mu<S, M64>(c);
  if (em != cudaSuccess) return em;
  // at most 8192 CTAs: the handle's partials buffer holds at least that many
  const int nb = int(std::min<long long>(std::min<long long>((long long)c.kp.ny * c.kp.nz, 8LL * num_sms()), 8192LL));
  if (nblocks) *nblocks = nb;
  k_obs3d<S><<<nb, 256, 0, c.stream>>>(c.kp, static_cast<const float*>(c.fin), static_cast<const float*>(c.rin),
                                       static_cast<const float*>(c.mu), c.aux);
  return cudaGetLastError();
}

template <int S, class P>
cudaError_t launch(const Launch& c, int mode, int* nblocks) {
  if constexpr (std::is_same<P, PrecF32>::value && !Sch<S>::ISO) {
    if (mode == MODE_OBS && c.mu) return launch_obs_split<S>(c, nblocks);
  }
  if constexpr (std::is_same<P, PrecF32M64>::value && !Sch<S>::ISO && !Sch<S>::GF) {
    // line schemes with the FP64 EOS chemical potential: the split path
    if (c.mu) {
      if (mode == MODE_OBS) return launch_obs_split<S, true>(c, nblocks);
      if (mode == MODE_STEP || mode == MODE_STEP_OBS) {
        const bool obs = mode == MODE_STEP_OBS;
        return c.kp.omega == 1.0 ? launch_split<S, true, true>(c, nblocks, obs)
                                 : launch_split<S, false, true>(c, nblocks, obs);
      }
    }
  }
  if constexpr (std::is_same<P, PrecF32>::value) {
    if (mode == MODE_STEP || mode == MODE_STEP_OBS) {
      const bool obs = mode == MODE_STEP_OBS;
      if constexpr (!Sch<S>::ISO)
        return c.kp.omega == 1.0 ? launch_split<S, true>(c, nblocks, obs) : launch_split<S, false>(c, nblocks, obs);
      if (obs) return cudaErrorNotSupported;
      return c.kp.omega == 1.0 ? launch_fast<S, true>(c, nblocks) : launch_fast<S, false>(c, nblocks);
    }
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

long long step3d_obs_ctas(const KParams& kp) {
  return (long long)((kp.nx + TX3 - 1) / TX3) * ((kp.ny + TY3 - 1) / TY3) * ((kp.nz + ZC3 - 1) / ZC3);
}

bool make_coll3d_tmap(const void* f, const KParams& kp, void* out, int rows) {
  if (kp.nx % 4 != 0 || (reinterpret_cast<uintptr_t>(f) & 15) != 0) return false;
  // the driver's encoder, looked up once (a function-local static is
  // initialised once even when several host threads get here together)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  const cuuint64_t dims[4] = {cuuint64_t(kp.nx), cuuint64_t(kp.ny), cuuint64_t(kp.nz), 19};
  const cuuint64_t strides[3] = {cuuint64_t(kp.nx) * 4, cuuint64_t(kp.nx) * kp.ny * 4, cuuint64_t(kp.n) * 4};
  if (rows < 1 || rows > 32) return false;
  const cuuint32_t box[4] = {cuuint32_t(FW), cuuint32_t(rows), 1, 19};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return encode(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(f), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
// one thread per node of the band edge rows: blockIdx.y = 2 band + (0: first row, 1: last row)
__global__ void k_zero_edges(const KParams p, const float* __restrict__ rin, float* __restrict__ rout,
                             unsigned long long* bad, long long t) {
  const RowBands bands(p.ny, CY);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= p.nx) return;
  const int b = int(blockIdx.y) >> 1;
  const int y = (blockIdx.y & 1) ? bands.start(b + 1) - 1 : bands.start(b);
  const long long o = (long long)blockIdx.z * p.nx * p.ny + (long long)y * p.nx + x;
  rout[o] = 0.f;
  if (!(float(p.rho_ref) + rin[o] > 0.f)) atomicMin(bad, (unsigned long long)t);
}
// one thread per node of the tile edge columns: blockIdx.y = 2 tile + (0: first column, 1: last column)
__global__ void k_zero_edge_cols(const KParams p, const float* __restrict__ rin, float* __restrict__ rout,
                                 unsigned long long* bad, long long t) {
  const ColTiles tiles(p.nx);
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= p.ny) return;
  const int k = int(blockIdx.y) >> 1;
  const int x = (blockIdx.y & 1) ? tiles.start(k + 1) - 1 : tiles.start(k);
  const long long o = (long long)blockIdx.z * p.nx * p.ny + (long long)y * p.nx + x;
  rout[o] = 0.f;
  if (!(float(p.rho_ref) + rin[o] > 0.f)) atomicMin(bad, (unsigned long long)t);
}
}  // namespace

cudaError_t coll3d_zero_edges(const KParams& kp, const float* rin, float* rout, unsigned long long* bad, long long t,
                              cudaStream_t st) {
  if (!rin || !rout || !bad || kp.nz > 65535) return cudaErrorInvalidValue;
  const dim3 g((kp.nx + 127) / 128, 2 * RowBands(kp.ny, CY).nb, kp.nz);
  k_zero_edges<<<g, 128, 0, st>>>(kp, rin, rout, bad, t);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
  const dim3 gc((kp.ny + 127) / 128, 2 * ColTiles(kp.nx).nt, kp.nz);
  k_zero_edge_cols<<<gc, 128, 0, st>>>(kp, rin, rout, bad, t);
  return cudaGetLastError();
}

bool coll3d_gf_ok(const Launch& c) {
  return c.kp.nx % 4 == 0 && aligned16(c.fin) && aligned16(c.rin) && c.tmap && c.rout;
}

cudaError_t coll3d_gf_step(const Launch& c, int* nblocks) {
  if (!coll3d_gf_ok(c) || !c.gi.gmu || !c.gi.grho) return cudaErrorNotSupported;
  const int zc = c.zc > 0 ? c.zc : split_zchunk_heuristic(c.kp, 0, TYC, 2);
  if (nblocks) *nblocks = int(coll3d_ctas(c.kp, zc));
  return c.kp.omega == 1.0 ? launch_coll<S_CFDS4, true, true, false>(c, zc)
                           : launch_coll<S_CFDS4, false, true, false>(c, zc);
}

cudaError_t mu3d_pass(const Launch& c, int order, bool zero_edges) {
  if (order == 4) return launch_mu<S_EFDS4>(c, zero_edges);
  if (order == 6) return launch_mu<S_EFDS6>(c, zero_edges);
  return cudaErrorNotSupported;
}

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
