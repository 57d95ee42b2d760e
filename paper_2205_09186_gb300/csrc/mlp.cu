// Warm-start network: a small fully connected GELU network (FP32) that maps
// droplet parameters to an initial radial density profile.  Forward, backward
// (mean-squared error) and Adam run as CUDA kernels; the training loop stays
// on the device.  There is no counterpart in the paper: the network only
// supplies initial conditions that the solver then relaxes.
//
// Parameter layout (as in the C ABI): per layer W (out x in, row-major) then b.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm.h"

namespace {

constexpr int SB = 32;     // samples per CTA
constexpr int MAXW = 128;  // widest layer supported
constexpr int MAXL = 8;    // layers supported

struct Net {
  int nl;
  int sizes[MAXL + 1];
  long long woff[MAXL], boff[MAXL];  // parameter offsets
};

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// forward for a block of SB samples; pre-activations z[l][s][o] and
// activations kept for backward in global scratch (act: per layer B x width)
__global__ void k_mlp_forward(const Net net, const float* __restrict__ P, const float* __restrict__ x, int B,
                              float* __restrict__ y, float* __restrict__ zs, float* __restrict__ hs) {
  __shared__ float h[SB][MAXW + 1];
  __shared__ float hn[SB][MAXW + 1];
  const int s0 = blockIdx.x * SB;
  const int ns = min(SB, B - s0);
  const int in0 = net.sizes[0];
  for (int idx = threadIdx.x; idx < SB * in0; idx += blockDim.x) {
    const int s = idx / in0, i = idx - s * in0;
    h[s][i] = s < ns ? x[(long long)(s0 + s) * in0 + i] : 0.f;
  }
  __syncthreads();
  long long zoff = 0;
  for (int l = 0; l < net.nl; ++l) {
    const int in = net.sizes[l], out = net.sizes[l + 1];
    const float* W = P + net.woff[l];
    const float* b = P + net.boff[l];
    for (int o = threadIdx.x; o < out; o += blockDim.x) {
      float acc[SB];
#pragma unroll
      for (int s = 0; s < SB; ++s) acc[s] = b[o];
      for (int i = 0; i < in; ++i) {
        const float w = W[(long long)o * in + i];
#pragma unroll
        for (int s = 0; s < SB; ++s) acc[s] += w * h[s][i];
      }
#pragma unroll
      for (int s = 0; s < SB; ++s) {
        if (s < ns) zs[zoff + (long long)(s0 + s) * out + o] = acc[s];
        hn[s][o] = (l < net.nl - 1) ? gelu(acc[s]) : acc[s];
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < SB * out; idx += blockDim.x) {
      const int s = idx / out, o = idx - s * out;
      h[s][o] = hn[s][o];
      if (s < ns && l < net.nl - 1) hs[zoff + (long long)(s0 + s) * out + o] = hn[s][o];
    }
    __syncthreads();
    zoff += (long long)B * out;
  }
  const int nout = net.sizes[net.nl];
  for (int idx = threadIdx.x; idx < ns * nout; idx += blockDim.x) {
    const int s = idx / nout, o = idx - s * nout;
    y[(long long)(s0 + s) * nout + o] = h[s][o];
  }
}

// backward for a block of samples: per-CTA partial gradients (deterministic
// final reduction in k_reduce); loss partial per CTA
__global__ void k_mlp_backward(const Net net, const float* __restrict__ P, const float* __restrict__ x,
                               const float* __restrict__ t, int B, const float* __restrict__ y,
                               const float* __restrict__ zs, const float* __restrict__ hs, float* __restrict__ gpart,
                               long long nparam, float* __restrict__ lpart) {
  __shared__ float d[SB][MAXW + 1];
  __shared__ float dn[SB][MAXW + 1];
  __shared__ float hin[SB][MAXW + 1];
  __shared__ float red[256];
  const int s0 = blockIdx.x * SB;
  const int ns = min(SB, B - s0);
  const int nl = net.nl, nout = net.sizes[nl];
  const float scale = 2.f / (float(B) * float(nout));
  float lsum = 0.f;
  for (int idx = threadIdx.x; idx < SB * nout; idx += blockDim.x) {
    const int s = idx / nout, o = idx - s * nout;
    float v = 0.f;
    if (s < ns) {
      const float e = y[(long long)(s0 + s) * nout + o] - t[(long long)(s0 + s) * nout + o];
      lsum += e * e;
      v = e * scale;
    }
    d[s][o] = v;
  }
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
  // offsets of the stored activations per layer
  long long zoff[MAXL];
  long long acc = 0;
  for (int l = 0; l < nl; ++l) { zoff[l] = acc; acc += (long long)B * net.sizes[l + 1]; }
  float* g = gpart + (long long)blockIdx.x * nparam;
  for (int l = nl - 1; l >= 0; --l) {
    const int in = net.sizes[l], out = net.sizes[l + 1];
    // input activations of layer l
    for (int idx = threadIdx.x; idx < SB * in; idx += blockDim.x) {
      const int s = idx / in, i = idx - s * in;
      float v = 0.f;
      if (s < ns) v = (l == 0) ? x[(long long)(s0 + s) * in + i] : hs[zoff[l - 1] + (long long)(s0 + s) * in + i];
      hin[s][i] = v;
    }
    __syncthreads();
    // dW[o][i] = sum_s d[s][o] hin[s][i]; db[o] = sum_s d[s][o]
    for (int idx = threadIdx.x; idx < out * in; idx += blockDim.x) {
      const int o = idx / in, i = idx - o * in;
      float a = 0.f;
#pragma unroll 8
      for (int s = 0; s < SB; ++s) a += d[s][o] * hin[s][i];
      g[net.woff[l] + idx] = a;
    }
    for (int o = threadIdx.x; o < out; o += blockDim.x) {
      float a = 0.f;
      for (int s = 0; s < SB; ++s) a += d[s][o];
      g[net.boff[l] + o] = a;
    }
    if (l > 0) {
      const float* W = P + net.woff[l];
      for (int idx = threadIdx.x; idx < SB * in; idx += blockDim.x) {
        const int s = idx / in, i = idx - s * in;
        float a = 0.f;
        for (int o = 0; o < out; ++o) a += W[(long long)o * in + i] * d[s][o];
        const float z = s < ns ? zs[zoff[l - 1] + (long long)(s0 + s) * in + i] : 0.f;
        dn[s][i] = a * gelu_d(z);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < SB * in; idx += blockDim.x) {
        const int s = idx / in, i = idx - s * in;
        d[s][i] = dn[s][i];
      }
    }
    __syncthreads();
  }
}

// gradient = sum over CTAs of the partials (fixed order); loss likewise
__global__ void k_reduce(const float* __restrict__ gpart, int nblk, long long nparam, float* __restrict__ grad,
                         const float* __restrict__ lpart, float* __restrict__ loss, float lscale) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < nparam) {
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += gpart[(long long)b * nparam + p];
    grad[p] = a;
  }
  if (p == 0) {
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += lpart[b];
    *loss = a * lscale;
  }
}

// Adam (Kingma and Ba): bias-corrected first and second moments
__global__ void k_adam(long long n, float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct lbm_mlp {
  Net net{};
  long long nparam = 0;
  int max_batch = 0;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  float *P = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *gpart = nullptr, *lpart = nullptr;
  float *x = nullptr, *t = nullptr, *y = nullptr, *zs = nullptr, *hs = nullptr, *loss = nullptr;
  size_t act_floats = 0;
  int ndata = 0;
  int adam_t = 0;
  std::vector<std::pair<void*, size_t>> blocks;
};

static void* malloc_cb(size_t b, void*) {
  void* p = nullptr;
  return cudaMalloc(&p, b) == cudaSuccess ? p : nullptr;
}
static void free_cb(void* p, size_t, void*) { cudaFree(p); }

static float* mget(lbm_mlp* m, size_t floats) {
  const size_t b = floats * 4 + 256;
  void* p = m->alloc.alloc(b, m->alloc.ctx);
  if (p) m->blocks.push_back({p, b});
  return static_cast<float*>(p);
}

extern "C" void lbm_mlp_destroy(lbm_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (auto& b : m->blocks) m->alloc.free(b.first, b.second, m->alloc.ctx);
  delete m;
}

extern "C" int lbm_mlp_create(const int* sizes, int nlayers, int max_batch, void* stream, const lbm_allocator* alloc,
                              lbm_mlp** out) {
  if (!out || !sizes || nlayers < 1 || nlayers > MAXL || max_batch < 1) return LBM_EINVAL;
  *out = nullptr;
  for (int l = 0; l <= nlayers; ++l)
    if (sizes[l] < 1 || sizes[l] > MAXW) return LBM_EINVAL;
  lbm_mlp* m = new (std::nothrow) lbm_mlp();
  if (!m) return LBM_ENOMEM;
  m->stream = static_cast<cudaStream_t>(stream);
  if (alloc && alloc->alloc && alloc->free) m->alloc = *alloc;
  else { m->alloc.alloc = malloc_cb; m->alloc.free = free_cb; m->alloc.ctx = nullptr; }
  m->net.nl = nlayers;
  long long off = 0;
  size_t act = 0;
  for (int l = 0; l <= nlayers; ++l) m->net.sizes[l] = sizes[l];
  for (int l = 0; l < nlayers; ++l) {
    m->net.woff[l] = off;
    off += (long long)sizes[l + 1] * sizes[l];
    m->net.boff[l] = off;
    off += sizes[l + 1];
    act += size_t(sizes[l + 1]);
  }
  m->nparam = off;
  m->max_batch = max_batch;
  m->act_floats = act * size_t(max_batch);
  const int nblk = (max_batch + SB - 1) / SB;
  m->P = mget(m, off);
  m->m = mget(m, off);
  m->v = mget(m, off);
  m->grad = mget(m, off);
  m->gpart = mget(m, size_t(off) * nblk);
  m->lpart = mget(m, size_t(nblk));
  m->x = mget(m, size_t(max_batch) * sizes[0]);
  m->t = mget(m, size_t(max_batch) * sizes[nlayers]);
  m->y = mget(m, size_t(max_batch) * sizes[nlayers]);
  m->zs = mget(m, m->act_floats);
  m->hs = mget(m, m->act_floats);
  m->loss = mget(m, 1);
  if (!m->P || !m->m || !m->v || !m->grad || !m->gpart || !m->lpart || !m->x || !m->t || !m->y || !m->zs || !m->hs ||
      !m->loss) {
    lbm_mlp_destroy(m);
    return LBM_ENOMEM;
  }
  cudaMemsetAsync(m->m, 0, size_t(off) * 4, m->stream);
  cudaMemsetAsync(m->v, 0, size_t(off) * 4, m->stream);
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) { lbm_mlp_destroy(m); return LBM_ECUDA; }
  *out = m;
  return LBM_OK;
}

extern "C" long long lbm_mlp_param_count(const lbm_mlp* m) { return m ? m->nparam : -1; }

extern "C" int lbm_mlp_set_params(lbm_mlp* m, const float* host) {
  if (!m || !host) return LBM_EINVAL;
  cudaError_t e = cudaMemcpyAsync(m->P, host, size_t(m->nparam) * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, size_t(m->nparam) * 4, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, size_t(m->nparam) * 4, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  m->adam_t = 0;
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_mlp_get_params(lbm_mlp* m, float* host) {
  if (!m || !host) return LBM_EINVAL;
  cudaError_t e = cudaMemcpyAsync(host, m->P, size_t(m->nparam) * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

static cudaError_t run_forward(lbm_mlp* m, const float* dx, int B, float* dy) {
  const int nblk = (B + SB - 1) / SB;
  k_mlp_forward<<<nblk, 128, 0, m->stream>>>(m->net, m->P, dx, B, dy, m->zs, m->hs);
  return cudaGetLastError();
}

static cudaError_t run_grad(lbm_mlp* m, const float* dx, const float* dt, int B) {
  cudaError_t e = run_forward(m, dx, B, m->y);
  if (e != cudaSuccess) return e;
  const int nblk = (B + SB - 1) / SB;
  k_mlp_backward<<<nblk, 256, 0, m->stream>>>(m->net, m->P, dx, dt, B, m->y, m->zs, m->hs, m->gpart, m->nparam,
                                              m->lpart);
  const int nout = m->net.sizes[m->net.nl];
  k_reduce<<<unsigned((m->nparam + 255) / 256), 256, 0, m->stream>>>(m->gpart, nblk, m->nparam, m->grad, m->lpart,
                                                                      m->loss, 1.f / (float(B) * float(nout)));
  return cudaGetLastError();
}

extern "C" int lbm_mlp_forward(lbm_mlp* m, const float* host_x, int batch, float* host_y) {
  if (!m || !host_x || !host_y || batch < 1 || batch > m->max_batch) return LBM_EINVAL;
  const int in = m->net.sizes[0], out = m->net.sizes[m->net.nl];
  cudaError_t e = cudaMemcpyAsync(m->x, host_x, size_t(batch) * in * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = run_forward(m, m->x, batch, m->y);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_y, m->y, size_t(batch) * out * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_mlp_loss_grad(lbm_mlp* m, const float* host_x, const float* host_t, int batch, float* host_loss,
                                 float* host_grad) {
  if (!m || !host_x || !host_t || batch < 1 || batch > m->max_batch) return LBM_EINVAL;
  const int in = m->net.sizes[0], out = m->net.sizes[m->net.nl];
  cudaError_t e = cudaMemcpyAsync(m->x, host_x, size_t(batch) * in * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->t, host_t, size_t(batch) * out * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = run_grad(m, m->x, m->t, batch);
  if (e == cudaSuccess && host_grad)
    e = cudaMemcpyAsync(host_grad, m->grad, size_t(m->nparam) * 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess && host_loss) e = cudaMemcpyAsync(host_loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_mlp_set_data(lbm_mlp* m, const float* host_x, const float* host_t, int n) {
  if (!m || !host_x || !host_t || n < 1 || n > m->max_batch) return LBM_EINVAL;
  const int in = m->net.sizes[0], out = m->net.sizes[m->net.nl];
  cudaError_t e = cudaMemcpyAsync(m->x, host_x, size_t(n) * in * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->t, host_t, size_t(n) * out * 4, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  m->ndata = n;
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

// iters full-batch Adam steps on the data set by lbm_mlp_set_data; the final
// loss (of the parameters before the last update) is returned in *host_loss
extern "C" int lbm_mlp_train(lbm_mlp* m, int iters, float lr, float* host_loss) {
  if (!m || iters < 0 || m->ndata < 1) return LBM_EINVAL;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < iters; ++it) {
    cudaError_t e = run_grad(m, m->x, m->t, m->ndata);
    if (e != cudaSuccess) return LBM_ECUDA;
    m->adam_t += 1;
    const float c1 = 1.f - std::pow(b1, float(m->adam_t)), c2 = 1.f - std::pow(b2, float(m->adam_t));
    k_adam<<<unsigned((m->nparam + 255) / 256), 256, 0, m->stream>>>(m->nparam, m->P, m->m, m->v, m->grad, lr, b1, b2,
                                                                      eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  if (host_loss) e = cudaMemcpyAsync(host_loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
