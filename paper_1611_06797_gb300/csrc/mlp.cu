// Pair-energy surrogate of the learned form: a 3-layer perceptron (n_in -> H -> H -> 1,
// tanh hidden units, H <= 64, FP32) trained on pair energies that the exact kernel
// produces, used to estimate the exchange energy of weak pairs that are then not
// contracted.  The paper has no counterpart; it belongs to the batching / screening forms
// of this library.  Training and inference are hand-written kernels: one thread per
// sample, weights in shared memory, per-block gradients as outer-product sums in shared
// memory, block partials summed in a fixed order, Adam updates on the device.  Training
// is deterministic: no atomics anywhere.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ltmp2.h"

namespace {

constexpr int kMaxIn = 16;
constexpr int kMaxH = 64;
constexpr int kThreads = 128;

struct Dims {
  int n_in, h;
  int w1, b1, w2, b2, w3, b3, total;  // offsets into the parameter vector
};

Dims make_dims(int n_in, int h) {
  Dims d;
  d.n_in = n_in;
  d.h = h;
  d.w1 = 0;
  d.b1 = d.w1 + h * n_in;
  d.w2 = d.b1 + h;
  d.b2 = d.w2 + h * h;
  d.w3 = d.b2 + h;
  d.b3 = d.w3 + h;
  d.total = d.b3 + 1;
  return d;
}

// forward pass of one sample; h1, h2 receive the hidden activations
__device__ float forward(const Dims &d, const float *__restrict__ w, const float *x, float *h1, float *h2) {
  for (int k = 0; k < d.h; ++k) {
    float a = w[d.b1 + k];
    for (int q = 0; q < d.n_in; ++q) a += w[d.w1 + k * d.n_in + q] * x[q];
    h1[k] = tanhf(a);
  }
  for (int k = 0; k < d.h; ++k) {
    float a = w[d.b2 + k];
    for (int q = 0; q < d.h; ++q) a += w[d.w2 + k * d.h + q] * h1[q];
    h2[k] = tanhf(a);
  }
  float o = w[d.b3];
  for (int k = 0; k < d.h; ++k) o += w[d.w3 + k] * h2[k];
  return o;
}

__global__ void k_mlp_predict(Dims d, const float *__restrict__ params, const float *__restrict__ X, int n,
                              const float *__restrict__ xmean, const float *__restrict__ xstd, float ymean,
                              float ystd, float *__restrict__ y) {
  extern __shared__ float w[];
  for (int k = threadIdx.x; k < d.total; k += blockDim.x) w[k] = params[k];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kMaxIn], h1[kMaxH], h2[kMaxH];
  for (int q = 0; q < d.n_in; ++q) x[q] = (X[(size_t)s * d.n_in + q] - xmean[q]) / xstd[q];
  y[s] = ymean + ystd * forward(d, w, x, h1, h2);
}

// Mean-squared-error gradient of the block's samples -> partial[block][total]; loss ->
// lpart[block].  Phase 1: one thread per sample runs forward and backward and leaves its
// activations and error signals in shared memory; phase 2: threads over parameters sum
// the block's outer products in a fixed order (no atomics).
__global__ void k_mlp_grad(Dims d, const float *__restrict__ params, const float *__restrict__ Xs,
                           const float *__restrict__ ys, int n, float *__restrict__ partial,
                           float *__restrict__ lpart) {
  extern __shared__ float sm[];
  const int B = blockDim.x, H = d.h;
  float *w = sm;                                  // [total]
  float *H1 = w + d.total;                        // [B][H] layer-1 activations
  float *D2 = H1 + (size_t)B * H;                 // [B][H] error at layer-2 pre-activations
  float *DZ = D2 + (size_t)B * H;                 // [B][H] error at layer-1 pre-activations
  float *O2 = DZ + (size_t)B * H;                 // [B][H] dout * h2
  float *XS = O2 + (size_t)B * H;                 // [B][n_in]
  float *DO = XS + (size_t)B * d.n_in;            // [B] dout
  for (int k = threadIdx.x; k < d.total; k += B) w[k] = params[k];
  __shared__ float lred[kThreads];
  __syncthreads();
  const int t = threadIdx.x, s = blockIdx.x * B + t;
  float loss = 0.f;
  {
    float x[kMaxIn], h1[kMaxH], h2[kMaxH];
    float dout = 0.f;
    if (s < n) {
      for (int q = 0; q < d.n_in; ++q) x[q] = Xs[(size_t)s * d.n_in + q];
      const float o = forward(d, w, x, h1, h2);
      const float r = o - ys[s];
      loss = r * r;
      dout = 2.f * r / (float)n;
    } else {
      for (int q = 0; q < d.n_in; ++q) x[q] = 0.f;
      for (int k = 0; k < H; ++k) { h1[k] = 0.f; h2[k] = 0.f; }
    }
    DO[t] = dout;
    for (int q = 0; q < d.n_in; ++q) XS[t * d.n_in + q] = x[q];
    for (int k = 0; k < H; ++k) {
      H1[t * H + k] = h1[k];
      O2[t * H + k] = dout * h2[k];
      D2[t * H + k] = dout * w[d.w3 + k] * (1.f - h2[k] * h2[k]);
    }
    for (int q = 0; q < H; ++q) {
      float a = 0.f;
      for (int k = 0; k < H; ++k) a += w[d.w2 + k * H + q] * D2[t * H + k];
      DZ[t * H + q] = a * (1.f - h1[q] * h1[q]);
    }
  }
  lred[t] = loss;
  __syncthreads();
  float *out = partial + (size_t)blockIdx.x * d.total;
  for (int k = t; k < d.total; k += B) {
    float g = 0.f;
    if (k >= d.w2 && k < d.b2) {            // W2[r][c]: sum_s D2[s][r] H1[s][c]
      const int r = (k - d.w2) / H, c = (k - d.w2) % H;
      for (int q = 0; q < B; ++q) g += D2[q * H + r] * H1[q * H + c];
    } else if (k >= d.w1 && k < d.b1) {     // W1[r][c]: sum_s DZ[s][r] X[s][c]
      const int r = (k - d.w1) / d.n_in, c = (k - d.w1) % d.n_in;
      for (int q = 0; q < B; ++q) g += DZ[q * H + r] * XS[q * d.n_in + c];
    } else if (k >= d.b1 && k < d.w2) {
      for (int q = 0; q < B; ++q) g += DZ[q * H + (k - d.b1)];
    } else if (k >= d.b2 && k < d.w3) {
      for (int q = 0; q < B; ++q) g += D2[q * H + (k - d.b2)];
    } else if (k >= d.w3 && k < d.b3) {
      for (int q = 0; q < B; ++q) g += O2[q * H + (k - d.w3)];
    } else {
      for (int q = 0; q < B; ++q) g += DO[q];
    }
    out[k] = g;
  }
  for (int wdt = B / 2; wdt > 0; wdt >>= 1) {
    if (t < wdt) lred[t] += lred[t + wdt];
    __syncthreads();
  }
  if (t == 0) lpart[blockIdx.x] = lred[0];
}

// sum the block partials in a fixed order and take one Adam step
__global__ void k_mlp_adam(Dims d, int nblocks, const float *__restrict__ partial, float *__restrict__ params,
                           float *__restrict__ m, float *__restrict__ v, float lr, float b1t, float b2t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.total) return;
  float gsum = 0.f;
  for (int b = 0; b < nblocks; ++b) gsum += partial[(size_t)b * d.total + k];
  const float beta1 = 0.9f, beta2 = 0.999f;
  m[k] = beta1 * m[k] + (1.f - beta1) * gsum;
  v[k] = beta2 * v[k] + (1.f - beta2) * gsum * gsum;
  const float mh = m[k] / (1.f - b1t), vh = v[k] / (1.f - b2t);
  params[k] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

unsigned long long splitmix(unsigned long long &s) {
  unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct ltmp2_mlp {
  Dims d;
  int device = 0;
  float *params = nullptr, *m = nullptr, *v = nullptr;
  std::vector<float> xmean, xstd;
  float ymean = 0.f, ystd = 1.f;
  float resid = 0.f;   // root-mean-square training residual, in the units of the targets
  int steps = 0;
  ~ltmp2_mlp() {
    cudaFree(params);
    cudaFree(m);
    cudaFree(v);
  }
};

extern "C" {

int ltmp2_mlp_create(int n_in, int width, unsigned long long seed, ltmp2_mlp **out) {
  if (!out || n_in < 1 || n_in > kMaxIn || width < 1 || width > kMaxH) return LTMP2_ERR_INVALID_ARG;
  *out = nullptr;
  ltmp2_mlp *net = new (std::nothrow) ltmp2_mlp();
  if (!net) return LTMP2_ERR_OOM;
  net->d = make_dims(n_in, width);
  cudaGetDevice(&net->device);
  const size_t bytes = sizeof(float) * net->d.total;
  if (cudaMalloc(&net->params, bytes) != cudaSuccess || cudaMalloc(&net->m, bytes) != cudaSuccess ||
      cudaMalloc(&net->v, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return LTMP2_ERR_OOM;
  }
  // Glorot-uniform weights from a seeded host generator, zero biases
  std::vector<float> h(net->d.total, 0.f);
  unsigned long long s = seed;
  auto uni = [&](float lim) { return lim * (2.f * (float)((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.f); };
  const Dims &d = net->d;
  for (int k = 0; k < d.h * d.n_in; ++k) h[d.w1 + k] = uni(std::sqrt(6.f / (d.n_in + d.h)));
  for (int k = 0; k < d.h * d.h; ++k) h[d.w2 + k] = uni(std::sqrt(6.f / (2.f * d.h)));
  for (int k = 0; k < d.h; ++k) h[d.w3 + k] = uni(std::sqrt(6.f / (d.h + 1.f)));
  if (cudaMemcpy(net->params, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->m, 0, bytes) != cudaSuccess || cudaMemset(net->v, 0, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return LTMP2_ERR_CUDA;
  }
  net->xmean.assign(n_in, 0.f);
  net->xstd.assign(n_in, 1.f);
  *out = net;
  return LTMP2_OK;
}

int ltmp2_mlp_train(ltmp2_mlp *net, const float *X, const float *y, int n, int epochs, float lr, float *final_loss) {
  if (!net || !X || !y || n < 1 || epochs < 1 || !(lr > 0.f)) return LTMP2_ERR_INVALID_ARG;
  const Dims &d = net->d;
  // standardise inputs and targets with the training set's moments
  for (int q = 0; q < d.n_in; ++q) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
      const double x = X[(size_t)i * d.n_in + q];
      if (!std::isfinite(x)) return LTMP2_ERR_INVALID_ARG;
      s += x;
      s2 += x * x;
    }
    const double mu = s / n, var = s2 / n - mu * mu;
    net->xmean[q] = (float)mu;
    net->xstd[q] = (float)(var > 1e-20 ? std::sqrt(var) : 1.0);
  }
  {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) {
      if (!std::isfinite(y[i])) return LTMP2_ERR_INVALID_ARG;
      s += y[i];
      s2 += (double)y[i] * y[i];
    }
    const double mu = s / n, var = s2 / n - mu * mu;
    net->ymean = (float)mu;
    net->ystd = (float)(var > 1e-30 ? std::sqrt(var) : 1.0);
  }
  std::vector<float> xs((size_t)n * d.n_in), ys(n);
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < d.n_in; ++q)
      xs[(size_t)i * d.n_in + q] = (X[(size_t)i * d.n_in + q] - net->xmean[q]) / net->xstd[q];
    ys[i] = (y[i] - net->ymean) / net->ystd;
  }
  const int nblocks = (n + kThreads - 1) / kThreads;
  float *dX = nullptr, *dy = nullptr, *part = nullptr, *lp = nullptr;
  auto cleanup = [&]() {
    cudaFree(dX);
    cudaFree(dy);
    cudaFree(part);
    cudaFree(lp);
  };
  if (cudaMalloc(&dX, sizeof(float) * xs.size()) != cudaSuccess || cudaMalloc(&dy, sizeof(float) * n) != cudaSuccess ||
      cudaMalloc(&part, sizeof(float) * (size_t)nblocks * d.total) != cudaSuccess ||
      cudaMalloc(&lp, sizeof(float) * nblocks) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return LTMP2_ERR_OOM;
  }
  cudaMemcpy(dX, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(dy, ys.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  const size_t smem = sizeof(float) * (d.total + (size_t)kThreads * (4 * d.h + d.n_in + 1));
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return LTMP2_ERR_CUDA;
  }
  double b1t = 1.0, b2t = 1.0;
  for (int ep = 0; ep < epochs; ++ep) {
    ++net->steps;
    b1t *= 0.9;
    b2t *= 0.999;
    k_mlp_grad<<<nblocks, kThreads, smem>>>(d, net->params, dX, dy, n, part, lp);
    k_mlp_adam<<<(d.total + 255) / 256, 256>>>(d, nblocks, part, net->params, net->m, net->v, lr, (float)b1t,
                                               (float)b2t);
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    std::vector<float> l(nblocks);
    cudaMemcpy(l.data(), lp, sizeof(float) * nblocks, cudaMemcpyDeviceToHost);
    double t = 0;
    for (float x : l) t += x;
    const double mse = t / n;  // mean squared error of the standardised targets
    if (final_loss) *final_loss = (float)mse;
    net->resid = (float)(std::sqrt(mse) * net->ystd);
  }
  cleanup();
  return e == cudaSuccess ? LTMP2_OK : LTMP2_ERR_CUDA;
}

int ltmp2_mlp_predict(const ltmp2_mlp *net, const float *X, int n, float *y) {
  if (!net || !X || !y || n < 1) return LTMP2_ERR_INVALID_ARG;
  const Dims &d = net->d;
  float *dX = nullptr, *dy = nullptr, *dm = nullptr, *ds = nullptr;
  int rc = LTMP2_OK;
  if (cudaMalloc(&dX, sizeof(float) * (size_t)n * d.n_in) != cudaSuccess ||
      cudaMalloc(&dy, sizeof(float) * n) != cudaSuccess || cudaMalloc(&dm, sizeof(float) * d.n_in) != cudaSuccess ||
      cudaMalloc(&ds, sizeof(float) * d.n_in) != cudaSuccess) {
    cudaGetLastError();
    rc = LTMP2_ERR_OOM;
  }
  if (!rc) {
    cudaMemcpy(dX, X, sizeof(float) * (size_t)n * d.n_in, cudaMemcpyHostToDevice);
    cudaMemcpy(dm, net->xmean.data(), sizeof(float) * d.n_in, cudaMemcpyHostToDevice);
    cudaMemcpy(ds, net->xstd.data(), sizeof(float) * d.n_in, cudaMemcpyHostToDevice);
    k_mlp_predict<<<(n + kThreads - 1) / kThreads, kThreads, sizeof(float) * d.total>>>(d, net->params, dX, n, dm, ds,
                                                                                       net->ymean, net->ystd, dy);
    if (cudaMemcpy(y, dy, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = LTMP2_ERR_CUDA;
  }
  cudaFree(dX);
  cudaFree(dy);
  cudaFree(dm);
  cudaFree(ds);
  return rc;
}

int ltmp2_mlp_residual(const ltmp2_mlp *net, float *sigma) {
  if (!net || !sigma) return LTMP2_ERR_INVALID_ARG;
  *sigma = net->resid;
  return LTMP2_OK;
}

void ltmp2_mlp_destroy(ltmp2_mlp *net) { delete net; }

}  // extern "C"
