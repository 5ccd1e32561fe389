// Learned sizing of the Krylov dimensions: a 16 -> 64 -> 64 -> 2 float MLP (ReLU) that
// reads 16 features of the first outer coefficients and predicts (log k*, log l*).
// Forward, backward and Adam are hand-written kernels; training runs on the GPU.
//
// Parameter vector (5378 floats): W1 [64][16], b1 [64], W2 [64][64], b2 [64],
// W3 [2][64], b3 [2] (row-major, out x in). Loss: mean over samples of the squared
// error summed over the two outputs.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ov_internal.h"

namespace ov {

constexpr int kIn = 16, kHid = 64, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid, kNParams = kOffB3 + kOut;
static_assert(kNParams == 5378, "parameter layout");
constexpr int kMlpThreads = 128;

// One thread per sample; parameters staged in shared memory. z1, z2 (pre-activations)
// are stored when not NULL (training).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float* __restrict__ theta, int n,
                                                             const float* __restrict__ X, float* z1, float* z2,
                                                             float* Y) {
  __shared__ float th[kNParams];
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[(size_t)s * kIn + i];
  float a1[kHid];
#pragma unroll 4
  for (int o = 0; o < kHid; ++o) {
    float acc = th[kOffB1 + o];
#pragma unroll
    for (int i = 0; i < kIn; ++i) acc = fmaf(th[kOffW1 + o * kIn + i], x[i], acc);
    if (z1) z1[(size_t)s * kHid + o] = acc;
    a1[o] = fmaxf(acc, 0.f);
  }
  float y0 = th[kOffB3], y1 = th[kOffB3 + 1];
  for (int o = 0; o < kHid; ++o) {
    float acc = th[kOffB2 + o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) acc = fmaf(th[kOffW2 + o * kHid + i], a1[i], acc);
    if (z2) z2[(size_t)s * kHid + o] = acc;
    const float a2 = fmaxf(acc, 0.f);
    y0 = fmaf(th[kOffW3 + o], a2, y0);
    y1 = fmaf(th[kOffW3 + kHid + o], a2, y1);
  }
  Y[(size_t)s * kOut + 0] = y0;
  Y[(size_t)s * kOut + 1] = y1;
}

// Per-sample back-propagation: d3 = 2 (y - t) / n, d2 = (W3^T d3) * [z2 > 0],
// d1 = (W2^T d2) * [z1 > 0]; also the squared error of the sample.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_delta(const float* __restrict__ theta, int n,
                                                           const float* __restrict__ z1, const float* __restrict__ z2,
                                                           const float* __restrict__ Yp, const float* __restrict__ Yt,
                                                           float* d1, float* d2, float* d3, float* sqerr) {
  __shared__ float th[kNParams];
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float e0 = Yp[(size_t)s * 2] - Yt[(size_t)s * 2], e1 = Yp[(size_t)s * 2 + 1] - Yt[(size_t)s * 2 + 1];
  sqerr[s] = e0 * e0 + e1 * e1;
  const float g0 = 2.f * e0 / n, g1 = 2.f * e1 / n;
  d3[(size_t)s * 2] = g0;
  d3[(size_t)s * 2 + 1] = g1;
  float dd2[kHid];
#pragma unroll 4
  for (int o = 0; o < kHid; ++o) {
    const float v = th[kOffW3 + o] * g0 + th[kOffW3 + kHid + o] * g1;
    dd2[o] = z2[(size_t)s * kHid + o] > 0.f ? v : 0.f;
    d2[(size_t)s * kHid + o] = dd2[o];
  }
  for (int i = 0; i < kHid; ++i) {
    float v = 0.f;
#pragma unroll
    for (int o = 0; o < kHid; ++o) v = fmaf(th[kOffW2 + o * kHid + i], dd2[o], v);
    d1[(size_t)s * kHid + i] = z1[(size_t)s * kHid + i] > 0.f ? v : 0.f;
  }
}

// One thread per parameter: gradient = sum over samples (fixed order) of
// delta(out) * activation(in).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_wgrad(int n, const float* __restrict__ X,
                                                           const float* __restrict__ z1, const float* __restrict__ z2,
                                                           const float* __restrict__ d1, const float* __restrict__ d2,
                                                           const float* __restrict__ d3, float* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNParams) return;
  float acc = 0.f;
  if (p < kOffB1) {
    const int o = (p - kOffW1) / kIn, i = (p - kOffW1) % kIn;
    for (int s = 0; s < n; ++s) acc = fmaf(d1[(size_t)s * kHid + o], X[(size_t)s * kIn + i], acc);
  } else if (p < kOffW2) {
    const int o = p - kOffB1;
    for (int s = 0; s < n; ++s) acc += d1[(size_t)s * kHid + o];
  } else if (p < kOffB2) {
    const int o = (p - kOffW2) / kHid, i = (p - kOffW2) % kHid;
    for (int s = 0; s < n; ++s) acc = fmaf(d2[(size_t)s * kHid + o], fmaxf(z1[(size_t)s * kHid + i], 0.f), acc);
  } else if (p < kOffW3) {
    const int o = p - kOffB2;
    for (int s = 0; s < n; ++s) acc += d2[(size_t)s * kHid + o];
  } else if (p < kOffB3) {
    const int o = (p - kOffW3) / kHid, i = (p - kOffW3) % kHid;
    for (int s = 0; s < n; ++s) acc = fmaf(d3[(size_t)s * kOut + o], fmaxf(z2[(size_t)s * kHid + i], 0.f), acc);
  } else {
    const int o = p - kOffB3;
    for (int s = 0; s < n; ++s) acc += d3[(size_t)s * kOut + o];
  }
  grad[p] = acc;
}

// Adam (Kingma & Ba 2015) with bias correction; t >= 1 is the step number.
__global__ void k_mlp_adam(float* theta, const float* __restrict__ grad, float* m, float* v, int t, float lr,
                           float b1, float b2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNParams) return;
  const float g = grad[p];
  const float mn = b1 * m[p] + (1.f - b1) * g;
  const float vn = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mn;
  v[p] = vn;
  const float mh = mn / (1.f - powf(b1, (float)t));
  const float vh = vn / (1.f - powf(b2, (float)t));
  theta[p] -= lr * mh / (sqrtf(vh) + eps);
}

// fixed-order sum of n values (one block)
__global__ void k_sum(const float* __restrict__ x, int n, float* out) {
  __shared__ double red[kMlpThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) s += red[i];
    *out = (float)(s / n);
  }
}

struct MlpBufs {
  float *theta = nullptr, *X = nullptr, *Y = nullptr, *Yp = nullptr, *z1 = nullptr, *z2 = nullptr, *d1 = nullptr,
        *d2 = nullptr, *d3 = nullptr, *sq = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  void free_all() {
    float* all[] = {theta, X, Y, Yp, z1, z2, d1, d2, d3, sq, grad, m, v, loss};
    for (float* p : all)
      if (p) cudaFree(p);
  }
  bool alloc(int n) {
    auto A = [](float** p, size_t k) { return cudaMalloc(p, sizeof(float) * std::max<size_t>(k, 1)) == cudaSuccess; };
    return A(&theta, kNParams) && A(&X, (size_t)n * kIn) && A(&Y, (size_t)n * kOut) && A(&Yp, (size_t)n * kOut) &&
           A(&z1, (size_t)n * kHid) && A(&z2, (size_t)n * kHid) && A(&d1, (size_t)n * kHid) &&
           A(&d2, (size_t)n * kHid) && A(&d3, (size_t)n * kOut) && A(&sq, n) && A(&grad, kNParams) &&
           A(&m, kNParams) && A(&v, kNParams) && A(&loss, 1);
  }
};

static cudaError_t loss_grad_dev(MlpBufs& b, int n, const float* X, const float* Y, cudaStream_t st) {
  const int nb = (n + kMlpThreads - 1) / kMlpThreads;
  k_mlp_forward<<<nb, kMlpThreads, 0, st>>>(b.theta, n, X, b.z1, b.z2, b.Yp);
  k_mlp_delta<<<nb, kMlpThreads, 0, st>>>(b.theta, n, b.z1, b.z2, b.Yp, Y, b.d1, b.d2, b.d3, b.sq);
  k_mlp_wgrad<<<(kNParams + kMlpThreads - 1) / kMlpThreads, kMlpThreads, 0, st>>>(n, X, b.z1, b.z2, b.d1, b.d2,
                                                                                  b.d3, b.grad);
  k_sum<<<1, kMlpThreads, 0, st>>>(b.sq, n, b.loss);
  return cudaGetLastError();
}

cudaError_t mlp_predict_device(const float* theta_dev, int n, const float* X_dev, float* Y_dev, cudaStream_t st) {
  const int nb = (n + kMlpThreads - 1) / kMlpThreads;
  k_mlp_forward<<<nb, kMlpThreads, 0, st>>>(theta_dev, n, X_dev, nullptr, nullptr, Y_dev);
  return cudaGetLastError();
}

int mlp_num_params() { return kNParams; }

}  // namespace ov

using namespace ov;

extern "C" int ov_mlp_forward(const float* theta, int n, const float* X, float* Y) {
  if (!theta || !X || !Y || n < 1) return OV_ERR_ARG;
  MlpBufs b;
  if (!b.alloc(n)) {
    b.free_all();
    return OV_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpy(b.theta, theta, sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_predict_device(b.theta, n, b.X, b.Yp, 0);
  if (e == cudaSuccess) e = cudaMemcpy(Y, b.Yp, sizeof(float) * n * kOut, cudaMemcpyDeviceToHost);
  b.free_all();
  return e == cudaSuccess ? OV_OK : OV_ERR_CUDA;
}

extern "C" int ov_mlp_loss_grad(const float* theta, int n, const float* X, const float* Y, float* loss, float* grad) {
  if (!theta || !X || !Y || n < 1) return OV_ERR_ARG;
  MlpBufs b;
  if (!b.alloc(n)) {
    b.free_all();
    return OV_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpy(b.theta, theta, sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.Y, Y, sizeof(float) * n * kOut, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = loss_grad_dev(b, n, b.X, b.Y, 0);
  if (e == cudaSuccess && grad) e = cudaMemcpy(grad, b.grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss) e = cudaMemcpy(loss, b.loss, sizeof(float), cudaMemcpyDeviceToHost);
  b.free_all();
  return e == cudaSuccess ? OV_OK : OV_ERR_CUDA;
}

extern "C" int ov_mlp_train(float* theta, int n, const float* X, const float* Y, int epochs, int batch, float lr,
                            unsigned seed, float* loss_history, int n_val, const float* Xv, const float* Yv,
                            float* val_history) {
  if (!theta || !X || !Y || n < 1 || epochs < 1 || !(lr > 0.f)) return OV_ERR_ARG;
  if (n_val < 0 || (n_val > 0 && (!Xv || !Yv))) return OV_ERR_ARG;
  if (batch <= 0 || batch > n) batch = n;
  MlpBufs b, bv;
  float* best = nullptr;
  auto cleanup = [&]() {
    b.free_all();
    bv.free_all();
    if (best) cudaFree(best);
  };
  if (!b.alloc(n) || (n_val > 0 && !bv.alloc(n_val)) || cudaMalloc(&best, sizeof(float) * kNParams) != cudaSuccess) {
    cleanup();
    return OV_ERR_NOMEM;
  }
  cudaError_t e = cudaMemcpy(b.theta, theta, sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(best, theta, sizeof(float) * kNParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.m, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess) e = cudaMemset(b.v, 0, sizeof(float) * kNParams);
  if (e == cudaSuccess && n_val > 0) {
    e = cudaMemcpy(bv.X, Xv, sizeof(float) * n_val * kIn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bv.Y, Yv, sizeof(float) * n_val * kOut, cudaMemcpyHostToDevice);
  }
  std::vector<int> perm(n);
  std::vector<float> Xs((size_t)n * kIn), Ys((size_t)n * kOut);
  for (int i = 0; i < n; ++i) perm[i] = i;
  unsigned state = seed ? seed : 0x9e3779b9u;
  auto rnd = [&]() {  // xorshift32
    state ^= state << 13;
    state ^= state >> 17;
    state ^= state << 5;
    return state;
  };
  float best_val = INFINITY;
  int t = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    if (batch < n) {  // a new deterministic shuffle per epoch
      for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[rnd() % (unsigned)(i + 1)]);
    }
    if (batch < n || ep == 0) {
      for (int i = 0; i < n; ++i) {
        memcpy(&Xs[(size_t)i * kIn], X + (size_t)perm[i] * kIn, sizeof(float) * kIn);
        memcpy(&Ys[(size_t)i * kOut], Y + (size_t)perm[i] * kOut, sizeof(float) * kOut);
      }
      e = cudaMemcpy(b.X, Xs.data(), sizeof(float) * n * kIn, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(b.Y, Ys.data(), sizeof(float) * n * kOut, cudaMemcpyHostToDevice);
    }
    for (int s0 = 0; s0 < n && e == cudaSuccess; s0 += batch) {
      const int nb = std::min(batch, n - s0);
      e = loss_grad_dev(b, nb, b.X + (size_t)s0 * kIn, b.Y + (size_t)s0 * kOut, 0);
      if (e != cudaSuccess) break;
      ++t;
      k_mlp_adam<<<(kNParams + 127) / 128, 128>>>(b.theta, b.grad, b.m, b.v, t, lr, 0.9f, 0.999f, 1e-8f);
      e = cudaGetLastError();
    }
    if (loss_history && e == cudaSuccess) {
      // full-data loss after the epoch
      e = loss_grad_dev(b, n, b.X, b.Y, 0);
      if (e == cudaSuccess) e = cudaMemcpy(&loss_history[ep], b.loss, sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (n_val > 0 && e == cudaSuccess) {
      // validation loss with the current parameters; keep the best parameters
      e = cudaMemcpy(bv.theta, b.theta, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice);
      if (e == cudaSuccess) e = loss_grad_dev(bv, n_val, bv.X, bv.Y, 0);
      float lv = INFINITY;
      if (e == cudaSuccess) e = cudaMemcpy(&lv, bv.loss, sizeof(float), cudaMemcpyDeviceToHost);
      if (val_history) val_history[ep] = lv;
      if (e == cudaSuccess && lv < best_val) {
        best_val = lv;
        e = cudaMemcpy(best, b.theta, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice);
      }
    }
  }
  const float* src = n_val > 0 ? best : b.theta;
  if (e == cudaSuccess) e = cudaMemcpy(theta, src, sizeof(float) * kNParams, cudaMemcpyDeviceToHost);
  cleanup();
  return e == cudaSuccess ? OV_OK : OV_ERR_CUDA;
}
