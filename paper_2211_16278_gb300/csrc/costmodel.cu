// Learned cost model of the tile autotuner: a two-hidden-layer tanh MLP that maps the
// features of a (workload shape, tile candidate) pair to the predicted log launch time.
// It ranks the autotuner's candidates so only the most promising ones are timed. It never
// touches block values. Training runs on the GPU with this file's kernels: full-batch
// forward, backward and Adam in one CTA, with every reduction in a fixed order so that a
// training run is bitwise reproducible.
//
// Parameters (FP32), in this order: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
// Loss: mean squared error, L = (1/n) sum_s (f(x_s) - y_s)^2.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/bblock.h"

struct bblock_costmodel {
  int F = 0, H = 0, n_params = 0, device = 0;
  long long adam_t = 0;
  float* d_p = nullptr;     // parameters
  float* d_m = nullptr;     // Adam first moment
  float* d_v = nullptr;     // Adam second moment
};

namespace {

constexpr int kMaxF = 16, kMaxH = 64, kMaxSamples = 1 << 16, kThreads = 256;

int n_params_of(int F, int H) { return H * F + H + H * H + H + H + 1; }

struct Layout {
  int w1, b1, w2, b2, w3, b3;
};
__host__ __device__ inline Layout layout(int F, int H) {
  Layout l;
  l.w1 = 0;
  l.b1 = l.w1 + H * F;
  l.w2 = l.b1 + H;
  l.b2 = l.w2 + H * H;
  l.w3 = l.b2 + H;
  l.b3 = l.w3 + H;
  return l;
}

// Forward of one sample; a1, a2 receive the hidden activations.
__device__ float forward_one(const float* __restrict__ p, const float* __restrict__ x, int F,
                             int H, float* a1, float* a2) {
  const Layout L = layout(F, H);
  for (int i = 0; i < H; ++i) {
    float z = p[L.b1 + i];
    for (int f = 0; f < F; ++f) z = fmaf(p[L.w1 + i * F + f], x[f], z);
    a1[i] = tanhf(z);
  }
  float y = p[L.b3];
  for (int j = 0; j < H; ++j) {
    float z = p[L.b2 + j];
    for (int i = 0; i < H; ++i) z = fmaf(p[L.w2 + j * H + i], a1[i], z);
    a2[j] = tanhf(z);
    y = fmaf(p[L.w3 + j], a2[j], y);
  }
  return y;
}

__global__ void k_mlp_predict(const float* __restrict__ p, const float* __restrict__ X, int n,
                              int F, int H, float* __restrict__ y) {
  float a1[kMaxH], a2[kMaxH];
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    y[s] = forward_one(p, X + (size_t)s * F, F, H, a1, a2);
}

// `epochs` full-batch steps of forward, backward and (if update) Adam, in one CTA.
// Scratch: A1, A2, D1, D2 [n][H]; g [n]. Writes the last step's gradient and loss.
__global__ void __launch_bounds__(kThreads) k_mlp_train(
    float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
    const float* __restrict__ X, const float* __restrict__ yt, int n, int F, int H, int epochs,
    int update, float lr, long long t0, float* __restrict__ A1, float* __restrict__ A2,
    float* __restrict__ D1, float* __restrict__ D2, float* __restrict__ g,
    float* __restrict__ grad_out, float* __restrict__ loss_out) {
  __shared__ double part[kThreads];
  const int tid = threadIdx.x;
  const Layout L = layout(F, H);
  const int P = L.b3 + 1;
  const float b1c = 0.9f, b2c = 0.999f, eps = 1e-8f;
  for (int e = 0; e < epochs; ++e) {
    // forward, residual gradient dL/dy_s = 2 (f(x_s) - y_s) / n
    double lpart = 0.0;
    for (int s = tid; s < n; s += kThreads) {
      const float y = forward_one(p, X + (size_t)s * F, F, H, A1 + (size_t)s * H, A2 + (size_t)s * H);
      const float r = y - yt[s];
      g[s] = 2.f * r / (float)n;
      lpart += (double)r * r;
    }
    part[tid] = lpart;
    __syncthreads();
    // back through the hidden layers, per sample
    for (int s = tid; s < n; s += kThreads) {
      const float* a1 = A1 + (size_t)s * H;
      const float* a2 = A2 + (size_t)s * H;
      float* d2 = D2 + (size_t)s * H;
      float* d1 = D1 + (size_t)s * H;
      for (int j = 0; j < H; ++j) d2[j] = g[s] * p[L.w3 + j] * (1.f - a2[j] * a2[j]);
      for (int i = 0; i < H; ++i) {
        float acc = 0.f;
        for (int j = 0; j < H; ++j) acc = fmaf(d2[j], p[L.w2 + j * H + i], acc);
        d1[i] = acc * (1.f - a1[i] * a1[i]);
      }
    }
    __syncthreads();
    // parameter gradients: sums over samples in index order
    for (int q = tid; q < P; q += kThreads) {
      float gr = 0.f;
      if (q < L.b1) {
        const int i = q / F, f = q - i * F;
        for (int s = 0; s < n; ++s) gr = fmaf(D1[(size_t)s * H + i], X[(size_t)s * F + f], gr);
      } else if (q < L.w2) {
        const int i = q - L.b1;
        for (int s = 0; s < n; ++s) gr += D1[(size_t)s * H + i];
      } else if (q < L.b2) {
        const int j = (q - L.w2) / H, i = (q - L.w2) - j * H;
        for (int s = 0; s < n; ++s) gr = fmaf(D2[(size_t)s * H + j], A1[(size_t)s * H + i], gr);
      } else if (q < L.w3) {
        const int j = q - L.b2;
        for (int s = 0; s < n; ++s) gr += D2[(size_t)s * H + j];
      } else if (q < L.b3) {
        const int j = q - L.w3;
        for (int s = 0; s < n; ++s) gr = fmaf(g[s], A2[(size_t)s * H + j], gr);
      } else {
        for (int s = 0; s < n; ++s) gr += g[s];
      }
      if (e == epochs - 1) grad_out[q] = gr;
      if (update) {
        const long long t = t0 + e + 1;
        m[q] = b1c * m[q] + (1.f - b1c) * gr;
        v[q] = b2c * v[q] + (1.f - b2c) * gr * gr;
        const float mh = m[q] / (1.f - powf(b1c, (float)t));
        const float vh = v[q] / (1.f - powf(b2c, (float)t));
        p[q] -= lr * mh / (sqrtf(vh) + eps);
      }
    }
    if (tid == 0 && e == epochs - 1) {
      double l = 0.0;
      for (int k = 0; k < kThreads; ++k) l += part[k];
      *loss_out = (float)(l / n);
    }
    __syncthreads();
  }
}

// splitmix64: deterministic initial weights (Glorot-uniform ranges)
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Scratch {
  float *X = nullptr, *y = nullptr, *A1 = nullptr, *A2 = nullptr, *D1 = nullptr, *D2 = nullptr,
        *g = nullptr, *grad = nullptr, *loss = nullptr;
  bool ok = false;
  Scratch(int n, int F, int H, int P) {
    ok = cudaMalloc(&X, sizeof(float) * (size_t)n * F) == cudaSuccess &&
         cudaMalloc(&y, sizeof(float) * (size_t)n) == cudaSuccess &&
         cudaMalloc(&A1, sizeof(float) * (size_t)n * H) == cudaSuccess &&
         cudaMalloc(&A2, sizeof(float) * (size_t)n * H) == cudaSuccess &&
         cudaMalloc(&D1, sizeof(float) * (size_t)n * H) == cudaSuccess &&
         cudaMalloc(&D2, sizeof(float) * (size_t)n * H) == cudaSuccess &&
         cudaMalloc(&g, sizeof(float) * (size_t)n) == cudaSuccess &&
         cudaMalloc(&grad, sizeof(float) * (size_t)P) == cudaSuccess &&
         cudaMalloc(&loss, sizeof(float)) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~Scratch() {
    cudaFree(X); cudaFree(y); cudaFree(A1); cudaFree(A2); cudaFree(D1); cudaFree(D2);
    cudaFree(g); cudaFree(grad); cudaFree(loss);
  }
};

int run_train(bblock_costmodel* cm, const float* X, const float* y, int n, int epochs, int update,
              float lr, float* loss, float* grad) {
  if (!cm || !X || !y || n < 1 || n > kMaxSamples || epochs < 1) return BBLOCK_ERR_INVALID_ARG;
  if (cudaSetDevice(cm->device) != cudaSuccess) { cudaGetLastError(); return BBLOCK_ERR_CUDA; }
  Scratch sc(n, cm->F, cm->H, cm->n_params);
  if (!sc.ok) return BBLOCK_ERR_OOM;
  if (cudaMemcpy(sc.X, X, sizeof(float) * (size_t)n * cm->F, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(sc.y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  k_mlp_train<<<1, kThreads>>>(cm->d_p, cm->d_m, cm->d_v, sc.X, sc.y, n, cm->F, cm->H, epochs,
                               update, lr, cm->adam_t, sc.A1, sc.A2, sc.D1, sc.D2, sc.g, sc.grad,
                               sc.loss);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  if (update) cm->adam_t += epochs;
  if ((loss && cudaMemcpy(loss, sc.loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (grad && cudaMemcpy(grad, sc.grad, sizeof(float) * cm->n_params, cudaMemcpyDeviceToHost) !=
                   cudaSuccess)) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  return BBLOCK_OK;
}

}  // namespace

extern "C" {

int bblock_costmodel_create(bblock_costmodel** out, int n_features, int hidden, uint64_t seed,
                            int device) {
  if (!out) return BBLOCK_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_features < 1 || n_features > kMaxF || hidden < 1 || hidden > kMaxH) return BBLOCK_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return BBLOCK_ERR_CUDA; }
  bblock_costmodel* cm = new bblock_costmodel();
  cm->F = n_features;
  cm->H = hidden;
  cm->device = device;
  cm->n_params = n_params_of(n_features, hidden);
  const size_t bytes = sizeof(float) * cm->n_params;
  if (cudaMalloc(&cm->d_p, bytes) != cudaSuccess || cudaMalloc(&cm->d_m, bytes) != cudaSuccess ||
      cudaMalloc(&cm->d_v, bytes) != cudaSuccess) {
    cudaGetLastError();
    bblock_costmodel_destroy(cm);
    return BBLOCK_ERR_OOM;
  }
  std::vector<float> p(cm->n_params, 0.f);
  const Layout L = layout(cm->F, cm->H);
  uint64_t st = seed;
  auto uni = [&](float r) { return (float)((splitmix(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * r; };
  const float r1 = sqrtf(6.f / (cm->F + cm->H)), r2 = sqrtf(6.f / (2 * cm->H)), r3 = sqrtf(6.f / (cm->H + 1));
  for (int q = L.w1; q < L.b1; ++q) p[q] = uni(r1);
  for (int q = L.w2; q < L.b2; ++q) p[q] = uni(r2);
  for (int q = L.w3; q < L.b3; ++q) p[q] = uni(r3);
  if (cudaMemcpy(cm->d_p, p.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(cm->d_m, 0, bytes) != cudaSuccess || cudaMemset(cm->d_v, 0, bytes) != cudaSuccess) {
    cudaGetLastError();
    bblock_costmodel_destroy(cm);
    return BBLOCK_ERR_CUDA;
  }
  *out = cm;
  return BBLOCK_OK;
}

void bblock_costmodel_destroy(bblock_costmodel* cm) {
  if (!cm) return;
  cudaSetDevice(cm->device);
  cudaFree(cm->d_p);
  cudaFree(cm->d_m);
  cudaFree(cm->d_v);
  cudaGetLastError();
  delete cm;
}

int bblock_costmodel_num_params(const bblock_costmodel* cm) { return cm ? cm->n_params : 0; }

int bblock_costmodel_get_params(bblock_costmodel* cm, float* out, int n) {
  if (!cm || !out || n != cm->n_params) return BBLOCK_ERR_INVALID_ARG;
  if (cudaSetDevice(cm->device) != cudaSuccess ||
      cudaMemcpy(out, cm->d_p, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  return BBLOCK_OK;
}

int bblock_costmodel_set_params(bblock_costmodel* cm, const float* in, int n) {
  if (!cm || !in || n != cm->n_params) return BBLOCK_ERR_INVALID_ARG;
  const size_t bytes = sizeof(float) * n;
  if (cudaSetDevice(cm->device) != cudaSuccess ||
      cudaMemcpy(cm->d_p, in, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(cm->d_m, 0, bytes) != cudaSuccess || cudaMemset(cm->d_v, 0, bytes) != cudaSuccess) {
    cudaGetLastError();
    return BBLOCK_ERR_CUDA;
  }
  cm->adam_t = 0;
  return BBLOCK_OK;
}

int bblock_costmodel_gradient(bblock_costmodel* cm, const float* X, const float* y, int n,
                              float* loss, float* grad) {
  return run_train(cm, X, y, n, 1, 0, 0.f, loss, grad);
}

int bblock_costmodel_train(bblock_costmodel* cm, const float* X, const float* y, int n, int epochs,
                           float lr, float* final_loss) {
  if (!(lr > 0.f)) return BBLOCK_ERR_INVALID_ARG;
  return run_train(cm, X, y, n, epochs, 1, lr, final_loss, nullptr);
}

int bblock_costmodel_predict(bblock_costmodel* cm, const float* X, int n, float* y) {
  if (!cm || !X || !y || n < 1 || n > kMaxSamples) return BBLOCK_ERR_INVALID_ARG;
  if (cudaSetDevice(cm->device) != cudaSuccess) { cudaGetLastError(); return BBLOCK_ERR_CUDA; }
  float *dX = nullptr, *dy = nullptr;
  if (cudaMalloc(&dX, sizeof(float) * (size_t)n * cm->F) != cudaSuccess ||
      cudaMalloc(&dy, sizeof(float) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dX);
    return BBLOCK_ERR_OOM;
  }
  int rc = BBLOCK_OK;
  if (cudaMemcpy(dX, X, sizeof(float) * (size_t)n * cm->F, cudaMemcpyHostToDevice) != cudaSuccess) rc = BBLOCK_ERR_CUDA;
  if (rc == BBLOCK_OK) {
    k_mlp_predict<<<(n + kThreads - 1) / kThreads, kThreads>>>(cm->d_p, dX, n, cm->F, cm->H, dy);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(y, dy, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = BBLOCK_ERR_CUDA;
  }
  cudaGetLastError();
  cudaFree(dX);
  cudaFree(dy);
  return rc;
}

}  // extern "C"
