// mlp.cu -- the learned screen's network: a 4 -> 64 -> 64 -> 1 multilayer perceptron
// (tanh hidden layers, FP32) that predicts log10 of a term's norm from
//   (level n, |l|_2, log10 t_m, log10 ||s_b||_F).
// Hand-written kernels: parameter initialisation, batched forward, full-batch
// gradient of the mean squared error (deterministic two-pass reduction) and Adam.
//
// Parameter layout (MRA_MLP_PARAMS floats): W1[64][4], b1[64], W2[64][64], b2[64],
// W3[64], b3, then the fixed input/output standardisation x_mean[4], x_std[4],
// y_mean, y_std (not trained).  Network output o is the standardised target:
//   z = (x - x_mean) / x_std,  h1 = tanh(W1 z + b1),  h2 = tanh(W2 h1 + b2),
//   o = W3 . h2 + b3,          prediction = o * y_std + y_mean.
#include <math.h>

#include "mlp.cuh"

namespace mra {

namespace {

// counter-based uniform in [0,1): splitmix64 of (seed, index)
__device__ __forceinline__ double u01(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void mlp_init_kernel(float *p, uint64_t seed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NP) return;
  // uniform(-a, a) with a = sqrt(6 / (fan_in + fan_out)) for weights, zero biases
  double a = 0.0;
  if (i < MLP_B1) a = sqrt(6.0 / (MLP_IN + MLP_H));
  else if (i >= MLP_W2 && i < MLP_B2) a = sqrt(6.0 / (MLP_H + MLP_H));
  else if (i >= MLP_W3 && i < MLP_B3) a = sqrt(6.0 / (MLP_H + 1));
  p[i] = (float)((2.0 * u01(seed, (uint64_t)i) - 1.0) * a);
}

// per-feature and target mean/std over n rows (one block, deterministic)
__global__ void mlp_norm_kernel(float *p, const float *x, const float *y, int64_t n) {
  __shared__ double red[5][2][256];
  double s[5] = {0, 0, 0, 0, 0}, q[5] = {0, 0, 0, 0, 0};
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    for (int f = 0; f < 4; ++f) {
      double v = x[r * 4 + f];
      s[f] += v;
      q[f] += v * v;
    }
    double v = y[r];
    s[4] += v;
    q[4] += v * v;
  }
  for (int f = 0; f < 5; ++f) {
    red[f][0][threadIdx.x] = s[f];
    red[f][1][threadIdx.x] = q[f];
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int f = 0; f < 5; ++f) {
        red[f][0][threadIdx.x] += red[f][0][threadIdx.x + o];
        red[f][1][threadIdx.x] += red[f][1][threadIdx.x + o];
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int f = 0; f < 5; ++f) {
      double m = n > 0 ? red[f][0][0] / n : 0.0;
      double var = n > 0 ? red[f][1][0] / n - m * m : 1.0;
      double sd = var > 1e-12 ? sqrt(var) : 1.0;
      if (f < 4) {
        p[MLP_XMEAN + f] = (float)m;
        p[MLP_XSTD + f] = (float)sd;
      } else {
        p[MLP_YMEAN] = (float)m;
        p[MLP_YSTD] = (float)sd;
      }
    }
  }
}

__global__ void mlp_forward_kernel(const float *__restrict__ p, const float *__restrict__ x, int64_t n,
                                   float *__restrict__ y) {
  __shared__ __align__(16) float sp[MLP_NALL];
  for (int i = threadIdx.x; i < MLP_NALL; i += blockDim.x) sp[i] = p[i];
  __syncthreads();
#pragma unroll 1
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    float in[4] = {x[r * 4], x[r * 4 + 1], x[r * 4 + 2], x[r * 4 + 3]};
    y[r] = mlp_predict(sp, in);
  }
}

// Gradient of L = (1/n) sum_r (o_r - (y_r - y_mean)/y_std)^2.  Each block handles a
// contiguous chunk of rows, keeps the chunk's activations in shared memory and writes
// its partial gradient; grad_reduce_kernel then sums the partials in block order.
constexpr int GB_ROWS = 16;  // rows per block-chunk (activations stay in 48 KB of shared memory)
__global__ void __launch_bounds__(256) mlp_grad_partial_kernel(const float *__restrict__ p,
                                                               const float *__restrict__ x,
                                                               const float *__restrict__ y, int64_t n,
                                                               int64_t chunk, float *__restrict__ part,
                                                               double *__restrict__ loss_part) {
  __shared__ float sp[MLP_NALL];
  __shared__ float z[GB_ROWS][4], h1[GB_ROWS][MLP_H], h2[GB_ROWS][MLP_H], d2[GB_ROWS][MLP_H],
      d1[GB_ROWS][MLP_H], dout[GB_ROWS];
  __shared__ double lred[256];
  for (int i = threadIdx.x; i < MLP_NALL; i += blockDim.x) sp[i] = p[i];
  float g[(MLP_NP + 255) / 256];
#pragma unroll
  for (int q = 0; q < (MLP_NP + 255) / 256; ++q) g[q] = 0.f;
  double lsum = 0.0;
  const int64_t r_begin = (int64_t)blockIdx.x * chunk, r_end = min(n, r_begin + chunk);
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  for (int64_t c0 = r_begin; c0 < r_end; c0 += GB_ROWS) {
    const int nr = (int)min((int64_t)GB_ROWS, r_end - c0);
    // forward: z, h1
    for (int e = threadIdx.x; e < nr * 4; e += blockDim.x) {
      int r = e / 4, f = e % 4;
      z[r][f] = (x[(c0 + r) * 4 + f] - sp[MLP_XMEAN + f]) / sp[MLP_XSTD + f];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * MLP_H; e += blockDim.x) {
      int r = e / MLP_H, j = e % MLP_H;
      float a = sp[MLP_B1 + j];
      for (int i = 0; i < 4; ++i) a += sp[MLP_W1 + j * 4 + i] * z[r][i];
      h1[r][j] = tanhf(a);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * MLP_H; e += blockDim.x) {
      int r = e / MLP_H, j = e % MLP_H;
      float a = sp[MLP_B2 + j];
      for (int i = 0; i < MLP_H; ++i) a += sp[MLP_W2 + j * MLP_H + i] * h1[r][i];
      h2[r][j] = tanhf(a);
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      int r = threadIdx.x;
      float o = sp[MLP_B3];
      for (int i = 0; i < MLP_H; ++i) o += sp[MLP_W3 + i] * h2[r][i];
      float t = (y[c0 + r] - sp[MLP_YMEAN]) / sp[MLP_YSTD];
      float e = o - t;
      lsum += (double)e * (double)e;
      dout[r] = 2.0f * e * inv_n;
    }
    __syncthreads();
    // backward: d2 = dout W3 (1 - h2^2); d1 = (W2^T d2)(1 - h1^2)
    for (int e = threadIdx.x; e < nr * MLP_H; e += blockDim.x) {
      int r = e / MLP_H, j = e % MLP_H;
      d2[r][j] = dout[r] * sp[MLP_W3 + j] * (1.0f - h2[r][j] * h2[r][j]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * MLP_H; e += blockDim.x) {
      int r = e / MLP_H, i = e % MLP_H;
      float a = 0.f;
      for (int j = 0; j < MLP_H; ++j) a += sp[MLP_W2 + j * MLP_H + i] * d2[r][j];
      d1[r][i] = a * (1.0f - h1[r][i] * h1[r][i]);
    }
    __syncthreads();
    // parameter gradients of this chunk, thread-owned parameters (fixed summation order)
#pragma unroll
    for (int q = 0; q < (MLP_NP + 255) / 256; ++q) {
      int i = threadIdx.x + 256 * q;
      if (i >= MLP_NP) continue;
      float a = 0.f;
      if (i < MLP_B1) {
        int j = i / 4, f = i % 4;
        for (int r = 0; r < nr; ++r) a += d1[r][j] * z[r][f];
      } else if (i < MLP_W2) {
        int j = i - MLP_B1;
        for (int r = 0; r < nr; ++r) a += d1[r][j];
      } else if (i < MLP_B2) {
        int j = (i - MLP_W2) / MLP_H, l = (i - MLP_W2) % MLP_H;
        for (int r = 0; r < nr; ++r) a += d2[r][j] * h1[r][l];
      } else if (i < MLP_W3) {
        int j = i - MLP_B2;
        for (int r = 0; r < nr; ++r) a += d2[r][j];
      } else if (i < MLP_B3) {
        int j = i - MLP_W3;
        for (int r = 0; r < nr; ++r) a += dout[r] * h2[r][j];
      } else {
        for (int r = 0; r < nr; ++r) a += dout[r];
      }
      g[q] += a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (MLP_NP + 255) / 256; ++q) {
    int i = threadIdx.x + 256 * q;
    if (i < MLP_NP) part[(int64_t)blockIdx.x * MLP_NP + i] = g[q];
  }
  lred[threadIdx.x] = lsum;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) lred[threadIdx.x] += lred[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = lred[0];
}

__global__ void grad_reduce_kernel(const float *part, int nblocks, float *grad, const double *loss_part,
                                   int64_t n, double *loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NP) {
    float a = 0.f;
    for (int b = 0; b < nblocks; ++b) a += part[(int64_t)b * MLP_NP + i];
    grad[i] = a;
  }
  if (i == 0) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += loss_part[b];
    *loss = n > 0 ? l / n : 0.0;
  }
}

__global__ void adam_kernel(float *p, float *m, float *v, const float *g, float lr, float b1, float b2,
                            float eps, int step) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NP) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float mh = mi / (1.f - powf(b1, (float)step));
  float vh = vi / (1.f - powf(b2, (float)step));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// rows of one minibatch: counter-based sample with replacement
__global__ void gather_batch_kernel(const float *x, const float *y, int64_t n, int batch, uint64_t seed,
                                    int step, float *bx, float *by) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= batch) return;
  int64_t src = (int64_t)(u01(seed ^ (0xA5A5A5A5ull * (uint64_t)(step + 1)), (uint64_t)r) * (double)n);
  if (src >= n) src = n - 1;
  for (int f = 0; f < 4; ++f) bx[r * 4 + f] = x[src * 4 + f];
  by[r] = y[src];
}

}  // namespace

int mlp_grad_blocks(int64_t n) {
  int64_t chunk = 1024;
  int64_t nb = (n + chunk - 1) / chunk;
  return (int)(nb < 1 ? 1 : (nb > 1024 ? 1024 : nb));
}

size_t mlp_grad_workspace(int64_t n) {
  return (size_t)mlp_grad_blocks(n) * (MLP_NP * sizeof(float) + sizeof(double)) + 64;
}

cudaError_t mlp_init(float *p, uint64_t seed, cudaStream_t s) {
  mlp_init_kernel<<<counted((MLP_NP + 255) / 256), 256, 0, s>>>(p, seed);
  return cudaGetLastError();
}

cudaError_t mlp_fit_norm(float *p, const float *x, const float *y, int64_t n, cudaStream_t s) {
  mlp_norm_kernel<<<counted(1), 256, 0, s>>>(p, x, y, n);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const float *p, const float *x, int64_t n, float *y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  mlp_forward_kernel<<<counted((unsigned)blocks), 256, 0, s>>>(p, x, n, y);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float *p, const float *x, const float *y, int64_t n, float *grad, double *d_loss,
                     void *ws, cudaStream_t s) {
  int nb = mlp_grad_blocks(n);
  int64_t chunk = (n + nb - 1) / nb;
  float *part = (float *)ws;
  double *lpart = (double *)(((uintptr_t)(part + (size_t)nb * MLP_NP) + 15) & ~(uintptr_t)15);
  mlp_grad_partial_kernel<<<counted(nb), 256, 0, s>>>(p, x, y, n, chunk, part, lpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  grad_reduce_kernel<<<counted((MLP_NP + 255) / 256), 256, 0, s>>>(part, nb, grad, lpart, n, d_loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, float lr, int step, cudaStream_t s) {
  adam_kernel<<<counted((MLP_NP + 255) / 256), 256, 0, s>>>(p, m, v, g, lr, 0.9f, 0.999f, 1e-8f, step);
  return cudaGetLastError();
}

cudaError_t mlp_gather_batch(const float *x, const float *y, int64_t n, int batch, uint64_t seed, int step,
                             float *bx, float *by, cudaStream_t s) {
  gather_batch_kernel<<<counted((batch + 255) / 256), 256, 0, s>>>(x, y, n, batch, seed, step, bx, by);
  return cudaGetLastError();
}

}  // namespace mra
