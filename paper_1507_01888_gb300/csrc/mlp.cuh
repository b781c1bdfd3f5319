// mlp.cuh -- layout of the learned screen's network and its single-row forward pass.
#pragma once

#include "mra_internal.cuh"

namespace mra {

constexpr int MLP_IN = 4, MLP_H = 64;
constexpr int MLP_W1 = 0;                          // [64][4]
constexpr int MLP_B1 = MLP_W1 + MLP_H * MLP_IN;     // [64]
constexpr int MLP_W2 = MLP_B1 + MLP_H;              // [64][64]
constexpr int MLP_B2 = MLP_W2 + MLP_H * MLP_H;      // [64]
constexpr int MLP_W3 = MLP_B2 + MLP_H;              // [64]
constexpr int MLP_B3 = MLP_W3 + MLP_H;              // scalar
constexpr int MLP_NP = MLP_B3 + 1;                  // trainable parameters (4545)
constexpr int MLP_XMEAN = MLP_NP, MLP_XSTD = MLP_NP + 4, MLP_YMEAN = MLP_NP + 8, MLP_YSTD = MLP_NP + 9;
constexpr int MLP_NALL = MLP_NP + 10;               // with the standardisation (4555)
static_assert(MLP_NALL == MRA_MLP_PARAMS, "parameter count must match mra.h");
static_assert(MLP_W1 % 4 == 0 && MLP_W2 % 4 == 0, "float4 rows of the network must be 16-byte aligned");

// Predicted log10 of a term's norm for features x[4]; p in shared or global memory, 16-byte
// aligned.  The hidden activations stay in registers (every index below is compile-time);
// the 64 x 64 layer is read as float4 rows.
__device__ __forceinline__ float mlp_predict(const float *p, const float *x) {
  float z[MLP_IN];
#pragma unroll
  for (int f = 0; f < MLP_IN; ++f) z[f] = (x[f] - p[MLP_XMEAN + f]) / p[MLP_XSTD + f];
  float h1[MLP_H];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) {
    const float4 w = *(const float4 *)(p + MLP_W1 + j * MLP_IN);
    float a = p[MLP_B1 + j];
    a += w.x * z[0];
    a += w.y * z[1];
    a += w.z * z[2];
    a += w.w * z[3];
    h1[j] = tanhf(a);
  }
  float o = p[MLP_B3];
#pragma unroll 1
  for (int j = 0; j < MLP_H; ++j) {
    const float4 *row = (const float4 *)(p + MLP_W2 + j * MLP_H);
    float a = p[MLP_B2 + j];
#pragma unroll
    for (int i4 = 0; i4 < MLP_H / 4; ++i4) {
      const float4 w = row[i4];
      a += w.x * h1[4 * i4];
      a += w.y * h1[4 * i4 + 1];
      a += w.z * h1[4 * i4 + 2];
      a += w.w * h1[4 * i4 + 3];
    }
    o += p[MLP_W3 + j] * tanhf(a);
  }
  return o * p[MLP_YSTD] + p[MLP_YMEAN];
}

int mlp_grad_blocks(int64_t n);
size_t mlp_grad_workspace(int64_t n);
cudaError_t mlp_init(float *p, uint64_t seed, cudaStream_t s);
cudaError_t mlp_fit_norm(float *p, const float *x, const float *y, int64_t n, cudaStream_t s);
cudaError_t mlp_forward(const float *p, const float *x, int64_t n, float *y, cudaStream_t s);
cudaError_t mlp_grad(const float *p, const float *x, const float *y, int64_t n, float *grad, double *d_loss,
                     void *ws, cudaStream_t s);
cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, float lr, int step, cudaStream_t s);
cudaError_t mlp_gather_batch(const float *x, const float *y, int64_t n, int batch, uint64_t seed, int step,
                             float *bx, float *by, cudaStream_t s);

}  // namespace mra
