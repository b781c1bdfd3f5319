// peak.cu -- FP64 throughput of this GPU, measured: the rate a loop of independent DFMA chains
// reaches on the FP64 units and the rate a loop of FP64 warp-level MMAs (mma.sync m16n8k16,
// DMMA) reaches, each timed with CUDA events over the whole device.  The FP64 apply kernel
// (three k x k mode products per term in DFMA) is measured against the DFMA figure.
#include <algorithm>

#include "mra_internal.cuh"

namespace mra {

namespace {

// sink for the probes' results: written only if a sum takes an impossible value, so that the
// compiler keeps the arithmetic
static __device__ double g_peak_sink;

constexpr int PEAK_THREADS = 256;
constexpr int DFMA_CHAINS = 16;

// Each thread runs DFMA_CHAINS independent chains x <- x a + b (a < 1, so x stays bounded), the
// loop unrolled so that loop control takes few issue slots.
__global__ void __launch_bounds__(PEAK_THREADS) dfma_probe_kernel(int iters, double a, double b) {
  double x[DFMA_CHAINS];
#pragma unroll
  for (int c = 0; c < DFMA_CHAINS; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < DFMA_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < DFMA_CHAINS; ++c) s += x[c];
  if (s == -1.0) g_peak_sink = s;
}

// Each warp runs four independent accumulator sets through mma.sync m16n8k16 f64
// (16 x 8 x 16 multiply-adds per warp and instruction).
__global__ void __launch_bounds__(PEAK_THREADS) dmma_probe_kernel(int iters, double a, double b) {
  double d[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int j = 0; j < 4; ++j) d[s][j] = 0.0;
  const double a0 = a, a1 = b * 0.5, a2 = a * 0.25, a3 = b, a4 = a, a5 = b * 0.5, a6 = a * 0.25, a7 = b;
  const double b0 = b, b1 = a * 0.5, b2 = b * 0.25, b3 = a;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
          "{%12,%13,%14,%15}, {%0,%1,%2,%3};"
          : "+d"(d[s][0]), "+d"(d[s][1]), "+d"(d[s][2]), "+d"(d[s][3])
          : "d"(a0), "d"(a1), "d"(a2), "d"(a3), "d"(a4), "d"(a5), "d"(a6), "d"(a7), "d"(b0), "d"(b1), "d"(b2),
            "d"(b3));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += d[q][j];
  if (s == -1.0) g_peak_sink = s;
}

// TFLOP/s of `kern` with `iters` iterations: best of three timed launches after one warm-up.
int time_probe(void (*kern)(int, double, double), unsigned grid, int iters, double flops_per_launch,
               cudaStream_t s, double *tflops) {
  cudaEvent_t e0, e1;
  MRA_CUDA_TRY(cudaEventCreate(&e0));
  MRA_CUDA_TRY(cudaEventCreate(&e1));
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    MRA_CUDA_TRY(cudaEventRecord(e0, s));
    kern<<<counted(grid), PEAK_THREADS, 0, s>>>(iters, 0.9999999, 1e-7);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cudaEventRecord(e1, s));
    MRA_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    MRA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms > 0.f) best = std::max(best, flops_per_launch / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return MRA_OK;
}

}  // namespace

}  // namespace mra

using namespace mra;

extern "C" int mra_measure_fp64_peak(double seconds, double *dfma_tflops, double *dmma_tflops, void *stream) {
  if (!(seconds > 0.0) || seconds > 60.0) return fail(MRA_ERR_ARG, "mra_measure_fp64_peak: seconds %g not in (0, 60]", seconds);
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  MRA_CUDA_TRY(cudaGetDevice(&dev));
  MRA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)sms * 8;  // eight CTAs of 256 threads per SM: full occupancy
  const double threads = (double)grid * PEAK_THREADS;
  const double per_probe = seconds / 8.0;   // four launches of each probe
  // DFMA: calibrate the iteration count on a short launch, then time launches of ~per_probe s
  double t = 0.0;
  int it = 1 << 12;
  int rc = time_probe(dfma_probe_kernel, grid, it, threads * it * DFMA_CHAINS * 2.0, s, &t);
  if (rc != MRA_OK) return rc;
  if (t > 0.0) it = (int)std::min(1e9, std::max(1e3, per_probe * t * 1e12 / (threads * DFMA_CHAINS * 2.0)));
  rc = time_probe(dfma_probe_kernel, grid, it, threads * it * DFMA_CHAINS * 2.0, s, &t);
  if (rc != MRA_OK) return rc;
  if (dfma_tflops) *dfma_tflops = t;
  // DMMA: 2 * 16 * 8 * 16 flops per warp and instruction, four instructions per iteration
  const double warps = threads / 32.0, per_it = warps * 4.0 * 2.0 * 16 * 8 * 16;
  it = 1 << 10;
  rc = time_probe(dmma_probe_kernel, grid, it, per_it * it, s, &t);
  if (rc != MRA_OK) return rc;
  if (t > 0.0) it = (int)std::min(1e9, std::max(1e2, per_probe * t * 1e12 / per_it));
  rc = time_probe(dmma_probe_kernel, grid, it, per_it * it, s, &t);
  if (rc != MRA_OK) return rc;
  if (dmma_tflops) *dmma_tflops = t;
  return MRA_OK;
}
