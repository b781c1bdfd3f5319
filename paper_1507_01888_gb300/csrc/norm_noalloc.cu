// norm_noalloc.cu -- mra_norm_noalloc: the tree-norm reduction without any device
// allocation, for callers that cannot allocate device memory (see include/mra.h).
//
// Scratch lives in one file-scope __device__ array of fixed size, shared by every
// call on a device.  Host code never uses the array's name as an address: every
// call asks the runtime for the array's device address in the current device's
// context with cudaGetSymbolAddress and passes that pointer to the kernels.  The
// lookup is not cached, so a new primary context (after cudaDeviceReset) gets its
// own address; once the module is loaded in a context the lookup allocates nothing.

#include "mra_internal.cuh"

namespace mra {

namespace {

// [0, MAX) per-box squared norms, [MAX] the total.  Every slot a call reads is
// written earlier in the same call, so nothing needs clearing between calls.
static __device__ __align__(256) double g_norm_scratch[MRA_NOALLOC_MAX_BOXES + 32];

__global__ void sq_norm_kernel(int64_t n, int k3, const double *coeffs, double *sq,
                               double *per_box) {
  int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (b >= n) return;
  const double *s = coeffs + b * k3;
  double a = 0.0;
  for (int e = lane; e < k3; e += 32) a += s[e] * s[e];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) {
    sq[b] = a;
    if (per_box) per_box[b] = sqrt(a);
  }
}

// One CTA of 1024 threads: fixed-order partial sums, then a tree reduction.
__global__ void sum_kernel(int64_t n, const double *sq, double *total) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += sq[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = red[0];
}

// Device address of the scratch array in the current device's context.  The first lookup in a
// context loads the library's device code there (lazy module loading), which brings the array
// into that device's memory; later lookups only read the address.
int scratch_for_current_device(double **out) {
  int dev = 0;
  MRA_CUDA_TRY(cudaGetDevice(&dev));
  double *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void **)&p, g_norm_scratch);
  if (e != cudaSuccess || !p)
    return fail(MRA_ERR_CUDA, "mra_norm_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                cudaGetErrorString(e));
  *out = p;
  return MRA_OK;
}

}  // namespace

}  // namespace mra

using namespace mra;

extern "C" int mra_norm_noalloc(const mra_tree_view *t, double *per_box, double *total,
                                void *stream) {
  if (!t) return fail(MRA_ERR_ARG, "mra_norm_noalloc: NULL tree view");
  if (t->n < 0 || t->cap < 0 || t->n > t->cap) return fail(MRA_ERR_ARG, "mra_norm_noalloc: bad n/cap");
  if (t->k < 1 || t->k > MRA_MAX_K) return fail(MRA_ERR_ARG, "mra_norm_noalloc: k=%d invalid", t->k);
  if (t->n > MRA_NOALLOC_MAX_BOXES)
    return fail(MRA_ERR_CAPACITY,
                "mra_norm_noalloc: %lld boxes exceed the fixed scratch of %d boxes; use mra_norm",
                (long long)t->n, (int)MRA_NOALLOC_MAX_BOXES);
  if (t->n > 0 && !t->coeffs) return fail(MRA_ERR_ARG, "mra_norm_noalloc: NULL coefficients");
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MRA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = t->n;
  const int k3 = t->k * t->k * t->k;
  double *sq = scratch, *tot = scratch + MRA_NOALLOC_MAX_BOXES;
  if (n > 0) {
    const int wpb = 8;
    sq_norm_kernel<<<counted((unsigned)((n + wpb - 1) / wpb)), 32 * wpb, 0, s>>>(n, k3, t->coeffs, sq, per_box);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  sum_kernel<<<counted(1), 1024, 0, s>>>(n, sq, tot);
  MRA_CUDA_TRY(cudaGetLastError());
  double h = 0.0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&h, tot, sizeof(double), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (total) *total = sqrt(h);
  return MRA_OK;
}
