// mra_internal.cuh -- shared declarations of libmra's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mra.h"

namespace mra {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);

#define MRA_CUDA_TRY(call)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::mra::fail(MRA_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,  \
                         cudaGetErrorString(e_));                                   \
  } while (0)

// ---------------------------------------------------------------- launch count
// Every kernel launch of the library takes its grid through counted(), so that
// mra_launch_count reports how many kernels the library has launched.
void note_launch();
long long launch_total();
template <class G>
inline G counted(G grid) {
  note_launch();
  return grid;
}

// ---------------------------------------------------------------- device memory
// Scratch of the host-orchestrated calls comes from a stream-ordered pool of the library's
// own (one per device) that keeps freed memory for the next call instead of returning it to
// the driver at every synchronisation, as the default pool does; mra_release_memory trims it.
cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s);

// ---------------------------------------------------------------- index checks
// The checking build (-DMRA_DEBUG) routes indices of the hot kernels' gathers and scatters
// through MRA_IDX(i, n): an index outside [0, n) is replaced by 0, so the access stays in
// bounds, and the first failing source line is kept in a device word of the translation unit,
// which mra_debug_status reads.  In the release build MRA_IDX(i, n) is i.
#ifdef MRA_DEBUG
static __device__ int g_debug_line;
template <class I, class N>
__device__ __forceinline__ I debug_idx(I i, N n, int line) {
  if (i < 0 || (long long)i >= (long long)n) {
    atomicCAS(&g_debug_line, 0, line);
    return (I)0;
  }
  return i;
}
#define MRA_IDX(i, n) ::mra::debug_idx((i), (n), __LINE__)
// the translation unit's first failing line since the last read (0: none), cleared
static inline int debug_take_line(cudaStream_t s) {
  int h = 0, z = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_debug_line, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbolAsync(g_debug_line, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return h;
}
#else
#define MRA_IDX(i, n) (i)
static inline int debug_take_line(cudaStream_t) { return 0; }
#endif
int debug_line_apply(cudaStream_t s);
int debug_line_split(cudaStream_t s);
int debug_line_src(cudaStream_t s);

// ---------------------------------------------------------------- keys
__host__ __device__ inline uint64_t make_key(int n, int64_t x, int64_t y, int64_t z) {
  return ((uint64_t)n << 57) | ((uint64_t)x << 38) | ((uint64_t)y << 19) | (uint64_t)z;
}
__host__ __device__ inline int key_level(uint64_t k) { return (int)(k >> 57); }
__host__ __device__ inline int64_t key_x(uint64_t k) { return (int64_t)((k >> 38) & 0x7FFFF); }
__host__ __device__ inline int64_t key_y(uint64_t k) { return (int64_t)((k >> 19) & 0x7FFFF); }
__host__ __device__ inline int64_t key_z(uint64_t k) { return (int64_t)(k & 0x7FFFF); }

// ---------------------------------------------------------------- operator
// Block table: for each level n in [min_level, max_level], D(n) = min(max_disp, 2^n-1),
// blocks R[n][m][l + D(n)][i][j] (k*k doubles) starting at level_off[n - min_level] blocks.
struct Operator {
  int kernel = 0;
  double mu = 0.0;
  int M = 0, k = 0;
  double L = 0.0;
  int min_level = 0, max_level = 0, max_disp = 0;
  double h_fit = 0.0, s_lo = 0.0, fit_err = 0.0, r_lo = 0.0, r_hi = 0.0, fit_eps = 0.0;
  bool r_hi_auto = false;                 // r_hi derived from (L, fit_eps, mu) at creation
  bool non_standard = false;              // made by mra_operator_ns_create (blocks gathered, not fitted)
  std::vector<double> c, t;               // host copies of the fit
  std::vector<int> D;                     // per level (index n - min_level)
  std::vector<int64_t> level_off;         // first block index of each level
  int64_t n_blocks = 0;
  double *d_c = nullptr, *d_t = nullptr;  // device fit
  double *d_R = nullptr;                  // device blocks, n_blocks * k*k
  double *d_N = nullptr;                  // device block norms, n_blocks
  int *d_D = nullptr;                     // device copy of D (20 entries, by absolute level)
  int64_t *d_level_off = nullptr;         // device copy (20 entries, by absolute level; -1 = absent)
  // split-precision copies of the blocks for the tensor-core path (lazily built)
  void *d_Rsplit = nullptr;
  int split_pieces = 0;
};

// ---------------------------------------------------------------- host helpers
void gauss_legendre(int n, double *x, double *w);  // nodes/weights on [-1,1]
void two_scale(int k, double *U /* [2][k][k] */);  // U^(c)[i][j], Sec. 2.2
void free_operator(Operator *op);

// ---------------------------------------------------------------- launchers (setup)
cudaError_t launch_fit_search(double mu, int M, double r_lo, double r_hi, int stride, const int *d_pts, int npts,
                              const int *d_cands, int n_cands, double stop, double *d_err, cudaStream_t s);
cudaError_t launch_blocks(const Operator &op, const double *d_glx, const double *d_glw,
                          cudaStream_t s);
cudaError_t launch_project_boxes(int ng, const double *d_g /*[5][ng]*/, int k, double L,
                                 int64_t nbox, const uint64_t *d_keys, double *d_out,
                                 cudaStream_t s);
cudaError_t launch_refine_test(int k, int64_t nparent, const double *d_parent,
                               const double *d_child, const double *d_U, double *d_dnorm,
                               cudaStream_t s);
}  // namespace mra
