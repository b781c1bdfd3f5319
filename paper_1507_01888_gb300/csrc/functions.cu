// functions.cu -- products and inner products of functions held on different leaf trees.
//
// Two trees of disjoint leaves are first brought onto their common refinement: each tree's
// leaves plus zero boxes at the other tree's leaf keys are summed down (mra_reconstruct), which
// gives both functions on the same leaves.  The product then uses the third representation of
// Sec. 2.1: the values at the k Gauss-Legendre points of every box.  With V[q][i] = phi_i(x_q)
// and weights w_q on (0,1), a leaf of width h holds f = h^{-3/2} (V x V x V) s at its points,
// and coefficients come back as s = h^{3/2} (V^T W)^{x3} f, so the product's coefficients are
//     s_ab = h^{-3/2} (V^T W)^{x3} [ (V^{x3} s_a) * (V^{x3} s_b) ],
// the product interpolated at the points.  The inner product is the coefficient dot product
// over the common leaves (the basis is orthonormal).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cub/cub.cuh>

#include "mra_internal.cuh"

namespace mra {
namespace {

// c <- alpha c over n * k3 coefficients (grid-stride).
__global__ void scale_kernel(int64_t n, double alpha, double *c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c[i] *= alpha;
}

// Coefficients of the union leaves: the tree's own where the key is its, zero elsewhere.
__global__ void ext_rows_kernel(int64_t n, int k3, const int64_t *src, const double *coeffs, double *out) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t s = src[i];
  for (int e = threadIdx.x; e < k3; e += blockDim.x) out[i * k3 + e] = s >= 0 ? coeffs[s * k3 + e] : 0.0;
}

// One CTA per leaf: s_ab = h^{-3/2} (V^T W)^{x3} [(V^{x3} s_a) (V^{x3} s_b)].  VW[q][i] holds
// V[q][i] and VW[k*k + i*k + q] holds w_q V[q][i].  Shared memory: 4 k^3 doubles.
__global__ void product_kernel(int k, double L, int64_t n, const uint64_t *keys, const double *a, const double *b,
                               const double *VW, double *out) {
  extern __shared__ double sh[];
  const int64_t leaf = blockIdx.x;
  if (leaf >= n) return;
  const int k2 = k * k, k3 = k2 * k;
  double *x = sh, *y = x + k3, *t = y + k3, *u = t + k3;
  const double *V = VW, *VtW = VW + k2;
  const double h = 2.0 * L / (double)(1LL << key_level(keys[leaf]));
  // values of a (into x) and of b (into y): three mode products each
  for (int pass = 0; pass < 2; ++pass) {
    const double *src = pass == 0 ? a : b;
    double *dst = pass == 0 ? x : y;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) t[e] = src[leaf * k3 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // u[q][j][l] = sum_i V[q][i] t[i][j][l]
      const int q = e / k2, r = e % k2;
      double v = 0.0;
      for (int i = 0; i < k; ++i) v += V[q * k + i] * t[i * k2 + r];
      u[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // t[q][p][l] = sum_j V[p][j] u[q][j][l]
      const int q = e / k2, p = (e / k) % k, l = e % k;
      double v = 0.0;
      for (int j = 0; j < k; ++j) v += V[p * k + j] * u[(q * k + j) * k + l];
      t[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // dst[q][p][r] = sum_l V[r][l] t[q][p][l]
      const int qp = e / k, r = e % k;
      double v = 0.0;
      for (int l = 0; l < k; ++l) v += V[r * k + l] * t[qp * k + l];
      dst[e] = v;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k3; e += blockDim.x) t[e] = x[e] * y[e];
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // back: u[i][p][r] = sum_q VtW[i][q] t[q][p][r]
    const int i = e / k2, r = e % k2;
    double v = 0.0;
    for (int q = 0; q < k; ++q) v += VtW[i * k + q] * t[q * k2 + r];
    u[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    const int i = e / k2, j = (e / k) % k, r = e % k;
    double v = 0.0;
    for (int p = 0; p < k; ++p) v += VtW[j * k + p] * u[(i * k + p) * k + r];
    x[e] = v;
  }
  __syncthreads();
  const double scale = 1.0 / (h * sqrt(h));
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    const int ij = e / k, l = e % k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += VtW[l * k + r] * x[ij * k + r];
    out[leaf * k3 + e] = scale * v;
  }
}

__global__ void dot_rows_kernel(int64_t n, int k3, const double *a, const double *b, double *d) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int e = lane; e < k3; e += 32) s += a[i * k3 + e] * b[i * k3 + e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) d[i] = s;
}

// Device buffers released on scope exit (stream-ordered).
struct Pool {
  cudaStream_t s;
  std::vector<void *> held;
  explicit Pool(cudaStream_t st) : s(st) {}
  ~Pool() {
    for (void *p : held) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  }
  void *get(size_t bytes) {
    void *p = nullptr;
    if (pool_malloc(&p, bytes ? bytes : 1, s) != cudaSuccess) return nullptr;
    held.push_back(p);
    return p;
  }
};

int check_leaf_view(const mra_tree_view *v, const char *what) {
  if (!v) return fail(MRA_ERR_ARG, "%s: NULL tree", what);
  if (v->n < 0 || (v->n > 0 && (!v->keys || !v->coeffs))) return fail(MRA_ERR_ARG, "%s: bad tree view", what);
  if (v->k < 1 || v->k > MRA_MAX_K) return fail(MRA_ERR_ARG, "%s: k=%d outside 1..%d", what, v->k, MRA_MAX_K);
  return MRA_OK;
}

// Both trees on their common leaves: keys (shared), and each tree's coefficients there.
int align(const mra_tree_view &a, const mra_tree_view &b, Pool &pool, cudaStream_t s, int64_t *n_out,
          uint64_t **keys_out, double **ca, double **cb) {
  const int k = a.k, k3 = k * k * k;
  std::vector<uint64_t> ka(a.n), kb(b.n);
  if (a.n) MRA_CUDA_TRY(cudaMemcpyAsync(ka.data(), a.keys, (size_t)a.n * 8, cudaMemcpyDeviceToHost, s));
  if (b.n) MRA_CUDA_TRY(cudaMemcpyAsync(kb.data(), b.keys, (size_t)b.n * 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  for (size_t i = 1; i < ka.size(); ++i)
    if (ka[i] <= ka[i - 1]) return fail(MRA_ERR_ARG, "mra_multiply/inner: first tree's keys not sorted and unique");
  for (size_t i = 1; i < kb.size(); ++i)
    if (kb[i] <= kb[i - 1]) return fail(MRA_ERR_ARG, "mra_multiply/inner: second tree's keys not sorted and unique");
  if (ka == kb) {  // already on the same leaves
    *n_out = a.n;
    *keys_out = a.keys;
    *ca = a.coeffs;
    *cb = b.coeffs;
    return MRA_OK;
  }
  std::vector<uint64_t> u;
  std::set_union(ka.begin(), ka.end(), kb.begin(), kb.end(), std::back_inserter(u));
  const int64_t nu = (int64_t)u.size();
  std::vector<int64_t> ia(nu), ib(nu);
  for (int64_t i = 0; i < nu; ++i) {
    auto pa = std::lower_bound(ka.begin(), ka.end(), u[i]);
    auto pb = std::lower_bound(kb.begin(), kb.end(), u[i]);
    ia[i] = (pa != ka.end() && *pa == u[i]) ? pa - ka.begin() : -1;
    ib[i] = (pb != kb.end() && *pb == u[i]) ? pb - kb.begin() : -1;
  }
  uint64_t *du = (uint64_t *)pool.get(nu * 8);
  int64_t *dia = (int64_t *)pool.get(nu * 8), *dib = (int64_t *)pool.get(nu * 8);
  double *ea = (double *)pool.get(nu * k3 * 8), *eb = (double *)pool.get(nu * k3 * 8);
  if (!du || !dia || !dib || !ea || !eb) return fail(MRA_ERR_CUDA, "mra_multiply/inner: out of device memory");
  MRA_CUDA_TRY(cudaMemcpyAsync(du, u.data(), nu * 8, cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(dia, ia.data(), nu * 8, cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(dib, ib.data(), nu * 8, cudaMemcpyHostToDevice, s));
  if (nu > 0) {
    ext_rows_kernel<<<counted((unsigned)nu), 128, 0, s>>>(nu, k3, dia, a.coeffs, ea);
    ext_rows_kernel<<<counted((unsigned)nu), 128, 0, s>>>(nu, k3, dib, b.coeffs, eb);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  // sum both down to the common leaves; a tree whose own leaves turn out to be the common
  // leaves (the other tree's are all at or above them) is used as it is
  uint64_t *rk[2] = {nullptr, nullptr};
  double *rc[2] = {nullptr, nullptr};
  int64_t rn[2] = {0, 0};
  const bool b_finer = b.n >= a.n;  // reconstruct the coarser tree first
  for (int pass = 0; pass < 2; ++pass) {
    const int w = (pass == 0) == b_finer ? 0 : 1;
    if (pass == 1) {
      const std::vector<uint64_t> &own = w == 0 ? ka : kb;
      const int o = 1 - w;
      if (rn[o] == (int64_t)own.size()) {
        std::vector<uint64_t> got(rn[o]);
        if (rn[o]) {
          MRA_CUDA_TRY(cudaMemcpyAsync(got.data(), rk[o], rn[o] * 8, cudaMemcpyDeviceToHost, s));
          MRA_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (got == own) {
          rk[w] = w == 0 ? a.keys : b.keys;
          rc[w] = w == 0 ? a.coeffs : b.coeffs;
          rn[w] = rn[o];
          break;
        }
      }
    }
    int64_t cap = std::max<int64_t>(8 * nu, 1);
    while (true) {
      rk[w] = (uint64_t *)pool.get(cap * 8);
      rc[w] = (double *)pool.get(cap * k3 * 8);
      if (!rk[w] || !rc[w]) return fail(MRA_ERR_CUDA, "mra_multiply/inner: out of device memory");
      mra_tree_view in{nu, nu, du, w == 0 ? ea : eb, k, a.L};
      mra_tree_view out{0, cap, rk[w], rc[w], k, a.L};
      const int rc2 = mra_reconstruct(&in, &out, (void *)s);
      if (rc2 == MRA_ERR_CAPACITY && out.n > cap) {
        cap = out.n;
        continue;
      }
      if (rc2 != MRA_OK) return rc2;
      rn[w] = out.n;
      break;
    }
  }
  if (rn[0] != rn[1]) return fail(MRA_ERR_NUMERIC, "mra_multiply/inner: the common refinements differ");
  std::vector<uint64_t> k0(rn[0]), k1(rn[1]);
  if (rn[0]) {
    MRA_CUDA_TRY(cudaMemcpyAsync(k0.data(), rk[0], rn[0] * 8, cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(k1.data(), rk[1], rn[1] * 8, cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (k0 != k1) return fail(MRA_ERR_NUMERIC, "mra_multiply/inner: the common refinements differ");
  *n_out = rn[0];
  *keys_out = rk[0];
  *ca = rc[0];
  *cb = rc[1];
  return MRA_OK;
}

}  // namespace
}  // namespace mra

using namespace mra;

extern "C" int mra_multiply(const mra_tree_view *a, const mra_tree_view *b, mra_tree_view *out, void *stream) {
  int rc = check_leaf_view(a, "mra_multiply(a)");
  if (rc) return rc;
  rc = check_leaf_view(b, "mra_multiply(b)");
  if (rc) return rc;
  if (!out || out->k != a->k || out->cap < 0 || (out->cap > 0 && (!out->keys || !out->coeffs)))
    return fail(MRA_ERR_ARG, "mra_multiply: bad output view");
  if (b->k != a->k || b->L != a->L) return fail(MRA_ERR_ARG, "mra_multiply: trees of different k or L");
  out->L = a->L;
  if (a->n == 0 || b->n == 0) {
    out->n = 0;
    return MRA_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  int64_t n = 0;
  uint64_t *keys = nullptr;
  double *ca = nullptr, *cb = nullptr;
  rc = align(*a, *b, pool, s, &n, &keys, &ca, &cb);
  if (rc) return rc;
  if (n > out->cap) {
    out->n = n;
    return fail(MRA_ERR_CAPACITY, "mra_multiply: %lld leaves, capacity %lld", (long long)n, (long long)out->cap);
  }
  const int k = a->k, k3 = k * k * k;
  // V[q][i] = phi_i(x_q) and w_q V[q][i] (stored transposed) at the k Gauss-Legendre points on (0,1)
  std::vector<double> gx(k), gw(k), VW(2 * k * k);
  gauss_legendre(k, gx.data(), gw.data());
  for (int q = 0; q < k; ++q) {
    const double xq = 0.5 * (gx[q] + 1.0), wq = 0.5 * gw[q], t = 2.0 * xq - 1.0;
    double p0 = 1.0, p1 = t;
    for (int i = 0; i < k; ++i) {
      double P = i == 0 ? 1.0 : (i == 1 ? t : 0.0);
      if (i >= 2) {
        P = ((2.0 * i - 1.0) * t * p1 - (i - 1.0) * p0) / i;
        p0 = p1;
        p1 = P;
      }
      const double phi = sqrt(2.0 * i + 1.0) * P;
      VW[q * k + i] = phi;
      VW[k * k + i * k + q] = wq * phi;
    }
  }
  double *dVW = (double *)pool.get(VW.size() * 8);
  if (!dVW) return fail(MRA_ERR_CUDA, "mra_multiply: out of device memory");
  MRA_CUDA_TRY(cudaMemcpyAsync(dVW, VW.data(), VW.size() * 8, cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaFuncSetAttribute(product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(4 * k3 * sizeof(double))));
  product_kernel<<<counted((unsigned)n), 128, 4 * k3 * sizeof(double), s>>>(k, a->L, n, keys, ca, cb, dVW, out->coeffs);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cudaMemcpyAsync(out->keys, keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  out->n = n;
  return MRA_OK;
}

extern "C" int mra_inner(const mra_tree_view *a, const mra_tree_view *b, double *result, void *stream) {
  int rc = check_leaf_view(a, "mra_inner(a)");
  if (rc) return rc;
  rc = check_leaf_view(b, "mra_inner(b)");
  if (rc) return rc;
  if (!result) return fail(MRA_ERR_ARG, "mra_inner: NULL result");
  if (b->k != a->k || b->L != a->L) return fail(MRA_ERR_ARG, "mra_inner: trees of different k or L");
  *result = 0.0;
  if (a->n == 0 || b->n == 0) return MRA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Pool pool(s);
  int64_t n = 0;
  uint64_t *keys = nullptr;
  double *ca = nullptr, *cb = nullptr;
  rc = align(*a, *b, pool, s, &n, &keys, &ca, &cb);
  if (rc) return rc;
  const int k3 = a->k * a->k * a->k;
  double *d = (double *)pool.get(n * 8), *sum = (double *)pool.get(8);
  if (!d || !sum) return fail(MRA_ERR_CUDA, "mra_inner: out of device memory");
  dot_rows_kernel<<<counted((unsigned)((n + 7) / 8)), 256, 0, s>>>(n, k3, ca, cb, d);
  MRA_CUDA_TRY(cudaGetLastError());
  size_t tb = 0;
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(nullptr, tb, d, sum, (int)n, s));
  void *tmp = pool.get(tb);
  if (!tmp) return fail(MRA_ERR_CUDA, "mra_inner: out of device memory");
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tb, d, sum, (int)n, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(result, sum, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  return MRA_OK;
}

extern "C" int mra_scale(mra_tree_view *t, double alpha, void *stream) {
  if (!t) return fail(MRA_ERR_ARG, "mra_scale: NULL tree view");
  if (t->n < 0 || t->n > t->cap) return fail(MRA_ERR_ARG, "mra_scale: bad n/cap");
  if (t->k < 1 || t->k > MRA_MAX_NS_K) return fail(MRA_ERR_ARG, "mra_scale: k=%d invalid", t->k);
  if (!std::isfinite(alpha)) return fail(MRA_ERR_ARG, "mra_scale: alpha is not finite");
  if (t->n == 0) return MRA_OK;
  if (!t->coeffs) return fail(MRA_ERR_ARG, "mra_scale: NULL coefficients");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = t->n * (int64_t)t->k * t->k * t->k;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
  scale_kernel<<<counted(grid), 256, 0, s>>>(n, alpha, t->coeffs);
  MRA_CUDA_TRY(cudaGetLastError());
  return MRA_OK;
}
