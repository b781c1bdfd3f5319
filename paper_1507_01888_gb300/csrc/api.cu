// api.cu -- the extern "C" entry points declared in include/mra.h.
#include <atomic>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <cub/cub.cuh>
#include <vector>

#include "apply_internal.cuh"
#include "mlp.cuh"

namespace mra {

static thread_local char g_err[1024] = "no error";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

// n-point Gauss-Legendre rule on [-1,1] (Newton iteration on P_n).
void gauss_legendre(int n, double *x, double *w) {
  const double pi = 3.14159265358979323846264338327950288;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5)), pn = 0.0, pm = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      pm = 1.0;
      pn = z;
      for (int m = 1; m < n; ++m) {
        double nx = ((2.0 * m + 1.0) * z * pn - m * pm) / (m + 1.0);
        pm = pn;
        pn = nx;
      }
      if (n == 1) { pn = z; pm = 1.0; }
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    pm = 1.0;
    pn = z;
    for (int m = 1; m < n; ++m) {
      double nx = ((2.0 * m + 1.0) * z * pn - m * pm) / (m + 1.0);
      pm = pn;
      pn = nx;
    }
    if (n == 1) { pn = z; pm = 1.0; }
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Two-scale matrices U^{(c)}[i][j] = 2^{-1/2} int_0^1 phi_i(y) phi_j((y+c)/2) dy (Sec. 2.2).
void two_scale(int k, double *U /* [2][k][k] */) {
  int nq = k + 2;
  std::vector<double> x(nq), w(nq);
  gauss_legendre(nq, x.data(), w.data());
  auto phi = [k](double t, double *out) {
    double xx = 2.0 * t - 1.0, p0 = 1.0, p1 = xx;
    out[0] = 1.0;
    if (k > 1) out[1] = sqrt(3.0) * xx;
    for (int m = 1; m + 1 < k; ++m) {
      double p2 = ((2.0 * m + 1.0) * xx * p1 - m * p0) / (m + 1.0);
      p0 = p1;
      p1 = p2;
      out[m + 1] = sqrt(2.0 * m + 3.0) * p2;
    }
  };
  double pi_[MRA_MAX_K], pj[MRA_MAX_K];
  for (int c = 0; c < 2; ++c) {
    double *Uc = U + c * k * k;
    for (int i = 0; i < k * k; ++i) Uc[i] = 0.0;
    for (int q = 0; q < nq; ++q) {
      double y = 0.5 * (x[q] + 1.0), wy = 0.5 * w[q];
      phi(y, pi_);
      phi(0.5 * (y + c), pj);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Uc[i * k + j] += wy * pi_[i] * pj[j] / sqrt(2.0);
    }
  }
}

void free_operator(Operator *op) {
  if (!op) return;
  cudaFree(op->d_c);
  cudaFree(op->d_t);
  cudaFree(op->d_R);
  cudaFree(op->d_N);
  cudaFree(op->d_D);
  cudaFree(op->d_level_off);
  cudaFree(op->d_Rsplit);
  delete op;
}

namespace {
__global__ void gather_rows_kernel(int64_t n, int row, const double *src, const int64_t *from,
                                   double *dst, int64_t dst_base) {
  int64_t r = blockIdx.x;
  if (r >= n) return;
  const double *a = src + from[r] * row;
  double *b = dst + (dst_base + r) * row;
  for (int e = threadIdx.x; e < row; e += blockDim.x) b[e] = a[e];
}
__global__ void gather_sorted_kernel(int64_t n, int row, const double *src, const int *perm,
                                     double *dst) {
  int64_t r = blockIdx.x;
  if (r >= n) return;
  const double *a = src + (int64_t)perm[r] * row;
  double *b = dst + r * row;
  for (int e = threadIdx.x; e < row; e += blockDim.x) b[e] = a[e];
}
__global__ void iota32(int64_t n, int *p) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int)i;
}
}  // namespace

std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }

constexpr int MAX_POOL_DEVICES = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[MAX_POOL_DEVICES] = {};

cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_POOL_DEVICES) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pools[dev], &props);
      if (e != cudaSuccess) {
        g_pools[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;  // never released at a synchronisation; trimmed on request
      e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

}  // namespace mra

namespace mra {
// The Gaussian fit of the operator's kernel (mu_fit = 0: 1/r) on [r_lo, r_hi]: op->h_fit, s_lo,
// fit_err, c, t (host copies).
static int fit_operator(Operator *op, double mu_fit, int M, double r_lo, double r_hi, cudaStream_t s) {
  // The grid's argmin of the max relative error over the 3000 points, the first (lowest
  // index) of equal minima.  Exact with far fewer evaluations: the maximum over 16 of the
  // points (the three at each end of the range, where the truncation of the Gaussian sum shows,
  // and twelve spread over it) is a lower bound of each candidate's error, so candidates are
  // evaluated in full in increasing order of that bound until the bound exceeds the best full
  // error found; no candidate left out can reach it.  The batches of full evaluations grow
  // from 16 (a handful are usually enough), and a full evaluation stops once it exceeds the
  // best error found before its batch (such a candidate can neither win nor tie).
  const int NC = 116 * 113, NP = 3000, BATCH = 256;
  std::vector<int> sub;
  for (int q = 0; q < 3; ++q) {
    sub.push_back(q);
    sub.push_back(NP - 1 - q);
  }
  for (int q = 0; q < 12; ++q) sub.push_back((int)lround(q * (NP - 1) / 11.0));
  std::sort(sub.begin(), sub.end());
  sub.erase(std::unique(sub.begin(), sub.end()), sub.end());
  double *d_err = nullptr;
  int *d_cand = nullptr;
  if (pool_malloc((void **)&d_err, NC * sizeof(double), s) != cudaSuccess ||
      pool_malloc((void **)&d_cand, (BATCH + 256) * sizeof(int), s) != cudaSuccess) {
    if (d_err) cudaFreeAsync(d_err, s);
    cudaStreamSynchronize(s);
    return fail(MRA_ERR_CUDA, "fit search: out of device memory");
  }
  int *d_pts = d_cand + BATCH;
  std::vector<double> lower(NC), full(NC, -1.0);
  cudaError_t e = cudaMemcpyAsync(d_pts, sub.data(), sub.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_fit_search(mu_fit, M, r_lo, r_hi, 1, d_pts, (int)sub.size(), nullptr, NC, INFINITY, d_err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lower.data(), d_err, NC * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  std::vector<int> order(NC);
  for (int q = 0; q < NC; ++q) order[q] = q;
  // NaN bounds (never produced by the finite grid) sort last and are evaluated like the rest
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const bool na = std::isnan(lower[a]), nb = std::isnan(lower[b]);
    return na != nb ? nb : (!na && lower[a] < lower[b]);
  });
  int best = -1, pos = 0, batch = 16;
  while (e == cudaSuccess && pos < NC && (best < 0 || !(lower[order[pos]] > full[best]))) {
    const int nb = std::min(batch, NC - pos);
    batch = std::min(2 * batch, BATCH);
    std::vector<double> part(nb);
    e = cudaMemcpyAsync(d_cand, order.data() + pos, nb * sizeof(int), cudaMemcpyHostToDevice, s);
    const double stop = best < 0 ? INFINITY : full[best];
    if (e == cudaSuccess) e = launch_fit_search(mu_fit, M, r_lo, r_hi, 1, nullptr, 0, d_cand, nb, stop, d_err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), d_err, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int q = 0; q < nb && e == cudaSuccess; ++q) {
      const int c = order[pos + q];
      full[c] = part[q];
      if (best < 0 || part[q] < full[best] || (part[q] == full[best] && c < best)) best = c;
    }
    pos += nb;
  }
  cudaFreeAsync(d_err, s);
  cudaFreeAsync(d_cand, s);
  const cudaError_t ef = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return fail(MRA_ERR_CUDA, "fit search: %s", cudaGetErrorString(e));
  op->h_fit = (5.0 + best / 113) / 100.0;
  op->s_lo = (best % 113 - 100.0) / 4.0;
  op->fit_err = full[best];
  if (!std::isfinite(op->fit_err)) return fail(MRA_ERR_NUMERIC, "fit search produced a non-finite error");
  op->c.resize(M);
  op->t.resize(M);
  const double pi = 3.14159265358979323846264338327950288;
  for (int m = 0; m < M; ++m) {
    double sm = op->s_lo + m * op->h_fit;
    op->c[m] = 2.0 / sqrt(pi) * op->h_fit * exp(sm - mu_fit * mu_fit * exp(-2.0 * sm) / 4.0);
    op->t[m] = exp(2.0 * sm);
  }
  return MRA_OK;
}

}  // namespace mra

using namespace mra;

extern "C" {

const char *mra_last_error(void) { return g_err; }

const char *mra_version(void) { return "mra-gb300 0.1 (sm_103a)"; }

int64_t mra_abi_sizeof(const char *name) {
  if (!name) return -1;
  const std::string n(name);
  if (n == "mra_gauss_sum") return (int64_t)sizeof(mra_gauss_sum);
  if (n == "mra_tree_view") return (int64_t)sizeof(mra_tree_view);
  if (n == "mra_apply_opts") return (int64_t)sizeof(mra_apply_opts);
  if (n == "mra_apply_stats") return (int64_t)sizeof(mra_apply_stats);
  if (n == "mra_compare_result") return (int64_t)sizeof(mra_compare_result);
  return -1;
}

long long mra_launch_count(void) { return mra::g_launches.load(std::memory_order_relaxed); }

int mra_release_memory(void) {
  std::lock_guard<std::mutex> lock(mra::g_pool_mu);
  for (int d = 0; d < mra::MAX_POOL_DEVICES; ++d) {
    if (!mra::g_pools[d]) continue;
    const cudaError_t e = cudaMemPoolTrimTo(mra::g_pools[d], 0);
    if (e != cudaSuccess) return fail(MRA_ERR_CUDA, "mra_release_memory: %s", cudaGetErrorString(e));
  }
  return MRA_OK;
}

int mra_debug_status(int *line, void *stream) {
  if (!line) return fail(MRA_ERR_ARG, "mra_debug_status: NULL line");
  cudaStream_t s = (cudaStream_t)stream;
  const int a = debug_line_apply(s), b = debug_line_split(s), c = debug_line_src(s);
  if (a < 0 || b < 0 || c < 0) return fail(MRA_ERR_CUDA, "mra_debug_status: reading the check words failed");
  *line = a ? a : (b ? b : c);
  return MRA_OK;
}

int mra_debug_selftest(void *stream) { return debug_selftest_run((cudaStream_t)stream); }

int mra_operator_create(int kernel, double mu, int M, double fit_eps, double r_lo, double r_hi,
                        int k, double L, int min_level, int max_level, int max_disp,
                        mra_operator **out, void *stream) {
  if (!out) return fail(MRA_ERR_ARG, "mra_operator_create: out is NULL");
  *out = nullptr;
  if (kernel != MRA_POISSON && kernel != MRA_BSH)
    return fail(MRA_ERR_ARG, "mra_operator_create: unknown kernel %d", kernel);
  if (kernel == MRA_BSH && !(mu > 0.0)) return fail(MRA_ERR_ARG, "mra_operator_create: BSH needs mu > 0");
  if (M < 1 || M > MRA_MAX_TERMS) return fail(MRA_ERR_ARG, "mra_operator_create: M=%d outside 1..%d", M, MRA_MAX_TERMS);
  if (k < 1 || k > MRA_MAX_K) return fail(MRA_ERR_ARG, "mra_operator_create: k=%d outside 1..%d", k, MRA_MAX_K);
  if (!(L > 0.0)) return fail(MRA_ERR_ARG, "mra_operator_create: L must be > 0");
  if (min_level < 0 || max_level > MRA_MAX_LEVEL || min_level > max_level)
    return fail(MRA_ERR_ARG, "mra_operator_create: levels %d..%d invalid", min_level, max_level);
  if (max_disp < 0 || max_disp > 127) return fail(MRA_ERR_ARG, "mra_operator_create: max_disp outside 0..127");
  if (!(r_lo > 0.0)) return fail(MRA_ERR_ARG, "mra_operator_create: r_lo must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  const bool r_hi_auto = !(r_hi > 0.0);
  if (r_hi_auto) {
    r_hi = 2.0 * L;
    if (kernel == MRA_BSH) {
      if (!(fit_eps > 0.0 && fit_eps < 1.0)) return fail(MRA_ERR_ARG, "mra_operator_create: fit_eps in (0,1) needed");
      r_hi = std::min(r_hi, log(1.0 / fit_eps) / mu);
    }
  }
  if (!(r_hi > r_lo)) return fail(MRA_ERR_ARG, "mra_operator_create: empty fit range");
  double mu_fit = kernel == MRA_BSH ? mu : 0.0;
  Operator *op = new Operator();
  op->kernel = kernel;
  op->mu = mu_fit;
  op->M = M;
  op->k = k;
  op->L = L;
  op->min_level = min_level;
  op->max_level = max_level;
  op->max_disp = max_disp;
  op->r_lo = r_lo;
  op->r_hi = r_hi;
  op->r_hi_auto = r_hi_auto;
  op->fit_eps = fit_eps;
  auto bail = [&](int code) { free_operator(op); return code; };
  // ---- fit: grid search on the device, argmin on the host (first strict minimum)
  {
    const int rcf = fit_operator(op, mu_fit, M, r_lo, r_hi, s);
    if (rcf != MRA_OK) return bail(rcf);
  }
  // ---- block table layout
  std::vector<int> Dabs(20, 0);
  std::vector<int64_t> off_abs(20, -1);
  int64_t nb = 0;
  for (int n = min_level; n <= max_level; ++n) {
    int64_t maxl = (1LL << n) - 1;
    int D = (int)std::min<int64_t>(max_disp, maxl);
    Dabs[n] = D;
    off_abs[n] = nb;
    nb += (int64_t)M * (2 * D + 1);
  }
  op->n_blocks = nb;
  size_t kk = (size_t)k * k;
  if (cudaMalloc((void **)&op->d_c, M * 8) != cudaSuccess ||
      cudaMalloc((void **)&op->d_t, M * 8) != cudaSuccess ||
      cudaMalloc((void **)&op->d_R, nb * kk * 8) != cudaSuccess ||
      cudaMalloc((void **)&op->d_N, nb * 8) != cudaSuccess ||
      cudaMalloc((void **)&op->d_D, 20 * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&op->d_level_off, 20 * sizeof(int64_t)) != cudaSuccess)
    return bail(fail(MRA_ERR_CUDA, "mra_operator_create: cudaMalloc failed"));
  double *d_gl = nullptr;
  std::vector<double> glx(k + 1), glw(k + 1);
  gauss_legendre(k + 1, glx.data(), glw.data());
  cudaError_t e = cudaMalloc((void **)&d_gl, 2 * (k + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(op->d_c, op->c.data(), M * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(op->d_t, op->t.data(), M * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(op->d_D, Dabs.data(), 20 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(op->d_level_off, off_abs.data(), 20 * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_gl, glx.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_gl + k + 1, glw.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s);
  for (int n = min_level; n <= max_level; ++n) {
    op->D.push_back(Dabs[n]);
    op->level_off.push_back(off_abs[n]);
  }
  if (e == cudaSuccess) e = launch_blocks(*op, d_gl, d_gl + k + 1, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_gl);
  if (e != cudaSuccess) return bail(fail(MRA_ERR_CUDA, "operator blocks: %s", cudaGetErrorString(e)));
  {
    int rc = split_blocks_build(*op, s);  // BF16 pieces of every block for the tensor-core path
    if (rc != MRA_OK) return bail(rc);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(MRA_ERR_CUDA, "split blocks: %s", cudaGetErrorString(e)));
  }
  *out = reinterpret_cast<mra_operator *>(op);
  return MRA_OK;
}

int mra_operator_blocks(int kernel, double mu, int M, double fit_eps, double r_lo, double r_hi,
                        int k, double L, int min_level, int max_level, int max_disp,
                        mra_operator **out, void *stream) {
  return mra_operator_create(kernel, mu, M, fit_eps, r_lo, r_hi, k, L, min_level, max_level, max_disp, out, stream);
}

int mra_operator_refit(mra_operator *h, double mu, int *blocks_reused, void *stream) {
  Operator *op = reinterpret_cast<Operator *>(h);
  if (!op) return fail(MRA_ERR_ARG, "mra_operator_refit: NULL operator");
  if (op->kernel != MRA_BSH) return fail(MRA_ERR_ARG, "mra_operator_refit: only the BSH kernel depends on mu");
  if (op->non_standard)
    return fail(MRA_ERR_ARG, "mra_operator_refit: refit the operator it was made from and create it again");
  if (!(mu > 0.0)) return fail(MRA_ERR_ARG, "mra_operator_refit: mu must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  const double r_hi = op->r_hi_auto ? std::min(2.0 * op->L, log(1.0 / op->fit_eps) / mu) : op->r_hi;
  if (!(r_hi > op->r_lo)) return fail(MRA_ERR_ARG, "mra_operator_refit: empty fit range");
  Operator fitted;
  const int rc = fit_operator(&fitted, mu, op->M, op->r_lo, r_hi, s);
  if (rc != MRA_OK) return rc;
  // the exponents t_m depend on (h, s_lo) only: equal grid points give the same blocks
  const bool same = fitted.h_fit == op->h_fit && fitted.s_lo == op->s_lo;
  op->mu = mu;
  op->r_hi = r_hi;
  op->h_fit = fitted.h_fit;
  op->s_lo = fitted.s_lo;
  op->fit_err = fitted.fit_err;
  op->c = fitted.c;
  op->t = fitted.t;
  MRA_CUDA_TRY(cudaMemcpyAsync(op->d_c, op->c.data(), op->M * 8, cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(op->d_t, op->t.data(), op->M * 8, cudaMemcpyHostToDevice, s));
  if (!same) {
    const int k = op->k;
    double *d_gl = nullptr;
    std::vector<double> glx(k + 1), glw(k + 1);
    gauss_legendre(k + 1, glx.data(), glw.data());
    cudaError_t e = cudaMalloc((void **)&d_gl, 2 * (k + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_gl, glx.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_gl + k + 1, glw.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_blocks(*op, d_gl, d_gl + k + 1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_gl);
    if (e != cudaSuccess) return fail(MRA_ERR_CUDA, "operator blocks: %s", cudaGetErrorString(e));
  }
  const int rc2 = split_blocks_build(*op, s, true);  // the c_m-scaled pieces change with c_m
  if (rc2 != MRA_OK) return rc2;
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (blocks_reused) *blocks_reused = same ? 1 : 0;
  return MRA_OK;
}

int mra_operator_fit(const mra_operator *h, double *c, double *t, double *hf, double *s_lo,
                     double *max_rel_err) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  if (!op) return fail(MRA_ERR_ARG, "mra_operator_fit: NULL operator");
  if (c) memcpy(c, op->c.data(), op->M * 8);
  if (t) memcpy(t, op->t.data(), op->M * 8);
  if (hf) *hf = op->h_fit;
  if (s_lo) *s_lo = op->s_lo;
  if (max_rel_err) *max_rel_err = op->fit_err;
  return MRA_OK;
}

int mra_operator_info(const mra_operator *h, int *k, int *M, int *min_level, int *max_level,
                      int *max_disp, double *L) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  if (!op) return fail(MRA_ERR_ARG, "mra_operator_info: NULL operator");
  if (k) *k = op->k;
  if (M) *M = op->M;
  if (min_level) *min_level = op->min_level;
  if (max_level) *max_level = op->max_level;
  if (max_disp) *max_disp = op->max_disp;
  if (L) *L = op->L;
  return MRA_OK;
}

int mra_operator_block(const mra_operator *h, int level, int m, int l, double *R, double *norm) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  if (!op) return fail(MRA_ERR_ARG, "mra_operator_block: NULL operator");
  if (level < op->min_level || level > op->max_level || m < 0 || m >= op->M)
    return fail(MRA_ERR_ARG, "mra_operator_block: (level %d, term %d) not in the table", level, m);
  int D = op->D[level - op->min_level];
  if (l < -D || l > D) return fail(MRA_ERR_ARG, "mra_operator_block: |l|=%d > %d", l < 0 ? -l : l, D);
  int64_t blk = op->level_off[level - op->min_level] + (int64_t)m * (2 * D + 1) + (l + D);
  size_t kk = (size_t)op->k * op->k;
  if (R) MRA_CUDA_TRY(cudaMemcpy(R, op->d_R + blk * kk, kk * 8, cudaMemcpyDeviceToHost));
  if (norm) MRA_CUDA_TRY(cudaMemcpy(norm, op->d_N + blk, 8, cudaMemcpyDeviceToHost));
  return MRA_OK;
}

int mra_operator_free(mra_operator *h) {
  free_operator(reinterpret_cast<Operator *>(h));
  return MRA_OK;
}

int mra_project(const mra_gauss_sum *f, int k, double L, double thresh, int init_level,
                int max_level, int uniform_level, mra_tree_view *out, void *stream) {
  if (!f || !out) return fail(MRA_ERR_ARG, "mra_project: NULL argument");
  if (f->n < 0 || (f->n > 0 && (!f->coef || !f->expnt || !f->cx || !f->cy || !f->cz)))
    return fail(MRA_ERR_ARG, "mra_project: bad Gaussian sum");
  if (k < 1 || k > MRA_MAX_K) return fail(MRA_ERR_ARG, "mra_project: k=%d outside 1..%d", k, MRA_MAX_K);
  if (!(L > 0.0)) return fail(MRA_ERR_ARG, "mra_project: L must be > 0");
  for (int g = 0; g < f->n; ++g)
    if (!(f->expnt[g] > 0.0)) return fail(MRA_ERR_ARG, "mra_project: exponent %d must be > 0", g);
  cudaStream_t s = (cudaStream_t)stream;
  int ng = f->n;
  const int k3 = k * k * k;
  std::vector<double> hg(5 * (size_t)std::max(ng, 1));
  for (int g = 0; g < ng; ++g) {
    hg[g] = f->coef[g];
    hg[ng + g] = f->expnt[g];
    hg[2 * ng + g] = f->cx[g];
    hg[3 * ng + g] = f->cy[g];
    hg[4 * ng + g] = f->cz[g];
  }
  double *d_g = nullptr;
  MRA_CUDA_TRY(pool_malloc((void **)&d_g, hg.size() * 8, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(d_g, hg.data(), hg.size() * 8, cudaMemcpyHostToDevice, s));
  out->k = k;
  out->L = L;
  if (uniform_level >= 0) {
    if (uniform_level > 10) { cudaFreeAsync(d_g, s); return fail(MRA_ERR_ARG, "mra_project: uniform level > 10"); }
    int64_t nb = 1LL << uniform_level, total = nb * nb * nb;
    if (total > out->cap) {
      cudaFreeAsync(d_g, s);
      out->n = total;
      return fail(MRA_ERR_CAPACITY, "mra_project: %lld boxes needed, cap %lld", (long long)total, (long long)out->cap);
    }
    std::vector<uint64_t> keys(total);
    for (int64_t b = 0; b < total; ++b) keys[b] = make_key(uniform_level, b / (nb * nb), (b / nb) % nb, b % nb);
    MRA_CUDA_TRY(cudaMemcpyAsync(out->keys, keys.data(), total * 8, cudaMemcpyHostToDevice, s));
    MRA_CUDA_TRY(launch_project_boxes(ng, d_g, k, L, total, out->keys, out->coeffs, s));
    MRA_CUDA_TRY(cudaFreeAsync(d_g, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
    out->n = total;
    return MRA_OK;
  }
  if (init_level < 1 || max_level < init_level || max_level > MRA_MAX_LEVEL) {
    cudaFreeAsync(d_g, s);
    return fail(MRA_ERR_ARG, "mra_project: levels init=%d max=%d invalid", init_level, max_level);
  }
  // ---- adaptive refinement, one level of parents at a time, in chunks
  std::vector<double> U(2 * k * k);
  two_scale(k, U.data());
  double *d_U = nullptr;
  MRA_CUDA_TRY(pool_malloc((void **)&d_U, U.size() * 8, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(d_U, U.data(), U.size() * 8, cudaMemcpyHostToDevice, s));
  int pl = init_level - 1;
  std::vector<uint64_t> parents;
  {
    int64_t nb = 1LL << pl;
    for (int64_t b = 0; b < nb * nb * nb; ++b) parents.push_back(make_key(pl, b / (nb * nb), (b / nb) % nb, b % nb));
  }
  const int64_t CH = 8192;  // parents per chunk
  uint64_t *d_keys = nullptr;
  double *d_box = nullptr, *d_dn = nullptr;
  int64_t *d_from = nullptr;
  MRA_CUDA_TRY(pool_malloc((void **)&d_keys, CH * 9 * 8, s));
  MRA_CUDA_TRY(pool_malloc((void **)&d_box, (size_t)CH * 9 * k3 * 8, s));
  MRA_CUDA_TRY(pool_malloc((void **)&d_dn, CH * 8, s));
  MRA_CUDA_TRY(pool_malloc((void **)&d_from, CH * 8 * 8, s));
  // leaves accumulate in a growing device buffer
  int64_t leaf_cap = 1 << 14, n_leaf = 0;
  double *d_leaf = nullptr;
  MRA_CUDA_TRY(pool_malloc((void **)&d_leaf, (size_t)leaf_cap * k3 * 8, s));
  std::vector<uint64_t> leaf_keys;
  std::vector<double> dn(CH);
  std::vector<uint64_t> ck(CH * 9);
  std::vector<int64_t> from(CH * 8);
  int rc = MRA_OK;
  while (!parents.empty() && rc == MRA_OK) {
    std::vector<uint64_t> next;
    for (size_t p0 = 0; p0 < parents.size() && rc == MRA_OK; p0 += CH) {
      int64_t np = std::min<int64_t>(CH, (int64_t)parents.size() - (int64_t)p0);
      for (int64_t p = 0; p < np; ++p) {
        uint64_t key = parents[p0 + p];
        ck[p] = key;
        int n = key_level(key);
        int64_t x = key_x(key), y = key_y(key), z = key_z(key);
        for (int c = 0; c < 8; ++c)
          ck[np + 8 * p + c] = make_key(n + 1, 2 * x + ((c >> 2) & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c & 1));
      }
      MRA_CUDA_TRY(cudaMemcpyAsync(d_keys, ck.data(), np * 9 * 8, cudaMemcpyHostToDevice, s));
      MRA_CUDA_TRY(launch_project_boxes(ng, d_g, k, L, np * 9, d_keys, d_box, s));
      MRA_CUDA_TRY(launch_refine_test(k, np, d_box, d_box + (size_t)np * k3, d_U, d_dn, s));
      MRA_CUDA_TRY(cudaMemcpyAsync(dn.data(), d_dn, np * 8, cudaMemcpyDeviceToHost, s));
      MRA_CUDA_TRY(cudaStreamSynchronize(s));
      int64_t nf = 0;
      for (int64_t p = 0; p < np; ++p) {
        int n = key_level(ck[p]);
        bool forced = (n + 1 >= max_level);
        if (!std::isfinite(dn[p])) { rc = fail(MRA_ERR_NUMERIC, "mra_project: non-finite refinement norm"); break; }
        bool refine = !forced && dn[p] > thresh;
        for (int c = 0; c < 8; ++c) {
          if (refine) next.push_back(ck[np + 8 * p + c]);
          else {
            leaf_keys.push_back(ck[np + 8 * p + c]);
            from[nf++] = np + 8 * p + c;
          }
        }
      }
      if (rc != MRA_OK || nf == 0) continue;
      if (n_leaf + nf > leaf_cap) {
        int64_t nc = std::max(leaf_cap * 2, n_leaf + nf);
        double *grown = nullptr;
        MRA_CUDA_TRY(pool_malloc((void **)&grown, (size_t)nc * k3 * 8, s));
        MRA_CUDA_TRY(cudaMemcpyAsync(grown, d_leaf, (size_t)n_leaf * k3 * 8, cudaMemcpyDeviceToDevice, s));
        MRA_CUDA_TRY(cudaFreeAsync(d_leaf, s));
        d_leaf = grown;
        leaf_cap = nc;
      }
      MRA_CUDA_TRY(cudaMemcpyAsync(d_from, from.data(), nf * 8, cudaMemcpyHostToDevice, s));
      gather_rows_kernel<<<counted((unsigned)nf), 128, 0, s>>>(nf, k3, d_box, d_from, d_leaf, n_leaf);
      MRA_CUDA_TRY(cudaGetLastError());
      n_leaf += nf;
      MRA_CUDA_TRY(cudaStreamSynchronize(s));  // ck/from are reused by the next chunk
    }
    parents.swap(next);
  }
  if (rc == MRA_OK && n_leaf > out->cap) {
    out->n = n_leaf;
    rc = fail(MRA_ERR_CAPACITY, "mra_project: %lld boxes needed, cap %lld", (long long)n_leaf, (long long)out->cap);
  }
  if (rc == MRA_OK && n_leaf > 0) {
    // sort leaves by key: permutation via radix sort, then gather rows
    uint64_t *d_lk = nullptr;
    int *d_pi = nullptr, *d_po = nullptr;
    void *tmp = nullptr;
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, (uint64_t *)nullptr, (uint64_t *)nullptr, (int *)nullptr,
                                    (int *)nullptr, (int)n_leaf);
    MRA_CUDA_TRY(pool_malloc((void **)&d_lk, n_leaf * 8, s));
    MRA_CUDA_TRY(pool_malloc((void **)&d_pi, n_leaf * 4, s));
    MRA_CUDA_TRY(pool_malloc((void **)&d_po, n_leaf * 4, s));
    MRA_CUDA_TRY(pool_malloc(&tmp, tb, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(d_lk, leaf_keys.data(), n_leaf * 8, cudaMemcpyHostToDevice, s));
    iota32<<<counted((unsigned)((n_leaf + 255) / 256)), 256, 0, s>>>(n_leaf, d_pi);
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, d_lk, out->keys, d_pi, d_po, (int)n_leaf, 0, 64, s));
    gather_sorted_kernel<<<counted((unsigned)n_leaf), 128, 0, s>>>(n_leaf, k3, d_leaf, d_po, out->coeffs);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cudaFreeAsync(d_lk, s));
    MRA_CUDA_TRY(cudaFreeAsync(d_pi, s));
    MRA_CUDA_TRY(cudaFreeAsync(d_po, s));
    MRA_CUDA_TRY(cudaFreeAsync(tmp, s));
    out->n = n_leaf;
  }
  cudaFreeAsync(d_keys, s);
  cudaFreeAsync(d_box, s);
  cudaFreeAsync(d_dn, s);
  cudaFreeAsync(d_from, s);
  cudaFreeAsync(d_leaf, s);
  cudaFreeAsync(d_U, s);
  cudaFreeAsync(d_g, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == MRA_OK && e != cudaSuccess) rc = fail(MRA_ERR_CUDA, "mra_project: %s", cudaGetErrorString(e));
  return rc;
}

static int check_view(const mra_tree_view *v, const char *what, bool need_data) {
  if (!v) return fail(MRA_ERR_ARG, "%s: NULL tree view", what);
  if (v->n < 0 || v->cap < 0 || v->n > v->cap) return fail(MRA_ERR_ARG, "%s: bad n/cap", what);
  if (need_data && v->n > 0 && (!v->keys || !v->coeffs)) return fail(MRA_ERR_ARG, "%s: NULL buffers", what);
  if (v->k < 1 || v->k > MRA_MAX_K) return fail(MRA_ERR_ARG, "%s: k=%d invalid", what, v->k);
  return MRA_OK;
}

static int check_opts(const Operator *op, const mra_tree_view *in, const mra_apply_opts *o) {
  if (!op) return fail(MRA_ERR_ARG, "mra_apply: NULL operator");
  if (!o) return fail(MRA_ERR_ARG, "mra_apply: NULL options");
  int rc = check_view(in, "mra_apply(in)", true);
  if (rc) return rc;
  if (in->k != op->k) return fail(MRA_ERR_ARG, "mra_apply: tree k=%d, operator k=%d", in->k, op->k);
  if (in->L != op->L) return fail(MRA_ERR_ARG, "mra_apply: tree L differs from operator L");
  if (o->precision != MRA_PREC_FP64 && o->precision != MRA_PREC_SPLIT_BF16)
    return fail(MRA_ERR_ARG, "mra_apply: unknown precision %d", o->precision);
  if (o->screen != MRA_SCREEN_NONE && o->screen != MRA_SCREEN_NORM && o->screen != MRA_SCREEN_LEARNED)
    return fail(MRA_ERR_ARG, "mra_apply: unknown screen %d", o->screen);
  if (o->screen == MRA_SCREEN_LEARNED && (!o->mlp || !(o->tau > 0.0)))
    return fail(MRA_ERR_ARG, "mra_apply: the learned screen needs a model and tau > 0");
  if (o->stencil != MRA_STENCIL_SHELLS && o->stencil != MRA_STENCIL_NEAREST)
    return fail(MRA_ERR_ARG, "mra_apply: unknown stencil %d", o->stencil);
  if (o->stencil == MRA_STENCIL_SHELLS && (o->max_disp < 0 || o->max_disp > op->max_disp))
    return fail(MRA_ERR_ARG, "mra_apply: max_disp %d outside 0..%d", o->max_disp, op->max_disp);
  if (o->stencil == MRA_STENCIL_NEAREST && op->max_disp < 1)
    return fail(MRA_ERR_ARG, "mra_apply: nearest stencil needs an operator with max_disp >= 1");
  if (o->screen != MRA_SCREEN_NONE && !(o->tau >= 0.0)) return fail(MRA_ERR_ARG, "mra_apply: tau must be >= 0");
  if (o->precision == MRA_PREC_SPLIT_BF16 && (o->pieces < 2 || o->pieces > 3))
    return fail(MRA_ERR_ARG, "mra_apply: pieces must be 2 or 3");
  if (o->dest_hi != 0 && o->dest_lo >= o->dest_hi)
    return fail(MRA_ERR_ARG, "mra_apply: empty destination range");
  return MRA_OK;
}

int mra_apply_workspace_size(const mra_operator *h, const mra_tree_view *in, const mra_apply_opts *o,
                             size_t *bytes) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  int rc = check_opts(op, in, o);
  if (rc) return rc;
  if (!bytes) return fail(MRA_ERR_ARG, "mra_apply_workspace_size: NULL bytes");
  *bytes = apply_workspace_bytes(*op, *o, in->n);
  return MRA_OK;
}

int mra_apply(const mra_operator *h, const mra_tree_view *in, const mra_apply_opts *o,
              mra_tree_view *out, void *workspace, size_t workspace_bytes, mra_apply_stats *stats,
              void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  int rc = check_opts(op, in, o);
  if (rc) return rc;
  rc = check_view(out, "mra_apply(out)", false);
  if (rc) return rc;
  if (out->k != op->k) return fail(MRA_ERR_ARG, "mra_apply: output k=%d, operator k=%d", out->k, op->k);
  if (in->n > 0 && !workspace) return fail(MRA_ERR_ARG, "mra_apply: NULL workspace");
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_apply: more than 2^31 source boxes");
  out->L = op->L;
  return apply_run(*op, *in, *o, *out, workspace, workspace_bytes, stats, (cudaStream_t)stream);
}

int mra_apply_host(const mra_operator *h, const mra_tree_view *in, const mra_apply_opts *o, mra_tree_view *out,
                   mra_apply_stats *stats, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  int rc = check_opts(op, in, o);
  if (rc) return rc;
  rc = check_view(out, "mra_apply_host(out)", false);
  if (rc) return rc;
  if (out->k != op->k) return fail(MRA_ERR_ARG, "mra_apply_host: output k=%d, operator k=%d", out->k, op->k);
  if (out->cap > 0 && (!out->keys || !out->coeffs)) return fail(MRA_ERR_ARG, "mra_apply_host: NULL output buffers");
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_apply_host: more than 2^31 source boxes");
  out->L = op->L;
  if (in->n == 0) {
    out->n = 0;
    if (stats) *stats = mra_apply_stats{};
    return MRA_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = in->n, cap = out->cap, k3 = (int64_t)op->k * op->k * op->k;
  const size_t wb = apply_workspace_bytes(*op, *o, n);
  void *d_ik = nullptr, *d_ic = nullptr, *d_ok = nullptr, *d_oc = nullptr, *ws = nullptr;
  cudaError_t e = pool_malloc(&d_ik, (size_t)n * 8, s);
  if (e == cudaSuccess) e = pool_malloc(&d_ic, (size_t)(n * k3) * 8, s);
  if (e == cudaSuccess) e = pool_malloc(&d_ok, (size_t)std::max<int64_t>(cap, 1) * 8, s);
  if (e == cudaSuccess) e = pool_malloc(&d_oc, (size_t)(std::max<int64_t>(cap, 1) * k3) * 8, s);
  if (e == cudaSuccess) e = pool_malloc(&ws, wb, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ik, in->keys, (size_t)n * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ic, in->coeffs, (size_t)(n * k3) * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    mra_tree_view din{n, n, (uint64_t *)d_ik, (double *)d_ic, op->k, op->L};
    mra_tree_view dout{0, cap, (uint64_t *)d_ok, (double *)d_oc, op->k, op->L};
    rc = apply_run(*op, din, *o, dout, ws, wb, stats, s);
    out->n = dout.n;
    if (rc == MRA_OK && dout.n > 0) {
      e = cudaMemcpyAsync(out->keys, d_ok, (size_t)dout.n * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out->coeffs, d_oc, (size_t)(dout.n * k3) * 8, cudaMemcpyDeviceToHost, s);
    }
  }
  for (void *p : {d_ik, d_ic, d_ok, d_oc, ws})
    if (p) cudaFreeAsync(p, s);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(MRA_ERR_CUDA, "mra_apply_host: %s", cudaGetErrorString(e));
  if (rc != MRA_OK) return rc;
  if (es != cudaSuccess) return fail(MRA_ERR_CUDA, "mra_apply_host: %s", cudaGetErrorString(es));
  return MRA_OK;
}

int mra_apply_batched(const mra_operator *h, int nfunc, const mra_tree_view *in, const int64_t *in_offsets,
                      const mra_apply_opts *o, mra_tree_view *out, int64_t *out_offsets, void *workspace,
                      size_t workspace_bytes, mra_apply_stats *stats, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  int rc = check_opts(op, in, o);
  if (rc) return rc;
  rc = check_view(out, "mra_apply_batched(out)", false);
  if (rc) return rc;
  if (nfunc < 1 || nfunc > MRA_MAX_FUNCS) return fail(MRA_ERR_ARG, "mra_apply_batched: nfunc=%d", nfunc);
  if (o->dest_hi != 0) return fail(MRA_ERR_ARG, "mra_apply_batched: no destination range with several functions");
  if (!in_offsets || !out_offsets) return fail(MRA_ERR_ARG, "mra_apply_batched: NULL offsets");
  if (in_offsets[0] != 0 || in_offsets[nfunc] != in->n)
    return fail(MRA_ERR_ARG, "mra_apply_batched: offsets must run from 0 to in->n");
  for (int f = 0; f < nfunc; ++f)
    if (in_offsets[f + 1] < in_offsets[f]) return fail(MRA_ERR_ARG, "mra_apply_batched: offsets decrease");
  if (out->k != op->k) return fail(MRA_ERR_ARG, "mra_apply_batched: output k differs");
  if (in->n > 0 && !workspace) return fail(MRA_ERR_ARG, "mra_apply_batched: NULL workspace");
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_apply_batched: more than 2^31 source boxes");
  out->L = op->L;
  return apply_run(*op, *in, *o, *out, workspace, workspace_bytes, stats, (cudaStream_t)stream, nfunc, in_offsets,
                   out_offsets);
}

int mra_log_terms(const mra_operator *h, const mra_tree_view *in, const mra_apply_opts *o, int64_t max_terms,
                  uint64_t seed, float *features, float *log_norms, int64_t *n_logged, void *workspace,
                  size_t workspace_bytes, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  int rc = check_opts(op, in, o);
  if (rc) return rc;
  if (!n_logged || max_terms < 0 || (max_terms > 0 && (!features || !log_norms)))
    return fail(MRA_ERR_ARG, "mra_log_terms: bad output arguments");
  if (in->n > 0 && !workspace) return fail(MRA_ERR_ARG, "mra_log_terms: NULL workspace");
  if (max_terms >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_log_terms: max_terms >= 2^31");
  return log_terms_run(*op, *in, *o, max_terms, seed, features, log_norms, n_logged, workspace,
                       workspace_bytes, (cudaStream_t)stream);
}

int mra_mlp_init(float *params, uint64_t seed, void *stream) {
  if (!params) return fail(MRA_ERR_ARG, "mra_mlp_init: NULL params");
  cudaStream_t s = (cudaStream_t)stream;
  MRA_CUDA_TRY(cudaMemsetAsync(params, 0, MLP_NALL * sizeof(float), s));
  MRA_CUDA_TRY(mlp_init(params, seed, s));
  const float ident[10] = {0, 0, 0, 0, 1, 1, 1, 1, 0, 1};
  MRA_CUDA_TRY(cudaMemcpyAsync(params + MLP_XMEAN, ident, sizeof(ident), cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  return MRA_OK;
}

int mra_mlp_standardize(float *params, const float *x, const float *y, int64_t n, void *stream) {
  if (!params || n < 1 || !x || !y) return fail(MRA_ERR_ARG, "mra_mlp_standardize: bad arguments");
  MRA_CUDA_TRY(mlp_fit_norm(params, x, y, n, (cudaStream_t)stream));
  return MRA_OK;
}

int mra_mlp_forward(const float *params, const float *x, int64_t n, float *out, void *stream) {
  if (!params || n < 0 || (n > 0 && (!x || !out))) return fail(MRA_ERR_ARG, "mra_mlp_forward: bad arguments");
  MRA_CUDA_TRY(mlp_forward(params, x, n, out, (cudaStream_t)stream));
  return MRA_OK;
}

static size_t mlp_ws(int64_t n) {
  size_t a = (mlp_grad_workspace(n) + 255) & ~(size_t)255;
  size_t b = ((size_t)n * 5 * sizeof(float) + 255) & ~(size_t)255;
  size_t c = ((size_t)MLP_NALL * sizeof(float) + 255) & ~(size_t)255;
  return a + b + c + 256;
}

int mra_mlp_workspace_size(int64_t n, size_t *bytes) {
  if (!bytes || n < 1) return fail(MRA_ERR_ARG, "mra_mlp_workspace_size: bad arguments");
  *bytes = mlp_ws(n);
  return MRA_OK;
}

int mra_mlp_grad(const float *params, const float *x, const float *y, int64_t n, float *grad, double *loss,
                 void *ws, size_t ws_bytes, void *stream) {
  if (!params || n < 1 || !x || !y || !grad || !ws) return fail(MRA_ERR_ARG, "mra_mlp_grad: bad arguments");
  if (ws_bytes < mlp_ws(n)) return fail(MRA_ERR_CAPACITY, "mra_mlp_grad: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)ws;
  size_t a = (mlp_grad_workspace(n) + 255) & ~(size_t)255;
  double *d_loss = (double *)(w + mlp_ws(n) - 256);
  MRA_CUDA_TRY(mlp_grad(params, x, y, n, grad, d_loss, w, s));
  (void)a;
  double h = 0.0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = h;
  return MRA_OK;
}

int mra_mlp_train(float *params, float *adam_state, const float *x, const float *y, int64_t n, int batch,
                  int steps, int step0, float lr, uint64_t seed, double *final_loss, void *ws, size_t ws_bytes,
                  void *stream) {
  if (!params || !adam_state || !x || !y || n < 1 || batch < 1 || steps < 0 || step0 < 0 || !(lr > 0.f) || !ws)
    return fail(MRA_ERR_ARG, "mra_mlp_train: bad arguments");
  if (ws_bytes < mlp_ws(batch)) return fail(MRA_ERR_CAPACITY, "mra_mlp_train: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)ws;
  size_t a = (mlp_grad_workspace(batch) + 255) & ~(size_t)255;
  float *bx = (float *)(w + a);
  float *by = bx + (size_t)batch * 4;
  size_t b = ((size_t)batch * 5 * sizeof(float) + 255) & ~(size_t)255;
  float *grad = (float *)(w + a + b);
  double *d_loss = (double *)(w + mlp_ws(batch) - 256);
  for (int st = 0; st < steps; ++st) {
    MRA_CUDA_TRY(mlp_gather_batch(x, y, n, batch, seed, step0 + st, bx, by, s));
    MRA_CUDA_TRY(mlp_grad(params, bx, by, batch, grad, d_loss, w, s));
    MRA_CUDA_TRY(mlp_adam(params, adam_state, adam_state + MLP_NALL, grad, lr, step0 + st + 1, s));
  }
  double h = 0.0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (final_loss) *final_loss = h;
  return MRA_OK;
}

int mra_norm(const mra_tree_view *t, double *per_box, double *total, void *stream) {
  int rc = check_view(t, "mra_norm", true);
  if (rc) return rc;
  return norm_run(*t, per_box, total, (cudaStream_t)stream);
}

int mra_compare(const mra_tree_view *test, const mra_tree_view *ref, mra_compare_result *res,
                void *stream) {
  int rc = check_view(test, "mra_compare(test)", true);
  if (rc) return rc;
  rc = check_view(ref, "mra_compare(ref)", true);
  if (rc) return rc;
  if (!res) return fail(MRA_ERR_ARG, "mra_compare: NULL result");
  return compare_run(*test, *ref, res, (cudaStream_t)stream);
}

}  // extern "C"
