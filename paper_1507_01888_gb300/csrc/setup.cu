// setup.cu -- set-up kernels: Gaussian-fit search, 1-D operator blocks, projection.
//
// Everything here is FP64 and runs once per operator or per input function;
// none of it is on the timed apply path.  Compiled with --fmad=false so that
// the fit search evaluates its error exactly as written.
#include <math.h>

#include "mra_internal.cuh"

namespace mra {

namespace {

constexpr int GLQ = 20;  // points per panel of the composite Gauss-Legendre rules
__constant__ double c_glx[GLQ], c_glw[GLQ];

__device__ __forceinline__ void legendre_phi(int k, double x01, double *out) {
  // phi_i(x) = sqrt(2i+1) P_i(2x-1), i < k (Sec. 2.1, eq. scalingfunc); zero outside [0,1]
  if (x01 < 0.0 || x01 > 1.0) {
    for (int i = 0; i < k; ++i) out[i] = 0.0;
    return;
  }
  double x = 2.0 * x01 - 1.0, p0 = 1.0, p1 = x;
  out[0] = 1.0;
  if (k > 1) out[1] = sqrt(3.0) * x;
  for (int m = 1; m + 1 < k; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - (double)m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
    out[m + 1] = sqrt(2.0 * m + 3.0) * p2;
  }
}

// --------------------------------------------------------------------------- fit search
// One CTA per candidate (h, s_lo) of the grid h = (5+i)/100, s_lo = (j-100)/4:
// max over the log-spaced points p = 0, stride, 2 stride, ... < 3000 (or, when `pts` is given,
// over the npts points pts[0..npts), npts <= blockDim) of
// |sum_m c_m exp(-t_m r_p^2) - K(r_p)| / K(r_p).  Over all points this is the candidate's
// error; over a subset it is a lower bound of it (a maximum over some of the same values).
// `cands` lists the candidates to evaluate (NULL: every candidate, in grid order).  A CTA
// stops early once its running maximum exceeds `stop` (a full error found already; +inf:
// never) and then writes that partial maximum, which exceeds `stop` too; errors at or below
// `stop` are exact.
constexpr int FIT_NS = 113, FIT_NP = 3000;  // s_lo values per h (116 h values), points

__global__ void fit_search_kernel(double mu, int M, double r_lo, double r_hi, int stride, const int *pts,
                                  int npts, const int *cands, double stop, double *err) {
  extern __shared__ double sh[];
  double *c = sh, *t = sh + M;
  __shared__ double red[32];
  const int cand = cands ? cands[blockIdx.x] : (int)blockIdx.x;
  int i = cand / FIT_NS, j = cand % FIT_NS;
  double h = (5.0 + i) / 100.0, s_lo = (j - 100.0) / 4.0;
  const double two_over_sqrtpi = 2.0 / sqrt(3.14159265358979323846264338327950288);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double s = s_lo + m * h;
    c[m] = two_over_sqrtpi * h * exp(s - mu * mu * exp(-2.0 * s) / 4.0);
    t[m] = exp(2.0 * s);
  }
  __syncthreads();
  double worst = 0.0;
  const int span = pts ? (int)blockDim.x : FIT_NP;
  for (int p0 = 0; p0 < span; p0 += blockDim.x * stride) {  // block-uniform trip count
    const int p = pts ? (threadIdx.x < npts ? pts[threadIdx.x] : FIT_NP) : p0 + threadIdx.x * stride;
    if (p < FIT_NP) {
      double r = r_lo * pow(r_hi / r_lo, (double)p / (double)(FIT_NP - 1));
      double K = exp(-mu * r) / r, sum = 0.0;
      for (int m = 0; m < M; ++m) sum += c[m] * exp(-t[m] * r * r);
      double e = fabs(sum - K) / K;
      worst = e > worst ? e : worst;
    }
    if (__syncthreads_or(worst > stop)) break;
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) w = fmax(w, red[q]);
    err[blockIdx.x] = w;
  }
}

// --------------------------------------------------------------------------- blocks
// R^n_{m,l}[i][j] = h int_{-1}^{1} exp(-T (z+l)^2) C_ij(z) dz,
//   C_ij(z) = int_{max(0,z)}^{min(1,1+z)} phi_i(u) phi_j(u-z) du  (exact: (k+1)-point GL),
// the cross-correlation form of h int int phi_i(u) exp(-T(u-v+l)^2) phi_j(v) du dv with z = u - v.
// The outer integral runs over w = z + l on the two halves z in [-1,0], [0,1]
// (C has a kink at z = 0), restricted to |w| <= sqrt(wmin^2 + 46/T) (the rest is
// below e^-46 of the maximum on that half), with uniform panels no wider than
// min(1/8, 1/(2 sqrt T), 1/(T wmin)) and 20-point Gauss-Legendre per panel.
struct HalfRange {
  double lo, hi;
  int npan;
};

__device__ HalfRange half_range(double T, double wa, double wb) {
  HalfRange r;
  double wmin = wa > 0.0 ? wa : (wb < 0.0 ? -wb : 0.0);
  r.lo = wa;
  r.hi = wb;
  double width = 0.125;
  if (T > 0.0) {
    double W = sqrt(wmin * wmin + 46.0 / T);
    if (-W > r.lo) r.lo = -W;
    if (W < r.hi) r.hi = W;
    width = fmin(width, 0.5 / sqrt(T));
    if (wmin > 0.0) width = fmin(width, 1.0 / (T * wmin));
  }
  if (r.hi <= r.lo) {
    r.npan = 0;
    return r;
  }
  double np = ceil((r.hi - r.lo) / width);
  r.npan = (int)fmin(np, 1024.0);
  return r;
}

constexpr int ZB = 8;  // z nodes per shared-memory round

__global__ void blocks_kernel(int k, double L, int min_level, int nlev, const int *Dlev,
                              const int64_t *level_off, const double *t, int M, const double *glxk,
                              const double *glwk, double *R, double *N) {
  extern __shared__ double sm[];
  // phi tables for ZB z-nodes: A[zb][q][i] = phi_i(u_q), B[zb][q][j] = phi_j(u_q - z)
  int kq = k + 1;
  double *A = sm;
  double *B = A + ZB * kq * k;
  double *wq = B + ZB * kq * k;  // [ZB][kq] quadrature weight (incl. Gaussian and Jacobians)
  __shared__ double red[32];
  int64_t blk = blockIdx.x;
  int lev = min_level;
  for (int q = 0; q < nlev; ++q)
    if (blk >= level_off[min_level + q]) lev = min_level + q;
  int D = Dlev[lev];
  int nl = 2 * D + 1;
  int64_t local = blk - level_off[lev];
  int m = (int)(local / nl);
  int l = (int)(local % nl) - D;
  double h = 2.0 * L / (double)(1LL << lev);
  double T = t[m] * h * h;
  HalfRange hr[2] = {half_range(T, -1.0 + l, 0.0 + l), half_range(T, 0.0 + l, 1.0 + l)};
  int n0 = hr[0].npan * GLQ, ntot = n0 + hr[1].npan * GLQ;
  int tid = threadIdx.x;
  int ii = tid / k, jj = tid % k;
  double acc = 0.0;
  for (int base = 0; base < ntot; base += ZB) {
    // build tables for nodes base..base+ZB-1
    for (int e = tid; e < ZB * kq; e += blockDim.x) {
      int zb = e / kq, q = e % kq;
      int node = base + zb;
      double wgt = 0.0, z = 0.0;
      if (node < ntot) {
        int half = node < n0 ? 0 : 1;
        int idx = half ? node - n0 : node;
        int p = idx / GLQ, g = idx % GLQ;
        const HalfRange &r = hr[half];
        double pw = (r.hi - r.lo) / r.npan;
        double w = r.lo + pw * (p + 0.5 + 0.5 * c_glx[g]);
        z = w - (double)l;
        double ua = z > 0.0 ? z : 0.0, ub = z < 0.0 ? 1.0 + z : 1.0;
        double u = ua + (ub - ua) * 0.5 * (glxk[q] + 1.0);
        wgt = 0.5 * pw * c_glw[g] * exp(-T * w * w) * 0.5 * (ub - ua) * glwk[q];
        legendre_phi(k, u, A + (zb * kq + q) * k);
        legendre_phi(k, u - z, B + (zb * kq + q) * k);
      } else {
        for (int i = 0; i < k; ++i) {
          A[(zb * kq + q) * k + i] = 0.0;
          B[(zb * kq + q) * k + i] = 0.0;
        }
      }
      wq[zb * kq + q] = wgt;
    }
    __syncthreads();
    if (tid < k * k) {
      for (int e = 0; e < ZB * kq; ++e) acc += wq[e] * A[e * k + ii] * B[e * k + jj];
    }
    __syncthreads();
  }
  double v = (tid < k * k) ? h * acc : 0.0;
  if (tid < k * k) R[blk * k * k + tid] = v;
  double s2 = v * v;
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((tid & 31) == 0) red[tid >> 5] = s2;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    N[blk] = sqrt(s);
  }
}

// --------------------------------------------------------------------------- projection
// s_b[ix][iy][iz] = sum_g coef_g h^{3/2} X_g[ix] Y_g[iy] Z_g[iz],
// X_g[i] = int_0^1 exp(-a_g h^2 (u - uc)^2) phi_i(u) du, uc = (c_g + L)/h - b_x  (eq. projection).
// One warp per (Gaussian, dimension) 1-D integral over the offset w = u - uc,
// with the same panel rule as the blocks; lanes stride over the nodes.
__global__ void project_kernel(int ng, const double *g, int k, double L, const uint64_t *keys,
                               double *out) {
  extern __shared__ double F[];  // [ng][3][k]
  uint64_t key = keys[blockIdx.x];
  int n = key_level(key);
  int64_t bxyz[3] = {key_x(key), key_y(key), key_z(key)};
  double h = 2.0 * L / (double)(1LL << n);
  const double *coef = g, *ex = g + ng;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int task = warp; task < 3 * ng; task += nw) {
    int gi = task / 3, d = task % 3;
    double cc = g[(2 + d) * ng + gi];
    double T = ex[gi] * h * h;
    double x = (cc + L) / h;               // uc = x - b
    double wa = (double)bxyz[d] - x;       // w at u = 0
    double wb = (double)(bxyz[d] + 1) - x; // w at u = 1
    HalfRange r = half_range(T, wa, wb);
    double acc[MRA_MAX_K];
    for (int i = 0; i < k; ++i) acc[i] = 0.0;
    int nn = r.npan * GLQ;
    double pw = r.npan > 0 ? (r.hi - r.lo) / r.npan : 0.0;
    double ph[MRA_MAX_K];
    for (int node = lane; node < nn; node += 32) {
      int p = node / GLQ, q = node % GLQ;
      double w = r.lo + pw * (p + 0.5 + 0.5 * c_glx[q]);
      double wt = 0.5 * pw * c_glw[q] * exp(-T * w * w);
      double u = w - wa;  // u = w + uc, formed from the box end
      legendre_phi(k, u, ph);
      for (int i = 0; i < k; ++i) acc[i] += wt * ph[i];
    }
    for (int i = 0; i < k; ++i) {
      double v = acc[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) F[(gi * 3 + d) * k + i] = v;
    }
  }
  __syncthreads();
  double h32 = h * sqrt(h);
  int k3 = k * k * k;
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    int ix = e / (k * k), iy = (e / k) % k, iz = e % k;
    double s = 0.0;
    for (int gi = 0; gi < ng; ++gi)
      s += coef[gi] * h32 * F[(gi * 3 + 0) * k + ix] * F[(gi * 3 + 1) * k + iy] *
           F[(gi * 3 + 2) * k + iz];
    out[(int64_t)blockIdx.x * k3 + e] = s;
  }
}

// --------------------------------------------------------------------------- refinement test
// For parent p: sum over its 8 children c of || s_c - (U^{cx} x U^{cy} x U^{cz}) s_p ||_F^2,
// with U^{(c)}[i][j] = 2^{-1/2} int_0^1 phi_i(y) phi_j((y+c)/2) dy (Sec. 2.2, P^{n+1} = P^n + Q^n).
__global__ void refine_test_kernel(int k, const double *parent, const double *child,
                                   const double *U, double *dnorm) {
  extern __shared__ double sm[];
  int k3 = k * k * k;
  double *sp = sm, *t1 = sp + k3, *t2 = t1 + k3;
  __shared__ double red[32];
  const double *ps = parent + (int64_t)blockIdx.x * k3;
  for (int e = threadIdx.x; e < k3; e += blockDim.x) sp[e] = ps[e];
  __syncthreads();
  double part = 0.0;
  for (int c = 0; c < 8; ++c) {
    const double *Ux = U + ((c >> 2) & 1) * k * k;
    const double *Uy = U + ((c >> 1) & 1) * k * k;
    const double *Uz = U + (c & 1) * k * k;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {
      int a = e / (k * k), b = (e / k) % k, cc = e % k;
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += Ux[a * k + j] * sp[(j * k + b) * k + cc];
      t1[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {
      int a = e / (k * k), b = (e / k) % k, cc = e % k;
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += Uy[b * k + j] * t1[(a * k + j) * k + cc];
      t2[e] = s;
    }
    __syncthreads();
    const double *cs = child + ((int64_t)blockIdx.x * 8 + c) * k3;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) {
      int a = e / (k * k), b = (e / k) % k, cc = e % k;
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += Uz[cc * k + j] * t2[(a * k + b) * k + j];
      double d = cs[e] - s;
      part += d * d;
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    dnorm[blockIdx.x] = sqrt(s);
  }
}

bool g_gl_uploaded = false;

cudaError_t upload_gl() {
  static double x[GLQ], w[GLQ];
  if (!g_gl_uploaded) {
    gauss_legendre(GLQ, x, w);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_glx, x, sizeof(x));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_glw, w, sizeof(w));
  g_gl_uploaded = true;
  return e;
}

}  // namespace

cudaError_t launch_fit_search(double mu, int M, double r_lo, double r_hi, int stride, const int *d_pts, int npts,
                              const int *d_cands, int n_cands, double stop, double *d_err, cudaStream_t s) {
  if (d_pts && (npts < 1 || npts > 256)) return cudaErrorInvalidValue;
  fit_search_kernel<<<counted((unsigned)n_cands), 256, 2 * M * sizeof(double), s>>>(
      mu, M, r_lo, r_hi, stride, d_pts, npts, d_cands, stop, d_err);
  return cudaGetLastError();
}

cudaError_t launch_blocks(const Operator &op, const double *d_glxk, const double *d_glwk,
                          cudaStream_t s) {
  cudaError_t e = upload_gl();
  if (e != cudaSuccess) return e;
  int kq = op.k + 1;
  size_t smem = (size_t)(2 * ZB * kq * op.k + ZB * kq) * sizeof(double);
  int threads = 256;
  int nlev = op.max_level - op.min_level + 1;
  blocks_kernel<<<counted((unsigned)op.n_blocks), threads, smem, s>>>(op.k, op.L, op.min_level, nlev, op.d_D,
                                                             op.d_level_off, op.d_t, op.M, d_glxk,
                                                             d_glwk, op.d_R, op.d_N);
  return cudaGetLastError();
}

cudaError_t launch_project_boxes(int ng, const double *d_g, int k, double L, int64_t nbox,
                                 const uint64_t *d_keys, double *d_out, cudaStream_t s) {
  if (nbox <= 0) return cudaSuccess;
  cudaError_t e = upload_gl();
  if (e != cudaSuccess) return e;
  size_t smem = (size_t)ng * 3 * k * sizeof(double);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  project_kernel<<<counted((unsigned)nbox), 256, smem, s>>>(ng, d_g, k, L, d_keys, d_out);
  return cudaGetLastError();
}

cudaError_t launch_refine_test(int k, int64_t nparent, const double *d_parent,
                               const double *d_child, const double *d_U, double *d_dnorm,
                               cudaStream_t s) {
  if (nparent <= 0) return cudaSuccess;
  size_t smem = (size_t)3 * k * k * k * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(refine_test_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  refine_test_kernel<<<counted((unsigned)nparent), 256, smem, s>>>(k, d_parent, d_child, d_U, d_dnorm);
  return cudaGetLastError();
}

}  // namespace mra
