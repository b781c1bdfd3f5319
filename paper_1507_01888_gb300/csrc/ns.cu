// ns.cu -- the operator in non-standard form and its apply on uniform trees (Sec. 2.2).
//
// With P^{n+1} = P^n + Q^n the level-N operator T^N = P^N T P^N splits into
//     T^N = T^{n0} + sum_{n=n0}^{N-1} (A^n + B^n + C^n),
// A^n = Q^n T Q^n, B^n = Q^n T P^n, C^n = P^n T Q^n.  On level n's 2k basis -- a box's
// children's k^3 coefficients side by side, S[(cx,i)][(cy,j)][(cz,l)] -- the level-(n+1)
// operator has the blocks
//     R2k^n_{m,l}[(ci,i)][(cj,j)] = R^{n+1}_{m, 2l+ci-cj}[i][j]
// and A^n + B^n + C^n = T2k^n - Ubar T^n Ubar^T with Ubar[(c,i)][j] = U^(c)[i][j].  Its
// blocks decay with the displacement (A as r^(-2k-1), B and C as r^(-k-1)), so a small
// displacement range per level reaches the operator's long range through the coarse levels.
//
// The apply (uniform level N, every box present):
//   compress   s^n = (Ubar^T)^{x3} S^n, S^n = children of level n, for n = N-1 .. n0;
//   coarsest   r^{n0} = T^{n0} s^{n0} with every displacement of level n0;
//   per level  Y^n = T2k^n S^n and Z^n = T^n s^n (the library's apply on level n's boxes,
//              |l|_inf <= max_disp, FP64 or split BF16), then
//              r^{n+1}(children of b) = (Ubar)^{x3} (r^n_b - Z^n_b) + Y^n_b;
// r^N is the result.  With every displacement it equals the plain level-N apply.
#include <algorithm>
#include <vector>

#include <cub/cub.cuh>

#include "apply_internal.cuh"

namespace mra {

namespace {

// ---------------------------------------------------------------- 2k blocks
// Blocks of one level of the non-standard operator from the level-(n+1) blocks of op.
__global__ void ns_blocks_kernel(int k, int M, int D, const double *Rop, int64_t op_base, int Dc,
                                 double *Rns, int64_t ns_base) {
  const int nl = 2 * D + 1, nlc = 2 * Dc + 1, kk = 2 * k;
  const int q = blockIdx.x;  // m * nl + (l + D)
  if (q >= M * nl) return;
  const int m = q / nl, l = q % nl - D;
  double *B = Rns + (ns_base + q) * (int64_t)kk * kk;
  for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
    const int I = e / kk, J = e % kk, ci = I / k, i = I % k, cj = J / k, j = J % k;
    const int lc = 2 * l + ci - cj;
    B[e] = Rop[(op_base + (int64_t)m * nlc + lc + Dc) * k * k + i * k + j];
  }
}

// Frobenius norm of every block (for the norm screen).
__global__ void block_norms_kernel(int64_t nblocks, int kk2, const double *R, double *N) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nblocks) return;
  double s = 0.0;
  for (int e = lane; e < kk2; e += 32) {
    const double v = R[b * kk2 + e];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) N[b] = sqrt(s);
}

// ---------------------------------------------------------------- uniform levels
// Keys of every box of level n in key order (x slowest): box i at (i / nb^2, i / nb % nb, i % nb).
__global__ void level_keys_kernel(int n, int64_t nbox, uint64_t *keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox) return;
  const int64_t nb = 1LL << n;
  keys[i] = make_key(n, i / (nb * nb), (i / nb) % nb, i % nb);
}

__global__ void check_uniform_kernel(int n, int64_t nbox, const uint64_t *keys, int *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbox) return;
  const int64_t nb = 1LL << n;
  if (keys[i] != make_key(n, i / (nb * nb), (i / nb) % nb, i % nb)) atomicExch(err, 1);
}

// Rows of an apply's output (keys of level n, any subset) into a zeroed dense level array.
__global__ void scatter_dense_kernel(int64_t n_rows, const uint64_t *keys, const double *rows, int rowlen,
                                     double *dense) {
  const int64_t r = blockIdx.x;
  if (r >= n_rows) return;
  const uint64_t key = keys[r];
  const int64_t nb = 1LL << key_level(key);
  const int64_t d = (key_x(key) * nb + key_y(key)) * nb + key_z(key);
  for (int e = threadIdx.x; e < rowlen; e += blockDim.x) dense[d * rowlen + e] = rows[r * rowlen + e];
}

// ---------------------------------------------------------------- two-scale transforms
// One CTA per box of level n: S = the children (dense level n+1) as a (2k)^3 tensor, written
// out, and s = (Ubar^T)^{x3} S.  Shared memory: S (2k)^3, a k (2k)^2, b k^2 (2k) doubles.
__global__ void compress_kernel(int k, int n, const double *fine, const double *Ub, double *S_out,
                                double *s_out) {
  extern __shared__ double sh[];
  const int kk = 2 * k, k3 = k * k * k, kk3 = kk * kk * kk;
  double *S = sh, *a = S + kk3, *b = a + k * kk * kk;
  const int64_t box = blockIdx.x, nb = 1LL << n, nf = 2 * nb;
  const int64_t x = box / (nb * nb), y = (box / nb) % nb, z = box % nb;
  for (int e = threadIdx.x; e < kk3; e += blockDim.x) {
    const int I = e / (kk * kk), J = (e / kk) % kk, Lq = e % kk;
    const int64_t child = ((2 * x + I / k) * nf + 2 * y + J / k) * nf + 2 * z + Lq / k;
    const double v = fine[child * k3 + ((I % k) * k + J % k) * k + Lq % k];
    S[e] = v;
    S_out[box * kk3 + e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * kk * kk; e += blockDim.x) {  // a[i][J][L] = sum_I Ub[I][i] S[I][J][L]
    const int i = e / (kk * kk), q = e % (kk * kk);
    double v = 0.0;
    for (int I = 0; I < kk; ++I) v += Ub[I * k + i] * S[I * kk * kk + q];
    a[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k * kk; e += blockDim.x) {  // b[i][j][L] = sum_J Ub[J][j] a[i][J][L]
    const int i = e / (k * kk), j = (e / kk) % k, Lq = e % kk;
    double v = 0.0;
    for (int J = 0; J < kk; ++J) v += Ub[J * k + j] * a[(i * kk + J) * kk + Lq];
    b[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // s[i][j][l] = sum_L Ub[L][l] b[i][j][L]
    const int q = e / k, l = e % k;
    double v = 0.0;
    for (int Lq = 0; Lq < kk; ++Lq) v += Ub[Lq * k + l] * b[q * kk + Lq];
    s_out[box * k3 + e] = v;
  }
}

// One CTA per box of level n: r^{n+1}(children) = (Ubar)^{x3} (r_b - Z_b) + Y_b, into the
// dense level n+1 array.  Shared memory: d k^3, a (2k) k^2, b (2k)^2 k doubles.
__global__ void sum_down_kernel(int k, int n, const double *r, const double *Z, const double *Y,
                                const double *Ub, double *fine) {
  extern __shared__ double sh[];
  const int kk = 2 * k, k2 = k * k, k3 = k2 * k, kk3 = kk * kk * kk;
  double *d = sh, *a = d + k3, *b = a + kk * k2;
  const int64_t box = blockIdx.x, nb = 1LL << n, nf = 2 * nb;
  const int64_t x = box / (nb * nb), y = (box / nb) % nb, z = box % nb;
  for (int e = threadIdx.x; e < k3; e += blockDim.x) d[e] = r[box * k3 + e] - Z[box * k3 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < kk * k2; e += blockDim.x) {  // a[I][j][l] = sum_i Ub[I][i] d[i][j][l]
    const int I = e / k2, q = e % k2;
    double v = 0.0;
    for (int i = 0; i < k; ++i) v += Ub[I * k + i] * d[i * k2 + q];
    a[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * kk * k; e += blockDim.x) {  // b[I][J][l] = sum_j Ub[J][j] a[I][j][l]
    const int I = e / (kk * k), J = (e / k) % kk, l = e % k;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Ub[J * k + j] * a[(I * k + j) * k + l];
    b[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk3; e += blockDim.x) {  // + sum_l Ub[L][l] b[I][J][l] + Y
    const int I = e / (kk * kk), J = (e / kk) % kk, Lq = e % kk;
    double v = Y[box * kk3 + e];
    for (int l = 0; l < k; ++l) v += Ub[Lq * k + l] * b[(I * kk + J) * k + l];
    const int64_t child = ((2 * x + I / k) * nf + 2 * y + J / k) * nf + 2 * z + Lq / k;
    fine[child * k3 + ((I % k) * k + J % k) * k + Lq % k] = v;
  }
}

// ---------------------------------------------------------------- adaptive trees
__device__ __forceinline__ int64_t find_sorted(const uint64_t *keys, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const uint64_t v = keys[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Leaf checks: keys strictly increasing, every leaf deeper than n0; deepest level -> *maxlev.
__global__ void leaf_check_kernel(int64_t n, const uint64_t *keys, int n0, int *err, int *maxlev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lv = key_level(keys[i]);
  if (lv <= n0 || (i > 0 && keys[i] <= keys[i - 1])) atomicExch(err, 1);
  atomicMax(maxlev, lv);
}

// Ancestor on level n of every leaf deeper than n (others: the largest key, dropped later).
// Entry (j, i): the level-(n0+j) ancestor of leaf i when the leaf is deeper, else the largest key.
__global__ void ancestor_kernel(int64_t n_leaf, const uint64_t *keys, int n0, int nlev, uint64_t *anc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_leaf * nlev) return;
  const int64_t i = e % n_leaf;
  const int n = n0 + (int)(e / n_leaf);
  const uint64_t k = keys[i];
  const int lv = key_level(k);
  anc[e] = lv > n ? make_key(n, key_x(k) >> (lv - n), key_y(k) >> (lv - n), key_z(k) >> (lv - n)) : ~0ull;
}

// One CTA per interior node of level n: its children (leaves or interior nodes of level n+1)
// as the (2k)^3 tensor S, and s = (Ubar^T)^{x3} S.  A missing child sets *err.
__global__ void compress_tree_kernel(int k, int n, const uint64_t *ikeys, int64_t n_int, const uint64_t *lkeys,
                                     const double *lcoeffs, int64_t n_leaf, const uint64_t *ckeys,
                                     const double *ccoeffs, int64_t n_child_int, const double *Ub, double *S_out,
                                     double *s_out, int *err) {
  extern __shared__ double sh[];
  __shared__ const double *src[8];
  const int kk = 2 * k, k3 = k * k * k, kk3 = kk * kk * kk;
  double *S = sh, *a = S + kk3, *b = a + k * kk * kk;
  const int64_t box = blockIdx.x;
  if (box >= n_int) return;
  const uint64_t key = ikeys[box];
  if (threadIdx.x < 8) {
    const int cx = threadIdx.x >> 2, cy = (threadIdx.x >> 1) & 1, cz = threadIdx.x & 1;
    const uint64_t ck = make_key(n + 1, 2 * key_x(key) + cx, 2 * key_y(key) + cy, 2 * key_z(key) + cz);
    const int64_t li = find_sorted(lkeys, n_leaf, ck);
    const double *p = nullptr;
    if (li >= 0) {
      p = lcoeffs + li * k3;
    } else {
      const int64_t ci = find_sorted(ckeys, n_child_int, ck);
      if (ci >= 0) p = ccoeffs + ci * k3;
    }
    if (!p) atomicExch(err, 2);
    src[threadIdx.x] = p;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk3; e += blockDim.x) {
    const int I = e / (kk * kk), J = (e / kk) % kk, Lq = e % kk;
    const double *p = src[((I / k) << 2) | ((J / k) << 1) | (Lq / k)];
    const double v = p ? p[((I % k) * k + J % k) * k + Lq % k] : 0.0;
    S[e] = v;
    S_out[box * kk3 + e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * kk * kk; e += blockDim.x) {
    const int i = e / (kk * kk), q = e % (kk * kk);
    double v = 0.0;
    for (int I = 0; I < kk; ++I) v += Ub[I * k + i] * S[I * kk * kk + q];
    a[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k * kk; e += blockDim.x) {
    const int i = e / (k * kk), j = (e / kk) % k, Lq = e % kk;
    double v = 0.0;
    for (int J = 0; J < kk; ++J) v += Ub[J * k + j] * a[(i * kk + J) * kk + Lq];
    b[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    const int q = e / k, l = e % k;
    double v = 0.0;
    for (int Lq = 0; Lq < kk; ++Lq) v += Ub[Lq * k + l] * b[q * kk + Lq];
    s_out[box * k3 + e] = v;
  }
}

// The halo of the level's sources: every in-cell box within |l|_inf <= D of one (others: the
// largest key, dropped later).
__global__ void halo_kernel(int64_t ni, const uint64_t *ikeys, int D, uint64_t *out) {
  const int w = 2 * D + 1, w3 = w * w * w;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ni * w3) return;
  const uint64_t k = ikeys[e / w3];
  const int l = (int)(e % w3), lx = l / (w * w) - D, ly = (l / w) % w - D, lz = l % w - D;
  const int n = key_level(k);
  const int64_t nb = 1LL << n, x = key_x(k) + lx, y = key_y(k) + ly, z = key_z(k) + lz;
  out[e] = (x < 0 || x >= nb || y < 0 || y >= nb || z < 0 || z >= nb) ? ~0ull : make_key(n, x, y, z);
}

// Every node p of R_n: refined when it lies in the sources' halo (every box an unscreened apply
// of the level would reach); its output rows of the level's two applies, if any.
// The halo's count *nh is read on the device (its last key may be the largest key, which no
// node has).
__global__ void reach_kernel(int64_t nr, const uint64_t *rkeys, const uint64_t *hkeys, const int64_t *nh,
                             const uint64_t *ykeys, int64_t ny, const uint64_t *zkeys, int64_t nz, int64_t *yi,
                             int64_t *zi, int *refine, int *leaf) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nr) return;
  yi[p] = find_sorted(ykeys, ny, rkeys[p]);
  zi[p] = find_sorted(zkeys, nz, rkeys[p]);
  const bool in = find_sorted(hkeys, *nh, rkeys[p]) >= 0;
  refine[p] = in ? 1 : 0;
  leaf[p] = in ? 0 : 1;
}

// Every target row of an apply must be a node of R_n.
__global__ void targets_in_kernel(int64_t nt, const uint64_t *tkeys, const uint64_t *rkeys, int64_t nr, int *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  if (find_sorted(rkeys, nr, tkeys[i]) < 0) atomicExch(err, 3);
}

// Result leaves of this level: nodes of R_n that no apply reached, appended at out + base.
__global__ void emit_leaves_kernel(int64_t nr, int k3, const uint64_t *rkeys, const double *r, const int *leaf,
                                   const int *leaf_pos, int64_t base, int64_t cap, uint64_t *okeys, double *ocoeffs) {
  const int64_t p = blockIdx.x;
  if (p >= nr || !leaf[p]) return;
  const int64_t o = base + leaf_pos[p];
  if (o >= cap) return;
  if (threadIdx.x == 0) okeys[o] = rkeys[p];
  for (int e = threadIdx.x; e < k3; e += blockDim.x) ocoeffs[o * k3 + e] = r[p * k3 + e];
}

// One CTA per reached node p: its children get (Ubar)^{x3} (r_p - Z_p) + Y_p (absent rows as
// zero), written at 8 ref_pos[p] + child in the unsorted level-(n+1) arrays.
__global__ void sum_down_tree_kernel(int k, int64_t nr, const uint64_t *rkeys, const double *r, const int *refine,
                                     const int *ref_pos, const int64_t *yi, const double *Y, const int64_t *zi,
                                     const double *Z, const double *Ub, uint64_t *ckeys, double *cr) {
  extern __shared__ double sh[];
  const int64_t p = blockIdx.x;
  if (p >= nr || !refine[p]) return;
  const int kk = 2 * k, k2 = k * k, k3 = k2 * k, kk3 = kk * kk * kk;
  double *d = sh, *a = d + k3, *b = a + kk * k2;
  const int64_t y = yi[p], z = zi[p], base = 8 * (int64_t)ref_pos[p];
  for (int e = threadIdx.x; e < k3; e += blockDim.x) d[e] = r[p * k3 + e] - (z >= 0 ? Z[z * k3 + e] : 0.0);
  const uint64_t key = rkeys[p];
  if (threadIdx.x < 8) {
    const int cx = threadIdx.x >> 2, cy = (threadIdx.x >> 1) & 1, cz = threadIdx.x & 1;
    ckeys[base + threadIdx.x] =
        make_key(key_level(key) + 1, 2 * key_x(key) + cx, 2 * key_y(key) + cy, 2 * key_z(key) + cz);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * k2; e += blockDim.x) {
    const int I = e / k2, q = e % k2;
    double v = 0.0;
    for (int i = 0; i < k; ++i) v += Ub[I * k + i] * d[i * k2 + q];
    a[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * kk * k; e += blockDim.x) {
    const int I = e / (kk * k), J = (e / k) % kk, l = e % k;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Ub[J * k + j] * a[(I * k + j) * k + l];
    b[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk3; e += blockDim.x) {
    const int I = e / (kk * kk), J = (e / kk) % kk, Lq = e % kk;
    double v = y >= 0 ? Y[y * kk3 + e] : 0.0;
    for (int l = 0; l < k; ++l) v += Ub[Lq * k + l] * b[(I * kk + J) * k + l];
    const int child = ((I / k) << 2) | ((J / k) << 1) | (Lq / k);
    cr[(base + child) * k3 + ((I % k) * k + J % k) * k + Lq % k] = v;
  }
}

__global__ void gather_rows_ns_kernel(int64_t n, int rowlen, const int *perm, const double *src, double *dst) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t from = perm[i];
  for (int e = threadIdx.x; e < rowlen; e += blockDim.x) dst[i * rowlen + e] = src[from * rowlen + e];
}

__global__ void iota_ns_kernel(int64_t n, int *v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (int)i;
}

// ---------------------------------------------------------------- reconstruct
// Level of the shallowest input box above box b or b itself (the input is sorted and unique).
__global__ void top_level_kernel(int64_t n, const uint64_t *keys, int *top) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const uint64_t k = keys[b];
  const int lv = key_level(k);
  int t = lv;
  for (int m = 0; m < lv; ++m)
    if (find_sorted(keys, n, make_key(m, key_x(k) >> (lv - m), key_y(k) >> (lv - m), key_z(k) >> (lv - m))) >= 0) {
      t = m;
      break;
    }
  top[b] = t;
}

// Interior boxes of levels n0 .. n0+nlev-1 at once: entry (j, b) is the level-(n0+j) ancestor of
// input box b when b is deeper and has an input box at or above that level on its path, else
// the largest key (dropped after the sort: its level field is beyond every level).
__global__ void interior_all_kernel(int64_t n_in, const uint64_t *keys, const int *top, int n0, int nlev,
                                    uint64_t *out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_in * nlev) return;
  const int64_t b = e % n_in;
  const int n = n0 + (int)(e / n_in);
  const uint64_t k = keys[b];
  const int lv = key_level(k);
  out[e] = (lv > n && top[b] <= n) ? make_key(n, key_x(k) >> (lv - n), key_y(k) >> (lv - n), key_z(k) >> (lv - n))
                                   : ~0ull;
}
// off[l] = first position of level l (0 <= l <= 20) in the sorted keys[0 .. *n)
__global__ void level_offsets_kernel(const uint64_t *keys, const int64_t *n, int64_t *off) {
  const int l = threadIdx.x;
  if (l > 20) return;
  const uint64_t x = (uint64_t)l << 57;
  int64_t a = 0, b = *n;
  while (a < b) {
    const int64_t m = (a + b) / 2;
    if (keys[m] < x) a = m + 1;
    else b = m;
  }
  off[l] = a;
}

// Input boxes of level n in [lo, hi): tops join the level's boxes (appended after `base`
// passed-down boxes, at their rank pos[b] - pos0 among the level's tops), the others add their
// coefficients to the passed-down box of the same key.
__global__ void tops_kernel(int64_t lo, int64_t hi, int n, const int *top, const uint64_t *keys, const double *coeffs,
                            int k3, const int *pos, int pos0, int64_t base, uint64_t *rkeys, double *rv) {
  const int64_t b = lo + blockIdx.x;
  if (b >= hi || top[b] != n) return;
  const int64_t o = base + (pos[b] - pos0);
  if (threadIdx.x == 0) rkeys[o] = keys[b];
  for (int e = threadIdx.x; e < k3; e += blockDim.x) rv[o * k3 + e] = coeffs[b * k3 + e];
}
// flag[b] = 1 for the input boxes that are tops (no input box above them), flag[n] = 0
__global__ void top_flags_kernel(int64_t n, const uint64_t *keys, const int *top, int *flag) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b > n) return;
  flag[b] = b < n && top[b] == key_level(keys[b]) ? 1 : 0;
}
// the level's interior boxes found among its boxes must be all of them (a consistent tree)
__global__ void inner_count_check_kernel(const int *ipos, int64_t nr, int64_t ni, int *err) {
  if (ipos[nr] != ni) atomicExch(err, 2);
}
__global__ void add_inputs_kernel(int64_t lo, int64_t hi, int n, const int *top, const uint64_t *keys,
                                  const double *coeffs, int k3, const uint64_t *rkeys, int64_t nr, double *rv,
                                  int *err) {
  const int64_t b = lo + blockIdx.x;
  if (b >= hi || top[b] == n) return;
  __shared__ int64_t p;
  if (threadIdx.x == 0) p = find_sorted(rkeys, nr, keys[b]);
  __syncthreads();
  if (p < 0) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  for (int e = threadIdx.x; e < k3; e += blockDim.x) rv[p * k3 + e] += coeffs[b * k3 + e];
}

// Is box p of the level interior (passes down) or a leaf of the result?
__global__ void classify_kernel(int64_t nr, const uint64_t *rkeys, const uint64_t *ikeys, int64_t ni, int *inner,
                                int *leaf) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nr) return;
  const bool in = find_sorted(ikeys, ni, rkeys[p]) >= 0;
  inner[p] = in ? 1 : 0;
  leaf[p] = in ? 0 : 1;
}

// One CTA per interior box: its eight children get Ubar^{x3} s (two-scale relation).
__global__ void pass_down_kernel(int k, int64_t nr, const uint64_t *rkeys, const double *rv, const int *inner,
                                 const int *pos, int64_t ninner, const double *Ub, uint64_t *ckeys, double *cv,
                                 int *err) {
  extern __shared__ double sh[];
  const int64_t p = blockIdx.x;
  if (p >= nr || !inner[p]) return;
  if (pos[p] >= ninner) {  // more interior boxes than the level has room for: inconsistent tree
    if (threadIdx.x == 0) atomicExch(err, 2);
    return;
  }
  const int kk = 2 * k, k2 = k * k, k3 = k2 * k, kk3 = kk * kk * kk;
  double *d = sh, *a = d + k3, *b = a + kk * k2;
  const int64_t base = 8 * (int64_t)pos[p];
  for (int e = threadIdx.x; e < k3; e += blockDim.x) d[e] = rv[p * k3 + e];
  const uint64_t key = rkeys[p];
  if (threadIdx.x < 8) {
    const int cx = threadIdx.x >> 2, cy = (threadIdx.x >> 1) & 1, cz = threadIdx.x & 1;
    ckeys[base + threadIdx.x] =
        make_key(key_level(key) + 1, 2 * key_x(key) + cx, 2 * key_y(key) + cy, 2 * key_z(key) + cz);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * k2; e += blockDim.x) {
    const int I = e / k2, q = e % k2;
    double v = 0.0;
    for (int i = 0; i < k; ++i) v += Ub[I * k + i] * d[i * k2 + q];
    a[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk * kk * k; e += blockDim.x) {
    const int I = e / (kk * k), J = (e / k) % kk, l = e % k;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Ub[J * k + j] * a[(I * k + j) * k + l];
    b[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk3; e += blockDim.x) {
    const int I = e / (kk * kk), J = (e / kk) % kk, Lq = e % kk;
    double v = 0.0;
    for (int l = 0; l < k; ++l) v += Ub[Lq * k + l] * b[(I * kk + J) * k + l];
    const int child = ((I / k) << 2) | ((J / k) << 1) | (Lq / k);
    cv[(base + child) * k3 + ((I % k) * k + J % k) * k + Lq % k] = v;
  }
}

// ---------------------------------------------------------------- truncate
// One CTA per leaf of level n (sorted keys): a leaf with even (x, y, z) whose seven siblings
// are leaves too forms S from the eight, s = (Ubar^T)^{x3} S and the detail
// d = S - Ubar^{x3} s; if ||d||_F <= thresh the eight are marked gone, the parent (key, s) is
// appended at an atomic slot of the level above and ||d||^2 is kept at the first child's slot.
// Shared memory: the filter's two intermediates (4k^3, 2k^3) and s (k^3), the unfilter's
// intermediates reusing the filter's; S itself (8k^3) is staged too when s_smem is set, and
// read from the children's rows otherwise (k > 12, where it does not fit).
__global__ void truncate_level_kernel(int k, int n, int64_t nl, const uint64_t *keys, const double *v, double thresh,
                                      const double *Ub, int *gone, double *d2, uint64_t *pkeys, double *pv,
                                      int *pcount, int s_smem) {
  extern __shared__ double sh[];
  __shared__ int64_t idx[8];
  __shared__ int all;
  __shared__ double red[8];
  const int64_t i = blockIdx.x;
  if (i >= nl) return;
  const uint64_t key = keys[i];
  const int64_t x = key_x(key), y = key_y(key), z = key_z(key);
  if ((x & 1) || (y & 1) || (z & 1)) return;
  const int kk = 2 * k, k3 = k * k * k, kk3 = kk * kk * kk;
  double *a = sh, *b = a + k * kk * kk, *sv = b + k * k * kk, *S = sv + k3;
  double *c = b, *e = a;  // the unfilter's intermediates (kk k^2 and kk^2 k) once a and b are consumed
  if (threadIdx.x == 0) all = 1;
  __syncthreads();
  if (threadIdx.x < 8) {
    const int cx = threadIdx.x >> 2, cy = (threadIdx.x >> 1) & 1, cz = threadIdx.x & 1;
    idx[threadIdx.x] = find_sorted(keys, nl, make_key(n, x + cx, y + cy, z + cz));
    if (idx[threadIdx.x] < 0) atomicExch(&all, 0);
  }
  __syncthreads();
  if (!all) return;
  // S[(I, J, L)] = child (I/k, J/k, L/k)'s coefficient (I%k, J%k, L%k)
  auto s_at = [&](int q) {
    const int I = q / (kk * kk), J = (q / kk) % kk, Lq = q % kk;
    const int64_t src = idx[((I / k) << 2) | ((J / k) << 1) | (Lq / k)];
    return v[src * k3 + ((I % k) * k + J % k) * k + Lq % k];
  };
  if (s_smem) {
    for (int q = threadIdx.x; q < kk3; q += blockDim.x) S[q] = s_at(q);
    __syncthreads();
  }
  for (int q = threadIdx.x; q < k * kk * kk; q += blockDim.x) {  // filter
    const int ii = q / (kk * kk), r = q % (kk * kk);
    double t = 0.0;
    for (int I = 0; I < kk; ++I) t += Ub[I * k + ii] * (s_smem ? S[I * kk * kk + r] : s_at(I * kk * kk + r));
    a[q] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k * k * kk; q += blockDim.x) {
    const int ii = q / (k * kk), j = (q / kk) % k, Lq = q % kk;
    double t = 0.0;
    for (int J = 0; J < kk; ++J) t += Ub[J * k + j] * a[(ii * kk + J) * kk + Lq];
    b[q] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k3; q += blockDim.x) {
    const int r = q / k, l = q % k;
    double t = 0.0;
    for (int Lq = 0; Lq < kk; ++Lq) t += Ub[Lq * k + l] * b[r * kk + Lq];
    sv[q] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kk * k * k; q += blockDim.x) {  // unfilter of s
    const int I = q / (k * k), r = q % (k * k);
    double t = 0.0;
    for (int ii = 0; ii < k; ++ii) t += Ub[I * k + ii] * sv[ii * k * k + r];
    c[q] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kk * kk * k; q += blockDim.x) {
    const int I = q / (kk * k), J = (q / k) % kk, l = q % k;
    double t = 0.0;
    for (int j = 0; j < k; ++j) t += Ub[J * k + j] * c[(I * k + j) * k + l];
    e[q] = t;
  }
  __syncthreads();
  double part = 0.0;
  for (int q = threadIdx.x; q < kk3; q += blockDim.x) {
    const int I = q / (kk * kk), J = (q / kk) % kk, Lq = q % kk;
    double t = 0.0;
    for (int l = 0; l < k; ++l) t += Ub[Lq * k + l] * e[(I * kk + J) * k + l];
    const double dd = (s_smem ? S[q] : s_at(q)) - t;
    part += dd * dd;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  __shared__ int slot;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const bool merge = sqrt(tot) <= thresh;
    slot = -1;
    if (merge) {
      for (int cc = 0; cc < 8; ++cc) gone[idx[cc]] = 1;
      d2[i] = tot;
      slot = atomicAdd(pcount, 1);
      pkeys[slot] = make_key(n - 1, x >> 1, y >> 1, z >> 1);
    }
  }
  __syncthreads();
  if (slot >= 0)
    for (int q = threadIdx.x; q < k3; q += blockDim.x) pv[(int64_t)slot * k3 + q] = sv[q];
}

__global__ void keep_flags_kernel(int64_t n, const uint64_t *keys, const int *gone, int *keep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keep[i] = gone[i] || keys[i] == ~0ull ? 0 : 1;  // the largest key pads the level
}
// the level's survivor count and merged squared detail into per-level slots
__global__ void level_totals_kernel(const int *kpos, int64_t nl, const double *dsum, int n, int *cnt, double *d2l) {
  cnt[n] = kpos[nl];
  d2l[n] = *dsum;
}

inline size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
inline int64_t boxes(int n) { return 1LL << (3 * n); }

// Options of the per-level applies and of the coarsest level's complete apply.
mra_apply_opts level_opts(const mra_apply_opts &o) { return o; }
mra_apply_opts coarse_opts(const mra_apply_opts &o, int n0) {
  mra_apply_opts c = o;
  c.stencil = MRA_STENCIL_SHELLS;
  c.max_disp = (int)((1LL << n0) - 1);
  return c;
}

// Workspace of mra_apply_ns: dense s^n, S^n (n0 <= n < N), r ping-pong, Y, Z (level N-1
// sizes), Ubar, an error word, one level's keys, the per-level apply outputs (keys +
// coefficients of Y and of Z / the coarse r), and the largest per-level apply workspace.
struct NsLayout {
  std::vector<size_t> s, S;
  size_t rA, rB, Yd, Zd, Ub, err, keys, yk, yc, zk, zc, apply, total;
  size_t apply_bytes;
};

NsLayout ns_layout(const Operator &op, const Operator &ns, int N, int n0, const mra_apply_opts &o) {
  NsLayout L{};
  const int k = op.k, kk = 2 * k;
  const size_t k3 = (size_t)k * k * k, kk3 = (size_t)kk * kk * kk;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = al(off + (bytes ? bytes : 1));
    return at;
  };
  L.s.assign(N + 1, 0);
  L.S.assign(N + 1, 0);
  for (int n = n0; n < N; ++n) {
    L.s[n] = take(boxes(n) * k3 * 8);
    L.S[n] = take(boxes(n) * kk3 * 8);
  }
  const int64_t nt = boxes(N - 1);
  L.rA = take(nt * k3 * 8);
  L.rB = take(nt * k3 * 8);
  L.Yd = take(nt * kk3 * 8);
  L.Zd = take(nt * k3 * 8);
  L.Ub = take((size_t)kk * k * 8);
  L.err = take(8);
  L.keys = take(nt * 8);
  L.yk = take(nt * 8);
  L.yc = take(nt * kk3 * 8);
  L.zk = take(nt * 8);
  L.zc = take(nt * k3 * 8);
  size_t ab = apply_workspace_bytes(op, coarse_opts(o, n0), boxes(n0));
  for (int n = n0; n < N; ++n) {
    ab = std::max(ab, apply_workspace_bytes(op, level_opts(o), boxes(n)));
    ab = std::max(ab, apply_workspace_bytes(ns, level_opts(o), boxes(n)));
  }
  L.apply_bytes = ab;
  L.apply = take(ab);
  L.total = off;
  return L;
}

int ns_check(const Operator *op, const Operator *ns, const mra_tree_view *in, int n0, const mra_apply_opts *o,
             int *N_out) {
  if (!op || !ns) return fail(MRA_ERR_ARG, "mra_apply_ns: NULL operator");
  if (!in || !o) return fail(MRA_ERR_ARG, "mra_apply_ns: NULL argument");
  if (ns->k != 2 * op->k || ns->M != op->M || ns->L != op->L)
    return fail(MRA_ERR_ARG, "mra_apply_ns: the second operator is not the non-standard form of the first");
  if (in->k != op->k || in->L != op->L) return fail(MRA_ERR_ARG, "mra_apply_ns: tree k or L differs from the operator");
  if (in->n <= 0 || !in->keys || !in->coeffs) return fail(MRA_ERR_ARG, "mra_apply_ns: empty input tree");
  int N = -1;
  for (int n = 1; n <= 10; ++n)
    if (in->n == boxes(n)) N = n;
  if (N < 0) return fail(MRA_ERR_ARG, "mra_apply_ns: %lld boxes is not a whole level 1..10", (long long)in->n);
  if (n0 < 0 || n0 >= N) return fail(MRA_ERR_ARG, "mra_apply_ns: coarsest level %d outside 0..%d", n0, N - 1);
  if (n0 < op->min_level || N - 1 > op->max_level || n0 < ns->min_level || N - 1 > ns->max_level)
    return fail(MRA_ERR_ARG, "mra_apply_ns: levels %d..%d outside the operators' tables", n0, N - 1);
  if (o->precision != MRA_PREC_FP64 && o->precision != MRA_PREC_SPLIT_BF16)
    return fail(MRA_ERR_ARG, "mra_apply_ns: unknown precision %d", o->precision);
  if (o->precision == MRA_PREC_SPLIT_BF16 && (o->pieces < 2 || o->pieces > 3))
    return fail(MRA_ERR_ARG, "mra_apply_ns: pieces must be 2 or 3");
  if (o->dest_hi != 0) return fail(MRA_ERR_ARG, "mra_apply_ns: no destination range in the non-standard form");
  if (o->precision == MRA_PREC_SPLIT_BF16 && ns->k > MRA_MAX_K)
    return fail(MRA_ERR_UNSUPPORTED, "mra_apply_ns: order 2k=%d is applied in FP64 only (split precision to %d)",
                ns->k, MRA_MAX_K);
  if (o->screen != MRA_SCREEN_NONE && o->screen != MRA_SCREEN_NORM)
    return fail(MRA_ERR_ARG, "mra_apply_ns: screen must be MRA_SCREEN_NONE or MRA_SCREEN_NORM");
  if (o->screen == MRA_SCREEN_NORM && !(o->tau >= 0.0)) return fail(MRA_ERR_ARG, "mra_apply_ns: tau must be >= 0");
  if (o->stencil != MRA_STENCIL_SHELLS && o->stencil != MRA_STENCIL_NEAREST)
    return fail(MRA_ERR_ARG, "mra_apply_ns: unknown stencil %d", o->stencil);
  const int D = o->stencil == MRA_STENCIL_NEAREST ? 1 : o->max_disp;
  if (D < 0 || D > ns->max_disp || D > op->max_disp)
    return fail(MRA_ERR_ARG, "mra_apply_ns: max_disp %d outside the operators' range", D);
  if ((1LL << n0) - 1 > op->max_disp)
    return fail(MRA_ERR_ARG, "mra_apply_ns: the complete level-%d apply needs an operator with max_disp >= %lld", n0,
                (long long)((1LL << n0) - 1));
  *N_out = N;
  return MRA_OK;
}

}  // namespace

}  // namespace mra

using namespace mra;

extern "C" int mra_operator_ns_create(const mra_operator *h, int max_disp, mra_operator **out, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  if (!op || !out) return fail(MRA_ERR_ARG, "mra_operator_ns_create: NULL argument");
  *out = nullptr;
  if (2 * op->k > MRA_MAX_NS_K)
    return fail(MRA_ERR_ARG, "mra_operator_ns_create: 2k=%d above %d", 2 * op->k, MRA_MAX_NS_K);
  if (op->max_level <= op->min_level)
    return fail(MRA_ERR_ARG, "mra_operator_ns_create: the operator needs at least two levels");
  if (max_disp < 0) return fail(MRA_ERR_ARG, "mra_operator_ns_create: max_disp < 0");
  cudaStream_t s = (cudaStream_t)stream;
  Operator *ns = new Operator();
  auto bail = [&](int code) {
    free_operator(ns);
    return code;
  };
  ns->kernel = op->kernel;
  ns->non_standard = true;
  ns->mu = op->mu;
  ns->M = op->M;
  ns->k = 2 * op->k;
  ns->L = op->L;
  ns->min_level = op->min_level;
  ns->max_level = op->max_level - 1;
  ns->max_disp = max_disp;
  ns->h_fit = op->h_fit;
  ns->s_lo = op->s_lo;
  ns->fit_err = op->fit_err;
  ns->r_lo = op->r_lo;
  ns->r_hi = op->r_hi;
  ns->c = op->c;
  ns->t = op->t;
  std::vector<int> Dabs(20, 0);
  std::vector<int64_t> off_abs(20, -1);
  int64_t nb = 0;
  for (int n = ns->min_level; n <= ns->max_level; ++n) {
    const int D = (int)std::min<int64_t>(max_disp, (1LL << n) - 1);
    if (2 * D + 1 > op->D[n + 1 - op->min_level])
      return bail(fail(MRA_ERR_ARG, "mra_operator_ns_create: level %d needs the operator's max_disp >= %d", n + 1,
                       2 * D + 1));
    Dabs[n] = D;
    off_abs[n] = nb;
    ns->D.push_back(D);
    ns->level_off.push_back(nb);
    nb += (int64_t)ns->M * (2 * D + 1);
  }
  ns->n_blocks = nb;
  const size_t kk2 = (size_t)ns->k * ns->k;
  if (cudaMalloc((void **)&ns->d_c, ns->M * 8) != cudaSuccess || cudaMalloc((void **)&ns->d_t, ns->M * 8) != cudaSuccess ||
      cudaMalloc((void **)&ns->d_R, nb * kk2 * 8) != cudaSuccess || cudaMalloc((void **)&ns->d_N, nb * 8) != cudaSuccess ||
      cudaMalloc((void **)&ns->d_D, 20 * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&ns->d_level_off, 20 * sizeof(int64_t)) != cudaSuccess)
    return bail(fail(MRA_ERR_CUDA, "mra_operator_ns_create: cudaMalloc failed"));
  cudaError_t e = cudaMemcpyAsync(ns->d_c, ns->c.data(), ns->M * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ns->d_t, ns->t.data(), ns->M * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ns->d_D, Dabs.data(), 20 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ns->d_level_off, off_abs.data(), 20 * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  for (int n = ns->min_level; n <= ns->max_level && e == cudaSuccess; ++n) {
    const int li = n - ns->min_level, lc = n + 1 - op->min_level;
    const int D = ns->D[li];
    ns_blocks_kernel<<<counted((unsigned)(ns->M * (2 * D + 1))), 256, 0, s>>>(op->k, ns->M, D, op->d_R, op->level_off[lc],
                                                                       op->D[lc], ns->d_R, ns->level_off[li]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    block_norms_kernel<<<counted((unsigned)((nb + 7) / 8)), 256, 0, s>>>(nb, (int)kk2, ns->d_R, ns->d_N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(fail(MRA_ERR_CUDA, "mra_operator_ns_create: %s", cudaGetErrorString(e)));
  if (ns->k <= MRA_MAX_K) {  // BF16 pieces of the 2k blocks for the tensor-core path
    int rc = split_blocks_build(*ns, s);
    if (rc != MRA_OK) return bail(rc);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(fail(MRA_ERR_CUDA, "mra_operator_ns_create: %s", cudaGetErrorString(e)));
  *out = reinterpret_cast<mra_operator *>(ns);
  return MRA_OK;
}

extern "C" int mra_apply_ns_workspace_size(const mra_operator *h, const mra_operator *hns, const mra_tree_view *in,
                                           int n0, const mra_apply_opts *o, size_t *bytes) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  const Operator *ns = reinterpret_cast<const Operator *>(hns);
  if (!bytes) return fail(MRA_ERR_ARG, "mra_apply_ns_workspace_size: NULL bytes");
  int N = 0;
  int rc = ns_check(op, ns, in, n0, o, &N);
  if (rc) return rc;
  *bytes = ns_layout(*op, *ns, N, n0, *o).total;
  return MRA_OK;
}

extern "C" int mra_apply_ns(const mra_operator *h, const mra_operator *hns, const mra_tree_view *in, int n0,
                            const mra_apply_opts *o, mra_tree_view *out, void *workspace, size_t workspace_bytes,
                            mra_apply_stats *stats, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  const Operator *ns = reinterpret_cast<const Operator *>(hns);
  int N = 0;
  int rc = ns_check(op, ns, in, n0, o, &N);
  if (rc) return rc;
  if (!out || !out->keys || !out->coeffs || out->k != op->k)
    return fail(MRA_ERR_ARG, "mra_apply_ns: output view missing or of another k");
  if (out->cap < in->n) {
    out->n = in->n;
    return fail(MRA_ERR_CAPACITY, "mra_apply_ns: output capacity %lld < %lld", (long long)out->cap,
                (long long)in->n);
  }
  const NsLayout Lw = ns_layout(*op, *ns, N, n0, *o);
  if (!workspace || workspace_bytes < Lw.total)
    return fail(MRA_ERR_CAPACITY, "mra_apply_ns: workspace of %zu bytes < %zu needed", workspace_bytes, Lw.total);
  cudaStream_t s = (cudaStream_t)stream;
  char *w = (char *)workspace;
  const int k = op->k, kk = 2 * k;
  const int k3 = k * k * k, kk3 = kk * kk * kk;
  double *Ub = (double *)(w + Lw.Ub);
  int *d_err = (int *)(w + Lw.err);
  uint64_t *keys = (uint64_t *)(w + Lw.keys);
  // Ubar[(c,i)][j] = U^(c)[i][j]
  std::vector<double> U(2 * k * k), Ubh(2 * k * k);
  two_scale(k, U.data());
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ubh[(c * k + i) * k + j] = U[c * k * k + i * k + j];
  MRA_CUDA_TRY(cudaMemcpyAsync(Ub, Ubh.data(), Ubh.size() * 8, cudaMemcpyHostToDevice, s));
  MRA_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  check_uniform_kernel<<<counted((unsigned)((in->n + 255) / 256)), 256, 0, s>>>(N, in->n, in->keys, d_err);
  MRA_CUDA_TRY(cudaGetLastError());
  int herr = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) return fail(MRA_ERR_ARG, "mra_apply_ns: the input is not every box of level %d in key order", N);

  // ---- compress: S^n and s^n for n = N-1 .. n0
  const size_t sh_c = (size_t)(kk3 + k * kk * kk + k * k * kk) * 8;
  const size_t sh_d = (size_t)(k3 + kk * k * k + kk * kk * k) * 8;
  MRA_CUDA_TRY(cudaFuncSetAttribute(compress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_c));
  MRA_CUDA_TRY(cudaFuncSetAttribute(sum_down_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_d));
  for (int n = N - 1; n >= n0; --n) {
    const double *fine = n == N - 1 ? in->coeffs : (const double *)(w + Lw.s[n + 1]);
    compress_kernel<<<counted((unsigned)boxes(n)), 256, sh_c, s>>>(k, n, fine, Ub, (double *)(w + Lw.S[n]),
                                                          (double *)(w + Lw.s[n]));
    MRA_CUDA_TRY(cudaGetLastError());
  }

  mra_apply_stats acc{};
  auto add_stats = [&](const mra_apply_stats &st) {
    acc.pairs += st.pairs;
    acc.terms_kept += st.terms_kept;
    acc.terms_screened += st.terms_screened;
    acc.terms_issued += st.terms_issued;
    acc.sources_truncated += st.sources_truncated;
    acc.skipped_bound += st.skipped_bound;
    acc.kernel_ms += st.kernel_ms;
    acc.main_kernel_ms += st.main_kernel_ms;
    acc.mma_passes += st.mma_passes;
    acc.kernel = st.kernel;
    acc.algo_flops += st.algo_flops;
    for (int q = 0; q <= MRA_MAX_LEVEL; ++q) {
      acc.level_sources[q] += st.level_sources[q];
      acc.level_terms_kept[q] += st.level_terms_kept[q];
    }
  };
  void *aws = w + Lw.apply;
  // one apply on every box of level n: its output rows scattered into a zeroed dense array
  auto level_apply = [&](const Operator &opx, int n, const double *coeffs, const mra_apply_opts &oo,
                         uint64_t *okeys, double *ocoeffs, double *dense) -> int {
    const int64_t nbx = boxes(n);
    const int rowlen = opx.k * opx.k * opx.k;
    level_keys_kernel<<<counted((unsigned)((nbx + 255) / 256)), 256, 0, s>>>(n, nbx, keys);
    MRA_CUDA_TRY(cudaGetLastError());
    mra_tree_view vin{nbx, nbx, keys, const_cast<double *>(coeffs), opx.k, opx.L};
    mra_tree_view vout{0, nbx, okeys, ocoeffs, opx.k, opx.L};
    mra_apply_stats st{};
    int rc2 = apply_run(opx, vin, oo, vout, aws, Lw.apply_bytes, &st, s);
    if (rc2 != MRA_OK) return rc2;
    add_stats(st);
    MRA_CUDA_TRY(cudaMemsetAsync(dense, 0, (size_t)nbx * rowlen * 8, s));
    if (vout.n > 0) {
      scatter_dense_kernel<<<counted((unsigned)vout.n), 128, 0, s>>>(vout.n, okeys, ocoeffs, rowlen, dense);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    return MRA_OK;
  };
  uint64_t *yk = (uint64_t *)(w + Lw.yk), *zk = (uint64_t *)(w + Lw.zk);
  double *yc = (double *)(w + Lw.yc), *zc = (double *)(w + Lw.zc);
  double *Yd = (double *)(w + Lw.Yd), *Zd = (double *)(w + Lw.Zd);
  double *rcur = (double *)(w + Lw.rA), *rnext = (double *)(w + Lw.rB);

  // ---- coarsest level: T^{n0} with every displacement
  rc = level_apply(*op, n0, (const double *)(w + Lw.s[n0]), coarse_opts(*o, n0), zk, zc, rcur);
  if (rc != MRA_OK) return rc;
  // ---- levels n0 .. N-1
  for (int n = n0; n < N; ++n) {
    rc = level_apply(*ns, n, (const double *)(w + Lw.S[n]), level_opts(*o), yk, yc, Yd);
    if (rc != MRA_OK) return rc;
    rc = level_apply(*op, n, (const double *)(w + Lw.s[n]), level_opts(*o), zk, zc, Zd);
    if (rc != MRA_OK) return rc;
    double *fine = n == N - 1 ? out->coeffs : rnext;
    sum_down_kernel<<<counted((unsigned)boxes(n)), 256, sh_d, s>>>(k, n, rcur, Zd, Yd, Ub, fine);
    MRA_CUDA_TRY(cudaGetLastError());
    std::swap(rcur, rnext);
  }
  MRA_CUDA_TRY(cudaMemcpyAsync(out->keys, in->keys, (size_t)in->n * 8, cudaMemcpyDeviceToDevice, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  out->n = in->n;
  out->L = op->L;
  if (stats) {
    acc.n_in = in->n;
    acc.n_out = in->n;
    *stats = acc;
  }
  return MRA_OK;
}

// ---------------------------------------------------------------- adaptive trees
// The non-standard form apply on an adaptive tree (leaves of a complete octree, every leaf
// deeper than n0).  Sources of level n are the interior nodes I_n (S = children, s = filter);
// the result tree starts with every box of level n0 (r = T^{n0} s^{n0}, every displacement)
// and at each level refines the nodes in the halo of the level's sources -- every box an
// unscreened apply reaches, |l|_inf <= D (children get Ubar^{x3} (r_p - Z_p) + Y_p, absent
// rows of screened applies as zero); the other nodes, and every node of the deepest leaf
// level, are the result's leaves.  The halo keeps every later level's targets inside the
// result: a target's parent lies in the previous level's halo.
extern "C" int mra_apply_ns_tree(const mra_operator *h, const mra_operator *hns, const mra_tree_view *in, int n0,
                                 const mra_apply_opts *o, mra_tree_view *out, mra_apply_stats *stats, void *stream) {
  const Operator *op = reinterpret_cast<const Operator *>(h);
  const Operator *ns = reinterpret_cast<const Operator *>(hns);
  if (!op || !ns || !in || !o || !out) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: NULL argument");
  if (ns->k != 2 * op->k || ns->M != op->M || ns->L != op->L)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: the second operator is not the non-standard form of the first");
  if (in->k != op->k || in->L != op->L) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: tree k or L differs");
  if (in->n <= 0 || !in->keys || !in->coeffs) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: empty input tree");
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: more than 2^31 leaves");
  if (out->k != op->k || out->cap < 0 || (out->cap > 0 && (!out->keys || !out->coeffs)))
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: bad output view");
  if (o->dest_hi != 0) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: no destination range in the non-standard form");
  if (o->precision != MRA_PREC_FP64 && o->precision != MRA_PREC_SPLIT_BF16)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: unknown precision %d", o->precision);
  if (o->precision == MRA_PREC_SPLIT_BF16 && (o->pieces < 2 || o->pieces > 3))
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: pieces must be 2 or 3");
  if (o->screen != MRA_SCREEN_NONE && o->screen != MRA_SCREEN_NORM)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: screen must be MRA_SCREEN_NONE or MRA_SCREEN_NORM");
  if (o->stencil != MRA_STENCIL_SHELLS && o->stencil != MRA_STENCIL_NEAREST)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: unknown stencil %d", o->stencil);
  const int D = o->stencil == MRA_STENCIL_NEAREST ? 1 : o->max_disp;
  if (D < 0 || D > ns->max_disp || D > op->max_disp)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: max_disp %d outside the operators' range", D);
  if (n0 < 0 || (1LL << n0) - 1 > op->max_disp)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: the complete level-%d apply needs max_disp >= %lld", n0,
                (long long)((1LL << n0) - 1));
  cudaStream_t s = (cudaStream_t)stream;
  const int k = op->k, kk = 2 * k, k3 = k * k * k;
  const int64_t n_leaf = in->n;
  std::vector<void *> held;  // stream-ordered allocations, released on every return
  struct Release {
    std::vector<void *> &v;
    cudaStream_t s;
    ~Release() {
      for (void *p : v) cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } release{held, s};
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (pool_malloc(&p, bytes ? bytes : 1, s) != cudaSuccess) return nullptr;
    held.push_back(p);
    return p;
  };
  auto drop = [&](void *p) {  // release one allocation early
    auto it = std::find(held.begin(), held.end(), p);
    if (it != held.end()) {
      cudaFreeAsync(p, s);
      held.erase(it);
    }
  };
#define NS_ALLOC(var, type, count)                                                              \
  type *var = (type *)dalloc((size_t)(count) * sizeof(type));                                   \
  if (!var) return fail(MRA_ERR_CUDA, "mra_apply_ns_tree: out of device memory (%s)", #var);

  // ---- leaves: order, depth
  NS_ALLOC(d_int, int, 4);
  MRA_CUDA_TRY(cudaMemsetAsync(d_int, 0, 4 * sizeof(int), s));
  leaf_check_kernel<<<counted((unsigned)((n_leaf + 255) / 256)), 256, 0, s>>>(n_leaf, in->keys, n0, d_int, d_int + 1);
  MRA_CUDA_TRY(cudaGetLastError());
  int hint[2] = {0, 0};
  MRA_CUDA_TRY(cudaMemcpyAsync(hint, d_int, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (hint[0]) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: leaves must be sorted, unique and deeper than level %d", n0);
  const int Nmax = hint[1];
  if (n0 < op->min_level || Nmax - 1 > op->max_level || n0 < ns->min_level || Nmax - 1 > ns->max_level)
    return fail(MRA_ERR_ARG, "mra_apply_ns_tree: levels %d..%d outside the operators' tables", n0, Nmax - 1);
  NS_ALLOC(Ub, double, kk * k);
  std::vector<double> U(2 * k * k), Ubh(2 * k * k);
  two_scale(k, U.data());
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ubh[(c * k + i) * k + j] = U[c * k * k + i * k + j];
  MRA_CUDA_TRY(cudaMemcpyAsync(Ub, Ubh.data(), Ubh.size() * 8, cudaMemcpyHostToDevice, s));

  // ---- interior nodes of every level: the leaves' ancestors, sorted and unique, all levels in
  // one sort (keys order by level first, so each level is one range)
  std::vector<uint64_t *> Ik(Nmax + 1, nullptr);
  std::vector<int64_t> In(Nmax + 1, 0);
  {
    const int nlev = std::max(Nmax - n0, 1);
    if (n_leaf * nlev >= (int64_t)INT32_MAX) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: too many leaves x levels");
    const int64_t na = n_leaf * nlev;
    NS_ALLOC(anc, uint64_t, na);
    NS_ALLOC(anc_s, uint64_t, na);
    NS_ALLOC(d_nsel, int64_t, 1);
    NS_ALLOC(d_off, int64_t, 21);
    size_t t1 = 0, t2 = 0;
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, t1, anc, anc_s, (int)na, 0, 64, s));
    MRA_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, t2, anc_s, anc, d_nsel, (int)na, s));
    size_t tb = std::max(t1, t2);
    NS_ALLOC(tmp, unsigned char, tb);
    ancestor_kernel<<<counted((unsigned)((na + 255) / 256)), 256, 0, s>>>(n_leaf, in->keys, n0, nlev, anc);
    MRA_CUDA_TRY(cudaGetLastError());
    size_t tt = tb;
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tt, anc, anc_s, (int)na, 0, 64, s));
    tt = tb;
    MRA_CUDA_TRY(cub::DeviceSelect::Unique(tmp, tt, anc_s, anc, d_nsel, (int)na, s));
    level_offsets_kernel<<<counted(1), 32, 0, s>>>(anc, d_nsel, d_off);
    MRA_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> off(21);
    MRA_CUDA_TRY(cudaMemcpyAsync(off.data(), d_off, 21 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
    for (int n = n0; n < Nmax; ++n) {
      Ik[n] = anc + off[n];
      In[n] = off[n + 1] - off[n];
    }
    drop(anc_s);
    drop(tmp);
  }
  if (In[n0] != boxes(n0)) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: level %d is not complete", n0);

  // ---- compress, from the deepest interior level up
  const size_t sh_c = (size_t)(kk * kk * kk + k * kk * kk + k * k * kk) * 8;
  const size_t sh_d = (size_t)(k3 + kk * k * k + kk * kk * k) * 8;
  MRA_CUDA_TRY(cudaFuncSetAttribute(compress_tree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_c));
  MRA_CUDA_TRY(cudaFuncSetAttribute(sum_down_tree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_d));
  std::vector<double *> Sn(Nmax + 1, nullptr), sn(Nmax + 1, nullptr);
  for (int n = Nmax - 1; n >= n0; --n) {
    NS_ALLOC(S, double, In[n] * kk * kk * kk);
    NS_ALLOC(sv, double, In[n] * k3);
    Sn[n] = S;
    sn[n] = sv;
    const bool deeper = n + 1 < Nmax;
    compress_tree_kernel<<<counted((unsigned)In[n]), 256, sh_c, s>>>(k, n, Ik[n], In[n], in->keys, in->coeffs, n_leaf,
                                                            deeper ? Ik[n + 1] : nullptr, deeper ? sn[n + 1] : nullptr,
                                                            deeper ? In[n + 1] : 0, Ub, S, sv, d_int);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  MRA_CUDA_TRY(cudaMemcpyAsync(hint, d_int, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (hint[0]) return fail(MRA_ERR_ARG, "mra_apply_ns_tree: the leaves are not a complete octree");

  mra_apply_stats acc{};
  // one library apply on the given boxes of one level; its output allocated here
  auto run_apply = [&](const Operator &opx, int64_t nsrc, uint64_t *skeys, double *scoeffs,
                       const mra_apply_opts &oo, int64_t cap, uint64_t **okeys, double **ocoeffs,
                       int64_t *nout) -> int {
    const size_t wb = apply_workspace_bytes(opx, oo, nsrc);
    void *ws = dalloc(wb);
    *okeys = (uint64_t *)dalloc((size_t)cap * 8);
    *ocoeffs = (double *)dalloc((size_t)cap * opx.k * opx.k * opx.k * 8);
    if (!ws || !*okeys || !*ocoeffs) return fail(MRA_ERR_CUDA, "mra_apply_ns_tree: out of device memory");
    mra_tree_view vin{nsrc, nsrc, skeys, scoeffs, opx.k, opx.L};
    mra_tree_view vout{0, cap, *okeys, *ocoeffs, opx.k, opx.L};
    mra_apply_stats st{};
    const int rc2 = apply_run(opx, vin, oo, vout, ws, wb, &st, s);
    drop(ws);
    if (rc2 != MRA_OK) return rc2;
    acc.pairs += st.pairs;
    acc.terms_kept += st.terms_kept;
    acc.terms_screened += st.terms_screened;
    acc.terms_issued += st.terms_issued;
    acc.skipped_bound += st.skipped_bound;
    acc.kernel_ms += st.kernel_ms;
    acc.main_kernel_ms += st.main_kernel_ms;
    acc.mma_passes += st.mma_passes;
    acc.kernel = st.kernel;
    acc.algo_flops += st.algo_flops;
    for (int q = 0; q <= MRA_MAX_LEVEL; ++q) {
      acc.level_sources[q] += st.level_sources[q];
      acc.level_terms_kept[q] += st.level_terms_kept[q];
    }
    *nout = vout.n;
    return MRA_OK;
  };

  // ---- coarsest level: every box, T^{n0} with every displacement
  int64_t nR = boxes(n0);
  uint64_t *Rk = Ik[n0];
  NS_ALLOC(r0, double, nR * k3);
  double *R = r0;
  {
    uint64_t *ok;
    double *oc;
    int64_t no = 0;
    int rc = run_apply(*op, nR, Rk, sn[n0], coarse_opts(*o, n0), nR, &ok, &oc, &no);
    if (rc != MRA_OK) return rc;
    MRA_CUDA_TRY(cudaMemsetAsync(R, 0, (size_t)nR * k3 * 8, s));
    if (no > 0) {
      scatter_dense_kernel<<<counted((unsigned)no), 128, 0, s>>>(no, ok, oc, k3, R);  // level n0 is complete: dense order
      MRA_CUDA_TRY(cudaGetLastError());
    }
    drop(ok);
    drop(oc);
  }
  int64_t nout = 0;
  const int64_t cap = out->cap;
  const int64_t w3 = (int64_t)(2 * D + 1) * (2 * D + 1) * (2 * D + 1);
  for (int n = n0; n < Nmax; ++n) {
    const int64_t tcap = std::min<int64_t>(boxes(n), In[n] * w3);
    uint64_t *yk, *zk;
    double *yc, *zc;
    int64_t ny = 0, nz = 0;
    int rc = run_apply(*ns, In[n], Ik[n], Sn[n], level_opts(*o), tcap, &yk, &yc, &ny);
    if (rc != MRA_OK) return rc;
    rc = run_apply(*op, In[n], Ik[n], sn[n], level_opts(*o), tcap, &zk, &zc, &nz);
    if (rc != MRA_OK) return rc;
    MRA_CUDA_TRY(cudaMemsetAsync(d_int, 0, sizeof(int), s));
    if (ny > 0) targets_in_kernel<<<counted((unsigned)((ny + 255) / 256)), 256, 0, s>>>(ny, yk, Rk, nR, d_int);
    if (nz > 0) targets_in_kernel<<<counted((unsigned)((nz + 255) / 256)), 256, 0, s>>>(nz, zk, Rk, nR, d_int);
    MRA_CUDA_TRY(cudaGetLastError());
    // the halo of the level's sources, sorted and unique
    const int64_t nh_all = In[n] * w3;
    NS_ALLOC(hal, uint64_t, nh_all);
    NS_ALLOC(hal_s, uint64_t, nh_all);
    NS_ALLOC(hk, uint64_t, nh_all);
    NS_ALLOC(d_nh, int64_t, 1);
    MRA_CUDA_TRY(cudaMemsetAsync(d_nh, 0, 8, s));
    if (nh_all > 0) {
      halo_kernel<<<counted((unsigned)((nh_all + 255) / 256)), 256, 0, s>>>(In[n], Ik[n], D, hal);
      MRA_CUDA_TRY(cudaGetLastError());
      size_t t1 = 0, t2 = 0;
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, t1, hal, hal_s, (int)nh_all, 0, 64, s));
      MRA_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, t2, hal_s, hk, d_nh, (int)nh_all, s));
      NS_ALLOC(tmph, unsigned char, std::max(t1, t2));
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmph, t1, hal, hal_s, (int)nh_all, 0, 64, s));
      MRA_CUDA_TRY(cub::DeviceSelect::Unique(tmph, t2, hal_s, hk, d_nh, (int)nh_all, s));
      drop(tmph);
    }
    NS_ALLOC(yi, int64_t, nR);
    NS_ALLOC(zi, int64_t, nR);
    NS_ALLOC(refine, int, nR + 1);
    NS_ALLOC(leaf, int, nR + 1);
    NS_ALLOC(ref_pos, int, nR + 1);
    NS_ALLOC(leaf_pos, int, nR + 1);
    if (nR > 0) {
      reach_kernel<<<counted((unsigned)((nR + 255) / 256)), 256, 0, s>>>(nR, Rk, hk, d_nh, yk, ny, zk, nz, yi, zi, refine, leaf);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    MRA_CUDA_TRY(cudaMemsetAsync(refine + nR, 0, sizeof(int), s));
    MRA_CUDA_TRY(cudaMemsetAsync(leaf + nR, 0, sizeof(int), s));
    size_t tb = 0;
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, refine, ref_pos, (int)(nR + 1), s));
    NS_ALLOC(tmp, unsigned char, tb);
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, refine, ref_pos, (int)(nR + 1), s));
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, leaf, leaf_pos, (int)(nR + 1), s));
    int hcount[2] = {0, 0};
    MRA_CUDA_TRY(cudaMemcpyAsync(&hcount[0], ref_pos + nR, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(&hint[0], d_int, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
    if (hint[0]) return fail(MRA_ERR_NUMERIC, "mra_apply_ns_tree: a level-%d apply reached a box outside the result tree", n);
    const int64_t nref = hcount[0], nleaf_here = nR - nref;
    if (nleaf_here > 0 && nR > 0) {
      emit_leaves_kernel<<<counted((unsigned)nR), 128, 0, s>>>(nR, k3, Rk, R, leaf, leaf_pos, nout, cap, out->keys, out->coeffs);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    nout += nleaf_here;
    // children of the reached nodes, then in key order
    const int64_t nC = 8 * nref;
    NS_ALLOC(cku, uint64_t, nC);
    NS_ALLOC(cru, double, nC * k3);
    if (nref > 0) {
      sum_down_tree_kernel<<<counted((unsigned)nR), 256, sh_d, s>>>(k, nR, Rk, R, refine, ref_pos, yi, yc, zi, zc, Ub, cku, cru);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    NS_ALLOC(cks, uint64_t, nC);
    NS_ALLOC(crs, double, nC * k3);
    NS_ALLOC(idx, int, nC);
    NS_ALLOC(idx_s, int, nC);
    if (nC > 0) {
      iota_ns_kernel<<<counted((unsigned)((nC + 255) / 256)), 256, 0, s>>>(nC, idx);
      MRA_CUDA_TRY(cudaGetLastError());
      size_t ts = 0;
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, ts, cku, cks, idx, idx_s, (int)nC, 0, 64, s));
      NS_ALLOC(tmp2, unsigned char, ts);
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp2, ts, cku, cks, idx, idx_s, (int)nC, 0, 64, s));
      gather_rows_ns_kernel<<<counted((unsigned)nC), 128, 0, s>>>(nC, k3, idx_s, cru, crs);
      MRA_CUDA_TRY(cudaGetLastError());
      drop(tmp2);
    }
    for (void *p : {(void *)yk, (void *)yc, (void *)zk, (void *)zc, (void *)yi, (void *)zi, (void *)refine,
                    (void *)leaf, (void *)ref_pos, (void *)leaf_pos, (void *)tmp, (void *)cku, (void *)cru,
                    (void *)idx, (void *)idx_s, (void *)hal, (void *)hal_s, (void *)hk, (void *)d_nh})
      drop(p);
    if (Rk != Ik[n0]) drop(Rk);
    drop(R);
    Rk = cks;
    R = crs;
    nR = nC;
  }
  // the deepest level: every node is a result leaf
  if (nR > 0 && nout < cap) {
    const int64_t ncopy = std::min<int64_t>(nR, cap - nout);
    MRA_CUDA_TRY(cudaMemcpyAsync(out->keys + nout, Rk, (size_t)ncopy * 8, cudaMemcpyDeviceToDevice, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(out->coeffs + nout * k3, R, (size_t)ncopy * k3 * 8, cudaMemcpyDeviceToDevice, s));
  }
  nout += nR;
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (stats) {
    acc.n_in = n_leaf;
    acc.n_out = nout;
    *stats = acc;
  }
  out->L = op->L;
  if (nout > cap) {
    out->n = nout;
    return fail(MRA_ERR_CAPACITY, "mra_apply_ns_tree: %lld result leaves, capacity %lld", (long long)nout,
                (long long)cap);
  }
  out->n = nout;
  return MRA_OK;
#undef NS_ALLOC
}


// ---------------------------------------------------------------- reconstruct (host)
extern "C" int mra_reconstruct(const mra_tree_view *in, mra_tree_view *out, void *stream) {
  if (!in || !out) return fail(MRA_ERR_ARG, "mra_reconstruct: NULL argument");
  if (in->n < 0 || (in->n > 0 && (!in->keys || !in->coeffs))) return fail(MRA_ERR_ARG, "mra_reconstruct: bad input");
  if (in->k < 1 || in->k > MRA_MAX_K) return fail(MRA_ERR_ARG, "mra_reconstruct: k=%d outside 1..%d", in->k, MRA_MAX_K);
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_reconstruct: more than 2^31 boxes");
  if (out->k != in->k || out->cap < 0 || (out->cap > 0 && (!out->keys || !out->coeffs)))
    return fail(MRA_ERR_ARG, "mra_reconstruct: bad output view");
  out->L = in->L;
  if (in->n == 0) {
    out->n = 0;
    return MRA_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int k = in->k, kk = 2 * k, k3 = k * k * k;
  const int64_t n_in = in->n;
  std::vector<void *> held;
  struct Release {
    std::vector<void *> &v;
    cudaStream_t s;
    ~Release() {
      for (void *p : v) cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } release{held, s};
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (pool_malloc(&p, bytes ? bytes : 1, s) != cudaSuccess) return nullptr;
    held.push_back(p);
    return p;
  };
  auto drop = [&](void *p) {
    auto it = std::find(held.begin(), held.end(), p);
    if (it != held.end()) {
      cudaFreeAsync(p, s);
      held.erase(it);
    }
  };
#define RC_ALLOC(var, type, count)                                                              \
  type *var = (type *)dalloc((size_t)(count) * sizeof(type));                                   \
  if (!var) return fail(MRA_ERR_CUDA, "mra_reconstruct: out of device memory (%s)", #var);

  // order and the level ranges of the sorted input
  std::vector<uint64_t> hk(n_in);
  MRA_CUDA_TRY(cudaMemcpyAsync(hk.data(), in->keys, (size_t)n_in * 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int64_t> lo(21, n_in), hi(21, n_in);
  for (int64_t i = 0; i < n_in; ++i) {
    if (i > 0 && hk[i] <= hk[i - 1]) return fail(MRA_ERR_ARG, "mra_reconstruct: keys must be sorted and unique");
    const int lv = key_level(hk[i]);
    if (lv > 19) return fail(MRA_ERR_ARG, "mra_reconstruct: level %d above 19", lv);
  }
  for (int n = 0; n <= 20; ++n) {
    lo[n] = std::lower_bound(hk.begin(), hk.end(), (uint64_t)n << 57) - hk.begin();
    hi[n] = n < 20 ? std::lower_bound(hk.begin(), hk.end(), (uint64_t)(n + 1) << 57) - hk.begin() : n_in;
  }
  const int nmin = key_level(hk.front()), nmax = key_level(hk.back());
  RC_ALLOC(Ub, double, kk * k);
  std::vector<double> U(2 * k * k), Ubh(2 * k * k);
  two_scale(k, U.data());
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ubh[(c * k + i) * k + j] = U[c * k * k + i * k + j];
  MRA_CUDA_TRY(cudaMemcpyAsync(Ub, Ubh.data(), Ubh.size() * 8, cudaMemcpyHostToDevice, s));
  RC_ALLOC(top, int, n_in);
  top_level_kernel<<<counted((unsigned)((n_in + 255) / 256)), 256, 0, s>>>(n_in, in->keys, top);
  MRA_CUDA_TRY(cudaGetLastError());
  RC_ALLOC(d_err, int, 1);
  MRA_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  // Every size of the level loop is known in advance, so the loop runs without a host
  // synchronisation: the interior boxes of all levels (one sort), the tops of all levels
  // (one scan), one copy to the host.  A level's boxes are the 8 children of the previous
  // level's interior boxes and its tops; its interior boxes are exactly the interior keys of
  // the level (checked on the device), the others are leaves of the result.
  const int nlev = std::max(nmax - nmin, 1);
  if (n_in * nlev >= (int64_t)INT32_MAX) return fail(MRA_ERR_ARG, "mra_reconstruct: too many boxes x levels");
  const int64_t na = n_in * nlev;
  RC_ALLOC(anc, uint64_t, na);
  RC_ALLOC(iall, uint64_t, na);
  RC_ALLOC(d_nsel, int64_t, 1);
  RC_ALLOC(d_ioff, int64_t, 21);
  RC_ALLOC(tflag, int, n_in + 1);
  RC_ALLOC(tpos, int, n_in + 1);
  interior_all_kernel<<<counted((unsigned)((na + 255) / 256)), 256, 0, s>>>(n_in, in->keys, top, nmin, nlev, anc);
  MRA_CUDA_TRY(cudaGetLastError());
  top_flags_kernel<<<counted((unsigned)((n_in + 256) / 256)), 256, 0, s>>>(n_in, in->keys, top, tflag);
  MRA_CUDA_TRY(cudaGetLastError());
  {
    size_t tb = 0, t2 = 0, t3 = 0;
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, anc, iall, (int)na, 0, 64, s));
    MRA_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, t2, iall, anc, d_nsel, (int)na, s));
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, t3, tflag, tpos, (int)(n_in + 1), s));
    tb = std::max(tb, std::max(t2, t3));
    RC_ALLOC(tmp, unsigned char, tb);
    size_t tt = tb;
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tt, anc, iall, (int)na, 0, 64, s));
    tt = tb;
    MRA_CUDA_TRY(cub::DeviceSelect::Unique(tmp, tt, iall, anc, d_nsel, (int)na, s));
    tt = tb;
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tt, tflag, tpos, (int)(n_in + 1), s));
    drop(tmp);
  }
  uint64_t *ik_all = anc;  // the unique interior keys, in key order (so level by level)
  level_offsets_kernel<<<counted(1), 32, 0, s>>>(ik_all, d_nsel, d_ioff);
  MRA_CUDA_TRY(cudaGetLastError());
  std::vector<int64_t> ioff(21);
  std::vector<int> tposh(n_in + 1);
  MRA_CUDA_TRY(cudaMemcpyAsync(ioff.data(), d_ioff, 21 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(tposh.data(), tpos, (size_t)(n_in + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  drop(iall);
  const size_t sh_d = (size_t)(k3 + kk * k * k + kk * kk * k) * 8;
  MRA_CUDA_TRY(cudaFuncSetAttribute(pass_down_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_d));
  uint64_t *Ck = nullptr;  // boxes passed down to the current level (unsorted) and their values
  double *Cv = nullptr;
  int64_t nC = 0, nout = 0;
  const int64_t cap = out->cap;
  for (int n = nmin; n <= nmax; ++n) {
    const int64_t ni = ioff[n + 1] - ioff[n];  // interior boxes of level n
    const uint64_t *ik = ik_all + ioff[n];
    // the level's boxes: passed down, then the tops of this level; in key order
    const int64_t nl = hi[n] - lo[n];
    const int ntop = tposh[hi[n]] - tposh[lo[n]];
    const int64_t nr = nC + ntop;
    RC_ALLOC(uk, uint64_t, nr);
    RC_ALLOC(uv, double, nr * k3);
    if (nC > 0) {
      MRA_CUDA_TRY(cudaMemcpyAsync(uk, Ck, (size_t)nC * 8, cudaMemcpyDeviceToDevice, s));
      MRA_CUDA_TRY(cudaMemcpyAsync(uv, Cv, (size_t)nC * k3 * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (ntop > 0) {
      tops_kernel<<<counted((unsigned)nl), 128, 0, s>>>(lo[n], hi[n], n, top, in->keys, in->coeffs, k3, tpos,
                                                        tposh[lo[n]], nC, uk, uv);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    RC_ALLOC(rk, uint64_t, nr);
    RC_ALLOC(rv, double, nr * k3);
    RC_ALLOC(idx, int, nr);
    RC_ALLOC(idx_s, int, nr);
    if (nr > 0) {
      iota_ns_kernel<<<counted((unsigned)((nr + 255) / 256)), 256, 0, s>>>(nr, idx);
      MRA_CUDA_TRY(cudaGetLastError());
      size_t tsp = 0;
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tsp, uk, rk, idx, idx_s, (int)nr, 0, 64, s));
      RC_ALLOC(tmp4, unsigned char, tsp);
      MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp4, tsp, uk, rk, idx, idx_s, (int)nr, 0, 64, s));
      gather_rows_ns_kernel<<<counted((unsigned)nr), 128, 0, s>>>(nr, k3, idx_s, uv, rv);
      MRA_CUDA_TRY(cudaGetLastError());
      drop(tmp4);
    }
    if (nl > 0) {  // input boxes below a top add their coefficients
      add_inputs_kernel<<<counted((unsigned)nl), 128, 0, s>>>(lo[n], hi[n], n, top, in->keys, in->coeffs, k3, rk, nr, rv, d_err);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    // leaves out, interior boxes passed down
    RC_ALLOC(inner, int, nr + 1);
    RC_ALLOC(leaf, int, nr + 1);
    RC_ALLOC(ipos, int, nr + 1);
    RC_ALLOC(lpos, int, nr + 1);
    MRA_CUDA_TRY(cudaMemsetAsync(inner + nr, 0, sizeof(int), s));
    MRA_CUDA_TRY(cudaMemsetAsync(leaf + nr, 0, sizeof(int), s));
    if (nr > 0) {
      classify_kernel<<<counted((unsigned)((nr + 255) / 256)), 256, 0, s>>>(nr, rk, ik, ni, inner, leaf);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    size_t tsc = 0;
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tsc, inner, ipos, (int)(nr + 1), s));
    RC_ALLOC(tmp5, unsigned char, tsc);
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp5, tsc, inner, ipos, (int)(nr + 1), s));
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp5, tsc, leaf, lpos, (int)(nr + 1), s));
    inner_count_check_kernel<<<counted(1), 1, 0, s>>>(ipos, nr, ni, d_err);
    MRA_CUDA_TRY(cudaGetLastError());
    if (nr - ni > 0) {
      emit_leaves_kernel<<<counted((unsigned)nr), 128, 0, s>>>(nr, k3, rk, rv, leaf, lpos, nout, cap, out->keys, out->coeffs);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    nout += std::max<int64_t>(nr - ni, 0);
    const int64_t nnext = 8 * ni;
    RC_ALLOC(nk, uint64_t, nnext);
    RC_ALLOC(nv, double, nnext * k3);
    if (ni > 0 && nr > 0) {
      pass_down_kernel<<<counted((unsigned)nr), 256, sh_d, s>>>(k, nr, rk, rv, inner, ipos, ni, Ub, nk, nv, d_err);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    for (void *p : {(void *)uk, (void *)uv, (void *)rk, (void *)rv, (void *)idx, (void *)idx_s, (void *)inner,
                    (void *)leaf, (void *)ipos, (void *)lpos, (void *)tmp5})
      drop(p);
    if (Ck) drop(Ck);
    if (Cv) drop(Cv);
    Ck = nk;
    Cv = nv;
    nC = nnext;
  }
  int herr = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr == 1) return fail(MRA_ERR_NUMERIC, "mra_reconstruct: an input box has no place in the result");
  if (herr) return fail(MRA_ERR_NUMERIC, "mra_reconstruct: the interior boxes of a level are inconsistent");
  if (nC != 0) return fail(MRA_ERR_NUMERIC, "mra_reconstruct: boxes passed below the deepest level");
  if (nout > cap) {
    out->n = nout;
    return fail(MRA_ERR_CAPACITY, "mra_reconstruct: %lld leaves, capacity %lld", (long long)nout, (long long)cap);
  }
  out->n = nout;
  return MRA_OK;
#undef RC_ALLOC
}


// ---------------------------------------------------------------- truncate (host)
extern "C" int mra_truncate(const mra_tree_view *in, double thresh, mra_tree_view *out, double *err2, void *stream) {
  if (!in || !out) return fail(MRA_ERR_ARG, "mra_truncate: NULL argument");
  if (in->n < 0 || (in->n > 0 && (!in->keys || !in->coeffs))) return fail(MRA_ERR_ARG, "mra_truncate: bad input");
  if (in->k < 1 || in->k > MRA_MAX_K) return fail(MRA_ERR_ARG, "mra_truncate: k=%d outside 1..%d", in->k, MRA_MAX_K);
  if (in->n >= (1LL << 31)) return fail(MRA_ERR_ARG, "mra_truncate: more than 2^31 leaves");
  if (!(thresh >= 0.0)) return fail(MRA_ERR_ARG, "mra_truncate: thresh must be >= 0");
  if (out->k != in->k || out->cap < 0 || (out->cap > 0 && (!out->keys || !out->coeffs)))
    return fail(MRA_ERR_ARG, "mra_truncate: bad output view");
  out->L = in->L;
  if (err2) *err2 = 0.0;
  if (in->n == 0) {
    out->n = 0;
    return MRA_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int k = in->k, kk = 2 * k, k3 = k * k * k;
  const int64_t n_in = in->n;
  std::vector<void *> held;
  struct Release {
    std::vector<void *> &v;
    cudaStream_t s;
    ~Release() {
      for (void *p : v) cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } release{held, s};
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (pool_malloc(&p, bytes ? bytes : 1, s) != cudaSuccess) return nullptr;
    held.push_back(p);
    return p;
  };
#define TR_ALLOC(var, type, count)                                                              \
  type *var = (type *)dalloc((size_t)(count) * sizeof(type));                                   \
  if (!var) return fail(MRA_ERR_CUDA, "mra_truncate: out of device memory (%s)", #var);

  std::vector<uint64_t> hk(n_in);
  MRA_CUDA_TRY(cudaMemcpyAsync(hk.data(), in->keys, (size_t)n_in * 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int64_t i = 1; i < n_in; ++i)
    if (hk[i] <= hk[i - 1]) return fail(MRA_ERR_ARG, "mra_truncate: keys must be sorted and unique");
  if (key_level(hk.back()) > 19) return fail(MRA_ERR_ARG, "mra_truncate: level above 19");
  std::vector<int64_t> lo(21), hi(21);
  for (int n = 0; n <= 20; ++n) {
    lo[n] = std::lower_bound(hk.begin(), hk.end(), (uint64_t)n << 57) - hk.begin();
    hi[n] = n < 20 ? std::lower_bound(hk.begin(), hk.end(), (uint64_t)(n + 1) << 57) - hk.begin() : n_in;
  }
  TR_ALLOC(Ub, double, kk * k);
  std::vector<double> U(2 * k * k), Ubh(2 * k * k);
  two_scale(k, U.data());
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Ubh[(c * k + i) * k + j] = U[c * k * k + i * k + j];
  MRA_CUDA_TRY(cudaMemcpyAsync(Ub, Ubh.data(), Ubh.size() * 8, cudaMemcpyHostToDevice, s));
  // S stays in shared memory up to k = 12 (120 k^3 bytes); above, only the filter's pieces (56 k^3)
  const int s_smem = k <= 12 ? 1 : 0;
  const size_t sh = (size_t)(k * kk * kk + k * k * kk + k3 + (s_smem ? kk * kk * kk : 0)) * 8;
  MRA_CUDA_TRY(cudaFuncSetAttribute(truncate_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  TR_ALLOC(pcount, int, 1);
  TR_ALLOC(d_cnt, int, 20);
  TR_ALLOC(d_d2l, double, 20);
  MRA_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 20 * sizeof(int), s));
  MRA_CUDA_TRY(cudaMemsetAsync(d_d2l, 0, 20 * sizeof(double), s));
  // The level loop runs without a host synchronisation.  The parents merged from level n+1
  // are at most an eighth of that level's leaves, so every array is sized by that bound; the
  // merged parents are written at atomic slots of an array prefilled with the largest key,
  // which sorts after every real key, is never a leaf of a sibling group and is not kept.
  // The survivors of each level stay on the device until the counts are read at the end.
  std::vector<uint64_t *> keep_k(20, nullptr);
  std::vector<double *> keep_v(20, nullptr);
  uint64_t *mk = nullptr;  // parents merged from the level below (unsorted, padded)
  double *mv = nullptr;
  int64_t nm = 0;  // bound on their number
  const int top = key_level(hk.back());
  for (int n = top; n >= 0; --n) {
    // this level's leaves: the input's, then the merged parents, in key order
    const int64_t ni = hi[n] - lo[n], nl = ni + nm;
    if (nl == 0) continue;
    TR_ALLOC(uk, uint64_t, nl);
    TR_ALLOC(uv, double, nl * k3);
    if (ni > 0) {
      MRA_CUDA_TRY(cudaMemcpyAsync(uk, in->keys + lo[n], (size_t)ni * 8, cudaMemcpyDeviceToDevice, s));
      MRA_CUDA_TRY(cudaMemcpyAsync(uv, in->coeffs + lo[n] * k3, (size_t)ni * k3 * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (nm > 0) {
      MRA_CUDA_TRY(cudaMemcpyAsync(uk + ni, mk, (size_t)nm * 8, cudaMemcpyDeviceToDevice, s));
      MRA_CUDA_TRY(cudaMemcpyAsync(uv + ni * k3, mv, (size_t)nm * k3 * 8, cudaMemcpyDeviceToDevice, s));
    }
    TR_ALLOC(lk, uint64_t, nl);
    TR_ALLOC(lv, double, nl * k3);
    TR_ALLOC(idx, int, nl);
    TR_ALLOC(idx_s, int, nl);
    iota_ns_kernel<<<counted((unsigned)((nl + 255) / 256)), 256, 0, s>>>(nl, idx);
    MRA_CUDA_TRY(cudaGetLastError());
    size_t tsp = 0;
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tsp, uk, lk, idx, idx_s, (int)nl, 0, 64, s));
    TR_ALLOC(tmp, unsigned char, tsp);
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tsp, uk, lk, idx, idx_s, (int)nl, 0, 64, s));
    gather_rows_ns_kernel<<<counted((unsigned)nl), 128, 0, s>>>(nl, k3, idx_s, uv, lv);
    MRA_CUDA_TRY(cudaGetLastError());
    // merges into level n-1
    TR_ALLOC(gone, int, nl + 1);
    TR_ALLOC(d2, double, nl);
    MRA_CUDA_TRY(cudaMemsetAsync(gone, 0, (size_t)(nl + 1) * sizeof(int), s));
    MRA_CUDA_TRY(cudaMemsetAsync(d2, 0, (size_t)nl * 8, s));
    MRA_CUDA_TRY(cudaMemsetAsync(pcount, 0, sizeof(int), s));
    const int64_t np_max = n > 0 ? nl / 8 : 0;
    TR_ALLOC(pk, uint64_t, np_max + 1);
    TR_ALLOC(pv, double, (np_max + 1) * k3);
    MRA_CUDA_TRY(cudaMemsetAsync(pk, 0xFF, (size_t)(np_max + 1) * 8, s));
    if (n > 0) {
      truncate_level_kernel<<<counted((unsigned)nl), 256, sh, s>>>(k, n, nl, lk, lv, thresh, Ub, gone, d2, pk, pv, pcount,
                                                                   s_smem);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    // survivors, compacted in key order
    TR_ALLOC(keep, int, nl + 1);
    TR_ALLOC(kpos, int, nl + 1);
    keep_flags_kernel<<<counted((unsigned)((nl + 255) / 256)), 256, 0, s>>>(nl, lk, gone, keep);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cudaMemsetAsync(keep + nl, 0, sizeof(int), s));
    size_t tsc = 0;
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tsc, keep, kpos, (int)(nl + 1), s));
    size_t tsr = 0;
    double *dsum = nullptr;
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(nullptr, tsr, d2, dsum, (int)nl, s));
    TR_ALLOC(tmp2, unsigned char, std::max(tsc, tsr));
    TR_ALLOC(dsum_d, double, 1);
    MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp2, tsc, keep, kpos, (int)(nl + 1), s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp2, tsr, d2, dsum_d, (int)nl, s));
    level_totals_kernel<<<counted(1), 1, 0, s>>>(kpos, nl, dsum_d, n, d_cnt, d_d2l);
    MRA_CUDA_TRY(cudaGetLastError());
    TR_ALLOC(kk_, uint64_t, nl);
    TR_ALLOC(kv, double, nl * k3);
    emit_leaves_kernel<<<counted((unsigned)nl), 128, 0, s>>>(nl, k3, lk, lv, keep, kpos, 0, nl, kk_, kv);
    MRA_CUDA_TRY(cudaGetLastError());
    keep_k[n] = kk_;
    keep_v[n] = kv;
    mk = pk;
    mv = pv;
    nm = np_max;
  }
  std::vector<int> keep_n(20);
  std::vector<double> d2l(20);
  MRA_CUDA_TRY(cudaMemcpyAsync(keep_n.data(), d_cnt, 20 * sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(d2l.data(), d_d2l, 20 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  double e2 = 0.0;
  for (int n = top; n >= 0; --n) e2 += d2l[n];
  int64_t nout = 0;
  for (int n = 0; n < 20; ++n) nout += keep_n[n];
  if (nout > out->cap) {
    out->n = nout;
    return fail(MRA_ERR_CAPACITY, "mra_truncate: %lld leaves, capacity %lld", (long long)nout, (long long)out->cap);
  }
  int64_t o = 0;
  for (int n = 0; n < 20; ++n) {
    if (keep_n[n] == 0) continue;
    MRA_CUDA_TRY(cudaMemcpyAsync(out->keys + o, keep_k[n], (size_t)keep_n[n] * 8, cudaMemcpyDeviceToDevice, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(out->coeffs + o * k3, keep_v[n], (size_t)keep_n[n] * k3 * 8, cudaMemcpyDeviceToDevice, s));
    o += keep_n[n];
  }
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  out->n = nout;
  if (err2) *err2 = e2;
  return MRA_OK;
#undef TR_ALLOC
}
