// apply.cu -- the apply path: source norms, norm screen and work list, sort on the
// destination key, FP64 gather-apply, and the norm/compare reductions.
//
// Work list.  For every source box b (level n) and displacement l in D(b) the
// screen computes, per Gaussian term m, the bound
//     B = |c_m| * ||R^n_{m,lx}||_F * ||R^n_{m,ly}||_F * ||R^n_{m,lz}||_F * ||s_b||_F
// and keeps the term iff B >= tau (the sum of FP32 logs of the five factors decides first, the
// FP64 product wherever that sum is within its error margin of log2 tau, so every decision is
// the FP64 product's).  A (b, l) pair with at least one kept term
// becomes a record {dest key = key(n, b + l), b, l, kept-term mask}.  Records
// are sorted on the destination key (stable radix sort), so the records of one
// destination are contiguous; each destination box is then produced by one
// CTA that gathers its sources and sums their terms in registers, and written
// exactly once.  No atomics touch the result.
#include <cmath>
#include <algorithm>

#include <cub/cub.cuh>

#include "apply_internal.cuh"
#include "mlp.cuh"

namespace mra {

namespace {

__global__ void iota_kernel(int64_t n, int *p) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int)i;
}

__global__ void square_kernel(int64_t n, const double *a, double *b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i] * a[i];
}

__global__ void max_kernel_single(int64_t n, const double *a, double *out) {
  __shared__ double red[1024];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, a[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- per-box norms
__global__ void box_norm_kernel(int64_t n, int k3, const double *coeffs, double *norms) {
  int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (b >= n) return;
  const double *s = coeffs + b * k3;
  double a = 0.0;
  for (int e = lane; e < k3; e += 32) a += s[e] * s[e];
  a = warp_sum(a);
  if (lane == 0) norms[b] = sqrt(a);
}

// ---------------------------------------------------------------- screen
// One warp per source box.  pass 0 counts records, pass 1 writes them at off[b].
constexpr int LD_Q = 13;  // |l|^2 classes with a stored learned-screen decision (|l|_inf <= 2)
struct ScreenArgs {
  int64_t n_in;
  const uint64_t *keys;
  const double *snorm;
  int M;
  const double *c;
  const double *N;            // block norms
  const int *Dlev;            // operator D per absolute level
  const int64_t *level_off;   // operator first block per absolute level (-1 absent)
  int stencil, dmax, screen;
  double tau;
  // outputs
  int *dstop;
  int64_t *cnt;               // records per box (pass 0)
  const int64_t *off;         // record offsets (pass 1)
  uint64_t *rec_key;
  int *rec_src;
  int *rec_l;                 // packed (lx+128) | (ly+128)<<8 | (lz+128)<<16
  uint64_t *rec_mask;         // 2 words per record
  int64_t *box_kept, *box_screened;
  double *box_skipped;
  int *box_trunc;
  int *err;
  int64_t rec_cap;            // records the workspace holds (index checks of the checking build)
  uint64_t dest_lo, dest_hi;  // keep destinations with keys in [dest_lo, dest_hi); dest_hi = 0: all
  // learned screen (MRA_SCREEN_LEARNED): drop a kept term when mlp(features) < learned_cut
  const float *mlp;
  const double *t;            // Gaussian exponents (features)
  float learned_cut[MRA_MAX_LEVEL + 1];  // per source level: log10(tau) - delta (-inf: keep all)
  int64_t *box_learned;
  double *box_lbound;
  // pass 0 stores the kept-term mask of every (box, l) it screens, l at index
  // ((lx + dmax) S + ly + dmax) S + lz + dmax with S = 2 dmax + 1; pass 1 writes the records
  // from these masks (the same decisions, nothing recomputed)
  uint64_t *box_mask;         // [n_in][S^3][2]
  // exact filter of the bound in log2 (pass 0): FP32 log2 of every block norm (indexed like N)
  // and of every |c_m|; a term is decided from the FP32 sum of the five logs when it lies more
  // than SCREEN_LMARGIN from log2(tau), else from the FP64 product
  const float *lN, *lc;
  int lfilter;
  float ltau_hi, ltau_lo;
  // several functions in one apply: boxes [fn_off[f], fn_off[f+1]) belong to function f,
  // and records sort on (f, level, x, y, z) packed as f<<53 | n<<48 | x<<32 | y<<16 | z
  int nfunc;
  const int64_t *fn_off;
};

// Margin (in log2) of the screen's FP32 filter.  The five FP32 logs of a bound are each within
// half an ulp (<= 2^-14 for |log2| < 2048) of the true ones and the four FP32 additions of sums
// below 2^13 in magnitude each add at most 2^-12: at most 1.3e-3 in all, under the margin, so a
// term the filter decides is decided as the FP64 product would decide it.
constexpr float SCREEN_LMARGIN = 1.0f / 256.0f;

// FP32 log2 of the block norms and of |c_m| (-inf for 0), for the screen's filter.
__global__ void screen_log_tables_kernel(int64_t n_blocks, int M, const double *N, const double *c, float *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_blocks + M; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = i < n_blocks ? N[i] : fabs(c[i - n_blocks]);
    out[i] = v > 0.0 ? (float)log2(v) : -INFINITY;
  }
}

// Sort key of a destination box of function f in a batched apply (levels <= 15).
__device__ __forceinline__ uint64_t batched_key(int f, int n, int64_t x, int64_t y, int64_t z) {
  return ((uint64_t)f << 53) | ((uint64_t)n << 48) | ((uint64_t)x << 32) | ((uint64_t)y << 16) | (uint64_t)z;
}
__device__ __forceinline__ uint64_t public_key(uint64_t bk) {
  return make_key((int)((bk >> 48) & 31), (int64_t)((bk >> 32) & 0xFFFF), (int64_t)((bk >> 16) & 0xFFFF),
                  (int64_t)(bk & 0xFFFF));
}

// PASS 0 screens and counts (LEARNED: with the learned screen), PASS 1 writes the records.
template <int PASS, bool LEARNED = false>
__global__ void __launch_bounds__(256, LEARNED ? 1 : 2) screen_kernel(ScreenArgs a) {
  extern __shared__ __align__(16) float mlp_sh[];  // the learned screen's parameters, when used
  __shared__ uint64_t drop_sh[8][LD_Q][2];  // per warp: learned-screen drop bits by |l|^2 class
  const float *mlp = LEARNED ? a.mlp : nullptr;
  if (mlp && PASS == 0) {
    for (int i = threadIdx.x; i < MLP_NALL; i += blockDim.x) mlp_sh[i] = mlp[i];
    __syncthreads();
  }
  int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  if (b >= a.n_in) return;
  uint64_t key = a.keys[b];
  int n = key_level(key);
  int64_t x = key_x(key), y = key_y(key), z = key_z(key);
  int64_t nb = 1LL << n;
  if (a.level_off[n] < 0) {
    if (lane == 0 && PASS == 0) atomicExch(a.err, 1);  // level outside the operator's table
    return;
  }
  int func = 0;
  if (a.nfunc > 1) {
    if (n > 15) {
      if (lane == 0 && PASS == 0) atomicExch(a.err, 3);  // batched sort keys hold levels <= 15
      return;
    }
    int lo = 0, hi = a.nfunc - 1;  // last f with fn_off[f] <= b
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (a.fn_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    func = lo;
  }
  int Dop = a.Dlev[n];
  int D = a.stencil == MRA_STENCIL_NEAREST ? 1 : a.dmax;
  if (D > Dop) D = Dop;
  if (D > nb - 1) D = (int)(nb - 1);
  const int S = 2 * a.dmax + 1;
  uint64_t *bmask = a.box_mask + (size_t)b * S * S * S * 2;
  auto mask_at = [&](int lx, int ly, int lz) {
    return bmask + (((lx + a.dmax) * S + ly + a.dmax) * S + lz + a.dmax) * 2;
  };
  if (PASS == 1) {
    // the records, in pass 0's order, from its masks: shells before the one it stopped at
    int64_t wpos = a.off[b];
    const int dstop = a.dstop[b];
    for (int d = 0; d <= D && d < dstop; ++d)
      for (int lx = -d; lx <= d; ++lx)
        for (int ly = -d; ly <= d; ++ly)
          for (int lz = -d; lz <= d; ++lz) {
            if (max(abs(lx), max(abs(ly), abs(lz))) != d) continue;
            if (x + lx < 0 || x + lx >= nb || y + ly < 0 || y + ly >= nb || z + lz < 0 || z + lz >= nb) continue;
            const uint64_t tkey = make_key(n, x + lx, y + ly, z + lz);
            if (!(a.dest_hi == 0 || (tkey >= a.dest_lo && tkey < a.dest_hi))) continue;
            const uint64_t *mk = mask_at(lx, ly, lz);
            const uint64_t m0 = mk[0], m1 = mk[1];
            if (!(m0 | m1)) continue;
            if (lane == 0) {
              const int64_t wp = MRA_IDX(wpos, a.rec_cap);
              a.rec_key[wp] = a.nfunc > 1 ? batched_key(func, n, x + lx, y + ly, z + lz)
                                          : make_key(n, x + lx, y + ly, z + lz);
              a.rec_src[wp] = (int)b;
              a.rec_l[wp] = (lx + 128) | ((ly + 128) << 8) | ((lz + 128) << 16);
              a.rec_mask[2 * wp] = m0;
              a.rec_mask[2 * wp + 1] = m1;
            }
            ++wpos;
          }
    return;
  }
  int nl = 2 * Dop + 1;
  const double *Nl = a.N + a.level_off[n];
  double sn = a.snorm[b];
  int64_t count = 0, kept = 0, screened = 0, learned = 0;
  double skipped = 0.0, lbound = 0.0;
  const float log_sn = (float)log10(fmax(sn, 1e-300));
  // learned screen: drop bits of every (|l|^2 class, term) this box can meet, by the network
  // (terms the norm screen would drop anyway are never looked up)
  uint64_t(*drop)[2] = drop_sh[wib];
  if (mlp && D <= 2) {
    for (int q = 0; q <= 3 * D * D; ++q) {
      bool occurs = false;  // q = lx^2 + ly^2 + lz^2 with |l|_inf <= D
      for (int u = 0; u <= D; ++u)
        for (int v = 0; v <= D; ++v)
          for (int w = 0; w <= D; ++w) occurs |= u * u + v * v + w * w == q;
      uint64_t w0 = 0ull, w1 = 0ull;
      if (occurs) {
        for (int m0 = 0; m0 < a.M; m0 += 32) {
          const int m = m0 + lane;
          bool dr = false;
          if (m < a.M) {
            float f[4] = {(float)n, sqrtf((float)q), (float)log10(a.t[m]), log_sn};
            dr = mlp_predict(mlp_sh, f) < a.learned_cut[n];
          }
          const uint64_t bal = (uint64_t)__ballot_sync(0xffffffffu, dr) << (m0 & 63);
          if (m0 < 64) w0 |= bal; else w1 |= bal;
        }
      }
      if (lane == 0) {
        drop[q][0] = w0;
        drop[q][1] = w1;
      }
    }
    __syncwarp();
  }
  // log2 |c_m| of this lane's terms (m = 32 j + lane), log2 of the box norm
  float lcm[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) lcm[j] = a.lfilter && 32 * j + lane < a.M ? a.lc[32 * j + lane] : 0.f;
  const float lsn = sn > 0.0 ? (float)log2(sn) : -INFINITY;
  const float *lNl = a.lfilter ? a.lN + a.level_off[n] : nullptr;
  // the bounds of terms the filter drops, as an FP32 sum per lane, and how many (its rounding
  // bound: a sum of n non-negative FP32 terms is within (n - 1) 2^-24 of its value)
  float skipped32 = 0.f;
  int n32 = 0;
  // the FP64 bound (((|c_m| N_x) N_y) N_z) |s_b|, in the oracle's order
  auto bound64 = [&](int m, int lx, int ly, int lz) {
    return fabs(a.c[m]) * Nl[m * nl + lx + Dop] * Nl[m * nl + ly + Dop] * Nl[m * nl + lz + Dop] * sn;
  };
  int d;
  for (d = 0; d <= D; ++d) {
    int any = 0;
    for (int lx = -d; lx <= d; ++lx)
      for (int ly = -d; ly <= d; ++ly) {
        if (x + lx < 0 || x + lx >= nb || y + ly < 0 || y + ly >= nb) continue;
        // log2 of the bound's first three factors, the same for every l_z
        float lq[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m = 32 * j + lane;
          lq[j] = a.lfilter && m < a.M ? (lcm[j] + lNl[m * nl + lx + Dop]) + lNl[m * nl + ly + Dop] : 0.f;
        }
        for (int lz = -d; lz <= d; ++lz) {
          int m_inf = max(abs(lx), max(abs(ly), abs(lz)));
          if (m_inf != d) continue;
          if (z + lz < 0 || z + lz >= nb) continue;
          // destinations outside the caller's key range are screened (so that the shell logic
          // is that of the whole apply) but neither counted nor emitted
          const uint64_t tkey = make_key(n, x + lx, y + ly, z + lz);
          const bool owned = a.dest_hi == 0 || (tkey >= a.dest_lo && tkey < a.dest_hi);
          uint64_t mask[2] = {0ull, 0ull};
          bool norm_kept = false;  // any term of this l passes the norm screen
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int m0 = 32 * j;
            if (m0 >= a.M) break;
            const int m = m0 + lane;
            bool keep = false;
            double B = 0.0;
            bool have_B = false;   // B holds the FP64 bound
            float b_up = 0.f;      // an upper bound of the bound, where the filter dropped the term
            bool dropped_by_model = false;
            if (m < a.M) {
              if (a.screen == MRA_SCREEN_NONE) {
                keep = true;
              } else {
                bool decided = false;
                if (a.lfilter) {
                  const float lb = (lq[j] + lNl[m * nl + lz + Dop]) + lsn;
                  if (lb >= a.ltau_hi) {
                    keep = decided = true;
                  } else if (lb < a.ltau_lo) {
                    decided = true;
                    b_up = fmaxf(exp2f(lb + SCREEN_LMARGIN), 1.5e-45f);
                  }
                }
                if (!decided) {
                  B = bound64(m, lx, ly, lz);
                  have_B = true;
                  keep = B >= a.tau;
                }
              }
              if (keep && mlp) {
                const int q = lx * lx + ly * ly + lz * lz;
                bool dr;
                if (D <= 2) {
                  dr = (drop[q][m >> 6] >> (m & 63)) & 1ull;
                } else {  // wide stencils: evaluate the network for this term
                  float f[4] = {(float)n, sqrtf((float)q), (float)log10(a.t[m]), log_sn};
                  dr = mlp_predict((const float *)mlp_sh, f) < a.learned_cut[n];
                }
                if (dr) {
                  keep = false;
                  dropped_by_model = true;
                  if (!have_B) B = bound64(m, lx, ly, lz);
                }
              }
            }
            if (owned) {  // per-lane sums, reduced over the warp once per box
              if (mlp) {
                learned += __popc(__ballot_sync(0xffffffffu, dropped_by_model));
                if (dropped_by_model) lbound += B;
              }
              if (m < a.M && !keep && !dropped_by_model) {
                if (have_B) {
                  skipped += B;
                } else {
                  skipped32 += b_up;
                  ++n32;
                }
              }
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            mask[j >> 1] |= (uint64_t)bal << (m0 & 63);
            if (mlp) norm_kept |= __ballot_sync(0xffffffffu, keep || dropped_by_model) != 0u;
          }
          // the shells follow the norm screen: the learned screen removes terms it kept, and a shell
          // whose kept terms it all removes does not end the shells (their terms count as its drops)
          if (norm_kept) any = 1;
          if (owned && lane == 0) {
            uint64_t *mk = mask_at(lx, ly, lz);
            mk[0] = mask[0];
            mk[1] = mask[1];
          }
          int pk = __popcll(mask[0]) + __popcll(mask[1]);
          if (pk == 0) {
            if (owned) screened += a.M;
            continue;
          }
          any = 1;
          if (!owned) continue;
          kept += pk;
          screened += a.M - pk;
          ++count;
        }
      }
    if (a.stencil == MRA_STENCIL_SHELLS && !any) break;
  }
  skipped += (double)skipped32 * (1.0 + n32 * 0x1p-24);
  skipped = warp_sum(skipped);
  lbound = warp_sum(lbound);
  if (lane == 0) {
    a.cnt[b] = count;
    a.dstop[b] = d;
    a.box_kept[b] = kept;
    a.box_screened[b] = screened;
    a.box_skipped[b] = skipped;
    a.box_trunc[b] = (a.stencil == MRA_STENCIL_SHELLS && d == D + 1) ? 1 : 0;
    a.box_learned[b] = learned;
    a.box_lbound[b] = lbound;
  }
}

// ---------------------------------------------------------------- destination segments
__global__ void head_flags_kernel(int64_t P, const uint64_t *skey, int *head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  head[i] = (i == 0 || skey[i] != skey[i - 1]) ? 1 : 0;
}

__global__ void segments_kernel(int64_t P, const uint64_t *skey, const int *head,
                                const int *dest_id /*inclusive scan*/, uint64_t *dest_key,
                                int64_t *seg, int64_t *n_dest, int batched, int *dest_func) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  if (head[i]) {
    int64_t d = dest_id[i] - 1;
    dest_key[d] = batched ? public_key(skey[i]) : skey[i];
    if (batched) dest_func[d] = (int)(skey[i] >> 53);
    seg[d] = i;
  }
  if (i == P - 1) {
    *n_dest = dest_id[i];
    seg[dest_id[i]] = P;
  }
}

// offsets[f] = first destination of function f (dest_func is sorted), offsets[nfunc] = n
__global__ void func_offsets_kernel(int64_t n, const int *dest_func, int nfunc, int64_t *offsets) {
  for (int f = threadIdx.x; f <= nfunc; f += blockDim.x) {
    int64_t lo = 0, hi = n;  // first index with dest_func >= f
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (dest_func[mid] < f) lo = mid + 1; else hi = mid;
    }
    offsets[f] = lo;
  }
}

// ---------------------------------------------------------------- FP64 gather-apply
// One CTA per destination box.  For each of its records (source b, l, mask)
// and each kept term m:  t1 = s x_1 Rx, t2 = t1 x_2 Ry, t3 = t2 x_3 Rz,
// acc += c_m t3 (Sec. 2.3), acc held in registers across all records.
// PT accumulators per thread: k^3 <= 256 PT (PT = 16 up to k = 16, 32 for the non-standard
// form's orders up to 20).
constexpr int F64_THREADS = 256;

template <int PT>
__global__ void __launch_bounds__(F64_THREADS) apply_f64_kernel(
    int k, int M, const double *c, const double *R, const int *Dlev, const int64_t *level_off,
    const uint64_t *in_keys, const double *in_coeffs, const int64_t *seg, const int *perm,
    const int *rec_src, const int *rec_l, const uint64_t *rec_mask, const uint64_t *dest_key,
    uint64_t *out_keys, double *out_coeffs, int64_t n_src, int64_t n_rec, int64_t n_blocks) {
  extern __shared__ double sm[];
  int k2 = k * k, k3 = k2 * k;
  double *s = sm, *t1 = s + k3, *t2 = t1 + k3, *Rs = t2 + k3;  // Rs: 3 * k2
  int64_t dst = blockIdx.x;
  uint64_t dkey = dest_key[dst];
  int n = key_level(dkey);
  int Dop = Dlev[n];
  int nl = 2 * Dop + 1;
  double acc[PT];
#pragma unroll
  for (int q = 0; q < PT; ++q) acc[q] = 0.0;
  int64_t r0 = seg[dst], r1 = seg[dst + 1];
  for (int64_t r = r0; r < r1; ++r) {
    int p = MRA_IDX(perm[MRA_IDX(r, n_rec)], n_rec);
    int src = MRA_IDX(rec_src[p], n_src);
    int lp = rec_l[p];
    int lx = (lp & 255) - 128, ly = ((lp >> 8) & 255) - 128, lz = ((lp >> 16) & 255) - 128;
    uint64_t mk[2] = {rec_mask[2 * (int64_t)p], rec_mask[2 * (int64_t)p + 1]};
    __syncthreads();
    const double *sb = in_coeffs + (int64_t)src * k3;
    for (int e = threadIdx.x; e < k3; e += blockDim.x) s[e] = sb[e];
    for (int w = 0; w < 2; ++w) {
      uint64_t bits = mk[w];
      while (bits) {
        int m = w * 64 + __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        __syncthreads();
        const int64_t lo = level_off[n];
        const double *Rx = R + MRA_IDX(lo + (int64_t)m * nl + lx + Dop, n_blocks) * k2;
        const double *Ry = R + MRA_IDX(lo + (int64_t)m * nl + ly + Dop, n_blocks) * k2;
        const double *Rz = R + MRA_IDX(lo + (int64_t)m * nl + lz + Dop, n_blocks) * k2;
        for (int e = threadIdx.x; e < k2; e += blockDim.x) {
          Rs[e] = Rx[e];
          Rs[k2 + e] = Ry[e];
          Rs[2 * k2 + e] = Rz[e];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // t1[ix][jy][jz]
          int ix = e / k2, rest = e % k2;
          double v = 0.0;
          for (int j = 0; j < k; ++j) v += Rs[ix * k + j] * s[j * k2 + rest];
          t1[e] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < k3; e += blockDim.x) {  // t2[ix][iy][jz]
          int ix = e / k2, iy = (e / k) % k, jz = e % k;
          double v = 0.0;
          for (int j = 0; j < k; ++j) v += Rs[k2 + iy * k + j] * t1[ix * k2 + j * k + jz];
          t2[e] = v;
        }
        __syncthreads();
        double cm = c[m];
#pragma unroll
        for (int q = 0; q < PT; ++q) {  // acc += c_m t3[ix][iy][iz]
          int e = threadIdx.x + q * F64_THREADS;
          if (e < k3) {
            int base = (e / k) * k, iz = e % k;
            double v = 0.0;
            for (int j = 0; j < k; ++j) v += Rs[2 * k2 + iz * k + j] * t2[base + j];
            acc[q] += cm * v;
          }
        }
      }
    }
  }
  double *o = out_coeffs + dst * k3;
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    int e = threadIdx.x + q * F64_THREADS;
    if (e < k3) o[e] = acc[q];
  }
  if (threadIdx.x == 0) out_keys[dst] = dkey;
}

// ---------------------------------------------------------------- compare
// For each test box: squared norms of test, of the matching ref box (by key)
// and of their difference.  Boxes only in ref are handled by ref_only_kernel.
__global__ void compare_kernel(int64_t nt, const uint64_t *tk, const double *tc, int64_t nr,
                               const uint64_t *rk, const double *rc, int k3, double *d2,
                               double *t2, double *r2, double *rel, int *match) {
  int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (b >= nt) return;
  uint64_t key = tk[b];
  int64_t lo = 0, hi = nr - 1, pos = -1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    uint64_t v = rk[mid];
    if (v == key) { pos = mid; break; }
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  const double *a = tc + b * k3;
  const double *r = pos >= 0 ? rc + pos * k3 : nullptr;
  double sd = 0.0, st = 0.0, sr = 0.0;
  for (int e = lane; e < k3; e += 32) {
    double av = a[e], rv = r ? r[e] : 0.0;
    sd += (av - rv) * (av - rv);
    st += av * av;
    sr += rv * rv;
  }
  sd = warp_sum(sd);
  st = warp_sum(st);
  sr = warp_sum(sr);
  if (lane == 0) {
    d2[b] = sd;
    t2[b] = st;
    r2[b] = sr;
    rel[b] = pos >= 0 ? (sr > 0.0 ? sqrt(sd / sr) : (sd > 0.0 ? INFINITY : 0.0)) : 0.0;
    match[b] = pos >= 0 ? 1 : 0;
  }
}

// Per source level: boxes and kept triples (a shared-memory histogram per CTA, then one
// integer atomic per level: the sums are exact whatever the order).
__global__ void level_counts_kernel(int64_t n, const uint64_t *keys, const int64_t *kept, int64_t *lev) {
  __shared__ unsigned long long hb[MRA_MAX_LEVEL + 1], ht[MRA_MAX_LEVEL + 1];
  if (threadIdx.x <= MRA_MAX_LEVEL) hb[threadIdx.x] = ht[threadIdx.x] = 0ull;
  __syncthreads();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int l = key_level(keys[b]);
    atomicAdd(&hb[l], 1ull);
    atomicAdd(&ht[l], (unsigned long long)kept[b]);
  }
  __syncthreads();
  if (threadIdx.x <= MRA_MAX_LEVEL) {
    if (hb[threadIdx.x]) atomicAdd((unsigned long long *)&lev[threadIdx.x], hb[threadIdx.x]);
    if (ht[threadIdx.x]) atomicAdd((unsigned long long *)&lev[MRA_MAX_LEVEL + 1 + threadIdx.x], ht[threadIdx.x]);
  }
}

// The checking build's self test: one index outside its range through MRA_IDX.
__global__ void debug_selftest_kernel(int *sink) {
  const int i = MRA_IDX(5, 3);
  sink[i] = 1;
}

// Fixed-size (graph) mode: the record count the screen computed against the captured one.
__global__ void fixed_count_check_kernel(const int64_t *off, const int64_t *cnt, int64_t n_in, int64_t P,
                                         const int *d_err, int *status) {
  int st = 0;
  if (off[n_in - 1] + cnt[n_in - 1] != P) st |= 1;
  if (*d_err) st |= 4;
  if (st) atomicOr(status, st);
}
__global__ void fixed_dest_check_kernel(const int64_t *ndest, int64_t nd, int *status) {
  if (*ndest != nd) atomicOr(status, 2);
}

// One CTA per level n: the sum of v over the boxes of level n (keys sorted, so the level's boxes
// are contiguous), reduced in a fixed order (deterministic).
__global__ void level_sum_kernel(int64_t n, const uint64_t *keys, const double *v, double *out,
                                 int64_t *count) {
  __shared__ double red[32];
  const int lev = blockIdx.x;
  auto lower = [&](uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const int64_t b0 = lower((uint64_t)lev << 57);
  const int64_t b1 = lev >= MRA_MAX_LEVEL ? n : lower((uint64_t)(lev + 1) << 57);
  double s = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += v[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[lev] = t;
    if (count) count[lev] = b1 - b0;
  }
}

__global__ void ref_only_kernel(int64_t nr, const uint64_t *rk, const double *rc, int64_t nt,
                                const uint64_t *tk, int k3, double *r2_all, double *r2_only,
                                int *only) {
  int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (b >= nr) return;
  uint64_t key = rk[b];
  int64_t lo = 0, hi = nt - 1;
  bool found = false;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    uint64_t v = tk[mid];
    if (v == key) { found = true; break; }
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  const double *r = rc + b * k3;
  double s = 0.0;
  for (int e = lane; e < k3; e += 32) s += r[e] * r[e];
  s = warp_sum(s);
  if (lane == 0) {
    r2_all[b] = s;
    r2_only[b] = found ? 0.0 : s;
    only[b] = found ? 0 : 1;
  }
}

}  // namespace

// ============================================================== host side

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

int apply_max_disp(const Operator &op, const mra_apply_opts &o) {
  int D = o.stencil == MRA_STENCIL_NEAREST ? 1 : o.max_disp;
  if (D > op.max_disp) D = op.max_disp;
  if (D < 0) D = 0;
  return D;
}

int64_t apply_max_records(const Operator &op, const mra_apply_opts &o, int64_t n_in) {
  int64_t w = 2 * apply_max_disp(op, o) + 1;
  return n_in * w * w * w;
}

// Workspace layout (all offsets 256-byte aligned):
//   per box: snorm, dstop, cnt, off, kept, screened, skipped, trunc, learned, lbound, and the
//     screen's kept-term masks of its (2 dmax + 1)^3 displacements
//   per record: key, src, l, mask[2], sorted key, perm in/out, head, dest id
//   per destination (<= records): dest key, seg (+1)
//   CUB temp storage (max over scan / sort / reduce needs)
struct Layout {
  size_t snorm, dstop, cnt, off, kept, screened, skipped, trunc, learned, lbound, bmask, ltab;
  size_t rkey, rsrc, rl, rmask, skey, pin, pout, head, did, dkey, seg, ndest, dfunc, fnoff, lev, split, tmp;
  size_t split_bytes, tmp_bytes, total;
};

static Layout make_layout(int64_t n_in, int64_t P, int dmax, int64_t n_tab, bool src_path = false) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + (bytes ? bytes : 1));
    return at;
  };
  int64_t nb = n_in > 0 ? n_in : 1, np = P > 0 ? P : 1;
  L.snorm = take(nb * 8);
  L.dstop = take(nb * 4);
  L.cnt = take(nb * 8);
  L.off = take(nb * 8);
  L.kept = take(nb * 8);
  L.screened = take(nb * 8);
  L.skipped = take(nb * 8);
  L.trunc = take(nb * 4);
  L.learned = take(nb * 8);
  L.lbound = take(nb * 8);
  const int64_t S = 2 * (int64_t)dmax + 1;
  L.bmask = take(nb * S * S * S * 16);
  L.ltab = take((size_t)n_tab * 4);
  L.rkey = take(np * 8);
  L.rsrc = take(np * 4);
  L.rl = take(np * 4);
  L.rmask = take(np * 16);
  L.skey = take(np * 8);
  L.pin = take(np * 4);
  L.pout = take(np * 4);
  L.head = take(np * 4);
  L.did = take(np * 4);
  L.dkey = take(np * 8);
  L.seg = take((np + 1) * 8);
  L.ndest = take(8);
  L.dfunc = take(np * 4);
  L.fnoff = take((MRA_MAX_FUNCS + 1) * 8);
  L.lev = take(2 * (MRA_MAX_LEVEL + 1) * 8);
  L.split_bytes = src_path ? std::max(split_workspace_bytes(np), src_workspace_bytes(nb)) : split_workspace_bytes(np);
  L.split = take(L.split_bytes);
  // CUB temporary storage: the largest of the calls below
  size_t a = 0, b = 0, c = 0, d = 0, e = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, a, (int64_t *)nullptr, (int64_t *)nullptr, (int)nb);
  cub::DeviceScan::InclusiveSum(nullptr, b, (int *)nullptr, (int *)nullptr, (int)np);
  cub::DeviceRadixSort::SortPairs(nullptr, c, (uint64_t *)nullptr, (uint64_t *)nullptr,
                                  (int *)nullptr, (int *)nullptr, (int)np);
  cub::DeviceReduce::Sum(nullptr, d, (double *)nullptr, (double *)nullptr, (int)nb);
  cub::DeviceReduce::Sum(nullptr, e, (int64_t *)nullptr, (int64_t *)nullptr, (int)nb);
  size_t t = a;
  for (size_t v : {b, c, d, e}) t = v > t ? v : t;
  L.tmp_bytes = t;
  L.tmp = take(t);
  L.total = o;
  return L;
}

// The records' largest |l|_inf on level n: the stencil's radius within the operator's and the cell's.
static int records_disp(const Operator &op, const mra_apply_opts &o, int n) {
  int D = apply_max_disp(op, o);
  if (n < op.min_level || n > op.max_level) return 0;
  const int Dop = op.D[n - op.min_level];
  if (D > Dop) D = Dop;
  if ((int64_t)D > (1LL << n) - 1) D = (int)((1LL << n) - 1);
  return D;
}

bool apply_uses_src_path(const Operator &op, const mra_apply_opts &o) {
  if (o.precision != MRA_PREC_SPLIT_BF16 || o.split_kernel == MRA_SPLIT_DEST) return false;
  int dmax = 0;
  for (int n = op.min_level; n <= op.max_level; ++n) dmax = std::max(dmax, records_disp(op, o, n));
  return src_path_supported(op.k, dmax);
}

size_t apply_workspace_bytes(const Operator &op, const mra_apply_opts &o, int64_t n_in) {
  return make_layout(n_in, apply_max_records(op, o, n_in), apply_max_disp(op, o), op.n_blocks + op.M,
                     apply_uses_src_path(op, o)).total;
}

// Pointers into a carved workspace.
struct WsPtrs {
  double *snorm;
  int *dstop;
  int64_t *cnt, *off, *bkept, *bscr, *blearned;
  double *bskip, *blbound;
  uint64_t *bmask;
  float *ltab;
  int *btrunc;
  uint64_t *rkey, *skey, *rmask, *dkey;
  int *rsrc, *rl, *pin, *pout, *head, *did;
  int64_t *seg, *ndest;
  int *dfunc;
  int64_t *fnoff;
  int64_t *lev;  // per level: source boxes, kept triples
  void *tmp;
  size_t tmpb;
};

static WsPtrs carve(const Layout &L, void *ws) {
  char *w = (char *)ws;
  WsPtrs p{};
  p.snorm = (double *)(w + L.snorm);
  p.dstop = (int *)(w + L.dstop);
  p.cnt = (int64_t *)(w + L.cnt);
  p.off = (int64_t *)(w + L.off);
  p.bkept = (int64_t *)(w + L.kept);
  p.bscr = (int64_t *)(w + L.screened);
  p.bskip = (double *)(w + L.skipped);
  p.btrunc = (int *)(w + L.trunc);
  p.blearned = (int64_t *)(w + L.learned);
  p.blbound = (double *)(w + L.lbound);
  p.bmask = (uint64_t *)(w + L.bmask);
  p.ltab = (float *)(w + L.ltab);
  p.rkey = (uint64_t *)(w + L.rkey);
  p.skey = (uint64_t *)(w + L.skey);
  p.rsrc = (int *)(w + L.rsrc);
  p.rl = (int *)(w + L.rl);
  p.rmask = (uint64_t *)(w + L.rmask);
  p.pin = (int *)(w + L.pin);
  p.pout = (int *)(w + L.pout);
  p.head = (int *)(w + L.head);
  p.did = (int *)(w + L.did);
  p.dkey = (uint64_t *)(w + L.dkey);
  p.seg = (int64_t *)(w + L.seg);
  p.ndest = (int64_t *)(w + L.ndest);
  p.dfunc = (int *)(w + L.dfunc);
  p.fnoff = (int64_t *)(w + L.fnoff);
  p.lev = (int64_t *)(w + L.lev);
  p.tmp = w + L.tmp;
  p.tmpb = L.tmp_bytes;
  return p;
}

// Source norms, norm (and learned) screen, record counts, scan and record emission.
// On return *P_out holds the number of records (written in source order).
static int screen_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o, const WsPtrs &w,
                      int64_t Pmax, mra_apply_stats *stats, int64_t *P_out, cudaStream_t s, int nfunc = 1,
                      const FixedSizes *fx = nullptr) {
  const int k = op.k, k3 = k * k * k;
  const int64_t n_in = in.n;
  // error flag lives in the first word of the dest-count slot until it is used
  int *d_err = (int *)w.ndest;
  MRA_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int64_t), s));
  const int wpb = 8;  // warps per CTA for per-box kernels
  unsigned gboxes = (unsigned)((n_in + wpb - 1) / wpb);
  box_norm_kernel<<<counted(gboxes), 32 * wpb, 0, s>>>(n_in, k3, in.coeffs, w.snorm);
  MRA_CUDA_TRY(cudaGetLastError());

  ScreenArgs a{};
  a.n_in = n_in;
  a.keys = in.keys;
  a.snorm = w.snorm;
  a.M = op.M;
  a.c = op.d_c;
  a.N = op.d_N;
  a.Dlev = op.d_D;
  a.level_off = op.d_level_off;
  a.stencil = o.stencil;
  a.dmax = apply_max_disp(op, o);
  a.screen = o.screen == MRA_SCREEN_LEARNED ? MRA_SCREEN_NORM : o.screen;
  a.tau = o.tau;
  // the log2 filter, where a norm screen runs with a threshold log2 can represent
  a.lfilter = a.screen != MRA_SCREEN_NONE && o.tau > 0.0 && std::isfinite(std::log2(o.tau)) ? 1 : 0;
  if (a.lfilter) {
    const double lt = std::log2(o.tau);
    a.ltau_hi = (float)(lt + SCREEN_LMARGIN);
    a.ltau_lo = (float)(lt - SCREEN_LMARGIN);
    a.lN = w.ltab;
    a.lc = w.ltab + op.n_blocks;
    screen_log_tables_kernel<<<counted((unsigned)std::min<int64_t>((op.n_blocks + op.M + 255) / 256, 1024)), 256, 0,
                               s>>>(op.n_blocks, op.M, op.d_N, op.d_c, w.ltab);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  a.dstop = w.dstop;
  a.cnt = w.cnt;
  a.off = w.off;
  a.rec_key = w.rkey;
  a.rec_src = w.rsrc;
  a.rec_l = w.rl;
  a.rec_mask = w.rmask;
  a.box_kept = w.bkept;
  a.box_screened = w.bscr;
  a.box_skipped = w.bskip;
  a.box_trunc = w.btrunc;
  a.err = d_err;
  a.rec_cap = Pmax;
  a.dest_lo = o.dest_lo;
  a.dest_hi = o.dest_hi;
  a.mlp = o.screen == MRA_SCREEN_LEARNED ? o.mlp : nullptr;
  a.t = op.d_t;
  for (int n = 0; n <= MRA_MAX_LEVEL; ++n) {
    const double dl = o.delta_level ? o.delta_level[n] : o.delta;
    a.learned_cut[n] = isinf(dl) && dl > 0 ? -INFINITY : (float)(log10(o.tau) - dl);
  }
  a.box_learned = w.blearned;
  a.box_lbound = w.blbound;
  a.box_mask = w.bmask;
  a.nfunc = nfunc;
  a.fn_off = w.fnoff;
  const size_t ssm = a.mlp ? (size_t)MLP_NALL * sizeof(float) : 0;
  if (a.mlp)
    screen_kernel<0, true><<<counted(gboxes), 32 * wpb, ssm, s>>>(a);
  else
    screen_kernel<0, false><<<counted(gboxes), 32 * wpb, 0, s>>>(a);
  MRA_CUDA_TRY(cudaGetLastError());
  void *tmp = w.tmp;
  size_t tmpb = w.tmpb;
  MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tmpb, w.cnt, w.off, (int)n_in, s));
  if (fx) {  // graph mode: the captured record count, checked on the device
    fixed_count_check_kernel<<<counted(1), 1, 0, s>>>(w.off, w.cnt, n_in, fx->P, d_err, fx->status);
    MRA_CUDA_TRY(cudaGetLastError());
    if (fx->P > 0) {
      screen_kernel<1><<<counted(gboxes), 32 * wpb, 0, s>>>(a);
      MRA_CUDA_TRY(cudaGetLastError());
    }
    *P_out = fx->P;
    return MRA_OK;
  }
  // statistics reduced on the device (deterministic), read with the record count
  int64_t *red_i = w.seg;  // seg is free until the segments pass
  double *red_d = (double *)(w.seg + 4);
  if (stats) {
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.bkept, red_i + 0, (int)n_in, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.bscr, red_i + 1, (int)n_in, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.btrunc, (int *)(red_i + 2), (int)n_in, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.blearned, red_i + 3, (int)n_in, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.bskip, red_d, (int)n_in, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, w.blbound, red_d + 1, (int)n_in, s));
    MRA_CUDA_TRY(cudaMemsetAsync(w.lev, 0, 2 * (MRA_MAX_LEVEL + 1) * sizeof(int64_t), s));
    level_counts_kernel<<<counted((unsigned)std::min<int64_t>((n_in + 255) / 256, 1024)), 256, 0, s>>>(
        n_in, in.keys, w.bkept, w.lev);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  int64_t h_last[2] = {0, 0};
  int h_err = 0;
  int64_t hs[4] = {0, 0, 0, 0};
  double hd[2] = {0.0, 0.0};
  int64_t hl[2 * (MRA_MAX_LEVEL + 1)] = {};
  MRA_CUDA_TRY(cudaMemcpyAsync(&h_last[0], w.off + n_in - 1, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(&h_last[1], w.cnt + n_in - 1, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (stats) {
    MRA_CUDA_TRY(cudaMemcpyAsync(hs, red_i, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(hd, red_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaMemcpyAsync(hl, w.lev, sizeof(hl), cudaMemcpyDeviceToHost, s));
  }
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (h_err == 3)
    return fail(MRA_ERR_UNSUPPORTED, "mra_apply_batched: levels above 15 are not supported");
  if (h_err)
    return fail(MRA_ERR_ARG, "mra_apply: an input box lies on a level the operator does not cover "
                "(levels %d..%d)", op.min_level, op.max_level);
  const int64_t P = h_last[0] + h_last[1];
  if (P > Pmax) return fail(MRA_ERR_CAPACITY, "mra_apply: internal record bound exceeded");
  if (stats) {
    int ntr = 0;
    memcpy(&ntr, &hs[2], sizeof(int));
    *stats = mra_apply_stats{};
    stats->n_in = n_in;
    stats->terms_kept = hs[0];
    stats->terms_screened = hs[1] - hs[3];  // the norm screen's drops; the model's are below
    stats->sources_truncated = ntr;
    stats->skipped_bound = hd[0];
    stats->pairs = P;
    stats->terms_issued = hs[0];
    stats->terms_learned_skipped = hs[3];
    stats->learned_skipped_bound = hd[1];
    stats->algo_flops = (double)hs[0] * (6.0 * op.k * op.k * op.k * op.k + (double)op.k * op.k * op.k);
    for (int n = 0; n <= MRA_MAX_LEVEL; ++n) {
      stats->level_sources[n] = hl[n];
      stats->level_terms_kept[n] = hl[MRA_MAX_LEVEL + 1 + n];
    }
  }
  if (P > 0) {
    screen_kernel<1><<<counted(gboxes), 32 * wpb, 0, s>>>(a);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  *P_out = P;
  return MRA_OK;
}

int apply_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o,
              mra_tree_view &out, void *ws, size_t ws_bytes, mra_apply_stats *stats,
              cudaStream_t s, int nfunc, const int64_t *in_offsets, int64_t *out_offsets,
              const FixedSizes *fx) {
  const int k = op.k, k3 = k * k * k;
  const int64_t n_in = in.n;
  const int64_t Pmax = apply_max_records(op, o, n_in);
  const bool src_path = apply_uses_src_path(op, o);
  Layout L = make_layout(n_in, Pmax, apply_max_disp(op, o), op.n_blocks + op.M, src_path);
  if (ws_bytes < L.total)
    return fail(MRA_ERR_CAPACITY, "mra_apply: workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  WsPtrs W = carve(L, ws);
  char *w = (char *)ws;
  uint64_t *rkey = W.rkey, *skey = W.skey, *rmask = W.rmask, *dkey = W.dkey;
  int *rsrc = W.rsrc, *rl = W.rl, *pin = W.pin, *pout = W.pout, *head = W.head, *did = W.did;
  int64_t *seg = W.seg, *ndest = W.ndest;
  void *tmp = W.tmp;
  size_t tmpb = W.tmpb;
  if (fx) stats = nullptr;  // graph mode: nothing is read back
  if (out_offsets && !fx)
    for (int f = 0; f <= nfunc; ++f) out_offsets[f] = 0;
  if (n_in == 0) {
    out.n = 0;
    if (stats) *stats = mra_apply_stats{};
    return MRA_OK;
  }
  if (nfunc > 1) {
    if (fx)
      MRA_CUDA_TRY(cudaMemcpyAsync(W.fnoff, fx->d_in_offsets, (nfunc + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    else
      MRA_CUDA_TRY(cudaMemcpyAsync(W.fnoff, in_offsets, (nfunc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }
  int64_t P = 0;
  int rc0 = screen_run(op, in, o, W, Pmax, stats, &P, s, nfunc, fx);
  if (rc0 != MRA_OK) return rc0;
  if (P == 0) {
    out.n = 0;
    return MRA_OK;
  }
  // sort record indices on the destination key
  {
    unsigned g = (unsigned)((P + 255) / 256);
    iota_kernel<<<counted(g), 256, 0, s>>>(P, pin);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmpb, rkey, skey, pin, pout, (int)P, 0, 64, s));
    head_flags_kernel<<<counted(g), 256, 0, s>>>(P, skey, head);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp, tmpb, head, did, (int)P, s));
    segments_kernel<<<counted(g), 256, 0, s>>>(P, skey, head, did, dkey, seg, ndest, nfunc > 1, W.dfunc);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  int64_t nd = 0;
  if (fx) {
    fixed_dest_check_kernel<<<counted(1), 1, 0, s>>>(ndest, fx->nd, fx->status);
    MRA_CUDA_TRY(cudaGetLastError());
    nd = fx->nd;
  } else {
    MRA_CUDA_TRY(cudaMemcpyAsync(&nd, ndest, 8, cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (nd > out.cap) {
    out.n = nd;
    return fail(MRA_ERR_CAPACITY, "mra_apply: output holds %lld boxes, %lld needed",
                (long long)out.cap, (long long)nd);
  }
  if (fx) {
    // graph mode: the output offsets of the sizing run stand
  } else if (nfunc > 1 && out_offsets) {  // first destination of each function (destinations sorted by function)
    func_offsets_kernel<<<counted(1), 256, 0, s>>>(nd, W.dfunc, nfunc, W.fnoff);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cudaMemcpyAsync(out_offsets, W.fnoff, (nfunc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MRA_CUDA_TRY(cudaStreamSynchronize(s));
  } else if (out_offsets) {
    out_offsets[0] = 0;
    out_offsets[1] = nd;
  }
  int rc;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evk0 = nullptr, evk1 = nullptr;
  if (stats) {
    MRA_CUDA_TRY(cudaEventCreate(&ev0));
    MRA_CUDA_TRY(cudaEventCreate(&ev1));
    if (src_path) {
      MRA_CUDA_TRY(cudaEventCreate(&evk0));
      MRA_CUDA_TRY(cudaEventCreate(&evk1));
    }
  }
  ApplyWork wk{};
  wk.n_dest = nd;
  wk.P = P;
  wk.seg = seg;
  wk.perm = pout;
  wk.did = did;
  wk.skey = skey;
  wk.rec_src = rsrc;
  wk.rec_l = rl;
  wk.rec_mask = rmask;
  wk.dest_key = dkey;
  wk.rec_cnt = W.cnt;
  wk.rec_off = W.off;
  wk.box_kept = W.bkept;
  wk.split_ws = w + L.split;
  wk.split_ws_bytes = L.split_bytes;
  wk.ev0 = ev0;
  wk.ev1 = ev1;
  wk.evk0 = evk0;
  wk.evk1 = evk1;
  wk.fx = fx;
  if (stats)
    stats->kernel = o.precision == MRA_PREC_FP64 ? MRA_KERNEL_F64 : src_path ? MRA_KERNEL_SPLIT_SRC : MRA_KERNEL_SPLIT_DEST;
  if (o.precision == MRA_PREC_FP64) {
    if (ev0) MRA_CUDA_TRY(cudaEventRecord(ev0, s));
    size_t smem = (size_t)(3 * k3 + 3 * k * k) * sizeof(double);
    auto kern = k3 <= 16 * F64_THREADS ? apply_f64_kernel<16> : apply_f64_kernel<32>;
    if (smem > 48 * 1024)
      MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<counted((unsigned)nd), F64_THREADS, smem, s>>>(
        k, op.M, op.d_c, op.d_R, op.d_D, op.d_level_off, in.keys, in.coeffs, seg, pout, rsrc, rl,
        rmask, dkey, out.keys, out.coeffs, n_in, P, op.n_blocks);
    MRA_CUDA_TRY(cudaGetLastError());
    if (ev1) MRA_CUDA_TRY(cudaEventRecord(ev1, s));
    rc = MRA_OK;
  } else if (src_path) {
    // the partial sums (one k^3 block of floats per record): the graph's own buffer when
    // recorded, else from the library's memory pool for this call
    int dap[MRA_MAX_LEVEL + 1];
    for (int n = 0; n <= MRA_MAX_LEVEL; ++n) dap[n] = records_disp(op, o, n);
    float *partial = fx ? fx->partial : nullptr;
    if (!fx) MRA_CUDA_TRY(pool_malloc((void **)&partial, (size_t)P * k3 * sizeof(float), s));
    if (!partial) return fail(MRA_ERR_ARG, "mra_apply: no partial-sum buffer for the recorded apply");
    int64_t passes = 0;
    rc = apply_src_run(op, in, o, out, wk, dap, partial, s, &passes);
    if (stats && rc == MRA_OK) stats->mma_passes = passes;
    if (!fx) cudaFreeAsync(partial, s);
    if (rc != MRA_OK) return rc;
  } else {
    rc = apply_split_run(op, in, o, out, wk, stats, s);
    if (rc != MRA_OK) return rc;
  }
  out.n = nd;
  if (stats) {
    stats->n_out = nd;
    MRA_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.0f;
    MRA_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    stats->kernel_ms = ms;
    stats->main_kernel_ms = ms;
    if (evk0) {
      MRA_CUDA_TRY(cudaEventElapsedTime(&ms, evk0, evk1));
      stats->main_kernel_ms = ms;
      cudaEventDestroy(evk0);
      cudaEventDestroy(evk1);
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  return rc;
}


// ---------------------------------------------------------------- training-data logging
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ bool sampled(uint64_t seed, int64_t p, int m, uint64_t thr) {
  return mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(p * 128 + m + 1)) <= thr;
}

__global__ void sample_count_kernel(int64_t P, const uint64_t *rmask, uint64_t seed, uint64_t thr,
                                    int64_t *cnt) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t c = 0;
  for (int w = 0; w < 2; ++w) {
    uint64_t bits = rmask[2 * p + w];
    while (bits) {
      int m = w * 64 + __ffsll((long long)bits) - 1;
      bits &= bits - 1;
      c += sampled(seed, p, m, thr) ? 1 : 0;
    }
  }
  cnt[p] = c;
}

// term list, stashed as ints in the feature rows until term_norm_kernel replaces them
__global__ void sample_write_kernel(int64_t P, const uint64_t *rmask, const int *rsrc, const int *rl,
                                    uint64_t seed, uint64_t thr, const int64_t *off, int64_t max_terms,
                                    float *features) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int64_t idx = off[p];
  for (int w = 0; w < 2; ++w) {
    uint64_t bits = rmask[2 * p + w];
    while (bits) {
      int m = w * 64 + __ffsll((long long)bits) - 1;
      bits &= bits - 1;
      if (!sampled(seed, p, m, thr)) continue;
      if (idx < max_terms) {
        int *row = (int *)(features + idx * 4);
        row[0] = rsrc[p];
        row[1] = rl[p];
        row[2] = m;
      }
      ++idx;
    }
  }
}

// One CTA per logged term: its features and log10 ||c_m (Rx x Ry x Rz) s_b||_F in FP64.
__global__ void term_norm_kernel(int k, const double *c, const double *t, const double *R, const int *Dlev,
                                 const int64_t *level_off, const uint64_t *keys, const double *coeffs,
                                 const double *snorm, float *features, float *log_norms) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ int info[3];
  const int k2 = k * k, k3 = k2 * k;
  double *s = sm, *t1 = s + k3, *t2 = t1 + k3, *Rs = t2 + k3;
  const int64_t q = blockIdx.x;
  if (threadIdx.x < 3) info[threadIdx.x] = ((const int *)(features + q * 4))[threadIdx.x];
  __syncthreads();
  const int src = info[0], lp = info[1], m = info[2];
  const int lx = (lp & 255) - 128, ly = ((lp >> 8) & 255) - 128, lz = ((lp >> 16) & 255) - 128;
  const int n = key_level(keys[src]);
  const int Dop = Dlev[n], nl = 2 * Dop + 1;
  const double *Rlev = R + level_off[n] * k2;
  const double *Rx = Rlev + ((int64_t)m * nl + lx + Dop) * k2;
  const double *Ry = Rlev + ((int64_t)m * nl + ly + Dop) * k2;
  const double *Rz = Rlev + ((int64_t)m * nl + lz + Dop) * k2;
  for (int e = threadIdx.x; e < k3; e += blockDim.x) s[e] = coeffs[(int64_t)src * k3 + e];
  for (int e = threadIdx.x; e < k2; e += blockDim.x) {
    Rs[e] = Rx[e];
    Rs[k2 + e] = Ry[e];
    Rs[2 * k2 + e] = Rz[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    int ix = e / k2, rest = e % k2;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Rs[ix * k + j] * s[j * k2 + rest];
    t1[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    int ix = e / k2, iy = (e / k) % k, jz = e % k;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Rs[k2 + iy * k + j] * t1[ix * k2 + j * k + jz];
    t2[e] = v;
  }
  __syncthreads();
  double acc = 0.0;
  for (int e = threadIdx.x; e < k3; e += blockDim.x) {
    int base = (e / k) * k, iz = e % k;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += Rs[2 * k2 + iz * k + j] * t2[base + j];
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    double norm = fabs(c[m]) * sqrt(tot);
    log_norms[q] = (float)log10(fmax(norm, 1e-300));
    features[q * 4 + 0] = (float)n;
    features[q * 4 + 1] = sqrtf((float)(lx * lx + ly * ly + lz * lz));
    features[q * 4 + 2] = (float)log10(t[m]);
    features[q * 4 + 3] = (float)log10(fmax(snorm[src], 1e-300));
  }
}

}  // namespace

int log_terms_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o, int64_t max_terms,
                  uint64_t seed, float *features, float *log_norms, int64_t *n_logged, void *ws,
                  size_t ws_bytes, cudaStream_t s) {
  *n_logged = 0;
  const int64_t n_in = in.n;
  if (n_in == 0 || max_terms <= 0) return MRA_OK;
  const int64_t Pmax = apply_max_records(op, o, n_in);
  Layout L = make_layout(n_in, Pmax, apply_max_disp(op, o), op.n_blocks + op.M);
  if (ws_bytes < L.total)
    return fail(MRA_ERR_CAPACITY, "mra_log_terms: workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  WsPtrs W = carve(L, ws);
  mra_apply_stats st{};
  int64_t P = 0;
  int rc = screen_run(op, in, o, W, Pmax, &st, &P, s);
  if (rc != MRA_OK || P == 0) return rc;
  const double frac = (double)max_terms / (double)(st.terms_kept > 0 ? st.terms_kept : 1);
  const uint64_t thr = frac >= 1.0 ? ~0ull : (uint64_t)(frac * 18446744073709551615.0);
  int64_t *cnt = (int64_t *)W.rkey, *off = (int64_t *)W.skey;  // free until a sort runs
  unsigned g = (unsigned)((P + 255) / 256);
  sample_count_kernel<<<counted(g), 256, 0, s>>>(P, W.rmask, seed, thr, cnt);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceScan::ExclusiveSum(W.tmp, W.tmpb, cnt, off, (int)P, s));
  int64_t last[2];
  MRA_CUDA_TRY(cudaMemcpyAsync(&last[0], off + P - 1, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(&last[1], cnt + P - 1, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t total = last[0] + last[1];
  const int64_t nlog = total < max_terms ? total : max_terms;
  if (nlog == 0) return MRA_OK;
  sample_write_kernel<<<counted(g), 256, 0, s>>>(P, W.rmask, W.rsrc, W.rl, seed, thr, off, max_terms, features);
  MRA_CUDA_TRY(cudaGetLastError());
  const int k = op.k;
  size_t smem = (size_t)(3 * k * k * k + 3 * k * k) * sizeof(double);
  if (smem > 48 * 1024)
    MRA_CUDA_TRY(cudaFuncSetAttribute(term_norm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  term_norm_kernel<<<counted((unsigned)nlog), 256, smem, s>>>(k, op.d_c, op.d_t, op.d_R, op.d_D, op.d_level_off, in.keys,
                                                      in.coeffs, W.snorm, features, log_norms);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  *n_logged = nlog;
  return MRA_OK;
}

// ---------------------------------------------------------------- norm / compare hosts

int norm_run(const mra_tree_view &t, double *per_box, double *total, cudaStream_t s) {
  int k3 = t.k * t.k * t.k;
  int64_t n = t.n;
  if (n == 0) {
    if (total) *total = 0.0;
    return MRA_OK;
  }
  double *buf = nullptr, *sq = nullptr, *dsum = nullptr;
  void *tmp = nullptr;
  size_t tmpb = 0;
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(nullptr, tmpb, (double *)nullptr, (double *)nullptr, (int)n));
  MRA_CUDA_TRY(pool_malloc((void **)&buf, n * 8 * 2 + 8 + tmpb + 512, s));
  sq = buf + n;
  dsum = sq + n;
  tmp = (void *)(((uintptr_t)(dsum + 1) + 255) & ~(uintptr_t)255);
  double *norms = per_box ? per_box : buf;
  const int wpb = 8;
  box_norm_kernel<<<counted((unsigned)((n + wpb - 1) / wpb)), 32 * wpb, 0, s>>>(n, k3, t.coeffs, norms);
  square_kernel<<<counted((unsigned)((n + 255) / 256)), 256, 0, s>>>(n, norms, sq);
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, sq, dsum, (int)n, s));
  double h = 0.0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&h, dsum, 8, cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaFreeAsync(buf, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (total) *total = sqrt(h);
  return MRA_OK;
}



int debug_line_apply(cudaStream_t s) { return debug_take_line(s); }

int debug_selftest_run(cudaStream_t s) {
  int *sink = nullptr;
  MRA_CUDA_TRY(pool_malloc((void **)&sink, sizeof(int), s));
  debug_selftest_kernel<<<counted(1), 1, 0, s>>>(sink);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cudaFreeAsync(sink, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  return MRA_OK;
}

int compare_run(const mra_tree_view &t, const mra_tree_view &r, mra_compare_result *res,
                cudaStream_t s) {
  if (t.k != r.k) return fail(MRA_ERR_ARG, "mra_compare: trees have different k");
  int k3 = t.k * t.k * t.k;
  int64_t nt = t.n, nr = r.n;
  int64_t nmax = (nt > nr ? nt : nr) + 1;
  size_t tmpb = 0, tb2 = 0;
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(nullptr, tmpb, (double *)nullptr, (double *)nullptr, (int)nmax));
  MRA_CUDA_TRY(cub::DeviceReduce::Sum(nullptr, tb2, (int *)nullptr, (int *)nullptr, (int)nmax));
  if (tb2 > tmpb) tmpb = tb2;
  char *buf = nullptr;
  size_t per = align_up(nmax * 8);
  size_t total = per * 8 + align_up(tmpb) + 256;
  MRA_CUDA_TRY(pool_malloc((void **)&buf, total, s));
  double *d2 = (double *)buf, *t2 = (double *)(buf + per), *r2 = (double *)(buf + 2 * per);
  double *rel = (double *)(buf + 3 * per), *ra = (double *)(buf + 4 * per);
  double *ro = (double *)(buf + 5 * per);
  int *match = (int *)(buf + 6 * per), *only = (int *)(buf + 7 * per);
  void *tmp = buf + 8 * per;
  double *sums = (double *)(buf + 8 * per + align_up(tmpb));  // 8 doubles
  constexpr int NLEV = MRA_MAX_LEVEL + 1;
  double *lev = nullptr;  // per level: test diff^2, ref-only diff^2, ref^2; ref box counts
  MRA_CUDA_TRY(pool_malloc((void **)&lev, 4 * NLEV * sizeof(double), s));
  MRA_CUDA_TRY(cudaMemsetAsync(lev, 0, 4 * NLEV * sizeof(double), s));
  const int wpb = 8;
  MRA_CUDA_TRY(cudaMemsetAsync(sums, 0, 8 * sizeof(double), s));
  if (nt > 0) {
    compare_kernel<<<counted((unsigned)((nt + wpb - 1) / wpb)), 32 * wpb, 0, s>>>(
        nt, t.keys, t.coeffs, nr, r.keys, r.coeffs, k3, d2, t2, r2, rel, match);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, d2, sums + 0, (int)nt, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, t2, sums + 1, (int)nt, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, match, (int *)(sums + 4), (int)nt, s));
    max_kernel_single<<<counted(1), 1024, 0, s>>>(nt, rel, sums + 5);
    level_sum_kernel<<<counted(NLEV), 256, 0, s>>>(nt, t.keys, d2, lev, nullptr);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  if (nr > 0) {
    ref_only_kernel<<<counted((unsigned)((nr + wpb - 1) / wpb)), 32 * wpb, 0, s>>>(nr, r.keys, r.coeffs, nt,
                                                                           t.keys, k3, ra, ro, only);
    MRA_CUDA_TRY(cudaGetLastError());
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, ra, sums + 2, (int)nr, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, ro, sums + 3, (int)nr, s));
    MRA_CUDA_TRY(cub::DeviceReduce::Sum(tmp, tmpb, only, (int *)(sums + 6), (int)nr, s));
    level_sum_kernel<<<counted(NLEV), 256, 0, s>>>(nr, r.keys, ro, lev + NLEV, nullptr);
    MRA_CUDA_TRY(cudaGetLastError());
    level_sum_kernel<<<counted(NLEV), 256, 0, s>>>(nr, r.keys, ra, lev + 2 * NLEV, (int64_t *)(lev + 3 * NLEV));
    MRA_CUDA_TRY(cudaGetLastError());
  }
  double h[8];
  double hl[4 * NLEV];
  MRA_CUDA_TRY(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(hl, lev, sizeof(hl), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaFreeAsync(buf, s));
  MRA_CUDA_TRY(cudaFreeAsync(lev, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int n = 0; n < NLEV; ++n) {
    res->level_diff_norm[n] = sqrt(hl[n] + hl[NLEV + n]);
    res->level_ref_norm[n] = sqrt(hl[2 * NLEV + n]);
    int64_t c = 0;
    memcpy(&c, &hl[3 * NLEV + n], sizeof(int64_t));
    res->level_ref_boxes[n] = c;
  }
  int n_common = 0, n_only_ref = 0;
  memcpy(&n_common, &h[4], sizeof(int));
  memcpy(&n_only_ref, &h[6], sizeof(int));
  res->diff_norm = sqrt(h[0] + h[3]);
  res->test_norm = sqrt(h[1]);
  res->ref_norm = sqrt(h[2]);
  res->rel_l2 = res->ref_norm > 0 ? res->diff_norm / res->ref_norm : res->diff_norm;
  res->max_box_rel = nt > 0 ? h[5] : 0.0;
  res->n_common = n_common;
  res->n_only_test = nt - n_common;
  res->n_only_ref = n_only_ref;
  return MRA_OK;
}

}  // namespace mra
