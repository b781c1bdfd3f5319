// apply_split.cu -- split-precision tensor-core apply (tcgen05, sm_103a).
//
// The three mode products of every kept term (Sec. 2.3),
//     t1 = s x_1 Rx,  t2 = t1 x_2 Ry,  t3 = t2 x_3 Rz,  r += c_m t3,
// run as BF16 tcgen05 MMAs with FP32 accumulation in tensor memory; every FP64
// or FP32 operand x is split into P BF16 pieces x = x0 + x1 (+ x2) and the
// products x_p y_q with p + q < P are kept.  The Gaussian-term sum and the
// per-box accumulation are FP64, in registers.
//
// Work decomposition (destination-stationary, no atomics): a CTA owns a tile of
// G consecutive destination boxes (slot i = 0..G-1).  Their records are grouped
// by (level, displacement l): one group gathers up to G sources s_i = b_i, one
// per slot, that share the blocks R^n_{m,lx}, R^n_{m,ly}, R^n_{m,lz}.  For each
// term m kept for any slot of the group, the G sources form the rows of three
// M x 16 x 16 GEMMs (M = G k^2, in tiles of 128 rows):
//   stage 1: rows (i, jy, jz), contraction jx, output ix    -> D1[(i,jy,jz)][ix]
//   stage 2: rows (i, jz, ix), contraction jy, output iy    -> D2[(i,jz,ix)][iy]
//   stage 3: rows (i, ix, iy), contraction jz, output iz    -> D3[(i,ix,iy)][iz]
// Each stage's output row (a, b, c) with column d is the next stage's operand
// element [contraction a][row (b, c, d)]: stored MN-major (rows contiguous),
// a thread writes its row's k outputs as one contiguous run.  The k x k block
// R_d is the K-major B operand (N = output index, K = input index), its P
// pieces stacked along N so that one MMA per A piece covers all kept products.
#include <cuda_bf16.h>

#include <cub/cub.cuh>

#include "apply_internal.cuh"
#include "tcgen05.cuh"

namespace mra {

namespace {

constexpr int SPLIT_THREADS = 256;      // 8 warps: two warps per tensor-memory lane quarter
constexpr int MAX_TILES = 7;            // 128-row MMA tiles per stage (G k^2 <= 896)
constexpr int MG_BYTES = 272;           // stride of the 8-row groups: 256 B of core matrices + 16 B
                                        // so that consecutive groups start 4 banks apart
constexpr int TILE_BYTES = 16 * MG_BYTES;  // one 128 x 16 BF16 operand tile
constexpr int BPIECE_BYTES = 512;       // one 16 x 16 BF16 block piece
constexpr int BSTAGE_BYTES = 3 * BPIECE_BYTES;
constexpr int MAX_G = 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_CYCLES = 4000000000LL;  // bounded mbarrier wait (~2 s)

__host__ __device__ inline int tile_boxes(int k) {
  int g = 896 / (k * k);
  return g > MAX_G ? MAX_G : (g < 1 ? 1 : g);
}

// byte offset of element (row m, contraction kk) in an MN-major operand: core
// matrices of 8 contraction rows x 8 consecutive rows (128 B); the two
// contraction groups of a row group 128 B apart (descriptor LBO), the 16 row
// groups of a 128-row tile MG_BYTES apart (descriptor SBO)
__device__ __forceinline__ uint32_t a_off(int m, int kk) {
  return (uint32_t)((m >> 7) * TILE_BYTES + ((m & 127) >> 3) * MG_BYTES + (kk >> 3) * 128 +
                    (kk & 7) * 16 + (m & 7) * 2);
}

__device__ __forceinline__ void split3(double x, __nv_bfloat16 &p0, __nv_bfloat16 &p1,
                                       __nv_bfloat16 &p2) {
  p0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(p0);
  p1 = __double2bfloat16(r);
  r -= (double)__bfloat162float(p1);
  p2 = __double2bfloat16(r);
}

__device__ __forceinline__ void split3f(float x, __nv_bfloat16 &p0, __nv_bfloat16 &p1,
                                        __nv_bfloat16 &p2) {
  p0 = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(p0);
  p1 = __float2bfloat16_rn(r);
  r -= __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r);
}

struct SplitArgs {
  int k, M, P, G, T;
  const double *c;
  const unsigned char *Bsplit;  // per block: 3 pieces x 512 B (K-major core-matrix layout)
  const int *Dlev;
  const int64_t *level_off;
  const double *in_coeffs;
  // work list
  int64_t n_dest;
  const uint64_t *dest_key;
  const int *perm, *did, *rec_src, *rec_l;
  const uint64_t *rec_mask;
  const int *val2;               // key2-sorted -> dest-sorted position
  const int *grp_start;          // [n_groups + 1]
  const int *tile_gstart;        // [n_tiles + 1]
  uint64_t *out_keys;
  double *out_coeffs;
  int *err;
};

// KC >= k: compile-time column count of the FP64 accumulators (8, 12 or 16).
template <int KC>
__global__ void __launch_bounds__(SPLIT_THREADS, 1) apply_split_kernel(SplitArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int k = a.k, k2 = k * k, k3 = k2 * k, P = a.P, G = a.G, T = a.T;
  const int rows = G * k2;
  unsigned char *A1 = smem;                               // [P][T][4096]
  unsigned char *A23 = A1 + P * T * TILE_BYTES;           // [P][T][4096]
  unsigned char *Bt = A23 + P * T * TILE_BYTES;           // [3 stages][1536]
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  __shared__ int slot_src[MAX_G];
  __shared__ uint64_t slot_mask[MAX_G][2];
  __shared__ uint64_t uni[2];
  __shared__ int g_level, g_l;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int quarter = warp & 3, half = warp >> 2;

  // zero all operand buffers once: the contraction padding (16 - k) and row padding stay zero
  {
    int4 *z = (int4 *)smem;
    int n16 = (2 * P * T * TILE_BYTES + 3 * BSTAGE_BYTES) / 16;
    for (int i = tid; i < n16; i += SPLIT_THREADS) z[i] = make_int4(0, 0, 0, 0);
  }
  const uint32_t bar_a = tc::smem_u32(&bar);
  if (tid == 0) tc::mbar_init(bar_a, 1);
  bool aborted = false;  // identical in every thread: set only from a CTA-wide vote
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_holder), TMEM_COLS);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  uint32_t phase = 0;

  double acc[4][KC];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < KC; ++j) acc[q][j] = 0.0;

  const uint32_t idesc_n[3] = {tc::idesc_bf16(128, 16, 1, 0), tc::idesc_bf16(128, 32, 1, 0),
                               tc::idesc_bf16(128, 48, 1, 0)};

  // Issue one stage: for every 128-row tile, the P MMAs over the A pieces.
  auto issue_stage = [&](const unsigned char *A, const unsigned char *B) {
    tc::fence_after_sync();
    const uint32_t bdesc_addr = tc::smem_u32(B);
    for (int t = 0; t < T; ++t) {
      uint32_t d = tmem + (uint32_t)(t * 48);
      for (int p = 0; p < P; ++p) {
        uint64_t ad = tc::smem_desc(tc::smem_u32(A + (p * T + t) * TILE_BYTES), 128, MG_BYTES);
        uint64_t bd = tc::smem_desc(bdesc_addr, 128, 256);
        // A piece p times B pieces 0..P-1-p (stacked along N) into column groups p..P-1
        tc::mma_bf16(d + 16 * p, ad, bd, idesc_n[P - 1 - p], p > 0 ? 1u : 0u);
      }
    }
    tc::mma_commit(bar_a);
  };

  // Every thread waits for the stage's MMAs; the CTA then agrees on the outcome.
  auto wait_mma = [&]() -> bool {
    bool ok = tc::mbar_wait(bar_a, phase, WAIT_CYCLES);
    phase ^= 1u;
    int bad = __syncthreads_or(!ok);
    if (bad) {
      aborted = true;
      if (tid == 0) atomicExch(a.err, 1);
    }
    tc::fence_after_sync();
    return !bad;
  };

  // Sum of this thread's P column groups of tile t (k values).
  auto load_tile = [&](int t, float *v) {
    uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(t * 48);
    float c0[16], c1[16], c2[16];
    tc::tmem_ld16(base, c0);
    if (P > 1) tc::tmem_ld16(base + 16, c1);
    if (P > 2) tc::tmem_ld16(base + 32, c2);
    tc::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float s = c0[j];
      if (P == 2) s = c1[j] + c0[j];
      if (P == 3) s = (c2[j] + c1[j]) + c0[j];
      v[j] = s;
    }
  };

  // write the k values of output row (b, c) with new index d into the next operand:
  // element [contraction a][row (i, b, c, d)] for d = 0..k-1.  For even k the run
  // starts on an even row, so pairs of rows share one 32-bit word.
  auto store_run = [&](unsigned char *A, int i, int a_idx, int b_idx, const float *v) {
    int mrow = i * k2 + b_idx * k;  // rows (i, b, d) for d = 0..k-1
    const int stride = T * TILE_BYTES;
    if ((k & 1) == 0) {
#pragma unroll
      for (int d = 0; d < 16; d += 2) {
        if (d < k) {
          __nv_bfloat16 a0, a1, a2, b0, b1, b2;
          split3f(v[d], a0, a1, a2);
          split3f(v[d + 1], b0, b1, b2);
          uint32_t off = a_off(mrow + d, a_idx);
          *(__nv_bfloat162 *)(A + off) = __halves2bfloat162(a0, b0);
          *(__nv_bfloat162 *)(A + stride + off) = __halves2bfloat162(a1, b1);
          if (P > 2) *(__nv_bfloat162 *)(A + 2 * stride + off) = __halves2bfloat162(a2, b2);
        }
      }
    } else {
      for (int d = 0; d < k; ++d) {
        __nv_bfloat16 p0, p1, p2;
        split3f(v[d], p0, p1, p2);
        uint32_t off = a_off(mrow + d, a_idx);
        *(__nv_bfloat16 *)(A + off) = p0;
        *(__nv_bfloat16 *)(A + stride + off) = p1;
        if (P > 2) *(__nv_bfloat16 *)(A + 2 * stride + off) = p2;
      }
    }
  };

  const int g0 = a.tile_gstart[tile], g1 = a.tile_gstart[tile + 1];
  for (int g = g0; g < g1 && !aborted; ++g) {
    const int r0 = a.grp_start[g], r1 = a.grp_start[g + 1];
    if (tid < MAX_G) {
      slot_src[tid] = -1;
      slot_mask[tid][0] = slot_mask[tid][1] = 0ull;
    }
    if (tid == 0) uni[0] = uni[1] = 0ull;
    __syncthreads();
    for (int r = r0 + tid; r < r1; r += SPLIT_THREADS) {
      int i = a.val2[r];
      int p = a.perm[i];
      int slot = (a.did[i] - 1) - tile * G;
      if (slot < 0 || slot >= G) {
        atomicExch(a.err, 2);
        continue;
      }
      slot_src[slot] = a.rec_src[p];
      slot_mask[slot][0] = a.rec_mask[2 * (int64_t)p];
      slot_mask[slot][1] = a.rec_mask[2 * (int64_t)p + 1];
      atomicOr((unsigned long long *)&uni[0], (unsigned long long)a.rec_mask[2 * (int64_t)p]);
      atomicOr((unsigned long long *)&uni[1], (unsigned long long)a.rec_mask[2 * (int64_t)p + 1]);
      if (r == r0) {
        g_l = a.rec_l[p];
        g_level = key_level(a.dest_key[a.did[i] - 1]);
      }
    }
    __syncthreads();
    // stage-1 operand: sources, rows (i, jy, jz), contraction jx (pairs of rows when k is even)
    if ((k & 1) == 0) {
      for (int e = tid; e < G * k3 / 2; e += SPLIT_THREADS) {
        int e2 = 2 * e;
        int i = e2 / k3, rest = e2 - i * k3;
        int jx = rest / k2, q = rest - jx * k2;
        int src = slot_src[i];
        double x0 = 0.0, x1 = 0.0;
        if (src >= 0) {
          double2 xx = *(const double2 *)(a.in_coeffs + (int64_t)src * k3 + rest);
          x0 = xx.x;
          x1 = xx.y;
        }
        __nv_bfloat16 a0, a1, a2, b0, b1, b2;
        split3(x0, a0, a1, a2);
        split3(x1, b0, b1, b2);
        uint32_t off = a_off(i * k2 + q, jx);
        *(__nv_bfloat162 *)(A1 + off) = __halves2bfloat162(a0, b0);
        *(__nv_bfloat162 *)(A1 + T * TILE_BYTES + off) = __halves2bfloat162(a1, b1);
        if (P > 2) *(__nv_bfloat162 *)(A1 + 2 * T * TILE_BYTES + off) = __halves2bfloat162(a2, b2);
      }
    } else {
      for (int e = tid; e < G * k3; e += SPLIT_THREADS) {
        int i = e / k3, rest = e - i * k3;
        int jx = rest / k2, q = rest - jx * k2;
        int src = slot_src[i];
        double x = src >= 0 ? a.in_coeffs[(int64_t)src * k3 + rest] : 0.0;
        __nv_bfloat16 p0, p1, p2;
        split3(x, p0, p1, p2);
        uint32_t off = a_off(i * k2 + q, jx);
        *(__nv_bfloat16 *)(A1 + off) = p0;
        *(__nv_bfloat16 *)(A1 + T * TILE_BYTES + off) = p1;
        if (P > 2) *(__nv_bfloat16 *)(A1 + 2 * T * TILE_BYTES + off) = p2;
      }
    }
    const int lev = g_level, lp = g_l;
    const int Dop = a.Dlev[lev], nl = 2 * Dop + 1;
    const int ld[3] = {(lp & 255) - 128, ((lp >> 8) & 255) - 128, ((lp >> 16) & 255) - 128};
    const int64_t lbase = a.level_off[lev];
    for (int w = 0; w < 2 && !aborted; ++w) {
      uint64_t bits = uni[w];
      while (bits && !aborted) {
        const int m = w * 64 + __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        // B operands of the three stages: blocks (m, lx), (m, ly), (m, lz)
        for (int e = tid; e < 3 * (BSTAGE_BYTES / 16); e += SPLIT_THREADS) {
          int st = e / (BSTAGE_BYTES / 16), q = e - st * (BSTAGE_BYTES / 16);
          int64_t blk = lbase + (int64_t)m * nl + ld[st] + Dop;
          ((int4 *)(Bt + st * BSTAGE_BYTES))[q] = ((const int4 *)(a.Bsplit + blk * BSTAGE_BYTES))[q];
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // ---- stage 1
        if (tid == 0) issue_stage(A1, Bt);
        if (!wait_mma()) break;
        for (int t = half; t < T; t += 2) {
          float v[16];
          load_tile(t, v);
          int m1 = t * 128 + quarter * 32 + lane;
          if (m1 < rows) {
            int i = m1 / k2, rem = m1 - i * k2, jy = rem / k, jz = rem - jy * k;
            store_run(A23, i, jy, jz, v);  // element [jy][(i, jz, ix)]
          }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // ---- stage 2
        if (tid == 0) issue_stage(A23, Bt + BSTAGE_BYTES);
        if (!wait_mma()) break;
        for (int t = half; t < T; t += 2) {  // stage-2 reads of A23 are complete: rewrite it
          float v[16];
          load_tile(t, v);
          int m2 = t * 128 + quarter * 32 + lane;
          if (m2 < rows) {
            int i = m2 / k2, rem = m2 - i * k2, jz = rem / k, ix = rem - jz * k;
            store_run(A23, i, jz, ix, v);  // element [jz][(i, ix, iy)]
          }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // ---- stage 3
        if (tid == 0) issue_stage(A23, Bt + 2 * BSTAGE_BYTES);
        if (!wait_mma()) break;
        const double cm = a.c[m];
#pragma unroll
        for (int q = 0; q < MAX_TILES / 2 + 1; ++q) {
          int t = half + 2 * q;
          if (t < T) {
            float v[16];
            load_tile(t, v);
            int m3 = t * 128 + quarter * 32 + lane;
            if (m3 < rows) {
              int i = m3 / k2;
              bool kept = (slot_mask[i][w] >> (m & 63)) & 1ull;
              double wgt = kept ? cm : 0.0;
#pragma unroll
              for (int j = 0; j < KC; ++j) acc[q][j] += wgt * (double)v[j];
            }
          }
        }
        tc::fence_before_sync();
        __syncthreads();
      }
    }
    __syncthreads();
  }
  // write the destinations: row (i, ix, iy), columns iz
  if (!aborted) {
#pragma unroll
    for (int q = 0; q < MAX_TILES / 2 + 1; ++q) {
      int t = half + 2 * q;
      int m3 = t * 128 + quarter * 32 + lane;
      if (t < T && m3 < rows) {
        int i = m3 / k2, rem = m3 - i * k2;
        int64_t dst = (int64_t)tile * G + i;
        if (dst < a.n_dest) {
          double *o = a.out_coeffs + dst * k3 + (int64_t)rem * k;
#pragma unroll
          for (int j = 0; j < KC; ++j)
            if (j < k) o[j] = acc[q][j];
          if (rem == 0) a.out_keys[dst] = a.dest_key[dst];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (aborted && tid == 0) tc::mbar_wait(bar_a, phase ^ 1u, WAIT_CYCLES);  // let in-flight MMAs finish
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- work-list kernels
__global__ void key2_kernel(int64_t P, int G, const int *perm, const int *did, const uint64_t *skey,
                            const int *rec_l, uint64_t *key2, int *val2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int p = perm[i];
  uint64_t tile = (uint64_t)((did[i] - 1) / G);
  uint64_t lev = (uint64_t)key_level(skey[i]);
  key2[i] = (tile << 32) | (lev << 24) | (uint64_t)(rec_l[p] & 0xFFFFFF);
  val2[i] = (int)i;
}

__global__ void groups_kernel(int64_t P, const uint64_t *key2s, int *head, int n_tiles) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  head[j] = (j == 0 || key2s[j] != key2s[j - 1]) ? 1 : 0;
}

__global__ void group_bounds_kernel(int64_t P, const uint64_t *key2s, const int *head,
                                    const int *gid, int *grp_start, int *tile_gstart, int n_tiles) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P) return;
  if (head[j]) {
    int g = gid[j] - 1;
    grp_start[g] = (int)j;
    uint64_t tile = key2s[j] >> 32;
    if (j == 0 || (key2s[j - 1] >> 32) != tile) tile_gstart[tile] = g;
  }
  if (j == P - 1) {
    grp_start[gid[j]] = (int)P;
    tile_gstart[n_tiles] = gid[j];
  }
}

// Block pieces in the K-major core-matrix layout the MMA reads: piece p of block
// R (N = output index i, K = input index j), element (i, j) at
// p*512 + (i/8)*256 + (j/8)*128 + (i%8)*16 + (j%8)*2; zero outside k x k.
__global__ void split_blocks_kernel(int64_t n_blocks, int k, const double *R, unsigned char *out) {
  int64_t blk = blockIdx.x;
  if (blk >= n_blocks) return;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    int i = e / 16, j = e % 16;
    double x = (i < k && j < k) ? R[blk * k * k + i * k + j] : 0.0;
    __nv_bfloat16 p0, p1, p2;
    split3(x, p0, p1, p2);
    uint32_t off = (i / 8) * 256 + (j / 8) * 128 + (i % 8) * 16 + (j % 8) * 2;
    unsigned char *b = out + blk * BSTAGE_BYTES;
    *(__nv_bfloat16 *)(b + off) = p0;
    *(__nv_bfloat16 *)(b + BPIECE_BYTES + off) = p1;
    *(__nv_bfloat16 *)(b + 2 * BPIECE_BYTES + off) = p2;
  }
}

}  // namespace

size_t split_workspace_bytes(int64_t P) {
  int64_t np = P > 0 ? P : 1;
  size_t t = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, t, (uint64_t *)nullptr, (uint64_t *)nullptr, (int *)nullptr,
                                  (int *)nullptr, (int)np);
  size_t s2 = 0;
  cub::DeviceScan::InclusiveSum(nullptr, s2, (int *)nullptr, (int *)nullptr, (int)np);
  if (s2 > t) t = s2;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al(np * 8) * 2 + al(np * 4) * 5 + al((np + 2) * 4) * 2 + al(t) + 256;
}

int split_blocks_build(Operator &op, cudaStream_t s) {
  if (op.d_Rsplit) return MRA_OK;
  MRA_CUDA_TRY(cudaMalloc(&op.d_Rsplit, (size_t)op.n_blocks * BSTAGE_BYTES));
  split_blocks_kernel<<<(unsigned)op.n_blocks, 128, 0, s>>>(op.n_blocks, op.k, op.d_R,
                                                            (unsigned char *)op.d_Rsplit);
  MRA_CUDA_TRY(cudaGetLastError());
  return MRA_OK;
}

int apply_split_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o,
                    mra_tree_view &out, const ApplyWork &wk, mra_apply_stats *stats,
                    cudaStream_t s) {
  if (!op.d_Rsplit) return fail(MRA_ERR_ARG, "mra_apply: operator has no split blocks");
  const int k = op.k, G = tile_boxes(k);
  const int T = (G * k * k + 127) / 128;
  if (T > MAX_TILES) return fail(MRA_ERR_UNSUPPORTED, "split apply: tile too large for k=%d", k);
  const int64_t P = wk.P, nd = wk.n_dest;
  const int n_tiles = (int)((nd + G - 1) / G);
  // carve the split-path workspace
  char *w = (char *)wk.split_ws;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int64_t np = P > 0 ? P : 1;
  uint64_t *key2 = (uint64_t *)w;
  uint64_t *key2s = (uint64_t *)(w + al(np * 8));
  char *q = w + 2 * al(np * 8);
  int *val2 = (int *)q; q += al(np * 4);
  int *val2s = (int *)q; q += al(np * 4);
  int *head = (int *)q; q += al(np * 4);
  int *gid = (int *)q; q += al(np * 4);
  int *err = (int *)q; q += al(np * 4);
  int *grp_start = (int *)q; q += al((np + 2) * 4);
  int *tile_gstart = (int *)q; q += al((np + 2) * 4);
  void *tmp = q;
  size_t tmpb = wk.split_ws_bytes - (size_t)(q - w);
  unsigned g = (unsigned)((P + 255) / 256);
  MRA_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  key2_kernel<<<g, 256, 0, s>>>(P, G, wk.perm, wk.did, wk.skey, wk.rec_l, key2, val2);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmpb, key2, key2s, val2, val2s, (int)P, 0, 64, s));
  groups_kernel<<<g, 256, 0, s>>>(P, key2s, head, n_tiles);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp, tmpb, head, gid, (int)P, s));
  group_bounds_kernel<<<g, 256, 0, s>>>(P, key2s, head, gid, grp_start, tile_gstart, n_tiles);
  MRA_CUDA_TRY(cudaGetLastError());

  SplitArgs a{};
  a.k = k;
  a.M = op.M;
  a.P = o.pieces;
  a.G = G;
  a.T = T;
  a.c = op.d_c;
  a.Bsplit = (const unsigned char *)op.d_Rsplit;
  a.Dlev = op.d_D;
  a.level_off = op.d_level_off;
  a.in_coeffs = in.coeffs;
  a.n_dest = nd;
  a.dest_key = wk.dest_key;
  a.perm = wk.perm;
  a.did = wk.did;
  a.rec_src = wk.rec_src;
  a.rec_l = wk.rec_l;
  a.rec_mask = wk.rec_mask;
  a.val2 = val2s;
  a.grp_start = grp_start;
  a.tile_gstart = tile_gstart;
  a.out_keys = out.keys;
  a.out_coeffs = out.coeffs;
  a.err = err;
  size_t smem = (size_t)2 * a.P * T * TILE_BYTES + 3 * BSTAGE_BYTES + 1024;
  void (*kern)(SplitArgs) = k <= 8 ? apply_split_kernel<8> : (k <= 12 ? apply_split_kernel<12> : apply_split_kernel<16>);
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (wk.ev0) MRA_CUDA_TRY(cudaEventRecord(wk.ev0, s));
  kern<<<(unsigned)n_tiles, SPLIT_THREADS, smem, s>>>(a);
  MRA_CUDA_TRY(cudaGetLastError());
  if (wk.ev1) MRA_CUDA_TRY(cudaEventRecord(wk.ev1, s));
  int herr = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr == 1) return fail(MRA_ERR_TIMEOUT, "split apply: a tensor-core completion wait gave up");
  if (herr) return fail(MRA_ERR_ARG, "split apply: inconsistent work list (%d)", herr);
  (void)stats;
  return MRA_OK;
}

}  // namespace mra
