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
constexpr int MG_BYTES = 272;           // stride of the 8-row groups: 256 B of core matrices + 16 B
                                        // so that consecutive groups start 4 banks apart
constexpr int TILE_BYTES = 16 * MG_BYTES;  // one 128 x 16 BF16 operand tile
constexpr int BPIECE_BYTES = 512;       // one 16 x 16 BF16 block piece
constexpr int BSTAGE_BYTES = 3 * BPIECE_BYTES;
constexpr int MAX_G = 32;
constexpr long long WAIT_CYCLES = 4000000000LL;  // bounded mbarrier wait (~2 s)


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

// Exact widening of an FP32 value to FP64 with integer operations (IEEE layouts:
// 8-bit exponent bias 127 -> 11-bit bias 1023, 23-bit -> 52-bit fraction), so that
// only the multiply-add of the term sum uses the FP64 pipe.  FP32 subnormals
// (|x| < 1.2e-38) become zero.
__device__ __forceinline__ double widen(float f) {
  uint32_t u = __float_as_uint(f);
  uint32_t e = (u >> 23) & 0xFFu;
  uint64_t sign = (uint64_t)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);
  uint64_t ee = (e == 0xFFu) ? 2047u : (uint64_t)(e + 896u);
  return __longlong_as_double((long long)(sign | (ee << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// Named barrier over one warpgroup (128 threads) with an OR vote.
__device__ __forceinline__ bool wg_vote_or(int barrier_id, bool flag) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)flag), "r"(barrier_id)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void wg_sync(int barrier_id) {
  asm volatile("bar.sync %0, 128;" ::"r"(barrier_id) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Compile-time tile shapes for an even k: TM tiles of 128 rows per stage and MINB CTAs per
// SM.  Variant 0 -- k <= 10: four tiles and two CTAs per SM (each CTA's serial chain of MMA
// waits and tensor-memory loads hides behind the other's); k >= 12: one CTA with more tiles.
// Variant 1 (k = 6, 8, 10): seven tiles, one CTA per SM (fewer, wider tiles).
__host__ __device__ constexpr int tm_for(int k, int v = 0) {
  return v == 1 ? 7 : (k <= 2 ? 1 : (k <= 10 ? 4 : (k <= 12 ? 6 : (k <= 14 ? 5 : 4))));
}
__host__ __device__ constexpr int minb_for(int k, int v = 0) { return v == 1 ? 1 : (k <= 10 ? 2 : 1); }
__host__ __device__ constexpr int g_for(int k, int v = 0) {
  return (128 * tm_for(k, v)) / (k * k) > MAX_G ? MAX_G : (128 * tm_for(k, v)) / (k * k);
}
// tensor-memory columns: D (48 T: three 16-column piece groups per tile), rounded to a
// power of two
__host__ __device__ constexpr uint32_t tmem_cols_for(int k, int v = 0) {
  return 48 * tm_for(k, v) <= 64 ? 64u
       : (48 * tm_for(k, v) <= 128 ? 128u : (48 * tm_for(k, v) <= 256 ? 256u : 512u));
}

// Split x and y into three BF16 pieces each (x = x0 + x1 + x2 to 24 bits), packed in pairs.
__device__ __forceinline__ void split_pair(float x, float y, __nv_bfloat162 &h0, __nv_bfloat162 &h1,
                                           __nv_bfloat162 &h2) {
  h0 = __floats2bfloat162_rn(x, y);
  float2 f0 = __bfloat1622float2(h0);
  float rx = x - f0.x, ry = y - f0.y;
  h1 = __floats2bfloat162_rn(rx, ry);
  float2 f1 = __bfloat1622float2(h1);
  h2 = __floats2bfloat162_rn(rx - f1.x, ry - f1.y);
}

// Warp roles: warpgroup 0 (warps 0-3) stages each group's sources, turns stage-1/2
// outputs into the next stage's operands, and its thread 0 issues every MMA and every
// block-tile copy (one term ahead); warpgroup 1 (warps 4-7) adds each term's stage-3
// output into the FP64 accumulators while warpgroup 0 works on the next term.
// An M=128 x K=16 MMA costs about the same for any N <= 128 (its A tile fetch bounds
// it), so every stage stacks the B pieces along N: A piece p times [B0 .. B(P-1-p)]
// into column groups p..P-1 of the tile's 48 columns of D ([0, 48T)).  Warpgroup 1
// copies stage 3's result to registers (summing the groups) and releases D before
// the next term's stage 1; the FP64 accumulation then runs alongside that term.
template <int K, int V>
__global__ void __launch_bounds__(SPLIT_THREADS, minb_for(K, V)) apply_split_kernel(SplitArgs a) {
  constexpr int TM = tm_for(K, V);
  extern __shared__ __align__(1024) unsigned char smem[];
  // k, k^2, k^3, G, T are compile-time: the index arithmetic below has no runtime division
  constexpr int k = K, k2 = K * K, k3 = K * K * K, G = g_for(K, V), T = (G * K * K + 127) / 128;
  const int P = a.P;
  constexpr int rows = G * k2;
  unsigned char *A1 = smem;                          // [P][T][TILE_BYTES] stage-1 operand (sources)
  unsigned char *A23 = A1 + P * T * TILE_BYTES;      // [P][T][TILE_BYTES] stage-2/3 operand
  unsigned char *Bt = A23 + P * T * TILE_BYTES;      // [2 buffers][3 stages][1536]
  __shared__ __align__(8) uint64_t bar12, bar3, bar_free, bar_drain, bar_b[2];
  __shared__ uint32_t tmem_holder;
  __shared__ int slot_src[MAX_G];
  __shared__ uint64_t slot_mask[MAX_G][2];
  __shared__ uint64_t uni[2];
  __shared__ int g_level, g_l, total_it;
  __shared__ double ring_c[4];
  __shared__ double c_sh[MRA_MAX_TERMS];
  __shared__ uint32_t ring_keep[4];
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, quarter = warp & 3;
  const int tile = blockIdx.x;
  const int g0 = a.tile_gstart[tile], g1 = a.tile_gstart[tile + 1];

  {  // zero the operand buffers once: contraction and row padding stay zero
    int4 *z = (int4 *)smem;
    int n16 = (2 * P * T * TILE_BYTES) / 16;
    for (int i = tid; i < n16; i += SPLIT_THREADS) z[i] = make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(&bar12), 1);
    tc::mbar_init(tc::smem_u32(&bar3), 1);
    tc::mbar_init(tc::smem_u32(&bar_free), 1);
    tc::mbar_init(tc::smem_u32(&bar_drain), 1);
    tc::mbar_init(tc::smem_u32(&bar_b[0]), 1);
    tc::mbar_init(tc::smem_u32(&bar_b[1]), 1);
    abort_flag = 0;
    total_it = 0;
  }
  for (int m = tid; m < a.M; m += SPLIT_THREADS) c_sh[m] = a.c[m];
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_holder), tmem_cols_for(K, V));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_proxy_async_smem();
  __syncthreads();
  if (warp == 0) {  // number of (group, term) iterations of this tile, for warpgroup 1
    int cnt = 0;
    for (int g = g0; g < g1; ++g) {
      uint64_t u0 = 0, u1 = 0;
      for (int r = a.grp_start[g] + lane; r < a.grp_start[g + 1]; r += 32) {
        int p = a.perm[a.val2[r]];
        u0 |= a.rec_mask[2 * (int64_t)p];
        u1 |= a.rec_mask[2 * (int64_t)p + 1];
      }
      for (int o = 16; o > 0; o >>= 1) {
        u0 |= __shfl_xor_sync(0xffffffffu, u0, o);
        u1 |= __shfl_xor_sync(0xffffffffu, u1, o);
      }
      cnt += __popcll(u0) + __popcll(u1);
    }
    if (lane == 0) total_it = cnt;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t b12 = tc::smem_u32(&bar12);
  const uint32_t b3 = tc::smem_u32(&bar3), bfree = tc::smem_u32(&bar_free);
  const uint32_t bb[2] = {tc::smem_u32(&bar_b[0]), tc::smem_u32(&bar_b[1])};
  const int nit = total_it;
  const uint32_t idesc16 = tc::idesc_bf16(128, 16, 1, 0);
  const uint32_t idesc_n[3] = {idesc16, tc::idesc_bf16(128, 32, 1, 0), tc::idesc_bf16(128, 48, 1, 0)};

  // stages 1 and 2: A piece p times B pieces 0..P-1-p (stacked along N) into column
  // groups p..P-1 of the tile's 48 columns of D12
  auto issue_stacked = [&](const unsigned char *A, const unsigned char *B) {
    for (int t = 0; t < T; ++t) {
      uint32_t d = tmem + (uint32_t)(t * 48);
      for (int p = 0; p < P; ++p) {
        uint64_t ad = tc::smem_desc(tc::smem_u32(A + (p * T + t) * TILE_BYTES), 128, MG_BYTES);
        uint64_t bd = tc::smem_desc(tc::smem_u32(B), 128, 256);
        tc::mma_bf16(d + 16 * p, ad, bd, idesc_n[P - 1 - p], p > 0 ? 1u : 0u);
      }
    }
  };

  if (wg == 0) {
    // ======================================================= warpgroup 0 + MMA / copy issue
    uint32_t p12 = 0;
    int it = 0;
    bool bad = false;
    auto wait12 = [&]() -> bool {
      bool ok = tc::mbar_wait(b12, p12, WAIT_CYCLES);
      p12 ^= 1u;
      bool any_bad = wg_vote_or(1, !ok || abort_flag);
      tc::fence_after_sync();
      return !any_bad;
    };
    // copies of the three blocks (m; lx, ly, lz) into buffer `buf`
    auto fetch_blocks = [&](int buf, int m, int64_t lbase, int nl, int Dop, int lx, int ly, int lz) {
      unsigned char *Bb = Bt + buf * 3 * BSTAGE_BYTES;
      tc::mbar_arrive_expect_tx(bb[buf], 3 * BSTAGE_BYTES);
      const int ls[3] = {lx, ly, lz};
#pragma unroll
      for (int st = 0; st < 3; ++st) {
        int64_t blk = lbase + (int64_t)m * nl + ls[st] + Dop;
        tc::bulk_g2s(tc::smem_u32(Bb + st * BSTAGE_BYTES), a.Bsplit + blk * BSTAGE_BYTES, BSTAGE_BYTES, bb[buf]);
      }
    };
    // element [contraction a][row (i, b, d)] for d = 0..k-1 of this thread's rows
    auto store_run = [&](int mrow, int a_idx, const float *v) {
      const int stride = T * TILE_BYTES;
#pragma unroll
      for (int d = 0; d < K; d += 2) {
        __nv_bfloat162 h0, h1, h2;
        split_pair(v[d], v[d + 1], h0, h1, h2);
        uint32_t off = a_off(mrow + d, a_idx);
        *(__nv_bfloat162 *)(A23 + off) = h0;
        *(__nv_bfloat162 *)(A23 + stride + off) = h1;
        if (P > 2) *(__nv_bfloat162 *)(A23 + 2 * stride + off) = h2;
      }
    };
    // tiles t0, t0+1 of D12 for this thread's lane (first K columns of each of the P
    // groups, summed smallest first), one wait for all loads
    auto load_d12_pair = [&](int t0, float (*v)[16]) {
      const uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float c[3][K];
        if (t0 + u < T) {
#pragma unroll
          for (int p = 0; p < 3; ++p)
            if (p < P) tc::tmem_ldk<K>(base + (uint32_t)((t0 + u) * 48 + 16 * p), c[p]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < K; ++j)
            v[u][j] = P == 3 ? (c[2][j] + c[1][j]) + c[0][j] : (P == 2 ? c[1][j] + c[0][j] : c[0][j]);
        }
      }
    };
    for (int g = g0; g < g1 && !bad; ++g) {
      const int r0 = a.grp_start[g], r1 = a.grp_start[g + 1];
      if (tid < MAX_G) {
        slot_src[tid] = -1;
        slot_mask[tid][0] = slot_mask[tid][1] = 0ull;
      }
      if (tid == 0) uni[0] = uni[1] = 0ull;
      wg_sync(1);
      for (int r = r0 + tid; r < r1; r += 128) {
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
      wg_sync(1);
      const int lev = g_level, lp = g_l;
      const int Dop = a.Dlev[lev], nl = 2 * Dop + 1;
      const int ldx = (lp & 255) - 128, ldy = ((lp >> 8) & 255) - 128, ldz = ((lp >> 16) & 255) - 128;
      const int64_t lbase = a.level_off[lev];
      uint64_t bits0 = uni[0], bits1 = uni[1];
      auto next_term = [&](uint64_t &b0, uint64_t &b1) -> int {  // pop the lowest kept term
        if (b0) { int m = __ffsll((long long)b0) - 1; b0 &= b0 - 1; return m; }
        if (b1) { int m = 64 + __ffsll((long long)b1) - 1; b1 &= b1 - 1; return m; }
        return -1;
      };
      int m = next_term(bits0, bits1);
      // first term of the group: its blocks were not prefetched (buffer it&1 was last read by
      // stage 3 of term it-2, complete since stage 1 of term it-1 completed)
      if (tid == 0 && m >= 0) fetch_blocks(it & 1, m, lbase, nl, Dop, ldx, ldy, ldz);
      // stage-1 operand: sources, rows (i, jy, jz), contraction jx (FP64 -> FP32 -> 3 BF16 pieces).
      // The previous group's stage-1 MMAs are complete (their stage 2 was waited for).
      for (int e = tid; e < G * k3 / 2; e += 128) {
        int e2 = 2 * e;
        int i = e2 / k3, rest = e2 - i * k3;
        int jx = rest / k2, q = rest - jx * k2;
        int src = slot_src[i];
        double2 xx = make_double2(0.0, 0.0);
        if (src >= 0) xx = *(const double2 *)(a.in_coeffs + (int64_t)src * k3 + rest);
        __nv_bfloat162 h0, h1, h2;
        split_pair((float)xx.x, (float)xx.y, h0, h1, h2);
        uint32_t off = a_off(i * k2 + q, jx);
        *(__nv_bfloat162 *)(A1 + off) = h0;
        *(__nv_bfloat162 *)(A1 + T * TILE_BYTES + off) = h1;
        if (P > 2) *(__nv_bfloat162 *)(A1 + 2 * T * TILE_BYTES + off) = h2;
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      wg_sync(1);
      while (m >= 0 && !bad) {
        const int buf = it & 1;
        const unsigned char *Bb = Bt + buf * 3 * BSTAGE_BYTES;
        const int m_next = next_term(bits0, bits1);
        if (tid == 0) {
          // term info for warpgroup 1 (ring slot it&3 was read by its iteration it-4, which
          // finished before the "D free" arrival that let stage 1 of term it-3 start)
          uint32_t keep = 0;
          const int w = m >> 6;
          for (int i = 0; i < G; ++i) keep |= (uint32_t)((slot_mask[i][w] >> (m & 63)) & 1ull) << i;
          ring_keep[it & 3] = keep;
          ring_c[it & 3] = c_sh[m];
          bool ok = tc::mbar_wait(bb[buf], (uint32_t)((it >> 1) & 1), WAIT_CYCLES);
          // D holds stage 3 of term it-1 until warpgroup 1 has copied it out
          if (ok && it > 0) ok = tc::mbar_wait(bfree, (uint32_t)((it - 1) & 1), WAIT_CYCLES);
          if (!ok) {
            abort_flag = 1;
          } else {
            tc::fence_after_sync();
            issue_stacked(A1, Bb);  // ---- stage 1: rows (i, jy, jz), contraction jx
            tc::mma_commit(b12);
          }
        }
        if (!wait12()) { bad = true; break; }
        // stage 1 done, hence also stage 3 of term it-1: buffer it+1 is free for the next term
        if (tid == 0 && m_next >= 0) fetch_blocks((it + 1) & 1, m_next, lbase, nl, Dop, ldx, ldy, ldz);
#pragma unroll
        for (int t0 = 0; t0 < TM; t0 += 2) {
          float v[2][16];
          load_d12_pair(t0, v);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int t = t0 + u;
            int m1 = t * 128 + quarter * 32 + lane;
            if (t < TM && t < T && m1 < rows) {
              int i = m1 / k2, rem = m1 - i * k2, jy = rem / k, jz = rem - jy * k;
              store_run(i * k2 + jz * k, jy, v[u]);  // element [jy][(i, jz, ix)]
            }
          }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        wg_sync(1);
        if (tid == 0) {  // ---- stage 2: rows (i, jz, ix), contraction jy
          tc::fence_after_sync();
          issue_stacked(A23, Bb + BSTAGE_BYTES);
          tc::mma_commit(b12);
        }
        if (!wait12()) { bad = true; break; }
#pragma unroll
        for (int t0 = 0; t0 < TM; t0 += 2) {
          float v[2][16];
          load_d12_pair(t0, v);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int t = t0 + u;
            int m2 = t * 128 + quarter * 32 + lane;
            if (t < TM && t < T && m2 < rows) {
              int i = m2 / k2, rem = m2 - i * k2, jz = rem / k, ix = rem - jz * k;
              store_run(i * k2 + ix * k, jz, v[u]);  // element [jz][(i, ix, iy)]
            }
          }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        wg_sync(1);
        if (tid == 0) {  // ---- stage 3: rows (i, ix, iy), contraction jz
          tc::fence_after_sync();
          issue_stacked(A23, Bb + 2 * BSTAGE_BYTES);
          tc::mma_commit(b3);
        }
        ++it;
        m = m_next;
        if (wg_vote_or(1, abort_flag)) { bad = true; break; }
      }
      wg_sync(1);
    }
    if (bad) abort_flag = 1;
  } else {
    // ======================================================= warpgroup 1: FP64 term sums
    double acc[TM][K];
#pragma unroll
    for (int t = 0; t < TM; ++t)
#pragma unroll
      for (int j = 0; j < K; ++j) acc[t][j] = 0.0;
    bool bad = false;
    const uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16);
    for (int it = 0; it < nit; ++it) {
      bool ok = tc::mbar_wait(b3, (uint32_t)(it & 1), WAIT_CYCLES);
      if (wg_vote_or(2, !ok || abort_flag)) {
        bad = true;
        break;
      }
      tc::fence_after_sync();
      const double cm = ring_c[it & 3];
      const uint32_t keep = ring_keep[it & 3];
      float v[TM][K];
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        if (t < T) {
          float c[3][K];
#pragma unroll
          for (int p = 0; p < 3; ++p)
            if (p < P) tc::tmem_ldk<K>(base + (uint32_t)(t * 48 + 16 * p), c[p]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < K; ++j)
            v[t][j] = P == 3 ? (c[2][j] + c[1][j]) + c[0][j] : (P == 2 ? c[1][j] + c[0][j] : c[0][j]);
        }
      }
      tc::fence_before_sync();
      wg_sync(2);
      if (tid == 128) mbar_arrive(bfree);  // D may take stage 1 of the next term
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        int m3 = t * 128 + quarter * 32 + lane;
        if (t < T && m3 < rows && ((keep >> (m3 / k2)) & 1u)) {
#pragma unroll
          for (int j = 0; j < K; ++j) acc[t][j] = fma(cm, widen(v[t][j]), acc[t][j]);
        }
      }
    }
    if (bad) abort_flag = 1;
    // write the destinations: row (i, ix, iy), columns iz
    if (!bad) {
#pragma unroll
      for (int t = 0; t < TM; ++t) {
        int m3 = t * 128 + quarter * 32 + lane;
        if (t < T && m3 < rows) {
          int i = m3 / k2, rem = m3 - i * k2;
          int64_t dst = (int64_t)tile * G + i;
          if (dst < a.n_dest) {
            double *o = a.out_coeffs + dst * k3 + (int64_t)rem * k;
#pragma unroll
            for (int j = 0; j < K; ++j) o[j] = acc[t][j];
            if (rem == 0) a.out_keys[dst] = a.dest_key[dst];
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (abort_flag) {
    // let any copy or MMA still in flight finish before the tensor memory is released: a
    // commit tracks every tcgen05 operation this thread issued before it
    if (tid == 0) {
      atomicExch(a.err, 1);
      tc::mma_commit(tc::smem_u32(&bar_drain));
      tc::mbar_wait(tc::smem_u32(&bar_drain), 0, WAIT_CYCLES);
    }
    __syncthreads();
  }
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols_for(K, V));
}

// ---------------------------------------------------------------- work-list kernels
__global__ void key2_kernel(int64_t P, int G, const int *perm, const int *did, const uint64_t *dest_key,
                            const int *rec_l, uint64_t *key2, int *val2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int p = perm[i];
  uint64_t tile = (uint64_t)((did[i] - 1) / G);
  uint64_t lev = (uint64_t)key_level(dest_key[did[i] - 1]);
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
  const int k = op.k;
  if (k & 1) return fail(MRA_ERR_UNSUPPORTED, "split apply: odd k=%d not supported (use MRA_PREC_FP64)", k);
  const int v = (o.tile_variant == 1 && (k == 6 || k == 8 || k == 10)) ? 1 : 0;
  const int G = g_for(k, v);
  const int T = (G * k * k + 127) / 128;
  if (T > tm_for(k, v)) return fail(MRA_ERR_UNSUPPORTED, "split apply: tile shape for k=%d", k);
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
  key2_kernel<<<g, 256, 0, s>>>(P, G, wk.perm, wk.did, wk.dest_key, wk.rec_l, key2, val2);
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
  size_t smem = (size_t)2 * a.P * T * TILE_BYTES + 6 * BSTAGE_BYTES;
  void (*kern)(SplitArgs) = nullptr;
  switch (k * 2 + v) {
    case 4: kern = apply_split_kernel<2, 0>; break;
    case 8: kern = apply_split_kernel<4, 0>; break;
    case 12: kern = apply_split_kernel<6, 0>; break;
    case 13: kern = apply_split_kernel<6, 1>; break;
    case 16: kern = apply_split_kernel<8, 0>; break;
    case 17: kern = apply_split_kernel<8, 1>; break;
    case 20: kern = apply_split_kernel<10, 0>; break;
    case 21: kern = apply_split_kernel<10, 1>; break;
    case 24: kern = apply_split_kernel<12, 0>; break;
    case 28: kern = apply_split_kernel<14, 0>; break;
    default: kern = apply_split_kernel<16, 0>; break;
  }
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
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
