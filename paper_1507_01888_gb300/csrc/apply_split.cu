// apply_split.cu -- split-precision tensor-core apply (tcgen05, sm_103a).
//
// The three mode products of every kept term (Sec. 2.3),
//     t1 = s x_1 Rx,  t2 = t1 x_2 Ry,  t3 = t2 x_3 Rz,  r += c_m t3,
// run as BF16 tcgen05 MMAs with FP32 accumulation in tensor memory; every FP64
// or FP32 operand x is split into P BF16 pieces x = x0 + x1 (+ x2) and the
// products x_p y_q with p + q < P are kept.  The Gaussian-term sums and the
// per-box accumulation are compensated FP32 sums in registers (a sum and its Kahan
// correction per coefficient), formed into FP64 at the end.
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
// Stage 3 multiplies by c_m R_z.  Each term's FP32 stage-3 output is added into per-slot
// compensated FP32 sums (Kahan); in one-slot tiles two consecutive terms are first summed in
// the tensor-memory accumulator (JOIN).
#include <atomic>

#include <cub/cub.cuh>

#include "apply_internal.cuh"
#include "split_common.cuh"
#include "tcgen05.cuh"

namespace mra {

namespace {

using namespace split;

constexpr int SPLIT_THREADS = 256;      // 8 warps: two warps per tensor-memory lane quarter
constexpr int BTERM_BYTES = 3 * BSTAGE_BYTES;   // the three blocks (x, y, z) of one term
constexpr int NBUF = 4;                         // most block buffers a CTA uses
constexpr int RING = 4;                         // term-info ring from warpgroup 0 to 1
constexpr int MAX_G = 32;
constexpr int JOIN = 2;                         // terms summed in tensor memory per flush


struct SplitArgs {
  int k, M, P;
  const unsigned char *Bsplit;    // per block: 3 pieces x 512 B (K-major core-matrix layout)
  const unsigned char *Bsplit_c;  // the same for c_m R (stage 3 carries the term coefficient)
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
  int inject_stall;  // test hook: CTA 0 never issues the block copies of its first term
  int64_t n_src, n_rec, n_blocks;  // sizes for the index checks of the checking build
};

// Tile shapes for an even k.  A CTA owns G consecutive destination boxes (slots) whose
// G k^2 operand rows fill T <= TT tiles of 128 rows.  Tensor memory holds the stage-1
// and stage-2 outputs (48 columns per tile each: three 16-column piece groups) and the
// stage-3 output (32 columns per tile: two groups): 128 T columns.  TT = 4 takes the whole
// tensor memory (one CTA per SM); TT = 2 leaves room for a second CTA on the SM and TT = 1
// for four.
__host__ __device__ constexpr int g_for(int k, int tt) {
  return (128 * tt) / (k * k) > MAX_G ? MAX_G : (128 * tt) / (k * k);
}
__host__ __device__ constexpr int t_for(int k, int tt) { return (g_for(k, tt) * k * k + 127) / 128; }
__host__ __device__ constexpr uint32_t tmem_cols_for(int T) { return T <= 1 ? 128u : (T <= 2 ? 256u : 512u); }
// block buffers (terms whose blocks are in shared memory) and how many terms ahead the
// copies run: the one-tile shape keeps three buffers so that four CTAs fit on an SM
__host__ __device__ constexpr int nbuf_for(int tt) { return tt == 1 ? 3 : NBUF; }
// CTAs per SM the launch bounds ask for: TT = 1 fills the 512 tensor-memory columns with
// four CTAs of 128 columns each
__host__ __device__ constexpr int minb_for(int tt) { return tt == 1 ? 4 : 4 / tt; }
// slots whose rows [i k^2, (i+1) k^2) meet tile t's rows [128 t, 128 t + 128)
__host__ __device__ constexpr uint32_t tile_slots(int t, int k2, int G) {
  uint32_t m = 0;
  for (int i = 0; i < G; ++i)
    if (i * k2 < 128 * (t + 1) && (i + 1) * k2 > 128 * t) m |= 1u << i;
  return m;
}

// Warp roles and the term pipeline.  Terms of a group flow through three MMA stages:
//   warpgroup 0 (warps 0-3) stages each group's sources (A1), turns the stage-1 output
//     D1 into the stage-2 operand A2; its threads 0, 32 and 64 issue the stage-1 MMAs, the
//     block copies and the stage-2 MMAs;
//   warpgroup 1 (warps 4-7) turns the stage-2 output D2 into the stage-3 operand A3; its
//     thread 160 issues the stage-3 MMAs into D3 (the coefficient c_m is folded into the
//     stage-3 blocks); while the next term's stage 2 runs it adds D3 into the per-slot
//     sums, for the slots that keep the term.
// So warpgroup 0 works on term j+1 while warpgroup 1 works on term j.  Tiles of 128 rows
// that hold no slot keeping the term are skipped in all three stages.
// mbarriers (one arrival each): bb[b] block copies landed; s1/s2/s3 stage done (commit);
// ring_full term info published; d2_free D2 read out; b_free[b] block buffer b released
// by the stage-3 MMAs that read it.  Each wait is bounded and gives up when the other
// warpgroup has aborted.
template <int K, int TT>
__global__ void __launch_bounds__(SPLIT_THREADS, minb_for(TT)) apply_split_kernel(SplitArgs a) {
  constexpr int k = K, k2 = K * K, k3 = K * K * K;
  constexpr int G = g_for(K, TT), rows = G * k2, T = t_for(K, TT);
  constexpr uint32_t NCOL = tmem_cols_for(T);
  constexpr int NB = nbuf_for(TT), AHEAD = NB - 2;  // block buffers; copies run AHEAD terms ahead
  extern __shared__ __align__(1024) unsigned char smem[];
  const int P = a.P;
  const int ptile = P * T * TILE_BYTES;
  unsigned char *A1 = smem;              // [P][T] tiles: stage-1 operand (sources)
  unsigned char *A2 = A1 + ptile;        // [P][T] tiles: stage-2 operand
  unsigned char *A3 = A2 + ptile;        // [P][T] tiles: stage-3 operand
  unsigned char *Bt = A3 + ptile;        // [NB][3 stages][1536]: the blocks of a term
  __shared__ __align__(8) uint64_t bar_s1, bar_s2, bar_s3, bar_ring, bar_d2free, bar_drain0, bar_drain1, bar_drain2;
  __shared__ __align__(8) uint64_t bar_bb[NBUF], bar_bfree[NBUF];
  __shared__ uint32_t tmem_holder;
  __shared__ int slot_src[MAX_G];
  __shared__ uint64_t slot_mask[MAX_G][2];
  __shared__ uint64_t uni[2];
  __shared__ int g_level, g_l, total_it, g_nterms;
  __shared__ unsigned char g_terms[MRA_MAX_TERMS];
  __shared__ uint32_t ring_keep[RING];
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, quarter = warp & 3;
  const int tile = blockIdx.x;
  const int g0 = a.tile_gstart[tile], g1 = a.tile_gstart[tile + 1];

  {  // zero the operand tiles once: contraction and row padding stay zero
    int4 *z = (int4 *)smem;
    int n16 = (3 * ptile) / 16;
    for (int i = tid; i < n16; i += SPLIT_THREADS) z[i] = make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(&bar_s1), 1);
    tc::mbar_init(tc::smem_u32(&bar_s2), 1);
    tc::mbar_init(tc::smem_u32(&bar_s3), 1);
    tc::mbar_init(tc::smem_u32(&bar_ring), 1);
    tc::mbar_init(tc::smem_u32(&bar_d2free), 1);
    tc::mbar_init(tc::smem_u32(&bar_drain0), 1);
    tc::mbar_init(tc::smem_u32(&bar_drain1), 1);
    tc::mbar_init(tc::smem_u32(&bar_drain2), 1);
    for (int b = 0; b < NB; ++b) {
      tc::mbar_init(tc::smem_u32(&bar_bb[b]), 1);
      tc::mbar_init(tc::smem_u32(&bar_bfree[b]), 1);
    }
    abort_flag = 0;
    total_it = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_holder), NCOL);
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
  const uint32_t tD1 = tmem, tD2 = tmem + 48u * T, tD3 = tmem + 96u * T;
  const uint32_t bs1 = tc::smem_u32(&bar_s1), bs2 = tc::smem_u32(&bar_s2), bs3 = tc::smem_u32(&bar_s3);
  const uint32_t bring = tc::smem_u32(&bar_ring), bd2free = tc::smem_u32(&bar_d2free);
  const int nit = total_it;
  // instruction descriptor of an M=128 x N x 16 MMA (A MN-major, B K-major), N = 16 n
  auto idesc_n = [](int n) { return tc::idesc_bf16(128, 16 * n, 1, 0); };
  auto tiles_of = [&](uint32_t keep) -> uint32_t {
    uint32_t tl = 0;
#pragma unroll
    for (int t = 0; t < T; ++t)
      if (keep & tile_slots(t, k2, G)) tl |= 1u << t;
    return tl;
  };
  auto adesc = [&](const unsigned char *A, int p, int t) {
    return tc::smem_desc(tc::smem_u32(A + (p * T + t) * TILE_BYTES), 128, MG_BYTES);
  };
  auto bdesc = [&](const unsigned char *B) { return tc::smem_desc(tc::smem_u32(B), 128, 256); };
  // stages 1 and 2: A piece p times B pieces 0..P-1-p (stacked along N) into column
  // groups p..P-1 of the tile's 48 columns
  auto issue_stacked = [&](uint32_t d, const unsigned char *A, const unsigned char *B, uint32_t tiles) {
    for (int t = 0; t < T; ++t) {
      if (!((tiles >> t) & 1u)) continue;
      for (int p = 0; p < P; ++p)
        tc::mma_bf16(d + (uint32_t)(t * 48 + 16 * p), adesc(A, p, t), bdesc(B), idesc_n(P - p), p > 0 ? 1u : 0u);
    }
  };
  // store units of a thread's run: 16-byte core-matrix rows when 8 divides k, else 4-byte pairs
  constexpr int U = K % 8 == 0 ? K / 8 : K / 2;
  // shared-memory addresses of the store units of element [contraction a][rows (i, b, 0..k-1)]
  // in the first piece of operand A (the others follow at T * TILE_BYTES): fixed per thread
  auto run_addrs = [&](const unsigned char *A, int mrow, int a_idx, uint32_t *addr) {
    const uint32_t a0 = tc::smem_u32(A);
#pragma unroll
    for (int u = 0; u < U; ++u) addr[u] = a0 + a_off(mrow + (K % 8 == 0 ? 8 : 2) * u, a_idx);
  };
  auto st32 = st_shared32;
  auto st128 = st_shared128;
  // a thread's k values split into P pieces, stored at its precomputed unit addresses
  auto store_units = [&](const uint32_t *addr, const float *v) {
    const uint32_t stride = T * TILE_BYTES;
    if constexpr (K % 8 == 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          __nv_bfloat162 h0, h1, h2;
          split_pair(v[8 * u + 2 * h], v[8 * u + 2 * h + 1], h0, h1, h2);
          w0[h] = *(uint32_t *)&h0;
          w1[h] = *(uint32_t *)&h1;
          w2[h] = *(uint32_t *)&h2;
        }
        st128(addr[u], w0[0], w0[1], w0[2], w0[3]);
        st128(addr[u] + stride, w1[0], w1[1], w1[2], w1[3]);
        if (P > 2) st128(addr[u] + 2 * stride, w2[0], w2[1], w2[2], w2[3]);
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        __nv_bfloat162 h0, h1, h2;
        split_pair(v[2 * u], v[2 * u + 1], h0, h1, h2);
        st32(addr[u], *(uint32_t *)&h0);
        st32(addr[u] + stride, *(uint32_t *)&h1);
        if (P > 2) st32(addr[u] + 2 * stride, *(uint32_t *)&h2);
      }
    }
  };
  // the first K columns of each of the P piece groups of tile t, summed smallest first
  // (groups P-1 and P-2 first, then group 0: two loads in flight at a time)
  auto load_d = [&](uint32_t dbase, int t, float *v) {
    const uint32_t base = dbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(t * 48);
    float c[2][K];
    if (P == 3) {
      tc::tmem_ldk<K>(base + 32u, c[0]);
      tc::tmem_ldk<K>(base + 16u, c[1]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] = c[0][j] + c[1][j];
    } else {
      tc::tmem_ldk<K>(base + 16u, v);
      tc::tmem_ld_wait();
    }
    tc::tmem_ldk<K>(base, c[0]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] += c[0][j];
  };

  if (wg == 0) {
    // ======================================================= warpgroup 0
    // where this thread's stage-1 output row (i, jy, jz) goes in the stage-2 operand:
    // element [jy][(i, jz, 0..k-1)]
    uint32_t a2_addr[T][U];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int m1 = min(t * 128 + quarter * 32 + lane, rows - 1);
      const int i = m1 / k2, rem = m1 - i * k2, jy = rem / k, jz = rem - jy * k;
      run_addrs(A2, i * k2 + jz * k, jy, a2_addr[t]);
    }
    uint32_t p1 = 0;
    int it = 0;
    int nfetch = 0;  // block copies issued (thread 32), for iterations 0 .. nfetch-1 in order
    bool bad = false;
    // copies of the three blocks (m; lx, ly, lz) of iteration `i` into buffer i % NB, once
    // the stage-3 MMAs of iteration i - NB (the buffer's previous user) are done
    auto fetch = [&](int i, int m, int64_t lbase, int nl, int Dop, int lx, int ly, int lz) -> bool {
      const int b = i % NB;
      if (i >= NB &&
          !tc::mbar_wait_or_abort(tc::smem_u32(&bar_bfree[b]), (uint32_t)((i / NB - 1) & 1), WAIT_CYCLES, &abort_flag))
        return false;
      unsigned char *Bb = Bt + b * BTERM_BYTES;
      const uint32_t bar = tc::smem_u32(&bar_bb[b]);
      if (a.inject_stall && blockIdx.x == 0 && i == 0) {  // the copies never land: the waits run out
        ++nfetch;
        return true;
      }
      tc::mbar_arrive_expect_tx(bar, 3 * BSTAGE_BYTES);
      const int64_t blk0 = lbase + (int64_t)m * nl + Dop;
      const int64_t bx = MRA_IDX(blk0 + lx, a.n_blocks), by = MRA_IDX(blk0 + ly, a.n_blocks),
                    bz = MRA_IDX(blk0 + lz, a.n_blocks);
      tc::bulk_g2s(tc::smem_u32(Bb), a.Bsplit + bx * BSTAGE_BYTES, BSTAGE_BYTES, bar);
      tc::bulk_g2s(tc::smem_u32(Bb + BSTAGE_BYTES), a.Bsplit + by * BSTAGE_BYTES, BSTAGE_BYTES, bar);
      tc::bulk_g2s(tc::smem_u32(Bb + 2 * BSTAGE_BYTES), a.Bsplit_c + bz * BSTAGE_BYTES, BSTAGE_BYTES, bar);
      ++nfetch;
      return true;
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
        int i = MRA_IDX(a.val2[MRA_IDX(r, a.n_rec)], a.n_rec);
        int p = MRA_IDX(a.perm[i], a.n_rec);
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
      if (tid == 32) {  // the group's terms in ascending order; blocks of its first AHEAD terms
        int n = 0;
        uint64_t b0 = uni[0], b1 = uni[1];
        while (b0) { g_terms[n++] = (unsigned char)(__ffsll((long long)b0) - 1); b0 &= b0 - 1; }
        while (b1) { g_terms[n++] = (unsigned char)(64 + __ffsll((long long)b1) - 1); b1 &= b1 - 1; }
        g_nterms = n;
        for (int j = 0; j < AHEAD && j < n; ++j)
          if (!fetch(it + j, g_terms[j], lbase, nl, Dop, ldx, ldy, ldz)) abort_flag = 1;
      }
      // stage-1 operand: sources, rows (i, jy, jz), contraction jx (FP64 -> FP32 -> 3 BF16
      // pieces).  The previous group's stage-1 MMAs are complete (their output was read).
      for (int e = tid; e < G * k3 / 2; e += 128) {
        int e2 = 2 * e;
        int i = e2 / k3, rest = e2 - i * k3;
        int jx = rest / k2, q = rest - jx * k2;
        int src = slot_src[i];
        double2 xx = make_double2(0.0, 0.0);
        if (src >= 0) xx = *(const double2 *)(a.in_coeffs + (int64_t)MRA_IDX(src, a.n_src) * k3 + rest);
        __nv_bfloat162 h0, h1, h2;
        split_pair((float)xx.x, (float)xx.y, h0, h1, h2);
        uint32_t off = a_off(i * k2 + q, jx);
        *(__nv_bfloat162 *)(A1 + off) = h0;
        *(__nv_bfloat162 *)(A1 + T * TILE_BYTES + off) = h1;
        if (P > 2) *(__nv_bfloat162 *)(A1 + 2 * T * TILE_BYTES + off) = h2;
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      if (wg_vote_or(1, abort_flag)) { bad = true; break; }
      const int nt = g_nterms;
      for (int j = 0; j < nt; ++j, ++it) {
        const int m = g_terms[j];
        const int b = it % NB;
        const unsigned char *Bb = Bt + b * BTERM_BYTES;
        uint32_t keep = 0;
        for (int i = 0; i < G; ++i) keep |= (uint32_t)((slot_mask[i][m >> 6] >> (m & 63)) & 1ull) << i;
        const uint32_t tiles = tiles_of(keep);
        // asynchronous issue is spread over three threads of different warps, so that
        // its latency overlaps: thread 0 stage 1, thread 32 the block copies AHEAD terms
        // ahead, thread 64 stage 2
        if (tid == 0) {
          bool ok = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / NB) & 1), WAIT_CYCLES, &abort_flag);
          if (ok) {
            tc::fence_after_sync();
            issue_stacked(tD1, A1, Bb, tiles);  // ---- stage 1: rows (i, jy, jz), contraction jx
            tc::mma_commit(bs1);
          } else {
            abort_flag = 1;
          }
        }
        if (tid == 32 && j + AHEAD < nt && !fetch(it + AHEAD, g_terms[j + AHEAD], lbase, nl, Dop, ldx, ldy, ldz))
          abort_flag = 1;
        // one warp polls the barriers; the others sleep in the vote.  A2 is free once the
        // previous term's stage 2 is done.
        bool ok = true;
        if (quarter == 0) {
          ok = tc::mbar_wait_or_abort(bs1, p1, WAIT_CYCLES, &abort_flag);
          if (ok && it > 0) ok = tc::mbar_wait_or_abort(bs2, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
        }
        p1 ^= 1u;
        if (wg_vote_or(1, !ok || abort_flag)) { bad = true; break; }
        tc::fence_after_sync();
        // stage-1 output -> stage-2 operand: element [jy][(i, jz, ix)]
#pragma unroll
        for (int t = 0; t < T; ++t) {
          if (!((tiles >> t) & 1u)) continue;
          float v[K];
          load_d(tD1, t, v);
          if (t * 128 + quarter * 32 + lane < rows) store_units(a2_addr[t], v);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        wg_sync(1);
        if (tid == 64) {  // ---- stage 2: rows (i, jz, ix), contraction jy
          bool ok2 = it == 0 || tc::mbar_wait_or_abort(bd2free, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
          if (ok2) {
            ring_keep[it % RING] = keep;
            mbar_arrive(bring);
            ok2 = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / NB) & 1), WAIT_CYCLES, &abort_flag);
          }
          if (ok2) {
            tc::fence_after_sync();
            issue_stacked(tD2, A2, Bb + BSTAGE_BYTES, tiles);
            tc::mma_commit(bs2);
          } else {
            abort_flag = 1;
          }
        }
      }
    }
    if (bad) abort_flag = 1;
    // block copies still in flight (after an abort) land before the CTA exits, and every
    // MMA an issuing thread started is complete before the tensor memory is released
    if (tid == 32) {
      for (int b = 0; b < NB && b < nfetch; ++b) {
        const int uses = (nfetch - 1 - b) / NB + 1;  // copies into buffer b
        tc::mbar_wait(tc::smem_u32(&bar_bb[b]), (uint32_t)((uses - 1) & 1), WAIT_CYCLES);
      }
    }
    if (tid == 0 || tid == 64) {
      const uint32_t bd = tc::smem_u32(tid == 0 ? &bar_drain0 : &bar_drain2);
      tc::mma_commit(bd);
      tc::mbar_wait(bd, 0, WAIT_CYCLES);
    }
  } else {
    // ======================================================= warpgroup 1
    // where this thread's stage-2 output row (i, jz, ix) goes in the stage-3 operand:
    // element [jz][(i, ix, 0..k-1)]
    uint32_t a3_addr[T][U];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int m2 = min(t * 128 + quarter * 32 + lane, rows - 1);
      const int i = m2 / k2, rem = m2 - i * k2, jz = rem / k, ix = rem - jz * k;
      run_addrs(A3, i * k2 + ix * k, jz, a3_addr[t]);
    }
    // per-slot sums as FP32 pairs hi + lo, added to with compensated (Kahan) summation on the
    // FP32 pipe; the FP64 pipe (1/64 rate) only forms hi + lo at the end.  In one-slot tiles up
    // to JOIN consecutive terms are summed in D3 by the stage-3 MMAs before one flush adds them.
    float hi[T][K], lo[T][K];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int j = 0; j < K; ++j) hi[t][j] = lo[t][j] = 0.f;
    bool bad = false;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    // add the terms summed in D3 (tiles `tl`, kept by slots `kp`) into the sums of this
    // thread's rows; rows of slots that do not keep them are skipped
    auto flush = [&](uint32_t tl, uint32_t kp) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        if (!((tl >> t) & 1u)) continue;
        const uint32_t base = tD3 + lane_off + (uint32_t)(t * 32);
        float c0[K], c1[K];
        tc::tmem_ldk<K>(base, c0);
        tc::tmem_ldk<K>(base + 16u, c1);
        tc::tmem_ld_wait();
        const int m3 = t * 128 + quarter * 32 + lane;
        if (m3 < rows && ((kp >> (m3 / k2)) & 1u)) {
#pragma unroll
          for (int j = 0; j < K; ++j) {  // lo holds minus the running compensation
            const float y = (c1[j] + c0[j]) + lo[t][j];
            const float s = hi[t][j] + y;
            lo[t][j] = y - (s - hi[t][j]);
            hi[t][j] = s;
          }
        }
      }
    };
    uint32_t prev_tiles = 0, prev_keep = 0;
    int joined = 0;  // terms summed in D3 since its last flush
    for (int it = 0; it < nit; ++it) {
      // one warp polls the barriers; the others sleep in the vote.  Then the previous
      // term's stage 3 is done too: A3 is free and D3 holds its output
      bool ok = true;
      if (quarter == 0) {
        ok = tc::mbar_wait_or_abort(bs2, (uint32_t)(it & 1), WAIT_CYCLES, &abort_flag) &&
             tc::mbar_wait_or_abort(bring, (uint32_t)(it & 1), WAIT_CYCLES, &abort_flag);
        if (ok && it > 0) ok = tc::mbar_wait_or_abort(bs3, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
      }
      if (wg_vote_or(2, !ok || abort_flag)) { bad = true; break; }
      tc::fence_after_sync();
      const uint32_t keep = ring_keep[it % RING];
      const uint32_t tiles = tiles_of(keep);
      // D2 -> registers, then D2 is released for the next term's stage 2
      float v[T][K];
#pragma unroll
      for (int t = 0; t < T; ++t)
        if ((tiles >> t) & 1u) load_d(tD2, t, v[t]);
      tc::fence_before_sync();
      wg_sync(2);
      if (tid == 128) mbar_arrive(bd2free);
      // stage-2 output -> stage-3 operand: element [jz][(i, ix, iy)]
#pragma unroll
      for (int t = 0; t < T; ++t) {
        if (!((tiles >> t) & 1u)) continue;
        if (t * 128 + quarter * 32 + lane < rows) store_units(a3_addr[t], v[t]);
      }
      // this term's stage 3 adds onto D3 when the tile holds one slot and D3 has room;
      // otherwise D3 is flushed first and overwritten.  With several slots the rounding of a
      // slot's sum would depend on which other slots share its tile (joins need equal keep
      // masks), and a destination's result would change with how its function is batched.
      const bool join = G == 1 && joined > 0 && joined < JOIN && keep == prev_keep;
      if (joined > 0 && !join) {
        flush(prev_tiles, prev_keep);
        joined = 0;
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      wg_sync(2);
      if (tid == 160) {  // a thread of another warp than the polling one issues stage 3
        const int b = it % NB;
        const unsigned char *B3 = Bt + b * BTERM_BYTES + 2 * BSTAGE_BYTES;
        bool okb = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / NB) & 1), WAIT_CYCLES, &abort_flag);
        if (okb) {
          tc::fence_after_sync();
          // ---- stage 3: rows (i, ix, iy), contraction jz, B = c_m R_z pieces.  Column
          // group 0 gets x0 y0 alone, group 1 the other products x_p y_q with p + q < P,
          // so the small products are summed among themselves
          for (int t = 0; t < T; ++t) {
            if (!((tiles >> t) & 1u)) continue;
            const uint32_t d = tD3 + (uint32_t)(t * 32);
            tc::mma_bf16(d, adesc(A3, 0, t), bdesc(B3), idesc_n(2), join ? 1u : 0u);      // x0 [y0 y1]
            tc::mma_bf16(d + 16u, adesc(A3, 1, t), bdesc(B3), idesc_n(1), 1u);            // x1 y0
            if (P == 3) {
              tc::mma_bf16(d + 16u, adesc(A3, 1, t), bdesc(B3 + BPIECE_BYTES), idesc_n(1), 1u);      // x1 y1
              tc::mma_bf16(d + 16u, adesc(A3, 2, t), bdesc(B3), idesc_n(1), 1u);                     // x2 y0
              tc::mma_bf16(d + 16u, adesc(A3, 0, t), bdesc(B3 + 2 * BPIECE_BYTES), idesc_n(1), 1u);  // x0 y2
            }
          }
          tc::mma_commit(bs3);
          tc::mma_commit(tc::smem_u32(&bar_bfree[b]));
        } else {
          abort_flag = 1;
        }
      }
      prev_tiles = tiles;
      prev_keep = keep;
      ++joined;
    }
    if (!bad && nit > 0) {
      bool ok = quarter != 0 || tc::mbar_wait_or_abort(bs3, (uint32_t)((nit - 1) & 1), WAIT_CYCLES, &abort_flag);
      if (wg_vote_or(2, !ok || abort_flag)) {
        bad = true;
      } else {
        tc::fence_after_sync();
        flush(prev_tiles, prev_keep);
      }
    }
    if (bad) abort_flag = 1;
    // write the destinations: row (i, ix, iy), columns iz
    if (!bad) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        int m3 = t * 128 + quarter * 32 + lane;
        if (m3 < rows) {
          int i = m3 / k2, rem = m3 - i * k2;
          int64_t dst = (int64_t)tile * G + i;
          if (dst < a.n_dest) {
            double *o = a.out_coeffs + dst * k3 + (int64_t)rem * k;
#pragma unroll
            for (int j = 0; j < K; ++j) o[j] = (double)hi[t][j] + (double)lo[t][j];
            if (rem == 0) a.out_keys[dst] = a.dest_key[dst];
          }
        }
      }
    }
    if (tid == 160) {
      tc::mma_commit(tc::smem_u32(&bar_drain1));
      tc::mbar_wait(tc::smem_u32(&bar_drain1), 0, WAIT_CYCLES);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (abort_flag && tid == 0) atomicExch(a.err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

// ---------------------------------------------------------------- work-list kernels
// Fixed-size (graph) mode: the kernel's error word into the graph's status.
__global__ void fixed_err_kernel(const int *err, int *status) {
  if (*err == 1) atomicOr(status, 8);
  else if (*err) atomicOr(status, 16);
}

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
// x R (N = output index i, K = input index j), element (i, j) at
// (i/8)*256 + (j/8)*128 + (i%8)*16 + (j%8)*2 of a 512-byte piece; zero outside k x k.  Blocks
// are numbered m * nl + (l + D) within one level; x = c[m] when c is given, else 1.  Piece p
// of block (m, l) sits at byte (m nl + l + D) 1536 + p 512 (block-major: the three pieces of a
// block together), or with piece_major at (m nl 3 + p nl + l + D) 512 (all displacements of
// one piece together, so that the pieces of consecutive displacements are consecutive).
__global__ void split_blocks_kernel(int64_t n_blocks, int k, int nl, const double *c, const double *R,
                                    unsigned char *out, int piece_major) {
  int64_t blk = blockIdx.x;
  if (blk >= n_blocks) return;
  const double x = c ? c[blk / nl] : 1.0;
  const int64_t m = blk / nl, l = blk - m * nl;
  for (int e = threadIdx.x; e < 256; e += blockDim.x) {
    int i = e / 16, j = e % 16;
    double y = (i < k && j < k) ? x * R[blk * k * k + i * k + j] : 0.0;
    __nv_bfloat16 pc[3];
    split3(y, pc[0], pc[1], pc[2]);
    uint32_t off = (i / 8) * 256 + (j / 8) * 128 + (i % 8) * 16 + (j % 8) * 2;
    for (int p = 0; p < 3; ++p) {
      const int64_t at = piece_major ? ((m * nl * 3 + p * nl + l) * BPIECE_BYTES)
                                     : (blk * BSTAGE_BYTES + p * BPIECE_BYTES);
      *(__nv_bfloat16 *)(out + at + off) = pc[p];
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- failure-path test hook
std::atomic<int> g_inject_stall{0};
bool take_injected_stall() { return g_inject_stall.exchange(0) != 0; }

void split_fixed_err(const int *err, int *status, cudaStream_t s) {
  fixed_err_kernel<<<counted(1), 1, 0, s>>>(err, status);
}

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

int split_blocks_build(Operator &op, cudaStream_t s, bool rebuild) {
  if (op.d_Rsplit && !rebuild) return MRA_OK;
  // three tables: the blocks R (stages 1 and 2) and c_m R (stage 3 of the destination-stationary
  // kernel), block-major; c_m R piece-major (stage 3 of the source-stationary kernel)
  if (!op.d_Rsplit) MRA_CUDA_TRY(cudaMalloc(&op.d_Rsplit, (size_t)3 * op.n_blocks * BSTAGE_BYTES));
  unsigned char *plain = (unsigned char *)op.d_Rsplit;
  unsigned char *scaled = plain + (size_t)op.n_blocks * BSTAGE_BYTES;
  unsigned char *zpack = plain + (size_t)2 * op.n_blocks * BSTAGE_BYTES;
  for (size_t li = 0; li < op.D.size(); ++li) {
    const int nl = 2 * op.D[li] + 1;
    const int64_t nb = (int64_t)op.M * nl, base = op.level_off[li];
    if (nb <= 0) continue;
    const double *R = op.d_R + base * op.k * op.k;
    split_blocks_kernel<<<counted((unsigned)nb), 128, 0, s>>>(nb, op.k, nl, nullptr, R, plain + base * BSTAGE_BYTES, 0);
    split_blocks_kernel<<<counted((unsigned)nb), 128, 0, s>>>(nb, op.k, nl, op.d_c, R, scaled + base * BSTAGE_BYTES, 0);
    split_blocks_kernel<<<counted((unsigned)nb), 128, 0, s>>>(nb, op.k, nl, op.d_c, R, zpack + base * BSTAGE_BYTES, 1);
    MRA_CUDA_TRY(cudaGetLastError());
  }
  return MRA_OK;
}

int apply_split_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o,
                    mra_tree_view &out, const ApplyWork &wk, mra_apply_stats *stats,
                    cudaStream_t s) {
  const int k = op.k;
  if (k > MRA_MAX_K) return fail(MRA_ERR_UNSUPPORTED, "split apply: order %d above %d (use MRA_PREC_FP64)", k, MRA_MAX_K);
  if (!op.d_Rsplit) return fail(MRA_ERR_ARG, "mra_apply: operator has no split blocks");
  if (k & 1) return fail(MRA_ERR_UNSUPPORTED, "split apply: odd k=%d not supported (use MRA_PREC_FP64)", k);
  const int tt = (k >= 4 && o.tile_variant == 1) ? 2 : (k >= 4 && k <= 10 && o.tile_variant == 2) ? 1 : 4;
  const int G = g_for(k, tt);
  const int T = t_for(k, tt);  // 128-row tiles per CTA
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
  key2_kernel<<<counted(g), 256, 0, s>>>(P, G, wk.perm, wk.did, wk.dest_key, wk.rec_l, key2, val2);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmpb, key2, key2s, val2, val2s, (int)P, 0, 64, s));
  groups_kernel<<<counted(g), 256, 0, s>>>(P, key2s, head, n_tiles);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp, tmpb, head, gid, (int)P, s));
  group_bounds_kernel<<<counted(g), 256, 0, s>>>(P, key2s, head, gid, grp_start, tile_gstart, n_tiles);
  MRA_CUDA_TRY(cudaGetLastError());

  SplitArgs a{};
  a.k = k;
  a.M = op.M;
  a.P = o.pieces;
  a.Bsplit = (const unsigned char *)op.d_Rsplit;
  a.Bsplit_c = a.Bsplit + (size_t)op.n_blocks * BSTAGE_BYTES;
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
  a.inject_stall = take_injected_stall() ? 1 : 0;
  a.n_src = in.n;
  a.n_rec = P;
  a.n_blocks = op.n_blocks;
  size_t smem = (size_t)3 * a.P * T * TILE_BYTES + (size_t)nbuf_for(tt) * BTERM_BYTES;
  // no more CTAs per SM than the tensor memory holds (512 columns): otherwise an extra
  // CTA's allocation would wait for a resident CTA to finish
  const size_t smem_floor = (size_t)233472 / (512 / tmem_cols_for(T) + 1);
  if (smem < smem_floor) smem = smem_floor;
  void (*kern)(SplitArgs) = nullptr;
  switch (k * 8 + tt) {
    case 2 * 8 + 4: kern = apply_split_kernel<2, 4>; break;
    case 4 * 8 + 4: kern = apply_split_kernel<4, 4>; break;
    case 4 * 8 + 2: kern = apply_split_kernel<4, 2>; break;
    case 4 * 8 + 1: kern = apply_split_kernel<4, 1>; break;
    case 6 * 8 + 4: kern = apply_split_kernel<6, 4>; break;
    case 6 * 8 + 2: kern = apply_split_kernel<6, 2>; break;
    case 6 * 8 + 1: kern = apply_split_kernel<6, 1>; break;
    case 8 * 8 + 4: kern = apply_split_kernel<8, 4>; break;
    case 8 * 8 + 2: kern = apply_split_kernel<8, 2>; break;
    case 8 * 8 + 1: kern = apply_split_kernel<8, 1>; break;
    case 10 * 8 + 4: kern = apply_split_kernel<10, 4>; break;
    case 10 * 8 + 2: kern = apply_split_kernel<10, 2>; break;
    case 10 * 8 + 1: kern = apply_split_kernel<10, 1>; break;
    case 12 * 8 + 2: kern = apply_split_kernel<12, 2>; break;
    case 12 * 8 + 4: kern = apply_split_kernel<12, 4>; break;
    case 14 * 8 + 2: kern = apply_split_kernel<14, 2>; break;
    case 14 * 8 + 4: kern = apply_split_kernel<14, 4>; break;
    case 16 * 8 + 2: kern = apply_split_kernel<16, 2>; break;
    default: kern = apply_split_kernel<16, 4>; break;
  }
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  if (wk.ev0) MRA_CUDA_TRY(cudaEventRecord(wk.ev0, s));
  kern<<<counted((unsigned)n_tiles), SPLIT_THREADS, smem, s>>>(a);
  MRA_CUDA_TRY(cudaGetLastError());
  if (wk.ev1) MRA_CUDA_TRY(cudaEventRecord(wk.ev1, s));
  if (wk.fx) {
    fixed_err_kernel<<<counted(1), 1, 0, s>>>(err, wk.fx->status);
    MRA_CUDA_TRY(cudaGetLastError());
    return MRA_OK;
  }
  int herr = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr == 1) return fail(MRA_ERR_TIMEOUT, "split apply: a tensor-core completion wait gave up");
  if (herr) return fail(MRA_ERR_ARG, "split apply: inconsistent work list (%d)", herr);
  (void)stats;
  return MRA_OK;
}

}  // namespace mra

namespace mra {
int debug_line_split(cudaStream_t s) { return debug_take_line(s); }
}  // namespace mra

extern "C" int mra_debug_inject_stall(void) {
  mra::g_inject_stall.store(1);
  return MRA_OK;
}
