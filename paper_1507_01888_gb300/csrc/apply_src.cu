// apply_src.cu -- source-stationary split-precision tensor-core apply (tcgen05, sm_103a).
//
// Every kept term (source b, displacement l = (lx, ly, lz), Gaussian term m) contributes
//     c_m  s_b x_1 R_{m,lx} x_2 R_{m,ly} x_3 R_{m,lz}                    (Sec. 2.3)
// to the destination b + l.  The first mode product depends on (b, m, lx) only and the first
// two on (b, m, lx, ly): the terms of one source with the same (lx, ly) and m differ only in
// their last block.  So the work is organised around the source:
//   * a CTA takes a tile of G sources of one level (their G k^2 coefficient rows fill one
//     128-row operand tile); their BF16 pieces are staged in shared memory once and reused for
//     every displacement and term;
//   * the tile's records are grouped by (lx, ly) and a window of three consecutive lz; for each
//     Gaussian term m that any record of the group keeps, one pass of three GEMMs runs on the
//     tensor cores:
//       stage 1: rows (i, jy, jz), contraction jx, block R_{m,lx}            -> D1[(i,jy,jz)][ix]
//       stage 2: rows (i, jz, ix), contraction jy, block R_{m,ly}            -> D2[(i,jz,ix)][iy]
//       stage 3: rows (i, ix, iy), contraction jz, blocks c_m R_{m,lz} of the three lz of the
//                window stacked along N                                    -> D3[(i,ix,iy)][(lz, iz)]
//     so one pass serves up to three terms;
//   * each record's sum over m (the partial result of source b for destination b + l) stays in
//     registers, as a plain FP32 sum or a compensated one (a sum and its Kahan correction per
//     coefficient; the `sums` option), and is written once, as FP32, to a partial buffer indexed
//     by the record; up to `join` consecutive terms kept by the same records are first summed by
//     the stage-3 MMAs in the tensor-memory accumulator;
//   * a second kernel sums the partials of every destination in FP32 pairs (error-free
//     TwoSum additions, about 48 bits), in the order of the records sorted on the destination
//     key, and writes each destination once in FP64 (no atomics on results).
// Operands are split into P BF16 pieces and the piece products p + q < P are kept; each stage
// stacks the B pieces along N (one MMA per A piece) into column groups g = p + q, which the
// epilogues sum smallest first.  The FP32 accumulation of one stage happens in tensor memory.
//
// Pipeline (two warpgroups, as in the destination-stationary kernel): warpgroup 0 stages the
// sources, turns D1 into the stage-2 operand and issues stages 1 and 2 and the block copies;
// warpgroup 1 turns D2 into the stage-3 operand and adds D3 into the record sums, and stage 3 is
// issued by a ninth warp (plain sums) or by a thread of warpgroup 1 (compensated sums), so the
// two warpgroups work on consecutive terms.  The kernel is persistent: CTAs take
// tiles from a device counter until none are left; tiles come heaviest first.
#include <cub/cub.cuh>

#include "apply_internal.cuh"
#include "split_common.cuh"
#include "tcgen05.cuh"

namespace mra {

namespace {

using namespace split;

constexpr int SRC_THREADS = 256;
constexpr int SRC_NB = 6;                          // block buffers (terms whose blocks are in shared memory)
constexpr int SRC_MAX_AHEAD = SRC_NB - 2;          // the block copies run up to this many terms ahead
constexpr int SRC_MAX_JOIN = 8;                    // most terms summed in tensor memory per flush
constexpr int SRC_RING = 4;                        // term-info ring from warpgroup 0 to 1
constexpr int SRC_MAX_G = 8;                       // sources per tile
constexpr int SRC_MAX_DAP = 2;                     // largest |l|_inf of the records (else the other kernel)
constexpr int SRC_SW = 2 * SRC_MAX_DAP + 1;        // (lx, ly) sweeps per dimension
constexpr int SRC_NWIN = (SRC_SW + 2) / 3;         // lz windows of three
constexpr int SRC_NG = SRC_SW * SRC_SW * SRC_NWIN; // groups per tile at most
constexpr int BX_OFF = 0, BY_OFF = BSTAGE_BYTES, BZ_OFF = 2 * BSTAGE_BYTES;
constexpr int BIT_BYTES = 2 * BSTAGE_BYTES + 3 * BSTAGE_BYTES;  // blocks x, y and the z window of one term
constexpr uint32_t D1_COL = 0, D2_COL = 48, D3_COL = 96;          // tensor-memory columns (3 groups of 16,
constexpr uint32_t SRC_TMEM_COLS = 256;                           // D3: 3 groups x 3 lz x 16)
constexpr int FLAG_GROUP_END = 1, FLAG_TERM = 2, FLAG_JOIN = 4;

__host__ __device__ constexpr int src_g(int k) {
  return (128 / (k * k)) > SRC_MAX_G ? SRC_MAX_G : 128 / (k * k);
}

struct SrcArgs {
  int k, M, P;
  const unsigned char *Bsplit;  // per block: 3 pieces x 512 B (stages 1, 2: the blocks R)
  const unsigned char *Bzpack;  // per (level, m): [piece][l][512 B] of c_m R (stage 3)
  const int *Dlev;              // operator displacement range per level
  int Dap[MRA_MAX_LEVEL + 1];   // records' displacement range per level (<= SRC_MAX_DAP)
  const int64_t *level_off;
  const uint64_t *in_keys;
  const double *in_coeffs;
  const int64_t *rec_cnt, *rec_off;  // records of each source: [rec_off[b], rec_off[b] + rec_cnt[b])
  const int *rec_l;
  const uint64_t *rec_mask;
  const int *tile_src;          // [n_tiles][G] source index, -1 = empty slot
  const int *n_tiles;           // device count
  int *tile_ctr;                // next tile (zero before the launch)
  float *partial;               // [n_rec][k^3]
  unsigned long long *pass_ctr; // passes of all CTAs (each CTA adds its own once)
  int *err;
  int inject_stall;             // test hook: the CTA that takes tile 0 never issues the copies of its first term
  int join;                     // terms summed in D3 by the stage-3 MMAs before one flush
  int join_all;                 // 1: join in tiles of several sources too (else those flush every term)
  int compensated;              // record sums: 1 = FP32 sum + Kahan correction, 0 = plain FP32 sum
  int ahead;                    // block copies run this many terms ahead (1 .. SRC_MAX_AHEAD)
  int64_t n_src, n_rec, n_blocks;
};

// PLAIN: record sums in plain FP32 (fewer registers), which leaves room for a ninth warp that issues
// stage 3, so that warpgroup 1 does not wait on that issue; otherwise compensated sums and thread
// 160 issues stage 3
template <int K, bool PLAIN>
__global__ void __launch_bounds__(PLAIN ? SRC_THREADS + 32 : SRC_THREADS, 2) apply_src_kernel(SrcArgs a) {
  constexpr int k2 = K * K, k3 = K * K * K;
  constexpr int G = src_g(K), rows = G * k2;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int P = a.P;
  unsigned char *A1 = smem;                    // [P] tiles: stage-1 operand (the tile's sources)
  unsigned char *A2 = A1 + 3 * TILE_BYTES;     // [P] tiles: stage-2 operand
  unsigned char *A3 = A2 + 3 * TILE_BYTES;     // [P] tiles: stage-3 operand
  unsigned char *Bt = A3 + 3 * TILE_BYTES;     // [SRC_NB][BIT_BYTES]: the blocks of a term
  // per-tile record table: record index and kept-term mask of (group, slot, lz in window)
  int *grp_rec = (int *)(Bt + SRC_NB * BIT_BYTES);                      // [SRC_NG][G][3]
  uint64_t *grp_mask = (uint64_t *)(grp_rec + SRC_NG * G * 3 + (SRC_NG * G * 3) % 2);  // [SRC_NG][G][3][2]
  uint64_t *grp_union = grp_mask + SRC_NG * G * 3 * 2;                  // [SRC_NG][2]
  __shared__ __align__(8) uint64_t bar_s1, bar_s2, bar_s3, bar_ring, bar_d2free, bar_drain0, bar_drain1, bar_drain2;
  __shared__ int s3_flags[SRC_RING];  // from warpgroup 1 to the stage-3 issuer: join / no more terms
  __shared__ volatile int s_nfetch;    // terms whose block copies thread 32 has issued
  __shared__ __align__(8) uint64_t bar_bb[SRC_NB], bar_bfree[SRC_NB];
  __shared__ uint32_t tmem_holder;
  __shared__ int t_src[SRC_MAX_G];
  __shared__ int s_tile, t_level, t_dap, t_dop;
  __shared__ long long t_lbase;
  __shared__ int ring_m[SRC_RING], ring_flags[SRC_RING];
  __shared__ uint32_t ring_keep[SRC_RING];
  __shared__ int ring_rec[SRC_RING][SRC_MAX_G * 3];
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, quarter = warp & 3;

  {  // zero the operand tiles once: contraction and row padding stay zero
    int4 *z = (int4 *)smem;
    const int n16 = (9 * TILE_BYTES) / 16;
    for (int i = tid; i < n16; i += (int)blockDim.x) z[i] = make_int4(0, 0, 0, 0);
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
    for (int b = 0; b < SRC_NB; ++b) {
      tc::mbar_init(tc::smem_u32(&bar_bb[b]), 1);
      tc::mbar_init(tc::smem_u32(&bar_bfree[b]), 1);
    }
    abort_flag = 0;
    s_nfetch = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_holder), SRC_TMEM_COLS);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t tD1 = tmem + D1_COL, tD2 = tmem + D2_COL, tD3 = tmem + D3_COL;
  const uint32_t bs1 = tc::smem_u32(&bar_s1), bs2 = tc::smem_u32(&bar_s2), bs3 = tc::smem_u32(&bar_s3);
  const uint32_t bring = tc::smem_u32(&bar_ring), bd2free = tc::smem_u32(&bar_d2free);
  auto idesc_n = [](int n) { return tc::idesc_bf16(128, 16 * n, 1, 0); };
  auto adesc = [&](const unsigned char *A, int p) {
    return tc::smem_desc(tc::smem_u32(A + p * TILE_BYTES), 128, MG_BYTES);
  };
  auto bdesc = [&](const unsigned char *B) { return tc::smem_desc(tc::smem_u32(B), 128, 256); };
  // A piece p times B pieces 0..P-1-p (stacked along N, nb blocks per piece) into column groups
  // p..P-1; the first MMA overwrites D unless acc0
  auto issue_stacked = [&](uint32_t d, const unsigned char *A, const unsigned char *B, int nb, uint32_t acc0) {
    for (int p = 0; p < P; ++p)
      tc::mma_bf16(d + (uint32_t)(16 * nb * p), adesc(A, p), bdesc(B), idesc_n(nb * (P - p)), p > 0 ? 1u : acc0);
  };
  // store units of a thread's run: 16-byte core-matrix rows when 8 divides k, else 4-byte pairs
  constexpr int U = K % 8 == 0 ? K / 8 : K / 2;
  auto run_addrs = [&](const unsigned char *A, int mrow, int a_idx, uint32_t *addr) {
    const uint32_t a0 = tc::smem_u32(A);
#pragma unroll
    for (int u = 0; u < U; ++u) addr[u] = a0 + a_off(mrow + (K % 8 == 0 ? 8 : 2) * u, a_idx);
  };
  // a thread's k values split into P pieces, stored at its precomputed unit addresses
  auto store_units = [&](const uint32_t *addr, const float *v) {
    const uint32_t stride = TILE_BYTES;
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
        st_shared128(addr[u], w0[0], w0[1], w0[2], w0[3]);
        st_shared128(addr[u] + stride, w1[0], w1[1], w1[2], w1[3]);
        if (P > 2) st_shared128(addr[u] + 2 * stride, w2[0], w2[1], w2[2], w2[3]);
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        __nv_bfloat162 h0, h1, h2;
        split_pair(v[2 * u], v[2 * u + 1], h0, h1, h2);
        st_shared32(addr[u], *(uint32_t *)&h0);
        st_shared32(addr[u] + stride, *(uint32_t *)&h1);
        if (P > 2) st_shared32(addr[u] + 2 * stride, *(uint32_t *)&h2);
      }
    }
  };
  // the first K columns of each of the P column groups (16 nb columns apart) starting at
  // column `col` of this warp's lanes, summed smallest first (groups P-1 and P-2 first, then
  // group 0: two loads in flight at a time)
  auto load_groups = [&](uint32_t col, int nb, float *v) {
    const uint32_t base = col + ((uint32_t)(32 * quarter) << 16);
    float c[2][K];
    if (P == 3) {
      tc::tmem_ldk<K>(base + 32u * nb, c[0]);
      tc::tmem_ldk<K>(base + 16u * nb, c[1]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] = c[0][j] + c[1][j];
    } else {
      tc::tmem_ldk<K>(base + 16u * nb, v);
      tc::tmem_ld_wait();
    }
    tc::tmem_ldk<K>(base, c[0]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] += c[0][j];
  };
  // warpgroup 1 hands a term (or the end) to the stage-3 issuer warp: named barrier 3, 128 + 32
  auto wg_arrive_issuer = [&]() { asm volatile("bar.arrive 3, 160;" ::: "memory"); };
  const int mrow = quarter * 32 + lane;  // this thread's row of the tile (lane of tensor memory)
  const int ahead = max(1, min(a.ahead, SRC_MAX_AHEAD));
  // tiles of several sources join only when asked: a join depends on all the tile's records,
  // so it would make a result depend on which sources share its tile
  const int join = (G == 1 || a.join_all) ? max(1, min(a.join, SRC_MAX_JOIN)) : 1;

  if (wg == 0) {
    // ======================================================= warpgroup 0
    // where this thread's stage-1 output row (i, jy, jz) goes in the stage-2 operand:
    // element [jy][(i, jz, 0..k-1)]
    uint32_t a2_addr[U];
    {
      const int m1 = min(mrow, rows - 1);
      const int i = m1 / k2, rem = m1 - i * k2, jy = rem / K, jz = rem - jy * K;
      run_addrs(A2, i * k2 + jz * K, jy, a2_addr);
    }
    uint32_t p1 = 0;
    int it = 0;       // terms issued by this CTA so far (all tiles)
    int nfetch = 0;   // block copies issued (thread 32), for iterations 0 .. nfetch-1 in order
    bool bad = false;
    bool stalled = false;  // test hook: set for the CTA that takes tile 0
    // the tile's iteration cursor of thread 32 (copies AHEAD terms ahead): group and the terms left
    int f_g = 0;
    uint64_t f_u0 = 0, f_u1 = 0;
    auto cursor_next = [&](int &g, uint64_t &u0, uint64_t &u1, int &m) -> bool {
      while (!(u0 | u1)) {
        if (++g >= SRC_NG) return false;
        u0 = grp_union[2 * g];
        u1 = grp_union[2 * g + 1];
      }
      if (u0) { m = __ffsll((long long)u0) - 1; u0 &= u0 - 1; }
      else { m = 64 + __ffsll((long long)u1) - 1; u1 &= u1 - 1; }
      return true;
    };
    // copies of the blocks of iteration i (term m of group g) into buffer i % SRC_NB, once
    // the stage-3 MMAs of iteration i - SRC_NB (the buffer's previous user) are done
    auto fetch = [&](int i, int g, int m) -> bool {
      const int b = i % SRC_NB;
      if (i >= SRC_NB &&
          !tc::mbar_wait_or_abort(tc::smem_u32(&bar_bfree[b]), (uint32_t)((i / SRC_NB - 1) & 1), WAIT_CYCLES,
                                  &abort_flag))
        return false;
      unsigned char *Bb = Bt + b * BIT_BYTES;
      const uint32_t bar = tc::smem_u32(&bar_bb[b]);
      ++nfetch;
      s_nfetch = nfetch;
      if (stalled) {  // the copies never land: the waits run out
        stalled = false;
        return true;
      }
      const int dap = t_dap, dop = t_dop, nl = 2 * dop + 1, sw = 2 * dap + 1;
      const int wi = g % SRC_NWIN, sxy = g / SRC_NWIN;
      const int lx = sxy / sw - dap, ly = sxy % sw - dap, lz0 = -dap + 3 * wi;
      const int lzf = max(lz0, -dop), lzl = min(lz0 + 2, dop), cnt = lzl - lzf + 1;
      const int64_t blk0 = t_lbase + (int64_t)m * nl + dop;
      const int64_t bx = MRA_IDX(blk0 + lx, a.n_blocks), by = MRA_IDX(blk0 + ly, a.n_blocks);
      const uint32_t zbytes = (uint32_t)(P * cnt * BPIECE_BYTES);
      tc::mbar_arrive_expect_tx(bar, 2 * BSTAGE_BYTES + zbytes);
      tc::bulk_g2s(tc::smem_u32(Bb + BX_OFF), a.Bsplit + bx * BSTAGE_BYTES, BSTAGE_BYTES, bar);
      tc::bulk_g2s(tc::smem_u32(Bb + BY_OFF), a.Bsplit + by * BSTAGE_BYTES, BSTAGE_BYTES, bar);
      // c_m R_{m,l} of the window's lz: piece q of block (m, l) at ((m nl) 3 + q nl + l + dop) 512 B
      const int64_t zreg = MRA_IDX(t_lbase + (int64_t)m * nl, a.n_blocks);
      const unsigned char *z0 = a.Bzpack + zreg * BSTAGE_BYTES;
      if (cnt == 3 && nl == 3) {
        tc::bulk_g2s(tc::smem_u32(Bb + BZ_OFF), z0, (uint32_t)(P * BSTAGE_BYTES), bar);
      } else {
        for (int q = 0; q < P; ++q)
          tc::bulk_g2s(tc::smem_u32(Bb + BZ_OFF + q * BSTAGE_BYTES + (lzf - lz0) * BPIECE_BYTES),
                       z0 + ((int64_t)q * nl + lzf + dop) * BPIECE_BYTES, (uint32_t)(cnt * BPIECE_BYTES), bar);
      }
      return true;
    };

    while (!bad) {
      // ---------------------------------------------------------------- next tile
      if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1);
      wg_sync(1);
      const int tile = s_tile;
      if (tile >= *a.n_tiles) break;
      if (a.inject_stall && tile == 0 && nfetch == 0) stalled = true;
      if (tid < G) t_src[tid] = a.tile_src[(int64_t)tile * G + tid];
      for (int e = tid; e < SRC_NG * G * 3; e += 128) {
        grp_rec[e] = -1;
        grp_mask[2 * e] = grp_mask[2 * e + 1] = 0ull;
      }
      for (int e = tid; e < 2 * SRC_NG; e += 128) grp_union[e] = 0ull;
      wg_sync(1);
      if (tid == 0) {
        const int b0 = MRA_IDX(t_src[0], a.n_src);
        const int n = key_level(a.in_keys[b0]);
        t_level = n;
        t_dop = a.Dlev[n];
        t_dap = a.Dap[n];
        t_lbase = a.level_off[n];
      }
      wg_sync(1);
      const int dap = t_dap, sw = 2 * dap + 1;
      // records of the tile's sources into the group table (a warp per slot)
      for (int i = quarter; i < G; i += 4) {
        const int src = t_src[i];
        if (src < 0) continue;
        const int64_t r0 = a.rec_off[MRA_IDX(src, a.n_src)], rc = a.rec_cnt[MRA_IDX(src, a.n_src)];
        for (int64_t r = lane; r < rc; r += 32) {
          const int64_t p = MRA_IDX(r0 + r, a.n_rec);
          const int lp = a.rec_l[p];
          const int lx = (lp & 255) - 128 + dap, ly = ((lp >> 8) & 255) - 128 + dap, lz = ((lp >> 16) & 255) - 128 + dap;
          if (lx < 0 || lx >= sw || ly < 0 || ly >= sw || lz < 0 || lz >= sw) {
            atomicExch(a.err, 2);
            continue;
          }
          const int g = (lx * sw + ly) * SRC_NWIN + lz / 3, w = lz % 3;
          const int e = (g * G + i) * 3 + w;
          const uint64_t m0 = a.rec_mask[2 * p], m1 = a.rec_mask[2 * p + 1];
          grp_rec[e] = (int)p;
          grp_mask[2 * e] = m0;
          grp_mask[2 * e + 1] = m1;
          atomicOr((unsigned long long *)&grp_union[2 * g], (unsigned long long)m0);
          atomicOr((unsigned long long *)&grp_union[2 * g + 1], (unsigned long long)m1);
        }
      }
      wg_sync(1);
      // thread 32: the copies of the tile's first AHEAD terms
      if (tid == 32) {
        f_g = -1;
        f_u0 = f_u1 = 0ull;
        int m;
        for (int j = 0; j < ahead; ++j) {
          int g0 = f_g;
          if (!cursor_next(f_g, f_u0, f_u1, m)) break;
          (void)g0;
          if (!fetch(it + j, f_g, m)) abort_flag = 1;
        }
      }
      // stage-1 operand: the tile's sources, rows (i, jy, jz), contraction jx (FP64 -> FP32 ->
      // P BF16 pieces).  The previous tile's stage-1 MMAs are complete (their output was read).
      for (int e = tid; e < G * k3 / 2; e += 128) {
        const int e2 = 2 * e;
        const int i = e2 / k3, rest = e2 - i * k3;
        const int jx = rest / k2, q = rest - jx * k2;
        const int src = t_src[i];
        double2 xx = make_double2(0.0, 0.0);
        if (src >= 0) xx = *(const double2 *)(a.in_coeffs + (int64_t)MRA_IDX(src, a.n_src) * k3 + rest);
        __nv_bfloat162 h0, h1, h2;
        split_pair((float)xx.x, (float)xx.y, h0, h1, h2);
        const uint32_t off = a_off(i * k2 + q, jx);
        *(__nv_bfloat162 *)(A1 + off) = h0;
        *(__nv_bfloat162 *)(A1 + TILE_BYTES + off) = h1;
        if (P > 2) *(__nv_bfloat162 *)(A1 + 2 * TILE_BYTES + off) = h2;
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      if (wg_vote_or(1, abort_flag)) { bad = true; break; }
      // ---------------------------------------------------------------- the tile's terms
      int cg = -1, cm = 0;
      uint64_t cu0 = 0ull, cu1 = 0ull;
      while (cursor_next(cg, cu0, cu1, cm)) {
        const int g = cg, m = cm;
        const bool group_end = !(cu0 | cu1);
        const int b = it % SRC_NB;
        const unsigned char *Bb = Bt + b * BIT_BYTES;
        uint32_t keep = 0;
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            const int e = (g * G + i) * 3 + w;
            keep |= (uint32_t)((grp_mask[2 * e + (m >> 6)] >> (m & 63)) & 1ull) << (3 * i + w);
          }
        // asynchronous issue is spread over three threads of different warps: thread 0
        // stage 1, thread 32 the block copies AHEAD terms ahead, thread 64 stage 2
        if (tid == 0) {
          bool ok = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / SRC_NB) & 1), WAIT_CYCLES,
                                           &abort_flag);
          if (ok) {
            tc::fence_after_sync();
            issue_stacked(tD1, A1, Bb + BX_OFF, 1, 0u);  // ---- stage 1: rows (i, jy, jz), contraction jx
            tc::mma_commit(bs1);
          } else {
            abort_flag = 1;
          }
        }
        if (tid == 32) {
          int m2;
          if (cursor_next(f_g, f_u0, f_u1, m2) && !fetch(it + ahead, f_g, m2)) abort_flag = 1;
        }
        bool ok = true;
        if (quarter == 0) {
          ok = tc::mbar_wait_or_abort(bs1, p1, WAIT_CYCLES, &abort_flag);
          if (ok && it > 0) ok = tc::mbar_wait_or_abort(bs2, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
        }
        p1 ^= 1u;
        if (wg_vote_or(1, !ok || abort_flag)) { bad = true; break; }
        tc::fence_after_sync();
        {  // stage-1 output -> stage-2 operand: element [jy][(i, jz, ix)]
          float v[K];
          load_groups(tD1, 1, v);
          if (mrow < rows) store_units(a2_addr, v);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        wg_sync(1);
        if (tid == 64) {  // ---- stage 2: rows (i, jz, ix), contraction jy
          bool ok2 = it == 0 || tc::mbar_wait_or_abort(bd2free, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
          if (ok2) {
            const int r = it % SRC_RING;
            ring_m[r] = m;
            ring_keep[r] = keep;
            ring_flags[r] = group_end ? FLAG_GROUP_END : 0;
            if (group_end)
              for (int e = 0; e < G * 3; ++e) ring_rec[r][e] = grp_rec[g * G * 3 + e];
            mbar_arrive(bring);
            ok2 = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / SRC_NB) & 1), WAIT_CYCLES,
                                         &abort_flag);
          }
          if (ok2) {
            tc::fence_after_sync();
            issue_stacked(tD2, A2, Bb + BY_OFF, 1, 0u);
            tc::mma_commit(bs2);
          } else {
            abort_flag = 1;
          }
        }
        ++it;
      }
      // a thread that left the loop early by the vote has bad set
    }
    // no more terms: tell warpgroup 1 (after it has read the last term's D2)
    if (!bad && tid == 64) {
      bool ok2 = it == 0 || tc::mbar_wait_or_abort(bd2free, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
      if (ok2) {
        ring_flags[it % SRC_RING] = FLAG_TERM;
        mbar_arrive(bring);
      } else {
        abort_flag = 1;
      }
    }
    if (bad) abort_flag = 1;
    // block copies still in flight (after an abort) land before the CTA exits, and every MMA an
    // issuing thread started is complete before the tensor memory is released
    if (tid == 32) {
      for (int b = 0; b < SRC_NB && b < nfetch; ++b) {
        const int uses = (nfetch - 1 - b) / SRC_NB + 1;  // copies into buffer b
        tc::mbar_wait(tc::smem_u32(&bar_bb[b]), (uint32_t)((uses - 1) & 1), WAIT_CYCLES);
      }
    }
    if (tid == 0 || tid == 64) {
      const uint32_t bd = tc::smem_u32(tid == 0 ? &bar_drain0 : &bar_drain2);
      tc::mma_commit(bd);
      tc::mbar_wait(bd, 0, WAIT_CYCLES);
    }
    if (tid == 0 && it > 0) atomicAdd(a.pass_ctr, (unsigned long long)it);
  } else if (wg == 1) {
    // ======================================================= warpgroup 1
    // where this thread's stage-2 output row (i, jz, ix) goes in the stage-3 operand:
    // element [jz][(i, ix, 0..k-1)]
    uint32_t a3_addr[U];
    {
      const int m2 = min(mrow, rows - 1);
      const int i = m2 / k2, rem = m2 - i * k2, jz = rem / K, ix = rem - jz * K;
      run_addrs(A3, i * k2 + ix * K, jz, a3_addr);
    }
    const int slot = mrow < rows ? mrow / k2 : -1;
    const int rem3 = mrow < rows ? mrow - slot * k2 : 0;  // (ix, iy) of this thread's stage-3 row
    // per (lz in window, iz): the record sum over terms as FP32 hi + running compensation lo
    float hi[3][K], lo[3][K];
#pragma unroll
    for (int w = 0; w < 3; ++w)
#pragma unroll
      for (int j = 0; j < K; ++j) hi[w][j] = lo[w][j] = 0.f;
    bool bad = false;
    // add D3 (the terms of one pass, kept as `kp`) into this thread's record sums
    auto flush = [&](uint32_t kp) {
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        uint32_t any = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) any |= (kp >> (3 * i + w)) & 1u;
        if (!any) continue;  // uniform over the CTA: the tensor-memory loads are warp-collective
        float v[K];
        load_groups(tD3 + (uint32_t)(16 * w), 3, v);
        if (slot >= 0 && ((kp >> (3 * slot + w)) & 1u)) {
          if constexpr (!PLAIN) {
#pragma unroll
            for (int j = 0; j < K; ++j) {  // lo holds minus the running compensation
              const float y = v[j] + lo[w][j];
              const float s = hi[w][j] + y;
              lo[w][j] = y - (s - hi[w][j]);
              hi[w][j] = s;
            }
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) hi[w][j] += v[j];
          }
        }
      }
    };
    // the record sums of a finished group to the partial buffer (FP32), then cleared
    auto write_group = [&](const int *rec) {
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        const int p = slot >= 0 ? rec[3 * slot + w] : -1;
        if (p >= 0) {
          float *o = a.partial + (int64_t)MRA_IDX(p, a.n_rec) * k3 + (int64_t)rem3 * K;
          if constexpr (K % 2 == 0) {
#pragma unroll
            for (int j = 0; j < K; j += 2) *(float2 *)(o + j) = make_float2(hi[w][j] + lo[w][j], hi[w][j + 1] + lo[w][j + 1]);
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) o[j] = hi[w][j] + lo[w][j];
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) hi[w][j] = lo[w][j] = 0.f;
      }
    };
    uint32_t prev_keep = 0;
    int prev_flags = 0, prev_slot = 0;
    int last_handed = -1;  // the last term handed to the stage-3 issuer (plain sums)
    int joined = 0;  // terms summed in D3 since its last flush
    int it = 0;
    for (;; ++it) {
      const int r = it % SRC_RING;
      bool ok = true;
      if (quarter == 0) ok = tc::mbar_wait_or_abort(bring, (uint32_t)(it & 1), WAIT_CYCLES, &abort_flag);
      if (wg_vote_or(2, !ok || abort_flag)) { bad = true; break; }
      const int flags = ring_flags[r];
      if (flags & FLAG_TERM) break;
      if (quarter == 0) {
        ok = tc::mbar_wait_or_abort(bs2, (uint32_t)(it & 1), WAIT_CYCLES, &abort_flag);
        if (ok && it > 0) ok = tc::mbar_wait_or_abort(bs3, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
      }
      if (wg_vote_or(2, !ok || abort_flag)) { bad = true; break; }
      tc::fence_after_sync();
      const uint32_t keep = ring_keep[r];
      // D2 -> registers, then D2 is released for the next term's stage 2
      float v[K];
      load_groups(tD2, 1, v);
      tc::fence_before_sync();
      wg_sync(2);
      if (tid == 128) mbar_arrive(bd2free);
      // the previous pass's D3 into the record sums and a finished group written out, unless this
      // term's stage 3 joins it in D3 (same group, same records keeping it, room left)
      const bool join_now = joined > 0 && joined < join && keep == prev_keep && !(prev_flags & FLAG_GROUP_END);
      if (it > 0 && !join_now) {
        flush(prev_keep);
        if (prev_flags & FLAG_GROUP_END) write_group(ring_rec[prev_slot]);
        joined = 0;
      }
      // stage-2 output -> stage-3 operand: element [jz][(i, ix, iy)]
      if (mrow < rows) store_units(a3_addr, v);
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      wg_sync(2);
      if constexpr (PLAIN) {  // the stage-3 issuer warp takes it from here (named barrier 3)
        if (tid == 128) s3_flags[it % SRC_RING] = join_now ? FLAG_JOIN : 0;
        __syncwarp();
        wg_arrive_issuer();
        last_handed = it;
      } else if (tid == 160) {  // a thread of another warp than the polling one issues stage 3
        const int b = it % SRC_NB;
        const unsigned char *B3 = Bt + b * BIT_BYTES + BZ_OFF;
        bool okb = tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / SRC_NB) & 1), WAIT_CYCLES,
                                          &abort_flag);
        if (okb) {
          tc::fence_after_sync();
          // ---- stage 3: rows (i, ix, iy), contraction jz, B = c_m R_{m,lz} of the window's three lz
          issue_stacked(tD3, A3, B3, 3, join_now ? 1u : 0u);
          tc::mma_commit(bs3);
          tc::mma_commit(tc::smem_u32(&bar_bfree[b]));
        } else {
          abort_flag = 1;
        }
      }
      prev_keep = keep;
      prev_flags = flags;
      prev_slot = r;
      ++joined;
    }
    if (!bad && it > 0) {
      bool ok = quarter != 0 || tc::mbar_wait_or_abort(bs3, (uint32_t)((it - 1) & 1), WAIT_CYCLES, &abort_flag);
      if (wg_vote_or(2, !ok || abort_flag)) {
        bad = true;
      } else {
        tc::fence_after_sync();
        flush(prev_keep);
        if (prev_flags & FLAG_GROUP_END) write_group(ring_rec[prev_slot]);
      }
    }
    if (bad) abort_flag = 1;
    if constexpr (PLAIN) {
      // no more terms for the stage-3 issuer (also after an abort), in the slot after the last
      // term handed over.  That term's stage 3 done means the issuer took it, so this arrival is
      // the only one pending on barrier 3; if it never completes within the bound, the issuer has
      // left on the abort and waits no more.
      bool send = true;
      if (last_handed >= 0) {
        bool ok = quarter != 0 || tc::mbar_wait(bs3, (uint32_t)(last_handed & 1), WAIT_CYCLES);
        send = !wg_vote_or(2, !ok);
      }
      if (send) {
        if (tid == 128) s3_flags[(last_handed + 1) % SRC_RING] = FLAG_TERM;
        __syncwarp();
        wg_arrive_issuer();
      }
    } else if (tid == 160) {
      tc::mma_commit(tc::smem_u32(&bar_drain1));
      tc::mbar_wait(tc::smem_u32(&bar_drain1), 0, WAIT_CYCLES);
    }
  } else if (PLAIN && warp == SRC_THREADS / 32) {
    // ======================================================= the stage-3 issuer (warp 8; lane 0 issues)
    // Warpgroup 1 hands each term over on named barrier 3 (its 128 threads arrive, this warp
    // waits: cheaper than an mbarrier round trip) and arrives once more when there are no more
    // terms, also after an abort, so the wait always ends.  The blocks of the next term are
    // checked as soon as their copies are known to be issued.
    int ready = -1;  // the term whose blocks lane 0 has already seen land
    for (int it = 0;; ++it) {
      asm volatile("bar.sync 3, 160;" ::: "memory");
      const int f = s3_flags[it % SRC_RING];
      if (f & FLAG_TERM) break;
      const int b = it % SRC_NB;
      const unsigned char *B3 = Bt + b * BIT_BYTES + BZ_OFF;
      if (lane == 0) {
        bool ok = ready == it ||
                  tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[b]), (uint32_t)((it / SRC_NB) & 1), WAIT_CYCLES, &abort_flag);
        if (ok) {
          tc::fence_after_sync();
          // ---- stage 3: rows (i, ix, iy), contraction jz, B = c_m R_{m,lz} of the window's three lz
          issue_stacked(tD3, A3, B3, 3, (f & FLAG_JOIN) ? 1u : 0u);
          tc::mma_commit(bs3);
          tc::mma_commit(tc::smem_u32(&bar_bfree[b]));
          const int nx = it + 1;  // the next term's blocks, if their copies are issued
          if (nx < s_nfetch &&
              tc::mbar_wait_or_abort(tc::smem_u32(&bar_bb[nx % SRC_NB]), (uint32_t)((nx / SRC_NB) & 1), WAIT_CYCLES,
                                     &abort_flag))
            ready = nx;
        } else {
          abort_flag = 1;
        }
      }
      // one decision for the whole warp (lane 0's view), so that no lane waits alone at bar.sync
      if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) break;
    }
    if (lane == 0) {
      tc::mma_commit(tc::smem_u32(&bar_drain1));
      tc::mbar_wait(tc::smem_u32(&bar_drain1), 0, WAIT_CYCLES);
    }
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (abort_flag && tid == 0) atomicExch(a.err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, SRC_TMEM_COLS);
}

// ---------------------------------------------------------------- work list: tiles of sources
// Sort key of a source: sources without records last; then (several sources per tile) by level,
// and heaviest (most kept terms) first.
__global__ void src_key_kernel(int64_t n, int G, const uint64_t *keys, const int64_t *cnt, const int64_t *kept,
                               uint64_t *skey, int *sval) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  uint64_t key;
  if (cnt[b] <= 0) {
    key = ~0ull;
  } else {
    const uint64_t w = (uint64_t)min(kept[b], (int64_t)0xFFFFFFFF);
    const uint64_t lev = G > 1 ? (uint64_t)key_level(keys[b]) : 0ull;
    key = (lev << 32) | (0xFFFFFFFFull - w);
  }
  skey[b] = key;
  sval[b] = (int)b;
}

// One thread: per level the first sorted position and the tile numbering; the tile count.
__global__ void src_tiles_kernel(int64_t n, int G, const uint64_t *skey, int *lev_first, int *tile_base,
                                 int *n_tiles) {
  if (threadIdx.x != 0) return;
  auto lower = [&](uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (skey[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (int)lo;
  };
  const int n_active = lower(~0ull);
  int tiles = 0;
  if (G == 1) {
    lev_first[0] = 0;
    tile_base[0] = 0;
    tiles = n_active;
  } else {
    for (int l = 0; l <= MRA_MAX_LEVEL; ++l) {
      const int f = lower((uint64_t)l << 32), e = min(lower((uint64_t)(l + 1) << 32), n_active);
      lev_first[l] = f;
      tile_base[l] = tiles;
      tiles += (e - f + G - 1) / G;
    }
  }
  *n_tiles = tiles;
}

__global__ void src_scatter_kernel(int64_t n, int G, const uint64_t *skey, const int *sval, const int *lev_first,
                                   const int *tile_base, int *tile_src) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || skey[i] == ~0ull) return;
  const int l = G > 1 ? (int)(skey[i] >> 32) : 0;
  const int j = (int)i - lev_first[l];
  tile_src[(int64_t)(tile_base[l] + j / G) * G + j % G] = sval[i];
}

// s + c += x: s is the running FP32 sum and c the FP32 sum of its rounding errors, each taken
// exactly by Knuth's TwoSum (the cascaded summation Sum2 of Ogita, Rump and Oishi), so that
// s + c carries about twice FP32's precision.
__device__ __forceinline__ void sum2_add(float &s, float &c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

// Sum the partials of every destination, records in destination order; one CTA per destination,
// every coefficient written once.  The FP32 partials are added in FP32 pairs (sum2_add: error
// about 2^-48 of the sum's magnitude, far below the partials' own 2^-24 rounding) and the pair is
// formed into FP64 once per coefficient; an FP64 addition per partial would cost a conversion
// and an add on the FP64 pipe for every one of them.  k^3 is a multiple of 4 for the orders this
// path covers: each thread takes four consecutive coefficients (16-byte streaming loads, read
// once) and four records at a time.
__global__ void dest_sum_kernel(int64_t nd, int k3, const int64_t *seg, const int *perm, const float *partial,
                                const uint64_t *dest_key, uint64_t *out_keys, double *out_coeffs, int64_t n_rec) {
  const int64_t d = blockIdx.x;
  if (d >= nd) return;
  const int64_t r0 = seg[d], r1 = seg[d + 1];
  const int q4 = k3 / 4;
  for (int e = threadIdx.x; e < q4; e += blockDim.x) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    auto add = [&](const float4 v) {
      sum2_add(s0, c0, v.x);
      sum2_add(s1, c1, v.y);
      sum2_add(s2, c2, v.z);
      sum2_add(s3, c3, v.w);
    };
    auto rec = [&](int64_t r) {
      const int64_t p = MRA_IDX((int64_t)perm[MRA_IDX(r, n_rec)], n_rec);
      return (const float4 *)(partial + p * k3) + e;
    };
    int64_t r = r0;
    for (; r + 4 <= r1; r += 4) {
      const float4 v0 = __ldcs(rec(r)), v1 = __ldcs(rec(r + 1)), v2 = __ldcs(rec(r + 2)), v3 = __ldcs(rec(r + 3));
      add(v0);
      add(v1);
      add(v2);
      add(v3);
    }
    for (; r < r1; ++r) add(__ldcs(rec(r)));
    const double a0 = (double)s0 + (double)c0, a1 = (double)s1 + (double)c1;
    const double a2 = (double)s2 + (double)c2, a3 = (double)s3 + (double)c3;
    double *o = out_coeffs + d * k3 + 4 * e;
    if (((uintptr_t)out_coeffs & 15) == 0) {  // the caller's buffer: 16-byte stores where aligned
      ((double2 *)o)[0] = make_double2(a0, a1);
      ((double2 *)o)[1] = make_double2(a2, a3);
    } else {
      o[0] = a0;
      o[1] = a1;
      o[2] = a2;
      o[3] = a3;
    }
  }
  if (threadIdx.x == 0) out_keys[d] = dest_key[d];
}

}  // namespace

// The source-stationary kernel covers even k from 4 to 10 (one 128-row tile per CTA, G k^2 <= 128
// with G <= 8 sources) and records with |l|_inf <= 2.
bool src_path_supported(int k, int max_rec_disp) {
  return (k == 4 || k == 6 || k == 8 || k == 10) && max_rec_disp <= SRC_MAX_DAP;
}

size_t src_workspace_bytes(int64_t n_in) {
  const int64_t nb = n_in > 0 ? n_in : 1;
  size_t t = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, t, (uint64_t *)nullptr, (uint64_t *)nullptr, (int *)nullptr,
                                  (int *)nullptr, (int)nb);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return 2 * al(nb * 8) + 2 * al(nb * 4) + al((nb + 2 * SRC_MAX_G + 64) * SRC_MAX_G * 4) +
         al(4 * (MRA_MAX_LEVEL + 2) * 4) + al(t) + 256;
}

int apply_src_run(const Operator &op, const mra_tree_view &in, const mra_apply_opts &o, mra_tree_view &out,
                  const ApplyWork &wk, const int *dap, float *partial, cudaStream_t s, int64_t *passes) {
  const int k = op.k, k3 = k * k * k;
  const int G = src_g(k);
  const int64_t P = wk.P, nd = wk.n_dest, n_in = in.n;
  const int64_t nb = n_in > 0 ? n_in : 1;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char *w = (char *)wk.split_ws;
  uint64_t *skey = (uint64_t *)w; w += al(nb * 8);
  uint64_t *skey2 = (uint64_t *)w; w += al(nb * 8);
  int *sval = (int *)w; w += al(nb * 4);
  int *sval2 = (int *)w; w += al(nb * 4);
  int *tile_src = (int *)w; w += al((nb + 2 * SRC_MAX_G + 64) * SRC_MAX_G * 4);
  int *small = (int *)w; w += al(4 * (MRA_MAX_LEVEL + 2) * 4);
  int *lev_first = small, *tile_base = small + (MRA_MAX_LEVEL + 2), *n_tiles = small + 2 * (MRA_MAX_LEVEL + 2);
  int *tile_ctr = n_tiles + 1, *err = n_tiles + 2;
  // the pass counter: bytes 256..263 of the zeroed scratch (its 45 ints end at byte 180; the
  // scratch is 256-byte aligned and 336 bytes long), so 8-byte aligned for the 64-bit atomic
  static_assert(3 * (MRA_MAX_LEVEL + 2) * 4 <= 256 && 256 + 8 <= 4 * (MRA_MAX_LEVEL + 2) * 4,
                "pass counter inside the scratch, after its ints");
  unsigned long long *pass_ctr = (unsigned long long *)((char *)small + 256);
  if (((uintptr_t)small & 255) != 0) return fail(MRA_ERR_ARG, "split apply: workspace not 256-byte aligned");
  void *tmp = w;
  size_t tmpb = wk.split_ws_bytes - (size_t)(w - (char *)wk.split_ws);
  const size_t tile_bytes = (size_t)(nb + 2 * SRC_MAX_G + 64) * SRC_MAX_G * 4;

  if (wk.ev0) MRA_CUDA_TRY(cudaEventRecord(wk.ev0, s));
  MRA_CUDA_TRY(cudaMemsetAsync(small, 0, 4 * (MRA_MAX_LEVEL + 2) * 4, s));
  MRA_CUDA_TRY(cudaMemsetAsync(tile_src, 0xFF, tile_bytes, s));
  const unsigned gb = (unsigned)((nb + 255) / 256);
  src_key_kernel<<<counted(gb), 256, 0, s>>>(n_in, G, in.keys, wk.rec_cnt, wk.box_kept, skey, sval);
  MRA_CUDA_TRY(cudaGetLastError());
  MRA_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmpb, skey, skey2, sval, sval2, (int)n_in, 0, 64, s));
  src_tiles_kernel<<<counted(1), 32, 0, s>>>(n_in, G, skey2, lev_first, tile_base, n_tiles);
  MRA_CUDA_TRY(cudaGetLastError());
  src_scatter_kernel<<<counted(gb), 256, 0, s>>>(n_in, G, skey2, sval2, lev_first, tile_base, tile_src);
  MRA_CUDA_TRY(cudaGetLastError());

  SrcArgs a{};
  a.k = k;
  a.M = op.M;
  a.P = o.pieces;
  if (a.P < 2 || a.P > 3) return fail(MRA_ERR_ARG, "split apply: pieces must be 2 or 3");
  a.Bsplit = (const unsigned char *)op.d_Rsplit;
  a.Bzpack = a.Bsplit + (size_t)2 * op.n_blocks * BSTAGE_BYTES;
  a.Dlev = op.d_D;
  for (int n = 0; n <= MRA_MAX_LEVEL; ++n) a.Dap[n] = dap[n];
  a.level_off = op.d_level_off;
  a.in_keys = in.keys;
  a.in_coeffs = in.coeffs;
  a.rec_cnt = wk.rec_cnt;
  a.rec_off = wk.rec_off;
  a.rec_l = wk.rec_l;
  a.rec_mask = wk.rec_mask;
  a.tile_src = tile_src;
  a.n_tiles = n_tiles;
  a.tile_ctr = tile_ctr;
  a.partial = partial;
  a.err = err;
  a.pass_ctr = pass_ctr;
  a.inject_stall = take_injected_stall() ? 1 : 0;
  a.join = o.join > 0 ? o.join : 2;
  a.join_all = o.join > 0 ? 1 : 0;
  a.compensated = o.sums == MRA_SUMS_COMPENSATED ? 1 : 0;
  a.ahead = o.ahead > 0 ? o.ahead : 2;
  a.n_src = n_in;
  a.n_rec = P;
  a.n_blocks = op.n_blocks;
  const size_t tables = (size_t)SRC_NG * G * 3 * 4 + 8 + (size_t)SRC_NG * G * 3 * 16 + (size_t)SRC_NG * 16;
  size_t smem = (size_t)9 * TILE_BYTES + (size_t)SRC_NB * BIT_BYTES + tables;
  // no more CTAs per SM than the tensor memory holds (two of 256 columns): otherwise an extra
  // CTA's allocation would wait for a resident CTA to finish
  const size_t smem_floor = (size_t)233472 / (512 / SRC_TMEM_COLS + 1) + 16;
  if (smem < smem_floor) smem = smem_floor;
  void (*kern)(SrcArgs) = nullptr;
  const bool plain = !a.compensated;
  switch (k * 2 + (plain ? 1 : 0)) {
    case 8: kern = apply_src_kernel<4, false>; break;
    case 9: kern = apply_src_kernel<4, true>; break;
    case 12: kern = apply_src_kernel<6, false>; break;
    case 13: kern = apply_src_kernel<6, true>; break;
    case 16: kern = apply_src_kernel<8, false>; break;
    case 17: kern = apply_src_kernel<8, true>; break;
    case 21: kern = apply_src_kernel<10, true>; break;
    default: kern = apply_src_kernel<10, false>; break;
  }
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int dev = 0, sms = 0;
  MRA_CUDA_TRY(cudaGetDevice(&dev));
  MRA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // persistent: two CTAs per SM (the tensor memory holds two of 256 columns), never more CTAs
  // than sources
  const int64_t max_tiles = G == 1 ? n_in : n_in / G + MRA_MAX_LEVEL + 1;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)sms, max_tiles));
  if (((uintptr_t)partial & 15) != 0 || k3 % 4 != 0)
    return fail(MRA_ERR_ARG, "split apply: partial-sum buffer not 16-byte aligned or k^3 = %d not a multiple of 4", k3);
  if (wk.evk0) MRA_CUDA_TRY(cudaEventRecord(wk.evk0, s));
  kern<<<counted(grid), plain ? SRC_THREADS + 32 : SRC_THREADS, smem, s>>>(a);
  MRA_CUDA_TRY(cudaGetLastError());
  if (wk.evk1) MRA_CUDA_TRY(cudaEventRecord(wk.evk1, s));
  dest_sum_kernel<<<counted((unsigned)std::max<int64_t>(nd, 1)), 256, 0, s>>>(
      nd, k3, wk.seg, wk.perm, partial, wk.dest_key, out.keys, out.coeffs, P);
  MRA_CUDA_TRY(cudaGetLastError());
  if (wk.ev1) MRA_CUDA_TRY(cudaEventRecord(wk.ev1, s));
  if (wk.fx) {
    split_fixed_err(err, wk.fx->status, s);
    return MRA_OK;
  }
  int herr = 0;
  unsigned long long hpass = 0;
  MRA_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaMemcpyAsync(&hpass, pass_ctr, sizeof(hpass), cudaMemcpyDeviceToHost, s));
  MRA_CUDA_TRY(cudaStreamSynchronize(s));
  if (passes) *passes = (int64_t)hpass;
  if (herr == 1) return fail(MRA_ERR_TIMEOUT, "split apply: a tensor-core completion wait gave up");
  if (herr) return fail(MRA_ERR_ARG, "split apply: inconsistent work list (%d)", herr);
  return MRA_OK;
}

}  // namespace mra

namespace mra {
int debug_line_src(cudaStream_t s) { return debug_take_line(s); }
}  // namespace mra
