// Persistent grouped level launch for the exact splits (64-column tiles,
// orders up to 4096): one CTA per SM walks the level's whole tile list
// (tiles b, b + G, b + 2G, ... of every product in the device table), so the
// per-CTA set-up (barriers, TMEM allocation, descriptor prefetch) is paid once
// per SM instead of once per tile, and the epilogue of one tile (fold, block
// maxima, re-split, stores) overlaps the loads and MMAs of the next:
//
//   warp 0  TMA producer over the ring (runs ahead across tile boundaries)
//   warp 1  tcgen05.mma issuer; NBUF k-block accumulator sets in TMEM
//   warp 2  TMEM owner
//   warp 3  stages the block exponents and record of the next four tiles
//           (one per group of 8 lanes), so the epilogue never waits on a
//           global load to start a tile
//
// The host gives one 16-byte record per tile (product, depth, origin, the
// two tensor-map indices), so the producer and MMA warps read one record
// per tile and prefetch the next.
//   warps 4-11  two groups of four: group g folds the finished k-blocks of
//           the CTA's tiles g, g + 2, g + 4, ... into float32 registers,
//           then writes the next operand's slices with plain global stores
//           (no staging in the ring, which the next tile is already
//           filling); warp w takes TMEM lane quadrant w % 4 and all 64
//           columns.  While one group re-splits and stores a tile, the other
//           folds the next tile's k-blocks, so the MMA warp does not wait
//           through the store phase (with one group of eight warps sharing
//           every tile, it waited for an accumulator set 40 % of its time
//           with three slices: only two sets of 3 x 64 columns fit TMEM, and
//           a tile of N <= 256 has at most four k-blocks)
//
// The arithmetic per tile is that of tc_fxb_group_kernel: the same k-block
// order, the same fold, the same slicing, so the results are bit-for-bit the
// same.  Every wait is bounded; an abort drains copies and MMAs, frees TMEM
// and reports MATPOW_ETIMEDOUT through the status word.
#include <cuda.h>
#include <cuda_bf16.h>

#include "fxb.cuh"
#include "internal.cuh"
#include "plan.h"
#include "tc_ptx.cuh"

#include <vector>

namespace mp {
namespace persist {

constexpr int BM = 128, BN = 64, BK = 64, THREADS = 384;
constexpr int EW = 8;      // epilogue warps (4..11)
constexpr int GW = 4;      // epilogue warps per group (one per TMEM lane quadrant)
constexpr int WC = BN;     // columns per epilogue thread
constexpr int KB_MAX = 64;  // N <= 4096
constexpr int EXPB = 4;     // tiles staged ahead by warp 3 (one per group of 8 lanes)
constexpr uint64_t WAIT_NS = 2000000000ull;


// Per-tile record staged by warp 3 for the epilogue: product index, k-blocks,
// origin, operand scale exponents, output exponent.
struct TileInfo {
  int di, KB, m0, n0, sx, sy;
  long long Ec;
};

template <int NSL>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = NSL * (A_BYTES + B_BYTES);
  static constexpr int RING = NSL == 3 ? 216 * 1024 : 192 * 1024;
  static constexpr int STAGES = RING / STAGE_BYTES;
  // accumulator sets (NSL x 64 columns each) that fit 512 TMEM columns
  static constexpr int NBUF = NSL == 3 ? 2 : 4;
  static constexpr int TMEM_COLS = 512;
  // barriers: full[S], empty[S], accfull[NBUF], accempty[NBUF], expfull[EXPB],
  // expempty[EXPB], drain, folded[2]; then tmem slot, abort flag, the two
  // epilogue groups' verdicts
  static constexpr int NBARS = 2 * STAGES + 2 * NBUF + 2 * EXPB + 1 + 2;
  static constexpr int BAR_BYTES = 256;
  static constexpr int EXP_INTS = 3 * KB_MAX;  // eA (2 block rows) + eB (1 block column)
  static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + BAR_BYTES + EXPB * EXP_INTS * 4 + 64 +
                              EXPB * (int)sizeof(TileInfo);
  static_assert(NBARS * 8 + 16 <= BAR_BYTES, "barrier area");
  static_assert(STAGES >= 2, "ring");
  static_assert(NBUF * NSL * BN <= TMEM_COLS, "TMEM");
};

}  // namespace persist

// Named barrier 1 + grp over the 4 warps of epilogue group grp.
__device__ __forceinline__ void grp_bar(int grp) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + grp) : "memory");
}

template <int NSL>
__global__ void __launch_bounds__(persist::THREADS, 1)
    tc_fxb_persist_kernel(const GemmDesc* __restrict__ descs, int tiles_total,
                          const int4* __restrict__ recs, const CUtensorMap* __restrict__ maps,
                          Scale* scales, unsigned* status) {
  using namespace persist;
  using C = Cfg<NSL>;
  constexpr int STAGES = C::STAGES, NBUF = C::NBUF;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + C::NBARS);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* epi_ok = (volatile int*)(tmem_slot + 2);  // [2]: one verdict per epilogue group
  int* expbuf = (int*)((uint8_t*)bars + C::BAR_BYTES);  // [EXPB][EXP_INTS]
  float* red = (float*)(expbuf + EXPB * C::EXP_INTS);   // [2 groups][4 quadrants] (16 slots)
  TileInfo* info = (TileInfo*)(red + 16);                // [EXPB]
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 2 * STAGES + NBUF);
  const uint32_t expfull0 = ptx::smem_u32(bars + 2 * STAGES + 2 * NBUF);
  const uint32_t expempty0 = ptx::smem_u32(bars + 2 * STAGES + 2 * NBUF + EXPB);
  const uint32_t drainb = ptx::smem_u32(bars + 2 * STAGES + 2 * NBUF + 2 * EXPB);
  // folded[g]: epilogue group g has folded every k-block of one of its tiles
  const uint32_t folded0 = ptx::smem_u32(bars + 2 * STAGES + 2 * NBUF + 2 * EXPB + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, GW);  // one arrival per warp of the folding group
    }
    for (int b = 0; b < EXPB; ++b) {
      ptx::mbar_init(expfull0 + 8 * b, 8);     // the 8 lanes of one group of warp 3
      ptx::mbar_init(expempty0 + 8 * b, 32 * GW);  // every thread of the tile's epilogue group
    }
    ptx::mbar_init(drainb, 1);
    for (int g = 0; g < 2; ++g) ptx::mbar_init(folded0 + 8 * g, GW);  // one arrival per warp of group g
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // recs[t] = {product | k-blocks << 24, m0 | n0 << 16, A map, B map}
  int gk = 0;  // k-blocks handled by this role so far (ring / accumulator phases)
  if (warp == 0) {
    if (lane == 0) {
      int4 r = blockIdx.x < tiles_total ? recs[blockIdx.x] : make_int4(0, 0, 0, 0);
      if (blockIdx.x < tiles_total) {
#pragma unroll
        for (int k = 0; k < NSL; ++k) {
          ptx::prefetch_tmap(maps + r.z + k);
          ptx::prefetch_tmap(maps + r.w + k);
        }
      }
      for (int tb = blockIdx.x; tb < tiles_total && !*abort_flag; tb += G) {
        // the next tile's record, loaded while this tile's copies are issued
        const int4 rn = tb + G < tiles_total ? recs[tb + G] : make_int4(0, 0, 0, 0);
        const int KB = r.x >> 24;
        const int m0 = r.y & 0xFFFF, n0 = r.y >> 16;
        const CUtensorMap* ax = maps + r.z;
        const CUtensorMap* by = maps + r.w;
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb, ++gk) {
          const int s = gk % STAGES;
          if (!ptx::mbar_wait(empty0 + 8 * s, ((gk / STAGES) & 1) ^ 1, abort_flag, WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const uint32_t fb = full0 + 8 * s;
          ptx::mbar_expect_tx(fb, C::STAGE_BYTES);
          const uint32_t base = ptx::smem_u32(smem + s * C::STAGE_BYTES);
          const int kx = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB)) * BK;
#pragma unroll
          for (int k = 0; k < NSL; ++k) ptx::tma_load_2d(base + k * C::A_BYTES, ax + k, kx, m0, fb);
          const uint32_t bbase = base + NSL * C::A_BYTES;
#pragma unroll
          for (int k = 0; k < NSL; ++k) ptx::tma_load_2d(bbase + k * C::B_BYTES, by + k, n0, kx, fb);
        }
        if (!ok) break;
        if (rn.z != r.z || rn.w != r.w) {
#pragma unroll
          for (int k = 0; k < NSL; ++k) {
            ptx::prefetch_tmap(maps + rn.z + k);
            ptx::prefetch_tmap(maps + rn.w + k);
          }
        }
        r = rn;
      }
      // no copy may still be in flight when the CTA ends
      for (int g = gk - STAGES < 0 ? 0 : gk - STAGES; g < gk; ++g) {
        int dummy = 0;
        ptx::mbar_wait(full0 + 8 * (g % STAGES), (g / STAGES) & 1, &dummy, WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int KB = blockIdx.x < tiles_total ? recs[blockIdx.x].x >> 24 : 0;
      for (int tb = blockIdx.x; tb < tiles_total && !*abort_flag; tb += G) {
        // the next tile's depth, loaded while this tile's MMAs are issued
        const int KBn = tb + G < tiles_total ? recs[tb + G].x >> 24 : 0;
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb, ++gk) {
          const int buf = gk % NBUF;
          const uint32_t t0 = tmem + (uint32_t)(buf * NSL * BN);
          if (!ptx::mbar_wait(accempty0 + 8 * buf, ((gk / NBUF) & 1) ^ 1, abort_flag, WAIT_NS)) {
            ok = false;
            break;
          }
          const int s = gk % STAGES;
          if (!ptx::mbar_wait(full0 + 8 * s, (gk / STAGES) & 1, abort_flag, WAIT_NS)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t a0 = ptx::smem_u32(smem + s * C::STAGE_BYTES);
          const uint32_t b0 = a0 + NSL * C::A_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            uint64_t ad[NSL], bd[NSL];
#pragma unroll
            for (int i = 0; i < NSL; ++i) {
              ad[i] = ptx::smem_desc(a0 + i * C::A_BYTES + 32 * k, 16, 1024);
              bd[i] = ptx::smem_desc(b0 + i * C::B_BYTES + 2048 * k, 8192, 1024);
            }
            const uint32_t acc = k == 0 ? 0u : 1u;
            fxb::slice_mmas<BN, NSL>(t0, ad, bd[0], acc);
          }
          ptx::mma_commit(empty0 + 8 * s);
          ptx::mma_commit(accfull0 + 8 * buf);
        }
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        KB = KBn;
      }
      ptx::mma_commit(drainb);
      int dummy = 0;
      ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
    }
  } else if (warp == 3) {
    // four groups of 8 lanes; group g stages the CTA's tiles g, g + 4, ...
    // (block exponents and the tile's record) into buffer (tile index) % 4,
    // so the dependent global loads of four tiles are in flight at once
    const int grp = lane >> 3, gl = lane & 7;
    for (int lt = grp;; lt += EXPB) {
      const int tb = blockIdx.x + lt * G;
      if (tb >= tiles_total || *abort_flag) break;
      const int4 r = recs[tb];
      const int di = r.x & 0xFFFFFF, KB = r.x >> 24;
      const int m0 = r.y & 0xFFFF, n0 = r.y >> 16;
      const GemmDesc& d = descs[di];
      const int e = lt & (EXPB - 1);
      if (!ptx::mbar_wait(expempty0 + 8 * e, ((lt / EXPB) & 1) ^ 1, abort_flag, WAIT_NS)) {
        *abort_flag = 1;
        break;
      }
      const int N = d.N;
      const int nb = fxb::nblocks(N);
      const size_t boff = fxb::bexp_offset(N, d.ld, NSL);
      const int* bx = (const int*)((const char*)d.X + boff);
      const int* byx = (const int*)((const char*)d.Y + boff);
      int* eA = expbuf + e * C::EXP_INTS;
      int* eB = eA + 2 * KB_MAX;
      const int I0 = m0 / fxb::BLK, J0 = n0 / fxb::BLK;
      for (int i = gl; i < 2 * KB; i += 8) {
        const int hh = i / KB, kb = i - hh * KB;
        eA[i] = (I0 + hh < nb) ? __ldcg(bx + (I0 + hh) * nb + kb) : 0;
      }
      for (int kb = gl; kb < KB; kb += 8) eB[kb] = (J0 < nb) ? __ldcg(byx + kb * nb + J0) : 0;
      if (gl == 0) {
        TileInfo ti;
        ti.di = di;
        ti.KB = KB;
        ti.m0 = m0;
        ti.n0 = n0;
        ti.sx = scale_exp_from_bits(scales[d.sx].maxbits);
        ti.sy = scale_exp_from_bits(scales[d.sy].maxbits);
        ti.Ec = scales[d.sx].E + scales[d.sy].E + ti.sx + ti.sy;
        info[e] = ti;
      }
      ptx::mbar_arrive(expfull0 + 8 * e);  // release: this lane's writes are visible
    }
  } else if (warp >= 4) {
    const int grp = (warp - 4) / GW;  // this group takes the CTA's tiles grp, grp + 2, ...
    const int q = warp & 3;           // TMEM lane quadrant: rows 32 q .. 32 q + 31
    const int h = q >> 1;             // the tile's 64-row block row
    const bool lead = q == 0 && lane == 0;
    float T[WC];
    // the other group's tiles (lt of the other parity): their k-blocks pass
    // by.  Each one's depth is read a tile ahead, so that the global load
    // overlaps this group's fold instead of delaying its next tile.
    if (grp == 1 && (int)blockIdx.x < tiles_total) gk += recs[blockIdx.x].x >> 24;
    for (int lt = grp;; lt += 2) {
      const int tb = blockIdx.x + lt * G;
      if (tb >= tiles_total) break;
      const int kb_skip = tb + G < tiles_total ? recs[tb + G].x >> 24 : 0;
      const int e = lt & (EXPB - 1);
      bool ok = true;
      int dummy = 0;
      // the other group has folded the tile before this one: every
      // accumulator phase up to it has been consumed, so the accfull waits
      // below are at most one phase ahead (a parity wait cannot tell phases
      // further apart).  Its store phase still overlaps this tile's fold.
      if (lt > 0 && !ptx::mbar_wait(folded0 + 8 * (grp ^ 1), ((lt - 1) >> 1) & 1, &dummy, 2 * WAIT_NS))
        ok = false;
      if (ok && !ptx::mbar_wait(expfull0 + 8 * e, (lt / EXPB) & 1, &dummy, 2 * WAIT_NS)) ok = false;
      const TileInfo ti = info[e];
      const int KB = ok ? ti.KB : 0;
      // the store phase's fields, loaded now and used after the fold (a
      // record that never arrived is not dereferenced)
      const GemmDesc& d = descs[ok ? ti.di : 0];
      const int N = d.N, ld = d.ld, mode = d.mode, sc = d.sc;
      const long long plane = d.plane;
      void* Cp = d.C;
      void* outp = d.out;
      long long* out_log2 = d.out_log2;
      const int row = ti.m0 + 32 * q + lane;
      const int c0 = ti.n0;
      const int* eA = expbuf + e * C::EXP_INTS;
      const int* eB = eA + 2 * KB_MAX;
#pragma unroll
      for (int j = 0; j < WC; ++j) T[j] = 0.f;
      for (int kb = 0; kb < KB; ++kb, ++gk) {
        const int buf = gk % NBUF;
        if (!ptx::mbar_wait(accfull0 + 8 * buf, (gk / NBUF) & 1, &dummy, 2 * WAIT_NS)) {
          ok = false;
          gk += KB - kb;  // keep the set phases of the k-blocks that follow
          break;
        }
        ptx::tc_fence_after();
        const int kr = fxb::rot_kb(kb, KB, fxb::tile_rot(ti.m0, ti.n0, KB));
        const float f = fxb::pow2f(eA[h * KB + kr] + eB[kr] - 16 - ti.sx - ti.sy);
        // the fold of fxb::fold on this thread's 64 columns, 32 at a time:
        // accumulator w at column offset w * BN of the k-block's set; the set
        // is released once its last columns are in registers
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * NSL * BN);
#pragma unroll
        for (int c = 0; c < WC / 32; ++c) {
          uint32_t rm[32], rc[32];
          if (NSL == 3) {
            uint32_t rd[32];
            ptx::tmem_ld_32x32b_x32(tq + 32 * c + BN, rc);
            ptx::tmem_ld_32x32b_x32(tq + 32 * c + 2 * BN, rd);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j)
              rc[j] = __float_as_uint(fmaf(__uint_as_float(rd[j]), 0.00390625f, __uint_as_float(rc[j])));
            ptx::tmem_ld_32x32b_x32(tq + 32 * c, rm);
            ptx::tmem_ld_wait();
          } else {
            ptx::tmem_ld_32x32b_x32(tq + 32 * c, rm);
            ptx::tmem_ld_32x32b_x32(tq + 32 * c + BN, rc);
            ptx::tmem_ld_wait();
          }
          if (c == WC / 32 - 1) {
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(accempty0 + 8 * buf);  // the set is in registers
          }
#pragma unroll
          for (int j = 0; j < 32; ++j)
            T[32 * c + j] =
                fmaf(fmaf(__uint_as_float(rc[j]), 0.00390625f, __uint_as_float(rm[j])), f, T[32 * c + j]);
        }
      }
      ptx::mbar_arrive(expempty0 + 8 * e);  // this tile's exponents and record are no longer read
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(folded0 + 8 * grp);  // the next tile's group may fold
      // one verdict for the group's warps (they share named barrier 1 + grp)
      grp_bar(grp);
      if (lead) epi_ok[grp] = ok && !*abort_flag;
      grp_bar(grp);
      if (!epi_ok[grp]) {
        *abort_flag = 1;
        break;
      }
      const bool first = ti.m0 == 0 && ti.n0 == 0;  // tile 0 of its product
      if (mode == OUT_INTERNAL) {
        if (first && lead) scales[sc].E = ti.Ec;
        // block maximum of the 64 x 64 block (rows of quadrants 2h, 2h + 1),
        // its exponent, then this thread's slices
        float m = 0.f;
#pragma unroll
        for (int j = 0; j < WC; ++j) m = fmaxf(m, fabsf(T[j]));
        m = warp_max(m);
        if (lane == 0) red[4 * grp + q] = m;
        grp_bar(grp);
        const float bm = fmaxf(red[4 * grp + 2 * h], red[4 * grp + 2 * h + 1]);
        const int ex = fxb::frexp_exp(bm);
        const int nb = fxb::nblocks(N);
        const int I = ti.m0 / fxb::BLK + h, J = ti.n0 / fxb::BLK;
        if ((q & 1) == 0 && lane == 0 && I < nb && J < nb) {
          ((int*)((char*)Cp + fxb::bexp_offset(N, ld, NSL)))[I * nb + J] = ex;
          if (bm > 0.f) atomicMax(&scales[sc].maxbits, __float_as_uint(bm));
        }
        // the stores: a lane holding a row would put each 16-byte store of a
        // warp on its own cache line (32 lines per instruction, which the
        // L1 data path shares with the next tile's copies and MMA operand
        // reads); transposed within 8-lane groups, lane 8 g + i holds
        // columns c0 + 8 i .. + 7 of rows 32 q + 8 g + j (j = 0..7), and a
        // warp store covers 4 rows x 128 contiguous bytes.  A group that
        // starts below N ends within the row's padding to ld (a multiple of
        // 8), which no product reads, and its columns past N hold exact zeros
        fxb::transpose8x8(T, lane);
        const int col = c0 + 8 * (lane & 7);
        const int r0 = ti.m0 + 32 * q + 8 * (lane >> 3);
        // two row chunks per pass, T[0..15], then the rest moves down: a short
        // loop body instead of eight unrolled copies (instruction fetch is
        // this kernel's largest stall)
#pragma unroll 1
        for (int j = 0; j < 8; j += 2) {
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            if (r0 + j + jj < N && col < N) {
              uint32_t w[NSL][4];
#pragma unroll
              for (int hh = 0; hh < 4; ++hh) {
                float x0[NSL], x1[NSL];
                fxb::slice_n<NSL>(T[8 * jj + 2 * hh], ex, x0);
                fxb::slice_n<NSL>(T[8 * jj + 2 * hh + 1], ex, x1);
#pragma unroll
                for (int k = 0; k < NSL; ++k) w[k][hh] = fxb::pack_bf16_exact(x0[k], x1[k]);
              }
              __nv_bfloat16* p1 = (__nv_bfloat16*)Cp + (size_t)(r0 + j + jj) * ld + col;
#pragma unroll
              for (int k = 0; k < NSL; ++k)
                *reinterpret_cast<uint4*>(p1 + k * plane) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
            }
          }
#pragma unroll
          for (int i = 0; i < WC - 16; ++i) T[i] = T[i + 16];
        }
        grp_bar(grp);  // red may be reused
      } else {
        if (first && lead && mode == OUT_USER_MANT && out_log2) *out_log2 = ti.Ec;
        if (row < N)
          store_row_f32<WC>(T, (float*)outp + (size_t)row * N, c0, N, mode == OUT_USER_MANT, ti.Ec, status, outp);
      }
      gk += kb_skip;
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cfg<NSL>::TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
}

// ---------------------------------------------------------------------------
// host side

cudaError_t tc_persist_init() {
  cudaError_t e = cudaFuncSetAttribute(tc_fxb_persist_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       persist::Cfg<2>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_fxb_persist_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             persist::Cfg<3>::SMEM);
  return e;
}

void persist_tile_records(const GemmDesc* descs, int count, int nsl, std::vector<int4>* out) {
  for (int k = 0; k < count; ++k) {
    const GemmDesc& d = descs[k];
    const int tiles_m = (d.N + persist::BM - 1) / persist::BM;
    const int KB = (d.N + persist::BK - 1) / persist::BK;
    for (int t = 0; t < tiles_m * d.tiles_n; ++t) {
      int tm, tn;
      tile_raster(t, tiles_m, d.tiles_n, &tm, &tn);
      out->push_back(make_int4(k | (KB << 24), (tm * persist::BM) | ((tn * persist::BN) << 16), d.map_x,
                               d.map_y + nsl));
    }
  }
}

cudaError_t launch_fxb_persist(const GemmDesc* d_descs, int tiles, const int4* d_tile_rec,
                               const void* d_maps, int nsl, int num_sms, Scale* scales, unsigned* status,
                               cudaStream_t s) {
  const int grid = tiles < num_sms ? tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  const CUtensorMap* maps = (const CUtensorMap*)d_maps;
  if (nsl == 3)
    tc_fxb_persist_kernel<3><<<grid, persist::THREADS, persist::Cfg<3>::SMEM, s>>>(
        d_descs, tiles, d_tile_rec, maps, scales, status);
  else
    tc_fxb_persist_kernel<2><<<grid, persist::THREADS, persist::Cfg<2>::SMEM, s>>>(
        d_descs, tiles, d_tile_rec, maps, scales, status);
  return cudaGetLastError();
}

}  // namespace mp
