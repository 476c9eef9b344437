// Exact-split BF16X3 products on CTA pairs (tcgen05 cta_group::2), for large
// orders.  The arithmetic is that of tc_fxb_kernel<128, 2> (fxb.cuh: integer
// slice products exact in the float32 TMEM accumulators, folded per 64-deep
// k-block with the block factors, re-split by 64 x 64 blocks), so every
// result is bit-for-bit the same; only the MMA's operands are spread over
// two SMs.
//
// The idea.  One 128 x 128 tile per SM issues, per 16-deep k-step,
// a1 [b1 | b2] (N = 256) and a2 b1 (N = 128): 20 KB of operand reads from
// shared memory, beside 16 KB of TMA writes into it, for 192 tensor-core
// cycles of work -- about 1.5x what shared memory delivers per cycle, so the
// tensor pipe runs at ~2/3 of its rate (measured: 575 ns of MMA execution
// per k-block against 371 ns at the full rate).  Two SMs computing a
// 256 x 128 tile with M = 256 MMAs each hold their own 128 rows of the A
// slices and half of the B slices' columns: per SM and k-step, three
// M = 256, N = 128 MMAs read 18 KB and the TMA writes 12 KB.
//
// CTA pair = cluster of 2 (rank 0 issues the MMAs).  Per k-block each CTA's
// TMA loads its a1, a2 rows and its 64 columns of b1, b2 into its own ring
// stage and completes on its own `full` barrier; rank 1 relays that to rank
// 0's `pfull` barrier (remote arrive, release at cluster scope).  Rank 0
// waits for both, issues the 12 MMAs of the k-block and commits, multicast to
// both CTAs, the stage's `empty` barrier and the accumulator buffer's `accfull`
// barrier.  Each CTA's epilogue warps fold their own TMEM rows and arrive on
// rank 0's `accempty` (16 warps; rank 1's by a relaxed remote arrive).  Every wait is bounded; a CTA that gives up
// drains, meets its peer at the closing cluster barrier and reports
// MATPOW_ETIMEDOUT.
//
// Used for N > 2048 (64 or more k-blocks), where every tile walks its
// k-blocks from 0 (fxb::tile_rot), so both CTAs of a pair fold in the same
// order as the one-CTA kernel.  Opt-in (MATPOW_OPT_PAIR): measured on a GB300
// at N = 8192 it takes 2.93 ms per product against the one-SM kernel's
// 2.47 ms.  Per k-block the MMA issuer still waits ~80 ns for accumulators
// and ~100 ns for operands, and the MMAs themselves take ~680 ns against
// ~575 ns on one SM: serving the peer's reads of its B half costs each SM
// the shared-memory bandwidth the halved B saves, while the A slices, read
// once per MMA, are not shared; only the TMA write traffic drops (12 KB per
// k-step against 16 KB).
#include <cuda.h>
#include <cuda_bf16.h>

#include "fxb.cuh"
#include "internal.cuh"
#include "plan.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace mp {

namespace pair {
constexpr int BM = 128, BN = 128, BK = 64, NSL = 2;
constexpr int EW = 8;                    // epilogue warps: 4 lane quadrants x 2 column halves
constexpr int WC = 64;                   // columns per epilogue warp
constexpr int THREADS = 128 + 32 * EW;   // TMA, MMA, TMEM, exponents + epilogue
constexpr int A_BYTES = BM * BK * 2;     // one slice, this CTA's 128 rows
constexpr int BH_BYTES = (BN / 2) * BK * 2;  // one slice, this CTA's 64 columns
constexpr int STAGE_BYTES = NSL * (A_BYTES + BH_BYTES);  // 48 KB
constexpr int STAGES = 4;
constexpr int RING = STAGES * STAGE_BYTES;              // 192 KB
constexpr int NG = BN / fxb::BLK;
constexpr int EXP_BYTES = (2 + NG) * fxb::MAX_KB * 4;
constexpr int NBARS = 3 * STAGES + 5;  // full, empty, pfull, accfull[2], accempty[2], drain
constexpr int SMEM = RING + 1024 + 256 + EXP_BYTES + 64;
constexpr int TMEM_COLS = 512;         // 2 buffers x (main | cross) x 128 columns
constexpr uint64_t WAIT_NS = 2000000000ull;
static_assert(NBARS * 8 + 16 <= 256, "barrier area");
static_assert(2 * 2 * BN <= TMEM_COLS, "TMEM");
}  // namespace pair

__device__ __forceinline__ uint32_t pair_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t pair_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void pair_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t pair_mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Arrive on the peer's mbarrier without release semantics.  Both uses order
// no memory writes, only completed hardware work: the relay arrives after its
// CTA's TMA bytes have landed (its own `full` phase completed), and an
// epilogue warp arrives after its tcgen05.ld's have completed
// (tcgen05.wait::ld) -- the peer's next MMAs may then overwrite those TMEM
// columns.  A release at cluster scope costs a cluster-wide fence (measured:
// ~570 ns per k-block on the epilogue's path, which the MMA issuer then waited
// for); relaxed, the arrive is a plain message.
__device__ __forceinline__ void pair_arrive_remote(uint32_t a) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(a) : "memory");
}
// Bounded wait on a local mbarrier that other CTAs of the cluster arrive at
// (acquire at cluster scope); gives up after budget_ns or once *abort is set.
__device__ __forceinline__ bool pair_wait(uint32_t bar, uint32_t parity, volatile int* abort, uint64_t budget_ns) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = ptx::globaltimer();
    if ((it & 255u) == 255u) {
      if (*abort) return false;
      if (ptx::globaltimer() - t0 > budget_ns) return false;
    }
  }
}

// One CTA of the pair computing rows m0 .. m0 + 127 (m0 = the pair's first
// row + 128 rank) and columns n0 .. n0 + 127 of product d.
__device__ __forceinline__ void fxb_pair_cta(const GemmDesc& d, int pt, const CUtensorMap* ax0,
                                             const CUtensorMap* ax1, const CUtensorMap* by0,
                                             const CUtensorMap* by1, const CUtensorMap* const (&cx)[2],
                                             Scale* scales, unsigned* status) {
  using namespace pair;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + RING);
  uint32_t* tmem_slot = (uint32_t*)(bars + NBARS);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* epi_ok = (volatile int*)(tmem_slot + 2);
  int* eA = (int*)(smem + RING + 256);
  int* eB = eA + 2 * fxb::MAX_KB;
  float* red = (float*)(eB + NG * fxb::MAX_KB);
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t pfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 3 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 3 * STAGES + 2);
  const uint32_t drainb = ptx::smem_u32(bars + 3 * STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = pair_rank();
  int tm2, tn;
  tile_raster(pt, (d.N + 2 * BM - 1) / (2 * BM), d.tiles_n, &tm2, &tn);  // 256-row pair tiles
  const int m0 = tm2 * 2 * BM + (int)rank * BM, n0 = tn * BN;
  const int N = d.N;
  const int KB = (N + BK - 1) / BK;
  const size_t boff = fxb::bexp_offset(N, d.ld, NSL);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
      ptx::mbar_init(pfull0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, 2 * EW);  // both CTAs' epilogue warps
    }
    ptx::mbar_init(drainb, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    ptx::prefetch_tmap(ax0);
    ptx::prefetch_tmap(ax1);
    ptx::prefetch_tmap(by0);
    ptx::prefetch_tmap(by1);
  }
  // both CTAs' barriers are initialised before any remote arrival or commit
  pair_sync();
  if (warp == 2) {
    ptx::tmem_alloc_pair(ptx::smem_u32(tmem_slot), TMEM_COLS);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer (both CTAs): own rows of a1, a2; own half of b1, b2
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = full0 + 8 * s;
        ptx::mbar_expect_tx(fb, STAGE_BYTES);
        const uint32_t base = ptx::smem_u32(smem + s * STAGE_BYTES);
        const int kx = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB)) * BK;
        ptx::tma_load_2d(base, ax0, kx, m0, fb);
        ptx::tma_load_2d(base + A_BYTES, ax1, kx, m0, fb);
        const int nb = n0 + (int)rank * (BN / 2);
        ptx::tma_load_2d(base + NSL * A_BYTES, by0, nb, kx, fb);
        ptx::tma_load_2d(base + NSL * A_BYTES + BH_BYTES, by1, nb, kx, fb);
        ++issued;
      }
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
        int dummy = 0;
        ptx::mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, &dummy, WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 1) {
      // ---- relay: this CTA's stage has landed -> rank 0's pfull
      const uint32_t pf0 = pair_mapa(pfull0, 0);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        if (!ptx::mbar_wait(full0 + 8 * s, (kb / STAGES) & 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        pair_arrive_remote(pf0 + 8 * s);
      }
    } else if (lane == 0) {
      // ---- MMA issuer (rank 0): 3 pair MMAs per 16-deep k-step
      constexpr uint32_t idesc = idesc_bf16(2 * BM, BN);
      for (int kb = 0; kb < KB; ++kb) {
        const int buf = kb & 1;
        const uint32_t tmain = tmem + (uint32_t)(buf * 2 * BN);
        const uint32_t tcross = tmain + BN;
        if (!pair_wait(accempty0 + 8 * buf, ((kb >> 1) & 1) ^ 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!ptx::mbar_wait(full0 + 8 * s, ph, abort_flag, WAIT_NS) ||
            !pair_wait(pfull0 + 8 * s, ph, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t a0 = ptx::smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b0 = a0 + NSL * A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t a1 = ptx::smem_desc(a0 + 32 * k, 16, 1024);
          const uint64_t a2 = ptx::smem_desc(a0 + A_BYTES + 32 * k, 16, 1024);
          const uint64_t b1 = ptx::smem_desc(b0 + 2048 * k, 8192, 1024);
          const uint64_t b2 = ptx::smem_desc(b0 + BH_BYTES + 2048 * k, 8192, 1024);
          const uint32_t acc = k == 0 ? 0u : 1u;
          ptx::mma_f16_pair(tmain, a1, b1, idesc, acc);   // a1 b1
          ptx::mma_f16_pair(tcross, a1, b2, idesc, acc);  // a1 b2
          ptx::mma_f16_pair(tcross, a2, b1, idesc, 1u);   // + a2 b1
        }
        ptx::mma_commit_pair_mc(empty0 + 8 * s, 0x3);
        ptx::mma_commit_pair_mc(accfull0 + 8 * buf, 0x3);
      }
      ptx::mma_commit_pair(drainb);
      int dummy = 0;
      ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
    }
  } else if (warp == 3) {
    fxb::load_tile_exponents<BN>((const int*)((const char*)d.X + boff), (const int*)((const char*)d.Y + boff), N,
                                 m0, n0, KB, eA, eB, lane);
    __syncwarp();
    asm volatile("bar.arrive 2, %0;" ::"n"(32 + 32 * EW) : "memory");
  } else if (warp >= 4) {
    // ---- epilogue (both CTAs): fold this CTA's 128 TMEM lanes
    const int e = warp - 4;
    const int q = warp & 3;
    const int cs = e >> 2;
    const int h = q >> 1;
    const int row = m0 + 32 * q + lane;
    const int nw = n0 + cs * WC;
    const int sx = scale_exp_from_bits(scales[d.sx].maxbits);
    const int sy = scale_exp_from_bits(scales[d.sy].maxbits);
    const uint32_t ae0 = pair_mapa(accempty0, 0);
    float T[WC];
#pragma unroll
    for (int j = 0; j < WC; ++j) T[j] = 0.f;
    asm volatile("bar.sync 2, %0;" ::"n"(32 + 32 * EW) : "memory");  // exponents staged
    bool ok = true;
    for (int kb = 0; kb < KB; ++kb) {
      const int buf = kb & 1;
      int dummy = 0;
      if (!ptx::mbar_wait(accfull0 + 8 * buf, (kb >> 1) & 1, &dummy, 2 * WAIT_NS)) {
        *abort_flag = 1;
        ok = false;
        break;
      }
      ptx::tc_fence_after();
      const int kr = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB));
      float fac[WC / 64];
#pragma unroll
      for (int g = 0; g < WC / 64; ++g)
        fac[g] = fxb::pow2f(eA[h * KB + kr] + eB[kr * NG + cs * (WC / 64) + g] - 16 - sx - sy);
      fxb::fold<WC, NSL>(T, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 2 * BN + cs * WC), fac, BN);
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          ptx::mbar_arrive(accempty0 + 8 * buf);
        else
          pair_arrive_remote(ae0 + 8 * buf);
      }
    }
    fxb::epi_bar<32 * EW>();
    if (e == 0 && lane == 0) *epi_ok = ok && !*abort_flag;
    fxb::epi_bar<32 * EW>();
    ok = *epi_ok != 0;
    const long long Ec = scales[d.sx].E + scales[d.sy].E + sx + sy;
    if (d.mode == OUT_INTERNAL) {
      if (pt == 0 && rank == 0 && e == 0 && lane == 0) scales[d.sc].E = Ec;
      // (the second CTA of the last pair row may lie wholly below row N - 1:
      // then it has nothing to store; the condition is the same for all its
      // epilogue warps, which share the named barriers inside)
      if (ok && m0 < N)  // every epilogue warp reaches the named barriers inside; the ring is idle
        fxb::store_slices_tma<WC, 32 * EW, NSL>(T, 32 * q + lane, m0, nw, q, lane, N, cs * (WC / 64), BN / 64,
                                                smem, cx, (int*)((char*)d.C + boff), &scales[d.sc].maxbits, red,
                                                e == 0 && lane == 0, n0);
    } else if (ok) {
      if (pt == 0 && rank == 0 && e == 0 && lane == 0 && d.mode == OUT_USER_MANT && d.out_log2) *d.out_log2 = Ec;
      if (row < N) {
        float* O = (float*)d.out + (size_t)row * N;
        store_row_f32<WC>(T, O, nw, N, d.mode == OUT_USER_MANT, Ec, status, d.out);
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // neither CTA leaves (or frees TMEM) while its peer may still read its
  // shared memory, write its TMEM or arrive at its barriers
  pair_sync();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
}

// Grid: 2 CTAs per 256 x 128 pair tile, the first product's pair tiles first.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(pair::THREADS, 1)
    tc_fxb_pair_kernel(const __grid_constant__ TcPairParams P, Scale* scales, unsigned* status) {
  int pt = blockIdx.x >> 1;
  const int which = (P.count > 1 && pt >= P.tiles0) ? 1 : 0;
  if (which) pt -= P.tiles0;
  const TcProblem& pr = P.p[which];
  const CUtensorMap* cx[2] = {&pr.cx[0], &pr.cx[1]};
  if (pair_nctarank() != 2) {  // launched without its clusters: nothing can run safely
    if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    return;
  }
  fxb_pair_cta(pr.d, pt, &pr.ax[0], &pr.ax[1], &pr.by[0], &pr.by[1], cx, scales, status);
}

cudaError_t tc_pair_init() {
  return cudaFuncSetAttribute(tc_fxb_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pair::SMEM);
}

int pair_tiles(int N) { return ((N + 2 * pair::BM - 1) / (2 * pair::BM)) * ((N + pair::BN - 1) / pair::BN); }

cudaError_t launch_fxb_pair(const TcPairParams& P, int pair_tiles_total, Scale* scales, unsigned* status,
                            cudaStream_t s) {
  tc_fxb_pair_kernel<<<2 * pair_tiles_total, pair::THREADS, pair::SMEM, s>>>(P, scales, status);
  return cudaGetLastError();
}

}  // namespace mp
