// The whole square-and-multiply chain (arXiv 1204.3052 Sec. 4.3) in ONE
// cooperative tensor-core launch, for small and medium N.
//
// For N up to ~1000 a product is a handful of 128-row tiles, so launching one
// kernel per level (plus a split pass) is dominated by launch and ramp-up
// latency.  Here every CTA stays resident for the whole power (cooperative
// launch, one CTA per SM, at most one output tile per CTA per level), keeps
// its TMEM allocation and its mbarrier ring across levels, and the levels are
// separated by grid-wide barriers:
//
//   prep:   block-scaled exact split of A, max|A| -> barrier
//   level:  tile product (TMA -> tcgen05.mma on integer slices -> exact
//           64-deep TMEM partial sums -> float32 registers with the block
//           factors) -> re-split by 64 x 64 blocks straight from registers,
//           block exponents, max|C| -> barrier
//   last:   the final product writes the user's float32 output directly.
//
// Compared with the level-by-level path this removes every kernel launch but
// one.  The arithmetic is that of fxb.cuh, identical to the level kernels'.
//
// Split-K: when a level has few tiles (N up to ~540), S = 2 or 4 CTAs of a
// thread-block cluster share one output tile, each taking a contiguous run of
// its (rotated) k-blocks.  The non-leading CTAs push their float32 partial
// tiles into the leader's shared memory (distributed shared memory stores,
// then a remote mbarrier arrival); the leader adds them in rank order and
// runs the epilogue.  The sum order differs from the single-CTA fold, so
// split-K results equal the level path's to rounding, not bit for bit.
//
// Every wait is bounded: an mbarrier or grid barrier that gives up sets
// MATPOW_ETIMEDOUT in the plan's status word, and all CTAs then leave the
// chain, drain their copies and MMAs and free TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "tc_ptx.cuh"
#include "fxb.cuh"

namespace mp {

namespace chain {
// warps 0-3: TMA, MMA, TMEM allocation, exponent staging; warps 4-11: the
// epilogue, warp 4 + 4 cs + q holding rows 32q.. and columns half cs of the tile
constexpr int BM = 128, BK = 64, THREADS = 384, NEPI = 256, CHUNK_KB = 4;
constexpr int MAX_LEVELS = 64;
constexpr uint64_t WAIT_NS = 2000000000ull;
// dynamic shared memory: the 227 KB per CTA less the per-level work table
// (static shared memory, WORK_BYTES)
constexpr int WORK_BYTES = 24 * MAX_LEVELS;
constexpr int SMEM_MAX = 227 * 1024 - WORK_BYTES;
template <int BN, int NSL, int S>
struct Cfg {
  static constexpr int NG = BN / fxb::BLK;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = NSL * (A_BYTES + B_BYTES);
  static constexpr int KB_MAX = 16;  // N <= 1024
  // after the ring: barriers (256 B), exponent tables, epilogue scratch, then
  // the split-K buffer at XOFF (16-byte aligned); 1024 B of alignment slack
  static constexpr int XOFF = 256 + (2 + NG) * KB_MAX * 4 + 64;
  static constexpr int EXTRA = 1024 + XOFF;
  // partial tiles of the S - 1 other CTAs of the cluster (leader only)
  static constexpr int XBUF = (S - 1) * BM * BN * 4;
  static constexpr int RING_WANT = NSL == 3 ? 216 * 1024 : 192 * 1024;
  static constexpr int RING_FIT = SMEM_MAX - EXTRA - XBUF;
  static constexpr int RING = RING_WANT < RING_FIT ? RING_WANT : RING_FIT;
  static constexpr int STAGES = RING / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + EXTRA + XBUF;
  static constexpr int TMEM_USED = 2 * NSL * BN;  // NSL accumulators x 2 buffers
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
  static_assert(TMEM_USED <= 512, "TMEM");
  static_assert(STAGES >= 2, "at least two ring stages");
  static_assert(NSL * 16384 * NG <= STAGES * STAGE_BYTES, "epilogue staging fits the ring");
  static_assert(SMEM <= SMEM_MAX, "shared memory");
};
struct Op {
  signed char xb, yb, cb, last;
  short sx, sy, sc, pad;
};
}  // namespace chain

// One power A^n of the launch (its own four buffers and scale slots).
struct ChainProblem {
  CUtensorMap amap[4][3];  // buffer b as the A operand: slice planes (box 64 x 128)
  CUtensorMap bmap[4][3];  // buffer b as the B operand: slice planes (box 64 x 64)
  void* slices[4];         // first slice plane of buffer b (the next at + plane elements)
  int* bexp[4];            // block exponents of buffer b
  long long plane;
  const float* A;
  float* out;
  long long* out_log2;
  Scale* scales;  // this power's slots (ops' slot numbers are relative to it)
  int N, ld, tiles_n, tiles_per_op;
  chain::Op ops[2 * chain::MAX_LEVELS];
};
constexpr int CHAIN_MAXP = 4;  // independent powers in one launch
// Up to four independent powers in one cooperative launch: level L of every
// power runs between the same pair of grid barriers; the CTAs of level L are
// dealt out to the powers' tiles in order (lvl_begin[L][p] = first CTA group
// of power p; lvl_begin[L][nprob] = the level's tile count).
struct ChainParams {
  ChainProblem pr[CHAIN_MAXP];
  unsigned* status;
  unsigned* gbar;
  int nprob, nlevels;
  int prep_begin[CHAIN_MAXP + 1];  // first 64 x 64 prep block of power p
  short lvl_begin[chain::MAX_LEVELS][CHAIN_MAXP + 1];
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---- thread-block cluster helpers (split-K)
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster executes this the same number of
// times (at kernel start and end only), so it cannot wait for a thread that
// never comes.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory address `a` of this CTA -> the same offset in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z),
               "f"(w)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(a), "r"(count)
               : "memory");
}
// Bounded wait on a local mbarrier whose arrivals come from other CTAs of the
// cluster (acquire at cluster scope).
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, uint64_t budget_ns) {
  const uint64_t t0 = ptx::globaltimer();
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
    if ((it & 255u) == 255u && ptx::globaltimer() - t0 > budget_ns) return false;
  }
}

// Grid-wide barrier number `k` (1, 2, ...) over `G` co-resident CTAs.
__device__ __forceinline__ bool grid_sync(unsigned* gbar, unsigned target, unsigned* status,
                                          volatile int* cta_abort) {
  __syncthreads();
  if (threadIdx.x == 0 && !*cta_abort) {
    __threadfence();
    atomicAdd(gbar, 1u);
    const uint64_t t0 = ptx::globaltimer();
    for (unsigned it = 0;; ++it) {
      if (ld_acquire_gpu(gbar) >= target) break;
      if ((it & 63u) == 63u) {
        if (*(volatile unsigned*)status & ST_TIMEOUT) {
          *cta_abort = 1;
          break;
        }
        if (ptx::globaltimer() - t0 > chain::WAIT_NS) {
          atomicOr(status, ST_TIMEOUT);
          *cta_abort = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  return !*cta_abort;
}

__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// One CTA's assignment at one level (24 bytes).
struct LevelWork {
  chain::Op op;
  short pi;  // power, or -1: no tile at this level
  short f;   // CTAs per tile at this level
  short t, m0, n0, N;
};
static_assert(sizeof(LevelWork) * chain::MAX_LEVELS <= chain::WORK_BYTES, "work table");

// The end of a tile's level work by the NT epilogue threads that own its rows
// (q_first: the first of their row quadrants; each thread holds WC columns
// from c0 = n0 + cs WC): one verdict over them, then the user output (final
// product) or the next operand's block exponents and slices.
template <int WC, int NSL, int NT>
__device__ __forceinline__ void chain_finish(float (&T)[WC], bool ok, volatile int* epi_ok,
                                             volatile int* abort_flag, int q, int cs, int lane, int row, int t,
                                             int m0, int n0, int N, const ChainProblem& Q, const chain::Op& op,
                                             long long Ec, unsigned* status, float* ered, int q_first) {
  const int c0 = n0 + cs * WC;
  const bool first = cs == 0 && lane == 0;
  fxb::epi_bar<NT>();
  if (q == q_first && first) *epi_ok = ok && !*abort_flag;
  fxb::epi_bar<NT>();
  ok = *epi_ok != 0;
  if (op.last) {
    if (ok) {
      if (t == 0 && q == 0 && first && Q.out_log2) *Q.out_log2 = Ec;
      // 16-byte stores where the rows allow
      if (row < N) store_row_f32<WC>(T, Q.out + (size_t)row * N, c0, N, Q.out_log2 != nullptr, Ec, status, Q.out);
    }
  } else {
    if (t == 0 && q == 0 && first) Q.scales[op.sc].E = Ec;
    if (ok)  // 16-byte stores straight from registers (the next level's copies
             // read them after the grid barrier)
      fxb::store_slices_part<WC, NT, NSL>(T, row, m0, n0, c0, q, cs, lane, N, Q.ld, (__nv_bfloat16*)Q.slices[op.cb],
                                          Q.plane, Q.bexp[op.cb], &Q.scales[op.sc].maxbits, ered);
    // the next level's TMA reads these stores after the grid barrier, whose
    // __syncthreads and single fenced arrival make every thread's stores
    // visible GPU-wide (as for the prep's stores); the proxy fence orders
    // them before async-proxy reads
    fence_proxy_async_global();
  }
}

template <int BN, int NSL, int S>
__device__ __forceinline__ void chain_body(const ChainParams& P) {
  using namespace chain;
  using C = Cfg<BN, NSL, S>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  // full[S], empty[S], accfull[2], accempty[2], drain, (tmem_slot, flags,
  // red), xbar, full2[S]: full completes with a stage's first A slice and
  // its B slices, full2 with the other A slices
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* epi_ok = (volatile int*)(tmem_slot + 2);
  float* red = (float*)(tmem_slot + 4);  // 8 floats
  constexpr int NG = C::NG;
  constexpr int WC = BN / 2;              // columns of one epilogue thread
  constexpr int NGW = WC < 64 ? 1 : WC / 64;  // its 64-column blocks
  int* eA = (int*)(smem + STAGES * C::STAGE_BYTES + 256);
  int* eB = eA + 2 * C::KB_MAX;
  float* ered = (float*)(eB + NG * C::KB_MAX);
  // split-K: partial tiles pushed by the other CTAs of the cluster, as
  // float4 [rank - 1][BN / 4][128 rows]; xbar completes once per level
  // ((S - 1) x NEPI arrivals: pushing threads arrive with weights that
  // complete it for every split factor)
  float4* xbuf = (float4*)(smem + STAGES * C::STAGE_BYTES + C::XOFF);
  const uint32_t xbar = ptx::smem_u32(bars + 2 * STAGES + 5 + 8);  // past tmem_slot..red
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drainb = ptx::smem_u32(bars + 2 * STAGES + 4);
  const uint32_t full2_0 = ptx::smem_u32(bars + 2 * STAGES + 14);
  static_assert((3 * STAGES + 14) * 8 <= 256, "barrier area");

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned G = gridDim.x;
  unsigned bar_no = 0;

  // the reads of this CTA's first two prep blocks go out before the setup
  float pv[2][16];
  const int n_prep = P.prep_begin[P.nprob];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int b = blockIdx.x + i * G;
    if (b < n_prep) {
      int pi = 0;
      while (pi + 1 < P.nprob && b >= P.prep_begin[pi + 1]) ++pi;
      const int nb = fxb::nblocks(P.pr[pi].N);
      const int lb = b - P.prep_begin[pi];
      fxb::prep_load(P.pr[pi].A, P.pr[pi].N, lb / nb, lb % nb, pv[i]);
    }
  }
  // split-K needs the launch's clusters of S; launched without them (each CTA
  // its own cluster), every CTA computes whole tiles
  const bool clustered = S > 1 && cluster_nctarank() == (uint32_t)S;
  const int crank = clustered ? (int)cluster_ctarank() : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(full2_0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, NEPI / 32);
    }
    ptx::mbar_init(drainb, 1);
    if (clustered) ptx::mbar_init(xbar, (S - 1) * NEPI);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  __syncthreads();  // barriers and the abort flag initialised
  __shared__ LevelWork s_work[chain::MAX_LEVELS];
  if (threadIdx.x < 256) {
    // ---- prep: block-scaled exact split of each A into its buffer 0,
    // max|A| into its slot 1 (threads 0..255 on named barrier 3, while the
    // other warps set up the levels)
    int i = 0;
    for (int b = blockIdx.x; b < n_prep; b += G, ++i) {
      int pi = 0;
      while (pi + 1 < P.nprob && b >= P.prep_begin[pi + 1]) ++pi;
      const ChainProblem& Q = P.pr[pi];
      const int nb = fxb::nblocks(Q.N);
      const int lb = b - P.prep_begin[pi];
      if (i < 2)
        fxb::prep_split<NSL, 256>(i == 0 ? pv[0] : pv[1], Q.N, Q.ld, lb / nb, lb % nb,
                                  (__nv_bfloat16*)Q.slices[0], Q.plane, Q.bexp[0], &Q.scales[1].maxbits, P.status,
                                  red);
      else
        fxb::prep_block<NSL, 256>(Q.A, Q.N, Q.ld, lb / nb, lb % nb, (__nv_bfloat16*)Q.slices[0], Q.plane,
                                  Q.bexp[0], &Q.scales[1].maxbits, P.status, red);
    }
    fence_proxy_async_global();
  } else if (warp == 8) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::TMEM_COLS);
    ptx::tmem_relinquish();
  } else if (warp == 9) {
    if (lane == 0)
      for (int pi = 0; pi < P.nprob; ++pi)
        for (int b = 0; b < 4; ++b)
          for (int k = 0; k < NSL; ++k) {
            ptx::prefetch_tmap(&P.pr[pi].amap[b][k]);
            ptx::prefetch_tmap(&P.pr[pi].bmap[b][k]);
          }
  } else {
    // this CTA's work at every level (tile, power, split), from the launch
    // tables in parameter space, once: one thread of warps 10-11 per level
    for (int L = threadIdx.x - 320; L < P.nlevels; L += 64) {
      // the level's split: f CTAs of a cluster share a tile, the largest f
      // (dividing S) with f x (tiles of the level) <= G; the cluster's S CTAs
      // then work on S / f tiles
      const int T_L = P.lvl_begin[L][P.nprob];
      int f = 1;
      if (clustered) {
        f = S;
        while (f > 1 && f * T_L > (int)G) f >>= 1;
      }
      const int t_all = clustered ? (int)(blockIdx.x / S) * (S / f) + crank / f : (int)blockIdx.x;
      LevelWork w;
      w.f = (short)f;
      w.pi = -1;
      w.t = 0;
      w.m0 = w.n0 = 0;
      w.N = (short)P.pr[0].N;
      w.op = P.pr[0].ops[2 * L];
      if (t_all < T_L) {
        int pi = 0;  // the power this CTA group works for at level L
        while (pi + 1 < P.nprob && t_all >= P.lvl_begin[L][pi + 1]) ++pi;
        const ChainProblem& Q = P.pr[pi];
        const int local = t_all - P.lvl_begin[L][pi];
        const int oi = local / Q.tiles_per_op;
        const int t = local - oi * Q.tiles_per_op;
        const int tm = t / Q.tiles_n, tn = t - tm * Q.tiles_n;
        w.pi = (short)pi;
        w.t = (short)t;
        w.op = Q.ops[2 * L + oi];
        w.N = (short)Q.N;
        w.m0 = (short)(tm * BM);
        w.n0 = (short)(tn * BN);
      }
      s_work[L] = w;
    }
  }
  // every CTA of the cluster has started and initialised its barriers before
  // any remote store or arrival
  if (clustered) cluster_sync_all();
  // the grid barrier's CTA barrier also publishes the work table and the
  // TMEM address
  ptx::tc_fence_before();
  grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag);
  ptx::tc_fence_after();
  fence_proxy_async_global();
  const uint32_t tmem = *tmem_slot;
  int kb_base = 0;  // k-blocks done by this CTA: ring and accumulator-buffer phases
  uint32_t xph = 0;  // phase of xbar (leader)
  float T[WC];
  for (int L = 0; L < P.nlevels && !*abort_flag; ++L) {
    // this CTA's work at level L, worked out at kernel start
    const LevelWork W = s_work[L];
    const int f = W.f;
    const int sub = crank / f;
    const int rank = crank - sub * f;  // rank within the tile's group; 0 leads
    const int lead_rank = sub * f;     // cluster rank of the group's leader
    const bool has = W.pi >= 0;
    const ChainProblem& Q = P.pr[has ? W.pi : 0];
    const int t = W.t;
    const chain::Op op = W.op;
    const int N = W.N;
    const int KB = (N + BK - 1) / BK;
    // this CTA's run of the tile's k-blocks (in the rotated visiting order)
    const int i0 = rank * KB / f, i1 = (rank + 1) * KB / f;
    const int nkb = i1 - i0;
    const int m0 = W.m0, n0 = W.n0;
    const int q = (warp - 4) & 3;    // TMEM lane quadrant: rows 32q .. 32q + 31
    const int cs = (warp - 4) >> 2;  // column half of the tile
    const int row = m0 + 32 * q + lane;

    if (has) {
      if (warp == 0) {
        if (lane == 0) {
          for (int kb = i0; kb < i1; ++kb) {
            const int g = kb_base + kb - i0;
            const int s = g % STAGES;
            const uint32_t ph = (g / STAGES) & 1;
            if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            // the first A slice and the B slices (the first MMAs' operands)
            // on full, the other A slices on full2
            const uint32_t fb = full0 + 8 * s, fb2 = full2_0 + 8 * s;
            ptx::mbar_expect_tx(fb, C::A_BYTES + NSL * C::B_BYTES);
            ptx::mbar_expect_tx(fb2, (NSL - 1) * C::A_BYTES);
            const uint32_t base = ptx::smem_u32(smem + s * C::STAGE_BYTES);
            const int kx = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB)) * BK;
            ptx::tma_load_2d(base, &Q.amap[op.xb][0], kx, m0, fb);
            const uint32_t bbase = base + NSL * C::A_BYTES;
#pragma unroll
            for (int c = 0; c < BN / 64; ++c)
#pragma unroll
              for (int k = 0; k < NSL; ++k)
                ptx::tma_load_2d(bbase + k * C::B_BYTES + c * 8192, &Q.bmap[op.yb][k], n0 + 64 * c, kx,
                                 fb);
#pragma unroll
            for (int k = 1; k < NSL; ++k)
              ptx::tma_load_2d(base + k * C::A_BYTES, &Q.amap[op.xb][k], kx, m0, fb2);
          }
        }
      } else if (warp == 1) {
        if (lane == 0) {
          for (int kb = i0; kb < i1; ++kb) {
            const int g = kb_base + kb - i0;
            const int buf = g & 1;
            const uint32_t t0 = tmem + (uint32_t)(buf * NSL * BN);
            if (!ptx::mbar_wait(accempty0 + 8 * buf, ((g >> 1) & 1) ^ 1, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            const int s = g % STAGES;
            const uint32_t ph = (g / STAGES) & 1;
            if (!ptx::mbar_wait(full0 + 8 * s, ph, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a0 = ptx::smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t b0 = a0 + NSL * C::A_BYTES;
            // slice-major: a_0 [b_0 | ... ] over the four k-steps (the k-step-0
            // MMA initialises every accumulator), then, once full2 completes,
            // a_i [b_0 | ... | b_(NSL-1-i)] for i >= 1.  The accumulators hold
            // exact integer sums, so this order gives fxb::slice_mmas' results.
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              ptx::mma_f16(t0, ptx::smem_desc(a0 + 32 * k, 16, 1024),
                           ptx::smem_desc(b0 + 2048 * k, 8192, 1024), idesc_bf16(128, NSL * BN),
                           k == 0 ? 0u : 1u);
            if (!ptx::mbar_wait(full2_0 + 8 * s, ph, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            ptx::tc_fence_after();
#pragma unroll
            for (int i = 1; i < NSL; ++i)
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                ptx::mma_f16(t0 + (uint32_t)(i * BN), ptx::smem_desc(a0 + i * C::A_BYTES + 32 * k, 16, 1024),
                             ptx::smem_desc(b0 + 2048 * k, 8192, 1024), idesc_bf16(128, (NSL - i) * BN), 1u);
            ptx::mma_commit(empty0 + 8 * s);
            ptx::mma_commit(accfull0 + 8 * buf);
          }
        }
      } else if (warp == 3) {
        fxb::load_tile_exponents<BN>(Q.bexp[op.xb], Q.bexp[op.yb], N, m0, n0, KB, eA, eB, lane);
        __syncwarp();
        asm volatile("bar.arrive 2, %0;" ::"n"(32 + NEPI) : "memory");
      } else if (warp >= 4) {
        const int h = q >> 1;
        // scale slots are written by other CTAs: read them from L2, not L1
        const int sx = scale_exp_from_bits(__ldcg(&Q.scales[op.sx].maxbits));
        const int sy = scale_exp_from_bits(__ldcg(&Q.scales[op.sy].maxbits));
        const long long Ec = __ldcg(&Q.scales[op.sx].E) + __ldcg(&Q.scales[op.sy].E) + sx + sy;
#pragma unroll
        for (int j = 0; j < WC; ++j) T[j] = 0.f;
        asm volatile("bar.sync 2, %0;" ::"n"(32 + NEPI) : "memory");  // exponents staged
        const int gb0 = cs * WC / 64;  // first 64-column block of this thread's columns
        bool ok = true;
        for (int kb = i0; kb < i1; ++kb) {
          const int g = kb_base + kb - i0;
          const int buf = g & 1;
          int dummy = 0;
          if (!ptx::mbar_wait(accfull0 + 8 * buf, (g >> 1) & 1, &dummy, 2 * WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const int kr = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB));
          float fac[NGW];
#pragma unroll
          for (int gg = 0; gg < NGW; ++gg)
            fac[gg] = fxb::pow2f(eA[h * KB + kr] + eB[kr * NG + gb0 + gg] - 16 - sx - sy);
          fxb::fold<WC, NSL>(T, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * NSL * BN + cs * WC), fac,
                             BN);
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(accempty0 + 8 * buf);
        }
        const int et = 32 * q + lane;  // tile row
        const int cq0 = cs * WC / 4;   // this thread's first float4 column
        // f = 2: the two CTAs of the tile each finish one 64-row block row
        // (warps q with q / 2 = rank) and send the other rows to the partner;
        // f = 4: the group's first CTA gathers the other three partial tiles
        const bool rows2 = f == 2;
        const bool mine = rows2 ? (q >> 1) == rank : rank == 0;
        if (rows2) {
          if (!mine) {
            // this row belongs to the partner's block row: push it there
            // (weighted: NEPI / 2 pushing threads complete the barrier)
            const uint32_t prt = (uint32_t)(lead_rank + 1 - rank);
            const uint32_t dst = mapa_rank(ptx::smem_u32(xbuf), prt);
#pragma unroll
            for (int c = 0; c < WC / 4; ++c)
              st_cluster_v4(dst + (uint32_t)(((cq0 + c) * 128 + et) * 16), T[4 * c], T[4 * c + 1], T[4 * c + 2],
                            T[4 * c + 3]);
            mbar_arrive_remote(mapa_rank(xbar, prt), (uint32_t)(2 * (S - 1)));
          } else {
            if (!mbar_wait_cluster(xbar, xph, 2 * WAIT_NS)) {
              *abort_flag = 1;
              ok = false;
            }
            if (ok) {
              const float4* src = xbuf + cq0 * 128 + et;
#pragma unroll
              for (int c = 0; c < WC / 4; ++c) {
                const float4 v = src[c * 128];
                T[4 * c] += v.x;
                T[4 * c + 1] += v.y;
                T[4 * c + 2] += v.z;
                T[4 * c + 3] += v.w;
              }
            }
          }
          xph ^= 1;  // both CTAs' barriers complete once per such level
        } else if (!mine) {
          // push this partial tile into the leader's buffer, then arrive there
          // (weighted so that every split factor completes the leader's
          // barrier, initialised for S - 1 pushing CTAs, in one phase)
          const uint32_t dst =
              mapa_rank(ptx::smem_u32(xbuf + (size_t)(rank - 1) * (BN / 4) * 128), (uint32_t)lead_rank);
#pragma unroll
          for (int c = 0; c < WC / 4; ++c)
            st_cluster_v4(dst + (uint32_t)(((cq0 + c) * 128 + et) * 16), T[4 * c], T[4 * c + 1], T[4 * c + 2],
                          T[4 * c + 3]);
          mbar_arrive_remote(mapa_rank(xbar, (uint32_t)lead_rank), (uint32_t)((S - 1) / (f - 1)));
        } else if (f > 1) {
          // the other CTAs' partial tiles, added in rank order
          if (!mbar_wait_cluster(xbar, xph, 2 * WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
          }
          xph ^= 1;
          if (ok) {
#pragma unroll 1
            for (int r = 1; r < f; ++r) {
              const float4* src = xbuf + (size_t)(r - 1) * (BN / 4) * 128 + cq0 * 128 + et;
#pragma unroll
              for (int c = 0; c < WC / 4; ++c) {
                const float4 v = src[c * 128];
                T[4 * c] += v.x;
                T[4 * c + 1] += v.y;
                T[4 * c + 2] += v.z;
                T[4 * c + 3] += v.w;
              }
            }
          }
        }
        if (mine) {
          if (rows2)  // four warps (one block row) share the named barriers
            chain_finish<WC, NSL, NEPI / 2>(T, ok, epi_ok, abort_flag, q, cs, lane, row, t, m0, n0, N, Q, op, Ec,
                                            P.status, ered, 2 * rank);
          else
            chain_finish<WC, NSL, NEPI>(T, ok, epi_ok, abort_flag, q, cs, lane, row, t, m0, n0, N, Q, op, Ec,
                                        P.status, ered, 0);
        }
      }
      kb_base += nkb;  // ring and accumulator counters advance only with work done
    }
    if (L + 1 == P.nlevels) break;  // every power's final product has been written
    // this level's slices, exponents and maxima are visible to every CTA
    if (!grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag)) break;
    fence_proxy_async_global();
  }

  // ---- teardown: no copy or MMA of this CTA may still be in flight
  if (warp == 0 && lane == 0) {
    for (int g = kb_base - STAGES < 0 ? 0 : kb_base - STAGES; g < kb_base; ++g) {
      int dummy = 0;
      ptx::mbar_wait(full0 + 8 * (g % STAGES), (g / STAGES) & 1, &dummy, WAIT_NS);
      ptx::mbar_wait(full2_0 + 8 * (g % STAGES), (g / STAGES) & 1, &dummy, WAIT_NS);
    }
  }
  if (warp == 1 && lane == 0) {
    ptx::mma_commit(drainb);
    int dummy = 0;
    ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 8) {  // the allocating warp
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.status, ST_TIMEOUT);
  // no CTA leaves while another of its cluster may still write to its shared memory
  if (clustered) cluster_sync_all();
}

// Whole chain, one CTA per tile.
template <int BN, int NSL>
__global__ void __launch_bounds__(chain::THREADS, 1) tc_chain_kernel(const __grid_constant__ ChainParams P) {
  chain_body<BN, NSL, 1>(P);
}

// Whole chain with split-K over clusters of S CTAs (the cluster shape is part
// of the kernel).
template <int BN, int NSL, int S>
__global__ void __cluster_dims__(S, 1, 1) __launch_bounds__(chain::THREADS, 1)
    tc_chain_split_kernel(const __grid_constant__ ChainParams P) {
  chain_body<BN, NSL, S>(P);
}

template <int BN, int NSL, int S>
struct ChainKernel {
  static constexpr auto fn = tc_chain_split_kernel<BN, NSL, S>;
};
template <int BN, int NSL>
struct ChainKernel<BN, NSL, 1> {
  static constexpr auto fn = tc_chain_kernel<BN, NSL>;
};

// ---------------------------------------------------------------------------
// host side

template <int BN, int NSL, int S>
static cudaError_t chain_attr() {
  return cudaFuncSetAttribute(ChainKernel<BN, NSL, S>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              chain::Cfg<BN, NSL, S>::SMEM);
}

cudaError_t tc_chain_init(matpow_plan_s*) {
  cudaError_t e = chain_attr<64, 2, 1>();
  if (e == cudaSuccess) e = chain_attr<128, 2, 1>();
  if (e == cudaSuccess) e = chain_attr<64, 3, 1>();
  if (e == cudaSuccess) e = chain_attr<64, 2, 2>();
  if (e == cudaSuccess) e = chain_attr<64, 2, 4>();
  if (e == cudaSuccess) e = chain_attr<64, 3, 2>();
  return e;
}

// Cooperative launch of G CTAs (in clusters of S: the split kernels carry
// their cluster shape).
template <int BN, int NSL, int S>
static cudaError_t chain_launch(ChainParams* P, int G, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(chain::THREADS);
  cfg.dynamicSmemBytes = chain::Cfg<BN, NSL, S>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ChainKernel<BN, NSL, S>::fn, *P);
}

// Clusters of S co-resident with one CTA per SM (0 if the query fails).
template <int BN, int NSL, int S>
static int chain_max_clusters() {
  static int cached = -1;
  if (cached >= 0) return cached;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S * 64);
  cfg.blockDim = dim3(chain::THREADS);
  cfg.dynamicSmemBytes = chain::Cfg<BN, NSL, S>::SMEM;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, ChainKernel<BN, NSL, S>::fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached = n;
  return n;
}

// The level at which each power's chain starts.  A power's products are
// sequential, but the powers of a launch are independent, so a chain shorter
// than the longest may start later.  A level lasts about as long as its
// deepest run of k-blocks per CTA, ceil(KB / f), where f is the split-K its
// tile count allows (the largest f <= smax with f x tiles <= the SMs); the
// powers are placed, longest first, at the start that minimises the sum of
// that depth over the levels (ties: the earliest start).  With smax = 1 every
// start is 0.
static void chain_place(const std::vector<LevelOps>* levels, const int* tpo, const int* kb, int nj, int nlevels,
                        int smax, int num_sms, int* start) {
  std::vector<int> order(nj);
  for (int j = 0; j < nj; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return levels[a].size() > levels[b].size(); });
  std::vector<int> tiles(nlevels, 0), deep(nlevels, 0);
  auto depth = [&](int T, int K) {
    if (T == 0) return 0;
    int f = smax;
    while (f > 1 && f * T > num_sms) f >>= 1;
    return (K + f - 1) / f;
  };
  for (int j : order) {
    const int len = (int)levels[j].size();
    int best = 0;
    long long best_cost = -1;
    for (int d = 0; d + len <= nlevels; ++d) {
      long long cost = 0;
      for (int L = 0; L < nlevels; ++L) {
        int T = tiles[L], K = deep[L];
        if (L >= d && L < d + len) {
          T += (int)levels[j][L - d].ops.size() * tpo[j];
          K = std::max(K, kb[j]);
        }
        cost += depth(T, K);
      }
      if (best_cost < 0 || cost < best_cost) {
        best_cost = cost;
        best = d;
      }
    }
    start[j] = best;
    for (int L = best; L < best + len; ++L) {
      tiles[L] += (int)levels[j][L - best].ops.size() * tpo[j];
      deep[L] = std::max(deep[L], kb[j]);
    }
  }
}

// Whole-chain launch of up to four independent powers (same tile width and
// slice count); *used stays false when the powers do not fit one cooperative
// wave (the caller then runs the level-by-level path).
matpow_status tc_chain_launch(matpow_plan_s* p, const ChainJob* jobs, int nj, cudaStream_t s, bool* used) {
  *used = false;
  const int fmt = plan_float_fmt(p);
  if (p->chain_mode == 0 || p->naive || !fmt_exact(fmt) || nj < 1 || nj > CHAIN_MAXP) return MATPOW_OK;
  const int nsl = fmt_slices(fmt);
  int maxN = 0, minKB = 1 << 30;
  for (int j = 0; j < nj; ++j) {
    const int N = jobs[j].N;
    if (jobs[j].n < 2 || N <= p->tiny_max || N > 1024) return MATPOW_OK;
    // three accumulators per buffer fit TMEM only at 64-wide tiles
    if (nsl == 3 && N > 768) return MATPOW_OK;
    maxN = std::max(maxN, N);
    minKB = std::min(minKB, (N + chain::BK - 1) / chain::BK);
  }
  // the tile table (chain_mode 1 only: modes 0 and 2 are explicit choices):
  // the whole chain or the level path, its tile width and split-K
  const matpow_tile_rule* rule = p->chain_mode == 1 ? plan_tile_rule(p, maxN) : nullptr;
  if (rule && rule->chain == 0) return MATPOW_OK;
  int BN = maxN <= 768 ? 64 : 128;
  if (rule && (rule->bn == 64 || (rule->bn == 128 && nsl == 2))) BN = rule->bn;
  if (BN == 128 && nj > 1) return MATPOW_OK;  // one tile width per launch
  static thread_local ChainParams P;  // ~20 KB: kept off the stack
  memset(&P, 0, sizeof P);
  std::vector<LevelOps> levels[CHAIN_MAXP];
  int nlevels = 0;
  for (int j = 0; j < nj; ++j) {
    build_schedule(jobs[j].n, &levels[j]);
    if ((int)levels[j].size() > chain::MAX_LEVELS) return MATPOW_OK;
    nlevels = std::max(nlevels, (int)levels[j].size());
  }
  // where each power's chain starts (the split-K the launch may use decides
  // which placement is best; see below for the split itself)
  const int want_s = rule ? rule->split_k : -1;  // -1: the largest that fits
  const bool may_split = p->chain_mode == 1 && BN == 64 && want_s != 1;
  int tpo[CHAIN_MAXP], kbj[CHAIN_MAXP], start[CHAIN_MAXP];
  for (int j = 0; j < nj; ++j) {
    const int N = jobs[j].N;
    tpo[j] = ((N + chain::BM - 1) / chain::BM) * ((N + BN - 1) / BN);
    kbj[j] = (N + chain::BK - 1) / chain::BK;
  }
  chain_place(levels, tpo, kbj, nj, nlevels, may_split ? (want_s > 1 ? want_s : nsl == 3 ? 2 : 4) : 1, p->num_sms,
              start);
  // CTA groups per level: the powers' tiles one after another
  int G1 = 0;
  for (int L = 0; L < nlevels; ++L) {
    int acc = 0;
    for (int j = 0; j < nj; ++j) {
      P.lvl_begin[L][j] = (short)acc;
      const int Lj = L - start[j];
      if (Lj >= 0 && Lj < (int)levels[j].size()) acc += (int)levels[j][Lj].ops.size() * tpo[j];
    }
    P.lvl_begin[L][nj] = (short)acc;
    G1 = std::max(G1, acc);
  }
  if (G1 > p->num_sms) return MATPOW_OK;
  // split-K: clusters of S = 2 or 4 CTAs; each level then splits its tiles
  // over f | S CTAs, the largest f with f x (its tiles) <= G.  The grid is
  // the smallest multiple of S covering S x (the largest level), capped by
  // the SMs; at least one level must be able to split, or S = 1.
  int S = 1, G = G1;
  if (may_split) {
    int minT = 1 << 30;
    for (int L = 0; L < nlevels; ++L) minT = std::min(minT, (int)P.lvl_begin[L][nj]);
    const int smax = nsl == 3 ? 2 : 4;
    for (int c = smax; c >= 2; c /= 2) {
      if (c > minKB || (want_s > 1 && c != want_s)) continue;
      const int g = std::min(c * G1, p->num_sms / c * c);
      if (g < G1 || 2 * minT > g) continue;  // no level could split
      const int mc = nsl == 3 ? chain_max_clusters<64, 3, 2>()
                     : c == 4 ? chain_max_clusters<64, 2, 4>() : chain_max_clusters<64, 2, 2>();
      if (mc >= g / c) {
        S = c;
        G = g;
        break;
      }
    }
  }

  int prep = 0;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < nj; ++j) {
    const ChainJob& J = jobs[j];
    ChainProblem& Q = P.pr[j];
    const int N = J.N;
    const int ld = ld_for(N, fmt);
    const long long plane = plane_offset_elems(N, fmt);
    for (int b = 0; b < 4; ++b) {
      const char* base = (const char*)J.buf[b];
      Q.slices[b] = J.buf[b];
      Q.bexp[b] = (int*)((char*)J.buf[b] + fxb::bexp_offset(N, ld, nsl));
      for (int k = 0; k < nsl; ++k)
        if (!tc_encode_bf16_map(&Q.amap[b][k], base + k * plane * 2, N, ld, 64, chain::BM) ||
            !tc_encode_bf16_map(&Q.bmap[b][k], base + k * plane * 2, N, ld, 64, 64))
          return fail(p, MATPOW_ECUDA, "cuTensorMapEncodeTiled failed (N=%d)", N);
    }
    Q.plane = plane;
    Q.A = J.A;
    Q.out = J.out;
    Q.out_log2 = (long long*)J.log2;
    Q.scales = J.scales;
    Q.N = N;
    Q.ld = ld;
    Q.tiles_n = (N + BN - 1) / BN;
    Q.tiles_per_op = ((N + chain::BM - 1) / chain::BM) * Q.tiles_n;
    const std::vector<LevelOps>& lv = levels[j];
    for (size_t L = 0; L < lv.size(); ++L)
      for (size_t i = 0; i < lv[L].ops.size(); ++i) {
        const Op& o = lv[L].ops[i];
        chain::Op& c = Q.ops[2 * (L + start[j]) + i];
        c.xb = (signed char)o.xb;
        c.yb = (signed char)o.yb;
        c.cb = (signed char)o.cb;
        c.sx = (short)o.sx;
        c.sy = (short)o.sy;
        c.sc = (short)o.sc;
        c.last = (L + 1 == lv.size() && i + 1 == lv[L].ops.size()) ? 1 : 0;
      }
    P.prep_begin[j] = prep;
    const int nb = fxb::nblocks(N);
    prep += nb * nb;
    if (e == cudaSuccess) e = cudaMemsetAsync(J.scales, 0, sizeof(Scale) * (2 + matpow_gemm_count(J.n)), s);
  }
  P.prep_begin[nj] = prep;
  P.nprob = nj;
  P.nlevels = nlevels;
  P.status = p->status;
  P.gbar = p->gbar;
  if (e == cudaSuccess) e = cudaMemsetAsync(p->gbar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemsetAsync");
  double flop = 0;
  for (int j = 0; j < nj; ++j) flop += 2.0 * jobs[j].N * (double)jobs[j].N * jobs[j].N * matpow_gemm_count(jobs[j].n);
  cudaEvent_t ev;
  timed_begin(p, s, &ev);
  if (nsl == 3)
    e = S == 2 ? chain_launch<64, 3, 2>(&P, G, s) : chain_launch<64, 3, 1>(&P, G, s);
  else if (BN == 64)
    e = S == 4 ? chain_launch<64, 2, 4>(&P, G, s)
        : S == 2 ? chain_launch<64, 2, 2>(&P, G, s) : chain_launch<64, 2, 1>(&P, G, s);
  else
    e = chain_launch<128, 2, 1>(&P, G, s);
  if (e != cudaSuccess && S > 1) {
    // a cooperative launch with clusters was refused: run without split-K
    cudaGetLastError();
    e = nsl == 3 ? chain_launch<64, 3, 1>(&P, G1, s) : chain_launch<64, 2, 1>(&P, G1, s);
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cooperative launch of tc_chain_kernel");
  timed_end(p, s, ev, MATPOW_KERNEL_TC, flop);
  p->launches++;
  *used = true;
  return MATPOW_OK;
}

matpow_status tc_chain_run(matpow_plan_s* p, const float* dA, int N, uint64_t n, float* dOut,
                           int64_t* dLog2, cudaStream_t s, bool* used) {
  ChainJob j{dA, N, n, dOut, dLog2, {p->buf[0], p->buf[1], p->buf[2], p->buf[3]}, p->scales};
  return tc_chain_launch(p, &j, 1, s, used);
}

}  // namespace mp
