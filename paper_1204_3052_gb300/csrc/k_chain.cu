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
//   prep:   max|A| -> barrier -> exact split of A into integer slices -> barrier
//   level:  tile product (TMA -> tcgen05.mma exact slices -> TMEM chunks ->
//           float32 registers) -> max|C| -> barrier -> re-split the tile from
//           registers with the now-known power-of-two scale, store the slices
//           -> barrier
//   last:   the final product writes the user's float32 output directly.
//
// Compared with the level-by-level path this removes every kernel launch but
// one, the float32 round trip of each partial product, and the split passes.
// The arithmetic is identical to the exact-split level kernel: integer slices
// a1, a2 of the normalised operands, exact 256-deep partial sums in TMEM,
// round-to-nearest folding in float32 registers, lagged power-of-two scales.
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

namespace mp {

namespace chain {
constexpr int BM = 128, BK = 64, THREADS = 256, CHUNK_KB = 4;
constexpr int MAX_LEVELS = 64;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int SMEM_RING = 192 * 1024;
template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);
  static constexpr int STAGES = SMEM_RING / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 512;
  static constexpr int TMEM_COLS = 4 * BN;
};
struct Op {
  signed char xb, yb, cb, last;
  short sx, sy, sc, pad;
};
}  // namespace chain

struct ChainParams {
  CUtensorMap amap[4][2];  // buffer b as the A operand: slices a1, a2 (box 64 x 128)
  CUtensorMap bmap[4][2];  // buffer b as the B operand: slices a1, a2 (box 64 x 64)
  void* slices[4];         // slice a1 plane of buffer b (a2 at + plane elements)
  long long plane;
  const float* A;
  float* out;
  long long* out_log2;
  Scale* scales;
  unsigned* status;
  unsigned* gbar;
  int N, ld, nlevels, tiles_n, tiles_per_op;
  signed char lvl_nops[chain::MAX_LEVELS];
  chain::Op ops[2 * chain::MAX_LEVELS];
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
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

template <int BN>
__global__ void __launch_bounds__(chain::THREADS, 1)
    tc_chain_kernel(const __grid_constant__ ChainParams P) {
  using namespace chain;
  using C = Cfg<BN>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  // full[S], empty[S], accfull[2], accempty[2], drain
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* red = (float*)(tmem_slot + 4);  // 8 floats
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drainb = ptx::smem_u32(bars + 2 * STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = P.N, ld = P.ld;
  const int KB = (N + BK - 1) / BK;
  const int NCH = (KB + CHUNK_KB - 1) / CHUNK_KB;
  const unsigned G = gridDim.x;
  unsigned bar_no = 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, 4);
    }
    ptx::mbar_init(drainb, 1);
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

  // ---- prep: max|A|, then the exact split of A into buffer 0
  {
    const size_t total = (size_t)N * N;
    float m = 0.f;
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)THREADS + threadIdx.x; i < total; i += (size_t)G * THREADS) {
      const float v = P.A[i];
      bad |= !isfinite(v);
      m = fmaxf(m, fabsf(v));
    }
    m = warp_max(m);
    if (lane == 0) red[warp] = m;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(P.status, ST_BADINPUT);
    if (threadIdx.x == 0) {
      float mm = red[0];
      for (int w = 1; w < THREADS / 32; ++w) mm = fmaxf(mm, red[w]);
      if (mm > 0.f) atomicMax(&P.scales[1].maxbits, __float_as_uint(mm));
    }
  }
  grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag);
  if (!*abort_flag) {
    const int s = scale_exp_from_bits(__ldcg(&P.scales[1].maxbits));
    __nv_bfloat16* a1 = (__nv_bfloat16*)P.slices[0];
    __nv_bfloat16* a2 = a1 + P.plane;
    const size_t total = (size_t)N * ld;
    for (size_t i = blockIdx.x * (size_t)THREADS + threadIdx.x; i < total; i += (size_t)G * THREADS) {
      const size_t r = i / ld;
      const int c = (int)(i - r * ld);
      const float u = c < N ? mul_pow2(P.A[r * N + c], 8 - s) : 0.f;
      const float h = rintf(u);
      a1[i] = __float2bfloat16_rn(h);
      a2[i] = __float2bfloat16_rn(rintf((u - h) * 256.f));
    }
    fence_proxy_async_global();
  }
  grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag);

  int kb_base = 0, ch_base = 0;  // ring and accumulator-buffer counters (per CTA)
  float T[BN];
  for (int L = 0; L < P.nlevels && !*abort_flag; ++L) {
    const int nops = P.lvl_nops[L];
    const int t_all = blockIdx.x;
    const bool has = t_all < nops * P.tiles_per_op;
    const int oi = has ? t_all / P.tiles_per_op : 0;
    const int t = has ? t_all - oi * P.tiles_per_op : 0;
    const chain::Op op = P.ops[2 * L + oi];
    const int tm = t / P.tiles_n, tn = t - (t / P.tiles_n) * P.tiles_n;
    const int m0 = tm * BM, n0 = tn * BN;
    const int q = warp - 4;
    const int row = m0 + 32 * q + lane;

    if (has) {
      if (warp == 0) {
        if (lane == 0) {
          const CUtensorMap* am1 = &P.amap[op.xb][0];
          const CUtensorMap* am2 = &P.amap[op.xb][1];
          const CUtensorMap* bm1 = &P.bmap[op.yb][0];
          const CUtensorMap* bm2 = &P.bmap[op.yb][1];
          for (int kb = 0; kb < KB; ++kb) {
            const int g = kb_base + kb;
            const int s = g % STAGES;
            const uint32_t ph = (g / STAGES) & 1;
            if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            const uint32_t fb = full0 + 8 * s;
            ptx::mbar_expect_tx(fb, C::STAGE_BYTES);
            const uint32_t base = ptx::smem_u32(smem + s * C::STAGE_BYTES);
            const int kx = kb * BK;
            ptx::tma_load_2d(base, am1, kx, m0, fb);
            ptx::tma_load_2d(base + C::A_BYTES, am2, kx, m0, fb);
            const uint32_t bbase = base + 2 * C::A_BYTES;
#pragma unroll
            for (int c = 0; c < BN / 64; ++c) {
              ptx::tma_load_2d(bbase + c * 8192, bm1, n0 + 64 * c, kx, fb);
              ptx::tma_load_2d(bbase + C::B_BYTES + c * 8192, bm2, n0 + 64 * c, kx, fb);
            }
          }
        }
      } else if (warp == 1) {
        if (lane == 0) {
          constexpr uint32_t idesc = idesc_bf16(BM, BN);
          for (int kb = 0; kb < KB; ++kb) {
            const int g = kb_base + kb;
            const int ch = ch_base + kb / CHUNK_KB;
            const int buf = ch & 1;
            const bool first = (kb % CHUNK_KB) == 0;
            const bool last = (kb % CHUNK_KB) == CHUNK_KB - 1 || kb == KB - 1;
            const uint32_t t_main = tmem + (uint32_t)(buf * 2 * BN);
            const uint32_t t_cross = t_main + BN;
            if (first && !ptx::mbar_wait(accempty0 + 8 * buf, ((ch >> 1) & 1) ^ 1, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            const int s = g % STAGES;
            if (!ptx::mbar_wait(full0 + 8 * s, (g / STAGES) & 1, abort_flag, WAIT_NS)) {
              *abort_flag = 1;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a1 = ptx::smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t a2 = a1 + C::A_BYTES;
            const uint32_t b1 = a1 + 2 * C::A_BYTES;
            const uint32_t b2 = b1 + C::B_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t ad1 = ptx::smem_desc(a1 + 32 * k, 16, 1024);
              const uint64_t ad2 = ptx::smem_desc(a2 + 32 * k, 16, 1024);
              const uint64_t bd1 = ptx::smem_desc(b1 + 2048 * k, 8192, 1024);
              const uint64_t bd2 = ptx::smem_desc(b2 + 2048 * k, 8192, 1024);
              const uint32_t acc = (first && k == 0) ? 0u : 1u;
              ptx::mma_f16(t_main, ad1, bd1, idesc, acc);
              ptx::mma_f16(t_cross, ad1, bd2, idesc, acc);
              ptx::mma_f16(t_cross, ad2, bd1, idesc, 1);
            }
            ptx::mma_commit(empty0 + 8 * s);
            if (last) ptx::mma_commit(accfull0 + 8 * buf);
          }
        }
      } else if (warp >= 4) {
#pragma unroll
        for (int j = 0; j < BN; ++j) T[j] = 0.f;
        for (int cc = 0; cc < NCH; ++cc) {
          const int ch = ch_base + cc;
          const int buf = ch & 1;
          int dummy = 0;
          if (!ptx::mbar_wait(accfull0 + 8 * buf, (ch >> 1) & 1, &dummy, 2 * WAIT_NS)) {
            *abort_flag = 1;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 2 * BN);
#pragma unroll
          for (int c = 0; c < BN / 32; ++c) {
            uint32_t rm[32], rc[32];
            ptx::tmem_ld_32x32b_x32(tq + 32 * c, rm);
            ptx::tmem_ld_32x32b_x32(tq + BN + 32 * c, rc);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j)
              T[32 * c + j] += __uint_as_float(rm[j]) + __uint_as_float(rc[j]) * 0.00390625f;
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(accempty0 + 8 * buf);
        }
        // stored value of the normalised-operand product
#pragma unroll
        for (int j = 0; j < BN; ++j) T[j] *= 1.52587890625e-05f;  // 2^-16
        // scale slots are written by other CTAs: read them from L2, not L1
        const int sx = scale_exp_from_bits(__ldcg(&P.scales[op.sx].maxbits));
        const int sy = scale_exp_from_bits(__ldcg(&P.scales[op.sy].maxbits));
        const long long Ec = __ldcg(&P.scales[op.sx].E) + __ldcg(&P.scales[op.sy].E) + sx + sy;
        if (op.last) {
          if (t == 0 && q == 0 && lane == 0 && P.out_log2) *P.out_log2 = Ec;
          if (row < N) {
            float* O = P.out + (size_t)row * N;
#pragma unroll
            for (int j = 0; j < BN; ++j) {
              const int c = n0 + j;
              if (c < N) O[c] = P.out_log2 ? T[j] : final_value(T[j], Ec, P.status);
            }
          }
        } else {
          if (t == 0 && q == 0 && lane == 0) P.scales[op.sc].E = Ec;
          float mx = 0.f;
          if (row < N) {
#pragma unroll
            for (int j = 0; j < BN; ++j)
              if (n0 + j < N) mx = fmaxf(mx, fabsf(T[j]));
          }
          mx = warp_max(mx);
          if (lane == 0 && mx > 0.f) atomicMax(&P.scales[op.sc].maxbits, __float_as_uint(mx));
        }
      }
    }
    if (has) {  // ring and accumulator counters advance only with work done
      kb_base += KB;
      ch_base += NCH;
    }
    if (P.ops[2 * L + nops - 1].last) break;  // the final product has been written
    // all maxima of this level are in
    if (!grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag)) break;
    if (has && warp >= 4 && !op.last) {
      const int s = scale_exp_from_bits(__ldcg(&P.scales[op.sc].maxbits));
      if (row < N) {
        __nv_bfloat16* a1 = (__nv_bfloat16*)P.slices[op.cb] + (size_t)row * ld + n0;
        __nv_bfloat16* a2 = a1 + P.plane;
        if (n0 + BN <= N) {
#pragma unroll
          for (int g8 = 0; g8 < BN / 8; ++g8) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float u0 = mul_pow2(T[8 * g8 + 2 * h], 8 - s);
              const float u1 = mul_pow2(T[8 * g8 + 2 * h + 1], 8 - s);
              const float h0 = rintf(u0), h1 = rintf(u1);
              __nv_bfloat162 hi = __floats2bfloat162_rn(h0, h1);
              __nv_bfloat162 lo = __floats2bfloat162_rn(rintf((u0 - h0) * 256.f), rintf((u1 - h1) * 256.f));
              hw[h] = *reinterpret_cast<uint32_t*>(&hi);
              lw[h] = *reinterpret_cast<uint32_t*>(&lo);
            }
            *reinterpret_cast<uint4*>(a1 + 8 * g8) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(a2 + 8 * g8) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < BN; ++j) {
            if (n0 + j < N) {
              const float u = mul_pow2(T[j], 8 - s);
              const float h = rintf(u);
              a1[j] = __float2bfloat16_rn(h);
              a2[j] = __float2bfloat16_rn(rintf((u - h) * 256.f));
            }
          }
        }
      }
      fence_proxy_async_global();
    }
    // the slices of this level are visible to every CTA's TMA
    if (!grid_sync(P.gbar, ++bar_no * G, P.status, abort_flag)) break;
    fence_proxy_async_global();
  }

  // ---- teardown: no copy or MMA of this CTA may still be in flight
  if (warp == 0 && lane == 0) {
    for (int g = kb_base - STAGES < 0 ? 0 : kb_base - STAGES; g < kb_base; ++g) {
      int dummy = 0;
      ptx::mbar_wait(full0 + 8 * (g % STAGES), (g / STAGES) & 1, &dummy, WAIT_NS);
    }
  }
  if (warp == 1 && lane == 0) {
    ptx::mma_commit(drainb);
    int dummy = 0;
    ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(P.status, ST_TIMEOUT);
}

// ---------------------------------------------------------------------------
// host side

cudaError_t tc_chain_init(matpow_plan_s*) {
  cudaError_t e = cudaFuncSetAttribute(tc_chain_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       chain::Cfg<64>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_chain_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              chain::Cfg<128>::SMEM);
}

matpow_status tc_chain_run(matpow_plan_s* p, const float* dA, int N, uint64_t n, float* dOut,
                           int64_t* dLog2, cudaStream_t s, bool* used) {
  *used = false;
  if (!p->use_chain || plan_float_fmt(p) != FMT_FX2 || n < 2 || N <= p->tiny_max || N > 1024)
    return MATPOW_OK;
  const int BN = N <= 768 ? 64 : 128;
  std::vector<LevelOps> levels;
  build_schedule(n, &levels);
  if ((int)levels.size() > chain::MAX_LEVELS) return MATPOW_OK;
  const int tiles_n = (N + BN - 1) / BN;
  const int tiles_per_op = ((N + chain::BM - 1) / chain::BM) * tiles_n;
  int maxops = 1;
  for (auto& lv : levels) maxops = std::max(maxops, (int)lv.ops.size());
  const int G = maxops * tiles_per_op;
  if (G > p->num_sms) return MATPOW_OK;

  static thread_local ChainParams P;  // ~4 KB: kept off the stack
  memset(&P, 0, sizeof P);
  const int fmt = FMT_FX2;
  const int ld = ld_for(N, fmt);
  const long long plane = plane_offset_elems(N, fmt);
  for (int b = 0; b < 4; ++b) {
    const char* base = (const char*)p->buf[b];
    P.slices[b] = p->buf[b];
    if (!tc_encode_bf16_map(&P.amap[b][0], base, N, ld, 64, chain::BM) ||
        !tc_encode_bf16_map(&P.amap[b][1], base + plane * 2, N, ld, 64, chain::BM) ||
        !tc_encode_bf16_map(&P.bmap[b][0], base, N, ld, 64, 64) ||
        !tc_encode_bf16_map(&P.bmap[b][1], base + plane * 2, N, ld, 64, 64))
      return fail(p, MATPOW_ECUDA, "cuTensorMapEncodeTiled failed (N=%d)", N);
  }
  P.plane = plane;
  P.A = dA;
  P.out = dOut;
  P.out_log2 = (long long*)dLog2;
  P.scales = p->scales;
  P.status = p->status;
  P.gbar = p->gbar;
  P.N = N;
  P.ld = ld;
  P.nlevels = (int)levels.size();
  P.tiles_n = tiles_n;
  P.tiles_per_op = tiles_per_op;
  for (size_t L = 0; L < levels.size(); ++L) {
    P.lvl_nops[L] = (signed char)levels[L].ops.size();
    for (size_t i = 0; i < levels[L].ops.size(); ++i) {
      const Op& o = levels[L].ops[i];
      chain::Op& c = P.ops[2 * L + i];
      c.xb = (signed char)o.xb;
      c.yb = (signed char)o.yb;
      c.cb = (signed char)o.cb;
      c.sx = (short)o.sx;
      c.sy = (short)o.sy;
      c.sc = (short)o.sc;
      c.last = (L + 1 == levels.size() && i + 1 == levels[L].ops.size()) ? 1 : 0;
    }
  }
  const int nslots = 2 + matpow_gemm_count(n);
  cudaError_t e = cudaMemsetAsync(p->scales, 0, sizeof(Scale) * nslots, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->gbar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemsetAsync");
  void* args[] = {&P};
  cudaEvent_t ev;
  timed_begin(p, s, &ev);
  if (BN == 64)
    e = cudaLaunchCooperativeKernel((const void*)tc_chain_kernel<64>, dim3(G), dim3(chain::THREADS),
                                    args, chain::Cfg<64>::SMEM, s);
  else
    e = cudaLaunchCooperativeKernel((const void*)tc_chain_kernel<128>, dim3(G), dim3(chain::THREADS),
                                    args, chain::Cfg<128>::SMEM, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaLaunchCooperativeKernel(tc_chain_kernel)");
  timed_end(p, s, ev, MATPOW_KERNEL_TC, 2.0 * N * (double)N * N * matpow_gemm_count(n));
  p->launches++;
  *used = true;
  return MATPOW_OK;
}

}  // namespace mp
