// Tensor-core products C = X * Y on sm_103a: TMA -> shared memory ->
// tcgen05.mma (kind::f16, bfloat16 operands) -> float32 accumulator in TMEM ->
// epilogue warps (tcgen05.ld) that apply the lagged power-of-two scale and
// write the stored result.
//
// The product is the matrix product of arXiv 1204.3052 Sec. 4.1, run inside
// the square-and-multiply chain of Sec. 4.3.  The paper's tiling through
// local memory (Sec. 4.3.2, 4.3.7) becomes TMA boxes in a multi-stage
// shared-memory ring; its vector loads (Sec. 4.3.5) become 128-byte swizzled
// TMA rows feeding the tensor cores; its barriers (Sec. 4.3.6) become
// mbarriers between the TMA, MMA and epilogue warps.
//
// Precisions:
//   PL = 1 (BF16):   one plane, one MMA per 16-deep k-step.
//   PL = 2 (BF16X3): x = hi + lo planes; hi*hi + hi*lo + lo*hi MMAs into one
//                    float32 accumulator (the lo*lo term, ~2^-16 relative,
//                    is dropped).
// Layout: X is the A operand (K-major rows, 64x128 boxes, 128-byte swizzle),
// row-major Y is the B operand in MN-major form (64x64 boxes per 64-column
// chunk, 128-byte swizzle), so no operand is ever transposed in memory.
//
// CTA: 256 threads.  Warp 0 issues TMA, warp 1 issues MMAs (one thread),
// warp 2 owns the TMEM allocation, warps 4-7 run the epilogue (each reads the
// 32 TMEM lanes = 32 rows of its quadrant).  Every wait is bounded in time; a
// CTA that gives up drains its copies and MMAs, frees TMEM, and reports
// MATPOW_ETIMEDOUT through the plan's status word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"
#include "plan.h"
#include "tc_ptx.cuh"
#include "tc_common.cuh"
#include "fxb.cuh"

namespace mp {

namespace tc {
constexpr int BM = 128, BK = 64, THREADS = 256;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr int SMEM_RING = 192 * 1024;
template <int BN, int PL>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = PL * (A_BYTES + B_BYTES);
  static constexpr int STAGES = SMEM_RING / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};
}  // namespace tc


template <int BN, int PL>
__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ TcPairParams P, Scale* scales, unsigned* status) {
  using namespace tc;
  using C = Cfg<BN, PL>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accb = ptx::smem_u32(bars + 2 * STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = blockIdx.x;
  const int which = (P.count > 1 && t >= P.tiles0) ? 1 : 0;
  if (which) t -= P.tiles0;
  const TcProblem& pr = P.p[which];
  const GemmDesc& d = pr.d;
  int tm, tn;
  tile_raster(t, (d.N + 127) / 128, d.tiles_n, &tm, &tn);  // 128-row tiles
  const int m0 = tm * BM, n0 = tn * BN;
  const int N = d.N;
  const int KB = (N + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    ptx::mbar_init(accb, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), BN);
    ptx::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    ptx::prefetch_tmap(&pr.ax[0]);
    ptx::prefetch_tmap(&pr.by[0]);
    if (PL == 2) {
      ptx::prefetch_tmap(&pr.ax[1]);
      ptx::prefetch_tmap(&pr.by[1]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = full0 + 8 * s;
        ptx::mbar_expect_tx(fb, C::STAGE_BYTES);
        const uint32_t base = ptx::smem_u32(smem + s * C::STAGE_BYTES);
        const int kx = kb * BK;
        ptx::tma_load_2d(base, &pr.ax[0], kx, m0, fb);
        if (PL == 2) ptx::tma_load_2d(base + C::A_BYTES, &pr.ax[1], kx, m0, fb);
        const uint32_t bbase = base + PL * C::A_BYTES;
#pragma unroll
        for (int c = 0; c < BN / 64; ++c) {
          ptx::tma_load_2d(bbase + c * 8192, &pr.by[0], n0 + 64 * c, kx, fb);
          if (PL == 2) ptx::tma_load_2d(bbase + C::B_BYTES + c * 8192, &pr.by[1], n0 + 64 * c, kx, fb);
        }
        ++issued;
      }
      // drain: every issued stage's copies have landed before the CTA can exit
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
        int dummy = 0;
        ptx::mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, &dummy, WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!ptx::mbar_wait(full0 + 8 * s, ph, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t a_hi = ptx::smem_u32(smem + s * C::STAGE_BYTES);
        const uint32_t a_lo = a_hi + C::A_BYTES;
        const uint32_t b_hi = a_hi + PL * C::A_BYTES;
        const uint32_t b_lo = b_hi + C::B_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t ad = ptx::smem_desc(a_hi + 32 * k, 16, 1024);
          const uint64_t bd = ptx::smem_desc(b_hi + 2048 * k, 8192, 1024);
          ptx::mma_f16(tmem, ad, bd, idesc, (kb | k) != 0);
          if (PL == 2) {
            const uint64_t bdl = ptx::smem_desc(b_lo + 2048 * k, 8192, 1024);
            const uint64_t adl = ptx::smem_desc(a_lo + 32 * k, 16, 1024);
            ptx::mma_f16(tmem, ad, bdl, idesc, 1);
            ptx::mma_f16(tmem, adl, bd, idesc, 1);
          }
        }
        ptx::mma_commit(empty0 + 8 * s);  // frees the stage when these MMAs are done
      }
      ptx::mma_commit(accb);  // accumulator complete (or drained, after an abort)
    }
  } else if (warp >= 4) {
    // ---- epilogue
    int dummy = 0;
    const bool ok = ptx::mbar_wait(accb, 0, &dummy, 2 * WAIT_NS);
    if (!ok) *abort_flag = 1;
    ptx::tc_fence_after();
    if (ok && !*abort_flag) {
      const int q = warp - 4;
      const int row = m0 + 32 * q + lane;
      const int sx = scale_exp_from_bits(scales[d.sx].maxbits);
      const int sy = scale_exp_from_bits(scales[d.sy].maxbits);
      const int sh = -(sx + sy);
      const long long Ec = scales[d.sx].E + scales[d.sy].E + sx + sy;
      if (t == 0 && q == 0 && lane == 0) {
        if (d.mode == OUT_INTERNAL) scales[d.sc].E = Ec;
        if (d.mode == OUT_USER_MANT && d.out_log2) *d.out_log2 = Ec;
      }
      float mx = 0.f;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * q) << 16) + 32 * c, r);
        ptx::tmem_ld_wait();
        const int col0 = n0 + 32 * c;
        if (row >= N || col0 >= N) continue;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = mul_pow2(__uint_as_float(r[j]), sh);
        if (d.mode == OUT_INTERNAL) {
          __nv_bfloat16* C0 = (__nv_bfloat16*)d.C + (size_t)row * d.ld + col0;
          __nv_bfloat16* C1 = C0 + d.plane;
          if (col0 + 32 <= N) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const float a = v[8 * g + 2 * h], b = v[8 * g + 2 * h + 1];
                __nv_bfloat162 hi = __floats2bfloat162_rn(a, b);
                hw[h] = *reinterpret_cast<uint32_t*>(&hi);
                if (PL == 2) {
                  __nv_bfloat162 lo = __floats2bfloat162_rn(a - __low2float(hi), b - __high2float(hi));
                  lw[h] = *reinterpret_cast<uint32_t*>(&lo);
                }
              }
              *reinterpret_cast<uint4*>(C0 + 8 * g) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              if (PL == 2) *reinterpret_cast<uint4*>(C1 + 8 * g) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) mx = fmaxf(mx, fabsf(v[j]));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (col0 + j < N) {
                __nv_bfloat16 hi = __float2bfloat16_rn(v[j]);
                C0[j] = hi;
                if (PL == 2) C1[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi));
                mx = fmaxf(mx, fabsf(v[j]));
              }
            }
          }
        } else {
          float* O = (float*)d.out + (size_t)row * N + col0;
          const bool mant = d.mode == OUT_USER_MANT;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col0 + j < N) O[j] = mant ? v[j] : final_value(v[j], Ec, status);
        }
      }
      if (d.mode == OUT_INTERNAL) {
        mx = warp_max(mx);
        if (lane == 0 && mx > 0.f) atomicMax(&scales[d.sc].maxbits, __float_as_uint(mx));
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, BN);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Exact block-scaled split products (BF16X3 default; arithmetic in fxb.cuh).
// Same warp roles as above, plus warp 3, which stages the tile's block
// exponents in shared memory.  The MMA accumulates each 64-deep k-block into
// one of two TMEM buffers (main, cross); the epilogue warps fold finished
// k-blocks into float32 registers with the block factors while the MMA fills
// the other buffer, then re-split the tile by 64 x 64 blocks straight into the
// next product's operand planes.

namespace fx {
template <int BN, int NSL>
struct Cfg {
  // epilogue warps: 4 lane quadrants x CS column slices of WC columns each
  static constexpr int CS = BN / 64;
  static constexpr int WC = BN / CS;
  static constexpr int EW = 4 * CS;
  static constexpr int THREADS = 128 + 32 * EW;
  static constexpr int NG = BN / fxb::BLK;
  static constexpr int A_BYTES = tc::BM * tc::BK * 2;
  static constexpr int B_BYTES = BN * tc::BK * 2;
  static constexpr int STAGE_BYTES = NSL * (A_BYTES + B_BYTES);
  static constexpr int RING = NSL == 3 ? 216 * 1024 : tc::SMEM_RING;
  static constexpr int STAGES = RING / STAGE_BYTES;
  static constexpr int EXP_BYTES = (2 + NG) * fxb::MAX_KB * 4;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256 + EXP_BYTES + 64;
  static constexpr int ACC = NSL;                 // accumulators per k-block buffer
  static constexpr int TMEM_USED = 2 * ACC * BN;  // 2 buffers
  static constexpr int TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
  static_assert(TMEM_USED <= 512, "TMEM");
};
}  // namespace fx

// One CTA = one output tile t of product d.  ax[k] / by[k]: slice k of X as
// the A operand / of Y as the B operand; cx[k]: slice k of C as TMA store
// target (param or global memory).  NSL = 2 (BF16X3) or 3 (BF16X6).
template <int BN, int NSL>
__device__ __forceinline__ void fxb_cta(const GemmDesc& d, int t, const CUtensorMap* const (&ax)[NSL],
                                        const CUtensorMap* const (&by)[NSL],
                                        const CUtensorMap* const (&cx)[NSL], Scale* scales,
                                        unsigned* status) {
  using namespace tc;
  using C = fx::Cfg<BN, NSL>;
  constexpr int EW = C::EW, WC = C::WC;
  constexpr int STAGES = C::STAGES;
  constexpr int NG = C::NG;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  // full[S], empty[S], accfull[2], accempty[2], drain
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  volatile int* epi_ok = (volatile int*)(tmem_slot + 2);
  int* eA = (int*)(smem + STAGES * C::STAGE_BYTES + 256);
  int* eB = eA + 2 * fxb::MAX_KB;
  float* red = (float*)(eB + NG * fxb::MAX_KB);
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drainb = ptx::smem_u32(bars + 2 * STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm, tn;
  tile_raster(t, (d.N + 127) / 128, d.tiles_n, &tm, &tn);  // 128-row tiles
  const int m0 = tm * BM, n0 = tn * BN;
  const int N = d.N;
  const int KB = (N + BK - 1) / BK;
  const size_t boff = fxb::bexp_offset(N, d.ld, NSL);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, EW);  // one arrival per epilogue warp
    }
    ptx::mbar_init(drainb, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), C::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
#pragma unroll
    for (int k = 0; k < NSL; ++k) {
      ptx::prefetch_tmap(ax[k]);
      ptx::prefetch_tmap(by[k]);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!ptx::mbar_wait(empty0 + 8 * s, ph ^ 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t fb = full0 + 8 * s;
        ptx::mbar_expect_tx(fb, C::STAGE_BYTES);
        const uint32_t base = ptx::smem_u32(smem + s * C::STAGE_BYTES);
        const int kx = fxb::rot_kb(kb, KB, fxb::tile_rot(m0, n0, KB)) * BK;
#pragma unroll
        for (int k = 0; k < NSL; ++k) ptx::tma_load_2d(base + k * C::A_BYTES, ax[k], kx, m0, fb);
        const uint32_t bbase = base + NSL * C::A_BYTES;
#pragma unroll
        for (int c = 0; c < BN / 64; ++c)
#pragma unroll
          for (int k = 0; k < NSL; ++k)
            ptx::tma_load_2d(bbase + k * C::B_BYTES + c * 8192, by[k], n0 + 64 * c, kx, fb);
        ++issued;
      }
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb) {
        int dummy = 0;
        ptx::mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1, &dummy, WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < KB; ++kb) {
        const int buf = kb & 1;
        const uint32_t t0 = tmem + (uint32_t)(buf * C::ACC * BN);
        if (!ptx::mbar_wait(accempty0 + 8 * buf, ((kb >> 1) & 1) ^ 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
          break;
        }
        const int s = kb % STAGES;
        if (!ptx::mbar_wait(full0 + 8 * s, (kb / STAGES) & 1, abort_flag, WAIT_NS)) {
          *abort_flag = 1;
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
      ptx::mma_commit(drainb);
      int dummy = 0;
      ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
    }
  } else if (warp == 3) {
    fxb::load_tile_exponents<BN>((const int*)((const char*)d.X + boff),
                                 (const int*)((const char*)d.Y + boff), N, m0, n0, KB, eA, eB, lane);
    __syncwarp();
    asm volatile("bar.arrive 2, %0;" ::"n"(32 + 32 * EW) : "memory");
  } else if (warp >= 4) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (= tile rows) and one slice
    // of WC columns
    const int e = warp - 4;
    const int q = warp & 3;
    const int cs = e >> 2;
    const int h = q >> 1;
    const int row = m0 + 32 * q + lane;
    const int nw = n0 + cs * WC;
    const int sx = scale_exp_from_bits(scales[d.sx].maxbits);
    const int sy = scale_exp_from_bits(scales[d.sy].maxbits);
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
      fxb::fold<WC, NSL>(T, tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * C::ACC * BN + cs * WC),
                         fac, BN);
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(accempty0 + 8 * buf);
    }
    // one verdict for all epilogue warps (they share named barriers below)
    fxb::epi_bar<32 * EW>();
    if (e == 0 && lane == 0) *epi_ok = ok && !*abort_flag;
    fxb::epi_bar<32 * EW>();
    ok = *epi_ok != 0;
    const long long Ec = scales[d.sx].E + scales[d.sy].E + sx + sy;
    if (d.mode == OUT_INTERNAL) {
      if (t == 0 && e == 0 && lane == 0) scales[d.sc].E = Ec;
      if (ok)  // every epilogue warp reaches the named barriers inside; the ring is idle
        fxb::store_slices_tma<WC, 32 * EW, NSL>(T, 32 * q + lane, m0, nw, q, lane, N, cs * (WC / 64),
                                                BN / 64, smem, cx, (int*)((char*)d.C + boff),
                                                &scales[d.sc].maxbits, red, e == 0 && lane == 0, n0);
    } else if (ok) {
      if (t == 0 && e == 0 && lane == 0 && d.mode == OUT_USER_MANT && d.out_log2) *d.out_log2 = Ec;
      if (row < N) {
        float* O = (float*)d.out + (size_t)row * N;
        const bool mant = d.mode == OUT_USER_MANT;
        store_row_f32<WC>(T, O, nw, N, mant, Ec, status, d.out);
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
}

template <int BN, int NSL>
__global__ void __launch_bounds__(fx::Cfg<BN, NSL>::THREADS, 1)
    tc_fxb_kernel(const __grid_constant__ TcPairParams P, Scale* scales, unsigned* status) {
  int t = blockIdx.x;
  const int which = (P.count > 1 && t >= P.tiles0) ? 1 : 0;
  if (which) t -= P.tiles0;
  const TcProblem& pr = P.p[which];
  const CUtensorMap* ax[NSL];
  const CUtensorMap* by[NSL];
  const CUtensorMap* cx[NSL];
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    ax[k] = &pr.ax[k];
    by[k] = &pr.by[k];
    cx[k] = &pr.cx[k];
  }
  fxb_cta<BN, NSL>(pr.d, t, ax, by, cx, scales, status);
}

// Grouped launch: products from a device table (any number of matrices),
// TMA descriptors from a device table: 2 NSL per stored buffer (A-role slices
// 0..NSL-1, then B-role slices), at index map_x / map_y / map_c.
template <int BN, int NSL>
__global__ void __launch_bounds__(fx::Cfg<BN, NSL>::THREADS, 1)
    tc_fxb_group_kernel(const GemmDesc* __restrict__ descs, int count,
                        const CUtensorMap* __restrict__ maps, Scale* scales, unsigned* status) {
  const int tb = blockIdx.x;
  int lo = 0, hi = count - 1;  // last desc with tile_begin <= tb
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile_begin <= tb) lo = mid; else hi = mid - 1;
  }
  const GemmDesc d = descs[lo];
  const CUtensorMap* ax[NSL];
  const CUtensorMap* by[NSL];
  const CUtensorMap* cx[NSL];
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    ax[k] = &maps[d.map_x + k];
    by[k] = &maps[d.map_y + NSL + k];
    cx[k] = &maps[d.map_c + k];
  }
  fxb_cta<BN, NSL>(d, tb - d.tile_begin, ax, by, cx, scales, status);
}

// A (float32, leading dimension N) -> block-scaled stored format, one CTA per
// 64 x 64 block.
template <int NSL>
__global__ void __launch_bounds__(256) prep_fxb_kernel(const float* __restrict__ A, int N, int ld,
                                                       __nv_bfloat16* dst, long long plane,
                                                       int* bexp, unsigned* maxbits,
                                                       unsigned* status) {
  __shared__ float red[8];
  const int nb = fxb::nblocks(N);
  const int I = blockIdx.x / nb, J = blockIdx.x - (blockIdx.x / nb) * nb;
  fxb::prep_block<NSL>(A, N, ld, I, J, dst, plane, bexp, maxbits, status, red);
}

// ---------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

template <int BN, int PL>
static cudaError_t set_attr() {
  return cudaFuncSetAttribute(tc_gemm_kernel<BN, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc::Cfg<BN, PL>::SMEM);
}

cudaError_t tc_init(matpow_plan_s*) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return cudaErrorNotSupported;
  cudaError_t e;
  if ((e = set_attr<64, 1>()) != cudaSuccess) return e;
  if ((e = set_attr<128, 1>()) != cudaSuccess) return e;
  if ((e = set_attr<256, 1>()) != cudaSuccess) return e;
  if ((e = set_attr<64, 2>()) != cudaSuccess) return e;
  if ((e = set_attr<128, 2>()) != cudaSuccess) return e;
  if ((e = set_attr<256, 2>()) != cudaSuccess) return e;
#define MP_FXB_ATTR(K, BN, NSL)                                                                  \
  if ((e = cudaFuncSetAttribute(K<BN, NSL>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                fx::Cfg<BN, NSL>::SMEM)) != cudaSuccess)                          \
    return e;
  MP_FXB_ATTR(tc_fxb_kernel, 64, 2)
  MP_FXB_ATTR(tc_fxb_kernel, 128, 2)
  MP_FXB_ATTR(tc_fxb_kernel, 64, 3)
  MP_FXB_ATTR(tc_fxb_group_kernel, 64, 2)
  MP_FXB_ATTR(tc_fxb_group_kernel, 128, 2)
  MP_FXB_ATTR(tc_fxb_group_kernel, 64, 3)
#undef MP_FXB_ATTR
  if ((e = tc_pair_init()) != cudaSuccess) return e;
  return tc_persist_init();
}

void tc_free(matpow_plan_s*) {}

static int pick_bn(matpow_plan_s* p, int N) {
  const int fmt = plan_float_fmt(p);
  if (fmt == FMT_FX3) return 64;  // three accumulators x 2 buffers fit TMEM at 64 columns
  const bool fx2 = fmt == FMT_FX2;
  if (p->tile_override == 64 || p->tile_override == 128 || p->tile_override == 256) {
    if (fx2 && p->tile_override == 256) return 128;
    return p->tile_override;
  }
  const int tb = plan_tile_field(p, N, &matpow_tile_rule::bn);  // the tile table's width
  if (tb == 64 || tb == 128) return tb;
  return tc_group_bn(N) == 64 ? 64 : (N <= 3072 || fx2) ? 128 : 256;
}

matpow_status tc_fill_desc(matpow_plan_s* p, GemmDesc* d, int* ntiles) {
  if (fmt_exact(plan_float_fmt(p)) && d->N > fxb::MAX_KB * fxb::BLK)
    return fail(p, MATPOW_EUNSUPPORTED, "exact split: N=%d above %d", d->N, fxb::MAX_KB * fxb::BLK);
  d->bn = pick_bn(p, d->N);
  d->tiles_n = (d->N + d->bn - 1) / d->bn;
  *ntiles = ((d->N + tc::BM - 1) / tc::BM) * d->tiles_n;
  return MATPOW_OK;
}

bool tc_encode_bf16_map(CUtensorMap* m, const void* base, int N, int ld, int box_inner, int box_outer) {
  cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)N};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool fill_problem(TcProblem* tp, const GemmDesc& d, int NPL) {
  tp->d = d;
  const size_t ps = (size_t)d.plane * 2;  // bytes between planes
  for (int k = 0; k < 3; ++k) {
    const int kk = k < NPL ? k : NPL - 1;
    if (!tc_encode_bf16_map(&tp->ax[k], (const char*)d.X + kk * ps, d.N, d.ld, 64, tc::BM)) return false;
    if (!tc_encode_bf16_map(&tp->by[k], (const char*)d.Y + kk * ps, d.N, d.ld, 64, 64)) return false;
    if (d.C) {  // TMA store targets of the output planes
      if (!tc_encode_bf16_map(&tp->cx[k], (const char*)d.C + kk * ps, d.N, d.ld, 64, tc::BM))
        return false;
    } else {
      tp->cx[k] = tp->ax[k];
    }
  }
  return true;
}

template <int BN, int PL>
static cudaError_t launch(const TcPairParams& P, int grid, Scale* scales, unsigned* status,
                          cudaStream_t s) {
  tc_gemm_kernel<BN, PL><<<grid, tc::THREADS, tc::Cfg<BN, PL>::SMEM, s>>>(P, scales, status);
  return cudaGetLastError();
}

matpow_status tc_launch_pair(matpow_plan_s* p, const GemmPair& g, cudaStream_t s) {
  const int fmt = plan_float_fmt(p);
  const int PL = fmt == FMT_BF16 ? 1 : 2;
  static thread_local TcPairParams P;  // ~3 KB: kept off the stack
  memset(&P, 0, sizeof P);
  P.count = g.count;
  for (int i = 0; i < g.count; ++i)
    if (!fill_problem(&P.p[i], g.d[i], fmt == FMT_FX3 ? 3 : PL))
      return fail(p, MATPOW_ECUDA, "cuTensorMapEncodeTiled failed (N=%d)", g.d[i].N);
  P.tiles0 = g.count > 1 ? g.d[1].tile_begin : g.tiles_total;
  const int bn = g.d[0].bn;
  cudaError_t e;
  bool on_pairs = fmt == FMT_FX2 && bn == 128 && p->pair;
  for (int i = 0; i < g.count; ++i) on_pairs = on_pairs && g.d[i].N > 2048 && g.d[i].bn == 128;
  if (on_pairs) {
    // 256 x 128 tiles over CTA pairs (same arithmetic, bit-identical results)
    P.tiles0 = pair_tiles(g.d[0].N);
    const int total = P.tiles0 + (g.count > 1 ? pair_tiles(g.d[1].N) : 0);
    if (g.count == 1) P.tiles0 = total;
    e = launch_fxb_pair(P, total, p->scales, p->status, s);
  } else if (fmt == FMT_FX3) {
    tc_fxb_kernel<64, 3><<<g.tiles_total, fx::Cfg<64, 3>::THREADS, fx::Cfg<64, 3>::SMEM, s>>>(
        P, p->scales, p->status);
    e = cudaGetLastError();
  } else if (fmt == FMT_FX2) {
    if (bn == 64)
      tc_fxb_kernel<64, 2><<<g.tiles_total, fx::Cfg<64, 2>::THREADS, fx::Cfg<64, 2>::SMEM, s>>>(
          P, p->scales, p->status);
    else
      tc_fxb_kernel<128, 2><<<g.tiles_total, fx::Cfg<128, 2>::THREADS, fx::Cfg<128, 2>::SMEM, s>>>(
          P, p->scales, p->status);
    e = cudaGetLastError();
  } else if (PL == 2)
    e = bn == 64 ? launch<64, 2>(P, g.tiles_total, p->scales, p->status, s)
        : bn == 128 ? launch<128, 2>(P, g.tiles_total, p->scales, p->status, s)
                    : launch<256, 2>(P, g.tiles_total, p->scales, p->status, s);
  else
    e = bn == 64 ? launch<64, 1>(P, g.tiles_total, p->scales, p->status, s)
        : bn == 128 ? launch<128, 1>(P, g.tiles_total, p->scales, p->status, s)
                    : launch<256, 1>(P, g.tiles_total, p->scales, p->status, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "tc_gemm_kernel launch");
  return MATPOW_OK;
}


cudaError_t launch_fxb_group(const GemmDesc* d_descs, int count, int tiles, const int4* d_tile_rec,
                             const void* d_maps, int bn, int nsl, int max_n, int num_sms, bool persist,
                             Scale* scales, unsigned* status, cudaStream_t s) {
  if (persist && d_tile_rec && bn == 64 && max_n <= 4096 && num_sms > 0)
    return launch_fxb_persist(d_descs, tiles, d_tile_rec, d_maps, nsl, num_sms, scales, status, s);
  const CUtensorMap* maps = (const CUtensorMap*)d_maps;
  if (nsl == 3)
    tc_fxb_group_kernel<64, 3><<<tiles, fx::Cfg<64, 3>::THREADS, fx::Cfg<64, 3>::SMEM, s>>>(
        d_descs, count, maps, scales, status);
  else if (bn == 64)
    tc_fxb_group_kernel<64, 2><<<tiles, fx::Cfg<64, 2>::THREADS, fx::Cfg<64, 2>::SMEM, s>>>(
        d_descs, count, maps, scales, status);
  else
    tc_fxb_group_kernel<128, 2><<<tiles, fx::Cfg<128, 2>::THREADS, fx::Cfg<128, 2>::SMEM, s>>>(
        d_descs, count, maps, scales, status);
  return cudaGetLastError();
}

matpow_status tc_launch_group_bn(matpow_plan_s* p, const GemmDesc* d_descs, int count, int tiles,
                                 const int4* d_tile_rec, const void* d_maps, int bn, int max_n,
                                 bool persist, Scale* scales, unsigned* status, cudaStream_t s) {
  const int fmt = plan_float_fmt(p);
  if (!fmt_exact(fmt))
    return fail(p, MATPOW_EUNSUPPORTED, "grouped tensor-core launches need the exact split");
  cudaError_t e = launch_fxb_group(d_descs, count, tiles, d_tile_rec, d_maps, bn, fmt_slices(fmt), max_n,
                                   p->num_sms, persist, scales, status, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "tc_fxb_group_kernel launch");
  return MATPOW_OK;
}

int tc_group_bn(int N, int nsl) { return (N <= 1024 || nsl == 3) ? 64 : 128; }

bool tc_encode_buffer_maps(CUtensorMap* m, const void* base, int N, int nsl) {
  const int fmt = nsl == 3 ? FMT_FX3 : FMT_FX2;
  const int ld = ld_for(N, fmt);
  const char* b = (const char*)base;
  const size_t ps = (size_t)plane_offset_elems(N, fmt) * 2;
  for (int k = 0; k < nsl; ++k)
    if (!tc_encode_bf16_map(&m[k], b + k * ps, N, ld, 64, tc::BM) ||
        !tc_encode_bf16_map(&m[nsl + k], b + k * ps, N, ld, 64, 64))
      return false;
  return true;
}

}  // namespace mp

namespace mp {

// Grouped block-scaled split: PrepDesc kind 0 covers nb x nb CTAs of its
// matrix; kinds 1 and 2 write the identity / a copy into the user's output.
__global__ void __launch_bounds__(256) prep_fxb_group_kernel(const PrepDesc* __restrict__ descs,
                                                             int count, Scale* scales,
                                                             unsigned* status) {
  __shared__ float red[8];
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (descs[mid].block_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const PrepDesc d = descs[lo];
  const int b = blockIdx.x - d.block_begin;
  const int N = d.N;
  if (d.kind != 0) {
    if (d.log2 && b == 0 && threadIdx.x == 0) *d.log2 = 0;
    const size_t total = (size_t)N * N;
    float* out = (float*)d.dst;
    for (size_t i = b * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)d.blocks * blockDim.x) {
      const size_t r = i / N, c = i - r * N;
      out[i] = d.kind == 1 ? (r == c ? 1.0f : 0.0f) : d.A[i];
    }
    return;
  }
  const int ld = ld_for(N, d.fmt);
  const int nb = fxb::nblocks(N);
  __nv_bfloat16* a1p = (__nv_bfloat16*)d.dst;
  const int nsl = fmt_slices(d.fmt);
  int* bexp = (int*)((char*)d.dst + fxb::bexp_offset(N, ld, nsl));
  if (nsl == 3)
    fxb::prep_block<3>(d.A, N, ld, b / nb, b % nb, a1p, d.plane, bexp, &scales[d.slot_stored].maxbits,
                       status, red);
  else
    fxb::prep_block<2>(d.A, N, ld, b / nb, b % nb, a1p, d.plane, bexp, &scales[d.slot_stored].maxbits,
                       status, red);
}

cudaError_t launch_prep_fxb_group(const PrepDesc* d, int count, int blocks, Scale* scales,
                                  unsigned* status, cudaStream_t s) {
  prep_fxb_group_kernel<<<blocks, 256, 0, s>>>(d, count, scales, status);
  return cudaGetLastError();
}

cudaError_t launch_prep_fxb(const float* A, int N, int fmt, void* dst, Scale* slot,
                            unsigned* status, cudaStream_t s) {
  const int ld = ld_for(N, fmt);
  const int nb = fxb::nblocks(N);
  const long long plane = plane_offset_elems(N, fmt);
  const int nsl = fmt_slices(fmt);
  int* bexp = (int*)((char*)dst + fxb::bexp_offset(N, ld, nsl));
  if (nsl == 3)
    prep_fxb_kernel<3><<<nb * nb, 256, 0, s>>>(A, N, ld, (__nv_bfloat16*)dst, plane, bexp,
                                               &slot->maxbits, status);
  else
    prep_fxb_kernel<2><<<nb * nb, 256, 0, s>>>(A, N, ld, (__nv_bfloat16*)dst, plane, bexp,
                                               &slot->maxbits, status);
  return cudaGetLastError();
}
}  // namespace mp
