// Exact products over the integers mod p on the tensor cores.
//
// A residue x in [0, p), p <= 65536, is stored as two balanced byte digits
// of its centred representative x' (x or x - p, |x'| <= p / 2):
// x' = 256 x1 + x0 with x0 in [-128, 127], x1 in [-128, 128], both exact in
// bfloat16.  For C = X Y mod p (arXiv 1204.3052 Sec. 4.1's product, inside
// Sec. 4.3's chain) the tensor cores form, per 256-deep chunk of k,
//     H  = sum x1 y1,   M1 = sum x1 y0,   M2 = sum x0 y1,   L = sum x0 y0,
// each a sum of at most 256 products of magnitude <= 2^14, i.e. within
// +-2^22: the float32 TMEM accumulators hold them exactly, and adding
// 1.5 * 2^23 turns each into its integer in the low bits of the float (one
// float add and one integer add per value instead of a float-to-integer
// conversion).  The epilogue warps keep 32-bit totals (within +-2^28 for
// N <= 16384), and at the end
//     c = (H * 2^16 + (M1 + M2) * 2^8 + L) mod p
// with Barrett reductions of the totals shifted by a multiple of p; a
// non-final product writes c's digits straight into the next product's
// operand planes.
//
// CTA: 384 threads.  Warp 0 TMA, warp 1 MMA (2 MMAs per 16-deep step), warp 2
// TMEM (2 buffers x 4 accumulators x 64 columns = 512), warps 4-11 epilogue
// (lane quadrant w % 4, column half (w - 4) / 4).  Every wait is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "plan.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace mp {

namespace tcm {
constexpr int BM = 128, BN = 64, BK = 64, CHUNK_KB = 4;
constexpr int EW = 8, THREADS = 128 + 32 * EW, WC = 32;
constexpr uint64_t WAIT_NS = 2000000000ull;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);
constexpr int STAGES = (192 * 1024) / STAGE_BYTES;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 512;
}  // namespace tcm

// x mod p for x < 2^32 with m = floor(2^32 / p): one correction step.
__device__ __forceinline__ unsigned barrett(unsigned x, unsigned p, unsigned m) {
  unsigned q = __umulhi(x, m);
  unsigned r = x - q * p;
  return r >= p ? r - p : r;
}

// Balanced byte digits (d1, d0) of the centred representative of x in [0, p).
__device__ __forceinline__ void modp_digits(unsigned x, unsigned p, int* d1, int* d0) {
  const int xc = x > (p >> 1) ? (int)x - (int)p : (int)x;
  const int lo = ((xc + 128) & 255) - 128;
  *d1 = (xc - lo) >> 8;  // xc - lo is a multiple of 256
  *d0 = lo;
}

// An exact integer-valued float v with |v| <= 2^22, plus 1.5 * 2^23, has the
// bits 0x4B400000 + v: totals of these bit patterns minus count * 0x4B400000
// (mod 2^32) are the exact integer totals.
constexpr float kMagic = 12582912.0f;
constexpr unsigned kMagicBits = 0x4B400000u;

// One output tile: its product, the operands' TMA descriptors (ax1/ax0: the
// high / low byte slices of X as the A operand, by1/by0: those of Y as the B
// operand) and its index within the product.
struct ModpTile {
  const GemmDesc* d;
  const CUtensorMap *ax1, *ax0, *by1, *by0;
  int t;
};

// Tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the launch's `total`
// 128 x 64 output tiles (tile_of(i) -> ModpTile).  The producer, MMA and
// epilogue roles run through the same tile sequence with running k-block and
// chunk counters, so with a grid below `total` (persistent) the next tile's
// loads and products proceed while the epilogue finishes the last one.
template <class TileOf>
__device__ __forceinline__ void modp_tiles(int total, TileOf tile_of, unsigned* status) {
  using namespace tcm;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  // full[S], empty[S], accfull[2], accempty[2], drain
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const uint32_t full0 = ptx::smem_u32(bars);
  const uint32_t empty0 = ptx::smem_u32(bars + STAGES);
  const uint32_t accfull0 = ptx::smem_u32(bars + 2 * STAGES);
  const uint32_t accempty0 = ptx::smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drainb = ptx::smem_u32(bars + 2 * STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(accfull0 + 8 * b, 1);
      ptx::mbar_init(accempty0 + 8 * b, EW);
    }
    ptx::mbar_init(drainb, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_slot), TMEM_COLS);
    ptx::tmem_relinquish();
  }
  if (warp == 0 && lane == 0 && (int)blockIdx.x < total) {
    const ModpTile f = tile_of((int)blockIdx.x);
    ptx::prefetch_tmap(f.ax1);
    ptx::prefetch_tmap(f.ax0);
    ptx::prefetch_tmap(f.by1);
    ptx::prefetch_tmap(f.by0);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;  // k-blocks issued so far (all tiles)
      bool ok = true;
      for (int i = blockIdx.x; ok && i < total; i += gridDim.x) {
        const ModpTile f = tile_of(i);
        int tm, tn;
        tile_raster(f.t, (f.d->N + BM - 1) / BM, f.d->tiles_n, &tm, &tn);
        const int m0 = tm * BM, n0 = tn * BN;
        const int KB = (f.d->N + BK - 1) / BK;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % STAGES;
          if (!ptx::mbar_wait(empty0 + 8 * s, ((g / STAGES) & 1) ^ 1, abort_flag, WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const uint32_t fb = full0 + 8 * s;
          ptx::mbar_expect_tx(fb, STAGE_BYTES);
          const uint32_t base = ptx::smem_u32(smem + s * STAGE_BYTES);
          const int kx = kb * BK;
          ptx::tma_load_2d(base, f.ax1, kx, m0, fb);                          // x1
          ptx::tma_load_2d(base + A_BYTES, f.ax0, kx, m0, fb);                // x0
          ptx::tma_load_2d(base + 2 * A_BYTES, f.by1, n0, kx, fb);            // y1
          ptx::tma_load_2d(base + 2 * A_BYTES + B_BYTES, f.by0, n0, kx, fb);  // y0
        }
      }
      // no copy may still be writing shared memory when the CTA exits
      for (int k = g - STAGES < 0 ? 0 : g - STAGES; k < g; ++k) {
        int dummy = 0;
        ptx::mbar_wait(full0 + 8 * (k % STAGES), (k / STAGES) & 1, &dummy, WAIT_NS);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc2 = idesc_bf16(BM, 2 * BN);
      int g = 0, gc = 0;  // k-blocks and chunks consumed so far (all tiles)
      bool ok = true;
      for (int i = blockIdx.x; ok && i < total; i += gridDim.x) {
        const ModpTile f = tile_of(i);
        const int KB = (f.d->N + BK - 1) / BK;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const bool first = (kb % CHUNK_KB) == 0;
          const bool last = (kb % CHUNK_KB) == CHUNK_KB - 1 || kb == KB - 1;
          const int buf = gc & 1;
          const uint32_t tH = tmem + (uint32_t)(buf * 4 * BN);
          if (first && !ptx::mbar_wait(accempty0 + 8 * buf, ((gc >> 1) & 1) ^ 1, abort_flag, WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const int s = g % STAGES;
          if (!ptx::mbar_wait(full0 + 8 * s, (g / STAGES) & 1, abort_flag, WAIT_NS)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t a1 = ptx::smem_u32(smem + s * STAGE_BYTES);
          const uint32_t a0 = a1 + A_BYTES;
          const uint32_t b1 = a1 + 2 * A_BYTES;  // y1, then y0 at + B_BYTES (one 64-column chunk)
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t ad1 = ptx::smem_desc(a1 + 32 * k, 16, 1024);
            const uint64_t ad0 = ptx::smem_desc(a0 + 32 * k, 16, 1024);
            const uint64_t bd1 = ptx::smem_desc(b1 + 2048 * k, 8192, 1024);
            const uint32_t acc = (first && k == 0) ? 0u : 1u;
            // the y1 and y0 planes lie next to each other at the MMA's 64-column
            // chunk stride: x1 [y1 | y0] -> H | M1 and x0 [y1 | y0] -> M2 | L
            ptx::mma_f16(tH, ad1, bd1, idesc2, acc);
            ptx::mma_f16(tH + 2 * BN, ad0, bd1, idesc2, acc);
          }
          ptx::mma_commit(empty0 + 8 * s);
          if (last) {
            ptx::mma_commit(accfull0 + 8 * buf);
            ++gc;
          }
        }
      }
      ptx::mma_commit(drainb);
      int dummy = 0;
      ptx::mbar_wait(drainb, 0, &dummy, WAIT_NS);
    }
  } else if (warp >= 4) {
    const int q = warp & 3;
    const int cs = (warp - 4) >> 2;
    int gc = 0;  // chunks drained so far (all tiles)
    bool ok = true;
    for (int i = blockIdx.x; ok && i < total; i += gridDim.x) {
      const ModpTile f = tile_of(i);
      const GemmDesc& d = *f.d;
      const int N = d.N;
      int tm, tn;
      tile_raster(f.t, (N + BM - 1) / BM, d.tiles_n, &tm, &tn);
      const int row = tm * BM + 32 * q + lane;
      const int nw = tn * BN + cs * WC;
      const int NCH = ((N + BK - 1) / BK + CHUNK_KB - 1) / CHUNK_KB;
      unsigned Ht[WC], Mt[WC], Lt[WC];
#pragma unroll
      for (int j = 0; j < WC; ++j) Ht[j] = Mt[j] = Lt[j] = 0u;
      for (int ch = 0; ch < NCH; ++ch, ++gc) {
        const int buf = gc & 1;
        if (!ptx::mbar_wait(accfull0 + 8 * buf, (gc >> 1) & 1, abort_flag, 2 * WAIT_NS)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 4 * BN + cs * WC);
        uint32_t r[32];
        ptx::tmem_ld_32x32b_x32(tq, r);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < WC; ++j) Ht[j] += __float_as_uint(__uint_as_float(r[j]) + kMagic);
        ptx::tmem_ld_32x32b_x32(tq + BN, r);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < WC; ++j) Mt[j] += __float_as_uint(__uint_as_float(r[j]) + kMagic);
        ptx::tmem_ld_32x32b_x32(tq + 2 * BN, r);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < WC; ++j) Mt[j] += __float_as_uint(__uint_as_float(r[j]) + kMagic);
        ptx::tmem_ld_32x32b_x32(tq + 3 * BN, r);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < WC; ++j) Lt[j] += __float_as_uint(__uint_as_float(r[j]) + kMagic);
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(accempty0 + 8 * buf);
      }
      if (!ok || *abort_flag || row >= N) continue;
      const unsigned pm = d.p;
      const unsigned bm = (unsigned)(0x100000000ull / pm);
      const unsigned c16 = (unsigned)((1ull << 16) % pm), c8 = 256u % pm;
      // totals within +-2^29; off: a multiple of p in [2^30, 2^30 + p)
      const unsigned off = pm * ((1u << 30) / pm + ((1u << 30) % pm ? 1u : 0u));
      const unsigned b1 = (unsigned)NCH * kMagicBits, b2 = 2u * b1;
      unsigned* res = Ht;  // c overwrites the H totals
#pragma unroll
      for (int j = 0; j < WC; ++j) {
        const unsigned h = barrett(Ht[j] - b1 + off, pm, bm), m = barrett(Mt[j] - b2 + off, pm, bm),
                       l = barrett(Lt[j] - b1 + off, pm, bm);
        const unsigned v = barrett(h * c16, pm, bm) + barrett(m * c8, pm, bm) + l;  // < 3p
        res[j] = barrett(v, pm, bm);
      }
      if (d.mode == OUT_INTERNAL) {
        // 16-byte groups of 8 columns: a group that starts below N ends within
        // the row's padding to ld (a multiple of 8), which no product reads;
        // its columns past N are zero (zero-filled operands)
        __nv_bfloat16* p1 = (__nv_bfloat16*)d.C + (size_t)row * d.ld + nw;
        __nv_bfloat16* p0 = p1 + d.plane;
#pragma unroll
        for (int g8 = 0; g8 < WC / 8; ++g8) {
          if (nw + 8 * g8 < N) {
            uint32_t w1[4], w0[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              int a1, a0, b1d, b0d;
              modp_digits(res[8 * g8 + 2 * h], pm, &a1, &a0);
              modp_digits(res[8 * g8 + 2 * h + 1], pm, &b1d, &b0d);
              __nv_bfloat162 hi = __floats2bfloat162_rn((float)a1, (float)b1d);
              __nv_bfloat162 lo = __floats2bfloat162_rn((float)a0, (float)b0d);
              w1[h] = *reinterpret_cast<uint32_t*>(&hi);
              w0[h] = *reinterpret_cast<uint32_t*>(&lo);
            }
            *reinterpret_cast<uint4*>(p1 + 8 * g8) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            *reinterpret_cast<uint4*>(p0 + 8 * g8) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
          }
        }
      } else {
        unsigned* O = (unsigned*)d.out + (size_t)row * N;
#pragma unroll
        for (int j = 0; j < WC; ++j)
          if (nw + j < N) O[nw + j] = res[j];
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
}

// Products of one level (one or two of the same order), persistent: grid =
// min(tiles, SMs).
__global__ void __launch_bounds__(tcm::THREADS, 1)
    tc_modp_kernel(const __grid_constant__ TcPairParams P, int total, unsigned* status) {
  modp_tiles(
      total,
      [&](int i) {
        const int which = (P.count > 1 && i >= P.tiles0) ? 1 : 0;
        const TcProblem& pr = P.p[which];
        return ModpTile{&pr.d, &pr.ax[0], &pr.ax[1], &pr.by[0], &pr.by[1], which ? i - P.tiles0 : i};
      },
      status);
}

// Grouped launch (server): products from a device table, each buffer's four
// TMA descriptors {x1, x0 as A; y1, y0 as B} from a device table at map_x
// (A role: + 0, 1) and map_y (B role: + 2, 3).  Persistent like the level
// launch when the grid is below the tile count.
__global__ void __launch_bounds__(tcm::THREADS, 1)
    tc_modp_group_kernel(const GemmDesc* __restrict__ descs, int count,
                         const CUtensorMap* __restrict__ maps, int total, unsigned* status) {
  modp_tiles(
      total,
      [&](int tb) {
        int lo = 0, hi = count - 1;  // last desc with tile_begin <= tb
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (descs[mid].tile_begin <= tb) lo = mid; else hi = mid - 1;
        }
        const GemmDesc& d = descs[lo];
        return ModpTile{&d, maps + d.map_x, maps + d.map_x + 1, maps + d.map_y + 2, maps + d.map_y + 3,
                        tb - d.tile_begin};
      },
      status);
}

// A (uint32, leading dimension N) -> balanced byte digits (x1, x0) as
// bfloat16 planes with leading dimension ld; entries >= p flag ST_BADINPUT.
__global__ void prep_modp_slices_kernel(const unsigned* __restrict__ A, int N, int ld, unsigned p,
                                        __nv_bfloat16* dst, long long plane, unsigned* status) {
  const size_t total = (size_t)N * ld;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / ld;
    const int c = (int)(i - r * ld);
    const unsigned v = c < N ? A[r * N + c] : 0u;
    bad |= v >= p;
    int d1, d0;
    modp_digits(v < p ? v : 0u, p, &d1, &d0);
    dst[i] = __float2bfloat16_rn((float)d1);
    dst[plane + i] = __float2bfloat16_rn((float)d0);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_BADINPUT);
}

// ---------------------------------------------------------------------------

cudaError_t tc_modp_init() {
  cudaError_t e = cudaFuncSetAttribute(tc_modp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcm::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_modp_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcm::SMEM);
  return e;
}

cudaError_t launch_modp_tc_group(const GemmDesc* d_descs, int count, int tiles, const void* d_maps,
                                 int num_sms, unsigned* status, cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  const int grid = num_sms > 0 && tiles > num_sms ? num_sms : tiles;
  tc_modp_group_kernel<<<grid, tcm::THREADS, tcm::SMEM, s>>>(d_descs, count, (const CUtensorMap*)d_maps,
                                                             tiles, status);
  return cudaGetLastError();
}

int tc_modp_tile_n() { return tcm::BN; }

cudaError_t launch_prep_modp_slices(const unsigned* A, int N, unsigned p, void* dst,
                                    unsigned* status, cudaStream_t s) {
  const int ld = ld_for(N, FMT_MODP);
  const long long plane = plane_offset_elems(N, FMT_MODP);
  const size_t total = (size_t)N * ld;
  size_t b = (total + 255) / 256;
  const int grid = (int)(b < 1216 ? (b ? b : 1) : 1216);
  prep_modp_slices_kernel<<<grid, 256, 0, s>>>(A, N, ld, p, (__nv_bfloat16*)dst, plane, status);
  return cudaGetLastError();
}

matpow_status tc_modp_launch_pair(matpow_plan_s* p, const GemmPair& g, cudaStream_t s) {
  TcPairParams P;
  memset(&P, 0, sizeof P);
  P.count = g.count;
  for (int i = 0; i < g.count; ++i) {
    const GemmDesc& d = g.d[i];
    TcProblem& tp = P.p[i];
    tp.d = d;
    const size_t lo = (size_t)d.plane * 2;
    if (!tc_encode_bf16_map(&tp.ax[0], d.X, d.N, d.ld, 64, tcm::BM) ||
        !tc_encode_bf16_map(&tp.ax[1], (const char*)d.X + lo, d.N, d.ld, 64, tcm::BM) ||
        !tc_encode_bf16_map(&tp.by[0], d.Y, d.N, d.ld, 64, 64) ||
        !tc_encode_bf16_map(&tp.by[1], (const char*)d.Y + lo, d.N, d.ld, 64, 64))
      return fail(p, MATPOW_ECUDA, "cuTensorMapEncodeTiled failed (N=%d)", d.N);
  }
  P.tiles0 = g.count > 1 ? g.d[1].tile_begin : g.tiles_total;
  const int grid = g.tiles_total < p->num_sms ? g.tiles_total : p->num_sms;
  tc_modp_kernel<<<grid, tcm::THREADS, tcm::SMEM, s>>>(P, g.tiles_total, p->status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(p, e, "tc_modp_kernel launch");
  return MATPOW_OK;
}

}  // namespace mp
