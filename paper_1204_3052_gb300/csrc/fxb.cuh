// Exact block-scaled split (the default MATPOW_BF16X3 arithmetic).
//
// A stored matrix S is cut into 64 x 64 blocks.  Block (I, J) with maximum
// |S| = m has exponent e = frexp exponent of m (m * 2^-e in [0.5, 1)) and its
// entries are written as two integer slices
//     u = s * 2^(8-e),  a1 = rint(u) in [-256, 256],  a2 = rint(256 (u - a1)) in [-128, 128],
// so s = 2^(e-16) (256 a1 + a2) to within 2^(e-17).  Integers of at most 8
// significant bits are exact in bfloat16, so the tensor core multiplies them
// exactly.  For a 64-deep k-block the products sum to
//     main  = sum a1 b1            (|main|  <= 64 * 2^16 = 2^22)
//     cross = sum a1 b2 + a2 b1    (|cross| <= 64 * 2^16 = 2^22)
// which the float32 TMEM accumulator holds exactly whatever its rounding.
// Each finished k-block is folded into float32 registers with
// round-to-nearest:
//     T += (main + cross / 256) * 2^(eX(I,kb) + eY(kb,J) - 16 - sX - sY)
// where eX, eY are the operands' block exponents and sX, sY their global
// (frexp) exponents; T is then the product of the two normalised operands
// (the lagged power-of-two scale of the chain).  The a2*b2 term (2^-16
// relative) is dropped.  The epilogue re-splits T by 64 x 64 blocks, so no
// global maximum is needed before the next product can start.
//
// With three slices (MATPOW_BF16X6) a third one a3 = rint(256 * remainder)
// extends the fixed point to 24 bits; six products a1b1 | a1b2 + a2b1 |
// a1b3 + a2b2 + a3b1 fill three accumulators (the third sums to below
// 64 * 81920 < 2^23 per k-block, still exact), and the dropped terms are
// 2^-24 relative: float32-class results.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace mp {
namespace fxb {

constexpr int BLK = 64;
constexpr int MAX_KB = 512;  // exponent table in shared memory: N <= 32768

__host__ __device__ inline size_t align1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

// Byte offset of the block-exponent table (int32, nb x nb) in a stored matrix
// of NSL slice planes.
__host__ __device__ inline size_t bexp_offset(int N, int ld, int NSL = 2) {
  return (size_t)NSL * align1k((size_t)N * ld * 2);
}
__host__ __device__ inline int nblocks(int N) { return (N + BLK - 1) / BLK; }

// 2^k as a float, exact for k in [-252, 254] (k below -252 gives 0).
__device__ __forceinline__ float pow2f(int k) {
  if (k >= -126 && k <= 127) return __int_as_float((127 + k) << 23);
  if (k < -252) return 0.f;
  return mul_pow2(1.0f, k);
}

// The i-th k-block a tile visits: tiles start at different k-blocks (tile_rot:
// (m0 + n0) / 128, the same for 64- and 128-wide tiles covering an element)
// so that CTAs sharing an operand band do not read the same lines at the same
// time.  The fold order follows it, identically in every kernel.
__device__ __forceinline__ int rot_kb(int i, int KB, int rot) {
  int k = i + rot % KB;
  return k >= KB ? k - KB : k;
}

// The rotation of the tile at (m0, n0) of a product with KB k-blocks:
// (m0 + n0) / 128 up to KB = 32 (N <= 2048); above, every tile starts at
// k-block 0 so that the CTAs of a wave move through k together and share each
// k-slab of their bands in L2.
__device__ __forceinline__ int tile_rot(int m0, int n0, int KB) { return KB > 32 ? 0 : (m0 + n0) / 128; }

__device__ __forceinline__ int frexp_exp(float m) { return scale_exp_from_bits(__float_as_uint(m)); }

// The bfloat16 pair (x0 low, x1 high) of two floats whose values are exact in
// bfloat16 (the integer slices: at most 8 significant bits), so that their
// low 16 bits are zero and rounding changes nothing: the upper halves, one
// byte permute instead of a conversion.
__device__ __forceinline__ uint32_t pack_bf16_exact(float x0, float x1) {
  return __byte_perm(__float_as_uint(x0), __float_as_uint(x1), 0x7632);
}

__device__ __forceinline__ void slice(float v, int e, float* h, float* l) {
  const float u = mul_pow2(v, 8 - e);
  *h = rintf(u);
  *l = rintf((u - *h) * 256.f);
}

// NSL integer slices of v relative to block exponent e:
//   u = v 2^(8-e); a0 = rint(u); a_k = rint(256 (previous remainder)).
template <int NSL>
__device__ __forceinline__ void slice_n(float v, int e, float (&a)[NSL]) {
  float u = mul_pow2(v, 8 - e);
#pragma unroll
  for (int k = 0; k < NSL; ++k) {
    a[k] = rintf(u);
    u = (u - a[k]) * 256.f;
  }
}

// The slice products of one 16-deep k-step into the NSL accumulators at TMEM
// column t0 (accumulator w at t0 + w BN collects a_i b_j with i + j = w).
// The B slice planes lie next to each other at the MMA's 64-column chunk
// stride, so the products that share an A slice go out as one wider MMA:
// a_i [b_0 | ... | b_(NSL-1-i)] with N = (NSL - i) BN, written to
// accumulators i .. NSL - 1.  acc = 0 on the k-block's first k-step (the
// first MMA then initialises every accumulator).  The sums are exact
// integers, so grouping the products this way changes no result.
template <int BN, int NSL>
__device__ __forceinline__ void slice_mmas(uint32_t t0, const uint64_t (&ad)[NSL], uint64_t bd0, uint32_t acc) {
  static_assert(NSL * BN <= 256, "MMA N");
#pragma unroll
  for (int i = 0; i < NSL; ++i)
    ptx::mma_f16(t0 + (uint32_t)(i * BN), ad[i], bd0, idesc_bf16(128, (NSL - i) * BN), i == 0 ? acc : 1u);
}

// Named barrier 1 over the NT epilogue threads (warps 4.. of the CTA).
template <int NT = 128>
__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Epilogue warps (q = warp % 4 owns rows 32q..32q+31 of the 128-row tile;
// rows 64h..64h+63 form block row h = q / 2).  T holds this thread's row `row`
// of the tile, columns n0..n0+BN-1.  Computes each 64 x 64 block's maximum
// over the warp pair, writes the block exponents and the NSL slice planes
// with plain global stores (a1p: first plane, the next at + plane elements)
// and folds the block maxima into the matrix maximum (*maxbits).  NT epilogue
// threads share named barrier 1; red: shared scratch of 4 * (BN / 64) floats.
template <int BN, int NT = 128, int NSL = 2>
__device__ __forceinline__ void store_slices(const float (&T)[BN], int row, int m0, int n0, int q,
                                             int lane, int N, int ld, __nv_bfloat16* a1p,
                                             long long plane, int* bexp, unsigned* maxbits,
                                             float* red) {
  constexpr int NG = BN / BLK;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < BLK; ++j) m = fmaxf(m, fabsf(T[BLK * g + j]));
    m = warp_max(m);
    if (lane == 0) red[q * NG + g] = m;
  }
  epi_bar<NT>();
  const int nb = nblocks(N);
  const int I = m0 / BLK + (q >> 1);
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const float bm = fmaxf(red[q * NG + g], red[(q ^ 1) * NG + g]);
    const int e = frexp_exp(bm);
    const int J = n0 / BLK + g;
    if ((q & 1) == 0 && lane == 0 && I < nb && J < nb) {
      bexp[I * nb + J] = e;
      if (bm > 0.f) atomicMax(maxbits, __float_as_uint(bm));
    }
    if (row < N) {
      // 16-byte groups of 8 columns; a group that starts below N ends within
      // the row's padding to ld (a multiple of 8), which no product reads, and
      // its columns past N hold exact zeros (zero-filled operands)
      const int c0 = n0 + BLK * g;
      __nv_bfloat16* p1 = a1p + (size_t)row * ld + c0;
#pragma unroll
      for (int g8 = 0; g8 < BLK / 8; ++g8) {
        if (c0 + 8 * g8 < N) {
          uint32_t w[NSL][4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            float x0[NSL], x1[NSL];
            slice_n<NSL>(T[BLK * g + 8 * g8 + 2 * h], e, x0);
            slice_n<NSL>(T[BLK * g + 8 * g8 + 2 * h + 1], e, x1);
#pragma unroll
            for (int k = 0; k < NSL; ++k) {
              w[k][h] = pack_bf16_exact(x0[k], x1[k]);
            }
          }
#pragma unroll
          for (int k = 0; k < NSL; ++k)
            *reinterpret_cast<uint4*>(p1 + k * plane + 8 * g8) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
        }
      }
    }
  }
  epi_bar<NT>();  // red may be reused
}

// store_slices for epilogue threads that each hold WC (32 or 64) of a
// tile's columns: T is row `row` of the tile at columns c0 .. c0 + WC - 1
// (c0 = the tile's n0 + cs WC, cs the thread's column part).  A 64 x 64
// block's maximum is reduced over the warps that hold it -- the quadrant
// pair (q, q ^ 1) and, for WC = 32, both column halves -- through red
// (8 floats per 64-column block of the tile); then the block exponent, the
// matrix maximum and this thread's slices as in store_slices.  NT epilogue
// threads share named barrier 1.
template <int WC, int NT, int NSL>
__device__ __forceinline__ void store_slices_part(const float (&T)[WC], int row, int m0, int n0, int c0, int q,
                                                  int cs, int lane, int N, int ld, __nv_bfloat16* a1p,
                                                  long long plane, int* bexp, unsigned* maxbits, float* red) {
  static_assert(WC == 32 || WC == 64, "column part");
  constexpr int NPART = 64 / WC;  // column parts per 64-column block
  const int gblk = (c0 - n0) / BLK;  // this thread's block within the tile
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < WC; ++j) m = fmaxf(m, fabsf(T[j]));
  m = warp_max(m);
  if (lane == 0) red[gblk * 8 + q * NPART + (NPART == 2 ? (cs & 1) : 0)] = m;
  epi_bar<NT>();
  const int nb = nblocks(N);
  const int I = m0 / BLK + (q >> 1);
  float bm = fmaxf(red[gblk * 8 + q * NPART], red[gblk * 8 + (q ^ 1) * NPART]);
  if (NPART == 2) bm = fmaxf(bm, fmaxf(red[gblk * 8 + q * NPART + 1], red[gblk * 8 + (q ^ 1) * NPART + 1]));
  const int e = frexp_exp(bm);
  const int J = n0 / BLK + gblk;
  if ((q & 1) == 0 && lane == 0 && (NPART == 1 || (cs & 1) == 0) && I < nb && J < nb) {
    bexp[I * nb + J] = e;
    if (bm > 0.f) atomicMax(maxbits, __float_as_uint(bm));
  }
  if (row < N) {
    // 16-byte groups of 8 columns, as in store_slices
    __nv_bfloat16* p1 = a1p + (size_t)row * ld + c0;
#pragma unroll
    for (int g8 = 0; g8 < WC / 8; ++g8) {
      if (c0 + 8 * g8 < N) {
        uint32_t w[NSL][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float x0[NSL], x1[NSL];
          slice_n<NSL>(T[8 * g8 + 2 * h], e, x0);
          slice_n<NSL>(T[8 * g8 + 2 * h + 1], e, x1);
#pragma unroll
          for (int k = 0; k < NSL; ++k) {
            w[k][h] = pack_bf16_exact(x0[k], x1[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < NSL; ++k)
          *reinterpret_cast<uint4*>(p1 + k * plane + 8 * g8) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
      }
    }
  }
  epi_bar<NT>();  // red may be reused
}

// Like store_slices, but the slice planes leave through TMA: each epilogue
// thread writes its row of every 64-column box into shared memory in the
// 128-byte-swizzled layout the tensor map expects (16-byte chunk c of row r at
// chunk position c ^ (r % 8)), then one thread stores each 128 x 64 box with
// one bulk-tensor instruction and waits for the writes to complete (they are
// read by TMA loads of the next product, after a barrier).
//   T: this thread's WC columns starting at nw (a multiple of 64); r: row in
//   the 128-row tile (32 q + lane); stage: 1024-aligned shared memory with
//   room for 2 planes x (number of boxes) x 16 KB; box0: index of this
//   warp's first box; c1, c2: the destination planes' tensor maps (box 64 x
//   128); leader: the one thread that issues the stores; NT epilogue threads.
template <int WC, int NT, int NSL = 2>
__device__ __forceinline__ void store_slices_tma(const float (&T)[WC], int r, int m0, int nw, int q,
                                                 int lane, int N, int box0, int nbox, uint8_t* stage,
                                                 const CUtensorMap* const (&cmap)[NSL], int* bexp,
                                                 unsigned* maxbits, float* red, bool leader, int n0) {
  constexpr int NG = WC / BLK;
  constexpr int BOX = NSL * 16384;  // bytes of one 128 x 64 box in all planes
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < BLK; ++j) m = fmaxf(m, fabsf(T[BLK * g + j]));
    m = warp_max(m);
    if (lane == 0) red[(box0 + g) * 4 + q] = m;
  }
  epi_bar<NT>();
  const int nb = nblocks(N);
  const int I = m0 / BLK + (q >> 1);
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const int b = box0 + g;
    const float bm = fmaxf(red[b * 4 + q], red[b * 4 + (q ^ 1)]);
    const int e = frexp_exp(bm);
    const int J = (nw + BLK * g) / BLK;
    if ((q & 1) == 0 && lane == 0 && I < nb && J < nb) {
      bexp[I * nb + J] = e;
      if (bm > 0.f) atomicMax(maxbits, __float_as_uint(bm));
    }
    uint8_t* p0 = stage + (size_t)b * BOX + r * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint32_t w[NSL][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float x0[NSL], x1[NSL];
        slice_n<NSL>(T[BLK * g + 8 * c + 2 * h], e, x0);
        slice_n<NSL>(T[BLK * g + 8 * c + 2 * h + 1], e, x1);
#pragma unroll
        for (int k = 0; k < NSL; ++k) {
          w[k][h] = pack_bf16_exact(x0[k], x1[k]);
        }
      }
      const int pos = (c ^ (r & 7)) * 16;
#pragma unroll
      for (int k = 0; k < NSL; ++k)
        *reinterpret_cast<uint4*>(p0 + 16384 * k + pos) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
    }
  }
  ptx::fence_proxy_async_smem();  // generic smem writes -> visible to the TMA engine
  epi_bar<NT>();
  if (leader) {
    for (int b = 0; b < nbox; ++b) {
      const uint32_t src = ptx::smem_u32(stage + (size_t)b * BOX);
#pragma unroll
      for (int k = 0; k < NSL; ++k) ptx::tma_store_2d(cmap[k], n0 + BLK * b, m0, src + 16384 * k);
    }
    ptx::bulk_commit();
    ptx::bulk_wait_all();
    ptx::fence_proxy_async_global();
  }
  epi_bar<NT>();  // the stage and red may be reused
}

// Transpose of 8 x 8 chunks of 8 floats within each group of 8 lanes (lane
// i = lane % 8 of group g = lane / 8), by three butterfly exchanges of half
// the chunks with the lane at distance 4, 2, 1.  Before: T[8 c + r] is
// element r of chunk c of the lane's own row.  After: T[8 j + r] is element
// r of chunk i of the row held by lane 8 g + j.  Every lane of the warp must
// take part.
__device__ __forceinline__ void transpose8x8(float (&T)[64], int lane) {
#pragma unroll
  for (int s = 4; s >= 1; s >>= 1) {
    const bool hi = (lane & s) != 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c & s) continue;  // chunk pair (c, c | s)
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float send = hi ? T[8 * c + r] : T[8 * (c | s) + r];
        const float recv = __shfl_xor_sync(0xffffffffu, send, s);
        if (hi)
          T[8 * c + r] = recv;
        else
          T[8 * (c | s) + r] = recv;
      }
    }
  }
}

// Fold one finished k-block into T with the block factors fac[g] (one per 64
// columns; BN = 32 takes fac[0]).  Accumulator k (0: main, 1: weight 2^-8,
// 2: weight 2^-16) sits at TMEM column tq + k * acc_stride.
template <int BN, int NSL = 2>
__device__ __forceinline__ void fold(float (&T)[BN], uint32_t tq, const float* fac,
                                     uint32_t acc_stride = BN) {
#pragma unroll
  for (int c = 0; c < BN / 32; ++c) {
    uint32_t rm[32], rc[32];
    ptx::tmem_ld_32x32b_x32(tq + 32 * c, rm);
    ptx::tmem_ld_32x32b_x32(tq + acc_stride + 32 * c, rc);
    if (NSL == 3) {
      uint32_t rd[32];
      ptx::tmem_ld_32x32b_x32(tq + 2 * acc_stride + 32 * c, rd);
      ptx::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 32; ++j)
        rc[j] = __float_as_uint(fmaf(__uint_as_float(rd[j]), 0.00390625f, __uint_as_float(rc[j])));
    } else {
      ptx::tmem_ld_wait();
    }
    const float f = fac[c / 2];
#pragma unroll
    for (int j = 0; j < 32; ++j)
      T[32 * c + j] = fmaf(fmaf(__uint_as_float(rc[j]), 0.00390625f, __uint_as_float(rm[j])), f,
                           T[32 * c + j]);
  }
}

// One 64 x 64 block (I, J) of a float32 matrix A (leading dimension N) split
// into the stored format by the first 256 threads of the CTA (with NB = 0
// any further threads take part in its barriers only; with NB = 256 they do
// not take part at all): block exponent, slices, matrix maximum, non-finite
// check.  red: 8 floats of shared scratch.  In two
// steps: prep_load reads this thread's 16 values of the block (so that a
// kernel can start the reads early), prep_split does the rest; prep_block
// runs both.
__device__ __forceinline__ void prep_load(const float* __restrict__ A, int N, int I, int J, float (&v)[16]) {
  const int tid = threadIdx.x;
  const int r = tid < 256 ? I * BLK + (tid >> 2) : N;  // idle threads: past the last row
  const int c0 = J * BLK + (tid & 3) * 16;
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = (r < N && c0 + j < N) ? A[(size_t)r * N + c0 + j] : 0.f;
}

// NB = 0: the CTA's barrier (every thread takes part); NB = 256: named
// barrier 3 over threads 0..255 alone (the other warps may do other work).
template <int NB>
__device__ __forceinline__ bool prep_sync_or(bool pred) {
  if constexpr (NB == 0) {
    return __syncthreads_or(pred);
  } else {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, 3, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(NB)
        : "memory");
    return r != 0;
  }
}
template <int NB>
__device__ __forceinline__ void prep_sync() {
  if constexpr (NB == 0)
    __syncthreads();
  else
    asm volatile("barrier.cta.sync 3, %0;" ::"n"(NB) : "memory");
}

template <int NSL = 2, int NB = 0>
__device__ __forceinline__ void prep_split(const float (&v)[16], int N, int ld, int I, int J,
                                           __nv_bfloat16* a1p, long long plane, int* bexp,
                                           unsigned* maxbits, unsigned* status, float* red) {
  const int tid = threadIdx.x;
  const bool act = tid < 256;
  const int r = act ? I * BLK + (tid >> 2) : N;
  const int c0 = J * BLK + (tid & 3) * 16;
  float m = 0.f;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    bad |= !isfinite(v[j]);
    m = fmaxf(m, fabsf(v[j]));
  }
  m = warp_max(m);
  if (act && (tid & 31) == 0) red[tid >> 5] = m;
  if (prep_sync_or<NB>(bad) && tid == 0) atomicOr(status, ST_BADINPUT);
  float bm = red[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) bm = fmaxf(bm, red[w]);
  const int e = frexp_exp(bm);
  const int nb = nblocks(N);
  if (tid == 0) {
    bexp[I * nb + J] = e;
    if (bm > 0.f) atomicMax(maxbits, __float_as_uint(bm));
  }
  if (r < N && c0 < ld) {
    __nv_bfloat16* p1 = a1p + (size_t)r * ld + c0;
    if (c0 + 16 <= ld) {
#pragma unroll
      for (int g8 = 0; g8 < 2; ++g8) {
        uint32_t w[NSL][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float x0[NSL], x1[NSL];
          slice_n<NSL>(v[8 * g8 + 2 * h], e, x0);
          slice_n<NSL>(v[8 * g8 + 2 * h + 1], e, x1);
#pragma unroll
          for (int k = 0; k < NSL; ++k) {
            w[k][h] = pack_bf16_exact(x0[k], x1[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < NSL; ++k)
          *reinterpret_cast<uint4*>(p1 + k * plane + 8 * g8) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (c0 + j < ld) {
          float x[NSL];
          slice_n<NSL>(v[j], e, x);
#pragma unroll
          for (int k = 0; k < NSL; ++k) p1[k * plane + j] = __float2bfloat16_rn(x[k]);
        }
      }
    }
  }
  prep_sync<NB>();  // red may be reused
}

template <int NSL = 2, int NB = 0>
__device__ __forceinline__ void prep_block(const float* __restrict__ A, int N, int ld, int I, int J,
                                           __nv_bfloat16* a1p, long long plane, int* bexp,
                                           unsigned* maxbits, unsigned* status, float* red) {
  float v[16];
  prep_load(A, N, I, J, v);
  prep_split<NSL, NB>(v, N, ld, I, J, a1p, plane, bexp, maxbits, status, red);
}

// Exponent table of one tile, staged in shared memory by warp 3:
// eA[h * KB + kb] = eX(I0 + h, kb) for the tile's two block rows,
// eB[kb * NG + g] = eY(kb, J0 + g) for its BN / 64 block columns.
template <int BN>
__device__ __forceinline__ void load_tile_exponents(const int* bexpX, const int* bexpY, int N, int m0,
                                                    int n0, int KB, int* eA, int* eB, int lane) {
  constexpr int NG = BN / BLK;
  const int nb = nblocks(N);
  const int I0 = m0 / BLK, J0 = n0 / BLK;
  for (int i = lane; i < 2 * KB; i += 32) {
    const int h = i / KB, kb = i - h * KB;
    eA[i] = (I0 + h < nb) ? __ldcg(bexpX + (I0 + h) * nb + kb) : 0;
  }
  for (int i = lane; i < NG * KB; i += 32) {
    const int kb = i / NG, g = i - kb * NG;
    eB[i] = (J0 + g < nb) ? __ldcg(bexpY + kb * nb + J0 + g) : 0;
  }
}

}  // namespace fxb
}  // namespace mp
