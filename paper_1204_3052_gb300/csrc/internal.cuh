// Internal types and helpers shared by the libmatpow kernels and host code.
// Nothing here is part of the C-ABI (include/matpow.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "matpow.h"

namespace mp {

// A stored matrix S stands for the true value T = S * 2^E.  maxbits collects
// max|S| as float bits (atomicMax on the bit pattern orders non-negative
// floats correctly); it must be zero before the kernel that writes S starts.
struct Scale {
  unsigned int maxbits;
  int pad;
  long long E;
};

// Deferred device status bits (OR-ed into the plan's status word).
enum : unsigned {
  ST_RANGE = 1u,     // a float32 output left the float32 range
  ST_BADINPUT = 2u,  // non-finite float input or an entry >= p
  ST_TIMEOUT = 4u,   // a bounded device wait gave up
};

// Internal storage formats of partial products.
enum Fmt : int {
  FMT_F32 = 0,     // float32, leading dimension roundup(N, 4)
  FMT_BF16 = 1,    // one bfloat16 plane, leading dimension roundup(N, 8)
  FMT_PLANES = 2,  // bfloat16 hi plane then lo plane (x ~ hi + lo), ld roundup(N, 8)
  FMT_MODP = 3,    // mod-p residues as two byte planes x = 256*x1 + x0 held in
                   // bfloat16 (exact integers 0..255): x1 plane then x0 plane
  FMT_U32 = 4,     // mod-p residues as uint32, leading dimension roundup(N, 4)
  FMT_FX2 = 5,     // exact block-scaled split: integer slices a1, a2 (two bfloat16
                   // planes) and an int32 exponent per 64 x 64 block; ld roundup(N, 8)
  FMT_FX3 = 6,     // the same with three slices a1, a2, a3
};

inline __host__ __device__ int fmt_slices(int fmt) { return fmt == FMT_FX3 ? 3 : 2; }
inline __host__ __device__ bool fmt_exact(int fmt) { return fmt == FMT_FX2 || fmt == FMT_FX3; }

// Where a product's result goes.
enum OutMode : int {
  OUT_INTERNAL = 0,    // stored matrix in the plan's format (and its max)
  OUT_USER_MANT = 1,   // user float32 array (ld N) holding the mantissa; E to out_log2
  OUT_USER_VALUE = 2,  // user float32 array (ld N) holding S*2^E rounded to float32
};

// One product C = X * Y of a grouped launch.
struct GemmDesc {
  const void* X;
  const void* Y;
  void* C;               // internal output (OUT_INTERNAL)
  void* out;             // user output (OUT_USER_*): float32 or uint32, leading dimension N
  long long* out_log2;   // user exponent (OUT_USER_MANT), may be null
  long long plane;       // element offset of the second plane (FMT_PLANES / FMT_MODP)
  int N;                 // order
  int ld;                // leading dimension (elements) of X, Y and internal C
  int sx, sy, sc;        // scale slots of X, Y, C (float paths)
  int mode;              // OutMode (mod p: OUT_INTERNAL or OUT_USER_VALUE)
  int tile_begin;        // first linear tile of this product in the launch
  int tiles_n;           // tiles along a row of C
  unsigned p;            // modulus (mod-p paths)
  int bn;                // tensor-core tile width (columns of C per CTA)
  int map_x, map_y;      // grouped tensor-core launches: TMA descriptors of X, Y and C
  int map_c, pad2_;      // (4 per buffer: A-role a1, a2, B-role a1, a2)
};

// Up to two products passed by value (one squaring level of one matrix:
// R <- R*P and P <- P*P, which both read P).
struct GemmPair {
  GemmDesc d[2];
  int count;
  int tiles_total;
};

inline __host__ __device__ int ld_for(int N, int fmt) {
  if (fmt == FMT_F32 || fmt == FMT_U32) return (N + 3) & ~3;
  return (N + 7) & ~7;
}

// Output tile t of a tiles_m x tiles_n grid, visited in groups of GM tile
// rows and column by column inside a group: a wave of consecutive CTAs covers
// a compact block of tiles, so it reads few row bands of X and column bands of
// Y, which stay in L2 while the wave runs; the next waves of the group reuse
// its row bands, and Y is streamed once per group (GM = 16 for tall grids).
// The arithmetic of a tile does not depend on when it runs.
__host__ __device__ inline void tile_raster(int t, int tiles_m, int tiles_n, int* tm, int* tn) {
  const int GM = tiles_m >= 32 ? 16 : 8;
  const int per = GM * tiles_n;
  const int g = t / per;
  const int r = t - g * per;
  const int rows = tiles_m - g * GM < GM ? tiles_m - g * GM : GM;
  *tm = g * GM + r % rows;
  *tn = r / rows;
}

// Exponent s with max * 2^-s in [0.5, 1) (frexp convention); 0 for max = 0.
__device__ __forceinline__ int scale_exp_from_bits(unsigned bits) {
  if (bits == 0u) return 0;
  unsigned biased = (bits >> 23) & 0xffu;
  if (biased == 0u) {  // subnormal maximum
    int e;
    (void)frexpf(__uint_as_float(bits), &e);
    return e;
  }
  return (int)biased - 126;
}

// x * 2^k for |k| up to ~250 without leaving the float range in an
// intermediate: two exact power-of-two multiplications.
__device__ __forceinline__ float mul_pow2(float x, int k) {
  int k1 = k / 2;
  int k2 = k - k1;
  return x * __int_as_float((127 + k1) << 23) * __int_as_float((127 + k2) << 23);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Final rescale of a stored value to float32 in float64 (S * 2^E).
__device__ __forceinline__ float final_value(float s, long long E, unsigned* status) {
  // Common case: s is a normal float and s 2^E is one too, so the result is
  // exact and is s with E added to its exponent field.  Zero, subnormal
  // operands and results outside the normal range take the float64 route
  // (one rounding to float32, overflow to +-inf, underflow to 0 or subnormal).
  const unsigned bits = __float_as_uint(s);
  const int es = (int)((bits >> 23) & 0xffu);
  if (es != 0 && es != 255 && E > -254 && E < 254) {
    const int et = es + (int)E;
    if (et >= 1 && et <= 254) return __uint_as_float(bits + ((unsigned)(int)E << 23));
  }
  long long Ec = E < -4000 ? -4000 : (E > 4000 ? 4000 : E);
  double v = ldexp((double)s, (int)Ec);
  float f = (float)v;
  if (s != 0.0f && (isinf(f) || f == 0.0f) && isfinite(s)) atomicOr(status, ST_RANGE);
  return f;
}

// One thread's row of a final float32 result: columns c0 .. c0 + W - 1 of
// row O (clipped at N), as mantissas (mant) or rescaled by 2^E (T is
// overwritten).  16-byte stores when every row of the N x N output starts on
// 16 bytes (N % 4 == 0 and a 16-byte aligned base); W and c0 are multiples of 4.
template <int W>
__device__ __forceinline__ void store_row_f32(float (&T)[W], float* O, int c0, int N, bool mant, long long E,
                                              unsigned* status, const void* out_base) {
  if (!mant) {
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (c0 + j < N) T[j] = final_value(T[j], E, status);
  }
  if ((N & 3) == 0 && ((uintptr_t)out_base & 15) == 0) {
#pragma unroll
    for (int j = 0; j < W; j += 4)
      if (c0 + j < N) *reinterpret_cast<float4*>(O + c0 + j) = make_float4(T[j], T[j + 1], T[j + 2], T[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (c0 + j < N) O[c0 + j] = T[j];
  }
}

}  // namespace mp

// Launchers implemented in the .cu files (host side).
namespace mp {
struct LaunchCtx {
  cudaStream_t stream;
  Scale* scales;
  unsigned* status;
};
cudaError_t launch_absmax_f32(const float* A, int N, Scale* slot, unsigned* status, cudaStream_t s);
cudaError_t launch_convert_f32(const float* A, int N, const Scale* raw, Scale* stored, int fmt,
                               void* dst, long long plane, cudaStream_t s);
cudaError_t launch_identity(void* out, int N, int is_u32, unsigned one, long long* log2,
                            cudaStream_t s);
cudaError_t launch_copy(const void* A, void* out, int N, long long* log2, cudaStream_t s);
// SIMT products on E x E tiles, E = simt_tile_edge(tiles of the launch at
// E = 128, SMs): 128 or 64; every descriptor's tiles_n counts E-wide tiles.
// split = simt_split(E, tiles of the launch at E, SMs): 2 runs each tile on a
// cluster of two CTAs, each summing half of k.
cudaError_t launch_simt_pair(const GemmPair& g, int edge, int split, Scale* scales, unsigned* status,
                             cudaStream_t s);
cudaError_t launch_simt_group(const GemmDesc* d_descs, int count, int tiles_total, int edge, int split,
                              Scale* scales, unsigned* status, cudaStream_t s);
int simt_tile_edge(int tiles128, int num_sms);
int simt_split(int edge, int tiles, int num_sms);
// Whole-chain kernel for small N: one CTA per matrix.
struct TinyDesc {
  const float* A;
  float* out;
  long long* log2;  // null: value mode
  unsigned long long n;
  int N;
  int pad_;
};
cudaError_t launch_selftest_wait(unsigned long long budget_ns, unsigned* status, cudaStream_t s);
// FP32 FFMA throughput probe: `blocks` CTAs of 256 threads, 8 x iters FFMA each.
cudaError_t launch_ffma_probe(long long iters, int blocks, unsigned* sink, cudaStream_t s);
cudaError_t launch_tiny_one(const TinyDesc& d, unsigned* status, cudaStream_t s);
cudaError_t launch_tiny_group(const TinyDesc* d_descs, int count, unsigned* status, cudaStream_t s);
int tiny_max_supported();
cudaError_t tiny_attrs();  // kernel attributes; called once per plan (outside any capture)
// mod p
cudaError_t launch_modp_check_convert(const unsigned* A, int N, unsigned p, unsigned* dst,
                                      unsigned* status, cudaStream_t s);
cudaError_t launch_modp_pair(const GemmPair& g, unsigned* status, cudaStream_t s);
cudaError_t launch_modp_group(const GemmDesc* d_descs, int count, int tiles_total, unsigned* status,
                              cudaStream_t s);
int modp_tile_edge();
}  // namespace mp

namespace mp {
// Per-matrix preparation of a batch (absmax, conversion) and the trivial
// powers n <= 1 of matrices too large for the whole-chain kernel.
struct PrepDesc {
  const float* A;
  void* dst;          // stored format (general path) or user output (trivial)
  long long* log2;    // trivial: user exponent or null
  long long plane;
  int N;
  int fmt;
  int slot_raw;       // scale slot of max|A|
  int slot_stored;    // scale slot of the stored A
  int block_begin;    // first CTA of this matrix in the launch
  int blocks;         // CTAs of this matrix
  int kind;           // 0: absmax/convert, 1: identity (n = 0), 2: copy (n = 1)
  int pad_;
};
// Float32 A (leading dimension N) -> the block-scaled exact split (FMT_FX2 or
// FMT_FX3) at dst; max|A| folds into slot->maxbits.  One CTA per 64 x 64 block.
cudaError_t launch_prep_fxb(const float* A, int N, int fmt, void* dst, Scale* slot,
                            unsigned* status, cudaStream_t s);
// Block-scaled split of many matrices (PrepDesc kind 0: nb x nb CTAs each;
// kinds 1, 2: identity / copy into the user's output).
cudaError_t launch_prep_fxb_group(const PrepDesc* d, int count, int blocks, Scale* scales,
                                  unsigned* status, cudaStream_t s);
cudaError_t launch_prep_absmax_group(const PrepDesc* d, int count, int blocks, Scale* scales,
                                     unsigned* status, cudaStream_t s);
cudaError_t launch_prep_convert_group(const PrepDesc* d, int count, int blocks, Scale* scales,
                                      cudaStream_t s);
}  // namespace mp
