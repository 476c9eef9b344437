// Float32 SIMT products on the CUDA cores.
//
//  * simt_gemm: C = X * Y for stored float32 matrices (arXiv 1204.3052
//    Sec. 4.1's c_ij = sum_k x_ik y_kj), tiled through shared memory
//    (Sec. 4.3.2, 4.3.7) with 128-bit vector loads (Sec. 4.3.5) and coalesced
//    row-major access (Sec. 4.3.3).  On sm_103a: a 128x128 CTA tile with an
//    8x8 register tile per thread, or 64x64 with 4x4 where 128-wide tiles
//    would leave most SMs idle; 16-deep k-steps double-buffered in shared
//    memory.  The epilogue applies the lagged power-of-two scale of the
//    operands, writes the stored result (or the user's float32 output) and
//    folds max|C| into the result's scale slot.
//  * tiny_chain: the whole square-and-multiply chain (Sec. 4.3) for N <= 64
//    in one CTA, with every partial product in shared memory.
#include "internal.cuh"

namespace mp {

namespace simt {
constexpr int BK = 16, THREADS = 256, PAD = 4;
// split-K over a cluster of two CTAs (64-wide tiles)
__device__ __forceinline__ uint32_t ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// both CTAs of the cluster execute the same two of these, so none waits for a
// thread that never arrives
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t peer(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
}  // namespace simt

// The tile edge E of a launch: 128 x 128 tiles (an 8 x 8 register tile per
// thread) unless they leave most SMs idle -- fewer 128-tiles than SMs, as for
// orders up to ~1500 -- then 64 x 64 tiles (4 x 4 per thread, four times the
// CTAs).
int simt_tile_edge(int tiles128, int num_sms) { return tiles128 < num_sms ? 64 : 128; }
// Split-K over clusters of two CTAs for 64-wide tiles that still number fewer
// than the SMs.
int simt_split(int edge, int tiles, int num_sms) { return edge == 64 && tiles < num_sms ? 2 : 1; }

// One E x E tile of one product (256 threads as 16 x 16, each holding an
// (E / 16) x (E / 16) register tile: rows 4 ty + 64 h + i, columns
// 4 tx + 64 h + j).  SPLIT = 2 (64-wide tiles, clusters of two CTAs): CTA
// rank r sums the k-steps of its half of k; rank 1 then stores its partial
// tile into rank 0's operand buffers through distributed shared memory and
// rank 0 adds it (rank 0's half + rank 1's half, in that order) and runs the
// epilogue.
template <int E, int SPLIT = 1>
__device__ __forceinline__ void simt_tile(const GemmDesc& d, int tile, Scale* scales,
                                          unsigned* status) {
  using namespace simt;
  static_assert(E == 64 || E == 128, "tile edge");
  static_assert(SPLIT == 1 || (SPLIT == 2 && E == 64), "split-K on 64-wide tiles");
  constexpr int T = E / 16;  // register tile edge
  constexpr int H = E / 64;  // 4-wide groups per register-tile edge
  // the operand buffers As [2][BK][E + PAD] and Bs (likewise), one array so
  // that a split tile's partial sums (T T THREADS floats) fit in them
  __shared__ __align__(16) float ops[2 * 2 * BK * (E + PAD)];
  static_assert(SPLIT == 1 || T * T * THREADS <= 2 * 2 * BK * (E + PAD), "partial tile fits");
  float (*As)[BK][E + PAD] = reinterpret_cast<float (*)[BK][E + PAD]>(ops);
  float (*Bs)[BK][E + PAD] = reinterpret_cast<float (*)[BK][E + PAD]>(ops + 2 * BK * (E + PAD));
  __shared__ float red[THREADS / 32];

  const int N = d.N, ld = d.ld;
  int tm, tn;
  tile_raster(tile, d.tiles_n, d.tiles_n, &tm, &tn);  // square tiles
  const int m0 = tm * E, n0 = tn * E;
  const float* __restrict__ X = (const float*)d.X;
  const float* __restrict__ Y = (const float*)d.Y;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // loader coordinates: X tile E rows x 16 k as float4 along k (rows xr + 64 h);
  // Y tile 16 k x E cols as float4 along n (k rows yk + (1024 / E) h)
  const int xr = tid >> 2, xq = tid & 3;
  const int yk = tid / (E / 4), yc = tid % (E / 4);

  float4 xa[H], yb[H];
  auto load_tile = [&](int k0) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
      int r = m0 + xr + 64 * h, k = k0 + 4 * xq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < N && k < N) {
        v = *reinterpret_cast<const float4*>(X + (size_t)r * ld + k);
        if (k + 1 >= N) v.y = 0.f;
        if (k + 2 >= N) v.z = 0.f;
        if (k + 3 >= N) v.w = 0.f;
      }
      xa[h] = v;
      int kk = k0 + yk + (1024 / E) * h, c = n0 + 4 * yc;
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (kk < N && c < N) {
        w = *reinterpret_cast<const float4*>(Y + (size_t)kk * ld + c);
        if (c + 1 >= N) w.y = 0.f;
        if (c + 2 >= N) w.z = 0.f;
        if (c + 3 >= N) w.w = 0.f;
      }
      yb[h] = w;
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int h = 0; h < H; ++h) {
      int r = xr + 64 * h;
      As[buf][4 * xq + 0][r] = xa[h].x;
      As[buf][4 * xq + 1][r] = xa[h].y;
      As[buf][4 * xq + 2][r] = xa[h].z;
      As[buf][4 * xq + 3][r] = xa[h].w;
      *reinterpret_cast<float4*>(&Bs[buf][yk + (1024 / E) * h][4 * yc]) = yb[h];
    }
  };

  float acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) acc[i][j] = 0.f;

  const int KT = (N + BK - 1) / BK;
  int kt0 = 0, kt1 = KT;
  uint32_t rank = 0;
  if constexpr (SPLIT == 2) {
    rank = ctarank();
    const int half = (KT + 1) / 2;
    kt0 = rank == 0 ? 0 : half;
    kt1 = rank == 0 ? half : KT;
  }
  load_tile(kt0 * BK);  // past N it loads zeros
  store_tile(0);
  __syncthreads();
  for (int kt = kt0; kt < kt1; ++kt) {
    const int buf = (kt - kt0) & 1;
    if (kt + 1 < kt1) load_tile((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[T], b[T];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const float4 av = *reinterpret_cast<const float4*>(&As[buf][k][64 * h + 4 * ty]);
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][k][64 * h + 4 * tx]);
        a[4 * h] = av.x; a[4 * h + 1] = av.y; a[4 * h + 2] = av.z; a[4 * h + 3] = av.w;
        b[4 * h] = bv.x; b[4 * h + 1] = bv.y; b[4 * h + 2] = bv.z; b[4 * h + 3] = bv.w;
      }
#pragma unroll
      for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < kt1) store_tile(buf ^ 1);
    __syncthreads();
  }
  if constexpr (SPLIT == 2) {
    cluster_barrier();  // both k-loops are done: rank 0's operand buffers are free
    if (rank == 1) {
      const uint32_t dst = peer(ops, 0);
#pragma unroll
      for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j)
          asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(dst + (uint32_t)(((i * T + j) * THREADS + tid) * 4)),
                       "f"(acc[i][j])
                       : "memory");
    }
    cluster_barrier();  // rank 1's partial tile is visible in rank 0's shared memory
    if (rank == 1) return;
#pragma unroll
    for (int i = 0; i < T; ++i)
#pragma unroll
      for (int j = 0; j < T; ++j) acc[i][j] += ops[(i * T + j) * THREADS + tid];
  }

  // ---- epilogue: lagged scale, store, max
  const int sx = scale_exp_from_bits(scales[d.sx].maxbits);
  const int sy = scale_exp_from_bits(scales[d.sy].maxbits);
  const int sh = -(sx + sy);
  const long long Ec = scales[d.sx].E + scales[d.sy].E + sx + sy;
  if (tile == 0 && tid == 0) {
    if (d.mode == OUT_INTERNAL) scales[d.sc].E = Ec;
    if (d.mode == OUT_USER_MANT && d.out_log2) *d.out_log2 = Ec;
  }
  float m = 0.f;
#pragma unroll
  for (int i = 0; i < T; ++i) {
    const int r = m0 + 64 * (i / 4) + 4 * ty + (i & 3);
    if (r >= N) continue;
#pragma unroll
    for (int hb = 0; hb < H; ++hb) {
      const int c = n0 + 64 * hb + 4 * tx;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = mul_pow2(acc[i][4 * hb + j], sh);
      if (d.mode == OUT_INTERNAL) {
        float* C = (float*)d.C + (size_t)r * ld;
        if (c + 3 < N) {
          *reinterpret_cast<float4*>(C + c) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c + j < N) C[c + j] = v[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < N) m = fmaxf(m, fabsf(v[j]));
      } else {
        float* O = (float*)d.out + (size_t)r * N;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < N) O[c + j] = d.mode == OUT_USER_MANT ? v[j] : final_value(v[j], Ec, status);
      }
    }
  }
  if (d.mode == OUT_INTERNAL) {
    m = warp_max(m);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    if (tid < 32) {
      m = tid < THREADS / 32 ? red[tid] : 0.f;
      m = warp_max(m);
      if (tid == 0 && m > 0.f) atomicMax(&scales[d.sc].maxbits, __float_as_uint(m));
    }
  }
}

template <int E>
__global__ void __launch_bounds__(simt::THREADS, 2)
    simt_pair_kernel(const GemmPair g, Scale* scales, unsigned* status) {
  int t = blockIdx.x;
  int which = (g.count > 1 && t >= g.d[1].tile_begin) ? 1 : 0;
  simt_tile<E>(g.d[which], t - g.d[which].tile_begin, scales, status);
}

// 64-wide tiles split over clusters of two CTAs (CTAs 2 t and 2 t + 1: tile t)
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(simt::THREADS, 2)
    simt_pair_split_kernel(const GemmPair g, Scale* scales, unsigned* status) {
  int t = blockIdx.x >> 1;
  int which = (g.count > 1 && t >= g.d[1].tile_begin) ? 1 : 0;
  simt_tile<64, 2>(g.d[which], t - g.d[which].tile_begin, scales, status);
}

template <int E>
__global__ void __launch_bounds__(simt::THREADS, 2)
    simt_group_kernel(const GemmDesc* __restrict__ descs, int count, Scale* scales,
                      unsigned* status) {
  int t = blockIdx.x;
  int lo = 0, hi = count - 1;  // last desc with tile_begin <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  GemmDesc d = descs[lo];
  simt_tile<E>(d, t - d.tile_begin, scales, status);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(simt::THREADS, 2)
    simt_group_split_kernel(const GemmDesc* __restrict__ descs, int count, Scale* scales, unsigned* status) {
  int t = blockIdx.x >> 1;
  int lo = 0, hi = count - 1;  // last desc with tile_begin <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  GemmDesc d = descs[lo];
  simt_tile<64, 2>(d, t - d.tile_begin, scales, status);
}

cudaError_t launch_simt_pair(const GemmPair& g, int edge, int split, Scale* scales, unsigned* status,
                             cudaStream_t s) {
  if (edge == 64 && split == 2)
    simt_pair_split_kernel<<<2 * g.tiles_total, simt::THREADS, 0, s>>>(g, scales, status);
  else if (edge == 64)
    simt_pair_kernel<64><<<g.tiles_total, simt::THREADS, 0, s>>>(g, scales, status);
  else
    simt_pair_kernel<128><<<g.tiles_total, simt::THREADS, 0, s>>>(g, scales, status);
  return cudaGetLastError();
}

cudaError_t launch_simt_group(const GemmDesc* d_descs, int count, int tiles_total, int edge, int split,
                              Scale* scales, unsigned* status, cudaStream_t s) {
  if (edge == 64 && split == 2)
    simt_group_split_kernel<<<2 * tiles_total, simt::THREADS, 0, s>>>(d_descs, count, scales, status);
  else if (edge == 64)
    simt_group_kernel<64><<<tiles_total, simt::THREADS, 0, s>>>(d_descs, count, scales, status);
  else
    simt_group_kernel<128><<<tiles_total, simt::THREADS, 0, s>>>(d_descs, count, scales, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Whole chain for N <= 64 in one CTA: P, R and a temporary T (64x64 float32
// each, zero-padded) live in shared memory for the entire power.  Every
// product is stored with an exact power-of-two scaling taken from its
// operands' maxima, the exponent carried in a 64-bit integer.

namespace tiny {
constexpr int NMAX = 64, LDS = 68, THREADS = 256;
}

int tiny_max_supported() { return tiny::NMAX; }

// Thread layout of a 64 x 64 product: thread t owns rows 4 (t / 16) + 0..3
// and columns 4 (t % 16) + 0..3.  Per 4-deep k-step it reads 4 float4 of X
// and 4 float4 of Y and makes 64 FMAs.  (One CTA of this kind is bound by
// shared-memory operand delivery near 1.8 us per product; wider register
// tiles, a split k range or warp-wide broadcasts of X measured no faster.)
__device__ __forceinline__ void tiny_load(const float* Xs, const float* Ys, int k, int r0, int c0, float4* a,
                                          float4* b) {
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(Xs + (r0 + i) * tiny::LDS + k);
#pragma unroll
  for (int q = 0; q < 4; ++q) b[q] = *reinterpret_cast<const float4*>(Ys + (k + q) * tiny::LDS + c0);
}

__device__ __forceinline__ void tiny_fma(const float4* a, const float4* b, float (*acc)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[i][0] = fmaf(av[q], b[q].x, acc[i][0]);
      acc[i][1] = fmaf(av[q], b[q].y, acc[i][1]);
      acc[i][2] = fmaf(av[q], b[q].z, acc[i][2]);
      acc[i][3] = fmaf(av[q], b[q].w, acc[i][3]);
    }
  }
}

// dst <- (Xs Ys) 2^shift, an exact power-of-two rescaling; this thread's
// share of max|dst| goes to red[warp].  Every output is one fmaf chain over
// ascending k.  dst is neither Xs nor Ys; the caller synchronises.
__device__ __forceinline__ void tiny_mul(const float* Xs, const float* Ys, float* dst, int kmax, int shift,
                                         float* red) {
  using namespace tiny;
  const int tid = threadIdx.x;
  const int r0 = 4 * (tid >> 4), c0 = 4 * (tid & 15);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  // Two operand sets in ping-pong: the next k-step's operands load while
  // this one's FMAs issue (the last step reloads its own: nothing is read
  // past row or column kmax - 1).
  float4 a0[4], b0[4], a1[4], b1[4];
  tiny_load(Xs, Ys, 0, r0, c0, a0, b0);
  for (int k = 0; k < kmax; k += 8) {
    tiny_load(Xs, Ys, k + 4 < kmax ? k + 4 : k, r0, c0, a1, b1);
    tiny_fma(a0, b0, acc);
    if (k + 4 >= kmax) break;
    tiny_load(Xs, Ys, k + 8 < kmax ? k + 8 : k + 4, r0, c0, a0, b0);
    tiny_fma(a1, b1, acc);
  }
  float m = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 v = make_float4(mul_pow2(acc[i][0], shift), mul_pow2(acc[i][1], shift),
                                 mul_pow2(acc[i][2], shift), mul_pow2(acc[i][3], shift));
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    *reinterpret_cast<float4*>(dst + (r0 + i) * LDS + c0) = v;
  }
  m = warp_max(m);
  if ((tid & 31) == 0) red[tid >> 5] = m;
}

// ---- four-CTA cluster form of the same chain (single powers): each CTA of a
// 2 x 2 cluster computes one 32 x 32 quadrant of every product and stores it
// into all four CTAs' copies of the result through distributed shared memory.
namespace tinyc {
constexpr int C = 4;
__device__ __forceinline__ uint32_t ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of the four CTAs executes the same sequence of these barriers
// (once after the set-up and once per product), so none waits for a thread
// that never arrives.
__device__ __forceinline__ void barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t peer(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_v2(uint32_t a, float x, float y) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ void st_f32(uint32_t a, float x) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(x) : "memory");
}
}  // namespace tinyc

// Quadrant (rq, cq) of dst <- (Xs Ys) 2^shift in every CTA of the cluster;
// thread t owns rows rq + 2 (t / 16) + 0..1 and columns cq + 2 (t % 16) + 0..1
// (one fmaf chain over ascending k per output, as in tiny_mul, so both forms
// give identical bits).  Each warp's max|.| goes to red[8 rank + warp] of
// every CTA.  The caller runs the cluster barrier after the call.
__device__ __forceinline__ void tinyc_mul(const float* Xs, const float* Ys, float* dst, int kmax, int shift,
                                          float* red, uint32_t rank) {
  using namespace tiny;
  const int tid = threadIdx.x;
  const int r = 32 * (int)(rank >> 1) + 2 * (tid >> 4), c = 32 * (int)(rank & 1) + 2 * (tid & 15);
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k = 0; k < kmax; k += 4) {
    const float4 a0 = *reinterpret_cast<const float4*>(Xs + r * LDS + k);
    const float4 a1 = *reinterpret_cast<const float4*>(Xs + (r + 1) * LDS + k);
    float2 b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = *reinterpret_cast<const float2*>(Ys + (k + q) * LDS + c);
    const float av[2][4] = {{a0.x, a0.y, a0.z, a0.w}, {a1.x, a1.y, a1.z, a1.w}};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[i][0] = fmaf(av[i][q], b[q].x, acc[i][0]);
        acc[i][1] = fmaf(av[i][q], b[q].y, acc[i][1]);
      }
  }
  float m = 0.f;
  float v[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    v[i][0] = mul_pow2(acc[i][0], shift);
    v[i][1] = mul_pow2(acc[i][1], shift);
    m = fmaxf(m, fmaxf(fabsf(v[i][0]), fabsf(v[i][1])));
  }
  *reinterpret_cast<float2*>(dst + r * LDS + c) = make_float2(v[0][0], v[0][1]);
  *reinterpret_cast<float2*>(dst + (r + 1) * LDS + c) = make_float2(v[1][0], v[1][1]);
#pragma unroll
  for (uint32_t p = 1; p < (uint32_t)tinyc::C; ++p) {
    const uint32_t q = (rank + p) % tinyc::C;
    tinyc::st_v2(tinyc::peer(dst + r * LDS + c, q), v[0][0], v[0][1]);
    tinyc::st_v2(tinyc::peer(dst + (r + 1) * LDS + c, q), v[1][0], v[1][1]);
  }
  m = warp_max(m);
  if ((tid & 31) == 0) {
    red[8 * rank + (tid >> 5)] = m;
#pragma unroll
    for (uint32_t p = 1; p < (uint32_t)tinyc::C; ++p)
      tinyc::st_f32(tinyc::peer(red + 8 * rank + (tid >> 5), (rank + p) % tinyc::C), m);
  }
}

// frexp exponent of the maximum gathered in red[W] (after a barrier).
template <int W>
__device__ __forceinline__ int tiny_red_exp(const float* red) {
  float m = red[0];
#pragma unroll
  for (int w = 1; w < W; ++w) m = fmaxf(m, red[w]);
  return scale_exp_from_bits(__float_as_uint(m));
}

// Every stored matrix S carries E (the matrix is S 2^E) and s, the frexp
// exponent of max|S|.  A product T = X Y is stored with a lagged rescaling:
//   S_T = (S_X S_Y) 2^-(s_X + s_Y),  E_T = E_X + E_Y + s_X + s_Y,
// so max|S_T| <= N, and s_T comes from the block reduction that the single
// barrier after the product completes.  The products see the same values up
// to exact powers of two as with normalised operands (one barrier per product
// instead of three).
template <bool CL>
__device__ __forceinline__ void tiny_chain(const TinyDesc& d, unsigned* status) {
  using namespace tiny;
  constexpr int W = CL ? 8 * tinyc::C : THREADS / 32;  // maxima gathered per product
  extern __shared__ __align__(16) float sm[];
  float* P = sm;
  float* R = sm + NMAX * LDS;
  float* T = sm + 2 * NMAX * LDS;
  __shared__ float red[2][W];  // alternate per product
  const int tid = threadIdx.x;
  const uint32_t rank = CL ? tinyc::ctarank() : 0u;
  const int N = d.N;
  const float* __restrict__ A = d.A;
  const int kmax = (N + 3) & ~3;

  // P = A normalised (E = frexp exponent of max|A|, so s = 0).  All of this
  // thread's loads of A are issued before any is used (one memory round trip).
  constexpr int PER = NMAX * NMAX / THREADS;
  const int NN = N * N;
  float v[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = tid + j * THREADS;
    v[j] = i < NN ? A[i] : 0.f;
  }
  for (int i = tid; i < NMAX * LDS; i += THREADS) {
    int r = i / LDS, c = i - r * LDS;
    if (r >= N || c >= N) P[i] = 0.f;
    R[i] = (r == c && r < N) ? 1.f : 0.f;
  }
  float m = 0.f;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    bad |= !isfinite(v[j]);
    m = fmaxf(m, fabsf(v[j]));
  }
  m = warp_max(m);
  if ((tid & 31) == 0) red[0][tid >> 5] = m;
  if (__syncthreads_or(bad) && tid == 0 && rank == 0) atomicOr(status, ST_BADINPUT);
  long long eP = tiny_red_exp<THREADS / 32>(red[0]), eR = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = tid + j * THREADS;
    if (i < NN) {
      const int r = i / N, c = i - r * N;
      P[r * LDS + c] = mul_pow2(v[j], -(int)eP);
    }
  }
  int sP = 0, sR = 0;
  if (CL)
    tinyc::barrier();  // every CTA has started and set up before any remote store
  else
    __syncthreads();

  bool haveR = false;
  int rb = 1;  // red buffer of the next product
  unsigned long long bits = d.n;
  while (bits) {
    if (bits & 1ull) {
      if (!haveR) {
        for (int i = tid; i < NMAX * LDS; i += THREADS) R[i] = P[i];
        eR = eP;
        sR = sP;
        haveR = true;
        __syncthreads();
      } else {
        if (CL) {
          tinyc_mul(R, P, T, kmax, -(sR + sP), red[rb], rank);
          tinyc::barrier();
        } else {
          tiny_mul(R, P, T, kmax, -(sR + sP), red[rb]);
          __syncthreads();
        }
        eR = eR + eP + sR + sP;
        sR = tiny_red_exp<W>(red[rb]);
        rb ^= 1;
        float* t = R; R = T; T = t;
      }
    }
    bits >>= 1;
    if (bits) {
      if (CL) {
        tinyc_mul(P, P, T, kmax, -2 * sP, red[rb], rank);
        tinyc::barrier();
      } else {
        tiny_mul(P, P, T, kmax, -2 * sP, red[rb]);
        __syncthreads();
      }
      eP = 2 * eP + 2 * sP;
      sP = tiny_red_exp<W>(red[rb]);
      rb ^= 1;
      float* t = P; P = T; T = t;
    }
  }
  // n == 0: R is the identity with exponent 0 (sR = 0: max|I| = 1 -> frexp 1;
  // written as is); otherwise the mantissa S_R 2^-s_R, exponent E_R + s_R
  const int shift = haveR ? -sR : 0;
  const long long eOut = haveR ? eR + sR : 0;
  if (d.log2 && tid == 0 && rank == 0) *d.log2 = eOut;
  // the cluster's CTAs write row blocks of 16 (no remote store follows the
  // last barrier, so a CTA may exit while the others still write)
  const int rbeg = CL ? 16 * (int)rank : 0, rend = CL ? min(N, rbeg + 16) : N;
  for (int i = rbeg * N + tid; i < rend * N; i += THREADS) {
    int r = i / N, c = i - r * N;
    float v = mul_pow2(R[r * LDS + c], shift);
    d.out[i] = d.log2 ? v : final_value(v, eOut, status);
  }
}

__global__ void __cluster_dims__(tinyc::C, 1, 1) __launch_bounds__(tiny::THREADS, 1)
    tiny_cluster_kernel(const TinyDesc d, unsigned* status) {
  tiny_chain<true>(d, status);
}

__global__ void __launch_bounds__(tiny::THREADS, 1) tiny_one_kernel(const TinyDesc d, unsigned* status) {
  tiny_chain<false>(d, status);
}

__global__ void __launch_bounds__(tiny::THREADS, 1)
    tiny_group_kernel(const TinyDesc* __restrict__ descs, unsigned* status) {
  TinyDesc d = descs[blockIdx.x];
  tiny_chain<false>(d, status);
}

static constexpr int kTinySmem = 3 * tiny::NMAX * tiny::LDS * (int)sizeof(float);

cudaError_t tiny_attrs() {
  cudaError_t e = cudaFuncSetAttribute(tiny_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kTinySmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tiny_one_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTinySmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tiny_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kTinySmem);
}

cudaError_t launch_tiny_one(const TinyDesc& d, unsigned* status, cudaStream_t s) {
  // Up to N = 32 a product is cheaper than the cluster's exchange and barrier.
  if (d.N > 32)
    tiny_cluster_kernel<<<tinyc::C, tiny::THREADS, kTinySmem, s>>>(d, status);
  else
    tiny_one_kernel<<<1, tiny::THREADS, kTinySmem, s>>>(d, status);
  return cudaGetLastError();
}

cudaError_t launch_tiny_group(const TinyDesc* d_descs, int count, unsigned* status, cudaStream_t s) {
  tiny_group_kernel<<<count, tiny::THREADS, kTinySmem, s>>>(d_descs, status);
  return cudaGetLastError();
}

}  // namespace mp
