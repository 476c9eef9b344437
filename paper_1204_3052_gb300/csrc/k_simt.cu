// Float32 SIMT products on the CUDA cores.
//
//  * simt_gemm: C = X * Y for stored float32 matrices (arXiv 1204.3052
//    Sec. 4.1's c_ij = sum_k x_ik y_kj), tiled through shared memory
//    (Sec. 4.3.2, 4.3.7) with 128-bit vector loads (Sec. 4.3.5) and coalesced
//    row-major access (Sec. 4.3.3).  On sm_103a: a 128x128 CTA tile, 16-deep
//    k-steps double-buffered in shared memory, an 8x8 register tile per
//    thread.  The epilogue applies the lagged power-of-two scale of the
//    operands, writes the stored result (or the user's float32 output) and
//    folds max|C| into the result's scale slot.
//  * tiny_chain: the whole square-and-multiply chain (Sec. 4.3) for N <= 64
//    in one CTA, with every partial product in shared memory.
#include "internal.cuh"

namespace mp {

namespace simt {
constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8;
constexpr int THREADS = (BM / TM) * (BN / TN);  // 256
constexpr int PAD = 4;
}  // namespace simt

int simt_tile_edge() { return simt::BM; }

// One 128x128 tile of one product.
__device__ __forceinline__ void simt_tile(const GemmDesc& d, int tile, Scale* scales,
                                          unsigned* status) {
  using namespace simt;
  __shared__ __align__(16) float As[2][BK][BM + PAD];
  __shared__ __align__(16) float Bs[2][BK][BN + PAD];
  __shared__ float red[THREADS / 32];

  const int N = d.N, ld = d.ld;
  int tm, tn;
  tile_raster(tile, d.tiles_n, d.tiles_n, &tm, &tn);  // square tiles
  const int m0 = tm * BM, n0 = tn * BN;
  const float* __restrict__ X = (const float*)d.X;
  const float* __restrict__ Y = (const float*)d.Y;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  // loader coordinates: X tile 128 rows x 16 k as float4 along k
  const int xr = tid >> 2, xq = tid & 3;  // rows xr, xr+64; k quad xq
  // Y tile 16 k x 128 cols as float4 along n
  const int yk = tid >> 5, yc = tid & 31;  // k rows yk, yk+8; col quad yc

  float4 xa[2], yb[2];
  auto load_tile = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int r = m0 + xr + 64 * h, k = k0 + 4 * xq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < N && k < N) {
        v = *reinterpret_cast<const float4*>(X + (size_t)r * ld + k);
        if (k + 1 >= N) v.y = 0.f;
        if (k + 2 >= N) v.z = 0.f;
        if (k + 3 >= N) v.w = 0.f;
      }
      xa[h] = v;
      int kk = k0 + yk + 8 * h, c = n0 + 4 * yc;
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
    for (int h = 0; h < 2; ++h) {
      int r = xr + 64 * h;
      As[buf][4 * xq + 0][r] = xa[h].x;
      As[buf][4 * xq + 1][r] = xa[h].y;
      As[buf][4 * xq + 2][r] = xa[h].z;
      As[buf][4 * xq + 3][r] = xa[h].w;
      *reinterpret_cast<float4*>(&Bs[buf][yk + 8 * h][4 * yc]) = yb[h];
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const int KT = (N + BK - 1) / BK;
  load_tile(0);
  store_tile(0);
  __syncthreads();
  for (int kt = 0; kt < KT; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < KT) load_tile((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[TM], b[TN];
      float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * ty]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tx]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * tx]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < KT) store_tile(buf ^ 1);
    __syncthreads();
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
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
    if (r >= N) continue;
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
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

__global__ void __launch_bounds__(simt::THREADS, 2)
    simt_pair_kernel(const GemmPair g, Scale* scales, unsigned* status) {
  int t = blockIdx.x;
  int which = (g.count > 1 && t >= g.d[1].tile_begin) ? 1 : 0;
  simt_tile(g.d[which], t - g.d[which].tile_begin, scales, status);
}

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
  simt_tile(d, t - d.tile_begin, scales, status);
}

cudaError_t launch_simt_pair(const GemmPair& g, Scale* scales, unsigned* status, cudaStream_t s) {
  simt_pair_kernel<<<g.tiles_total, simt::THREADS, 0, s>>>(g, scales, status);
  return cudaGetLastError();
}

cudaError_t launch_simt_group(const GemmDesc* d_descs, int count, int tiles_total, Scale* scales,
                              unsigned* status, cudaStream_t s) {
  simt_group_kernel<<<tiles_total, simt::THREADS, 0, s>>>(d_descs, count, scales, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Whole chain for N <= 64 in one CTA: P, R and a temporary T (64x64 float32
// each, zero-padded) live in shared memory for the entire power.  Every
// product is followed by an exact power-of-two renormalisation (max|.| in
// [0.5, 1)) with the exponent carried in a 64-bit integer.

namespace tiny {
constexpr int NMAX = 64, LDS = 68, THREADS = 256;
}

int tiny_max_supported() { return tiny::NMAX; }

// dst <- normalise(Xs * Ys); returns the applied exponent.  256 threads, each
// owns a 4x4 block of the 64x64 result.
__device__ __forceinline__ int tiny_mul(const float* Xs, const float* Ys, float* dst, int kmax,
                                        float* red) {
  using namespace tiny;
  const int tid = threadIdx.x;
  const int r0 = 4 * (tid >> 4), c0 = 4 * (tid & 15);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k = 0; k < kmax; k += 4) {
    float4 a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(Xs + (r0 + i) * LDS + k);
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = *reinterpret_cast<const float4*>(Ys + (k + q) * LDS + c0);
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
  float m = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) m = fmaxf(m, fabsf(acc[i][j]));
  m = warp_max(m);
  __syncthreads();  // all reads of Xs/Ys done before dst (which may alias) is written
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
#pragma unroll
  for (int w = 1; w < THREADS / 32; ++w) m = fmaxf(m, red[w]);
  const int s = scale_exp_from_bits(__float_as_uint(m));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float4 v = make_float4(mul_pow2(acc[i][0], -s), mul_pow2(acc[i][1], -s), mul_pow2(acc[i][2], -s),
                           mul_pow2(acc[i][3], -s));
    *reinterpret_cast<float4*>(dst + (r0 + i) * LDS + c0) = v;
  }
  __syncthreads();
  return s;
}

__device__ __forceinline__ void tiny_chain(const TinyDesc& d, unsigned* status) {
  using namespace tiny;
  extern __shared__ __align__(16) float sm[];
  float* P = sm;
  float* R = sm + NMAX * LDS;
  float* T = sm + 2 * NMAX * LDS;
  __shared__ float red[THREADS / 32];
  __shared__ int flag;
  const int tid = threadIdx.x;
  const int N = d.N;
  const float* __restrict__ A = d.A;
  const int kmax = (N + 3) & ~3;

  if (tid == 0) flag = 0;
  for (int i = tid; i < NMAX * LDS; i += THREADS) {
    int r = i / LDS, c = i - r * LDS;
    float v = (r < N && c < N) ? A[(size_t)r * N + c] : 0.f;
    P[i] = v;
    R[i] = (r == c && r < N) ? 1.f : 0.f;
  }
  __syncthreads();
  // normalise A
  float m = 0.f;
  bool bad = false;
  for (int i = tid; i < NMAX * LDS; i += THREADS) {
    bad |= !isfinite(P[i]);
    m = fmaxf(m, fabsf(P[i]));
  }
  if (bad) atomicOr(&flag, 1);
  m = warp_max(m);
  if ((tid & 31) == 0) red[tid >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < THREADS / 32; ++w) m = fmaxf(m, red[w]);
  long long eP = scale_exp_from_bits(__float_as_uint(m));
  for (int i = tid; i < NMAX * LDS; i += THREADS) P[i] = mul_pow2(P[i], -(int)eP);
  if (tid == 0 && flag) atomicOr(status, ST_BADINPUT);
  __syncthreads();

  long long eR = 0;
  bool haveR = false;
  unsigned long long bits = d.n;
  while (bits) {
    if (bits & 1ull) {
      if (!haveR) {
        for (int i = tid; i < NMAX * LDS; i += THREADS) R[i] = P[i];
        eR = eP;
        haveR = true;
        __syncthreads();
      } else {
        int s = tiny_mul(R, P, T, kmax, red);
        float* t = R; R = T; T = t;
        eR = eR + eP + s;
      }
    }
    bits >>= 1;
    if (bits) {
      int s = tiny_mul(P, P, T, kmax, red);
      float* t = P; P = T; T = t;
      eP = 2 * eP + s;
    }
  }
  // n == 0: R is the identity with exponent 0
  if (d.log2 && tid == 0) *d.log2 = eR;
  for (int i = tid; i < N * N; i += THREADS) {
    int r = i / N, c = i - r * N;
    float v = R[r * LDS + c];
    d.out[i] = d.log2 ? v : final_value(v, eR, status);
  }
}

__global__ void __launch_bounds__(tiny::THREADS, 1) tiny_one_kernel(const TinyDesc d, unsigned* status) {
  tiny_chain(d, status);
}

__global__ void __launch_bounds__(tiny::THREADS, 1)
    tiny_group_kernel(const TinyDesc* __restrict__ descs, unsigned* status) {
  TinyDesc d = descs[blockIdx.x];
  tiny_chain(d, status);
}

static constexpr int kTinySmem = 3 * tiny::NMAX * tiny::LDS * (int)sizeof(float);

cudaError_t tiny_attrs() {
  cudaError_t e = cudaFuncSetAttribute(tiny_one_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kTinySmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tiny_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kTinySmem);
}

cudaError_t launch_tiny_one(const TinyDesc& d, unsigned* status, cudaStream_t s) {
  tiny_one_kernel<<<1, tiny::THREADS, kTinySmem, s>>>(d, status);
  return cudaGetLastError();
}

cudaError_t launch_tiny_group(const TinyDesc* d_descs, int count, unsigned* status, cudaStream_t s) {
  tiny_group_kernel<<<count, tiny::THREADS, kTinySmem, s>>>(d_descs, status);
  return cudaGetLastError();
}

}  // namespace mp
