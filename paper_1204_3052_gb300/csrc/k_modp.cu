// Exact products over the integers mod p (p <= 65536) on the CUDA cores.
//
// C = (X * Y) mod p with X, Y entries in [0, p): every product x*y < 2^32,
// and a 64-bit accumulator holds the sum of up to 2^32 of them exactly, so
// each c_ij is the exact integer sum_k x_ik y_kj (arXiv 1204.3052 Sec. 4.1)
// reduced once.  A 64x64 CTA tile, 16-deep k-steps in shared memory, a 4x4
// register tile per thread with 32x32->64-bit multiply-adds.
#include "internal.cuh"

namespace mp {

namespace modp {
constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;
}

int modp_tile_edge() { return modp::BM; }

__global__ void modp_check_convert_kernel(const unsigned* __restrict__ A, int N, int ld, unsigned p,
                                          unsigned* dst, unsigned* status) {
  size_t total = (size_t)N * ld;
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i / ld;
    int c = (int)(i - r * ld);
    unsigned v = c < N ? A[r * N + c] : 0u;
    bad |= v >= p;
    dst[i] = v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_BADINPUT);
}

cudaError_t launch_modp_check_convert(const unsigned* A, int N, unsigned p, unsigned* dst,
                                      unsigned* status, cudaStream_t s) {
  int ld = ld_for(N, FMT_U32);
  size_t total = (size_t)N * ld;
  size_t b = (total + 255) / 256;
  int grid = (int)(b < 1216 ? (b ? b : 1) : 1216);
  modp_check_convert_kernel<<<grid, 256, 0, s>>>(A, N, ld, p, dst, status);
  return cudaGetLastError();
}

__device__ __forceinline__ void modp_tile(const GemmDesc& d, int tile) {
  using namespace modp;
  __shared__ __align__(16) unsigned As[BK][BM + 4];
  __shared__ __align__(16) unsigned Bs[BK][BN + 4];
  const int N = d.N, ld = d.ld;
  const unsigned p = d.p;
  const int tm = tile / d.tiles_n, tn = tile - tm * d.tiles_n;
  const int m0 = tm * BM, n0 = tn * BN;
  const unsigned* __restrict__ X = (const unsigned*)d.X;
  const unsigned* __restrict__ Y = (const unsigned*)d.Y;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  // loaders: X 64 rows x 16 k (one uint4 per thread), Y 16 k x 64 cols (one uint4)
  const int xr = tid >> 2, xq = tid & 3;
  const int yk = tid >> 4, yc = tid & 15;

  unsigned long long acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;

  for (int k0 = 0; k0 < N; k0 += BK) {
    {
      int r = m0 + xr, k = k0 + 4 * xq;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r < N && k < N) {
        v = *reinterpret_cast<const uint4*>(X + (size_t)r * ld + k);
        if (k + 1 >= N) v.y = 0;
        if (k + 2 >= N) v.z = 0;
        if (k + 3 >= N) v.w = 0;
      }
      As[4 * xq + 0][xr] = v.x;
      As[4 * xq + 1][xr] = v.y;
      As[4 * xq + 2][xr] = v.z;
      As[4 * xq + 3][xr] = v.w;
      int kk = k0 + yk, c = n0 + 4 * yc;
      uint4 w = make_uint4(0, 0, 0, 0);
      if (kk < N && c < N) {
        w = *reinterpret_cast<const uint4*>(Y + (size_t)kk * ld + c);
        if (c + 1 >= N) w.y = 0;
        if (c + 2 >= N) w.z = 0;
        if (c + 3 >= N) w.w = 0;
      }
      *reinterpret_cast<uint4*>(&Bs[yk][4 * yc]) = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      uint4 a = *reinterpret_cast<const uint4*>(&As[k][4 * ty]);
      uint4 b = *reinterpret_cast<const uint4*>(&Bs[k][4 * tx]);
      const unsigned av[4] = {a.x, a.y, a.z, a.w};
      const unsigned bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += (unsigned long long)av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + 4 * ty + i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + 4 * tx + j;
      if (c >= N) continue;
      unsigned v = (unsigned)(acc[i][j] % p);
      if (d.mode == OUT_INTERNAL)
        ((unsigned*)d.C)[(size_t)r * ld + c] = v;
      else
        ((unsigned*)d.out)[(size_t)r * N + c] = v;
    }
  }
}

__global__ void __launch_bounds__(modp::THREADS) modp_pair_kernel(const GemmPair g) {
  int t = blockIdx.x;
  int which = (g.count > 1 && t >= g.d[1].tile_begin) ? 1 : 0;
  modp_tile(g.d[which], t - g.d[which].tile_begin);
}

__global__ void __launch_bounds__(modp::THREADS)
    modp_group_kernel(const GemmDesc* __restrict__ descs, int count) {
  int t = blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (descs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  GemmDesc d = descs[lo];
  modp_tile(d, t - d.tile_begin);
}

cudaError_t launch_modp_pair(const GemmPair& g, unsigned* status, cudaStream_t s) {
  (void)status;
  modp_pair_kernel<<<g.tiles_total, modp::THREADS, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_modp_group(const GemmDesc* d_descs, int count, int tiles_total, unsigned* status,
                              cudaStream_t s) {
  (void)status;
  modp_group_kernel<<<tiles_total, modp::THREADS, 0, s>>>(d_descs, count);
  return cudaGetLastError();
}

}  // namespace mp
