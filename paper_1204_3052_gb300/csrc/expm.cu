// The matrix exponential e^A on the same squaring chain (scaling and
// squaring: Moler and Van Loan, "Nineteen dubious ways to compute the
// exponential of a matrix, twenty-five years later", SIAM Review 45 (2003),
// method 3).  arXiv 1204.3052's "matrix exponentiation" is A^n (Sec. 4.3);
// e^A is the other common meaning, and its cost is dominated by the same
// products and squarings:
//
//   s  = max(0, ceil(log2 ||A||_1))        (||A||_1: largest column sum)
//   B  = A 2^-s                             (exact), so ||B||_1 <= 1
//   T  = sum_{k <= 11} B^k / k!             (truncation < 1/12! ~ 2e-9 relative)
//      = P0 + B^4 (P1 + B^4 P2),  Pj = sum_{i < 4} B^i / (4j + i)!
//        (Paterson and Stockmeyer 1973: five products B^2, B^3, B^4 and two
//        outer ones instead of ten in Horner's rule)
//   e^A = T^(2^s)                           (matpow_f32: s squarings)
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "plan.h"

#define CK(plan, call)                                        \
  do {                                                        \
    cudaError_t ck_e = (call);                                \
    if (ck_e != cudaSuccess) return mp::cuda_fail(plan, ck_e, #call); \
  } while (0)

namespace mp {

namespace {

constexpr int kMats = 7;  // B, B^2, B^3, B^4, P0, P1, P2 (later Q, P1 + Q, R, T)

// Largest column sum of |A| (float64 sums); a non-finite entry makes it NaN
// or inf, whose bits exceed every finite value's.
__global__ void expm_norm1_kernel(const float* __restrict__ A, int N, unsigned* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += fabs((double)A[(size_t)i * N + j]);
  const float f = (float)s;
  atomicMax(out, isnan(f) ? 0x7fffffffu : __float_as_uint(f));
}

__global__ void expm_scale_kernel(const float* __restrict__ A, float* __restrict__ B, size_t n, int k) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    B[i] = mul_pow2(A[i], k);
}

struct Coef {
  double c[12];  // 1 / k!, k = 0 .. 11
};

// Pj = c[4j] I + c[4j+1] B + c[4j+2] B^2 + c[4j+3] B^3, summed in float64.
__global__ void expm_combo_kernel(const float* __restrict__ B, const float* __restrict__ B2,
                                  const float* __restrict__ B3, float* P0, float* P1, float* P2, int N,
                                  const Coef co) {
  const size_t n = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double d = (i / N == i % N) ? 1.0 : 0.0;
    const double b = B[i], b2 = B2[i], b3 = B3[i];
    float* P[3] = {P0, P1, P2};
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[j][i] = (float)(co.c[4 * j] * d + co.c[4 * j + 1] * b + co.c[4 * j + 2] * b2 + co.c[4 * j + 3] * b3);
  }
}

__global__ void expm_add_kernel(const float* __restrict__ X, const float* __restrict__ Y, float* Z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Z[i] = X[i] + Y[i];
}

// C = X Y for N <= 64: one thread per output, one fmaf chain over ascending k.
__global__ void expm_small_product_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                          float* __restrict__ C, int N) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= N) return;
  float acc = 0.f;
  for (int k = 0; k < N; ++k) acc = fmaf(X[(size_t)i * N + k], Y[(size_t)k * N + j], acc);
  C[(size_t)i * N + j] = acc;
}

int grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

matpow_status product(matpow_plan_s* p, const float* X, const float* Y, int N, float* out, cudaStream_t s) {
  if (N <= 64 && N <= p->tiny_max) {
    expm_small_product_kernel<<<N, 64, 0, s>>>(X, Y, out, N);
    CK(p, cudaGetLastError());
    p->launches++;
    return MATPOW_OK;
  }
  return enqueue_product_f32(p, X, Y, N, out, s);
}

}  // namespace
}  // namespace mp

using namespace mp;

extern "C" matpow_status matpow_expm(matpow_plan_t p, const float* dA, int N, float* dOut, int64_t* dLog2Scale,
                                     void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_expm: plan is NULL");
  if (N < 0 || N > p->max_n) return fail(p, MATPOW_EINVAL, "matpow_expm: N=%d outside [0, %d]", N, p->max_n);
  if (N == 0) return MATPOW_OK;
  if (!dA || !dOut) return fail(p, MATPOW_EINVAL, "matpow_expm: NULL matrix pointer");
  if (((uintptr_t)dA & 3) || ((uintptr_t)dOut & 3) || ((uintptr_t)dLog2Scale & 7))
    return fail(p, MATPOW_EINVAL, "matpow_expm: misaligned pointer");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  struct Restore {
    int dev;
    ~Restore() {
      int cur = 0;
      cudaGetDevice(&cur);
      if (cur != dev) cudaSetDevice(dev);
    }
  } restore{prev};
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)N * N, cap = (size_t)p->max_n * p->max_n;
  if (!p->expm_ws) {
    cudaError_t e = cudaMalloc(&p->expm_ws, kMats * cap * sizeof(float) + 256);
    if (e != cudaSuccess) {
      p->expm_ws = nullptr;
      return fail(p, MATPOW_ENOMEM, "matpow_expm: scratch of %zu bytes", kMats * cap * sizeof(float) + 256);
    }
  }
  float* M[kMats];
  for (int i = 0; i < kMats; ++i) M[i] = p->expm_ws + (size_t)i * cap;
  unsigned* dnorm = (unsigned*)(p->expm_ws + (size_t)kMats * cap);

  // s from ||A||_1 (read back: it fixes the number of squarings)
  CK(p, cudaMemsetAsync(dnorm, 0, sizeof(unsigned), s));
  expm_norm1_kernel<<<(N + 127) / 128, 128, 0, s>>>(dA, N, dnorm);
  CK(p, cudaGetLastError());
  p->launches++;
  unsigned hbits = 0;
  CK(p, cudaMemcpyAsync(&hbits, dnorm, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(p, cudaStreamSynchronize(s));
  float nrm;
  std::memcpy(&nrm, &hbits, sizeof nrm);
  if (!std::isfinite(nrm)) return fail(p, MATPOW_EINVAL, "matpow_expm: non-finite input");
  int sq = 0;
  if (nrm > 1.0f) sq = (int)std::ceil(std::log2((double)nrm));
  while (sq > 0 && std::ldexp((double)nrm, -(sq - 1)) <= 1.0) --sq;  // smallest s with ||A|| 2^-s <= 1
  while (std::ldexp((double)nrm, -sq) > 1.0) ++sq;
  if (sq > 62) return fail(p, MATPOW_EINVAL, "matpow_expm: ||A||_1 = %g is beyond 2^62", (double)nrm);

  // B = A 2^-s; B^2, B^3, B^4; the three Pj
  expm_scale_kernel<<<grid_for(nn), 256, 0, s>>>(dA, M[0], nn, -sq);
  CK(p, cudaGetLastError());
  p->launches++;
  matpow_status st;
  if ((st = product(p, M[0], M[0], N, M[1], s)) != MATPOW_OK) return st;  // B^2
  if ((st = product(p, M[1], M[0], N, M[2], s)) != MATPOW_OK) return st;  // B^3
  if ((st = product(p, M[1], M[1], N, M[3], s)) != MATPOW_OK) return st;  // B^4
  Coef co;
  double f = 1.0;
  for (int k = 0; k < 12; ++k) {
    if (k > 0) f *= k;
    co.c[k] = 1.0 / f;
  }
  expm_combo_kernel<<<grid_for(nn), 256, 0, s>>>(M[0], M[1], M[2], M[4], M[5], M[6], N, co);
  CK(p, cudaGetLastError());
  p->launches++;
  // T = P0 + B^4 (P1 + B^4 P2)
  if ((st = product(p, M[3], M[6], N, M[0], s)) != MATPOW_OK) return st;  // Q = B^4 P2
  expm_add_kernel<<<grid_for(nn), 256, 0, s>>>(M[5], M[0], M[5], nn);     // P1 + Q
  CK(p, cudaGetLastError());
  if ((st = product(p, M[3], M[5], N, M[1], s)) != MATPOW_OK) return st;  // R
  expm_add_kernel<<<grid_for(nn), 256, 0, s>>>(M[4], M[1], M[2], nn);     // T = P0 + R
  CK(p, cudaGetLastError());
  p->launches += 2;
  // e^A = T^(2^s)
  if (sq == 0) {
    CK(p, launch_copy(M[2], dOut, N, (long long*)dLog2Scale, s));
    p->launches++;
    return MATPOW_OK;
  }
  return matpow_f32(p, M[2], N, 1ull << sq, dOut, dLog2Scale, stream);
}
