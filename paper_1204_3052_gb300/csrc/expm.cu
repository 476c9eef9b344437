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
//        (Paterson and Stockmeyer 1973: B^2, B^3, B^4 -- one matpow_batched
//        call -- and two outer products instead of ten in Horner's rule)
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

// Column sums of |A| in float64: block (x, y) adds rows 16 y .. 16 y + 15 of
// columns 256 x .. 256 x + 255 into colsum (zeroed before).
constexpr int kNormRows = 16;
__global__ void expm_colsum_kernel(const float* __restrict__ A, int N, double* colsum) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int i0 = blockIdx.y * kNormRows, i1 = min(N, i0 + kNormRows);
  double s = 0.0;
  for (int i = i0; i < i1; ++i) s += fabs((double)A[(size_t)i * N + j]);
  atomicAdd(&colsum[j], s);
}

// ||A||_1 = the largest column sum, as float bits rounded upward from the
// float64 sum (so the float never falls below the true norm and the chosen s
// keeps ||A 2^-s||_1 <= 1); a non-finite entry makes a sum NaN or inf, whose
// bits (0x7fffffff for NaN) exceed every finite value's.
__global__ void expm_colmax_kernel(const double* __restrict__ colsum, int N, unsigned* out) {
  unsigned m = 0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float f = __double2float_ru(colsum[j]);
    m = max(m, isnan(f) ? 0x7fffffffu : __float_as_uint(f));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

struct Coef {
  float c[12];  // 1 / k!, k = 0 .. 11, rounded to float32
};

// x 2^k for the exponents of this kernel (k >= -500): exact while the result
// is normal; below 2^-250 relative the term is negligible and becomes 0.
__device__ __forceinline__ float scale_pow2(float x, long long k) {
  if (k < -250) return 0.f;
  return mul_pow2(x, (int)k);
}

// B^k = M_k 2^(E_k - k s) from the powers of A in mantissa form (exact
// power-of-two rescaling); Pj = c[4j] I + c[4j+1] B + c[4j+2] B^2 +
// c[4j+3] B^3 by float32 fmaf (largest power first); B^4 written over M_4.
__global__ void expm_combo_kernel(const float* __restrict__ A, const float* __restrict__ M2,
                                  const float* __restrict__ M3, float* M4, const long long* __restrict__ E,
                                  int sq, float* P0, float* P1, float* P2, int N, const Coef co) {
  const size_t n = (size_t)N * N;
  const long long e2 = E[0] - 2LL * sq, e3 = E[1] - 3LL * sq, e4 = E[2] - 4LL * sq;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = (i / N == i % N) ? 1.f : 0.f;
    const float b = mul_pow2(A[i], -sq), b2 = scale_pow2(M2[i], e2), b3 = scale_pow2(M3[i], e3);
    M4[i] = scale_pow2(M4[i], e4);
    float* P[3] = {P0, P1, P2};
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[j][i] = fmaf(co.c[4 * j + 3], b3, fmaf(co.c[4 * j + 2], b2, fmaf(co.c[4 * j + 1], b, co.c[4 * j] * d)));
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

matpow_status product(matpow_plan_s* p, const float* X, const float* Y, int N, float* out, cudaStream_t s,
                      bool keep_x = false) {
  if (N <= 64 && N <= p->tiny_max) {
    expm_small_product_kernel<<<N, 64, 0, s>>>(X, Y, out, N);
    CK(p, cudaGetLastError());
    p->launches++;
    return MATPOW_OK;
  }
  return enqueue_product_f32(p, X, Y, N, out, s, keep_x);
}

// B^4, P0 .. P2, T = P0 + B^4 (P1 + B^4 P2), e^A = T^(2^sq) on stream s.
matpow_status expm_tail(matpow_plan_s* p, const float* dA, int N, float* const* M, const long long* E, int sq,
                        float* dOut, int64_t* dLog2Scale, cudaStream_t s) {
  const size_t nn = (size_t)N * N;
  // B^4 and the three Pj
  Coef co;
  double f = 1.0;
  for (int k = 0; k < 12; ++k) {
    if (k > 0) f *= k;
    co.c[k] = (float)(1.0 / f);
  }
  expm_combo_kernel<<<grid_for(nn), 256, 0, s>>>(dA, M[1], M[2], M[3], E, sq, M[4], M[5], M[6], N, co);
  CK(p, cudaGetLastError());
  p->launches++;
  matpow_status st;
  // T = P0 + B^4 (P1 + B^4 P2)
  if ((st = product(p, M[3], M[6], N, M[0], s)) != MATPOW_OK) return st;  // Q = B^4 P2
  expm_add_kernel<<<grid_for(nn), 256, 0, s>>>(M[5], M[0], M[5], nn);     // P1 + Q
  CK(p, cudaGetLastError());
  if ((st = product(p, M[3], M[5], N, M[1], s, true)) != MATPOW_OK) return st;  // R (B^4 still split)
  expm_add_kernel<<<grid_for(nn), 256, 0, s>>>(M[4], M[1], M[2], nn);     // T = P0 + R
  CK(p, cudaGetLastError());
  p->launches += 2;
  // e^A = T^(2^s)
  if (sq == 0) {
    CK(p, launch_copy(M[2], dOut, N, (long long*)dLog2Scale, s));
    p->launches++;
    return MATPOW_OK;
  }
  return matpow_f32(p, M[2], N, 1ull << sq, dOut, dLog2Scale, s);
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
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(p, cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return fail(p, MATPOW_EINVAL, "matpow_expm: the stream is being captured (the norm is read back to the host)");
  const size_t nn = (size_t)N * N, cap = (size_t)p->max_n * p->max_n;
  if (!p->expm_ws) {
    const size_t bytes = kMats * cap * sizeof(float) + 16 + sizeof(double) * (size_t)p->max_n + 256;
    cudaError_t e = cudaMalloc(&p->expm_ws, bytes);
    if (e != cudaSuccess) {
      p->expm_ws = nullptr;
      return fail(p, MATPOW_ENOMEM, "matpow_expm: scratch of %zu bytes", bytes);
    }
  }
  if (!p->expm_ev) {
    CK(p, cudaEventCreateWithFlags(&p->expm_ev, cudaEventDisableTiming));
  }
  float* M[kMats];
  for (int i = 0; i < kMats; ++i) M[i] = p->expm_ws + (size_t)i * cap;
  double* colsum = (double*)(((uintptr_t)(p->expm_ws + (size_t)kMats * cap) + 15) & ~(uintptr_t)15);
  long long* E = (long long*)(colsum + p->max_n);  // exponents of A^2, A^3, A^4
  unsigned* dnorm = (unsigned*)(E + 4);

  // ||A||_1 on the device; its read-back (it fixes s) overlaps the powers
  // A^2, A^3, A^4, which do not depend on s (B^k = A^k 2^(-k s))
  CK(p, cudaMemsetAsync(colsum, 0, sizeof(double) * N, s));
  CK(p, cudaMemsetAsync(dnorm, 0, sizeof(unsigned), s));
  expm_colsum_kernel<<<dim3((N + 255) / 256, (N + kNormRows - 1) / kNormRows), 256, 0, s>>>(dA, N, colsum);
  CK(p, cudaGetLastError());
  expm_colmax_kernel<<<1, 256, 0, s>>>(colsum, N, dnorm);
  CK(p, cudaGetLastError());
  p->launches += 2;
  unsigned* hbits = p->h_status + 1;  // pinned word next to the status read-back
  CK(p, cudaMemcpyAsync(hbits, dnorm, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(p, cudaEventRecord(p->expm_ev, s));
  if (p->prec == MATPOW_FP32_SIMT || fmt_exact(plan_float_fmt(p)) || N <= p->tiny_max) {
    const float* as[3] = {dA, dA, dA};
    const int ns3[3] = {N, N, N};
    const uint64_t ks[3] = {2, 3, 4};
    float* outs[3] = {M[1], M[2], M[3]};
    matpow_status st = matpow_batched(p, 3, as, ns3, ks, outs, (int64_t*)E, stream);
    if (st != MATPOW_OK) return st;
  } else {  // precisions without grouped launches: three single powers
    for (int k = 0; k < 3; ++k) {
      matpow_status st = matpow_f32(p, dA, N, (uint64_t)(k + 2), M[k + 1], (int64_t*)(E + k), stream);
      if (st != MATPOW_OK) return st;
    }
  }
  CK(p, cudaEventSynchronize(p->expm_ev));
  float nrm;
  std::memcpy(&nrm, hbits, sizeof nrm);
  if (!std::isfinite(nrm)) {
    // the powers already enqueued flag the same input; that flag belongs to
    // this call's EINVAL, not to the next matpow_sync
    CK(p, cudaStreamSynchronize(s));
    CK(p, cudaMemsetAsync(p->status, 0, sizeof(unsigned), s));
    CK(p, cudaStreamSynchronize(s));
    return fail(p, MATPOW_EINVAL, "matpow_expm: non-finite input");
  }
  int sq = 0;
  if (nrm > 1.0f) sq = (int)std::ceil(std::log2((double)nrm));
  while (sq > 0 && std::ldexp((double)nrm, -(sq - 1)) <= 1.0) --sq;  // smallest s with ||A|| 2^-s <= 1
  while (std::ldexp((double)nrm, -sq) > 1.0) ++sq;
  if (sq > 62) return fail(p, MATPOW_EINVAL, "matpow_expm: ||A||_1 = %g is beyond 2^62", (double)nrm);

  // the rest depends only on s and the pointers: one CUDA graph per s
  GraphKey key{2, dA, dOut, dLog2Scale, N, (uint64_t)sq, 0};
  return run_graph_or_direct(p, key, s, [&](cudaStream_t st) {
    return expm_tail(p, dA, N, M, E, sq, dOut, dLog2Scale, st);
  });
}
