/*
 * Plain CPU oracle for the integer matrix power A^n.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (arXiv 1204.3052):
 *   - the matrix product as the plain triple loop of Sec. 4.1
 *     (c_ij accumulates a_ik * b_kj over k = 0..N-1, in increasing k);
 *   - A^n by "brute force": n copies of A multiplied one after another
 *     (Sec. 4.1 / Sec. 4.2, the power computed by repeating the product);
 *   - A^n by binary square-and-multiply, which needs about log2(n) products
 *     (Sec. 4.3): right-to-left over the bits of n, squaring P = A^(2^k) at
 *     each level and multiplying it into the result when bit k is set;
 *   - the same two methods over the integers modulo p (exact, uint64).
 *
 * Floating point: float64, IEEE round-to-nearest-even, no contraction into
 * fused multiply-add (built with -ffp-contract=off), no reassociation.  To
 * keep A^n in range for exponents up to 2^30, every product is followed by an
 * exact power-of-two rescale: the result is held as a mantissa matrix M and an
 * int64 exponent e with A^n = M * 2^e, where max|M| is in [0.5, 1) (or M = 0).
 * Scaling by a power of two is exact unless it leaves the normal range, so
 * this is the definition of A^n written in a wider exponent range.
 *
 * Loop order: i-k-j.  Each c_ij still accumulates its N terms in increasing k,
 * exactly as the i-j-k listing would, so the result is bit-identical; the
 * order only changes memory access.  Rows may be split across OpenMP threads,
 * which does not change any sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

/* Set the number of OpenMP threads used by the product loops (<=0: all). */
int oracle_set_threads(int threads) {
#ifdef _OPENMP
  if (threads <= 0) threads = omp_get_num_procs();
  omp_set_num_threads(threads);
  return threads;
#else
  (void)threads;
  return 1;
#endif
}

/* C = A * B for row-major N x N float64 (Sec. 4.1).  C must not alias A or B. */
void oracle_gemm_f64(int N, const double* A, const double* B, double* C) {
  int i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < N; ++i) {
    double* c = C + (size_t)i * N;
    for (int j = 0; j < N; ++j) c[j] = 0.0;
    for (int k = 0; k < N; ++k) {
      const double a = A[(size_t)i * N + k];
      const double* b = B + (size_t)k * N;
      for (int j = 0; j < N; ++j) c[j] = c[j] + a * b[j];
    }
  }
}

/* Rows r0 .. r1-1 of C = A * B (row-major N x N A, B; C holds r1 - r0 rows
 * of N): the same triple loop as oracle_gemm_f64 restricted to those rows, so
 * each entry equals the full product's bit for bit.  A bounded sample of one
 * large product for timing. */
void oracle_gemm_rows_f64(int N, int r0, int r1, const double* A, const double* B, double* C) {
  int i;
#pragma omp parallel for schedule(static)
  for (i = r0; i < r1; ++i) {
    double* c = C + (size_t)(i - r0) * N;
    for (int j = 0; j < N; ++j) c[j] = 0.0;
    for (int k = 0; k < N; ++k) {
      const double a = A[(size_t)i * N + k];
      const double* b = B + (size_t)k * N;
      for (int j = 0; j < N; ++j) c[j] = c[j] + a * b[j];
    }
  }
}

/* Rescale M (N x N) by a power of two so that max|M| is in [0.5, 1); add the
 * applied exponent to *e.  M = 0 is left alone. */
static void normalise(int N, double* M, int64_t* e) {
  double mx = 0.0;
  size_t total = (size_t)N * N;
  for (size_t t = 0; t < total; ++t) {
    double v = fabs(M[t]);
    if (v > mx) mx = v;
  }
  if (mx == 0.0 || !isfinite(mx)) return;
  int s;
  (void)frexp(mx, &s); /* mx = f * 2^s, f in [0.5, 1) */
  if (s == 0) return;
  for (size_t t = 0; t < total; ++t) M[t] = ldexp(M[t], -s);
  *e += s;
}

/* (M, e) <- (X * Y, ex + ey), normalised.  Scratch T is N x N. */
static void mul_scaled(int N, const double* X, int64_t ex, const double* Y, int64_t ey,
                       double* out, int64_t* eout, double* T) {
  oracle_gemm_f64(N, X, Y, T);
  memcpy(out, T, sizeof(double) * (size_t)N * N);
  *eout = ex + ey;
  normalise(N, out, eout);
}

/*
 * A^n as mantissa M and exponent *e (A^n = M * 2^e).
 * mode 0: square-and-multiply (Sec. 4.3); mode 1: n-1 repeated products
 * (Sec. 4.1/4.2).  n = 0 gives the identity, n = 1 a (normalised) copy.
 * *gemms receives the number of matrix products performed (nullable).
 */
int oracle_matpow_f64(int N, const double* A, uint64_t n, int mode, double* M,
                      int64_t* e, int64_t* gemms) {
  if (N < 0 || (N > 0 && (!A || !M || !e))) return ORACLE_EINVAL;
  if (gemms) *gemms = 0;
  if (N == 0) { *e = 0; return ORACLE_OK; }
  size_t NN = (size_t)N * N;
  *e = 0;
  if (n == 0) {
    memset(M, 0, sizeof(double) * NN);
    for (int i = 0; i < N; ++i) M[(size_t)i * N + i] = 1.0;
    normalise(N, M, e);
    return ORACLE_OK;
  }
  double* P = (double*)malloc(sizeof(double) * NN);
  double* T = (double*)malloc(sizeof(double) * NN);
  if (!P || !T) { free(P); free(T); return ORACLE_ENOMEM; }
  memcpy(P, A, sizeof(double) * NN);
  int64_t ep = 0;
  normalise(N, P, &ep);
  int64_t count = 0;
  if (mode == 1) {
    /* brute force: R = A, then R <- R * A, n-1 times */
    memcpy(M, P, sizeof(double) * NN);
    *e = ep;
    for (uint64_t t = 1; t < n; ++t) {
      mul_scaled(N, M, *e, P, ep, M, e, T);
      ++count;
    }
  } else {
    /* right-to-left binary: P = A^(2^k) at level k */
    int have_r = 0;
    uint64_t bits = n;
    while (bits) {
      if (bits & 1u) {
        if (!have_r) {
          memcpy(M, P, sizeof(double) * NN);
          *e = ep;
          have_r = 1;
        } else {
          mul_scaled(N, M, *e, P, ep, M, e, T);
          ++count;
        }
      }
      bits >>= 1;
      if (bits) {
        mul_scaled(N, P, ep, P, ep, P, &ep, T);
        ++count;
      }
    }
  }
  free(P);
  free(T);
  if (gemms) *gemms = count;
  return ORACLE_OK;
}

/* C = (A * B) mod p for row-major N x N integers in [0, p), p < 2^32.
 * For p < 2^16 each product is below 2^32, so N < 2^32 terms add up in uint64
 * without overflow and the sum is reduced once at the end.  For larger p each
 * product is reduced as it is added. */
void oracle_gemm_modp(int N, const uint64_t* A, const uint64_t* B, uint64_t p, uint64_t* C) {
  int i;
#pragma omp parallel for schedule(static)
  for (i = 0; i < N; ++i) {
    uint64_t* c = C + (size_t)i * N;
    for (int j = 0; j < N; ++j) c[j] = 0;
    for (int k = 0; k < N; ++k) {
      const uint64_t a = A[(size_t)i * N + k];
      const uint64_t* b = B + (size_t)k * N;
      if (p >= (1ull << 16)) {
        for (int j = 0; j < N; ++j) c[j] = (c[j] + (a * b[j]) % p) % p;
      } else {
        for (int j = 0; j < N; ++j) c[j] += a * b[j];
      }
    }
    for (int j = 0; j < N; ++j) c[j] %= p;
  }
}

/* A^n mod p (mode 0 square-and-multiply, mode 1 brute force). */
int oracle_matpow_modp(int N, const uint64_t* A, uint64_t n, uint64_t p, int mode,
                       uint64_t* out, int64_t* gemms) {
  if (N < 0 || p < 2 || p >= (1ull << 32) || (N > 0 && (!A || !out))) return ORACLE_EINVAL;
  if (gemms) *gemms = 0;
  if (N == 0) return ORACLE_OK;
  size_t NN = (size_t)N * N;
  for (size_t t = 0; t < NN; ++t)
    if (A[t] >= p) return ORACLE_EINVAL;
  if (n == 0) {
    memset(out, 0, sizeof(uint64_t) * NN);
    for (int i = 0; i < N; ++i) out[(size_t)i * N + i] = 1 % p;
    return ORACLE_OK;
  }
  uint64_t* P = (uint64_t*)malloc(sizeof(uint64_t) * NN);
  uint64_t* T = (uint64_t*)malloc(sizeof(uint64_t) * NN);
  if (!P || !T) { free(P); free(T); return ORACLE_ENOMEM; }
  memcpy(P, A, sizeof(uint64_t) * NN);
  int64_t count = 0;
  if (mode == 1) {
    memcpy(out, P, sizeof(uint64_t) * NN);
    for (uint64_t t = 1; t < n; ++t) {
      oracle_gemm_modp(N, out, P, p, T);
      memcpy(out, T, sizeof(uint64_t) * NN);
      ++count;
    }
  } else {
    int have_r = 0;
    uint64_t bits = n;
    while (bits) {
      if (bits & 1u) {
        if (!have_r) {
          memcpy(out, P, sizeof(uint64_t) * NN);
          have_r = 1;
        } else {
          oracle_gemm_modp(N, out, P, p, T);
          memcpy(out, T, sizeof(uint64_t) * NN);
          ++count;
        }
      }
      bits >>= 1;
      if (bits) {
        oracle_gemm_modp(N, P, P, p, T);
        memcpy(P, T, sizeof(uint64_t) * NN);
        ++count;
      }
    }
  }
  free(P);
  free(T);
  if (gemms) *gemms = count;
  return ORACLE_OK;
}
