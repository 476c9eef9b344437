/*
 * libmatpow — the integer matrix power A^n of a dense square matrix on one
 * NVIDIA GB300 GPU (sm_103a), by binary square-and-multiply.
 *
 * Operation (arXiv 1204.3052): given a dense N x N matrix A and an integer
 * power n, return A^n.  The paper's CPU method repeats the triple-loop matrix
 * product of Sec. 4.1 n-1 times; its GPU method (Sec. 4.3) multiplies "log(N)
 * times" instead of N times, i.e. binary square-and-multiply with
 * G(n) = floor(log2 n) + popcount(n) - 1 products, and moves the data between
 * host and device only a few times (Sec. 4.3.8).  This library keeps A, every
 * partial product and the result on the device and runs each product as a
 * hand-written CUDA kernel.
 *
 * Conventions for every call:
 *  - Matrices are row-major, N x N, densely packed (leading dimension N).
 *  - "device" pointers are CUDA global-memory addresses on the plan's device;
 *    "host" pointers are ordinary process memory.  Wherever a matrix is a
 *    "device" pointer it may also be page-locked host memory that the device
 *    addresses at the same pointer (cudaHostAlloc / cudaMallocHost memory
 *    under unified addressing; matpow_host_accessible() tells): the kernels
 *    then read A and write the result across the host link themselves (on a
 *    GB300, the NVLink-C2C to the Grace CPU).  Only the input read and the
 *    final result write touch such memory; every intermediate stays in the
 *    plan's device workspace.  Results are bit-identical to those of device
 *    buffers; for large transfers, copies by the copy engines into device
 *    buffers were measured faster.  The caller owns all memory
 *    it passes in; the library never frees it and keeps no reference after
 *    the work enqueued by the call has finished.
 *  - `stream` is a cudaStream_t (NULL: the legacy default stream).  Work is
 *    enqueued asynchronously on it; argument checks are synchronous.  Errors
 *    that only the device can see (a float result out of range, an entry >= p)
 *    are recorded in the plan and returned by matpow_sync().
 *  - No C++ exception crosses this interface.  Every call returns a
 *    matpow_status; matpow_last_error() gives a message for the last failure.
 *  - A plan is not thread-safe: use one plan per host thread.  A server
 *    (matpow_server_*) is internally locked and may be shared.
 */
#ifndef MATPOW_H
#define MATPOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MATPOW_VERSION 1

typedef enum matpow_status {
  MATPOW_OK = 0,
  MATPOW_EINVAL = 1,      /* bad argument (null pointer, N < 0, N > max_n, p out of range, entry >= p) */
  MATPOW_ENOMEM = 2,      /* device allocation failed or exceeds the plan's workspace limit */
  MATPOW_ECUDA = 3,       /* a CUDA runtime or driver call failed */
  MATPOW_EAGAIN = 4,      /* matpow_poll: the request is not finished yet */
  MATPOW_EBUSY = 5,       /* matpow_submit: the server's admission queue is full */
  MATPOW_ETIMEDOUT = 6,   /* a bounded wait (host or device) gave up */
  MATPOW_ERANGE = 7,      /* float result left the float32 range (the mantissa form is exact) */
  MATPOW_EUNSUPPORTED = 8 /* device is not sm_103 or the option is not supported */
} matpow_status;

/* Arithmetic of the float path (matpow_f32 / matpow_batched). */
typedef enum matpow_precision {
  MATPOW_FP32_SIMT = 0, /* float32 fused multiply-add products on the CUDA cores */
  MATPOW_BF16 = 1,      /* one bfloat16 tensor-core product per term, float32 accumulation */
  MATPOW_BF16X3 = 2,    /* each operand split into two bfloat16 parts, three tensor-core
                           products (hi*hi + hi*lo + lo*hi) with float32 accumulation; by
                           default the parts are exact 8-bit integer slices of each 64 x 64
                           block scaled by its power-of-two maximum (16-bit fixed point per
                           block), see MATPOW_OPT_SPLIT */
  MATPOW_BF16X6 = 3     /* three exact 8-bit slices per block (24-bit fixed point), six
                           tensor-core products a_i * b_j (i + j <= 2): float32-class results */
} matpow_precision;

typedef struct matpow_plan_s* matpow_plan_t;

/* ---- plan ---------------------------------------------------------------- */

/*
 * Create a plan on CUDA device `device` for matrices of order up to `max_n`
 * (>= 1) with float arithmetic `precision`.  The plan allocates its device
 * workspace here (partial products, scale exponents, status words); no later
 * call allocates device memory except matpow_batched, which grows a plan-owned
 * descriptor table on first use of a larger batch, and matpow_expm, which
 * allocates its scratch on its first call.  `workspace_bytes` = 0
 * lets the plan take what max_n needs (matpow_workspace_size); a nonzero
 * value is an upper limit, and the call fails with MATPOW_ENOMEM if the need
 * exceeds it.  Fails with MATPOW_EUNSUPPORTED if the device is not sm_103.
 * On success *plan owns the workspace until matpow_plan_destroy.
 */
matpow_status matpow_plan(matpow_plan_t* plan, int max_n, matpow_precision precision,
                          size_t workspace_bytes, int device);

/* Bytes of device workspace a plan for (max_n, precision) allocates. */
size_t matpow_workspace_size(int max_n, matpow_precision precision);

/* Free the plan and its workspace (synchronises the plan's device first). */
matpow_status matpow_plan_destroy(matpow_plan_t plan);

/* NUL-terminated message for the plan's last failure ("" if none).  Valid
 * until the next call on the plan.  plan may be NULL (last global error). */
const char* matpow_last_error(matpow_plan_t plan);

/*
 * Plan options (key, value):
 *   MATPOW_OPT_GRAPHS   1 (default): replay the level launches of a repeated
 *                       call from a cached CUDA graph; 0: launch directly.
 *   MATPOW_OPT_TIMING   1: record CUDA events around every product kernel on
 *                       the caller's stream (read with matpow_kernel_time); 0 (default).
 *   MATPOW_OPT_TINY_MAX largest N handled by the on-chip whole-chain path
 *                       (float32 products in shared memory: one CTA per
 *                       matrix, or for a single power with N > 32 one
 *                       four-CTA cluster; 0 disables it; default and
 *                       maximum 64).
 *   MATPOW_OPT_TILE     tensor-core tile width override (columns of C per CTA:
 *                       64, 128 or 256; 0 = the built-in choice by N).
 *   MATPOW_OPT_SPLIT    MATPOW_BF16X3 operand split: 0 (default) exact
 *                       fixed-point slices -- each matrix scaled by its
 *                       power-of-two maximum and cut into two 8-bit integer
 *                       slices, whose tensor-core partial sums are exact
 *                       integers; 1: floating hi/lo bfloat16 parts summed in
 *                       the tensor core's float32 accumulator (subject to the
 *                       accumulator's rounding toward zero, whose bias the
 *                       squaring chain amplifies).
 *   MATPOW_OPT_CHAIN    1 (default): for the exact splits (MATPOW_BF16X3 with
 *                       64 < N <= 1024, MATPOW_BF16X6 with 64 < N <= 768) run
 *                       the whole chain in one cooperative launch (grid
 *                       barriers between levels), with split-K over 2 or 4
 *                       CTAs of a thread-block cluster per tile when a level
 *                       has few tiles (results then equal the level path's
 *                       to rounding, not bit for bit); 2: the same without
 *                       split-K (bit-for-bit equal to the level path), and
 *                       MATPOW_FP32_SIMT products without their split-K over
 *                       two-CTA clusters (used when a launch has fewer
 *                       64 x 64 tiles than SMs), so that every result equals
 *                       that of the same matrix in a batch bit for bit;
 *                       0: one launch per level.
 *   MATPOW_OPT_MODP_TC  1 (default): matpow_mod_p with 64 < N <= 16384 runs on the
 *                       tensor cores (balanced byte digits of the residues,
 *                       exact partial sums); 0: 64-bit integer products on the
 *                       CUDA cores.
 *   MATPOW_OPT_PERSIST  1 (default): matpow_batched runs each level's 64-column
 *                       tensor-core tiles (orders up to 4096) in one persistent
 *                       launch, one CTA per SM walking the whole tile list; 0:
 *                       one CTA per tile.  Results are identical either way.
 *   MATPOW_OPT_PAIR     0 (default): one SM per 128 x 128 tile; 1: exact-split
 *                       BF16X3 products of orders above 2048 with 128-column
 *                       tiles run on CTA pairs: one 256 x 128 tile per two
 *                       SMs, M = 256 tensor-core MMAs (tcgen05 cta_group::2)
 *                       over both SMs' shared memory, each SM holding half of
 *                       the B operand.  Results are bit-for-bit those of the
 *                       one-SM kernel; it runs slower on a GB300 (N = 8192:
 *                       2.93 ms per product against 2.47 ms), since the
 *                       per-k-block accumulator hand-off then crosses SMs and
 *                       the pair saves no shared-memory operand reads.
 *   MATPOW_OPT_NAIVE    0 (default); 1: matpow_f32 with N above the whole-chain
 *                       limit (MATPOW_OPT_TINY_MAX) computes A^n the way the
 *                       paper's naive GPU method does (Sec. 4.2): n - 1
 *                       products R <- R A, one kernel launch each, with the
 *                       plan's product kernels and arithmetic.  A comparison
 *                       method: it costs n - 1 products instead of about
 *                       2 log2(n).
 */
enum { MATPOW_OPT_GRAPHS = 1, MATPOW_OPT_TIMING = 2, MATPOW_OPT_TINY_MAX = 3, MATPOW_OPT_TILE = 4,
       MATPOW_OPT_SPLIT = 5, MATPOW_OPT_CHAIN = 6, MATPOW_OPT_MODP_TC = 7, MATPOW_OPT_PERSIST = 8,
       MATPOW_OPT_NAIVE = 9, MATPOW_OPT_PAIR = 10 };
matpow_status matpow_plan_set_option(matpow_plan_t plan, int key, int64_t value);

/* ---- tile table (launch shapes per size class) ------------------------------ */

/*
 * The paper keeps a family of product kernels with tile shapes from 4 x 4 to
 * 16 x 16 and picks one by the problem size and the local memory available
 * (Sec. 4.3.7).  Here a plan may carry a tile table: rules, each for one
 * precision and one range of orders, that fix the launch shape of the
 * products; an autotuner (paper_1204_3052_gb300/autotune.py) measures the
 * candidates on the device and writes the winners as JSON.  Orders that no
 * rule covers keep the built-in choice, as does any field set to -1.
 * Explicit plan options win over the table: MATPOW_OPT_TILE over `bn`,
 * MATPOW_OPT_CHAIN 0 or 2 over `chain` and `split_k`, MATPOW_OPT_PERSIST 0
 * over `persist`.
 */
typedef struct matpow_tile_rule {
  int n_lo, n_hi; /* the rule covers orders N with n_lo < N <= n_hi */
  int precision;  /* matpow_precision the rule is for */
  int bn;         /* exact-split tile width, columns of C per CTA: 64 or 128 */
  int split_k;    /* whole-chain launches: CTAs of a cluster sharing one tile's k range: 1, 2, 4 */
  int chain;      /* single powers (and up to four side by side) with N <= 1024: 1 the
                     whole chain in one cooperative launch, 0 one launch per level */
  int persist;    /* matpow_batched levels of 64-column tiles: 1 one persistent CTA per SM
                     over the tile list, 0 one CTA per tile */
} matpow_tile_rule;

/* Replace the plan's tile table by `count` rules (copied; count = 0 clears
 * it).  MATPOW_EINVAL for a rule with n_lo >= n_hi, an unknown precision or
 * a field outside its values (bn: 64 or 128; split_k: 1, 2 or 4; chain,
 * persist: 0 or 1; -1 everywhere for "built-in"). */
matpow_status matpow_plan_set_tile_table(matpow_plan_t plan, const matpow_tile_rule* rules, int count);

/* Read a tile table from the JSON file at `path` (host path) into the plan:
 * {"rules": [{"precision": "bf16x6", "n_lo": 64, "n_hi": 128, "bn": 64,
 * "split_k": 2, "chain": 1, "persist": 1, ...}, ...]}; precision is one of
 * "fp32", "bf16", "bf16x3", "bf16x6"; omitted fields are -1; other keys are
 * ignored.  MATPOW_EINVAL (with the position in the message) for text that
 * does not parse or a rule that matpow_plan_set_tile_table rejects. */
matpow_status matpow_plan_load_tile_table(matpow_plan_t plan, const char* path);

/* Parse tile-table JSON text (NUL-terminated) into at most `cap` rules;
 * *count receives the number of rules in the text (may exceed cap).  Host
 * only, needs no device. */
matpow_status matpow_tile_table_parse(const char* json, matpow_tile_rule* rules, int cap, int* count);

/* The rule a table gives for (precision, N): the last rule in table order
 * that covers it, copied to *out; MATPOW_EAGAIN if none covers it (then
 * *out is all -1 but n_lo, n_hi, precision).  Host only. */
matpow_status matpow_tile_rule_lookup(const matpow_tile_rule* rules, int count, matpow_precision precision,
                                      int N, matpow_tile_rule* out);

/* ---- the power ------------------------------------------------------------ */

/*
 * A^n for float32 A (arXiv 1204.3052, Sec. 4.3: square-and-multiply, about
 * log2(n) products; the product itself is Sec. 4.1's c_ij = sum_k a_ik b_kj).
 *   dA          device, N*N float32, row-major; read only.
 *   N           matrix order, 0 <= N <= max_n (N = 0: nothing to do).
 *   n           power, any uint64 (n = 0: identity, n = 1: copy of A).
 *   dOut        device, N*N float32; may alias dA.
 *   dLog2Scale  device int64 or NULL.  If non-NULL the result is returned in
 *               mantissa form: dOut holds M and *dLog2Scale holds e with
 *               A^n = M * 2^e (max|M| <= N; never overflows).  If NULL, dOut
 *               holds A^n as M * 2^e rounded once to float32 (exact while
 *               the result is a normal float; one rounding into the
 *               subnormals); entries beyond the float32 range become +-inf
 *               or 0 and matpow_sync() then returns MATPOW_ERANGE.
 *   stream      cudaStream_t.
 * Intermediate powers are kept with a per-matrix power-of-two exponent so
 * that n up to 2^64-1 never overflows.  Asynchronous.
 */
matpow_status matpow_f32(matpow_plan_t plan, const float* dA, int N, uint64_t n, float* dOut,
                         int64_t* dLog2Scale, void* stream);

/*
 * A^n like matpow_f32 with MATPOW_FP32_SIMT products, for callers that may
 * not allocate device memory: code that runs under an allocator which owns
 * all of the device's memory (a framework's caching pool, a fixed budget set
 * at start-up), or latency-critical code that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  It takes no plan and calls no
 * allocating routine; its scratch (four 512 x 512 float32 buffers plus the
 * per-power scale slots, about 4 MiB) is an array compiled into the library,
 * present on every GPU that loads it until the process exits.  The paper has
 * no counterpart to this entry point.
 *   dA, N, n, dOut, dLog2Scale, stream: as in matpow_f32, on the calling
 *               thread's current device; 0 <= N <= 512, larger N fails with
 *               MATPOW_EINVAL (and a message naming the limit).
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and keeps it with the device's current context; a
 * call in a new context of that device (after cudaDeviceReset, say) looks
 * it up again.  Make the first call in each context before any stream
 * capture.
 * Every call uses the same scratch, so calls whose work overlaps on the GPU
 * (different streams, or threads without ordering) race and corrupt each
 * other: order them on one stream.  Device-side conditions that matpow_sync
 * reports for a plan (non-finite input, float32 range loss) are not reported
 * here; the mantissa form (dLog2Scale != NULL) never loses range.
 */
matpow_status matpow_f32_noalloc(const float* dA, int N, uint64_t n, float* dOut,
                                 int64_t* dLog2Scale, void* stream);

/*
 * The matrix exponential e^A of a float32 matrix.  (The paper's "matrix
 * exponentiation" is A^n; e^A is the other common meaning, computed here on
 * the same squaring chain by scaling and squaring: Moler and Van Loan,
 * SIAM Review 45 (2003), method 3.)
 *   s = max(0, ceil(log2 ||A||_1)) squarings (||A||_1: the largest column
 *   sum), B = A 2^-s, T = the degree-11 Taylor polynomial of e^B in
 *   Paterson-Stockmeyer form, T = P0 + B^4 (P1 + B^4 P2) (five products on
 *   the plan's product path: B^2, B^3, B^4 and the two outer ones), and
 *   e^A = T^(2^s) by matpow_f32 (s squarings).
 *   dA, dOut, dLog2Scale   as in matpow_f32; dOut may alias dA.
 * Reads ||A||_1 back to the host (it fixes s), so the call waits for the
 * stream up to that point; on a stream that is being captured it returns
 * MATPOW_EINVAL without enqueueing anything.  A non-finite entry or
 * ||A||_1 > 2^62 returns MATPOW_EINVAL.  The first call
 * on a plan allocates 7 max_n^2 float32 of scratch (MATPOW_ENOMEM if that
 * fails).  Accuracy: float32 class, the error growing with s (each squaring
 * doubles the relative error of the dominant eigenvalues).
 */
matpow_status matpow_expm(matpow_plan_t plan, const float* dA, int N, float* dOut, int64_t* dLog2Scale,
                          void* stream);

/*
 * A^n mod p for integer A (exact; the same square-and-multiply over Z/pZ).
 *   dA     device, N*N uint32 with every entry in [0, p); read only.
 *   p      modulus, 2 <= p <= 65536.
 *   dOut   device, N*N uint32, entries in [0, p); may alias dA.
 * An entry >= p is detected on the device: dOut is then unspecified and
 * matpow_sync() returns MATPOW_EINVAL.  Bit-exact.  Asynchronous.
 */
matpow_status matpow_mod_p(matpow_plan_t plan, const uint32_t* dA, int N, uint64_t n, uint32_t p,
                           uint32_t* dOut, void* stream);

/*
 * `count` independent float32 powers A_i^(n_i) of uneven orders, run level by
 * level: all products of one squaring level of all matrices go into one
 * grouped kernel launch (Sec. 4.3's method applied to a batch).
 *   dA, dOut     host arrays of `count` device pointers (N_i*N_i float32 each;
 *                dOut[i] may alias dA[i]).
 *   N, n         host arrays of `count` orders (0 <= N_i <= max_n) and powers.
 *   dLog2Scale   device array of `count` int64, or NULL (as in matpow_f32).
 * Asynchronous; the host arrays may be reused as soon as the call returns.
 */
matpow_status matpow_batched(matpow_plan_t plan, int count, const float* const* dA, const int* N,
                             const uint64_t* n, float* const* dOut, int64_t* dLog2Scale,
                             void* stream);

/*
 * Wait for the work enqueued on `stream` and return the first deferred
 * device status of the plan since the last matpow_sync (MATPOW_OK,
 * MATPOW_ERANGE, MATPOW_EINVAL for an entry >= p, MATPOW_ETIMEDOUT when a
 * kernel's bounded wait gave up), then clear it.
 */
matpow_status matpow_sync(matpow_plan_t plan, void* stream);

/*
 * Error-path self-test.  Launches one CTA that waits on a shared-memory
 * mbarrier that no thread ever arrives at, with the bounded wait every
 * tensor-core kernel of the library uses, given a budget of `budget_ns`
 * nanoseconds of the GPU's global timer (1000 <= budget_ns <= 10^10, else
 * MATPOW_EINVAL).  The wait gives up, the kernel records the timeout in the
 * plan's status word and returns; matpow_sync() then returns
 * MATPOW_ETIMEDOUT and the plan and the CUDA context stay usable.
 * Asynchronous.  For tests of the timeout path.
 */
matpow_status matpow_selftest_wait_timeout(matpow_plan_t plan, uint64_t budget_ns, void* stream);

/*
 * FP32 throughput probe (the roofline denominator of the float32 SIMT path).
 * Launches 8 CTAs of 256 threads per SM; every thread runs 8 independent
 * float32 fused multiply-add chains of `iters` steps on registers only
 * (`iters` a multiple of 16 in [16, 2^32], else MATPOW_EINVAL): exactly
 * 2 x 8 x iters x 256 x 8 x (SMs) flop, no memory traffic.  Time it with
 * CUDA events on `stream`.  Asynchronous.  (No counterpart in the paper,
 * whose Fermi figures are nominal.)
 */
matpow_status matpow_selftest_ffma(matpow_plan_t plan, int64_t iters, void* stream);

/* Streaming multiprocessors of the plan's device (sizes the probe above). */
int matpow_plan_sm_count(matpow_plan_t plan);

/*
 * 1 if `device` can address `ptr` at the same pointer, so that it may be
 * passed where a call takes a device matrix: global memory of that device,
 * managed memory, or page-locked host memory mapped at its host address.
 * 0 otherwise (pageable host memory, another device's memory, NULL, or a
 * failed query).  A host-side query (cudaPointerGetAttributes); no work is
 * enqueued.
 */
int matpow_host_accessible(const void* ptr, int device);

/* G(n) = floor(log2 n) + popcount(n) - 1 (0 for n <= 1): products that A^n takes. */
int matpow_gemm_count(uint64_t n);

/*
 * Timing of product kernels recorded under MATPOW_OPT_TIMING since the last
 * reset: kernel class `kind` (MATPOW_KERNEL_*), number of launches, total
 * milliseconds (CUDA events on the caller's stream; synchronises it), and the
 * algorithmic work those launches did (2*N^3 per product, summed) in flop.
 * reset != 0 clears the record afterwards.
 */
enum { MATPOW_KERNEL_SIMT = 0, MATPOW_KERNEL_TC = 1, MATPOW_KERNEL_TINY = 2, MATPOW_KERNEL_MODP = 3,
       MATPOW_KERNEL_AUX = 4, MATPOW_KERNEL_KINDS = 5 };
matpow_status matpow_kernel_time(matpow_plan_t plan, int kind, int64_t* launches, double* total_ms,
                                 double* flop, int reset);

/* Kernel launches the plan has issued since creation (all kernels, cumulative). */
int64_t matpow_launch_count(matpow_plan_t plan);

/* ---- serving ---------------------------------------------------------------- */

/*
 * A request server: continuous batching of independent A^n requests on one
 * device (the paper's method run for many users at once).  Requests are
 * admitted while their device footprint fits `hbm_budget_bytes` and fewer
 * than `max_inflight` are running; each scheduler step groups the next
 * product of every admitted request into one launch, so requests that
 * arrive later join the running batch at their own first level.
 */
typedef struct matpow_server_s* matpow_server_t;

typedef struct matpow_server_desc {
  int device;
  int max_n;                  /* largest order accepted */
  matpow_precision precision; /* float requests */
  size_t hbm_budget_bytes;    /* device bytes for in-flight partial products */
  int max_inflight;           /* admitted requests at most */
  int max_queue;              /* queued (not yet admitted) requests at most */
} matpow_server_desc;

typedef struct matpow_request {
  int N;               /* order, 1 <= N <= max_n */
  uint64_t n;          /* power */
  int kind;            /* 0: float32 A^n; 1: A^n mod p */
  uint32_t p;          /* modulus for kind 1 (2 <= p <= 65536) */
  const void* dA;      /* device input (float32 or uint32), read only, kept valid until done */
  void* dOut;          /* device output (float32 or uint32) */
  int64_t* dLog2Scale; /* kind 0: device int64 or NULL, as in matpow_f32 */
} matpow_request;

matpow_status matpow_server_create(matpow_server_t* server, const matpow_server_desc* desc);

/* Queue a request (non-blocking).  *ticket identifies it for matpow_poll.
 * MATPOW_EBUSY if the queue holds max_queue requests; MATPOW_EINVAL for a
 * bad request. */
matpow_status matpow_submit(matpow_server_t server, const matpow_request* req, uint64_t* ticket);

/* Wait up to timeout_us microseconds for request `ticket`: MATPOW_OK once its
 * output is complete on the device (the ticket is then retired),
 * MATPOW_EAGAIN / MATPOW_ETIMEDOUT if not finished (EAGAIN when
 * timeout_us == 0), or the request's error status. */
matpow_status matpow_poll(matpow_server_t server, uint64_t ticket, uint32_t timeout_us);

/* Latency record of retired requests: submit-to-completion microseconds for
 * up to `cap` requests (oldest first); returns how many were written. */
int64_t matpow_server_latencies(matpow_server_t server, double* us, int64_t cap);

/* Stop the scheduler, wait for in-flight work and free the server. */
matpow_status matpow_server_destroy(matpow_server_t server);

#ifdef __cplusplus
}
#endif
#endif /* MATPOW_H */
