// matpow_f32_noalloc: A^n with the float32 SIMT product kernels, using a
// fixed scratch array compiled into the library instead of a plan's
// workspace.  It allocates no device memory at any point.
//
// Scratch layout (one copy per GPU that loads the library, held until the
// process exits): four float32 partial-product buffers of 512 x 512, the
// scale slots {maxbits, exponent} of one power, and a status word.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.cuh"
#include "plan.h"

namespace {

constexpr int kMaxN = 512;
constexpr size_t kBufBytes = (size_t)kMaxN * kMaxN * sizeof(float);  // ld = 512, 1 MiB
constexpr int kSlots = 2 + 2 * 64;                                   // 2 + G(n) for any uint64 n
constexpr size_t kSlotBytes = kSlots * sizeof(mp::Scale);
constexpr size_t kScratchBytes = 4 * kBufBytes + kSlotBytes + 256;

// Device scratch shared by every call on a device.  In host code this name is
// only a stand-in: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;

// The scratch address is looked up once per device and kept with the CUDA
// context it belongs to: a context that is destroyed and re-created (after
// cudaDeviceReset, say) reloads the module, so the lookup is repeated then.
struct DevScratch {
  CUcontext ctx;
  unsigned char* ptr;
};
DevScratch g_dev_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
std::once_flag g_ctx_fn_once;

// The calling thread's current context, or null when it cannot be read.
CUcontext current_context() {
  std::call_once(g_ctx_fn_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = (CtxGetCurrentFn)fn;
  });
  CUcontext c = nullptr;
  if (!g_ctx_get_current || g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch array on the current device: set up on the
// first call in each context of the device (cudaGetSymbolAddress with that
// device current), reused afterwards.
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DevScratch& d = g_dev_scratch[dev];
  const CUcontext ctx = current_context();
  if (!d.ptr || !ctx || ctx != d.ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    d.ptr = (unsigned char*)ptr;
    d.ctx = current_context();  // the lookup initialises the context if it was not yet
  }
  *out = d.ptr;
  return cudaSuccess;
}

struct FixedOp {
  int xb, yb, cb, sx, sy, sc;
};

}  // namespace

using namespace mp;

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(nullptr, e_, #call); \
  } while (0)

extern "C" matpow_status matpow_f32_noalloc(const float* dA, int N, uint64_t n, float* dOut,
                                            int64_t* dLog2Scale, void* stream) {
  if (N < 0 || N > kMaxN)
    return fail(nullptr, MATPOW_EINVAL,
                "matpow_f32_noalloc: N=%d outside [0, %d], the size of its built-in scratch", N,
                kMaxN);
  if (N == 0) return MATPOW_OK;
  if (!dA || !dOut) return fail(nullptr, MATPOW_EINVAL, "matpow_f32_noalloc: NULL matrix pointer");
  if (((uintptr_t)dA & 3) || ((uintptr_t)dOut & 3) || ((uintptr_t)dLog2Scale & 7))
    return fail(nullptr, MATPOW_EINVAL, "matpow_f32_noalloc: misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    CK(launch_identity(dOut, N, 0, 0, (long long*)dLog2Scale, s));
    return MATPOW_OK;
  }
  if (n == 1) {
    CK(launch_copy(dA, dOut, N, (long long*)dLog2Scale, s));
    return MATPOW_OK;
  }
  unsigned char* base = nullptr;
  CK(scratch_for_current_device(&base));
  void* buf[4];
  for (int i = 0; i < 4; ++i) buf[i] = base + i * kBufBytes;
  Scale* scales = (Scale*)(base + 4 * kBufBytes);
  unsigned* status = (unsigned*)(base + 4 * kBufBytes + kSlotBytes);

  // slots and status start at zero on every call (the array keeps old contents)
  CK(cudaMemsetAsync(scales, 0, kSlotBytes + sizeof(unsigned), s));
  CK(launch_absmax_f32(dA, N, &scales[0], status, s));
  CK(launch_convert_f32(dA, N, &scales[0], &scales[1], FMT_F32, buf[0], 0, s));

  // right-to-left square-and-multiply over fixed arrays (no host allocation)
  const int ld = ld_for(N, FMT_F32);
  // N <= 512: at most 16 tiles of 128, so 64-wide SIMT tiles (four times the CTAs)
  constexpr int edge = 64;
  const int tn = (N + edge - 1) / edge;
  int refs[4] = {1, 0, 0, 0};
  auto take = [&]() {
    for (int i = 0; i < 4; ++i)
      if (refs[i] == 0) {
        refs[i] = 1;
        return i;
      }
    return -1;
  };
  int Pb = 0, Ps = 1, Rb = -1, Rs = -1, next_slot = 2;
  const int total_ops = matpow_gemm_count(n);
  int done_ops = 0;
  uint64_t bits = n;
  while (bits) {
    FixedOp ops[2];
    int nops = 0;
    int newRb = -1, newRs = -1, newPb = -1, newPs = -1;
    if (bits & 1ull) {
      if (Rb < 0) {
        Rb = Pb;
        Rs = Ps;
        refs[Pb]++;
      } else {
        newRb = take();
        newRs = next_slot++;
        ops[nops++] = {Rb, Pb, newRb, Rs, Ps, newRs};
      }
    }
    bits >>= 1;
    if (bits) {
      newPb = take();
      newPs = next_slot++;
      ops[nops++] = {Pb, Pb, newPb, Ps, Ps, newPs};
    }
    if (nops) {
      GemmPair g{};
      g.count = nops;
      int t = 0;
      for (int i = 0; i < nops; ++i) {
        const bool last = ++done_ops == total_ops;
        GemmDesc& d = g.d[i];
        d.X = buf[ops[i].xb];
        d.Y = buf[ops[i].yb];
        d.C = last ? nullptr : buf[ops[i].cb];
        d.out = last ? (void*)dOut : nullptr;
        d.out_log2 = last ? (long long*)dLog2Scale : nullptr;
        d.N = N;
        d.ld = ld;
        d.sx = ops[i].sx;
        d.sy = ops[i].sy;
        d.sc = ops[i].sc;
        d.mode = last ? (dLog2Scale ? OUT_USER_MANT : OUT_USER_VALUE) : OUT_INTERNAL;
        d.tile_begin = t;
        d.tiles_n = tn;
        t += tn * tn;
      }
      g.tiles_total = t;
      CK(launch_simt_pair(g, edge, 1, scales, status, s));
    }
    if (newRb >= 0) {
      refs[Rb]--;
      Rb = newRb;
      Rs = newRs;
    }
    if (newPb >= 0) {
      refs[Pb]--;
      Pb = newPb;
      Ps = newPs;
    }
  }
  return MATPOW_OK;
}
