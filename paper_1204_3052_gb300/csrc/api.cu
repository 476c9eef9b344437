// libmatpow C-ABI: plans, the square-and-multiply scheduler, graph replay,
// batching and timing.  Every product runs in the kernels of k_*.cu; this
// file only validates arguments, lays out the workspace and enqueues work.
//
// Method (arXiv 1204.3052 Sec. 4.3): A^n by binary square-and-multiply,
// right to left over the bits of n.  Level k holds P = A^(2^k); if bit k is
// set the partial result takes R <- R*P (the first set bit only copies P),
// and P <- P*P while higher bits remain.  Both products of a level read P and
// nothing else of the level, so they go into one grouped launch.  A is moved
// to the device once and all partial products stay there (Sec. 4.3.8).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"
#include "plan.h"

using namespace mp;

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

matpow_status mp::fail(matpow_plan_s* plan, matpow_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (plan) plan->err = buf;
  g_last_error = buf;
  return st;
}

matpow_status mp::cuda_fail(matpow_plan_s* plan, cudaError_t e, const char* what) {
  return fail(plan, MATPOW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(plan, call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(plan, e_, #call); \
  } while (0)

extern "C" const char* matpow_last_error(matpow_plan_t plan) {
  if (plan) return plan->err.c_str();
  return g_last_error.c_str();
}

extern "C" int matpow_gemm_count(uint64_t n) {
  if (n <= 1) return 0;
  int k = 63 - __builtin_clzll(n);
  return k + __builtin_popcountll(n) - 1;
}

// ---------------------------------------------------------------------------
// workspace layout

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t mp::matrix_bytes(int N, int fmt) {
  size_t ld = (size_t)ld_for(N, fmt);
  size_t e = (size_t)N * ld;
  switch (fmt) {
    case FMT_F32:
    case FMT_U32:
      return align_up(e * 4, 1024);
    case FMT_BF16:
      return align_up(e * 2, 1024);
    case FMT_FX2:
    case FMT_FX3: {  // two or three bfloat16 slice planes, then the block exponents
      size_t nb = ((size_t)N + 63) / 64;
      return fmt_slices(fmt) * align_up(e * 2, 1024) + align_up(nb * nb * 4, 1024);
    }
    default:  // two bfloat16 planes
      return 2 * align_up(e * 2, 1024);
  }
}



long long mp::plane_offset_elems(int N, int fmt) {
  size_t ld = (size_t)ld_for(N, fmt);
  return (long long)(align_up((size_t)N * ld * 2, 1024) / 2);
}

int mp::float_fmt(matpow_precision p) {
  switch (p) {
    case MATPOW_BF16:
      return FMT_BF16;
    case MATPOW_BF16X3:
      return FMT_FX2;
    case MATPOW_BF16X6:
      return FMT_FX3;
    default:
      return FMT_F32;
  }
}

int mp::plan_float_fmt(const matpow_plan_s* p) {
  int f = float_fmt(p->prec);
  if (f == FMT_FX2 && p->split_mode == 1) return FMT_PLANES;
  return f;
}

static size_t plan_bytes(int max_n, matpow_precision prec, size_t* buf_bytes) {
  // four partial products in the float format; the mod-p path reuses the
  // same buffers (uint32 or two bfloat16 planes take the same 4 bytes/entry)
  size_t bf = std::max(matrix_bytes(max_n, float_fmt(prec)), matrix_bytes(max_n, FMT_U32));
  bf = std::max(bf, matrix_bytes(max_n, FMT_MODP));
  if (prec == MATPOW_BF16X3) bf = std::max(bf, matrix_bytes(max_n, FMT_PLANES));
  if (buf_bytes) *buf_bytes = bf;
  return 4 * bf + align_up(sizeof(Scale) * kSingleSlots, 1024) + 1024;
}

extern "C" size_t matpow_workspace_size(int max_n, matpow_precision precision) {
  if (max_n < 1) return 0;
  return plan_bytes(max_n, precision, nullptr);
}

// ---------------------------------------------------------------------------
// plan

extern "C" matpow_status matpow_plan(matpow_plan_t* out, int max_n, matpow_precision precision,
                                     size_t workspace_bytes, int device) {
  if (!out) return fail(nullptr, MATPOW_EINVAL, "matpow_plan: out is NULL");
  *out = nullptr;
  if (max_n < 1) return fail(nullptr, MATPOW_EINVAL, "matpow_plan: max_n must be >= 1");
  if (precision != MATPOW_FP32_SIMT && precision != MATPOW_BF16 && precision != MATPOW_BF16X3 &&
      precision != MATPOW_BF16X6)
    return fail(nullptr, MATPOW_EINVAL, "matpow_plan: unknown precision %d", (int)precision);
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev)
    return fail(nullptr, MATPOW_EINVAL, "matpow_plan: device %d out of range (%d devices)", device,
                ndev);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, MATPOW_EUNSUPPORTED,
                "matpow_plan: device %d is sm_%d%d; libmatpow is built for sm_103a only", device,
                prop.major, prop.minor);
  size_t bufb = 0;
  size_t need = plan_bytes(max_n, precision, &bufb);
  if (workspace_bytes && need > workspace_bytes)
    return fail(nullptr, MATPOW_ENOMEM, "matpow_plan: needs %zu workspace bytes, limit %zu", need,
                workspace_bytes);

  auto* p = new (std::nothrow) matpow_plan_s();
  if (!p) return fail(nullptr, MATPOW_ENOMEM, "matpow_plan: host allocation failed");
  p->device = device;
  p->max_n = max_n;
  p->prec = precision;
  p->num_sms = prop.multiProcessorCount;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  e = cudaMalloc(&p->ws, need);
  if (e != cudaSuccess) {
    cudaSetDevice(prev);
    delete p;
    cudaGetLastError();
    return fail(nullptr, MATPOW_ENOMEM, "matpow_plan: cudaMalloc(%zu) failed: %s", need,
                cudaGetErrorString(e));
  }
  p->ws_bytes = need;
  char* base = (char*)p->ws;
  for (int i = 0; i < 4; ++i) p->buf[i] = base + i * bufb;
  p->buf_bytes = bufb;
  p->scales = (Scale*)(base + 4 * bufb);
  p->status = (unsigned*)(base + 4 * bufb + align_up(sizeof(Scale) * kSingleSlots, 1024));
  p->gbar = p->status + 32;  // own 128-byte line
  e = cudaMemset(p->ws, 0, need);
  if (e == cudaSuccess) e = tiny_attrs();
  if (e == cudaSuccess) e = tc_init(p);
  if (e == cudaSuccess) e = tc_chain_init(p);
  if (e == cudaSuccess) e = tc_modp_init();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_status, 4 * sizeof(unsigned));  // status, expm norm
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    matpow_plan_destroy(p);
    return cuda_fail(nullptr, e, "matpow_plan setup");
  }
  *out = p;
  return MATPOW_OK;
}

static void drop_graphs(matpow_plan_s* p) {
  for (auto& g : p->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
  }
  p->graphs.clear();
}

void mp::drop_plan_graphs(matpow_plan_s* p) { drop_graphs(p); }

extern "C" matpow_status matpow_plan_destroy(matpow_plan_t p) {
  if (!p) return MATPOW_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  drop_graphs(p);
  for (auto& k : p->timing)
    for (auto& ev : k.pending) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  for (auto& ev : p->event_pool) cudaEventDestroy(ev);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->ws) cudaFree(p->ws);
  if (p->expm_ws) cudaFree(p->expm_ws);
  if (p->expm_ev) cudaEventDestroy(p->expm_ev);
  batch_free(p);
  tc_free(p);
  if (p->h_status) cudaFreeHost(p->h_status);
  cudaSetDevice(prev);
  delete p;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_plan_set_option(matpow_plan_t p, int key, int64_t value) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_plan_set_option: plan is NULL");
  switch (key) {
    case MATPOW_OPT_GRAPHS:
      p->use_graphs = value != 0;
      if (!p->use_graphs) drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_TIMING:
      p->timing_on = value != 0;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_TINY_MAX:
      if (value < 0 || value > tiny_max_supported())
        return fail(p, MATPOW_EINVAL, "tiny_max must be in [0, %d]", tiny_max_supported());
      p->tiny_max = (int)value;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_TILE:
      if (value != 0 && value != 64 && value != 128 && value != 256)
        return fail(p, MATPOW_EINVAL, "tile width must be 0, 64, 128 or 256");
      p->tile_override = (int)value;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_CHAIN:
      if (value < 0 || value > 2) return fail(p, MATPOW_EINVAL, "chain mode must be 0, 1 or 2");
      p->chain_mode = (int)value;
      return MATPOW_OK;
    case MATPOW_OPT_NAIVE:
      p->naive = value != 0;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_PERSIST:
      p->persist = value != 0;
      return MATPOW_OK;
    case MATPOW_OPT_PAIR:
      p->pair = value != 0;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_MODP_TC:
      p->modp_tc = value != 0;
      drop_graphs(p);
      return MATPOW_OK;
    case MATPOW_OPT_SPLIT:
      if (value != 0 && value != 1) return fail(p, MATPOW_EINVAL, "split mode must be 0 or 1");
      p->split_mode = (int)value;
      drop_graphs(p);
      return MATPOW_OK;
    default:
      return fail(p, MATPOW_EINVAL, "unknown option %d", key);
  }
}

// ---------------------------------------------------------------------------
// timing

cudaEvent_t mp::take_event(matpow_plan_s* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void mp::timed_begin(matpow_plan_s* p, cudaStream_t s, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!p->timing_on) return;
  *ev = take_event(p);
  cudaEventRecord(*ev, s);
}

void mp::timed_end(matpow_plan_s* p, cudaStream_t s, cudaEvent_t ev, int kind, double flop) {
  if (!p->timing_on || !ev) return;
  cudaEvent_t e2 = take_event(p);
  cudaEventRecord(e2, s);
  p->timing[kind].pending.push_back({ev, e2});
  p->timing[kind].pending_flop.push_back(flop);
}

extern "C" matpow_status matpow_kernel_time(matpow_plan_t p, int kind, int64_t* launches,
                                            double* total_ms, double* flop, int reset) {
  if (!p || kind < 0 || kind >= MATPOW_KERNEL_KINDS)
    return fail(p, MATPOW_EINVAL, "matpow_kernel_time: bad arguments");
  auto& k = p->timing[kind];
  for (size_t i = 0; i < k.pending.size(); ++i) {
    cudaError_t e = cudaEventSynchronize(k.pending[i].second);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventSynchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, k.pending[i].first, k.pending[i].second);
    k.total_ms += ms;
    k.launches += 1;
    k.flop += k.pending_flop[i];
    p->event_pool.push_back(k.pending[i].first);
    p->event_pool.push_back(k.pending[i].second);
  }
  k.pending.clear();
  k.pending_flop.clear();
  if (launches) *launches = k.launches;
  if (total_ms) *total_ms = k.total_ms;
  if (flop) *flop = k.flop;
  if (reset) {
    k.launches = 0;
    k.total_ms = 0.0;
    k.flop = 0.0;
  }
  return MATPOW_OK;
}

extern "C" int64_t matpow_launch_count(matpow_plan_t p) { return p ? p->launches : 0; }

extern "C" int matpow_plan_sm_count(matpow_plan_t p) { return p ? p->num_sms : 0; }

extern "C" int matpow_host_accessible(const void* ptr, int device) {
  if (!ptr) return 0;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      return a.device == device ? 1 : 0;
    case cudaMemoryTypeManaged:
      return 1;
    case cudaMemoryTypeHost:  // page-locked: usable when mapped at its host address
      return a.devicePointer == ptr ? 1 : 0;
    default:
      return 0;
  }
}

// ---------------------------------------------------------------------------
// scheduling one power

// Build the level list for A^n with the stored A in buffer 0 / slot 1.
void mp::build_schedule(uint64_t n, std::vector<LevelOps>* levels) {
  levels->clear();
  int refs[4] = {1, 0, 0, 0};
  auto take = [&]() {
    for (int i = 0; i < 4; ++i)
      if (refs[i] == 0) {
        refs[i] = 1;
        return i;
      }
    return -1;  // unreachable: at most four matrices are live
  };
  int Pb = 0, Ps = 1, Rb = -1, Rs = -1, next_slot = 2;
  uint64_t bits = n;
  while (bits) {
    LevelOps lv;
    int newRb = -1, newRs = -1, newPb = -1, newPs = -1;
    if (bits & 1ull) {
      if (Rb < 0) {
        Rb = Pb;
        Rs = Ps;
        refs[Pb]++;
      } else {
        newRb = take();
        newRs = next_slot++;
        lv.ops.push_back({Rb, Pb, newRb, Rs, Ps, newRs, false});
      }
    }
    bits >>= 1;
    if (bits) {
      newPb = take();
      newPs = next_slot++;
      lv.ops.push_back({Pb, Pb, newPb, Ps, Ps, newPs, true});
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
    if (!lv.ops.empty()) levels->push_back(lv);
  }
}

static int tiles_for(int N, int edge) { return (N + edge - 1) / edge; }

// Enqueue every kernel of one float power on stream s (no graph logic here).
static matpow_status enqueue_f32(matpow_plan_s* p, const float* dA, int N, uint64_t n, float* dOut,
                                 int64_t* dLog2, cudaStream_t s) {
  cudaEvent_t ev;
  if (n == 0) {
    CK(p, launch_identity(dOut, N, 0, 0, (long long*)dLog2, s));
    p->launches++;
    return MATPOW_OK;
  }
  if (n == 1) {
    CK(p, launch_copy(dA, dOut, N, (long long*)dLog2, s));
    p->launches++;
    return MATPOW_OK;
  }
  if (N <= p->tiny_max) {
    TinyDesc d{dA, dOut, (long long*)dLog2, (unsigned long long)n, N, 0};
    timed_begin(p, s, &ev);
    CK(p, launch_tiny_one(d, p->status, s));
    timed_end(p, s, ev, MATPOW_KERNEL_TINY, 2.0 * N * N * (double)N * matpow_gemm_count(n));
    p->launches++;
    return MATPOW_OK;
  }
  const int fmt = plan_float_fmt(p);
  const long long plane = plane_offset_elems(N, fmt);
  const int ld = ld_for(N, fmt);
  const bool fx2 = fmt_exact(fmt);
  std::vector<LevelOps> levels;
  int nslots;
  if (p->naive) {
    // the comparison method (§4.2): n - 1 products R <- R A, one launch each;
    // R alternates between buffers 1 and 2 and scale slots 2 and 3 (a slot
    // is cleared before the product that writes it)
    for (uint64_t k = 1; k < n; ++k) {
      LevelOps lv;
      const int xb = k == 1 ? 0 : 1 + (int)(k & 1), xs = k == 1 ? 1 : 2 + (int)(k & 1);
      const int cb = 1 + (int)((k + 1) & 1), cs = 2 + (int)((k + 1) & 1);
      lv.ops.push_back({xb, 0, cb, xs, 1, cs, false});
      levels.push_back(lv);
    }
    nslots = 4;
  } else {
    build_schedule(n, &levels);
    nslots = 2 + matpow_gemm_count(n);
  }
  CK(p, cudaMemsetAsync(p->scales, 0, sizeof(Scale) * nslots, s));
  if (fx2) {
    // slot 1 describes A itself (exponent 0): block slices, max|A|
    CK(p, launch_prep_fxb(dA, N, fmt, p->buf[0], &p->scales[1], p->status, s));
    p->launches += 1;
  } else {
    CK(p, launch_absmax_f32(dA, N, &p->scales[0], p->status, s));
    CK(p, launch_convert_f32(dA, N, &p->scales[0], &p->scales[1], fmt, p->buf[0], plane, s));
    p->launches += 2;
  }
  const bool tc = p->prec != MATPOW_FP32_SIMT;
  for (size_t li = 0; li < levels.size(); ++li) {
    const LevelOps& lv = levels[li];
    GemmPair g{};
    g.count = (int)lv.ops.size();
    const int t128 = tiles_for(N, 128);
    const int edge = simt_tile_edge(g.count * t128 * t128, p->num_sms);  // SIMT tiles
    const int te = tiles_for(N, edge);
    const int split = p->chain_mode == 2 ? 1 : simt_split(edge, g.count * te * te, p->num_sms);
    int t = 0;
    for (int i = 0; i < g.count; ++i) {
      const Op& op = lv.ops[i];
      const bool last = (li + 1 == levels.size()) && (i + 1 == g.count);
      GemmDesc& d = g.d[i];
      d.X = p->buf[op.xb];
      d.Y = p->buf[op.yb];
      d.C = last ? nullptr : p->buf[op.cb];
      d.out = last ? (void*)dOut : nullptr;
      d.out_log2 = last ? (long long*)dLog2 : nullptr;
      d.plane = plane;
      d.N = N;
      d.ld = ld;
      d.sx = op.sx;
      d.sy = op.sy;
      d.sc = op.sc;
      d.mode = last ? (dLog2 ? OUT_USER_MANT : OUT_USER_VALUE) : OUT_INTERNAL;
      d.tile_begin = t;
      if (tc) {
        int nt = 0;
        matpow_status st = tc_fill_desc(p, &d, &nt);
        if (st != MATPOW_OK) return st;
        t += nt;
      } else {
        d.tiles_n = tiles_for(N, edge);
        t += d.tiles_n * d.tiles_n;
      }
    }
    g.tiles_total = t;
    if (p->naive && li >= 2)  // the slot this product writes held R two products ago
      CK(p, cudaMemsetAsync(&p->scales[lv.ops[0].sc], 0, sizeof(Scale), s));
    const double flop = 2.0 * N * (double)N * N * g.count;
    timed_begin(p, s, &ev);
    if (tc) {
      matpow_status st = tc_launch_pair(p, g, s);
      if (st != MATPOW_OK) return st;
      timed_end(p, s, ev, MATPOW_KERNEL_TC, flop);
    } else {
      CK(p, launch_simt_pair(g, edge, split, p->scales, p->status, s));
      timed_end(p, s, ev, MATPOW_KERNEL_SIMT, flop);
    }
    p->launches++;
  }
  return MATPOW_OK;
}

static matpow_status enqueue_modp(matpow_plan_s* p, const uint32_t* dA, int N, uint64_t n,
                                  uint32_t pmod, uint32_t* dOut, cudaStream_t s) {
  cudaEvent_t ev;
  if (n == 0) {
    CK(p, launch_identity(dOut, N, 1, 1u % pmod, nullptr, s));
    p->launches++;
    return MATPOW_OK;
  }
  if (n >= 2 && p->modp_tc && N > 64 && N <= 16384) {
    // tensor cores: byte slices, exact chunk sums, Barrett reduction
    const int ldm = ld_for(N, FMT_MODP);
    const long long plane = plane_offset_elems(N, FMT_MODP);
    CK(p, launch_prep_modp_slices(dA, N, pmod, p->buf[0], p->status, s));
    p->launches++;
    std::vector<LevelOps> levels;
    build_schedule(n, &levels);
    const int tn = (N + tc_modp_tile_n() - 1) / tc_modp_tile_n();
    const int tm = (N + 127) / 128;
    for (size_t li = 0; li < levels.size(); ++li) {
      const LevelOps& lv = levels[li];
      GemmPair g{};
      g.count = (int)lv.ops.size();
      int t = 0;
      for (int i = 0; i < g.count; ++i) {
        const Op& op = lv.ops[i];
        const bool last = (li + 1 == levels.size()) && (i + 1 == g.count);
        GemmDesc& d = g.d[i];
        d.X = p->buf[op.xb];
        d.Y = p->buf[op.yb];
        d.C = last ? nullptr : p->buf[op.cb];
        d.out = last ? (void*)dOut : nullptr;
        d.N = N;
        d.ld = ldm;
        d.plane = plane;
        d.mode = last ? OUT_USER_VALUE : OUT_INTERNAL;
        d.p = pmod;
        d.tile_begin = t;
        d.tiles_n = tn;
        t += tm * tn;
      }
      g.tiles_total = t;
      timed_begin(p, s, &ev);
      matpow_status st = tc_modp_launch_pair(p, g, s);
      if (st != MATPOW_OK) return st;
      timed_end(p, s, ev, MATPOW_KERNEL_MODP, 2.0 * N * (double)N * N * g.count);
      p->launches++;
    }
    return MATPOW_OK;
  }
  // check entries (and copy into the stored format) for every n >= 1
  const int ld = ld_for(N, FMT_U32);
  CK(p, launch_modp_check_convert(dA, N, pmod, (unsigned*)p->buf[0], p->status, s));
  p->launches++;
  if (n == 1) {
    CK(p, cudaMemcpy2DAsync(dOut, (size_t)N * 4, p->buf[0], (size_t)ld * 4, (size_t)N * 4, N,
                            cudaMemcpyDefault, s));  // dOut: device or mapped host memory
    return MATPOW_OK;
  }
  std::vector<LevelOps> levels;
  build_schedule(n, &levels);
  for (size_t li = 0; li < levels.size(); ++li) {
    const LevelOps& lv = levels[li];
    GemmPair g{};
    g.count = (int)lv.ops.size();
    int t = 0;
    for (int i = 0; i < g.count; ++i) {
      const Op& op = lv.ops[i];
      const bool last = (li + 1 == levels.size()) && (i + 1 == g.count);
      GemmDesc& d = g.d[i];
      d.X = p->buf[op.xb];
      d.Y = p->buf[op.yb];
      d.C = last ? nullptr : p->buf[op.cb];
      d.out = last ? (void*)dOut : nullptr;
      d.N = N;
      d.ld = ld;
      d.mode = last ? OUT_USER_VALUE : OUT_INTERNAL;
      d.p = pmod;
      d.tile_begin = t;
      d.tiles_n = tiles_for(N, modp_tile_edge());
      t += d.tiles_n * d.tiles_n;
    }
    g.tiles_total = t;
    timed_begin(p, s, &ev);
    CK(p, launch_modp_pair(g, p->status, s));
    timed_end(p, s, ev, MATPOW_KERNEL_MODP, 2.0 * N * (double)N * N * g.count);
    p->launches++;
  }
  return MATPOW_OK;
}

matpow_status mp::enqueue_product_f32(matpow_plan_s* p, const float* X, const float* Y, int N, float* out,
                                      cudaStream_t s, bool keep_x) {
  const int fmt = plan_float_fmt(p);
  const long long plane = plane_offset_elems(N, fmt);
  if (keep_x) {  // X's split and slot 1 stay; clear Y's and the output's slots
    CK(p, cudaMemsetAsync(&p->scales[2], 0, sizeof(Scale) * 2, s));
  } else {
    CK(p, cudaMemsetAsync(p->scales, 0, sizeof(Scale) * 4, s));
  }
  if (fmt_exact(fmt)) {
    if (!keep_x) CK(p, launch_prep_fxb(X, N, fmt, p->buf[0], &p->scales[1], p->status, s));
    CK(p, launch_prep_fxb(Y, N, fmt, p->buf[1], &p->scales[2], p->status, s));
    p->launches += keep_x ? 1 : 2;
  } else {
    if (!keep_x) {
      CK(p, launch_absmax_f32(X, N, &p->scales[0], p->status, s));
      CK(p, launch_convert_f32(X, N, &p->scales[0], &p->scales[1], fmt, p->buf[0], plane, s));
      p->launches += 2;
    }
    CK(p, cudaMemsetAsync(&p->scales[0], 0, sizeof(Scale), s));  // slot 0 again for Y's maximum
    CK(p, launch_absmax_f32(Y, N, &p->scales[0], p->status, s));
    CK(p, launch_convert_f32(Y, N, &p->scales[0], &p->scales[2], fmt, p->buf[1], plane, s));
    p->launches += 2;
  }
  GemmPair g{};
  g.count = 1;
  GemmDesc& d = g.d[0];
  d.X = p->buf[0];
  d.Y = p->buf[1];
  d.C = nullptr;
  d.out = out;
  d.out_log2 = nullptr;
  d.plane = plane;
  d.N = N;
  d.ld = ld_for(N, fmt);
  d.sx = 1;
  d.sy = 2;
  d.sc = 3;
  d.mode = OUT_USER_VALUE;
  d.tile_begin = 0;
  cudaEvent_t ev;
  const double flop = 2.0 * N * (double)N * N;
  timed_begin(p, s, &ev);
  if (p->prec != MATPOW_FP32_SIMT) {
    int nt = 0;
    matpow_status st = tc_fill_desc(p, &d, &nt);
    if (st != MATPOW_OK) return st;
    g.tiles_total = nt;
    st = tc_launch_pair(p, g, s);
    if (st != MATPOW_OK) return st;
    timed_end(p, s, ev, MATPOW_KERNEL_TC, flop);
  } else {
    const int t128 = tiles_for(N, 128);
    const int edge = simt_tile_edge(t128 * t128, p->num_sms);
    d.tiles_n = tiles_for(N, edge);
    g.tiles_total = d.tiles_n * d.tiles_n;
    const int split = p->chain_mode == 2 ? 1 : simt_split(edge, g.tiles_total, p->num_sms);
    CK(p, launch_simt_pair(g, edge, split, p->scales, p->status, s));
    timed_end(p, s, ev, MATPOW_KERNEL_SIMT, flop);
  }
  p->launches++;
  return MATPOW_OK;
}

// ---------------------------------------------------------------------------
// graph replay of repeated calls

template <class F>
static matpow_status run_maybe_graph(matpow_plan_s* p, const GraphKey& key, cudaStream_t s,
                                     F&& enqueue) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(p, cudaStreamIsCapturing(s, &cs));
  const bool graphable = p->use_graphs && !p->timing_on && cs == cudaStreamCaptureStatusNone;
  if (!graphable) return enqueue(s);
  for (auto& g : p->graphs) {
    if (g.key == key) {
      g.stamp = ++p->graph_clock;
      CK(p, cudaGraphLaunch(g.exec, s));
      p->launches += g.kernels;
      return MATPOW_OK;
    }
  }
  // capture on the plan's own stream, then launch into the caller's stream
  int64_t before = p->launches;
  CK(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  matpow_status st = enqueue(p->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
  if (st != MATPOW_OK) {
    if (graph) cudaGraphDestroy(graph);
    p->launches = before;
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaGraphInstantiate");
  GraphEntry ge;
  ge.key = key;
  ge.exec = exec;
  ge.kernels = p->launches - before;
  ge.stamp = ++p->graph_clock;
  p->launches = before;
  if (p->graphs.size() >= kMaxGraphs) {
    auto it = std::min_element(p->graphs.begin(), p->graphs.end(),
                               [](const GraphEntry& a, const GraphEntry& b) { return a.stamp < b.stamp; });
    cudaGraphExecDestroy(it->exec);
    p->graphs.erase(it);
  }
  p->graphs.push_back(ge);
  CK(p, cudaGraphLaunch(exec, s));
  p->launches += ge.kernels;
  return MATPOW_OK;
}

matpow_status mp::run_graph_or_direct(matpow_plan_s* p, const GraphKey& key, cudaStream_t s,
                                      const std::function<matpow_status(cudaStream_t)>& enqueue) {
  return run_maybe_graph(p, key, s, enqueue);
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != prev) cudaSetDevice(prev);
  }
};

extern "C" matpow_status matpow_f32(matpow_plan_t p, const float* dA, int N, uint64_t n, float* dOut,
                                    int64_t* dLog2Scale, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_f32: plan is NULL");
  if (N < 0 || N > p->max_n)
    return fail(p, MATPOW_EINVAL, "matpow_f32: N=%d outside [0, %d]", N, p->max_n);
  if (N == 0) return MATPOW_OK;
  if (!dA || !dOut) return fail(p, MATPOW_EINVAL, "matpow_f32: NULL matrix pointer");
  if (((uintptr_t)dA & 3) || ((uintptr_t)dOut & 3) || ((uintptr_t)dLog2Scale & 7))
    return fail(p, MATPOW_EINVAL, "matpow_f32: misaligned pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  bool used = false;
  matpow_status cst = tc_chain_run(p, dA, N, n, dOut, dLog2Scale, s, &used);
  if (cst != MATPOW_OK || used) return cst;
  GraphKey key{0, dA, dOut, dLog2Scale, N, n, 0};
  return run_maybe_graph(p, key, s, [&](cudaStream_t st) {
    return enqueue_f32(p, dA, N, n, dOut, dLog2Scale, st);
  });
}

extern "C" matpow_status matpow_mod_p(matpow_plan_t p, const uint32_t* dA, int N, uint64_t n,
                                      uint32_t pmod, uint32_t* dOut, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_mod_p: plan is NULL");
  if (N < 0 || N > p->max_n)
    return fail(p, MATPOW_EINVAL, "matpow_mod_p: N=%d outside [0, %d]", N, p->max_n);
  if (pmod < 2 || pmod > 65536)
    return fail(p, MATPOW_EINVAL, "matpow_mod_p: p=%u outside [2, 65536]", pmod);
  if (N == 0) return MATPOW_OK;
  if (!dA || !dOut) return fail(p, MATPOW_EINVAL, "matpow_mod_p: NULL matrix pointer");
  if (((uintptr_t)dA & 3) || ((uintptr_t)dOut & 3))
    return fail(p, MATPOW_EINVAL, "matpow_mod_p: misaligned pointer");
  DeviceGuard dg(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  GraphKey key{1, dA, dOut, nullptr, N, n, pmod};
  return run_maybe_graph(p, key, s, [&](cudaStream_t st) {
    return enqueue_modp(p, dA, N, n, pmod, dOut, st);
  });
}

extern "C" matpow_status matpow_selftest_wait_timeout(matpow_plan_t p, uint64_t budget_ns, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_selftest_wait_timeout: plan is NULL");
  if (budget_ns < 1000ull || budget_ns > 10000000000ull)
    return fail(p, MATPOW_EINVAL, "matpow_selftest_wait_timeout: budget_ns must be in [1e3, 1e10]");
  DeviceGuard dg(p->device);
  CK(p, launch_selftest_wait((unsigned long long)budget_ns, p->status, (cudaStream_t)stream));
  p->launches++;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_selftest_ffma(matpow_plan_t p, int64_t iters, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_selftest_ffma: plan is NULL");
  if (iters < 16 || iters > (int64_t)1 << 32 || (iters & 15))
    return fail(p, MATPOW_EINVAL, "matpow_selftest_ffma: iters must be a multiple of 16 in [16, 2^32]");
  DeviceGuard dg(p->device);
  // eight CTAs of 256 threads per SM: 64 warps, each with 8 independent chains
  CK(p, launch_ffma_probe((long long)iters, 8 * p->num_sms, p->status + 3, (cudaStream_t)stream));
  p->launches++;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_sync(matpow_plan_t p, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_sync: plan is NULL");
  DeviceGuard dg(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  CK(p, cudaStreamSynchronize(s));
  CK(p, cudaMemcpy(p->h_status, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  unsigned st = *p->h_status;
  if (st) CK(p, cudaMemset(p->status, 0, sizeof(unsigned)));
  if (st & ST_BADINPUT)
    return fail(p, MATPOW_EINVAL, "device: non-finite input or an entry >= p");
  if (st & ST_TIMEOUT) return fail(p, MATPOW_ETIMEDOUT, "device: a bounded wait gave up");
  if (st & ST_RANGE) return fail(p, MATPOW_ERANGE, "device: result outside the float32 range");
  return MATPOW_OK;
}
