// Request server: continuous batching of independent A^n requests.
//
// Each request is the paper's method (arXiv 1204.3052 Sec. 4.3) on its own
// matrix.  A scheduler thread owns one CUDA stream and loops:
//   1. admit queued requests (FIFO) while their device footprint fits the
//      arena and fewer than max_inflight run; each gets four partial-product
//      buffers, a chunk of scale slots and a status word;
//   2. build one step: the preparation of newly admitted requests, and the
//      NEXT level's products of every admitted request -- float products of
//      all requests in one grouped launch, mod-p products in another; small
//      float requests (N <= 64) run their whole chain in one grouped launch;
//   3. enqueue the step, record an event, and retire the requests whose last
//      product was in an earlier step whose event has completed.
// Requests that arrive while a step is on the GPU join the next step at their
// first level, so the batch changes every step (continuous batching); freed
// buffers are reused by later admissions in stream order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "plan.h"

using namespace mp;

namespace {

constexpr int kSlotsPerReq = 2 + 2 * 64;  // 2 + G(n) for any uint64 n
using Clock = std::chrono::steady_clock;

struct Range {
  size_t off, len;
};

// First-fit allocator over one device arena (offsets; 1 KB granularity).
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    free_.push_back({0, bytes});
  }
  bool alloc(size_t len, size_t* off) {
    len = (len + 1023) & ~(size_t)1023;
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].len >= len) {
        *off = free_[i].off;
        free_[i].off += len;
        free_[i].len -= len;
        if (!free_[i].len) free_.erase(free_.begin() + i);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t len) {
    len = (len + 1023) & ~(size_t)1023;
    auto it = std::lower_bound(free_.begin(), free_.end(), off,
                               [](const Range& r, size_t o) { return r.off < o; });
    it = free_.insert(it, {off, len});
    // merge neighbours
    size_t i = it - free_.begin();
    if (i + 1 < free_.size() && free_[i].off + free_[i].len == free_[i + 1].off) {
      free_[i].len += free_[i + 1].len;
      free_.erase(free_.begin() + i + 1);
    }
    if (i > 0 && free_[i - 1].off + free_[i - 1].len == free_[i].off) {
      free_[i - 1].len += free_[i].len;
      free_.erase(free_.begin() + i);
    }
  }

 private:
  std::vector<Range> free_;
};

struct Req {
  uint64_t ticket = 0;
  matpow_request r{};
  Clock::time_point t_submit, t_done;
  std::atomic<int> state{0};  // 0 queued, 1 active, 2 final work enqueued, 3 done
  matpow_status result = MATPOW_OK;
  // device resources
  size_t off = 0, bytes = 0;
  int chunk = -1;  // slot chunk index
  std::vector<LevelOps> levels;
  size_t next_level = 0;
  bool tiny = false;
  bool tcm = false;  // mod p on the tensor cores (byte-slice planes)
  bool prepared = false;
  uint64_t done_step = 0;
};

}  // namespace

struct matpow_server_s {
  matpow_server_desc desc{};
  int fmt = FMT_F32;  // FMT_FX2 / FMT_FX3: float levels on the tensor cores (exact split)
  int num_sms = 0;
  CUtensorMap* d_maps = nullptr;  // 24 TMA descriptors per slot chunk (4 buffers x 2 x 3)
  CUtensorMap* h_maps = nullptr;  // pinned host copy
  cudaStream_t stream = nullptr;
  void* arena_mem = nullptr;
  Arena arena;
  Scale* scales = nullptr;     // max_inflight * kSlotsPerReq slots
  unsigned* status = nullptr;  // word 0: step-wide; word 32 (c + 1): slot chunk c
  std::vector<unsigned> h_status;
  std::vector<int> free_chunks;
  // descriptor staging (two halves, each guarded by an event)
  void* d_tab = nullptr;
  void* h_tab[2] = {nullptr, nullptr};
  size_t tab_bytes = 0;
  cudaEvent_t tab_ev[2] = {nullptr, nullptr};
  int tab_i = 0;
  // steps
  std::deque<std::pair<uint64_t, cudaEvent_t>> step_events;
  std::vector<cudaEvent_t> event_pool;
  uint64_t step_no = 0;
  // requests
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<uint64_t, Req*> all;
  std::vector<double> latencies_us;
  uint64_t next_ticket = 1;
  bool stop = false;
  matpow_status fatal = MATPOW_OK;
  std::thread th;
  std::string err;
};

static matpow_status sfail(matpow_server_s* s, matpow_status st, const char* msg) {
  if (s) s->err = msg;
  return fail(nullptr, st, "%s", msg);
}

static size_t footprint(const matpow_server_s* s, const matpow_request& r) {
  if (r.kind == 1)  // uint32 (CUDA cores) or two byte-slice planes (tensor cores)
    return 4 * std::max(matrix_bytes(r.N, FMT_U32), matrix_bytes(r.N, FMT_MODP));
  return 4 * matrix_bytes(r.N, s->fmt);
}

static cudaEvent_t take_ev(matpow_server_s* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

static bool ensure_tab(matpow_server_s* s, size_t need) {
  if (need <= s->tab_bytes) return true;
  size_t n = std::max(need, s->tab_bytes * 2);
  cudaStreamSynchronize(s->stream);
  for (int i = 0; i < 2; ++i) {
    if (s->h_tab[i]) cudaFreeHost(s->h_tab[i]);
    s->h_tab[i] = nullptr;
  }
  if (s->d_tab) cudaFree(s->d_tab);
  s->d_tab = nullptr;
  if (cudaMalloc(&s->d_tab, 2 * n) != cudaSuccess) return false;
  for (int i = 0; i < 2; ++i)
    if (cudaMallocHost(&s->h_tab[i], n) != cudaSuccess) return false;
  s->tab_bytes = n;
  return true;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// One scheduler step (called with the lock NOT held; touches only scheduler state
// and requests in `active`, which submit/poll never modify).
static matpow_status run_step(matpow_server_s* s, std::vector<Req*>& act, uint64_t step) {
  std::vector<TinyDesc> tiny;
  std::vector<PrepDesc> prep;
  std::vector<GemmDesc> gf, gw, gm, gt;  // float (64-wide tiles), float (128-wide), mod p (CUDA / tensor cores)
  int tiles_f = 0, tiles_w = 0, tiles_m = 0, tiles_t = 0, maxn_f = 0;
  std::vector<Req*> modp_prep;
  for (Req* q : act) {
    if (q->state != 1) continue;
    const matpow_request& r = q->r;
    char* base = (char*)s->arena_mem + q->off;
    Scale* sl = s->scales + q->chunk * kSlotsPerReq;
    if (r.kind == 0 && q->tiny) {
      tiny.push_back({(const float*)r.dA, (float*)r.dOut, (long long*)r.dLog2Scale,
                      (unsigned long long)r.n, r.N, 0});
      q->state = 2;
      q->done_step = step;
      continue;
    }
    if (r.n <= 1) {  // identity or copy, through the prep table
      if (r.kind == 0) {
        PrepDesc d{};
        d.A = (const float*)r.dA;
        d.dst = r.dOut;
        d.log2 = (long long*)r.dLog2Scale;
        d.N = r.N;
        d.kind = r.n == 0 ? 1 : 2;
        prep.push_back(d);
        q->state = 2;
        q->done_step = step;
        continue;
      }
      if (r.n == 0) {
        cudaError_t e = launch_identity(r.dOut, r.N, 1, 1u % r.p, nullptr, s->stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "server identity");
        q->state = 2;
        q->done_step = step;
        continue;
      }
    }
    const size_t mb = q->bytes / 4;
    if (!q->prepared) {
      if (r.kind == 0) {
        PrepDesc d{};
        d.A = (const float*)r.dA;
        d.dst = base;
        d.N = r.N;
        d.fmt = s->fmt;
        d.plane = plane_offset_elems(r.N, s->fmt);
        d.slot_raw = (int)(sl - s->scales) + 0;
        d.slot_stored = (int)(sl - s->scales) + 1;
        d.kind = 0;
        prep.push_back(d);
      } else {
        modp_prep.push_back(q);
      }
      q->prepared = true;
      if (r.kind == 1 && r.n == 1) {  // copy after the entry check
        q->state = 2;
        q->done_step = step;
        continue;
      }
      continue;  // products start next step, after the preparation ran
    }
    // the next level of this request
    const LevelOps& lv = q->levels[q->next_level];
    const bool final_level = q->next_level + 1 == q->levels.size();
    for (size_t k = 0; k < lv.ops.size(); ++k) {
      const Op& op = lv.ops[k];
      const bool last = final_level && k + 1 == lv.ops.size();
      GemmDesc d{};
      d.X = base + op.xb * mb;
      d.Y = base + op.yb * mb;
      d.C = last ? nullptr : base + op.cb * mb;
      d.out = last ? r.dOut : nullptr;
      d.N = r.N;
      const int slot0 = (int)(sl - s->scales);
      d.sx = slot0 + op.sx;
      d.sy = slot0 + op.sy;
      d.sc = slot0 + op.sc;
      if (r.kind == 0) {
        d.out_log2 = last ? (long long*)r.dLog2Scale : nullptr;
        d.ld = ld_for(r.N, s->fmt);
        d.plane = plane_offset_elems(r.N, s->fmt);
        d.mode = last ? (r.dLog2Scale ? OUT_USER_MANT : OUT_USER_VALUE) : OUT_INTERNAL;
        if (fmt_exact(s->fmt)) {
          const int mpb = 2 * fmt_slices(s->fmt);
          d.bn = tc_group_bn(r.N, fmt_slices(s->fmt));
          d.tiles_n = (r.N + d.bn - 1) / d.bn;
          d.map_x = 24 * q->chunk + mpb * op.xb;
          d.map_y = 24 * q->chunk + mpb * op.yb;
          d.map_c = 24 * q->chunk + mpb * (last ? op.xb : op.cb);
          const int nt = ((r.N + 127) / 128) * d.tiles_n;
          if (d.bn == 64) {
            d.tile_begin = tiles_f;
            tiles_f += nt;
            maxn_f = std::max(maxn_f, r.N);
            gf.push_back(d);
          } else {
            d.tile_begin = tiles_w;
            tiles_w += nt;
            gw.push_back(d);
          }
        } else {
          // 128-wide SIMT tiles: a level's requests are gathered one by one
          d.tiles_n = (r.N + 127) / 128;
          d.tile_begin = tiles_f;
          tiles_f += d.tiles_n * d.tiles_n;
          gf.push_back(d);
        }
      } else if (q->tcm) {
        d.ld = ld_for(r.N, FMT_MODP);
        d.plane = plane_offset_elems(r.N, FMT_MODP);
        d.mode = last ? OUT_USER_VALUE : OUT_INTERNAL;
        d.p = r.p;
        d.bn = tc_modp_tile_n();
        d.tiles_n = (r.N + d.bn - 1) / d.bn;
        d.map_x = 24 * q->chunk + 4 * op.xb;
        d.map_y = 24 * q->chunk + 4 * op.yb;
        d.tile_begin = tiles_t;
        tiles_t += ((r.N + 127) / 128) * d.tiles_n;
        gt.push_back(d);
      } else {
        d.ld = ld_for(r.N, FMT_U32);
        d.mode = last ? OUT_USER_VALUE : OUT_INTERNAL;
        d.p = r.p;
        d.tiles_n = (r.N + modp_tile_edge() - 1) / modp_tile_edge();
        d.tile_begin = tiles_m;
        tiles_m += d.tiles_n * d.tiles_n;
        gm.push_back(d);
      }
    }
    q->next_level++;
    if (final_level) {
      q->state = 2;
      q->done_step = step;
    }
  }
  // prep CTA layout
  int prep_blocks = 0;
  for (auto& d : prep) {
    size_t e = (size_t)d.N * d.N;
    if (fmt_exact(s->fmt) && d.kind == 0) {
      const size_t nb = ((size_t)d.N + 63) / 64;
      d.blocks = (int)(nb * nb);
    } else {
      d.blocks = (int)std::min<size_t>(std::max<size_t>((e + 16383) / 16384, 1), 1024);
    }
    d.block_begin = prep_blocks;
    prep_blocks += d.blocks;
  }
  // stage tables
  const size_t o_t = 0;
  const size_t o_p = align256(o_t + tiny.size() * sizeof(TinyDesc));
  const size_t o_f = align256(o_p + prep.size() * sizeof(PrepDesc));
  const size_t o_w = align256(o_f + gf.size() * sizeof(GemmDesc));
  const size_t o_m = align256(o_w + gw.size() * sizeof(GemmDesc));
  // tile records of the 64-column float group (persistent kernel)
  std::vector<int4> trec;
  if (fmt_exact(s->fmt)) persist_tile_records(gf.data(), (int)gf.size(), fmt_slices(s->fmt), &trec);
  const size_t o_mt = align256(o_m + gm.size() * sizeof(GemmDesc));
  const size_t o_td = align256(o_mt + gt.size() * sizeof(GemmDesc));
  const size_t total = std::max<size_t>(align256(o_td + trec.size() * sizeof(int4)), 256);
  if (!ensure_tab(s, total)) return fail(nullptr, MATPOW_ENOMEM, "server: descriptor table");
  const int ti = s->tab_i;
  s->tab_i ^= 1;
  if (s->tab_ev[ti]) cudaEventSynchronize(s->tab_ev[ti]);  // its previous upload was consumed
  char* h = (char*)s->h_tab[ti];
  char* dd = (char*)s->d_tab + ti * s->tab_bytes;
  if (!tiny.empty()) memcpy(h + o_t, tiny.data(), tiny.size() * sizeof(TinyDesc));
  if (!prep.empty()) memcpy(h + o_p, prep.data(), prep.size() * sizeof(PrepDesc));
  if (!gf.empty()) memcpy(h + o_f, gf.data(), gf.size() * sizeof(GemmDesc));
  if (!gw.empty()) memcpy(h + o_w, gw.data(), gw.size() * sizeof(GemmDesc));
  if (!gm.empty()) memcpy(h + o_m, gm.data(), gm.size() * sizeof(GemmDesc));
  if (!gt.empty()) memcpy(h + o_mt, gt.data(), gt.size() * sizeof(GemmDesc));
  if (!trec.empty()) memcpy(h + o_td, trec.data(), trec.size() * sizeof(int4));
  cudaError_t e = cudaMemcpyAsync(dd, h, total, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: upload");
  if (!s->tab_ev[ti]) cudaEventCreateWithFlags(&s->tab_ev[ti], cudaEventDisableTiming);
  cudaEventRecord(s->tab_ev[ti], s->stream);
  unsigned* st0 = s->status;  // step-wide status word (chunk status words are per request)
  if (!tiny.empty()) {
    e = launch_tiny_group((const TinyDesc*)(dd + o_t), (int)tiny.size(), st0, s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: tiny");
  }
  if (!prep.empty()) {
    const PrepDesc* pd = (const PrepDesc*)(dd + o_p);
    if (fmt_exact(s->fmt)) {
      e = launch_prep_fxb_group(pd, (int)prep.size(), prep_blocks, s->scales, st0, s->stream);
    } else {
      e = launch_prep_absmax_group(pd, (int)prep.size(), prep_blocks, s->scales, st0, s->stream);
      if (e == cudaSuccess)
        e = launch_prep_convert_group(pd, (int)prep.size(), prep_blocks, s->scales, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: prep");
  }
  for (Req* q : modp_prep) {
    char* base = (char*)s->arena_mem + q->off;
    unsigned* st = s->status + (q->chunk + 1) * 32;
    if (q->tcm)
      e = launch_prep_modp_slices((const unsigned*)q->r.dA, q->r.N, q->r.p, base, st, s->stream);
    else
      e = launch_modp_check_convert((const unsigned*)q->r.dA, q->r.N, q->r.p, (unsigned*)base, st,
                                    s->stream);
    if (e == cudaSuccess && q->r.n == 1)
      e = cudaMemcpy2DAsync(q->r.dOut, (size_t)q->r.N * 4, base, (size_t)ld_for(q->r.N, FMT_U32) * 4,
                            (size_t)q->r.N * 4, q->r.N, cudaMemcpyDefault, s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: mod-p prep");
  }
  if (!gf.empty()) {
    if (fmt_exact(s->fmt))
      e = launch_fxb_group((const GemmDesc*)(dd + o_f), (int)gf.size(), tiles_f, (const int4*)(dd + o_td),
                           s->d_maps, 64, fmt_slices(s->fmt), maxn_f, s->num_sms, true, s->scales, st0,
                           s->stream);
    else
      e = launch_simt_group((const GemmDesc*)(dd + o_f), (int)gf.size(), tiles_f, 128, 1, s->scales, st0,
                            s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: float level");
  }
  if (!gw.empty()) {
    e = launch_fxb_group((const GemmDesc*)(dd + o_w), (int)gw.size(), tiles_w, nullptr, s->d_maps, 128,
                         fmt_slices(s->fmt), 0, s->num_sms, false, s->scales, st0, s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: float level");
  }
  if (!gm.empty()) {
    e = launch_modp_group((const GemmDesc*)(dd + o_m), (int)gm.size(), tiles_m, st0, s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: mod-p level");
  }
  if (!gt.empty()) {
    e = launch_modp_tc_group((const GemmDesc*)(dd + o_mt), (int)gt.size(), tiles_t, s->d_maps, s->num_sms,
                             st0, s->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "server: mod-p level");
  }
  cudaEvent_t ev = take_ev(s);
  cudaEventRecord(ev, s->stream);
  s->step_events.push_back({step, ev});
  return MATPOW_OK;
}

static void scheduler(matpow_server_s* s) {
  cudaSetDevice(s->desc.device);
  std::vector<Req*> act;
  uint64_t completed_step = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admission: FIFO while memory, slots and the in-flight cap allow
      while (!s->queue.empty() && (int)s->active.size() < s->desc.max_inflight &&
             !s->free_chunks.empty()) {
        Req* q = s->queue.front();
        size_t off = 0;
        const size_t fp = footprint(s, q->r);
        if (!s->arena.alloc(fp, &off)) break;
        s->queue.pop_front();
        q->off = off;
        q->bytes = fp;
        q->chunk = s->free_chunks.back();
        s->free_chunks.pop_back();
        q->state = 1;
        q->tiny = q->r.kind == 0 && q->r.N <= tiny_max_supported() && q->r.n >= 2;
        // mod p on the tensor cores from N > 64 (as matpow_mod_p does)
        q->tcm = q->r.kind == 1 && q->r.n >= 2 && q->r.N > 64 && q->r.N <= 16384;
        if (q->r.n >= 2) build_schedule(q->r.n, &q->levels);
        if ((fmt_exact(s->fmt) && q->r.kind == 0 && !q->tiny && q->r.n >= 2) || q->tcm) {
          // TMA descriptors of the request's four buffers, uploaded in stream
          // order before its first product
          const int nsl = q->tcm ? 2 : fmt_slices(s->fmt);
          CUtensorMap* hm = s->h_maps + 24 * q->chunk;
          const size_t mb = fp / 4;
          bool okm = true;
          for (int k = 0; k < 4 && okm; ++k)
            okm = tc_encode_buffer_maps(hm + 2 * nsl * k, (char*)s->arena_mem + off + k * mb, q->r.N,
                                        nsl);
          if (okm)
            okm = cudaMemcpyAsync(s->d_maps + 24 * q->chunk, hm, 24 * sizeof(CUtensorMap),
                                  cudaMemcpyHostToDevice, s->stream) == cudaSuccess;
          if (!okm) {
            q->state = 3;
            q->result = MATPOW_ECUDA;
            s->arena.release(off, fp);
            s->free_chunks.push_back(q->chunk);
            s->cv_done.notify_all();
            continue;
          }
        }
        s->active.push_back(q);
      }
      act = s->active;
      if (s->stop && act.empty() && s->queue.empty() && s->step_events.empty()) break;
      bool work = false;
      for (Req* q : act)
        if (q->state == 1) work = true;
      if (!work && s->step_events.empty()) {
        if (s->stop) break;
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    // chunk status words of new requests start at zero
    bool any = false;
    for (Req* q : act)
      if (q->state == 1) any = true;
    if (any) {
      for (Req* q : act)
        if (q->state == 1 && !q->prepared)
          cudaMemsetAsync(s->status + (q->chunk + 1) * 32, 0, sizeof(unsigned), s->stream);
      const uint64_t step = ++s->step_no;
      // scale slots of newly prepared requests start at zero
      for (Req* q : act)
        if (q->state == 1 && !q->prepared)
          cudaMemsetAsync(s->scales + q->chunk * kSlotsPerReq, 0, sizeof(Scale) * kSlotsPerReq,
                          s->stream);
      matpow_status st = run_step(s, act, step);
      if (st != MATPOW_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->fatal = st;
        for (Req* q : s->active) {
          q->state = 3;
          q->result = st;
        }
        s->active.clear();
        s->cv_done.notify_all();
        break;
      }
    }
    // retire finished steps (bounded: the loop keeps going either way)
    while (!s->step_events.empty()) {
      cudaError_t q = cudaEventQuery(s->step_events.front().second);
      if (q == cudaErrorNotReady) {
        if (!any) cudaEventSynchronize(s->step_events.front().second);
        else break;
        q = cudaSuccess;
      }
      completed_step = s->step_events.front().first;
      s->event_pool.push_back(s->step_events.front().second);
      s->step_events.pop_front();
      cudaMemcpy(s->h_status.data(), s->status, sizeof(unsigned) * s->h_status.size(),
                 cudaMemcpyDeviceToHost);
      const unsigned step_status = s->h_status[0];
      std::lock_guard<std::mutex> lk(s->mu);
      auto now = Clock::now();
      for (size_t i = 0; i < s->active.size();) {
        Req* r = s->active[i];
        if (r->state == 2 && r->done_step <= completed_step) {
          const unsigned bits = s->h_status[(r->chunk + 1) * 32] | step_status;
          r->result = (bits & ST_BADINPUT) ? MATPOW_EINVAL
                      : (bits & ST_RANGE) && r->r.kind == 0 && !r->r.dLog2Scale ? MATPOW_ERANGE
                                                                                 : MATPOW_OK;
          r->t_done = now;
          s->latencies_us.push_back(
              std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
          s->arena.release(r->off, r->bytes);
          s->free_chunks.push_back(r->chunk);
          s->active.erase(s->active.begin() + i);
          r->state = 3;
        } else {
          ++i;
        }
      }
      if (step_status) cudaMemsetAsync(s->status, 0, sizeof(unsigned), s->stream);
      s->cv_done.notify_all();
    }
  }
}

extern "C" matpow_status matpow_server_create(matpow_server_t* out, const matpow_server_desc* d) {
  if (!out || !d) return fail(nullptr, MATPOW_EINVAL, "matpow_server_create: NULL argument");
  *out = nullptr;
  if (d->max_n < 1 || d->max_inflight < 1 || d->max_queue < 1 || d->hbm_budget_bytes == 0)
    return fail(nullptr, MATPOW_EINVAL, "matpow_server_create: bad descriptor");
  if (d->precision != MATPOW_FP32_SIMT && d->precision != MATPOW_BF16 && d->precision != MATPOW_BF16X3 &&
      d->precision != MATPOW_BF16X6)
    return fail(nullptr, MATPOW_EINVAL, "matpow_server_create: unknown precision");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev)
    return fail(nullptr, MATPOW_EINVAL, "matpow_server_create: no such device");
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, d->device);
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, MATPOW_EUNSUPPORTED, "matpow_server_create: device is not sm_103");
  auto* s = new (std::nothrow) matpow_server_s();
  if (!s) return fail(nullptr, MATPOW_ENOMEM, "matpow_server_create: host allocation");
  s->desc = *d;
  s->num_sms = prop.multiProcessorCount;
  // grouped float levels: the exact-split tensor-core kernels for MATPOW_BF16X3
  // and MATPOW_BF16X6, the float32 SIMT kernels otherwise
  s->fmt = d->precision == MATPOW_BF16X3 ? FMT_FX2 : d->precision == MATPOW_BF16X6 ? FMT_FX3 : FMT_F32;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&s->arena_mem, d->hbm_budget_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->scales, sizeof(Scale) * kSlotsPerReq * d->max_inflight);
  s->h_status.assign((size_t)32 * (d->max_inflight + 1), 0u);
  if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(unsigned) * s->h_status.size());
  if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(unsigned) * s->h_status.size());
  if (e == cudaSuccess) e = tiny_attrs();
  if (e == cudaSuccess) {  // tensor maps: exact-split float levels and tensor-core mod p
    e = tc_init(nullptr);
    if (e == cudaSuccess) e = tc_modp_init();
    if (e == cudaSuccess) e = cudaMalloc(&s->d_maps, sizeof(CUtensorMap) * 24 * d->max_inflight);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_maps, sizeof(CUtensorMap) * 24 * d->max_inflight);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    matpow_server_destroy(s);
    cudaGetLastError();
    return fail(nullptr, MATPOW_ENOMEM, "matpow_server_create: device allocation failed");
  }
  s->arena.reset(d->hbm_budget_bytes);
  for (int i = d->max_inflight - 1; i >= 0; --i) s->free_chunks.push_back(i);
  s->th = std::thread(scheduler, s);
  *out = s;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_submit(matpow_server_t s, const matpow_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return fail(nullptr, MATPOW_EINVAL, "matpow_submit: NULL argument");
  if (r->N < 1 || r->N > s->desc.max_n) return sfail(s, MATPOW_EINVAL, "matpow_submit: N out of range");
  if (!r->dA || !r->dOut) return sfail(s, MATPOW_EINVAL, "matpow_submit: NULL matrix pointer");
  if (r->kind != 0 && r->kind != 1) return sfail(s, MATPOW_EINVAL, "matpow_submit: bad kind");
  if (r->kind == 1 && (r->p < 2 || r->p > 65536)) return sfail(s, MATPOW_EINVAL, "matpow_submit: bad p");
  if (footprint(s, *r) > s->desc.hbm_budget_bytes)
    return sfail(s, MATPOW_ENOMEM, "matpow_submit: request larger than the server's HBM budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != MATPOW_OK) return s->fatal;
  if ((int)s->queue.size() >= s->desc.max_queue) return MATPOW_EBUSY;
  Req* q = new Req();
  q->ticket = s->next_ticket++;
  q->r = *r;
  q->t_submit = Clock::now();
  s->queue.push_back(q);
  s->all[q->ticket] = q;
  *ticket = q->ticket;
  s->cv_sched.notify_one();
  return MATPOW_OK;
}

extern "C" matpow_status matpow_poll(matpow_server_t s, uint64_t ticket, uint32_t timeout_us) {
  if (!s) return fail(nullptr, MATPOW_EINVAL, "matpow_poll: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(s, MATPOW_EINVAL, "matpow_poll: unknown ticket");
  Req* q = it->second;
  if (q->state != 3 && timeout_us)
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return q->state == 3; });
  if (q->state != 3) return timeout_us ? MATPOW_ETIMEDOUT : MATPOW_EAGAIN;
  matpow_status st = q->result;
  s->all.erase(it);
  delete q;
  return st;
}

extern "C" int64_t matpow_server_latencies(matpow_server_t s, double* us, int64_t cap) {
  if (!s || !us || cap <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t n = std::min<int64_t>(cap, (int64_t)s->latencies_us.size());
  std::copy(s->latencies_us.begin(), s->latencies_us.begin() + n, us);
  return n;
}

extern "C" matpow_status matpow_server_destroy(matpow_server_t s) {
  if (!s) return MATPOW_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_sched.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->desc.device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& kv : s->all) delete kv.second;
  for (Req* q : s->queue)
    if (!s->all.count(q->ticket)) delete q;
  for (auto& e : s->step_events) cudaEventDestroy(e.second);
  for (auto e : s->event_pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (s->tab_ev[i]) cudaEventDestroy(s->tab_ev[i]);
    if (s->h_tab[i]) cudaFreeHost(s->h_tab[i]);
  }
  if (s->d_tab) cudaFree(s->d_tab);
  if (s->d_maps) cudaFree(s->d_maps);
  if (s->h_maps) cudaFreeHost(s->h_maps);
  if (s->scales) cudaFree(s->scales);
  if (s->status) cudaFree(s->status);
  if (s->arena_mem) cudaFree(s->arena_mem);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaSetDevice(prev);
  delete s;
  return MATPOW_OK;
}
