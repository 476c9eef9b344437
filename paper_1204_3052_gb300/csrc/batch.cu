// matpow_batched: many independent powers A_i^(n_i) of uneven orders.
//
// Small matrices (N <= the plan's whole-chain limit) run their entire chain
// in one CTA each, all in a single launch.  Larger ones are prepared by two
// grouped kernels (absmax, conversion) and then advanced level by level: the
// products of one squaring level of every matrix (arXiv 1204.3052 Sec. 4.3)
// form one grouped launch over a device table of product descriptors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "plan.h"

using namespace mp;

#define CK(plan, call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(plan, e_, #call); \
  } while (0)

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void mp::batch_free(matpow_plan_s* p) {
  BatchState& b = p->batch;
  if (b.ws) cudaFree(b.ws);
  if (b.scales) cudaFree(b.scales);
  if (b.descs) cudaFree(b.descs);
  if (b.h_descs) cudaFreeHost(b.h_descs);
  if (b.staged) cudaEventDestroy(b.staged);
  if (b.exec) cudaGraphExecDestroy(b.exec);
  b = BatchState();
}

static matpow_status grow(matpow_plan_s* p, void** ptr, size_t* cap, size_t need, bool host) {
  if (*cap >= need) return MATPOW_OK;
  size_t n = std::max(need, *cap * 3 / 2);
  void* q = nullptr;
  cudaError_t e;
  if (host) {
    if (p->batch.staged) cudaEventSynchronize(p->batch.staged);
    e = cudaMallocHost(&q, n);
  } else {
    cudaDeviceSynchronize();  // the old array may still be in use by queued work
    if (p->batch.exec) {      // the captured graph refers to the old array
      cudaGraphExecDestroy(p->batch.exec);
      p->batch.exec = nullptr;
      p->batch.sig.clear();
    }
    e = cudaMalloc(&q, n);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, MATPOW_ENOMEM, "matpow_batched: allocation of %zu bytes failed", n);
  }
  if (*ptr) {
    if (host) cudaFreeHost(*ptr); else cudaFree(*ptr);
  }
  *ptr = q;
  *cap = n;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_batched(matpow_plan_t p, int count, const float* const* dA,
                                        const int* N, const uint64_t* n, float* const* dOut,
                                        int64_t* dLog2Scale, void* stream) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_batched: plan is NULL");
  if (count < 0) return fail(p, MATPOW_EINVAL, "matpow_batched: count < 0");
  if (count == 0) return MATPOW_OK;
  if (!dA || !N || !n || !dOut) return fail(p, MATPOW_EINVAL, "matpow_batched: NULL array");
  for (int i = 0; i < count; ++i) {
    if (N[i] < 0 || N[i] > p->max_n)
      return fail(p, MATPOW_EINVAL, "matpow_batched: N[%d]=%d outside [0, %d]", i, N[i], p->max_n);
    if (N[i] > 0 && (!dA[i] || !dOut[i]))
      return fail(p, MATPOW_EINVAL, "matpow_batched: NULL matrix pointer at %d", i);
    if (((uintptr_t)dA[i] & 3) || ((uintptr_t)dOut[i] & 3))
      return fail(p, MATPOW_EINVAL, "matpow_batched: misaligned pointer at %d", i);
  }
  if ((uintptr_t)dLog2Scale & 7) return fail(p, MATPOW_EINVAL, "matpow_batched: misaligned dLog2Scale");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  cudaStream_t s = (cudaStream_t)stream;
  const int fmt = plan_float_fmt(p);
  const bool tc = p->prec != MATPOW_FP32_SIMT;

  // ---- up to four powers that all fit the whole-chain kernel: one
  // cooperative launch runs them side by side (level L of every power between
  // the same grid barriers)
  if (count <= 4 && fmt_exact(fmt) && p->chain_mode != 0 && !p->naive) {
    bool all = true;
    for (int i = 0; i < count && all; ++i)
      all = N[i] > p->tiny_max && N[i] <= 1024 && n[i] >= 2;
    if (all) {
      size_t need = 0, mb[4];
      int slots = 0, slot0[4];
      for (int i = 0; i < count; ++i) {
        mb[i] = matrix_bytes(N[i], fmt);
        need += 4 * mb[i];
        slot0[i] = slots;
        slots += 2 + matpow_gemm_count(n[i]);
      }
      matpow_status st;
      if ((st = grow(p, &p->batch.ws, &p->batch.ws_bytes, need, false))) return st;
      if ((st = grow(p, (void**)&p->batch.scales, &p->batch.scale_cap, sizeof(Scale) * slots, false)))
        return st;
      ChainJob jobs[4];
      size_t off = 0;
      for (int i = 0; i < count; ++i) {
        char* base = (char*)p->batch.ws + off;
        jobs[i] = ChainJob{dA[i], N[i], n[i], dOut[i], dLog2Scale ? dLog2Scale + i : nullptr,
                           {base, base + mb[i], base + 2 * mb[i], base + 3 * mb[i]},
                           p->batch.scales + slot0[i]};
        off += 4 * mb[i];
      }
      bool used = false;
      if ((st = tc_chain_launch(p, jobs, count, s, &used))) return st;
      if (used) return MATPOW_OK;
    }
  }

  // ---- replay: the same call as the last captured one needs no host work
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(p, cudaStreamIsCapturing(s, &cs));
  const bool graphable = p->use_graphs && !p->timing_on && cs == cudaStreamCaptureStatusNone;
  std::vector<uint64_t> sig;
  if (graphable) {
    sig.reserve(4 * (size_t)count + 6);
    sig.push_back((uint64_t)count);
    sig.push_back((uint64_t)(uintptr_t)dLog2Scale);
    sig.push_back((uint64_t)fmt);
    sig.push_back((uint64_t)p->tiny_max);
    sig.push_back((uint64_t)p->persist);
    sig.push_back((uint64_t)p->modp_tc);
    for (int i = 0; i < count; ++i) {
      sig.push_back((uint64_t)(uintptr_t)dA[i]);
      sig.push_back((uint64_t)(uintptr_t)dOut[i]);
      sig.push_back((uint64_t)N[i]);
      sig.push_back(n[i]);
    }
    if (p->batch.exec && sig == p->batch.sig) {
      CK(p, cudaGraphLaunch(p->batch.exec, s));
      p->launches += p->batch.exec_kernels;
      return MATPOW_OK;
    }
    if (p->batch.exec) {
      cudaGraphExecDestroy(p->batch.exec);
      p->batch.exec = nullptr;
      p->batch.sig.clear();
    }
  }

  // ---- classify
  std::vector<TinyDesc> tiny;
  std::vector<PrepDesc> prep;
  struct Big {
    int i;
    int slot0;
    size_t off;  // byte offset of this matrix's four buffers in the batch workspace
    size_t mb;   // bytes of one buffer
    std::vector<LevelOps> levels;
  };
  std::vector<Big> big;
  size_t ws_need = 0;
  int slots = 0;
  for (int i = 0; i < count; ++i) {
    if (N[i] == 0) continue;
    long long* lg = dLog2Scale ? (long long*)(dLog2Scale + i) : nullptr;
    if (N[i] <= p->tiny_max) {
      tiny.push_back({dA[i], dOut[i], lg, (unsigned long long)n[i], N[i], 0});
      continue;
    }
    if (n[i] <= 1) {
      PrepDesc d{};
      d.A = dA[i];
      d.dst = dOut[i];
      d.log2 = lg;
      d.N = N[i];
      d.kind = n[i] == 0 ? 1 : 2;
      prep.push_back(d);
      continue;
    }
    Big b;
    b.i = i;
    b.slot0 = slots;
    b.mb = matrix_bytes(N[i], fmt);
    b.off = ws_need;
    ws_need += 4 * b.mb;
    slots += 2 + matpow_gemm_count(n[i]);
    build_schedule(n[i], &b.levels);
    PrepDesc d{};
    d.A = dA[i];
    d.N = N[i];
    d.fmt = fmt;
    d.plane = plane_offset_elems(N[i], fmt);
    d.slot_raw = b.slot0;
    d.slot_stored = b.slot0 + 1;
    d.kind = 0;
    prep.push_back(d);
    big.push_back(std::move(b));
  }
  matpow_status st;
  const bool fx2 = fmt_exact(fmt);
  const int nsl = fmt_slices(fmt);
  const int mpb = 2 * nsl;  // TMA descriptors per buffer
  if (tc && !fx2 && !big.empty())
    return fail(p, MATPOW_EUNSUPPORTED,
                "matpow_batched: grouped tensor-core launches use the exact split (MATPOW_BF16X3 or MATPOW_BF16X6)");
  if ((st = grow(p, &p->batch.ws, &p->batch.ws_bytes, std::max<size_t>(ws_need, 1), false))) return st;
  size_t sc_bytes = sizeof(Scale) * std::max(slots, 1);
  if ((st = grow(p, (void**)&p->batch.scales, &p->batch.scale_cap, sc_bytes, false))) return st;
  // prep descriptors point into the workspace
  {
    size_t bi = 0;
    for (auto& d : prep)
      if (d.kind == 0) {
        d.dst = (char*)p->batch.ws + big[bi].off;
        ++bi;
      }
  }
  // ---- product descriptors per level; tensor-core levels get one launch per
  // kernel variant: 64-column tiles in the persistent kernel, 64-column tiles
  // one CTA each, 128-column tiles (built in: 64 columns for N <= 1024 or
  // three slices, 128 above; persistent where the plan allows it; the tile
  // table may choose per order range)
  struct Launch {
    int begin, count, tiles, bn, max_n, td;  // td: offset of the tile -> product table
    bool persist;
  };
  auto variant_of = [&](int Ni) -> int {
    int bn = tc_group_bn(Ni, nsl);
    const int tb = plan_tile_field(p, Ni, &matpow_tile_rule::bn);
    if (tb == 64 || (tb == 128 && nsl == 2)) bn = tb;
    if (bn == 128) return 2;
    bool per = p->persist;
    const int tp = plan_tile_field(p, Ni, &matpow_tile_rule::persist);
    if (p->persist && tp >= 0) per = tp == 1;
    return per ? 0 : 1;
  };
  int max_levels = 0;
  for (auto& b : big) max_levels = std::max(max_levels, (int)b.levels.size());
  std::vector<GemmDesc> gd;
  std::vector<std::vector<Launch>> lvl_launches(max_levels);
  std::vector<int4> trec;  // persistent-kernel tile records of every launch
  for (int L = 0; L < max_levels; ++L) {
    for (int pi = 0; pi < (tc ? 3 : 1); ++pi) {
      // SIMT: one tile edge for the whole launch (64 when its 128-tiles would
      // not fill the SMs); carried in the launch's bn
      int sedge = 128;
      if (!tc) {
        int t128 = 0;
        for (const Big& b : big)
          if (L < (int)b.levels.size()) {
            const int tt = (N[b.i] + 127) / 128;
            t128 += (int)b.levels[L].ops.size() * tt * tt;
          }
        sedge = simt_tile_edge(t128, p->num_sms);
      }
      const int bn = tc ? (pi == 2 ? 128 : 64) : sedge;
      int begin = (int)gd.size(), tiles = 0, max_n = 0;
      for (size_t bi = 0; bi < big.size(); ++bi) {
        const Big& b = big[bi];
        if (L >= (int)b.levels.size()) continue;
        const int Ni = N[b.i];
        if (tc && variant_of(Ni) != pi) continue;
        max_n = std::max(max_n, Ni);
        const bool final_level = L + 1 == (int)b.levels.size();
        const LevelOps& lv = b.levels[L];
        for (size_t k = 0; k < lv.ops.size(); ++k) {
          const Op& op = lv.ops[k];
          const bool last = final_level && k + 1 == lv.ops.size();
          char* base = (char*)p->batch.ws + b.off;
          GemmDesc d{};
          d.X = base + op.xb * b.mb;
          d.Y = base + op.yb * b.mb;
          d.C = last ? nullptr : base + op.cb * b.mb;
          d.out = last ? (void*)dOut[b.i] : nullptr;
          d.out_log2 = last && dLog2Scale ? (long long*)(dLog2Scale + b.i) : nullptr;
          d.plane = plane_offset_elems(Ni, fmt);
          d.N = Ni;
          d.ld = ld_for(Ni, fmt);
          d.sx = b.slot0 + op.sx;
          d.sy = b.slot0 + op.sy;
          d.sc = b.slot0 + op.sc;
          d.mode = last ? (dLog2Scale ? OUT_USER_MANT : OUT_USER_VALUE) : OUT_INTERNAL;
          d.tile_begin = tiles;
          if (tc) {
            d.bn = bn;
            d.tiles_n = (Ni + bn - 1) / bn;
            d.map_x = mpb * (4 * (int)bi + op.xb);
            d.map_y = mpb * (4 * (int)bi + op.yb);
            d.map_c = mpb * (4 * (int)bi + (last ? op.xb : op.cb));
            tiles += ((Ni + 127) / 128) * d.tiles_n;
          } else {
            d.tiles_n = (Ni + bn - 1) / bn;
            tiles += d.tiles_n * d.tiles_n;
          }
          gd.push_back(d);
        }
      }
      if ((int)gd.size() > begin) {
        const int td = (int)trec.size();
        if (tc && bn == 64) persist_tile_records(gd.data() + begin, (int)gd.size() - begin, nsl, &trec);
        lvl_launches[L].push_back({begin, (int)gd.size() - begin, tiles, bn, max_n, td, pi == 0});
      }
    }
  }
  // ---- TMA descriptors of every batch buffer (tensor-core levels), rebuilt
  // only when the layout (buffer addresses, orders) changed since the last call
  if (tc && !big.empty()) {
    std::vector<std::pair<const void*, int>> keys;
    keys.reserve(4 * big.size());
    for (auto& b : big)
      for (int k = 0; k < 4; ++k) keys.push_back({(char*)p->batch.ws + b.off + k * b.mb, N[b.i]});
    if (keys != p->batch.map_keys || p->batch.h_maps.size() != mpb * keys.size()) {
      p->batch.h_maps.resize(mpb * keys.size());
      for (size_t k = 0; k < keys.size(); ++k)
        if (!tc_encode_buffer_maps(&p->batch.h_maps[mpb * k], keys[k].first, keys[k].second, nsl))
          return fail(p, MATPOW_ECUDA, "matpow_batched: cuTensorMapEncodeTiled failed");
      const size_t mbytes = p->batch.h_maps.size() * sizeof(CUtensorMap);
      if ((st = grow(p, &p->batch.maps, &p->batch.maps_bytes, mbytes, false))) return st;
      CK(p, cudaMemcpy(p->batch.maps, p->batch.h_maps.data(), mbytes, cudaMemcpyHostToDevice));
      p->batch.map_keys = keys;
    }
  }
  // prep CTAs: one per 64 x 64 block (exact split), else about one per 16K entries
  int prep_blocks = 0;
  for (auto& d : prep) {
    size_t e = (size_t)d.N * d.N;
    if (fx2 && d.kind == 0) {
      const size_t nb = ((size_t)d.N + 63) / 64;
      d.blocks = (int)(nb * nb);
    } else {
      d.blocks = (int)std::min<size_t>(std::max<size_t>((e + 16383) / 16384, 1), 1024);
    }
    d.block_begin = prep_blocks;
    prep_blocks += d.blocks;
  }
  // ---- stage the three tables in one pinned buffer, upload once
  size_t o_tiny = 0;
  size_t o_prep = align_up(o_tiny + tiny.size() * sizeof(TinyDesc), 256);
  size_t o_gd = align_up(o_prep + prep.size() * sizeof(PrepDesc), 256);
  size_t o_td = align_up(o_gd + gd.size() * sizeof(GemmDesc), 256);
  size_t total = std::max<size_t>(align_up(o_td + trec.size() * sizeof(int4), 256), 256);
  if ((st = grow(p, &p->batch.h_descs, &p->batch.h_desc_bytes, total, true))) return st;
  if ((st = grow(p, &p->batch.descs, &p->batch.desc_bytes, total, false))) return st;
  if (!p->batch.staged) CK(p, cudaEventCreateWithFlags(&p->batch.staged, cudaEventDisableTiming));
  CK(p, cudaEventSynchronize(p->batch.staged));  // previous upload finished reading h_descs
  char* h = (char*)p->batch.h_descs;
  if (!tiny.empty()) memcpy(h + o_tiny, tiny.data(), tiny.size() * sizeof(TinyDesc));
  if (!prep.empty()) memcpy(h + o_prep, prep.data(), prep.size() * sizeof(PrepDesc));
  if (!gd.empty()) memcpy(h + o_gd, gd.data(), gd.size() * sizeof(GemmDesc));
  if (!trec.empty()) memcpy(h + o_td, trec.data(), trec.size() * sizeof(int4));
  CK(p, cudaMemcpyAsync(p->batch.descs, h, total, cudaMemcpyHostToDevice, s));
  CK(p, cudaEventRecord(p->batch.staged, s));
  char* dd = (char*)p->batch.descs;
  // ---- enqueue: directly, or captured once into a graph that later calls
  // with the same signature replay (the tables uploaded above stay valid
  // until a call with another signature rebuilds them)
  auto enqueue = [&](cudaStream_t s) -> matpow_status {
  cudaEvent_t ev;
  if (!tiny.empty()) {
    double flop = 0;
    for (auto& t : tiny) flop += 2.0 * t.N * (double)t.N * t.N * matpow_gemm_count(t.n);
    timed_begin(p, s, &ev);
    CK(p, launch_tiny_group((const TinyDesc*)(dd + o_tiny), (int)tiny.size(), p->status, s));
    timed_end(p, s, ev, MATPOW_KERNEL_TINY, flop);
    p->launches++;
  }
  if (!prep.empty()) {
    if (slots) CK(p, cudaMemsetAsync(p->batch.scales, 0, sizeof(Scale) * slots, s));
    const PrepDesc* pd = (const PrepDesc*)(dd + o_prep);
    if (fx2) {
      CK(p, launch_prep_fxb_group(pd, (int)prep.size(), prep_blocks, p->batch.scales, p->status, s));
      p->launches += 1;
    } else {
      CK(p, launch_prep_absmax_group(pd, (int)prep.size(), prep_blocks, p->batch.scales, p->status, s));
      CK(p, launch_prep_convert_group(pd, (int)prep.size(), prep_blocks, p->batch.scales, s));
      p->launches += 2;
    }
  }
  for (int L = 0; L < max_levels; ++L) {
    for (const Launch& la : lvl_launches[L]) {
      const GemmDesc* g = (const GemmDesc*)(dd + o_gd) + la.begin;
      double flop = 0;
      for (int k = 0; k < la.count; ++k) {
        const GemmDesc& d = gd[la.begin + k];
        flop += 2.0 * d.N * (double)d.N * d.N;
      }
      timed_begin(p, s, &ev);
      if (tc) {
        if ((st = tc_launch_group_bn(p, g, la.count, la.tiles, (const int4*)(dd + o_td) + la.td,
                                     p->batch.maps, la.bn, la.max_n, la.persist, p->batch.scales,
                                     p->status, s)))
          return st;
        timed_end(p, s, ev, MATPOW_KERNEL_TC, flop);
      } else {
        const int split = tc || p->chain_mode == 2 ? 1 : simt_split(la.bn, la.tiles, p->num_sms);
        CK(p, launch_simt_group(g, la.count, la.tiles, la.bn, split, p->batch.scales, p->status, s));
        timed_end(p, s, ev, MATPOW_KERNEL_SIMT, flop);
      }
      p->launches++;
    }
  }
  return MATPOW_OK;
  };
  if (!graphable) return enqueue(s);
  const int64_t before = p->launches;
  CK(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  matpow_status st2 = enqueue(p->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
  if (st2 != MATPOW_OK) {
    if (graph) cudaGraphDestroy(graph);
    p->launches = before;
    return st2;
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaGraphInstantiate");
  p->batch.exec = exec;
  p->batch.exec_kernels = p->launches - before;
  p->batch.sig.swap(sig);
  p->launches = before;
  CK(p, cudaGraphLaunch(exec, s));
  p->launches += p->batch.exec_kernels;
  return MATPOW_OK;
}
