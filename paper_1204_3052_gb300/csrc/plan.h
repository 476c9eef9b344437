// Host-side plan state of libmatpow (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace mp {

constexpr int kSingleSlots = 256;  // scale slots of one power: 2 + G(n) <= 2 + 126
constexpr size_t kMaxGraphs = 16;

// One product of the schedule: C(cb, sc) = X(xb, sx) * Y(yb, sy).
struct Op {
  int xb, yb, cb;
  int sx, sy, sc;
  bool square;
};
struct LevelOps {
  std::vector<Op> ops;  // one or two products that read the same P
};
void build_schedule(uint64_t n, std::vector<LevelOps>* levels);

struct GraphKey {
  int kind;  // 0 float, 1 mod p, 2 the e^A sequence after the norm (n = s)
  const void* A;
  void* out;
  void* log2;
  int N;
  uint64_t n;
  uint32_t p;
  bool operator==(const GraphKey& o) const {
    return kind == o.kind && A == o.A && out == o.out && log2 == o.log2 && N == o.N && n == o.n &&
           p == o.p;
  }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  uint64_t stamp = 0;
};

struct KernelTiming {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<double> pending_flop;
  int64_t launches = 0;
  double total_ms = 0.0;
  double flop = 0.0;
};

// Device arrays of matpow_batched, grown on demand and kept by the plan.
struct BatchState {
  void* ws = nullptr;           // per-matrix partial products
  size_t ws_bytes = 0;
  Scale* scales = nullptr;      // per-matrix scale slots
  size_t scale_cap = 0;
  void* descs = nullptr;        // GemmDesc / TinyDesc tables (device)
  size_t desc_bytes = 0;
  void* h_descs = nullptr;      // pinned staging for the tables
  size_t h_desc_bytes = 0;
  void* maps = nullptr;         // TMA descriptors of the batch buffers (device)
  size_t maps_bytes = 0;
  std::vector<CUtensorMap> h_maps;  // host copy; rebuilt when the layout changes
  std::vector<std::pair<const void*, int>> map_keys;  // (buffer, N) per 4 descriptors
  cudaEvent_t staged = nullptr; // the last upload from h_descs has been consumed
  // the last call captured as a CUDA graph: replayed while the call's
  // signature (pointers, orders, powers, options) is unchanged
  std::vector<uint64_t> sig;
  cudaGraphExec_t exec = nullptr;
  int64_t exec_kernels = 0;
};

}  // namespace mp

struct matpow_plan_s {
  int device = 0;
  int max_n = 0;
  matpow_precision prec = MATPOW_FP32_SIMT;
  int num_sms = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* buf[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t buf_bytes = 0;
  mp::Scale* scales = nullptr;
  unsigned* status = nullptr;
  unsigned* h_status = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::string err;
  // options
  bool use_graphs = true;
  bool timing_on = false;
  int tiny_max = 64;
  int tile_override = 0;
  int split_mode = 0;  // BF16X3: 0 exact fixed-point slices, 1 floating hi/lo planes
  int chain_mode = 1;  // whole-chain kernel: 0 off, 1 with split-K where it fits, 2 without
  bool modp_tc = true;    // mod-p products on the tensor cores (64 < N <= 16384)
  bool persist = true;    // batched 64-column levels: persistent grouped kernel
  bool naive = false;     // float powers by n - 1 products R <- R A (comparison method)
  bool pair = false;      // exact-split 128-column levels with N > 2048 on CTA pairs (opt-in)
  unsigned* gbar = nullptr;  // grid-barrier counter of the whole-chain kernel
  float* expm_ws = nullptr;  // matpow_expm scratch: 7 max_n^2 float32 + column sums, on first use
  cudaEvent_t expm_ev = nullptr;  // matpow_expm: the norm's read-back has landed
  // graphs
  std::vector<mp::GraphEntry> graphs;
  uint64_t graph_clock = 0;
  // timing
  mp::KernelTiming timing[MATPOW_KERNEL_KINDS];
  std::vector<cudaEvent_t> event_pool;
  int64_t launches = 0;
  // batching
  mp::BatchState batch;
  // tensor-core path state (tensor maps etc.), owned by k_tc.cu
  void* tc = nullptr;
  // tile table: launch shapes per order range (matpow_plan_set_tile_table)
  std::vector<matpow_tile_rule> tiles;
};

namespace mp {
matpow_status fail(matpow_plan_s* plan, matpow_status st, const char* fmt, ...);
// The tile-table rule that covers order N for the plan's precision (the
// last one in table order), or null; plan_tile_field gives one field of it
// (-1 when no rule covers N or the rule leaves the field to the built-in).
const matpow_tile_rule* plan_tile_rule(const matpow_plan_s* p, int N);
int plan_tile_field(const matpow_plan_s* p, int N, int matpow_tile_rule::*field);
// Destroy the plan's cached single-call CUDA graphs.
void drop_plan_graphs(matpow_plan_s* p);
matpow_status cuda_fail(matpow_plan_s* plan, cudaError_t e, const char* what);
size_t matrix_bytes(int N, int fmt);
long long plane_offset_elems(int N, int fmt);
int float_fmt(matpow_precision p);
int plan_float_fmt(const matpow_plan_s* p);  // float_fmt, with the split option applied
cudaEvent_t take_event(matpow_plan_s* p);
void timed_begin(matpow_plan_s* p, cudaStream_t s, cudaEvent_t* ev);
void timed_end(matpow_plan_s* p, cudaStream_t s, cudaEvent_t ev, int kind, double flop);
void batch_free(matpow_plan_s* p);
// tensor-core path (k_tc.cu)
cudaError_t tc_init(matpow_plan_s* p);  // kernel attributes, driver entry points
void tc_free(matpow_plan_s* p);
// Fill the tensor-core fields of d (tiles_n, tile count in *ntiles).
matpow_status tc_fill_desc(matpow_plan_s* p, GemmDesc* d, int* ntiles);
matpow_status tc_launch_pair(matpow_plan_s* p, const GemmPair& g, cudaStream_t s);
// 2-D bfloat16 tensor map over an N x N matrix (row stride ld), 128-byte swizzle.
bool tc_encode_bf16_map(CUtensorMap* m, const void* base, int N, int ld, int box_inner,
                        int box_outer);
// Whole square-and-multiply chain in one cooperative tensor-core launch
// (exact split; small and medium N).  *used = false when it does not apply.
matpow_status tc_chain_run(matpow_plan_s* p, const float* dA, int N, uint64_t n, float* dOut,
                           int64_t* dLog2, cudaStream_t s, bool* used);
// Run `enqueue` on s, or replay the CUDA graph captured from it the first
// time `key` was seen (the plan's graph cache; direct while timing or inside
// a caller's capture).
matpow_status run_graph_or_direct(matpow_plan_s* p, const GraphKey& key, cudaStream_t s,
                                  const std::function<matpow_status(cudaStream_t)>& enqueue);
// C = X Y of two float32 N x N matrices (N > tiny_max), value-mode float32
// output, through the plan's product path (uses buffers 0, 1, scale slots 0-3).
// keep_x: X is the previous call's X, still split in buffer 0 / slot 1.
matpow_status enqueue_product_f32(matpow_plan_s* p, const float* X, const float* Y, int N, float* out,
                                  cudaStream_t s, bool keep_x = false);
// One power of a multi-power whole-chain launch: input, order, power, output,
// its four stored-format buffers and its scale slots (2 + G(n)).
struct ChainJob {
  const float* A;
  int N;
  uint64_t n;
  float* out;
  int64_t* log2;
  void* buf[4];
  Scale* scales;
};
// Up to four independent powers (same tile width) in one cooperative launch.
matpow_status tc_chain_launch(matpow_plan_s* p, const ChainJob* jobs, int nj, cudaStream_t s, bool* used);
cudaError_t tc_chain_init(matpow_plan_s* p);
// tensor-core mod-p products (k_tcmodp.cu)
cudaError_t tc_modp_init();
int tc_modp_tile_n();
cudaError_t launch_prep_modp_slices(const unsigned* A, int N, unsigned p, void* dst,
                                    unsigned* status, cudaStream_t s);
matpow_status tc_modp_launch_pair(matpow_plan_s* p, const GemmPair& g, cudaStream_t s);
// Grouped tensor-core mod-p level launch (server): one CTA per 128 x 64 tile of
// every product in the device table; descriptors per buffer as for the exact
// split with two slices (x1, x0 as A at map_x, y1, y0 as B at map_y + 2).
cudaError_t launch_modp_tc_group(const GemmDesc* d_descs, int count, int tiles, const void* d_maps,
                                 int num_sms, unsigned* status, cudaStream_t s);
// Grouped exact-split level launch of the plan's batch (max_n: largest order
// among the products).
matpow_status tc_launch_group_bn(matpow_plan_s* p, const GemmDesc* d_descs, int count, int tiles,
                                 const int4* d_tile_rec, const void* d_maps, int bn, int max_n,
                                 bool persist, Scale* scales, unsigned* status, cudaStream_t s);
int tc_group_bn(int N, int nsl = 2);  // built-in tile width of grouped launches for order N
// Plan-free grouped exact-split launch (descriptor and TMA tables on the
// device): the persistent kernel (one CTA per SM over the whole tile list;
// d_tile_desc[t] = index of the product owning tile t | its k-blocks << 24)
// for 64-column tiles
// and orders up to 4096 when `persist` is set and the table is given, else
// one CTA per tile.
cudaError_t launch_fxb_group(const GemmDesc* d_descs, int count, int tiles, const int4* d_tile_rec,
                             const void* d_maps, int bn, int nsl, int max_n, int num_sms, bool persist,
                             Scale* scales, unsigned* status, cudaStream_t s);
cudaError_t tc_persist_init();
// CTA-pair exact-split products (k_tc2.cu): 256 x 128 tiles over two SMs.
struct TcPairParams;
cudaError_t tc_pair_init();
int pair_tiles(int N);
cudaError_t launch_fxb_pair(const TcPairParams& P, int pair_tiles_total, Scale* scales, unsigned* status,
                            cudaStream_t s);
// Per-tile records of a 64-column grouped level, in tile order: {product
// index | k-blocks << 24, m0 | n0 << 16, A-role map index, B-role map index}.
void persist_tile_records(const GemmDesc* descs, int count, int nsl, std::vector<int4>* out);
cudaError_t launch_fxb_persist(const GemmDesc* d_descs, int tiles, const int4* d_tile_rec,
                               const void* d_maps, int nsl, int num_sms, Scale* scales, unsigned* status,
                               cudaStream_t s);
// The 2 nsl TMA descriptors of one block-scaled buffer (A-role slices, then B-role).
bool tc_encode_buffer_maps(CUtensorMap* m, const void* base, int N, int nsl);
}  // namespace mp
