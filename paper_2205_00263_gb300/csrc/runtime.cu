// Host runtime of libmnbab: the C ABI declared in include/mnbab.h.
//
// Owns device memory (within an HBM budget), the per-network node pools,
// property tables and multi-neuron constraints, and drives the kernels of
// kernels.cu: back-substitution sweeps (Sec. 3.1), re-bounding after a split
// (Sec. 3.2, enforcing splits), the DeepPoly pass and projected-Adam
// optimisation with the adjoint sweep (Sec. 3.1), ACS branching (Sec. 3.2) and
// the FIFO branch-and-bound queue (Sec. 2.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <limits>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "mnbab.h"
#include "mnbab_internal.h"

using namespace mnbab;

namespace {

struct Err {
  mnbab_status code;
  std::string msg;
};

[[noreturn]] void fail(mnbab_status c, const std::string& m) { throw Err{c, m}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MNBAB_E_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

struct QNode {
  int slot;
  int64_t seq;
  int row;
  int depth;
  int split_layer;
};

struct HostLayer {
  int kind;
  int ci, hi, wi, co, ho, wo, k, s, p;
  std::vector<double> W, b;
};

}  // namespace

struct mnbab_ctx;

struct mnbab_net {
  int id = 0;
  mnbab_ctx* ctx = nullptr;
  NetDev nd{};
  std::vector<HostLayer> hops;   // affine ops
  int eop[MNBAB_MAXR + 2][2] = {{0}};  // affine op of the edges into node t
  float* lam = nullptr;          // per-layer coefficient buffers: layer s at lam_off[s], ld d[s]
  size_t lam_off[MNBAB_MAXR + 2] = {0};
  int R = 0, d0 = 0, SD = 0, n_out = 0, maxd = 0, maxd_relu = 0;
  int nslot = 0;
  // node pool
  PoolDev pool{};
  int cap = 0;
  std::vector<int> free_slots;
  std::vector<int> slot_split;  // host metadata per slot
  std::vector<int> slot_row;
  std::vector<int> slot_prop;
  std::vector<char> slot_used;
  // scratch
  int B = 0;          // batch capacity (objective rows)
  int pad_slot = -1;  // scratch node for padded graph rows
  std::vector<int> new_roots, new_root_props;  // root-bound slots awaiting initialisation
  float* atk = nullptr;  // adversarial pre-attack scratch (grown on demand)
  size_t atk_cap = 0;
  int chunk = 0;      // rows per back-substitution launch
  float *part = nullptr, *lb = nullptr;
  int *row_node = nullptr, *row_j = nullptr, *counter = nullptr;
  float* row_sign = nullptr;
  size_t rows_cap = 0;
  int *rb_nodes = nullptr, *ri_dst = nullptr, *ri_src = nullptr, *ri_row = nullptr;
  float *AP = nullptr, *GA = nullptr, *GB = nullptr, *GP = nullptr, *GPh = nullptr;
  float *Gz = nullptr, *Hz = nullptr, *X = nullptr, *Xb = nullptr, *GG = nullptr, *gp0 = nullptr;
  float *fout = nullptr, *score = nullptr, *bestb = nullptr, *gmax = nullptr;
  double *f64a = nullptr, *f64out = nullptr;
  float* splitk = nullptr;
  size_t splitk_floats = 0;
  int* cslots = nullptr;
  int *cand_idx = nullptr, *cand_count = nullptr;  // counterexample candidates picked on the device
  // the last fused optimisation launch: its profiling class and per-row work
  int fused_cat = -1;
  double fused_row_flops = 0.0, fused_row_bytes = 0.0;
  int *bslots = nullptr, *brows = nullptr, *acs_layer = nullptr, *acs_neuron = nullptr,
      *acs_fb = nullptr, *kid_parent = nullptr, *kid_slots = nullptr, *kid_layer = nullptr,
      *kid_neuron = nullptr;
  // optimised intermediate bounds (allocated on first use): per-set gradients
  // [B][SD], per-row best bounds and owning nodes, chunk segments, set slots
  float *iga = nullptr, *igb = nullptr, *ibest = nullptr;
  float* igg = nullptr;  // per-set gradients of the multi-neuron multipliers [B][EC]
  int *iorig = nullptr, *iseg = nullptr, *isrc = nullptr, *idst = nullptr;
  size_t iseg_cap = 0;
  // per-row a' checkpoints and gradients [icap][SD] of longer row chunks than
  // the batch buffers hold (null when icap = B: the batch buffers serve)
  float *iap = nullptr, *igar = nullptr, *igbr = nullptr;
  int icap = 0;
  float* xsum = nullptr;  // leaf completion: summed minimisers [B][d0]
  // multi-neuron constraint generation: combination rows of one chunk
  int* gen_cidx = nullptr;
  float* gen_coef = nullptr;
  int gen_cap = 0;
};

struct mnbab_prop {
  int index = 0;
  mnbab_net* net = nullptr;
  PropDev pd{};
  int root_slot = -1;
  int n_rows = 0;
  std::vector<float> lo, hi;
  std::vector<double> Wf, bf;  // folded last layer in FP64 (host check)
  std::deque<QNode> queue;
  int budget = 256;
  int bounded = 0;
  int64_t next_seq = 0;
  int verdict = MNBAB_UNKNOWN;
  bool done = false;
  bool unknown_leaf = false;
  std::vector<int> row_open, row_leaf, row_fals;
  std::vector<float> row_lb;
  std::vector<float> cex;
  int cex_row = -1;
  std::vector<mnbab_trace_rec> trace;
  int mnc_set[MNBAB_MAXR + 1] = {0};
  bool root_pending = false;         // root bounds not computed yet
  std::vector<int> root_row_slots;   // its row root nodes, initialised with the bounds
  bool admitted = true;              // false while queued in the request loop
  bool materialized = false;         // node slots allocated
  int inter_steps = 0;               // Adam steps of optimised root intermediate bounds
  int leaf_steps = 256;              // Adam steps of the exact completion of fully split leaves
  int atk_starts = 0, atk_steps = 0;  // pre-attack when the property starts (0: none)
  uint64_t atk_seed = 0;
  double timeout_s = 0.0;            // wall-clock limit from its first BaB step (0: none)
  double t_start = 0.0;              // time of its first BaB step
  bool timed_out = false;
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A request of the serving loop.
struct Request {
  uint64_t ticket = 0;
  mnbab_prop* p = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0, deadline = 0;
  int state = 0;    // 0 queued, 1 active, 2 done
  int reserve = 0;  // node slots reserved in its network's pool
  uint64_t bytes = 0;  // HBM of those slots (node state, parameters, moments)
  int timed_out = 0;
};

struct mnbab_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  uint64_t budget = 0, used = 0;
  int node_cap = 65536, EC = 0, row_chunk = 32768, gemm_path = 0;
  int attack_path = 0;  // 0 auto, 1 one kernel per (row, start), 2 per-layer kernels
  int* d_err = nullptr;  // device error flag of bounded device waits
  std::string err;
  std::vector<mnbab_net*> nets;
  std::vector<mnbab_prop*> props;
  PropDev* d_props = nullptr;
  int props_cap = 0;
  float* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  // pinned staging ring for small host-to-device copies: a copy's source is
  // copied here and the transfer runs asynchronously; the ring restarts after
  // every full stream synchronisation (all earlier transfers are done)
  unsigned char* pin = nullptr;
  size_t pin_cap = 0, pin_used = 0;
  // pinned landing area of the BaB step's device-to-host reads (Readback)
  unsigned char* rb = nullptr;
  size_t rb_cap = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  // profiling: kernel-class timing with CUDA events, launch and copy counters
  bool prof = false;
  uint64_t prof_mask = ~uint64_t(0);  // kernel classes timed with CUDA events
  // (class | (phase + 1) << 8 | graph-owned << 16, event pair)
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  int phase = -1;  // BaB step phase whose launches are being issued (-1: none)
  std::vector<cudaEvent_t> ev_free;
  int64_t launches = 0;
  int64_t acc_n[32] = {0};
  double acc_ms[32] = {0}, acc_flops[32] = {0}, acc_bytes[32] = {0};
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  // request loop
  std::vector<Request*> requests;        // by ticket - 1
  std::deque<Request*> req_queue;        // queued, FIFO
  std::vector<int> reserved;             // reserved node slots per network
  uint64_t serve_budget = 0;             // HBM bytes the active requests may hold (0: budget)
  uint64_t serve_bytes = 0;              // HBM bytes the active requests hold
  // CUDA graphs of the optimisation loop
  bool graphs = false;
  struct GraphEntry* cap = nullptr;  // entry being captured (Scope records into it)
  std::vector<struct GraphEntry*> graph_cache;
  std::vector<cudaEvent_t> graph_events;  // events owned by captured graphs
  std::vector<TcConv*> tc_convs;          // tensor-core convolution operands of all networks
  std::vector<TcFc*> tc_fcs;              // pre-split FC weights of all networks
};

// A captured optimisation loop: its executable graph, the kernel-class work it
// does per replay, and (when captured with profiling) its event pairs.
struct GraphEntry {
  int net_id, M, steps, gamma, prof;
  float hp[8];
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  int64_t n[32] = {0};
  double flops[32] = {0}, bytes[32] = {0};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pairs;
};

namespace {

void* dalloc(mnbab_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (c->used + bytes > c->budget)
    fail(MNBAB_E_BUDGET, "HBM budget exceeded (" + std::to_string(c->used + bytes) + " > " +
                             std::to_string(c->budget) + " bytes)");
  void* p = nullptr;
  ck(cudaMalloc(&p, bytes), "cudaMalloc");
  c->used += bytes;
  c->allocs.push_back({p, bytes});
  return p;
}

template <typename T>
T* dalloc_t(mnbab_ctx* c, size_t n) {
  return static_cast<T*>(dalloc(c, n * sizeof(T)));
}

void sync(mnbab_ctx* c);

void h2d_bytes(mnbab_ctx* c, void* dst, const void* src, size_t bytes) {
  c->h2d_bytes += (int64_t)bytes;
  if (!bytes) return;
  if (c->pin && bytes <= c->pin_cap / 4) {
    if (c->pin_used + bytes > c->pin_cap - 64) sync(c);  // every staged transfer has completed
    unsigned char* stage = c->pin + c->pin_used;
    std::memcpy(stage, src, bytes);
    c->pin_used += (bytes + 15) & ~size_t(15);
    ck(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, c->st), "H2D");
    return;
  }
  ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->st), "H2D");
}

template <typename T>
void h2d(mnbab_ctx* c, T* dst, const T* src, size_t n) {
  h2d_bytes(c, dst, src, n * sizeof(T));
}

template <typename T>
void d2h(mnbab_ctx* c, T* dst, const T* src, size_t n) {
  c->d2h_bytes += (int64_t)(n * sizeof(T));
  if (n) ck(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, c->st), "D2H");
}

// Device-to-host reads that do not block the host: a copy into pageable memory
// returns only once it has completed, so the reads of a step land in the
// context's pinned area and finish() moves them to their destinations after the
// next stream synchronisation.  Without room (or without the area) a read falls
// back to a direct, blocking copy.
struct Readback {
  mnbab_ctx* c;
  struct Item {
    void* dst;
    size_t off, bytes;
  };
  std::vector<Item> items;
  size_t used = 0;
  explicit Readback(mnbab_ctx* c_) : c(c_) {}
  template <typename T>
  void add(T* dst, const T* src, size_t n) {
    const size_t b = n * sizeof(T);
    if (!b) return;
    if (!c->rb || used + b > c->rb_cap) {
      d2h(c, dst, src, n);
      return;
    }
    c->d2h_bytes += (int64_t)b;
    ck(cudaMemcpyAsync(c->rb + used, src, b, cudaMemcpyDeviceToHost, c->st), "D2H");
    items.push_back({dst, used, b});
    used += (b + 15) & ~size_t(15);
  }
  // after a synchronisation of the stream
  void finish() {
    for (const Item& it : items) std::memcpy(it.dst, c->rb + it.off, it.bytes);
    items.clear();
    used = 0;
  }
};

enum Cat {
  C_BACKSUB_FC, C_BACKSUB_CONV, C_FWD_FC, C_FWD_CONV, C_INIT, C_REDUCE, C_GAMMA, C_ADAM, C_ACS,
  C_BOOK, C_WIN, C_FUSED, C_SWEEP, C_BACKSUB_CONV_TC, C_FWD_CONV_TC, C_FUSED_TC, NKCAT,
  // host wall time of the BaB step phases (stream work included up to their syncs)
  H_ROOTS = NKCAT, H_REBOUND, H_DEEPPOLY, H_OPTIMIZE, H_CONFIRM, H_FINISH,
  // device time of all kernel classes launched within each phase
  G_ROOTS, G_REBOUND, G_DEEPPOLY, G_OPTIMIZE, G_CONFIRM, G_FINISH, NCAT
};
constexpr int NPHASE = 6;
static_assert(NCAT <= 32, "profile arrays hold 32 classes");
const char* CAT_NAMES[NCAT] = {"backsub_fc_gemm", "backsub_conv_transpose", "forward_fc_gemm",
                               "forward_conv",    "init_rows",              "reduce_lb",
                               "gamma_terms",     "adam",                   "acs",
                               "bookkeeping",     "backsub_conv_window",    "opt_fused_chain",
                               "backsub_rows_fused", "backsub_conv_tc", "forward_conv_tc",
                               "opt_fused_chain_tc",
                               "step_roots_wall",        "step_rebound_wall",
                               "step_deeppoly_wall", "step_optimize_wall",  "step_confirm_wall",
                               "step_finish_wall", "phase_roots_gpu",        "phase_rebound_gpu",
                               "phase_deeppoly_gpu", "phase_optimize_gpu",   "phase_confirm_gpu",
                               "phase_finish_gpu"};

struct HostTimer {
  mnbab_ctx* c;
  std::chrono::steady_clock::time_point t;
  explicit HostTimer(mnbab_ctx* c_) : c(c_), t(std::chrono::steady_clock::now()) { c->phase = 0; }
  ~HostTimer() { c->phase = -1; }
  void lap(int cat);
};

void resolve_prof(mnbab_ctx* c) {
  for (auto& r : c->pending) {
    const bool owned = (r.first >> 16) & 1;  // event pair owned by a captured graph
    const int cat = r.first & 0xff, phase = ((r.first >> 8) & 0xff) - 1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.second.first, r.second.second) == cudaSuccess) {
      c->acc_ms[cat] += ms;
      if (phase >= 0 && phase < NPHASE) c->acc_ms[G_ROOTS + phase] += ms;
    }
    if (!owned) {
      c->ev_free.push_back(r.second.first);
      c->ev_free.push_back(r.second.second);
    }
  }
  c->pending.clear();
}

void sync(mnbab_ctx* c) {
  // the tensor-core error flag rides on the same synchronisation (pinned copy)
  int* flag = c->pin ? reinterpret_cast<int*>(c->pin + c->pin_cap - 64) : nullptr;
  const bool check = c->d_err && c->gemm_path != 1;
  if (check && flag)
    ck(cudaMemcpyAsync(flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "error flag");
  ck(cudaStreamSynchronize(c->st), "stream synchronize");
  c->pin_used = 0;
  ck(cudaGetLastError(), "kernel launch");
  if (!c->pending.empty()) resolve_prof(c);
  if (check) {
    int e = 0;
    if (flag) e = *flag;
    else ck(cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
    if (e) {
      cudaMemset(c->d_err, 0, sizeof(int));
      fail(MNBAB_E_TIMEOUT, "a tensor-core kernel timed out waiting for its MMAs");
    }
  }
}

cudaEvent_t get_event(mnbab_ctx* c) {
  if (c->ev_free.empty()) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "cudaEventCreate");
    return e;
  }
  cudaEvent_t e = c->ev_free.back();
  c->ev_free.pop_back();
  return e;
}

// Counts the launches of one kernel class and their algorithmic work; with
// profiling on, brackets them with CUDA events on the context's stream.
struct Scope {
  mnbab_ctx* c;
  int cat;
  cudaEvent_t a = nullptr, b = nullptr;
  Scope(mnbab_ctx* c_, int cat_, double flops, double bytes, int nl = 1) : c(c_), cat(cat_) {
    if (c->cap) {
      // inside a graph capture: the work is counted per replay; with profiling the
      // events become event-record nodes of the graph
      GraphEntry* g = c->cap;
      g->launches += nl;
      g->n[cat] += nl;
      g->flops[cat] += flops;
      g->bytes[cat] += bytes;
      if (g->prof && ((c->prof_mask >> cat) & 1)) {
        ck(cudaEventCreate(&a), "cudaEventCreate");
        ck(cudaEventCreate(&b), "cudaEventCreate");
        c->graph_events.push_back(a);
        c->graph_events.push_back(b);
        ck(cudaEventRecordWithFlags(a, c->st, cudaEventRecordExternal), "event record");
      }
      return;
    }
    c->launches += nl;
    c->acc_n[cat] += nl;
    c->acc_flops[cat] += flops;
    c->acc_bytes[cat] += bytes;
    if (c->prof && ((c->prof_mask >> cat) & 1)) {
      if (c->pending.size() > 8192) sync(c);
      a = get_event(c);
      b = get_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~Scope() {
    if (!a) return;
    if (c->cap) {
      cudaEventRecordWithFlags(b, c->st, cudaEventRecordExternal);
      c->cap->pairs.push_back({cat | ((c->phase + 1) << 8), {a, b}});
      return;
    }
    cudaEventRecord(b, c->st);
    c->pending.push_back({cat | ((c->phase + 1) << 8), {a, b}});
  }
};

void HostTimer::lap(int cat) {
  const auto now = std::chrono::steady_clock::now();
  if (c->prof) {
    c->acc_ms[cat] += std::chrono::duration<double, std::milli>(now - t).count();
    c->acc_n[cat] += 1;
  }
  c->phase = cat + 1 - H_ROOTS < NPHASE ? cat + 1 - H_ROOTS : -1;  // the phase that follows
  t = now;
}

double layer_macs(const LayerDev& L) {
  return L.kind == 1 ? (double)L.d_in * L.d_out : (double)L.co * L.ho * L.wo * L.ci * L.k * L.k;
}
double layer_wbytes(const LayerDev& L) {
  return 4.0 * (L.kind == 1 ? (double)L.d_in * L.d_out : (double)L.co * L.ci * L.k * L.k);
}

// ---------------------------------------------------------------------------
// node pool
// ---------------------------------------------------------------------------
int alloc_slot(mnbab_net* n) {
  if (n->free_slots.empty()) fail(MNBAB_E_BUDGET, "node pool exhausted");
  const int s = n->free_slots.back();
  n->free_slots.pop_back();
  n->slot_used[s] = 1;
  return s;
}

void free_slot(mnbab_net* n, int s) {
  if (s < 0 || s >= n->cap || !n->slot_used[s]) return;
  n->slot_used[s] = 0;
  n->free_slots.push_back(s);
}

// Device property table: grows by doubling (the previous table stays
// allocated until destroy: kernels already queued may still read it); a new or
// changed property uploads only its own entry.
void upload_prop(mnbab_ctx* c, int index) {
  const int np = (int)c->props.size();
  if (np > c->props_cap) {
    const int nc = std::max(64, np * 2);
    PropDev* nd = dalloc_t<PropDev>(c, nc);
    if (c->d_props && c->props_cap)
      ck(cudaMemcpyAsync(nd, c->d_props, (size_t)c->props_cap * sizeof(PropDev),
                         cudaMemcpyDeviceToDevice, c->st), "table copy");
    c->d_props = nd;
    c->props_cap = nc;
  }
  h2d(c, c->d_props + index, &c->props[index]->pd, 1);
}

// Bump allocator for per-property arrays (input box, folded last layer), so
// admitting a property issues no cudaMalloc in the common case.
float* prop_arena(mnbab_ctx* c, size_t nfloats) {
  nfloats = (nfloats + 63) & ~size_t(63);
  if (c->arena_used + nfloats > c->arena_cap) {
    const size_t cap = std::max(nfloats, (size_t)16 << 20);  // 64 MiB blocks
    c->arena = dalloc_t<float>(c, cap);
    c->arena_cap = cap;
    c->arena_used = 0;
  }
  float* p = c->arena + c->arena_used;
  c->arena_used += nfloats;
  return p;
}

Epi base_epi(mnbab_net* n, const int* row_node) {
  Epi e{};
  e.SD = n->SD;
  e.d0 = n->d0;
  e.row_node = row_node;
  e.pool = n->pool;
  e.props = n->ctx->d_props;
  e.part = n->part;
  e.nslot = n->nslot;
  e.bias_div = 1;
  e.gemm_path = n->ctx->gemm_path;
  e.err = n->ctx->d_err;
  e.ws = n->splitk;
  e.ws_floats = n->splitk_floats;
  return e;
}

void relu_epi(mnbab_net* n, Epi& e, int layer) {
  e.kind = EPI_RELU;
  e.layer = layer;
  e.off = n->nd.off[layer];
  e.bias = n->nd.bfull[layer];  // sum of the edge biases into zhat_layer, per neuron
  e.bias_div = 1;
}

float* lam_buf(mnbab_net* n, int s) { return n->lam + n->lam_off[s]; }

const LayerDev& edge_of(const mnbab_net* n, int t, int k) {
  return k == 0 ? n->nd.aff[t] : n->nd.aff2[t];
}
int src_of(const mnbab_net* n, int t, int k) { return k == 0 ? n->nd.src1[t] : n->nd.src2[t]; }

struct SweepOpts {
  bool final_mode = false;  // objective rows with the node's alpha, beta (gamma if has_gamma)
  bool has_gamma = false;
  bool store = false;       // keep a' checkpoints and x*
  bool track = false;       // keep best bound / minimiser per node
  bool keep_a0 = false;     // write the input coefficients a0 to the input buffer
};

// Back-substitutes rows that all start at zhat^(t) down to the input, node by
// node in descending order.  Every node's coefficients live in its own buffer;
// an edge into source s writes its contribution raw unless it is s's last
// consumer in this sweep, which adds the earlier contribution and applies s's
// ReLU (or concretisation) epilogue.
void sweep(mnbab_net* n, int t, const RowsDev& rows, const SweepOpts& o) {
  mnbab_ctx* c = n->ctx;
  if (rows.M <= 0) return;
  const NetDev& nd = n->nd;
  const bool unit = rows.cidx == nullptr;  // the fast paths take rows of one neuron
  if (unit && !o.final_mode && !o.store && !o.track && t == 1 && nd.n_edge[1] == 1 &&
      nd.src1[1] == 0) {
    // rows of layer 1: a dot product with the input box per row
    Scope sc(c, C_INIT, 2.0 * rows.M * nd.d[0], 12.0 * rows.M);
    launch_first_rows(nd, n->pool, c->d_props, rows, n->lb, c->st);
    return;
  }
  if (unit && !o.final_mode && !o.store && !o.track && sweep_chain_supported(nd, t)) {
    // dense intermediate-bound rows above a chain: persistent fused sweep
    double macs = nd.d[t - 1];
    for (int i = 1; i < t; ++i) macs += layer_macs(nd.aff[i]);
    Scope sc(c, C_SWEEP, 2.0 * rows.M * macs, 4.0 * rows.M * (nd.d[t - 1] + 4.0 * n->SD));
    launch_sweep_chain(nd, n->pool, c->d_props, rows, t, n->lb, c->st);
    return;
  }
  WinPlan wp;
  if (unit && !o.final_mode && !o.store && !o.track && win_plan(nd, t, wp)) {
    // intermediate-bound rows of a convolution neuron: receptive-field windows
    double macs = 0.0, elems = (double)nd.aff[t].ci * wp.h[t - 1] * wp.w[t - 1];
    for (int i = t - 1; i >= 1; --i) {
      const LayerDev& L = nd.aff[i];
      const double taps = std::ceil((double)L.k / L.s);
      macs += (double)L.ci * wp.h[i - 1] * wp.w[i - 1] * L.co * taps * taps;
      elems += (double)L.ci * wp.h[i - 1] * wp.w[i - 1];
    }
    Epi e = base_epi(n, rows.node);
    e.slot_base = 0;
    {
      Scope sc(c, C_WIN, 2.0 * rows.M * macs, 9.0 * rows.M * elems);
      launch_win_rows(nd, wp, rows, e, c->st);
    }
    Scope sc(c, C_REDUCE, 0.0, 4.0 * rows.M);
    launch_reduce_lb(rows.M, n->part, n->nslot, 1, nullptr, n->lb, false, rows.node, n->pool,
                     n->X, n->d0, c->st);
    return;
  }
  auto setup = [&](Epi& e, int layer) {
    if (layer >= 1) {
      relu_epi(n, e, layer);
      e.final_mode = o.final_mode;
      if (o.final_mode && o.has_gamma) {
        e.GP = n->GP;
        e.GPh = n->GPh;
      }
      if (o.store) e.AP = n->AP;
    } else {
      e.kind = EPI_CONC;
      if (o.store || o.track) e.X = n->X;
    }
  };
  // nodes reached from t, and the last (smallest) consumer of every source
  bool reached[MNBAB_MAXR + 2] = {false};
  int lastc[MNBAB_MAXR + 2];
  for (int s0 = 0; s0 <= MNBAB_MAXR + 1; ++s0) lastc[s0] = -1;
  reached[t] = true;
  for (int v = t; v >= 1; --v) {
    if (!reached[v]) continue;
    for (int k = 0; k < nd.n_edge[v]; ++k) {
      const int sidx = src_of(n, v, k);
      reached[sidx] = true;
      lastc[sidx] = v;  // descending scan: ends at the smallest consumer
    }
  }
  int need = 1;
  for (int v = t; v >= 1; --v)
    if (reached[v])
      for (int k = 0; k < nd.n_edge[v]; ++k)
        need += v == t ? 1 : backsub_slots(edge_of(n, v, k));
  if (need > n->nslot) fail(MNBAB_E_DEVICE, "partial-sum slots overflow");
  if (rows.M > n->chunk && rows.M > n->B) fail(MNBAB_E_DEVICE, "row block larger than scratch");
  bool written[MNBAB_MAXR + 2] = {false};
  int used = 0;
  bool conv_only = t <= nd.R;  // every edge met so far is a convolution
  for (int v = t; v >= 1; --v) {
    if (!reached[v]) continue;
    for (int k = 0; k < nd.n_edge[v]; ++k) {
      const int sidx = src_of(n, v, k);
      const bool last = lastc[sidx] == v;
      Epi e = base_epi(n, rows.node);
      if (last) setup(e, sidx);
      else e.kind = EPI_STORE;
      if (written[sidx]) {
        e.acc_in = lam_buf(n, sidx);
        e.acc_ld = nd.d[sidx];
      }
      e.slot_base = used;
      e.sparse_rows = conv_only ? 1 : 0;
      float* out = (sidx >= 1 || !last || o.keep_a0) ? lam_buf(n, sidx) : nullptr;
      if (v == t) {
        Scope sc(c, C_INIT, 0.0, 4.0 * rows.M * nd.d[sidx]);
        launch_init_rows(nd, t, k, rows, out, nd.d[sidx], e, c->st);
        used += 1;
      } else {
        const LayerDev& L = edge_of(n, v, k);
        Scope sc(c, L.kind == 1 ? C_BACKSUB_FC
                                : (conv_tc_chosen(L, 1, e, rows.M) ? C_BACKSUB_CONV_TC : C_BACKSUB_CONV),
                 2.0 * rows.M * layer_macs(L),
                 4.0 * rows.M * (L.d_out + (out ? L.d_in : 0)) + layer_wbytes(L));
        const int sl = launch_backsub(L, rows.M, lam_buf(n, v), nd.d[v], out, nd.d[sidx], e, c->st);
        if (last) used += sl;  // raw contributions write no offset partials
      }
      written[sidx] = true;
    }
    for (int k = 0; k < nd.n_edge[v]; ++k)
      if (edge_of(n, v, k).kind != MNBAB_CONV2D) conv_only = false;
  }
  Scope sc(c, C_REDUCE, 0.0, 4.0 * rows.M * used);
  launch_reduce_lb(rows.M, n->part, n->nslot, used,
                   (o.final_mode && o.has_gamma) ? n->gp0 : nullptr, n->lb, o.track, rows.node,
                   n->pool, n->X, n->d0, c->st);
}

// Re-bounds ReLU layers t > split layer of each node (Sec. 3.2, enforcing
// splits); rows are the node's unstable unsplit neurons, both sides.  The rows
// of every layer are collected up front (a layer's row set depends only on its
// own current bounds), so a pass costs one host synchronisation.  For fresh
// root slots (`fresh`: every bound infinite, nothing split) every neuron is a
// row, so the counts are known on the host and the pass does not synchronise.
int64_t rebound(mnbab_net* n, const std::vector<int>& slots, bool fresh = false) {
  mnbab_ctx* c = n->ctx;
  const int R = n->R;
  int64_t total = 0;
  std::vector<int> sel;
  for (int s : slots)
    if (n->slot_split[s] < R) sel.push_back(s);
  const int per = std::max(1, std::min(n->B, (int)(n->rows_cap / (2 * (size_t)n->SD))));
  std::vector<int> lay;
  for (size_t done = 0; done < sel.size(); done += per) {
    const int nb = (int)std::min(sel.size() - done, (size_t)per);
    int cnt[MNBAB_MAXR + 2] = {0};
    size_t region[MNBAB_MAXR + 2] = {0};
    size_t at = 0;
    ck(cudaMemsetAsync(n->counter, 0, (MNBAB_MAXR + 2) * sizeof(int), c->st), "memset");
    for (int t = 1; t <= R; ++t) {
      lay.clear();
      for (int k = 0; k < nb; ++k)
        if (n->slot_split[sel[done + k]] < t) lay.push_back(sel[done + k]);
      region[t] = at;
      cnt[t] = (int)lay.size();
      if (lay.empty()) continue;
      h2d(c, n->rb_nodes + (size_t)t * n->B, lay.data(), lay.size());
      Scope sc(c, C_BOOK, 0.0, 9.0 * lay.size() * n->nd.d[t]);
      launch_collect_rows((int)lay.size(), n->rb_nodes + (size_t)t * n->B, n->pool, n->nd.off[t],
                          n->nd.d[t], n->counter + t, n->row_node + at, n->row_j + at,
                          n->row_sign + at, c->st);
      at += 2 * lay.size() * (size_t)n->nd.d[t];
    }
    int M[MNBAB_MAXR + 2] = {0};
    if (fresh) {
      for (int t = 1; t <= R; ++t) M[t] = 2 * cnt[t] * n->nd.d[t];
    } else {
      d2h(c, M, n->counter, R + 1);
      sync(c);
    }
    for (int t = 1; t <= R; ++t) {
      if (!cnt[t] || !M[t]) continue;
      total += M[t];
      for (int s0 = 0; s0 < M[t]; s0 += n->chunk) {
        const int Mc = std::min(n->chunk, M[t] - s0);
        const size_t o = region[t] + s0;
        RowsDev r{Mc, n->row_node + o, n->row_j + o, n->row_sign + o};
        SweepOpts so;
        sweep(n, t, r, so);
        Scope sc(c, C_BOOK, 0.0, 24.0 * Mc);
        launch_update_bounds(Mc / 2, r.node, r.j, n->lb, n->pool, n->nd.off[t], c->st);
      }
    }
  }
  for (int s : slots) n->slot_split[s] = R;
  return total;
}

bool batch_has_gamma(mnbab_net* n, const std::vector<int>& slots) {
  for (int s : slots)
    if (n->ctx->props[n->slot_prop[s]]->pd.E > 0) return true;
  return false;
}

void upload_batch(mnbab_net* n, const std::vector<int>& slots) {
  std::vector<int> rows(slots.size());
  for (size_t i = 0; i < slots.size(); ++i) rows[i] = n->slot_row[slots[i]];
  h2d(n->ctx, n->bslots, slots.data(), slots.size());
  h2d(n->ctx, n->brows, rows.data(), rows.size());
}

RowsDev obj_rows(mnbab_net* n, int M) { return RowsDev{M, n->bslots, n->brows, nullptr}; }

// adjoint sweep from x* up through the ReLU layers (d lb / d ahat_t is the
// forward pass of the relaxed network at x*); a node with two edges stores the
// first edge's product and finishes with the second.
// Forward pass of the relaxed network at the rows' x* through ReLU layers
// 1 .. upto (all of them by default), writing d lb / d alpha and d lb / d beta.
void adjoint(mnbab_net* n, int M, bool has_gamma, int upto = -1) {
  mnbab_ctx* c = n->ctx;
  const NetDev& nd = n->nd;
  const int top = upto < 0 ? n->R : std::min(upto, n->R);
  for (int t = 1; t <= top; ++t) {
    for (int k = 0; k < nd.n_edge[t]; ++k) {
      const int sidx = src_of(n, t, k);
      Epi e = base_epi(n, n->bslots);
      e.part = nullptr;
      if (k == nd.n_edge[t] - 1) {
        e.kind = EPI_ADJ;
        e.layer = t;
        e.off = nd.off[t];
        e.AP = n->AP;
        e.GA = n->GA;
        e.GB = n->GB;
        if (has_gamma) {
          e.Gz = n->Gz;
          e.Hz = n->Hz;
        }
      } else {
        e.kind = EPI_STORE;
      }
      if (k > 0) {
        e.acc_in = lam_buf(n, t);
        e.acc_ld = nd.d[t];
      }
      const float* in = sidx == 0 ? n->X : lam_buf(n, sidx);
      const int ld_in = sidx == 0 ? n->d0 : nd.d[sidx];
      const LayerDev& L = edge_of(n, t, k);
      Scope sc(c, L.kind == 1 ? C_FWD_FC : (conv_tc_chosen(L, 0, e, M) ? C_FWD_CONV_TC : C_FWD_CONV),
               2.0 * M * layer_macs(L),
               4.0 * M * (L.d_in + L.d_out) + layer_wbytes(L));
      launch_forward(L, M, in, ld_in, lam_buf(n, t), nd.d[t], e, c->st);
    }
  }
  if (has_gamma) {
    Scope sc(c, C_GAMMA, 0.0, 4.0 * M * c->EC);
    launch_gamma_grad(M, n->bslots, n->pool, c->d_props, n->nd, n->Gz, n->Hz, n->GG, c->st);
  }
}

void run_optimize_body(mnbab_net* n, int M, bool has_gamma, const mnbab_adam& a,
                       const float* skip_lb = nullptr);

// Whether run_optimize takes the fused one-launch loop for this batch.
bool fused_path(mnbab_net* n, bool has_gamma, int steps) {
  return !has_gamma && n->ctx->gemm_path != 2 && fused_supported(n->nd, n->SD, n->d0, steps);
}

// Takes work back out of a kernel class's algorithmic counts (rows a launch was
// sized for that its kernel skipped).
void prof_sub(mnbab_ctx* c, int cat, double flops, double bytes) {
  c->acc_flops[cat] -= flops;
  c->acc_bytes[cat] -= bytes;
}

// The optimisation loop, replayed from a CUDA graph: the row count is padded up
// to a multiple of 64 with rows that point at the network's pad slot (its state
// is scratch: nothing reads it), so a handful of graphs cover every batch size.
// skip_lb (fused path without graphs only): rows whose DeepPoly bound is positive
// are not optimised.
void run_optimize(mnbab_net* n, int M, bool has_gamma, const mnbab_adam& a,
                  const float* skip_lb = nullptr) {
  mnbab_ctx* c = n->ctx;
  if (!c->graphs || n->pad_slot < 0) {
    run_optimize_body(n, M, has_gamma, a, skip_lb);
    return;
  }
  const int Mb = std::min(n->B, (M + 63) / 64 * 64);
  if (Mb > M) {
    std::vector<int> pad(Mb - M, n->pad_slot), zr(Mb - M, 0);
    h2d(c, n->bslots + M, pad.data(), pad.size());
    h2d(c, n->brows + M, zr.data(), zr.size());
  }
  const float hp[8] = {a.lr_alpha, a.lr_beta, a.lr_gamma, a.beta1, a.beta2, a.eps, a.grad_floor,
                       a.eps_rel};
  GraphEntry* g = nullptr;
  for (auto* e : c->graph_cache)
    if (e->net_id == n->id && e->M == Mb && e->steps == a.steps && e->gamma == (int)has_gamma &&
        e->prof == (int)c->prof && std::memcmp(e->hp, hp, sizeof(hp)) == 0)
      g = e;
  if (!g) {
    g = new GraphEntry();
    g->net_id = n->id;
    g->M = Mb;
    g->steps = a.steps;
    g->gamma = has_gamma;
    g->prof = c->prof;
    std::memcpy(g->hp, hp, sizeof(hp));
    cudaGraph_t graph = nullptr;
    ck(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "begin capture");
    c->cap = g;
    try {
      run_optimize_body(n, Mb, has_gamma, a);
    } catch (...) {
      c->cap = nullptr;
      cudaStreamEndCapture(c->st, &graph);
      if (graph) cudaGraphDestroy(graph);
      delete g;
      throw;
    }
    c->cap = nullptr;
    ck(cudaStreamEndCapture(c->st, &graph), "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      delete g;
      fail(MNBAB_E_DEVICE, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    c->graph_cache.push_back(g);
  }
  ck(cudaGraphLaunch(g->exec, c->st), "graph launch");
  c->launches += g->launches;
  for (int i = 0; i < 32; ++i) {
    c->acc_n[i] += g->n[i];
    c->acc_flops[i] += g->flops[i];
    c->acc_bytes[i] += g->bytes[i];
  }
  for (auto& pr : g->pairs) c->pending.push_back({(1 << 16) | pr.first, pr.second});
}

void run_optimize_body(mnbab_net* n, int M, bool has_gamma, const mnbab_adam& a,
                       const float* skip_lb) {
  mnbab_ctx* c = n->ctx;
  if (fused_path(n, has_gamma, a.steps)) {
    // the whole loop in one launch, one CTA per row
    FusedHP hp{};
    hp.steps = a.steps;
    hp.lr_a = a.lr_alpha;
    hp.lr_b = a.lr_beta;
    hp.b1 = a.beta1;
    hp.b2 = a.beta2;
    hp.eps_abs = a.eps;
    hp.eps_rel = a.eps_rel;
    hp.floor = a.grad_floor;
    double b1t = 1.0, b2t = 1.0;
    for (int s = 0; s < a.steps; ++s) {
      b1t *= a.beta1;
      b2t *= a.beta2;
      hp.bc1[s] = (float)(1.0 - b1t);
      hp.bc2[s] = (float)(1.0 - b2t);
    }
    double macs = 0.0;
    for (int t = 1; t <= n->R; ++t) macs += layer_macs(n->nd.aff[t]);
    // one conv layer's transposed convolution on the tensor cores (class
    // opt_fused_chain_tc) unless the SIMT path is forced
    const bool tc = c->gemm_path != 1 && fused_tc_layer(n->nd, n->SD, n->d0) > 0;
    n->fused_cat = tc ? C_FUSED_TC : C_FUSED;
    n->fused_row_flops = 2.0 * ((a.steps + 1.0) * (macs + n->nd.d[n->R]) + a.steps * macs);
    n->fused_row_bytes = (a.steps + 1.0) * n->SD * 66.0;
    Scope sc(c, n->fused_cat, M * n->fused_row_flops, M * n->fused_row_bytes);
    launch_opt_chain(M, n->nd, n->pool, c->d_props, n->bslots, n->brows, hp, n->AP, n->GB, tc,
                     c->d_err, c->st, skip_lb);
    return;
  }
  {
    Scope sc(c, C_BOOK, 0.0, 16.0 * M * (n->SD + c->EC));
    launch_zero_adam(M, n->bslots, n->pool, c->st);
  }
  SweepOpts o;
  o.final_mode = true;
  o.has_gamma = has_gamma;
  o.store = true;
  o.track = true;
  double b1t = 1.0, b2t = 1.0;
  for (int step = 0; step <= a.steps; ++step) {
    if (has_gamma) {
      Scope sc(c, C_GAMMA, 0.0, 4.0 * M * (c->EC + 2.0 * n->SD), 2);
      launch_gamma_proj(M, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
    }
    sweep(n, n->R + 1, obj_rows(n, M), o);
    if (step == a.steps) break;
    adjoint(n, M, has_gamma);
    b1t *= a.beta1;
    b2t *= a.beta2;
    Scope sc(c, C_ADAM, 0.0, 4.0 * M * (2.0 * n->SD + c->EC) * 8.0, 2);
    launch_adam(M, n->bslots, n->pool, c->d_props, n->SD, n->GA, n->GB, n->GG, n->gmax,
                a.grad_floor, a.lr_alpha, a.lr_beta, a.lr_gamma, a.beta1, a.beta2, a.eps,
                a.eps_rel, (float)(1.0 - b1t), (float)(1.0 - b2t), c->st);
  }
}

// FP32 forward pass of rows of `x` ([M][d0]) -> f_r in n->fout
void forward_rows(mnbab_net* n, int M, const float* x) {
  mnbab_ctx* c = n->ctx;
  const NetDev& nd = n->nd;
  for (int t = 1; t <= n->R; ++t) {
    for (int k = 0; k < nd.n_edge[t]; ++k) {
      const int sidx = src_of(n, t, k);
      Epi e = base_epi(n, n->bslots);
      e.part = nullptr;
      e.kind = k == nd.n_edge[t] - 1 ? EPI_FWD_RELU : EPI_STORE;
      if (k > 0) {
        e.acc_in = lam_buf(n, t);
        e.acc_ld = nd.d[t];
      }
      const float* in = sidx == 0 ? x : lam_buf(n, sidx);
      const int ld_in = sidx == 0 ? n->d0 : nd.d[sidx];
      const LayerDev& L = edge_of(n, t, k);
      Scope sc(c, L.kind == 1 ? C_FWD_FC : (conv_tc_chosen(L, 0, e, M) ? C_FWD_CONV_TC : C_FWD_CONV),
               2.0 * M * layer_macs(L),
               4.0 * M * (L.d_in + L.d_out) + layer_wbytes(L));
      launch_forward(L, M, in, ld_in, lam_buf(n, t), nd.d[t], e, c->st);
    }
  }
  const int sR = nd.src1[n->R + 1];
  const int dR = nd.d[sR];
  const float* z = sR == 0 ? x : lam_buf(n, sR);
  Scope sc(c, C_BOOK, 2.0 * M * dR, 8.0 * M * dR);
  launch_final_dot(M, n->bslots, n->pool, c->d_props, z, sR == 0 ? n->d0 : dR, dR, n->fout, c->st);
}

__global__ void k_gather_rows(int M, const int* idx, const float* src, int ld_src, float* dst,
                              int ld_dst, int w) {
  const int m = blockIdx.x;
  const float* s = src + (size_t)idx[m] * ld_src;
  for (int k = threadIdx.x; k < w; k += blockDim.x) dst[(size_t)m * ld_dst + k] = s[k];
}

// the same for the first *count rows (a count on the device; the grid covers the
// largest possible count)
__global__ void k_gather_rows_n(const int* count, const int* idx, const float* src, int ld_src,
                                float* dst, int ld_dst, int w) {
  const int m = blockIdx.x;
  if (m >= *count) return;
  const float* s = src + (size_t)idx[m] * ld_src;
  for (int k = threadIdx.x; k < w; k += blockDim.x) dst[(size_t)m * ld_dst + k] = s[k];
}

__global__ void k_gather1(int M, const int* idx, const float* src, float* dst) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) dst[m] = src[idx[m]];
}

mnbab_adam default_adam() {
  mnbab_adam a;
  a.steps = 20;
  a.lr_alpha = 0.1f;
  a.lr_beta = 0.05f;
  a.lr_gamma = 0.05f;
  a.beta1 = 0.9f;
  a.beta2 = 0.999f;
  a.eps = 1e-8f;
  a.grad_floor = 0.0f;
  a.eps_rel = 0.0f;  // standard Adam; the gradient-scaled eps is an option
  return a;
}

mnbab_net* net_of(mnbab_ctx* c, mnbab_node_id id, int* slot) {
  const int ni = (int)(id >> 32);
  const int s = (int)(id & 0xffffffff);
  if (ni < 0 || ni >= (int)c->nets.size()) fail(MNBAB_E_INVALID_ARG, "bad node id");
  mnbab_net* n = c->nets[ni];
  if (s < 0 || s >= n->cap || !n->slot_used[s]) fail(MNBAB_E_INVALID_ARG, "node id not live");
  *slot = s;
  return n;
}

mnbab_net* slots_of(mnbab_ctx* c, const mnbab_node_id* nodes, int nn, std::vector<int>& slots) {
  if (nn <= 0 || !nodes) fail(MNBAB_E_INVALID_ARG, "empty node list");
  mnbab_net* net = nullptr;
  slots.resize(nn);
  for (int i = 0; i < nn; ++i) {
    int s;
    mnbab_net* n = net_of(c, nodes[i], &s);
    if (net && n != net) fail(MNBAB_E_INVALID_ARG, "nodes of different networks in one batch");
    net = n;
    slots[i] = s;
  }
  if (nn > net->B) fail(MNBAB_E_INVALID_ARG, "batch larger than the context's batch capacity");
  return net;
}

void gather_best(mnbab_net* n, int M, float* host_out, Readback* rb = nullptr) {
  {
    Scope sc(n->ctx, C_BOOK, 0.0, 12.0 * M);
    k_gather1<<<(M + 255) / 256, 256, 0, n->ctx->st>>>(M, n->bslots, n->pool.BEST, n->bestb);
  }
  if (rb) rb->add(host_out, n->bestb, M);
  else d2h(n->ctx, host_out, n->bestb, M);
}

__global__ void k_acc_rows(size_t n, const float* x, float* acc) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] += x[i];
}

__global__ void k_scale_rows(size_t n, const float* x, float s, float* out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] * s;
}

// Exact completion of fully split nodes (Sec. 3.3): with every unstable neuron
// split, the network is affine on the node's region, so maximising the bound
// over beta (and gamma) reaches the region's exact minimum by LP duality, and
// every iterate's bound is a certified lower bound.  `steps` more projected
// Adam steps from the nodes' parameters (the node keeps the best bound); the
// average of the iterates' minimisers x* over the second half of the steps
// converges to a minimiser of the region and is checked in FP64 as a
// counterexample candidate.  best, f64 (f_r at the average) and xavg [M][d0]
// come back to the host.
void leaf_complete(mnbab_net* n, const std::vector<int>& slots, int steps, const mnbab_adam& a,
                   std::vector<float>& best, std::vector<double>& f64, std::vector<float>& xavg) {
  mnbab_ctx* c = n->ctx;
  const int M = (int)slots.size();
  const size_t nx = (size_t)M * n->d0;
  if (!n->xsum) n->xsum = dalloc_t<float>(c, (size_t)n->B * n->d0);
  upload_batch(n, slots);
  const bool g = batch_has_gamma(n, slots);
  {
    Scope sc(c, C_BOOK, 0.0, 16.0 * M * (n->SD + c->EC) + 4.0 * nx);
    launch_zero_adam(M, n->bslots, n->pool, c->st);
    launch_fill(n->xsum, nx, 0.f, c->st);
  }
  SweepOpts o;
  o.final_mode = true;
  o.has_gamma = g;
  o.store = true;
  o.track = true;
  double b1t = 1.0, b2t = 1.0;
  int cnt = 0;
  for (int step = 0; step <= steps; ++step) {
    if (g) {
      Scope sc(c, C_GAMMA, 0.0, 4.0 * M * (c->EC + 2.0 * n->SD), 2);
      launch_gamma_proj(M, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
    }
    sweep(n, n->R + 1, obj_rows(n, M), o);  // x* of this iterate in n->X
    if (2 * step >= steps) {
      Scope sc(c, C_BOOK, 0.0, 12.0 * nx);
      k_acc_rows<<<(unsigned)((nx + 255) / 256), 256, 0, c->st>>>(nx, n->X, n->xsum);
      ++cnt;
    }
    if (step == steps) break;
    adjoint(n, M, g);
    b1t *= a.beta1;
    b2t *= a.beta2;
    Scope sc(c, C_ADAM, 0.0, 4.0 * M * (2.0 * n->SD + c->EC) * 8.0, 2);
    launch_adam(M, n->bslots, n->pool, c->d_props, n->SD, n->GA, n->GB, n->GG, n->gmax,
                a.grad_floor, a.lr_alpha, a.lr_beta, a.lr_gamma, a.beta1, a.beta2, a.eps,
                a.eps_rel, (float)(1.0 - b1t), (float)(1.0 - b2t), c->st);
  }
  {
    Scope sc(c, C_BOOK, 0.0, 8.0 * nx);
    k_scale_rows<<<(unsigned)((nx + 255) / 256), 256, 0, c->st>>>(nx, n->xsum, 1.f / cnt, n->Xb);
  }
  {
    Scope sc(c, C_BOOK, 0.0, 8.0 * M * n->maxd, n->R + 2);
    launch_forward_f64(M, n->bslots, n->pool, c->d_props, n->nd, n->Xb, n->d0, n->f64a,
                       n->d0 + n->SD, n->f64out, c->st);
  }
  f64.resize(M);
  xavg.resize(nx);
  d2h(c, f64.data(), n->f64out, M);
  d2h(c, xavg.data(), n->Xb, nx);
  best.resize(M);
  gather_best(n, M, best.data());
  sync(c);
}

void setup_net(mnbab_ctx* c, mnbab_net* n) {
  // dims
  n->maxd = n->d0;
  n->maxd_relu = 1;
  for (int i = 1; i <= n->R; ++i) {
    n->maxd = std::max(n->maxd, n->nd.d[i]);
    n->maxd_relu = std::max(n->maxd_relu, n->nd.d[i]);
  }
  n->nslot = 4;
  for (int i = 1; i <= n->R + 1; ++i)
    for (int k = 0; k < n->nd.n_edge[i]; ++k)
      n->nslot += backsub_slots(k == 0 ? n->nd.aff[i] : n->nd.aff2[i]);
  // pool
  n->cap = c->node_cap;
  const size_t SD = n->SD, EC = c->EC, cap = n->cap;
  PoolDev& P = n->pool;
  P.SD = n->SD;
  P.EC = c->EC;
  P.d0 = n->d0;
  P.L = dalloc_t<float>(c, cap * SD);
  P.U = dalloc_t<float>(c, cap * SD);
  P.ALPHA = dalloc_t<float>(c, cap * SD);
  P.BETA = dalloc_t<float>(c, cap * SD);
  P.S = dalloc_t<int8_t>(c, cap * SD);
  P.MA = dalloc_t<float>(c, cap * SD);
  P.VA = dalloc_t<float>(c, cap * SD);
  P.MB = dalloc_t<float>(c, cap * SD);
  P.VB = dalloc_t<float>(c, cap * SD);
  P.GAM = dalloc_t<float>(c, cap * EC);
  P.MG = dalloc_t<float>(c, cap * EC);
  P.VG = dalloc_t<float>(c, cap * EC);
  P.BESTX = dalloc_t<float>(c, cap * n->d0);
  P.BEST = dalloc_t<float>(c, cap);
  P.prop = dalloc_t<int>(c, cap);
  P.row = dalloc_t<int>(c, cap);
  n->free_slots.resize(cap);
  for (int i = 0; i < (int)cap; ++i) n->free_slots[i] = (int)cap - 1 - i;
  n->slot_split.assign(cap, 0);
  n->slot_row.assign(cap, 0);
  n->slot_prop.assign(cap, 0);
  n->slot_used.assign(cap, 0);
  // pad slot: finite scratch state (l = u = 0, no splits, zero parameters)
  n->pad_slot = alloc_slot(n);
  {
    const size_t o = (size_t)n->pad_slot * SD;
    ck(cudaMemsetAsync(P.L + o, 0, SD * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.U + o, 0, SD * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.S + o, 0, SD, c->st), "memset");
    ck(cudaMemsetAsync(P.ALPHA + o, 0, SD * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.BETA + o, 0, SD * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.prop + n->pad_slot, 0, sizeof(int), c->st), "memset");
    ck(cudaMemsetAsync(P.row + n->pad_slot, 0, sizeof(int), c->st), "memset");
  }
  // scratch
  n->B = std::min(1024, std::max(1, (int)cap / 2));
  n->chunk = std::max(2, c->row_chunk & ~1);
  const size_t chunk = n->chunk, B = n->B;
  const size_t mrows = std::max(chunk, B);
  // per-layer coefficient buffers (input layer included)
  {
    size_t at = 0;
    for (int sidx = 0; sidx <= n->R; ++sidx) {
      n->lam_off[sidx] = at;
      at += mrows * (size_t)n->nd.d[sidx];
    }
    n->lam = dalloc_t<float>(c, at);
  }
  n->part = dalloc_t<float>(c, mrows * n->nslot);
  n->lb = dalloc_t<float>(c, mrows);
  n->rows_cap = std::max(chunk, std::min((size_t)2 * SD * B, (size_t)1 << 26));
  n->rows_cap = std::max(n->rows_cap, (size_t)2 * SD);
  n->row_node = dalloc_t<int>(c, n->rows_cap);
  n->row_j = dalloc_t<int>(c, n->rows_cap);
  // valid indices everywhere from the start (slot 0, neuron 0)
  ck(cudaMemsetAsync(n->row_node, 0, n->rows_cap * sizeof(int), c->st), "memset");
  ck(cudaMemsetAsync(n->row_j, 0, n->rows_cap * sizeof(int), c->st), "memset");
  n->row_sign = dalloc_t<float>(c, n->rows_cap);
  n->counter = dalloc_t<int>(c, MNBAB_MAXR + 2);
  n->rb_nodes = dalloc_t<int>(c, (size_t)(MNBAB_MAXR + 2) * B);
  n->ri_dst = dalloc_t<int>(c, 2 * B);
  n->ri_src = dalloc_t<int>(c, 2 * B);
  n->ri_row = dalloc_t<int>(c, 2 * B);
  n->AP = dalloc_t<float>(c, B * SD);
  n->GA = dalloc_t<float>(c, B * SD);
  n->GB = dalloc_t<float>(c, B * SD);
  n->GP = dalloc_t<float>(c, B * SD);
  n->GPh = dalloc_t<float>(c, B * SD);
  n->Gz = dalloc_t<float>(c, B * SD);
  n->Hz = dalloc_t<float>(c, B * SD);
  n->X = dalloc_t<float>(c, mrows * n->d0);
  n->Xb = dalloc_t<float>(c, B * n->d0);
  n->GG = dalloc_t<float>(c, B * std::max<size_t>(EC, 1));
  n->gp0 = dalloc_t<float>(c, B);
  n->fout = dalloc_t<float>(c, B);
  n->score = dalloc_t<float>(c, B);
  n->bestb = dalloc_t<float>(c, B);
  n->gmax = dalloc_t<float>(c, B);
  n->f64a = dalloc_t<double>(c, B * (size_t)(n->d0 + n->SD));
  n->f64out = dalloc_t<double>(c, B);
  n->cslots = dalloc_t<int>(c, B);
  n->cand_idx = dalloc_t<int>(c, B);
  n->cand_count = dalloc_t<int>(c, 1);
  // split-K workspace: 16 splits of a B x (widest FC layer) product
  {
    size_t wmax = 0;
    for (int i = 1; i <= n->R + 1; ++i)
      for (int k = 0; k < n->nd.n_edge[i]; ++k) {
        const LayerDev& L = k == 0 ? n->nd.aff[i] : n->nd.aff2[i];
        if (L.kind == 1) wmax = std::max(wmax, (size_t)std::max(L.d_in, L.d_out));
      }
    if (wmax) {
      n->splitk_floats = 16 * B * wmax;
      n->splitk = dalloc_t<float>(c, n->splitk_floats);
    }
  }
  // tensor-core GEMM: one workspace for the split coefficient rows of every
  // FC product of up to mrows rows (launches on the stream run in order)
  {
    size_t ws = 0;
    for (int i = 1; i <= n->R + 1; ++i)
      for (int k = 0; k < n->nd.n_edge[i]; ++k) {
        const LayerDev& L = k == 0 ? n->nd.aff[i] : n->nd.aff2[i];
        if (L.kind == 1 && L.tc) ws = std::max(ws, tc_fc_workspace_floats(L, (int)mrows));
      }
    if (ws) {
      float* buf = dalloc_t<float>(c, ws);
      for (int i = 1; i <= n->R + 1; ++i)
        for (int k = 0; k < n->nd.n_edge[i]; ++k) {
          const LayerDev& L = k == 0 ? n->nd.aff[i] : n->nd.aff2[i];
          if (L.kind == 1 && L.tc)
            tc_fc_set_workspace(static_cast<TcFc*>(const_cast<void*>(L.tc)), buf, ws);
        }
    }
  }
  n->bslots = dalloc_t<int>(c, B);
  n->brows = dalloc_t<int>(c, B);
  n->acs_layer = dalloc_t<int>(c, B);
  n->acs_neuron = dalloc_t<int>(c, B);
  n->acs_fb = dalloc_t<int>(c, B);
  n->kid_parent = dalloc_t<int>(c, B);
  n->kid_slots = dalloc_t<int>(c, 2 * B);
  n->kid_layer = dalloc_t<int>(c, B);
  n->kid_neuron = dalloc_t<int>(c, B);
  if (EC) {
    ck(cudaMemsetAsync(P.GAM, 0, cap * EC * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.MG, 0, cap * EC * sizeof(float), c->st), "memset");
    ck(cudaMemsetAsync(P.VG, 0, cap * EC * sizeof(float), c->st), "memset");
  }
}

// Cost of a split in each ReLU layer for cost-adjusted branching (App. B):
// affine layers cost their weight entries (FC) or d_out k^2 (conv), a ReLU layer
// d + #constraints; C_t sums the layers below zhat_t; a split at layer k costs
// the re-bounding of every later layer (2 d_t C_t each) plus one objective row.
void update_cab(mnbab_net* n, mnbab_prop* p) {
  const int R = n->R;
  double C[MNBAB_MAXR + 2] = {0};
  double acc = 0.0;
  for (int t = 1; t <= R; ++t) {
    for (int k = 0; k < n->nd.n_edge[t]; ++k) {
      const HostLayer& L = n->hops[n->eop[t][k]];
      acc += L.kind == MNBAB_FC ? (double)L.ci * L.co : (double)L.co * L.ho * L.wo * L.k * L.k;
    }
    C[t] = acc;
    acc += (double)n->nd.d[t] + (double)p->pd.mnc[t].e;
  }
  const double c_obj = acc + (R >= 1 ? (double)n->nd.d[R] : 0.0);
  for (int k = 1; k <= R; ++k) {
    double cost = c_obj;
    for (int t = k + 1; t <= R; ++t) cost += 2.0 * n->nd.d[t] * C[t];
    p->pd.cab_inv[k] = (float)(1.0 / cost);
  }
}

// Adversarial pre-attack (Sec. 4): sign-step PGD on every property row from
// n_starts starting points; best_out[r] / x_out[r] the row's smallest FP32
// margin over all iterates and its first minimiser.
// Forward pass of the attack candidates (the batch's slots) from points x:
// every ReLU layer's pre-activations go to the candidate slot's bounds and the
// layer buffers hold the activations; the margins land in n->fout.
void attack_forward(mnbab_net* n, int M, const float* x) {
  mnbab_ctx* c = n->ctx;
  const NetDev& nd = n->nd;
  for (int t = 1; t <= n->R; ++t) {
    for (int k = 0; k < nd.n_edge[t]; ++k) {
      const int sidx = src_of(n, t, k);
      Epi e = base_epi(n, n->bslots);
      e.part = nullptr;
      e.kind = EPI_STORE;
      if (k > 0) {
        e.acc_in = lam_buf(n, t);
        e.acc_ld = nd.d[t];
      }
      const float* in = sidx == 0 ? x : lam_buf(n, sidx);
      const int ld_in = sidx == 0 ? n->d0 : nd.d[sidx];
      const LayerDev& L = edge_of(n, t, k);
      Scope sc(c, L.kind == 1 ? C_FWD_FC : (conv_tc_chosen(L, 0, e, M) ? C_FWD_CONV_TC : C_FWD_CONV),
               2.0 * M * layer_macs(L), 4.0 * M * (L.d_in + L.d_out) + layer_wbytes(L));
      launch_forward(L, M, in, ld_in, lam_buf(n, t), nd.d[t], e, c->st);
    }
    Scope sc(c, C_BOOK, 0.0, 12.0 * M * nd.d[t]);
    launch_pattern_relu(M, n->bslots, n->pool, nd.off[t], nd.d[t], lam_buf(n, t), c->st);
  }
  const int sR = nd.src1[n->R + 1];
  const int dR = nd.d[sR];
  const float* z = sR == 0 ? x : lam_buf(n, sR);
  Scope sc(c, C_BOOK, 2.0 * M * dR, 8.0 * M * dR);
  launch_final_dot(M, n->bslots, n->pool, c->d_props, z, sR == 0 ? n->d0 : dR, dR, n->fout, c->st);
}

// Autotuner: for every affine edge, direction and row bucket up to max_rows,
// each kernel variant that takes the layer runs once untimed and three times
// timed (CUDA events on the context's stream, the fastest counts) on the
// network's coefficient buffers filled with 0.5, with a plain store
// epilogue; the fastest variant becomes the layer's choice for that bucket
// (larger buckets take the largest one timed).
int64_t autotune_impl(mnbab_net* n, int max_rows, std::vector<mnbab_tune_rec>& recs) {
  mnbab_ctx* c = n->ctx;
  NetDev& nd = n->nd;
  const int top = std::max(1, std::min(max_rows, std::max(n->chunk, n->B)));
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0), "cudaEventCreate");
  ck(cudaEventCreate(&e1), "cudaEventCreate");
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  for (int t = 1; t <= n->R; ++t)
    for (int k = 0; k < nd.n_edge[t]; ++k) {
      LayerDev& L = k == 0 ? nd.aff[t] : nd.aff2[t];
      const int sidx = src_of(n, t, k);
      for (int dir = 1; dir >= 0; --dir) {
        int last = 0;
        for (int b = 0; b < 6; ++b) {
          if (b > 0 && TUNE_ROWS[b - 1] >= top) {
            L.tune[dir][b] = (signed char)last;
            continue;
          }
          const int M = std::min(TUNE_ROWS[b], top);
          float* in = dir == 1 ? lam_buf(n, t) : lam_buf(n, sidx);
          const int ld_in = dir == 1 ? nd.d[t] : nd.d[sidx];
          float* out = dir == 1 ? lam_buf(n, sidx) : lam_buf(n, t);
          const int ld_out = dir == 1 ? nd.d[sidx] : nd.d[t];
          launch_fill(in, (size_t)M * ld_in, 0.5f, c->st);
          Epi e = base_epi(n, n->bslots);
          e.part = nullptr;
          e.kind = EPI_STORE;
          e.slot_base = 0;
          e.sparse_rows = 0;
          e.gemm_path = 0;
          mnbab_tune_rec rec{};
          rec.node = t;
          rec.edge = k;
          rec.dir = dir;
          rec.rows = M;
          float best = INFINITY;
          int bv = 0;
          for (int v = 0; v < NVARIANT; ++v) rec.ms[v] = -1.f;
          for (int v = 1; v < NVARIANT; ++v) {
            if (launch_affine_variant(v, dir, L, M, in, ld_in, out, ld_out, e, c->st) < 0) continue;
            sync(c);
            float ms = INFINITY;
            for (int rep = 0; rep < 3; ++rep) {
              ck(cudaEventRecord(e0, c->st), "cudaEventRecord");
              launch_affine_variant(v, dir, L, M, in, ld_in, out, ld_out, e, c->st);
              ck(cudaEventRecord(e1, c->st), "cudaEventRecord");
              ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
              float x = 0.f;
              ck(cudaEventElapsedTime(&x, e0, e1), "cudaEventElapsedTime");
              ms = std::min(ms, x);
            }
            rec.ms[v] = ms;
            if (ms < best) {
              best = ms;
              bv = v;
            }
          }
          sync(c);  // raises the device error flag of the bounded waits, if set
          rec.variant = bv;
          L.tune[dir][b] = (signed char)bv;
          last = bv;
          recs.push_back(rec);
        }
      }
    }
  return (int64_t)recs.size();
}

// Candidate slots of one chunk, released on every exit.
struct AttackSlots {
  mnbab_net* n;
  std::vector<int> s;
  ~AttackSlots() {
    for (int x : s) free_slot(n, x);
  }
};

// The pre-attack in the per-layer form, for any network the library loads:
// candidate q = r n_starts + s (row r, start s) is a scratch node slot; per
// iterate the forward kernels of the bounding path give the margin and write
// the pre-activations into the slot's bounds (l = u = zhat), and the DeepPoly
// back-substitution of the objective row through that slot (ReLU' = 1 where
// zhat >= 0, no splits or parameters) is the margin's gradient at the input.
// Candidates run in chunks of the batch capacity.  f64_out (nullable) gets
// each row's chosen point's margin in FP64 (device forward pass).
void attack_layers(mnbab_ctx* c, const mnbab_prop* p, int n_starts, int steps, const float* starts,
                   float* best_out, float* x_out, std::vector<double>* f64_out) {
  mnbab_net* n = p->net;
  const int nr = p->n_rows, d0 = n->d0, Q = nr * n_starts;
  const int Qc = std::min({Q, n->B, n->chunk, (int)n->free_slots.size()});
  if (Qc < 1) fail(MNBAB_E_BUDGET, "node pool exhausted");
  const size_t need = (size_t)n_starts * d0 + (size_t)Qc * (2 * (size_t)d0 + 1);
  if (n->atk_cap < need) {
    n->atk = dalloc_t<float>(c, need);
    n->atk_cap = need;
  }
  float* dst = n->atk;
  float* dX = dst + (size_t)n_starts * d0;
  float* dBx = dX + (size_t)Qc * d0;
  float* dBest = dBx + (size_t)Qc * d0;
  h2d(c, dst, starts, (size_t)n_starts * d0);
  std::vector<float> hb(Q), hx((size_t)Q * d0);
  for (int q0 = 0; q0 < Q; q0 += Qc) {
    const int M = std::min(Qc, Q - q0);
    AttackSlots sl{n, {}};
    for (int m = 0; m < M; ++m) {
      const int s = alloc_slot(n);
      sl.s.push_back(s);
      n->slot_prop[s] = p->index;
      n->slot_row[s] = (q0 + m) / n_starts;
    }
    upload_batch(n, sl.s);
    {
      Scope sc(c, C_BOOK, 0.0, 20.0 * M * n->SD);
      launch_attack_init(M, q0, n_starts, n->bslots, n->pool, p->index, c->d_props, dst, dX, dBest,
                         c->st);
    }
    for (int k = 0; k <= steps; ++k) {
      attack_forward(n, M, dX);
      {
        Scope sc(c, C_BOOK, 0.0, 8.0 * M * d0);
        launch_attack_best(M, n->fout, dX, d0, dBest, dBx, c->st);
      }
      if (k == steps) break;
      SweepOpts o;
      o.keep_a0 = true;
      sweep(n, n->R + 1, obj_rows(n, M), o);
      Scope sc(c, C_BOOK, 0.0, 12.0 * M * d0);
      launch_attack_step(M, lam_buf(n, 0), d0, dX, d0, c->d_props, p->index, steps, c->st);
    }
    d2h(c, hb.data() + q0, dBest, M);
    d2h(c, hx.data() + (size_t)q0 * d0, dBx, (size_t)M * d0);
    sync(c);
  }
  std::vector<float> xr((size_t)nr * d0);
  for (int r = 0; r < nr; ++r) {
    int bs = 0;
    for (int s0 = 1; s0 < n_starts; ++s0)
      if (hb[(size_t)r * n_starts + s0] < hb[(size_t)r * n_starts + bs]) bs = s0;  // first on ties
    best_out[r] = hb[(size_t)r * n_starts + bs];
    std::memcpy(xr.data() + (size_t)r * d0, hx.data() + ((size_t)r * n_starts + bs) * d0,
                (size_t)d0 * sizeof(float));
  }
  if (x_out) std::memcpy(x_out, xr.data(), xr.size() * sizeof(float));
  if (!f64_out) return;
  // FP64 margins of the chosen points (row r's point in a slot of row r)
  f64_out->assign(nr, 0.0);
  const int Rc = std::min({nr, n->B, (int)n->free_slots.size()});
  if (Rc < 1) fail(MNBAB_E_BUDGET, "node pool exhausted");
  for (int r0 = 0; r0 < nr; r0 += Rc) {
    const int M = std::min(Rc, nr - r0);
    AttackSlots sl{n, {}};
    for (int m = 0; m < M; ++m) {
      const int s = alloc_slot(n);
      sl.s.push_back(s);
      n->slot_prop[s] = p->index;
      n->slot_row[s] = r0 + m;
    }
    upload_batch(n, sl.s);
    launch_attack_init(M, r0, 1, n->bslots, n->pool, p->index, c->d_props, nullptr, nullptr,
                       nullptr, c->st);
    h2d(c, n->Xb, xr.data() + (size_t)r0 * d0, (size_t)M * d0);
    {
      Scope sc(c, C_BOOK, 2.0 * M * n->SD, 8.0 * M * (d0 + n->SD));
      launch_forward_f64(M, n->bslots, n->pool, c->d_props, n->nd, n->Xb, d0, n->f64a,
                         d0 + n->SD, n->f64out, c->st);
    }
    d2h(c, f64_out->data() + r0, n->f64out, M);
    sync(c);
  }
}

void attack_impl(mnbab_ctx* c, const mnbab_prop* p, int n_starts, int steps, const float* starts,
                 float* best_out, float* x_out, std::vector<double>* f64_out = nullptr) {
  mnbab_net* n = p->net;
  const bool fused = attack_supported(n->nd);
  if (c->attack_path == 1 && !fused)
    fail(MNBAB_E_UNSUPPORTED, "the one-kernel attack takes chain networks whose weights fit in "
                              "shared memory");
  if (c->attack_path == 2 || !fused) {
    attack_layers(c, p, n_starts, steps, starts, best_out, x_out, f64_out);
    return;
  }
  const int nr = p->n_rows, d0 = n->d0, nb = nr * n_starts;
  const size_t need = (size_t)n_starts * d0 + nb + (size_t)nb * d0;
  if (n->atk_cap < need) {
    n->atk = dalloc_t<float>(c, need);
    n->atk_cap = need;
  }
  float* dst = n->atk;
  float* dbest = dst + (size_t)n_starts * d0;
  float* dbx = dbest + nb;
  h2d(c, dst, starts, (size_t)n_starts * d0);
  {
    Scope sc(c, C_BOOK, 0.0, 4.0 * nb * d0);
    launch_attack_chain(n->nd, c->d_props, p->index, nr, dst, n_starts, steps, dbest, dbx, c->st);
  }
  std::vector<float> hb(nb), hx;
  d2h(c, hb.data(), dbest, nb);
  if (x_out) {
    hx.resize((size_t)nb * d0);
    d2h(c, hx.data(), dbx, hx.size());
  }
  sync(c);
  for (int r = 0; r < nr; ++r) {
    int bs = 0;
    for (int s0 = 1; s0 < n_starts; ++s0)
      if (hb[(size_t)r * n_starts + s0] < hb[(size_t)r * n_starts + bs]) bs = s0;  // first on ties
    best_out[r] = hb[(size_t)r * n_starts + bs];
    if (x_out)
      std::memcpy(x_out + (size_t)r * d0, hx.data() + ((size_t)r * n_starts + bs) * d0,
                  (size_t)d0 * sizeof(float));
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): the output at state
// seed + index * 0x9E3779B97F4A7C15, top 53 bits as a uniform in [0, 1)
double splitmix_uniform(uint64_t seed, uint64_t index) {
  uint64_t z = seed + (index + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// f_r(x) of a chain network in FP64 on the host (counterexample confirmation
// of the pre-attack): the affine layers of hops, ReLUs, the folded last layer.
double host_margin(const mnbab_net* n, const mnbab_prop* p, int row, const float* x) {
  std::vector<double> z(x, x + n->d0), h;
  for (int t = 1; t <= n->R; ++t) {
    const HostLayer& L = n->hops[n->eop[t][0]];
    if (L.kind == MNBAB_FC) {
      h.assign(L.co, 0.0);
      for (int o = 0; o < L.co; ++o) {
        double a = L.b[o];
        for (int i = 0; i < L.ci; ++i) a += L.W[(size_t)o * L.ci + i] * z[i];
        h[o] = a;
      }
    } else {
      h.assign((size_t)L.co * L.ho * L.wo, 0.0);
      for (int co = 0; co < L.co; ++co)
        for (int oy = 0; oy < L.ho; ++oy)
          for (int ox = 0; ox < L.wo; ++ox) {
            double a = L.b[co];
            for (int ci = 0; ci < L.ci; ++ci)
              for (int ky = 0; ky < L.k; ++ky)
                for (int kx = 0; kx < L.k; ++kx) {
                  const int iy = oy * L.s - L.p + ky, ix = ox * L.s - L.p + kx;
                  if (iy < 0 || iy >= L.hi || ix < 0 || ix >= L.wi) continue;
                  a += L.W[(((size_t)co * L.ci + ci) * L.k + ky) * L.k + kx] *
                       z[((size_t)ci * L.hi + iy) * L.wi + ix];
                }
            h[((size_t)co * L.ho + oy) * L.wo + ox] = a;
          }
    }
    for (double& v : h) v = v > 0.0 ? v : 0.0;
    z.swap(h);
  }
  const int dR = (int)z.size();
  double f = p->bf[row];
  for (int i = 0; i < dR; ++i) f += p->Wf[(size_t)row * dR + i] * z[i];
  return f;
}

// The pre-attack of a property that starts (Sec. 4: counterexamples are
// searched before branch-and-bound): the box centre and atk_starts - 1
// SplitMix64 points, atk_steps sign steps; a row whose minimiser has a
// negative FP64 margin falsifies the property before any node is bounded.
bool pre_attack(mnbab_ctx* c, mnbab_prop* p) {
  mnbab_net* n = p->net;
  const int d0 = n->d0, ns = p->atk_starts;
  std::vector<float> st((size_t)ns * d0), best(p->n_rows), x((size_t)p->n_rows * d0);
  for (int j = 0; j < d0; ++j) st[j] = (float)(0.5 * ((double)p->lo[j] + (double)p->hi[j]));
  for (int k = 1; k < ns; ++k)
    for (int j = 0; j < d0; ++j) {
      const double u = splitmix_uniform(p->atk_seed, (uint64_t)(k - 1) * d0 + j);
      st[(size_t)k * d0 + j] = (float)((double)p->lo[j] + ((double)p->hi[j] - p->lo[j]) * u);
    }
  const bool fused = c->attack_path != 2 && attack_supported(n->nd);
  std::vector<double> f64;
  attack_impl(c, p, ns, p->atk_steps, st.data(), best.data(), x.data(), fused ? nullptr : &f64);
  for (int r = 0; r < p->n_rows; ++r)
    if (best[r] < 0.f &&
        (fused ? host_margin(n, p, r, x.data() + (size_t)r * d0) : f64[r]) < 0.0) {
      p->verdict = MNBAB_FALSIFIED;
      p->done = true;
      p->cex.assign(x.begin() + (size_t)r * d0, x.begin() + (size_t)(r + 1) * d0);
      p->cex_row = r;
      p->row_fals[r] = 1;
      return true;
    }
  return false;
}

// Root bounds of every property of the network admitted since the last call,
// computed together in one re-bounding pass, then their row root nodes.
// Node slots of a property: the root-bound slot (l = -inf, u = +inf, re-bounded
// from layer 1 with the next batch of admissions) and one root node per row.
void materialize(mnbab_net* n, mnbab_prop* p) {
  mnbab_ctx* c = n->ctx;
  if (p->atk_starts > 0 && pre_attack(c, p)) {
    p->materialized = true;  // falsified before any node: nothing to bound
    return;
  }
  if ((int)n->free_slots.size() < p->n_rows + 1) fail(MNBAB_E_BUDGET, "node pool exhausted");
  const int rs = alloc_slot(n);
  p->root_slot = rs;
  n->slot_prop[rs] = p->index;
  n->slot_row[rs] = 0;
  n->slot_split[rs] = 0;
  // slot state (l = -inf, u = +inf, no splits, property index) is set for all
  // properties started together, in one launch (ensure_roots)
  n->new_roots.push_back(rs);
  n->new_root_props.push_back(p->index);
  for (int r = 0; r < p->n_rows; ++r) {
    const int sl = alloc_slot(n);
    n->slot_prop[sl] = p->index;
    n->slot_row[sl] = r;
    n->slot_split[sl] = n->R;
    p->root_row_slots.push_back(sl);
    p->queue.push_back(QNode{sl, p->next_seq++, r, 0, n->R});
    p->row_open[r]++;
  }
  p->root_pending = true;
  p->materialized = true;
}

// Optimised intermediate bounds (Sec. 3.1, parameter sharing).  For ReLU
// layers t = max(2, first_layer) .. R in order, the unstable unsplit neurons
// of t of every node give rows +e_j (lower bounds) and -e_j (upper bounds).
// Each (node, side) has one (alpha, beta) set over the layers below t, held in
// a scratch slot and shared by its rows.  A step bounds the rows (one sweep
// per chunk of rows), sums the rows' gradients per set and takes one projected
// Adam step per set; every row keeps its best bound, and the nodes' bounds of
// layer t are intersected with them before layer t + 1 is bounded.
int64_t optimize_intermediate_impl(mnbab_net* n, const std::vector<int>& slots, int first_layer,
                                   const mnbab_adam& a) {
  mnbab_ctx* c = n->ctx;
  const int nn = (int)slots.size();
  const int SD = n->SD, R = n->R;
  if (!n->iga) {
    // rows per sweep and adjoint: the batch capacity, or more where the
    // call's own per-row buffers fit in about 1 GB (an eighth of the free
    // budget at most); fewer, longer chunks mean fewer launches per step
    const size_t room = std::min<size_t>(1ull << 30, (c->budget - c->used) / 8);
    const size_t fit = std::min(room / (12 * (size_t)SD), (size_t)n->chunk);
    n->icap = n->B;
    if (fit > (size_t)n->B) {
      n->icap = (int)fit;
      n->iap = dalloc_t<float>(c, fit * SD);
      n->igar = dalloc_t<float>(c, fit * SD);
      n->igbr = dalloc_t<float>(c, fit * SD);
    }
    n->iga = dalloc_t<float>(c, (size_t)n->B * SD);
    n->igb = dalloc_t<float>(c, (size_t)n->B * SD);
    n->ibest = dalloc_t<float>(c, n->rows_cap);
    n->iorig = dalloc_t<int>(c, n->rows_cap);
    n->isrc = dalloc_t<int>(c, n->B);
    n->idst = dalloc_t<int>(c, n->B);
    n->iseg_cap = 3 * ((size_t)n->B + n->rows_cap / std::min(n->icap, n->chunk) + 2);
    n->iseg = dalloc_t<int>(c, n->iseg_cap);
  }
  // properties with multi-neuron constraints: the sets hold gamma as well, and
  // the rows' gamma projections and gradients use the batch buffers
  bool has_g = false;
  for (int s0 : slots) has_g = has_g || c->props[n->slot_prop[s0]]->pd.E > 0;
  if (has_g && !n->igg) n->igg = dalloc_t<float>(c, (size_t)n->B * c->EC);
  const int CH = has_g ? std::max(1, std::min(n->B, n->chunk))
                       : std::max(1, std::min(n->icap, n->chunk));
  // the sweeps and adjoints of this call use the per-row buffers above (and
  // read each row's slot from bslots); restored on every exit
  struct Swap {
    mnbab_net* n;
    float *ap, *ga, *gb;
    int* bs;
    ~Swap() {
      n->AP = ap;
      n->GA = ga;
      n->GB = gb;
      n->bslots = bs;
    }
  } swap{n, n->AP, n->GA, n->GB, n->bslots};
  if (n->iap && !has_g) {
    n->AP = n->iap;
    n->GA = n->igar;
    n->GB = n->igbr;
  }
  struct Scratch {
    mnbab_net* n;
    std::vector<int> slots;
    ~Scratch() {
      for (int s : slots) free_slot(n, s);
    }
  } tmp{n, {}};
  int64_t total = 0;
  std::vector<float> hl, hu;
  std::vector<int8_t> hs;
  for (int t = std::max(2, (int)first_layer); t <= R; ++t) {
    const int dt = n->nd.d[t], off = n->nd.off[t];
    hl.resize((size_t)nn * dt);
    hu.resize((size_t)nn * dt);
    hs.resize((size_t)nn * dt);
    for (int k = 0; k < nn; ++k) {
      const size_t q = (size_t)slots[k] * SD + off;
      d2h(c, hl.data() + (size_t)k * dt, n->pool.L + q, dt);
      d2h(c, hu.data() + (size_t)k * dt, n->pool.U + q, dt);
      d2h(c, hs.data() + (size_t)k * dt, n->pool.S + q, dt);
    }
    sync(c);
    // rows grouped by set: a node's lower rows, then its upper rows
    std::vector<int> rnode, rj, rorig, src, dst, set_lo, set_hi;
    std::vector<float> rsign;
    for (int k = 0; k < nn; ++k) {
      std::vector<int> idx;
      for (int j = 0; j < dt; ++j) {
        const size_t q = (size_t)k * dt + j;
        if (hl[q] < 0.f && hu[q] > 0.f && hs[q] == 0) idx.push_back(j);
      }
      if (idx.empty()) continue;
      for (int side = 0; side < 2; ++side) {
        const int ts = alloc_slot(n);
        tmp.slots.push_back(ts);
        n->slot_prop[ts] = n->slot_prop[slots[k]];
        n->slot_row[ts] = n->slot_row[slots[k]];
        n->slot_split[ts] = R;
        src.push_back(slots[k]);
        dst.push_back(ts);
        set_lo.push_back((int)rnode.size());
        for (int j : idx) {
          rnode.push_back(ts);
          rj.push_back(j);
          rsign.push_back(side == 0 ? 1.f : -1.f);
          rorig.push_back(slots[k]);
        }
        set_hi.push_back((int)rnode.size());
      }
    }
    const int M = (int)rnode.size(), nsets = (int)dst.size();
    if (M == 0) continue;
    if ((size_t)M > n->rows_cap)
      fail(MNBAB_E_BUDGET, "layer " + std::to_string(t) + " needs " + std::to_string(M) +
                               " intermediate-bound rows, more than the " +
                               std::to_string(n->rows_cap) +
                               "-row scratch of this network; pass fewer nodes per call");
    // per chunk of rows, the segments of its sets: (set, first row, end row)
    std::vector<int> seg, seg_at;
    for (int c0 = 0; c0 < M; c0 += CH) {
      const int c1 = std::min(M, c0 + CH);
      seg_at.push_back((int)seg.size() / 3);
      for (int st = 0; st < nsets; ++st) {
        const int lo = std::max(set_lo[st], c0), hi = std::min(set_hi[st], c1);
        if (lo < hi) seg.insert(seg.end(), {st, lo - c0, hi - c0});
      }
    }
    seg_at.push_back((int)seg.size() / 3);
    if (seg.size() > n->iseg_cap) fail(MNBAB_E_DEVICE, "segment scratch too small");
    h2d(c, n->row_node, rnode.data(), M);
    h2d(c, n->row_j, rj.data(), M);
    h2d(c, n->row_sign, rsign.data(), M);
    h2d(c, n->iorig, rorig.data(), M);
    h2d(c, n->isrc, src.data(), nsets);
    h2d(c, n->idst, dst.data(), nsets);
    h2d(c, n->iseg, seg.data(), seg.size());
    {
      Scope sc(c, C_BOOK, 0.0, 36.0 * nsets * SD);
      launch_set_init(nsets, n->isrc, n->idst, n->pool, c->st);
    }
    SweepOpts o;
    o.final_mode = true;
    o.has_gamma = has_g;
    double b1t = 1.0, b2t = 1.0;
    for (int step = 0; step <= a.steps; ++step) {
      const bool grad = step < a.steps;
      o.store = grad;
      if (grad) {
        ck(cudaMemsetAsync(n->iga, 0, (size_t)nsets * SD * sizeof(float), c->st), "memset");
        ck(cudaMemsetAsync(n->igb, 0, (size_t)nsets * SD * sizeof(float), c->st), "memset");
        if (has_g)
          ck(cudaMemsetAsync(n->igg, 0, (size_t)nsets * c->EC * sizeof(float), c->st), "memset");
      }
      for (int ci = 0, c0 = 0; c0 < M; ++ci, c0 += CH) {
        const int Mc = std::min(CH, M - c0);
        RowsDev r{Mc, n->row_node + c0, n->row_j + c0, n->row_sign + c0};
        if (has_g) {
          // gamma^T P, gamma^T Phat, gamma^T p of each row's set
          Scope sc(c, C_GAMMA, 0.0, 4.0 * Mc * (c->EC + 2.0 * n->SD), 2);
          launch_gamma_proj(Mc, r.node, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
        }
        sweep(n, t, r, o);
        {
          Scope sc(c, C_BOOK, 0.0, 12.0 * Mc);
          launch_rows_best(Mc, n->lb, n->ibest + c0, step == 0, c->st);
        }
        if (!grad) continue;
        // the adjoint reads each row's slot from bslots: point it at the chunk's rows
        n->bslots = n->row_node + c0;
        adjoint(n, Mc, has_g, t - 1);
        const int ns = seg_at[ci + 1] - seg_at[ci];
        Scope sc(c, C_ADAM, 0.0, 8.0 * (double)Mc * off + 16.0 * ns * off);
        launch_set_grad(ns, n->iseg + 3 * seg_at[ci], SD, off, n->GA, n->GB, n->iga, n->igb,
                        c->st);
        if (has_g)
          launch_set_grad_gamma(ns, n->iseg + 3 * seg_at[ci], n->idst, n->pool, c->d_props, t,
                                n->GG, n->igg, c->st);
      }
      if (!grad) break;
      b1t *= a.beta1;
      b2t *= a.beta2;
      Scope sc(c, C_ADAM, 0.0, 4.0 * nsets * 2.0 * SD * 8.0, 2);
      launch_adam(nsets, n->idst, n->pool, c->d_props, SD, n->iga, n->igb,
                  has_g ? n->igg : n->GG, n->gmax,
                  a.grad_floor, a.lr_alpha, a.lr_beta, a.lr_gamma, a.beta1, a.beta2, a.eps,
                  a.eps_rel, (float)(1.0 - b1t), (float)(1.0 - b2t), c->st);
    }
    {
      Scope sc(c, C_BOOK, 0.0, 20.0 * M);
      launch_set_update(M, n->iorig, n->row_j, n->row_sign, n->ibest, n->pool, off, c->st);
    }
    sync(c);
    for (int s : tmp.slots) free_slot(n, s);
    tmp.slots.clear();
    total += M;
  }
  sync(c);
  return total;
}

// Starts the given properties (all admitted properties of the network when
// `only` is null) and bounds every root still pending, in shared launches.
void ensure_roots(mnbab_net* n, mnbab_prop* const* only = nullptr, int n_only = 0) {
  mnbab_ctx* c = n->ctx;
  if (only) {
    for (int i = 0; i < n_only; ++i)
      if (only[i]->admitted && !only[i]->materialized) materialize(n, only[i]);
  } else {
    for (auto* p : c->props)
      if (p->net == n && p->admitted && !p->materialized) materialize(n, p);
  }
  for (size_t b0 = 0; b0 < n->new_roots.size(); b0 += 2 * (size_t)n->B) {
    const int nb = (int)std::min(n->new_roots.size() - b0, 2 * (size_t)n->B);
    h2d(c, n->ri_dst, n->new_roots.data() + b0, nb);
    h2d(c, n->ri_src, n->new_root_props.data() + b0, nb);
    Scope sc(c, C_BOOK, 0.0, 9.0 * nb * n->SD);
    launch_root_slot_init(nb, n->ri_dst, n->ri_src, n->pool, c->st);
  }
  n->new_roots.clear();
  n->new_root_props.clear();
  std::vector<mnbab_prop*> pend;
  for (auto* p : c->props)
    if (p->net == n && p->root_pending) pend.push_back(p);
  if (pend.empty()) return;
  std::vector<int> roots;
  for (auto* p : pend) roots.push_back(p->root_slot);
  rebound(n, roots, true);
  // optimised intermediate bounds of the roots that ask for them (Sec. 3.1,
  // parameter sharing), before the root nodes take the root bounds
  std::vector<std::pair<int, int>> want;  // (steps, root slot)
  for (auto* p : pend)
    if (p->inter_steps > 0) want.push_back({p->inter_steps, p->root_slot});
  std::sort(want.begin(), want.end());
  for (size_t i = 0; i < want.size();) {
    std::vector<int> grp;
    const int steps = want[i].first;
    // two parameter sets (lower, upper) per root; at least one root per group
    // so that the loop always advances (set_intermediate_steps refuses B < 2)
    while (i < want.size() && want[i].first == steps &&
           (grp.empty() || 2 * ((int)grp.size() + 1) <= n->B))
      grp.push_back(want[i++].second);
    mnbab_adam a = default_adam();
    a.steps = steps;
    optimize_intermediate_impl(n, grp, 2, a);
  }
  std::vector<int> dst, src, row;
  auto flush = [&]() {
    if (dst.empty()) return;
    h2d(c, n->ri_dst, dst.data(), dst.size());
    h2d(c, n->ri_src, src.data(), src.size());
    h2d(c, n->ri_row, row.data(), row.size());
    Scope sc(c, C_BOOK, 0.0, 25.0 * dst.size() * n->SD);
    launch_root_init((int)dst.size(), n->ri_dst, n->ri_src, n->ri_row, n->pool, c->st);
    // the index vectors were staged when they were enqueued: they can be reused
    dst.clear(); src.clear(); row.clear();
  };
  for (auto* p : pend) {
    for (size_t r = 0; r < p->root_row_slots.size(); ++r) {
      if ((int)dst.size() == 2 * n->B) flush();
      dst.push_back(p->root_row_slots[r]);
      src.push_back(p->root_slot);
      row.push_back((int)r);
    }
    p->root_pending = false;
    p->root_row_slots.clear();
  }
  flush();
}

// Uploads the constraint rows of one ReLU layer of a property (row form and
// CSR by neuron) and appends them to the property's gamma entries.
void set_mnc_impl(mnbab_ctx* c, mnbab_prop* p, int layer, int n_rows, int k, const int32_t* idx,
                  const float* P, const float* Phat, const float* pv) {
  if (p->mnc_set[layer]) fail(MNBAB_E_INVALID_ARG, "constraints of this layer already set");
  mnbab_net* n = p->net;
  const int d = n->nd.d[layer];
  if (p->pd.E + n_rows > c->EC)
    fail(MNBAB_E_BUDGET, "more constraint rows than mnbab_options.max_mnc_rows");
  for (int64_t q = 0; q < (int64_t)n_rows * k; ++q)
    if (idx[q] < 0 || idx[q] >= d) fail(MNBAB_E_INVALID_ARG, "constraint neuron index out of range");
  MncDev& m = p->pd.mnc[layer];
  m.e = n_rows;
  m.k = k;
  m.goff = p->pd.E;
  if (n_rows > 0) {
    const size_t nk = (size_t)n_rows * k;
    // CSR by neuron
    std::vector<int> cnt(d + 1, 0);
    for (size_t q = 0; q < nk; ++q) cnt[idx[q] + 1]++;
    for (int j = 0; j < d; ++j) cnt[j + 1] += cnt[j];
    std::vector<int> ce(nk), pos(cnt.begin(), cnt.end() - 1);
    std::vector<float> cP(nk), cPh(nk);
    for (int e = 0; e < n_rows; ++e)
      for (int kk = 0; kk < k; ++kk) {
        const size_t q = (size_t)e * k + kk;
        const int at = pos[idx[q]]++;
        ce[at] = e;
        cP[at] = P[q];
        cPh[at] = Phat[q];
      }
    int* didx = dalloc_t<int>(c, nk);
    float* dP = dalloc_t<float>(c, nk);
    float* dPh = dalloc_t<float>(c, nk);
    float* dp = dalloc_t<float>(c, n_rows);
    int* dcptr = dalloc_t<int>(c, d + 1);
    int* dce = dalloc_t<int>(c, nk);
    float* dcP = dalloc_t<float>(c, nk);
    float* dcPh = dalloc_t<float>(c, nk);
    h2d(c, didx, idx, nk);
    h2d(c, dP, P, nk);
    h2d(c, dPh, Phat, nk);
    h2d(c, dp, pv, n_rows);
    h2d(c, dcptr, cnt.data(), d + 1);
    h2d(c, dce, ce.data(), nk);
    h2d(c, dcP, cP.data(), nk);
    h2d(c, dcPh, cPh.data(), nk);
    m.idx = didx; m.P = dP; m.Ph = dPh; m.p = dp;
    m.cptr = dcptr; m.ce = dce; m.cP = dcP; m.cPh = dcPh;
  }
  p->pd.E += n_rows;
  p->mnc_set[layer] = 1;
  update_cab(n, p);
  upload_prop(c, p->index);
  sync(c);
}

// Multi-neuron constraints of every ReLU layer of a property from its root
// bounds: groups of three unstable neurons (sliding triples in the order of
// decreasing -l u / (u - l), ties by index, at most max_groups per layer), the
// DeepPoly lower bounds of the 26 octahedral directions of each group (one
// combination row each, back-substituted on the device with the root's
// DeepPoly relaxation of the layers below), then each group's rows from the
// hull of the lifted ReLU graph on the host (csrc/mnc_hull.cu, in parallel).
int64_t generate_mnc_impl(mnbab_ctx* c, mnbab_prop* p, int max_groups) {
  mnbab_net* n = p->net;
  for (int t = 1; t <= n->R; ++t)
    if (p->mnc_set[t]) fail(MNBAB_E_INVALID_ARG, "constraints of a layer are already set");
  mnbab_prop* only[1] = {p};
  ensure_roots(n, only, 1);
  if (!p->materialized) fail(MNBAB_E_INVALID_ARG, "property not admitted");
  if (p->root_slot < 0) {
    // decided when it started (its pre-attack found a counterexample): no node
    // will be bounded, so no constraints are needed
    for (int t = 1; t <= n->R; ++t) p->mnc_set[t] = 1;
    return 0;
  }
  const int SD = n->SD, rs = p->root_slot;
  std::vector<float> hl(SD), hu(SD);
  d2h(c, hl.data(), n->pool.L + (size_t)rs * SD, SD);
  d2h(c, hu.data(), n->pool.U + (size_t)rs * SD, SD);
  sync(c);
  static const int kDir[26][3] = {
      {-1, -1, -1}, {-1, -1, 0}, {-1, -1, 1}, {-1, 0, -1}, {-1, 0, 0}, {-1, 0, 1}, {-1, 1, -1},
      {-1, 1, 0},   {-1, 1, 1},  {0, -1, -1}, {0, -1, 0},  {0, -1, 1}, {0, 0, -1}, {0, 0, 1},
      {0, 1, -1},   {0, 1, 0},   {0, 1, 1},   {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1},
      {1, 0, 0},    {1, 0, 1},   {1, 1, -1},  {1, 1, 0},   {1, 1, 1}};
  const int chunk_groups = std::max(1, n->chunk / 26);  // rows per sweep <= the row chunk
  if (!n->gen_cidx) {
    n->gen_cap = chunk_groups * 26;
    n->gen_cidx = dalloc_t<int>(c, 3 * (size_t)n->gen_cap);
    n->gen_coef = dalloc_t<float>(c, 3 * (size_t)n->gen_cap);
  }
  int64_t total = 0;
  for (int t = 1; t <= n->R; ++t) {
    const int dt = n->nd.d[t], off = n->nd.off[t];
    std::vector<int> unst;
    for (int j = 0; j < dt; ++j)
      if (hl[off + j] < 0.f && hu[off + j] > 0.f) unst.push_back(j);
    const int ng = unst.size() >= 3 ? std::min((int)unst.size() - 2, max_groups) : 0;
    if (ng == 0) {
      set_mnc_impl(c, p, t, 0, 3, nullptr, nullptr, nullptr, nullptr);
      continue;
    }
    std::vector<double> key(dt, 0.0);
    for (int j : unst) {
      const double l = hl[off + j], u = hu[off + j];
      key[j] = -l * u / (u - l);
    }
    std::stable_sort(unst.begin(), unst.end(), [&](int a, int b) {
      return key[a] != key[b] ? key[a] > key[b] : a < b;
    });
    // octahedral bounds: 26 combination rows per group, in chunks
    std::vector<double> oct((size_t)ng * 26);
    std::vector<int> cidx, rnode;
    std::vector<float> coef;
    std::vector<float> lb;
    for (int g0 = 0; g0 < ng; g0 += chunk_groups) {
      const int gn = std::min(chunk_groups, ng - g0), Mc = gn * 26;
      cidx.resize(3 * (size_t)Mc);
      coef.resize(3 * (size_t)Mc);
      rnode.assign(Mc, rs);
      for (int g = 0; g < gn; ++g)
        for (int di = 0; di < 26; ++di)
          for (int k = 0; k < 3; ++k) {
            const size_t q = 3 * ((size_t)g * 26 + di) + k;
            cidx[q] = unst[g0 + g + k];
            coef[q] = (float)kDir[di][k];
          }
      h2d(c, n->gen_cidx, cidx.data(), cidx.size());
      h2d(c, n->gen_coef, coef.data(), coef.size());
      h2d(c, n->row_node, rnode.data(), rnode.size());
      RowsDev r{Mc, n->row_node, nullptr, nullptr, n->gen_cidx, n->gen_coef};
      SweepOpts so;
      sweep(n, t, r, so);
      lb.resize(Mc);
      d2h(c, lb.data(), n->lb, Mc);
      sync(c);
      for (int q = 0; q < Mc; ++q) oct[(size_t)g0 * 26 + q] = lb[q];
    }
    // hulls on the host, groups spread over the host threads
    std::vector<std::vector<MncRow>> rows(ng);
    const int nth = std::max(1, std::min(ng, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w)
      pool.emplace_back([&, w]() {
        for (int g = w; g < ng; g += nth) mnc_group_rows(oct.data() + (size_t)g * 26, rows[g]);
      });
    for (auto& th : pool) th.join();
    std::vector<int32_t> idx;
    std::vector<float> P, Ph, pv;
    for (int g = 0; g < ng; ++g)
      for (const MncRow& r : rows[g]) {
        for (int k = 0; k < 3; ++k) {
          idx.push_back(unst[g + k]);
          P.push_back((float)r.P[k]);
          Ph.push_back((float)r.Ph[k]);
        }
        pv.push_back((float)r.p);
      }
    const int nr = (int)pv.size();
    set_mnc_impl(c, p, t, nr, 3, idx.data(), P.data(), Ph.data(), pv.data());
    total += nr;
  }
  return total;
}

// ---------------------------------------------------------------------------
// BaB step (Sec. 2.2; Sec. 3.2)
// ---------------------------------------------------------------------------
struct Picked {
  mnbab_prop* p;
  QNode q;
};

void bab_step_impl(mnbab_ctx* c, mnbab_prop* const* props, int n_props, int max_nodes,
                   const mnbab_adam& adam, mnbab_step_stats* st) {
  std::memset(st, 0, sizeof(*st));
  if (n_props <= 0) return;
  const int64_t h2d0 = c->h2d_bytes, d2h0 = c->d2h_bytes;
  struct Fin {
    mnbab_ctx* c; mnbab_step_stats* st; int64_t a, b;
    ~Fin() { st->h2d_bytes = c->h2d_bytes - a; st->d2h_bytes = c->d2h_bytes - b; }
  } fin{c, st, h2d0, d2h0};
  mnbab_net* n = props[0]->net;
  for (int i = 0; i < n_props; ++i)
    if (props[i]->net != n) fail(MNBAB_E_INVALID_ARG, "properties of different networks");
  max_nodes = std::max(1, std::min(max_nodes, n->B));
  HostTimer ht(c);
  ensure_roots(n, props, n_props);
  ht.lap(H_ROOTS);
  {
    const double t = now_s();
    for (int i = 0; i < n_props; ++i)
      if (props[i]->materialized && props[i]->t_start == 0.0) props[i]->t_start = t;
  }
  // pop FIFO
  std::vector<Picked> picked;
  for (int i = 0; i < n_props && (int)picked.size() < max_nodes; ++i) {
    mnbab_prop* p = props[i];
    if (!p->materialized) continue;
    while (!p->done && !p->queue.empty() && p->bounded < p->budget &&
           (int)picked.size() < max_nodes) {
      picked.push_back({p, p->queue.front()});
      p->queue.pop_front();
      p->bounded++;
      p->row_open[picked.back().q.row]--;
    }
  }
  const int M = (int)picked.size();
  st->nodes_bounded = M;
  if (M > 0) {
    std::vector<int> slots(M);
    for (int i = 0; i < M; ++i) slots[i] = picked[i].q.slot;
    // 1. re-bound layers after the split layer
    st->rows_rebounded = rebound(n, slots);
    ht.lap(H_REBOUND);
    // 2. DeepPoly pass of the objective
    upload_batch(n, slots);
    {
      Scope sc(c, C_BOOK, 0.0, 8.0 * M);
      launch_set_best(M, n->bslots, n->pool, -INFINITY, c->st);
    }
    SweepOpts dp;
    dp.track = true;
    sweep(n, n->R + 1, obj_rows(n, M), dp);
    Readback rb(c);
    std::vector<float> lb_dp(M);
    rb.add(lb_dp.data(), n->lb, M);
    // On the fused path without graphs the whole batch goes to the optimiser,
    // whose kernel skips the rows the DeepPoly pass verified (read on the
    // device); the step then synchronises once for all of its results.
    const bool all_rows = !c->graphs && fused_path(n, batch_has_gamma(n, slots), adam.steps);
    if (!all_rows) {
      sync(c);
      rb.finish();
    }
    ht.lap(H_DEEPPOLY);
    // 3. projected Adam on the nodes DeepPoly does not verify; dev lists the
    // batch rows of the device arrays
    std::vector<int> dev;
    for (int i = 0; i < M; ++i)
      if (all_rows || !(lb_dp[i] > 0.f)) dev.push_back(i);
    std::vector<int> dslots(dev.size());
    for (size_t k = 0; k < dev.size(); ++k) dslots[k] = slots[dev[k]];
    const int Md = (int)dslots.size();
    std::vector<int> acs_ld(Md), acs_nd(Md), acs_fbd(Md), cand_d(Md);
    std::vector<float> f32d(Md);
    std::vector<double> f64(Md);
    std::vector<float> best(M);
    int n_cand = 0;
    if (Md > 0) {
      if (!all_rows) upload_batch(n, dslots);
      const bool g = batch_has_gamma(n, dslots);
      run_optimize(n, Md, g, adam, all_rows ? n->lb : nullptr);
      // 5. ACS at the final parameters (a' and gamma^T P of the last sweep)
      {
        Scope sc(c, C_ACS, 0.0, 4.0 * Md * n->SD * (g ? 5.0 : 4.0));
        launch_acs(Md, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->AP, g ? 1 : 0,
                   n->acs_layer, n->acs_neuron, n->score, n->acs_fb, c->st);
      }
      // 4. counterexample check at the best minimiser: FP32 forward pass of every
      // row, then the candidates (picked on the device) in FP64
      {
        Scope sc(c, C_BOOK, 0.0, 8.0 * Md * n->d0);
        k_gather_rows<<<Md, 128, 0, c->st>>>(Md, n->bslots, n->pool.BESTX, n->d0, n->Xb, n->d0,
                                             n->d0);
      }
      forward_rows(n, Md, n->Xb);
      {
        Scope sc(c, C_BOOK, 0.0, 16.0 * Md);
        launch_select_cand(Md, n->fout, n->bslots, n->pool.BEST, n->cand_idx, n->cslots,
                           n->cand_count, c->st);
      }
      {
        Scope sc(c, C_BOOK, 0.0, 8.0 * Md * n->d0);
        k_gather_rows_n<<<Md, 128, 0, c->st>>>(n->cand_count, n->cslots, n->pool.BESTX, n->d0,
                                               n->Xb, n->d0, n->d0);
      }
      {
        Scope sc(c, C_BOOK, 0.0, 8.0 * Md * n->maxd, n->R + 2);
        launch_forward_f64(Md, n->cslots, n->pool, c->d_props, n->nd, n->Xb, n->d0, n->f64a,
                           n->d0 + n->SD, n->f64out, c->st, n->cand_count);
      }
      rb.add(f32d.data(), n->fout, Md);
      rb.add(acs_ld.data(), n->acs_layer, Md);
      rb.add(acs_nd.data(), n->acs_neuron, Md);
      rb.add(acs_fbd.data(), n->acs_fb, Md);
      rb.add(&n_cand, n->cand_count, 1);
      rb.add(cand_d.data(), n->cand_idx, Md);
      rb.add(f64.data(), n->f64out, Md);
    }
    // best bound of every node (DeepPoly value for the verified ones)
    if (!all_rows) upload_batch(n, slots);
    gather_best(n, M, best.data(), &rb);
    sync(c);
    rb.finish();
    ht.lap(H_OPTIMIZE);
    // the optimised rows (batch indices) and their device rows
    std::vector<int> opt_idx, d_of;
    std::vector<int> o_of_d(Md, -1);
    for (int k = 0; k < Md; ++k) {
      if (all_rows && lb_dp[dev[k]] > 0.f) continue;
      o_of_d[k] = (int)opt_idx.size();
      opt_idx.push_back(dev[k]);
      d_of.push_back(k);
    }
    const int Mo = (int)opt_idx.size();
    if (all_rows && Md > Mo && n->fused_cat >= 0)
      prof_sub(c, n->fused_cat, (Md - Mo) * n->fused_row_flops, (Md - Mo) * n->fused_row_bytes);
    std::vector<int> oslots(Mo), acs_l(Mo), acs_n(Mo), acs_fb(Mo);
    std::vector<float> f32(Mo);
    for (int o = 0; o < Mo; ++o) {
      oslots[o] = slots[opt_idx[o]];
      acs_l[o] = acs_ld[d_of[o]];
      acs_n[o] = acs_nd[d_of[o]];
      acs_fb[o] = acs_fbd[d_of[o]];
      f32[o] = f32d[d_of[o]];
    }
    // FP64-confirmed candidates; the inputs of the falsifying ones are read back
    // only when there are any
    std::vector<int> cand_of(Mo, -1);
    bool any_neg = false;
    for (int k = 0; k < n_cand; ++k) {
      const int o = o_of_d[cand_d[k]];
      if (o >= 0) cand_of[o] = k;
      any_neg = any_neg || f64[k] < 0.0;
    }
    std::vector<float> xc;
    if (any_neg) {
      xc.resize((size_t)n_cand * n->d0);
      rb.add(xc.data(), n->Xb, xc.size());
      sync(c);
      rb.finish();
    }
    ht.lap(H_CONFIRM);
    // exact completion of fully split leaves the bound does not decide (Sec. 3.3)
    std::vector<int> leaf_of(Mo, -1);
    std::vector<double> leaf_f64;
    std::vector<float> leaf_x;
    {
      std::vector<int> lo_idx, ls;
      int lsteps = 0;
      for (int o = 0; o < Mo; ++o) {
        const int i = opt_idx[o];
        mnbab_prop* p = picked[i].p;
        const bool cex = cand_of[o] >= 0 && f64[cand_of[o]] < 0.0;
        if (acs_l[o] == 0 && !(best[i] > 0.f) && !cex && p->leaf_steps > 0 && !p->done) {
          lo_idx.push_back(o);
          ls.push_back(oslots[o]);
          lsteps = std::max(lsteps, p->leaf_steps);
        }
      }
      if (!ls.empty()) {
        std::vector<float> lbest;
        leaf_complete(n, ls, lsteps, adam, lbest, leaf_f64, leaf_x);
        for (size_t k = 0; k < lo_idx.size(); ++k) {
          leaf_of[lo_idx[k]] = (int)k;
          best[opt_idx[lo_idx[k]]] = lbest[k];
        }
      }
    }
    // host: verdicts, counterexample confirmation, children
    std::vector<int> par, lay, neu;
    std::vector<int> kidslots;
    std::vector<std::pair<int, int>> branch_of;  // (picked index, opt index)
    int oi = 0;
    for (int i = 0; i < M; ++i) {
      mnbab_prop* p = picked[i].p;
      const QNode& q = picked[i].q;
      mnbab_trace_rec rec{};
      rec.seq = q.seq;
      rec.row = q.row;
      rec.depth = q.depth;
      rec.lb_deeppoly = lb_dp[i];
      rec.lb = best[i];
      rec.f_xstar = NAN;
      rec.verdict = MNBAB_UNKNOWN;
      const bool optimised = oi < Mo && opt_idx[oi] == i;
      const int o = optimised ? oi++ : -1;
      rec.leaf = optimised && acs_l[o] == 0 ? 1 : 0;
      bool release = true;
      if (best[i] > 0.f) {
        rec.verdict = MNBAB_VERIFIED;
        st->nodes_verified++;
      } else {
        bool fals = false;
        if (optimised) {
          rec.f_xstar = f32[o];
          const int k = cand_of[o];
          if (k >= 0) {
            rec.f_xstar = (float)f64[k];
            if (f64[k] < 0.0) {
              fals = true;
              if (!p->done) {
                p->cex.assign(xc.begin() + (size_t)k * n->d0, xc.begin() + (size_t)(k + 1) * n->d0);
                p->cex_row = q.row;
              }
            }
          }
          const int lk = leaf_of[o];
          if (!fals && lk >= 0) {
            // a completed leaf: the averaged minimiser, confirmed in FP64
            rec.f_xstar = (float)leaf_f64[lk];
            if (leaf_f64[lk] < 0.0) {
              fals = true;
              if (!p->done) {
                p->cex.assign(leaf_x.begin() + (size_t)lk * n->d0,
                              leaf_x.begin() + (size_t)(lk + 1) * n->d0);
                p->cex_row = q.row;
              }
            }
          }
        }
        if (fals) {
          rec.verdict = MNBAB_FALSIFIED;
          st->nodes_falsified++;
          p->row_fals[q.row] = 1;
          if (!p->done) {
            p->verdict = MNBAB_FALSIFIED;
            p->done = true;
          }
        } else {
          p->row_lb[q.row] = std::min(p->row_lb[q.row], best[i]);
          if (optimised && acs_l[o] > 0 && !p->done) {
            rec.split_layer = acs_l[o];
            rec.split_neuron = acs_n[o];
            rec.fallback = acs_fb[o];
            par.push_back(q.slot);
            lay.push_back(acs_l[o]);
            neu.push_back(acs_n[o]);
            branch_of.push_back({i, o});
            release = false;
            st->nodes_branched++;
          } else if (!p->done) {
            p->unknown_leaf = true;
            p->row_leaf[q.row] = 1;
            st->nodes_leaf++;
          }
        }
      }
      p->trace.push_back(rec);
      if (release) free_slot(n, q.slot);
    }
    // children
    const int nb = (int)par.size();
    if (nb > 0) {
      kidslots.resize(2 * nb);
      for (int b = 0; b < nb; ++b) {
        kidslots[2 * b] = alloc_slot(n);
        kidslots[2 * b + 1] = alloc_slot(n);
      }
      h2d(c, n->kid_parent, par.data(), nb);
      h2d(c, n->kid_slots, kidslots.data(), 2 * nb);
      h2d(c, n->kid_layer, lay.data(), nb);
      h2d(c, n->kid_neuron, neu.data(), nb);
      {
        Scope sc(c, C_BOOK, 0.0, 3.0 * nb * (17.0 * n->SD + 4.0 * c->EC));
        launch_children(nb, n->kid_parent, n->kid_slots, n->kid_layer, n->kid_neuron, n->pool,
                        n->nd, c->st);
      }
      for (int b = 0; b < nb; ++b) {
        const Picked& pk = picked[branch_of[b].first];
        for (int k = 0; k < 2; ++k) {
          const int s = kidslots[2 * b + k];
          n->slot_split[s] = lay[b];
          n->slot_row[s] = pk.q.row;
          n->slot_prop[s] = n->slot_prop[pk.q.slot];
          pk.p->queue.push_back(QNode{s, pk.p->next_seq++, pk.q.row, pk.q.depth + 1, lay[b]});
          pk.p->row_open[pk.q.row]++;
        }
      }
      // no synchronisation: a freed parent slot is reused only by later work on
      // the same stream, after the children have copied it
      for (int b = 0; b < nb; ++b) free_slot(n, par[b]);
    }
  }
  ht.lap(H_FINISH);
  // property completion
  const double t_end = now_s();
  for (int i = 0; i < n_props; ++i) {
    mnbab_prop* p = props[i];
    if (!p->materialized) continue;
    if (!p->done && !p->queue.empty() && p->timeout_s > 0 && t_end - p->t_start > p->timeout_s) {
      p->verdict = MNBAB_UNKNOWN;
      p->done = true;
      p->timed_out = true;
    }
    if (p->done) {
      for (auto& q : p->queue) free_slot(n, q.slot);
      p->queue.clear();
    } else if (p->queue.empty()) {
      p->verdict = p->unknown_leaf ? MNBAB_UNKNOWN : MNBAB_VERIFIED;
      p->done = true;
    } else if (p->bounded >= p->budget) {
      p->verdict = MNBAB_UNKNOWN;
      p->done = true;
      for (auto& q : p->queue) free_slot(n, q.slot);
      p->queue.clear();
    }
    if (p->done) st->props_done++;
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
#define API_BEGIN(c)                                      \
  if (!(c)) return MNBAB_E_INVALID_ARG;                   \
  try {                                                   \
    ck(cudaSetDevice((c)->device), "cudaSetDevice");
#define API_END(c)                                        \
  return MNBAB_OK;                                        \
  }                                                       \
  catch (const Err& e) {                                  \
    (c)->err = e.msg;                                     \
    return e.code;                                        \
  }                                                       \
  catch (const std::exception& e) {                       \
    (c)->err = e.what();                                  \
    return MNBAB_E_DEVICE;                                \
  }

extern "C" {

mnbab_status mnbab_create(const mnbab_options* opt, mnbab_ctx** out) {
  if (!out) return MNBAB_E_INVALID_ARG;
  *out = nullptr;
  mnbab_ctx* c = new mnbab_ctx();
  mnbab_options o{};
  if (opt) o = *opt;
  c->device = o.device;
  c->budget = o.hbm_budget_bytes ? o.hbm_budget_bytes : (64ull << 30);
  c->node_cap = o.node_capacity > 0 ? o.node_capacity : 65536;
  c->EC = std::max(0, o.max_mnc_rows);
  c->row_chunk = std::min(o.row_chunk > 0 ? o.row_chunk : 32768, 65534);
  c->gemm_path = (o.gemm_path >= 0 && o.gemm_path <= 2) ? o.gemm_path : 0;
  c->graphs = o.use_graphs != 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    delete c;
    return MNBAB_E_DEVICE;
  }
  if (cudaSetDevice(c->device) != cudaSuccess) {
    delete c;
    return MNBAB_E_DEVICE;
  }
  if (o.stream && (cudaStream_t)o.stream != cudaStreamLegacy &&
      (cudaStream_t)o.stream != cudaStreamPerThread) {
    c->st = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MNBAB_E_DEVICE;
    }
    c->own_stream = true;
  }
  try {
    c->d_err = dalloc_t<int>(c, 1);
    void* pin = nullptr;
    if (cudaHostAlloc(&pin, (size_t)16 << 20, cudaHostAllocDefault) == cudaSuccess) {
      c->pin = static_cast<unsigned char*>(pin);
      c->pin_cap = (size_t)16 << 20;
    } else {
      cudaGetLastError();  // unpinned copies instead
    }
    void* rb = nullptr;
    if (cudaHostAlloc(&rb, (size_t)1 << 20, cudaHostAllocDefault) == cudaSuccess) {
      c->rb = static_cast<unsigned char*>(rb);
      c->rb_cap = (size_t)1 << 20;
    } else {
      cudaGetLastError();  // blocking reads instead
    }
    ck(cudaMemset(c->d_err, 0, sizeof(int)), "memset");
  } catch (const Err& e) {
    mnbab_destroy(c);
    return e.code;
  }
  *out = c;
  return MNBAB_OK;
}

void mnbab_destroy(mnbab_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->st);
  for (auto& r : c->pending) {
    if ((r.first >> 16) & 1) continue;  // owned by a graph: destroyed with graph_events
    cudaEventDestroy(r.second.first);
    cudaEventDestroy(r.second.second);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  for (auto* g : c->graph_cache) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
  }
  for (auto e : c->graph_events) cudaEventDestroy(e);
  for (auto& a : c->allocs) cudaFree(a.first);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->rb) cudaFreeHost(c->rb);
  for (auto* r : c->requests) delete r;
  for (auto* n : c->nets) delete n;
  for (auto* p : c->props) delete p;
  for (auto* t : c->tc_convs) tc_conv_destroy(t);
  for (auto* t : c->tc_fcs) tc_fc_destroy(t);
  if (c->own_stream) cudaStreamDestroy(c->st);
  delete c;
}

const char* mnbab_last_error(const mnbab_ctx* c) { return c ? c->err.c_str() : "null context"; }

// Device copy of one affine op (weights in the layouts the kernels read).
LayerDev upload_affine(mnbab_ctx* c, const HostLayer& h) {
  LayerDev L{};
  L.kind = h.kind;
  L.ci = h.ci; L.hi = h.hi; L.wi = h.wi; L.co = h.co; L.ho = h.ho; L.wo = h.wo;
  L.k = h.k; L.s = h.s; L.p = h.p;
  L.d_in = h.ci * h.hi * h.wi;
  L.d_out = h.co * h.ho * h.wo;
  std::vector<float> W(h.W.begin(), h.W.end()), b(h.b.begin(), h.b.end());
  float* dW = dalloc_t<float>(c, W.size());
  float* db = dalloc_t<float>(c, b.size());
  h2d(c, dW, W.data(), W.size());
  h2d(c, db, b.data(), b.size());
  L.W = dW;
  L.b = db;
  if (h.kind == MNBAB_FC) {
    std::vector<float> Wt((size_t)L.d_in * L.d_out);
    for (int o = 0; o < L.d_out; ++o)
      for (int k = 0; k < L.d_in; ++k) Wt[(size_t)k * L.d_out + o] = W[(size_t)o * L.d_in + k];
    float* dWt = dalloc_t<float>(c, Wt.size());
    h2d(c, dWt, Wt.data(), Wt.size());
    L.Wt = dWt;
    // pre-split TF32 weights and TMA tensor maps of the tensor-core GEMM
    TcFc* t = tc_fc_create(L, dalloc_t<float>(c, tc_fc_floats(L)), c->st);
    if (t) {
      c->tc_fcs.push_back(t);
      L.tc = t;
    }
  } else {
    if (!conv_supported(L))
      fail(MNBAB_E_UNSUPPORTED, "convolution row does not fit in shared memory");
    // weights pre-arranged for the row-resident kernels: channel blocks contiguous
    const int kk = L.k * L.k;
    std::vector<float> Wb((size_t)L.co * kk * L.ci), Wfw((size_t)L.ci * kk * L.co);
    for (int co = 0; co < L.co; ++co)
      for (int ci = 0; ci < L.ci; ++ci)
        for (int r = 0; r < kk; ++r) {
          const float w = W[((size_t)co * L.ci + ci) * kk + r];
          Wb[((size_t)co * kk + r) * L.ci + ci] = w;
          Wfw[((size_t)ci * kk + r) * L.co + co] = w;
        }
    float* dWb = dalloc_t<float>(c, Wb.size());
    float* dWf = dalloc_t<float>(c, Wfw.size());
    h2d(c, dWb, Wb.data(), Wb.size());
    h2d(c, dWf, Wfw.data(), Wfw.size());
    L.Wb = dWb;
    L.Wf = dWf;
    // pre-split TF32 weights and TMA tensor maps of the tensor-core convolutions
    const size_t tcf = tc_conv_floats(L);
    if (tcf) {
      TcConv* t = tc_conv_create(L, dalloc_t<float>(c, tcf), c->st);
      if (t) {
        c->tc_convs.push_back(t);
        L.tc = t;
      }
    }
  }
  return L;
}

mnbab_status mnbab_load_network(mnbab_ctx* c, const mnbab_layer_desc* layers, int32_t n_layers,
                                mnbab_net** out) {
  API_BEGIN(c)
  if (!layers || n_layers <= 0 || !out) fail(MNBAB_E_INVALID_ARG, "no layers");
  mnbab_net* n = new mnbab_net();
  n->ctx = c;
  n->id = (int)c->nets.size();
  // parse: ReLU layers get numbers 1..R; an affine op feeds the sum of its
  // consumer; an ADD concatenates the feeds of its two operands
  std::vector<int> relu_of(n_layers, -1);
  std::vector<std::vector<std::pair<int, int>>> feed(n_layers);  // (source node, affine op)
  std::vector<char> is_feed(n_layers, 0);
  std::vector<int> out_dim(n_layers, 0);
  std::vector<std::vector<std::pair<int, int>>> edges(1);
  int d0 = -1;
  auto op_index = [&](int i, int32_t src) {  // 0 = previous op, k >= 1 = op k - 1, -1 = input
    if (src == 0) return i - 1;
    if (src < 0) return -1;
    return (int)src - 1;
  };
  for (int i = 0; i < n_layers; ++i) {
    const mnbab_layer_desc& d = layers[i];
    if (d.kind == MNBAB_RELU) {
      if (i == 0 || !is_feed[i - 1]) fail(MNBAB_E_INVALID_ARG, "ReLU must follow an affine layer or ADD");
      if (feed[i - 1].size() > 2) fail(MNBAB_E_UNSUPPORTED, "more than two edges into a ReLU layer");
      edges.push_back(feed[i - 1]);
      relu_of[i] = (int)edges.size() - 1;
      out_dim[i] = out_dim[i - 1];
      continue;
    }
    if (d.kind == MNBAB_ADD) {
      const int a = op_index(i, d.src_a), b = op_index(i, d.src_b);
      if (d.src_a <= 0 || d.src_b <= 0 || a >= i || b >= i || !is_feed[a] || !is_feed[b])
        fail(MNBAB_E_INVALID_ARG, "ADD must sum two earlier affine layers");
      if (out_dim[a] != out_dim[b]) fail(MNBAB_E_INVALID_ARG, "ADD of different widths");
      feed[i] = feed[a];
      feed[i].insert(feed[i].end(), feed[b].begin(), feed[b].end());
      is_feed[i] = 1;
      out_dim[i] = out_dim[a];
      continue;
    }
    if (d.kind != MNBAB_FC && d.kind != MNBAB_CONV2D) fail(MNBAB_E_INVALID_ARG, "bad layer kind");
    if (!d.W || !d.b) fail(MNBAB_E_INVALID_ARG, "missing weights");
    HostLayer h{};
    h.kind = d.kind;
    if (d.kind == MNBAB_FC) {
      h.ci = d.in_c; h.co = d.out_c; h.hi = h.wi = h.ho = h.wo = 1; h.k = 1; h.s = 1; h.p = 0;
    } else {
      h.ci = d.in_c; h.hi = d.in_h; h.wi = d.in_w; h.co = d.out_c; h.ho = d.out_h; h.wo = d.out_w;
      h.k = d.k; h.s = d.stride; h.p = d.pad;
      if (h.k <= 0 || h.s <= 0 || h.p < 0 || h.ho != (h.hi + 2 * h.p - h.k) / h.s + 1 ||
          h.wo != (h.wi + 2 * h.p - h.k) / h.s + 1)
        fail(MNBAB_E_INVALID_ARG, "inconsistent convolution shape");
    }
    const int din = h.ci * h.hi * h.wi, dout = h.co * h.ho * h.wo;
    if (din <= 0 || dout <= 0) fail(MNBAB_E_INVALID_ARG, "empty layer");
    const int src_op = op_index(i, d.src_a);
    int snode = 0;
    if (src_op >= 0) {
      if (src_op >= i || relu_of[src_op] < 0)
        fail(MNBAB_E_INVALID_ARG, "an affine layer must read a ReLU output or the input");
      snode = relu_of[src_op];
      if (out_dim[src_op] != din) fail(MNBAB_E_INVALID_ARG, "layer sizes do not chain");
    } else {
      if (d0 >= 0 && d0 != din) fail(MNBAB_E_INVALID_ARG, "inconsistent input width");
      d0 = din;
    }
    const size_t nW = d.kind == MNBAB_FC ? (size_t)dout * din : (size_t)h.co * h.ci * h.k * h.k;
    h.W.assign(d.W, d.W + nW);
    h.b.assign(d.b, d.b + h.co);
    n->hops.push_back(std::move(h));
    feed[i] = {{snode, (int)n->hops.size() - 1}};
    is_feed[i] = 1;
    out_dim[i] = dout;
  }
  if (!is_feed[n_layers - 1]) fail(MNBAB_E_INVALID_ARG, "network must end with an affine layer");
  if (d0 < 0) fail(MNBAB_E_INVALID_ARG, "no layer reads the input");
  edges.push_back(feed[n_layers - 1]);
  n->R = (int)edges.size() - 2;
  if (n->R < 0 || n->R > MNBAB_MAXR) fail(MNBAB_E_UNSUPPORTED, "too many ReLU layers");
  if (edges.back().size() != 1 || n->hops[edges.back()[0].second].kind != MNBAB_FC)
    fail(MNBAB_E_UNSUPPORTED, "the last layer must be a single FC layer");
  NetDev& nd = n->nd;
  nd.R = n->R;
  n->d0 = d0;
  nd.d[0] = d0;
  std::vector<LayerDev> ops;
  for (const auto& h : n->hops) ops.push_back(upload_affine(c, h));
  int off = 0;
  for (int t = 1; t <= n->R + 1; ++t) {
    nd.n_edge[t] = (int)edges[t].size();
    nd.src1[t] = edges[t][0].first;
    nd.aff[t] = ops[edges[t][0].second];
    n->eop[t][0] = edges[t][0].second;
    if (nd.n_edge[t] > 1) {
      nd.src2[t] = edges[t][1].first;
      nd.aff2[t] = ops[edges[t][1].second];
      n->eop[t][1] = edges[t][1].second;
      if (nd.aff2[t].d_out != nd.aff[t].d_out) fail(MNBAB_E_INVALID_ARG, "ADD of different widths");
    }
    for (int k = 0; k < nd.n_edge[t]; ++k)
      if (edges[t][k].first >= t) fail(MNBAB_E_INVALID_ARG, "edges must point forward");
    if (t <= n->R) {
      nd.d[t] = nd.aff[t].d_out;
      nd.off[t] = off;
      off += nd.d[t];
      // per-neuron sum of the edge biases into zhat_t
      std::vector<float> bf(nd.d[t], 0.f);
      for (int k = 0; k < nd.n_edge[t]; ++k) {
        const HostLayer& h = n->hops[n->eop[t][k]];
        const int per = h.ho * h.wo;
        for (int j = 0; j < nd.d[t]; ++j) bf[j] += (float)h.b[j / per];
      }
      float* dbf = dalloc_t<float>(c, bf.size());
      h2d(c, dbf, bf.data(), bf.size());
      nd.bfull[t] = dbf;
    }
  }
  nd.off[n->R + 1] = off;
  nd.SD = off;
  n->SD = off;
  n->n_out = nd.aff[n->R + 1].d_out;
  nd.n_out = n->n_out;
  setup_net(c, n);
  sync(c);
  c->nets.push_back(n);
  *out = n;
  API_END(c)
}

mnbab_status mnbab_set_property(mnbab_ctx* c, const mnbab_net* cnet, const float* x_lo,
                                const float* x_hi, const float* C, const float* d, int32_t n_rows,
                                mnbab_prop** out) {
  API_BEGIN(c)
  mnbab_net* n = const_cast<mnbab_net*>(cnet);
  if (!n || n->ctx != c || !x_lo || !x_hi || !C || n_rows <= 0 || !out)
    fail(MNBAB_E_INVALID_ARG, "bad property arguments");
  for (int k = 0; k < n->d0; ++k)
    if (!(x_lo[k] <= x_hi[k])) fail(MNBAB_E_INVALID_ARG, "empty input box");
  mnbab_prop* p = new mnbab_prop();
  p->net = n;
  p->index = (int)c->props.size();
  p->n_rows = n_rows;
  p->lo.assign(x_lo, x_lo + n->d0);
  p->hi.assign(x_hi, x_hi + n->d0);
  // fold the property into the last layer (Sec. 2.1)
  const HostLayer& last = n->hops[n->eop[n->R + 1][0]];
  const int dR = last.ci, no = last.co;
  p->Wf.assign((size_t)n_rows * dR, 0.0);
  p->bf.assign(n_rows, 0.0);
  for (int r = 0; r < n_rows; ++r) {
    for (int o = 0; o < no; ++o) {
      const double cv = C[(size_t)r * no + o];
      if (cv == 0.0) continue;
      for (int k = 0; k < dR; ++k) p->Wf[(size_t)r * dR + k] += cv * last.W[(size_t)o * dR + k];
      p->bf[r] += cv * last.b[o];
    }
    if (d) p->bf[r] += d[r];
  }
  // input box, folded last layer and offsets in one arena block, one copy
  PropDev& pd = p->pd;
  auto up16 = [](size_t x) { return (x + 15) & ~size_t(15); };
  const size_t o_hi = up16(n->d0), o_wf = o_hi + up16(n->d0);
  const size_t o_bf = o_wf + up16(p->Wf.size()), tot = o_bf + up16(p->bf.size());
  std::vector<float> pack(tot, 0.f);
  std::copy(x_lo, x_lo + n->d0, pack.begin());
  std::copy(x_hi, x_hi + n->d0, pack.begin() + o_hi);
  for (size_t k = 0; k < p->Wf.size(); ++k) pack[o_wf + k] = (float)p->Wf[k];
  for (size_t k = 0; k < p->bf.size(); ++k) pack[o_bf + k] = (float)p->bf[k];
  float* blk = prop_arena(c, tot);
  h2d(c, blk, pack.data(), tot);
  float* dlo = blk;
  float* dhi = blk + o_hi;
  float* dWf = blk + o_wf;
  float* dbf = blk + o_bf;
  pd.lo = dlo; pd.hi = dhi; pd.Wf = dWf; pd.bf = dbf; pd.n_rows = n_rows; pd.E = 0;
  pd.cab = 0;
  update_cab(n, p);
  c->props.push_back(p);
  upload_prop(c, p->index);
  p->row_open.assign(n_rows, 0);
  p->row_leaf.assign(n_rows, 0);
  p->row_fals.assign(n_rows, 0);
  p->row_lb.assign(n_rows, INFINITY);
  // node slots are allocated when the property starts (materialize): right
  // away for direct use, on admission in the request loop
  *out = p;
  API_END(c)
}

mnbab_status mnbab_get_root_bounds(const mnbab_ctx* cc, const mnbab_prop* p, int32_t layer,
                                   float* l_out, float* u_out) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!p || !l_out || !u_out) fail(MNBAB_E_INVALID_ARG, "null argument");
  mnbab_net* n = p->net;
  if (layer < 1 || layer > n->R) fail(MNBAB_E_INVALID_ARG, "bad layer");
  ensure_roots(n);
  if (!p->materialized) fail(MNBAB_E_INVALID_ARG, "property is still queued in the request loop");
  const size_t base = (size_t)p->root_slot * n->SD + n->nd.off[layer];
  d2h(c, l_out, n->pool.L + base, n->nd.d[layer]);
  d2h(c, u_out, n->pool.U + base, n->nd.d[layer]);
  sync(c);
  API_END(c)
}

mnbab_status mnbab_set_mnc(mnbab_ctx* c, mnbab_prop* p, int32_t layer, int32_t n_rows, int32_t k,
                           const int32_t* idx, const float* P, const float* Phat, const float* pv) {
  API_BEGIN(c)
  if (!p || layer < 1 || layer > p->net->R || n_rows < 0 || k <= 0 || (n_rows && (!idx || !P ||
      !Phat || !pv)))
    fail(MNBAB_E_INVALID_ARG, "bad constraint arguments");
  set_mnc_impl(c, p, layer, n_rows, k, idx, P, Phat, pv);
  API_END(c)
}

mnbab_status mnbab_get_mnc(mnbab_ctx* c, const mnbab_prop* p, int32_t layer, int32_t max_rows,
                           int32_t* idx, float* P, float* Phat, float* pv, int32_t* n_out) {
  API_BEGIN(c)
  if (!p || layer < 1 || layer > p->net->R || !n_out || max_rows < 0)
    fail(MNBAB_E_INVALID_ARG, "bad arguments");
  const MncDev& m = p->pd.mnc[layer];
  *n_out = m.e;
  if (m.e > max_rows) fail(MNBAB_E_BUDGET, "more rows than max_rows");
  if (m.e > 0) {
    if (!idx || !P || !Phat || !pv) fail(MNBAB_E_INVALID_ARG, "null output");
    const size_t nk = (size_t)m.e * m.k;
    d2h(c, idx, m.idx, nk);
    d2h(c, P, m.P, nk);
    d2h(c, Phat, m.Ph, nk);
    d2h(c, pv, m.p, m.e);
    sync(c);
  }
  API_END(c)
}

mnbab_status mnbab_generate_mnc(mnbab_ctx* c, mnbab_prop* p, int32_t max_groups,
                                int64_t* rows_out) {
  API_BEGIN(c)
  if (!p || max_groups < 0) fail(MNBAB_E_INVALID_ARG, "bad arguments");
  const int64_t tot = generate_mnc_impl(c, p, max_groups);
  if (rows_out) *rows_out = tot;
  API_END(c)
}

mnbab_status mnbab_node_root(mnbab_ctx* c, mnbab_prop* p, int32_t row, mnbab_node_id* out) {
  API_BEGIN(c)
  if (!p || !out || row < 0 || row >= p->n_rows) fail(MNBAB_E_INVALID_ARG, "bad row");
  mnbab_net* n = p->net;
  ensure_roots(n);
  if (!p->materialized) fail(MNBAB_E_INVALID_ARG, "property is still queued in the request loop");
  const int s = alloc_slot(n);
  n->slot_prop[s] = p->index;
  n->slot_row[s] = row;
  n->slot_split[s] = n->R;
  const int src = p->root_slot;
  h2d(c, n->ri_dst, &s, 1);
  h2d(c, n->ri_src, &src, 1);
  h2d(c, n->ri_row, &row, 1);
  {
    Scope sc(c, C_BOOK, 0.0, 25.0 * n->SD);
    launch_root_init(1, n->ri_dst, n->ri_src, n->ri_row, n->pool, c->st);
  }
  sync(c);
  *out = ((int64_t)n->id << 32) | (int64_t)s;
  API_END(c)
}

mnbab_status mnbab_node_free(mnbab_ctx* c, mnbab_node_id node) {
  API_BEGIN(c)
  int s;
  mnbab_net* n = net_of(c, node, &s);
  free_slot(n, s);
  API_END(c)
}

mnbab_status mnbab_export_params(const mnbab_ctx* cc, mnbab_node_id node, void* buf,
                                 size_t* bytes) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!bytes) fail(MNBAB_E_INVALID_ARG, "null size");
  int s;
  mnbab_net* n = net_of(c, node, &s);
  const int E = c->props[n->slot_prop[s]]->pd.E;
  const size_t SD = n->SD;
  const size_t need = 16 + SD * (4 + 4 + 1 + 4 + 4) + (size_t)E * 4;
  if (!buf) {
    *bytes = need;
    return MNBAB_OK;
  }
  if (*bytes < need) fail(MNBAB_E_INVALID_ARG, "buffer too small");
  char* b = static_cast<char*>(buf);
  int32_t hdr[4] = {n->slot_split[s], n->R, n->SD, E};
  std::memcpy(b, hdr, 16);
  char* q = b + 16;
  d2h(c, (float*)q, n->pool.L + s * SD, SD); q += SD * 4;
  d2h(c, (float*)q, n->pool.U + s * SD, SD); q += SD * 4;
  d2h(c, (int8_t*)q, n->pool.S + s * SD, SD); q += SD;
  d2h(c, (float*)q, n->pool.ALPHA + s * SD, SD); q += SD * 4;
  d2h(c, (float*)q, n->pool.BETA + s * SD, SD); q += SD * 4;
  d2h(c, (float*)q, n->pool.GAM + (size_t)s * c->EC, E);
  sync(c);
  *bytes = need;
  API_END(c)
}

mnbab_status mnbab_import_params(mnbab_ctx* c, mnbab_node_id node, const void* buf, size_t bytes) {
  API_BEGIN(c)
  if (!buf) fail(MNBAB_E_INVALID_ARG, "null buffer");
  int s;
  mnbab_net* n = net_of(c, node, &s);
  const int E = c->props[n->slot_prop[s]]->pd.E;
  const size_t SD = n->SD;
  const size_t need = 16 + SD * (4 + 4 + 1 + 4 + 4) + (size_t)E * 4;
  if (bytes < need) fail(MNBAB_E_INVALID_ARG, "parameter block too small");
  const char* b = static_cast<const char*>(buf);
  int32_t hdr[4];
  std::memcpy(hdr, b, 16);
  if (hdr[1] != n->R || hdr[2] != n->SD || hdr[3] != E)
    fail(MNBAB_E_INVALID_ARG, "parameter block does not match the node's network / property");
  if (hdr[0] < 0 || hdr[0] > n->R) fail(MNBAB_E_INVALID_ARG, "bad split layer");
  const char* q = b + 16;
  h2d(c, n->pool.L + s * SD, (const float*)q, SD); q += SD * 4;
  h2d(c, n->pool.U + s * SD, (const float*)q, SD); q += SD * 4;
  h2d(c, n->pool.S + s * SD, (const int8_t*)q, SD); q += SD;
  h2d(c, n->pool.ALPHA + s * SD, (const float*)q, SD); q += SD * 4;
  h2d(c, n->pool.BETA + s * SD, (const float*)q, SD); q += SD * 4;
  h2d(c, n->pool.GAM + (size_t)s * c->EC, (const float*)q, E);
  sync(c);
  n->slot_split[s] = hdr[0];
  API_END(c)
}

mnbab_status mnbab_bound_batch(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                               float* lb_out, float* ub_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!lb_out) fail(MNBAB_E_INVALID_ARG, "null output");
  ensure_roots(n);
  rebound(n, slots);
  upload_batch(n, slots);
  const bool g = batch_has_gamma(n, slots);
  if (g) {
    Scope sc(c, C_GAMMA, 0.0, 4.0 * nn * (c->EC + 2.0 * n->SD), 2);
    launch_gamma_proj(nn, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
  }
  SweepOpts o;
  o.final_mode = true;
  o.has_gamma = g;
  o.store = true;
  sweep(n, n->R + 1, obj_rows(n, nn), o);
  d2h(c, lb_out, n->lb, nn);
  if (ub_out) {
    forward_rows(n, nn, n->X);
    d2h(c, ub_out, n->fout, nn);
  }
  sync(c);
  API_END(c)
}

mnbab_status mnbab_deeppoly_batch(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                                  float* lb_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!lb_out) fail(MNBAB_E_INVALID_ARG, "null output");
  upload_batch(n, slots);
  SweepOpts o;
  sweep(n, n->R + 1, obj_rows(n, nn), o);
  d2h(c, lb_out, n->lb, nn);
  sync(c);
  API_END(c)
}

mnbab_status mnbab_set_params(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                              const float* params) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!params) fail(MNBAB_E_INVALID_ARG, "null parameter array");
  const size_t SD = n->SD;
  size_t at = 0;
  for (int i = 0; i < nn; ++i) {
    const int s = slots[i];
    const int E = c->props[n->slot_prop[s]]->pd.E;
    h2d(c, n->pool.ALPHA + (size_t)s * SD, params + at, SD);
    at += SD;
    h2d(c, n->pool.BETA + (size_t)s * SD, params + at, SD);
    at += SD;
    if (E) h2d(c, n->pool.GAM + (size_t)s * c->EC, params + at, E);
    at += E;
  }
  sync(c);
  API_END(c)
}

mnbab_status mnbab_bound_grad(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                              float* lb_out, float* grad_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!lb_out || !grad_out) fail(MNBAB_E_INVALID_ARG, "null output");
  upload_batch(n, slots);
  const bool g = batch_has_gamma(n, slots);
  if (g) {
    Scope sc(c, C_GAMMA, 0.0, 4.0 * nn * (c->EC + 2.0 * n->SD), 2);
    launch_gamma_proj(nn, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
  }
  SweepOpts o;
  o.final_mode = true;
  o.has_gamma = g;
  o.store = true;
  sweep(n, n->R + 1, obj_rows(n, nn), o);
  adjoint(n, nn, g);
  d2h(c, lb_out, n->lb, nn);
  sync(c);
  size_t at = 0;
  for (int i = 0; i < nn; ++i) {
    const int E = c->props[n->slot_prop[slots[i]]]->pd.E;
    d2h(c, grad_out + at, n->GA + (size_t)i * n->SD, n->SD);
    at += n->SD;
    d2h(c, grad_out + at, n->GB + (size_t)i * n->SD, n->SD);
    at += n->SD;
    if (E) d2h(c, grad_out + at, n->GG + (size_t)i * c->EC, E);
    at += E;
  }
  sync(c);
  API_END(c)
}

mnbab_status mnbab_optimize(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                            const mnbab_adam* cfg, float* best_lb_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!best_lb_out) fail(MNBAB_E_INVALID_ARG, "null output");
  const mnbab_adam a = cfg ? *cfg : default_adam();
  if (a.steps < 0) fail(MNBAB_E_INVALID_ARG, "negative step count");
  upload_batch(n, slots);
  {
    Scope sc(c, C_BOOK, 0.0, 8.0 * nn);
    launch_set_best(nn, n->bslots, n->pool, -INFINITY, c->st);
  }
  run_optimize(n, nn, batch_has_gamma(n, slots), a);
  gather_best(n, nn, best_lb_out);
  sync(c);
  API_END(c)
}

mnbab_status mnbab_optimize_intermediate(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                                         int32_t first_layer, const mnbab_adam* cfg,
                                         int64_t* rows_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  const mnbab_adam a = cfg ? *cfg : default_adam();
  if (a.steps < 0) fail(MNBAB_E_INVALID_ARG, "negative step count");
  if (2 * nn > n->B) fail(MNBAB_E_INVALID_ARG, "more nodes than half the batch capacity");
  {
    // two sets of one node would update the same bounds concurrently
    std::vector<int> sorted(slots);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      fail(MNBAB_E_INVALID_ARG, "a node is listed twice");
  }
  const int64_t total = optimize_intermediate_impl(n, slots, first_layer, a);
  if (rows_out) *rows_out = total;
  API_END(c)
}

mnbab_status mnbab_set_intermediate_steps(mnbab_ctx* c, mnbab_prop* p, int32_t steps) {
  API_BEGIN(c)
  if (!p || steps < 0) fail(MNBAB_E_INVALID_ARG, "bad step count");
  if (p->materialized) fail(MNBAB_E_INVALID_ARG, "property already started");
  if (steps > 0 && p->net->B < 2)
    fail(MNBAB_E_INVALID_ARG,
         "optimised intermediate bounds need a batch capacity of at least 2 (node_capacity >= 4)");
  p->inter_steps = steps;
  API_END(c)
}

mnbab_status mnbab_score_branches(mnbab_ctx* c, const mnbab_node_id* nodes, int32_t nn,
                                  int32_t* layer_out, int32_t* neuron_out, float* score_out) {
  API_BEGIN(c)
  std::vector<int> slots;
  mnbab_net* n = slots_of(c, nodes, nn, slots);
  if (!layer_out || !neuron_out) fail(MNBAB_E_INVALID_ARG, "null output");
  upload_batch(n, slots);
  const bool g = batch_has_gamma(n, slots);
  if (g) {
    Scope sc(c, C_GAMMA, 0.0, 4.0 * nn * (c->EC + 2.0 * n->SD), 2);
    launch_gamma_proj(nn, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->gp0, c->st);
  }
  SweepOpts o;
  o.final_mode = true;
  o.has_gamma = g;
  o.store = true;
  sweep(n, n->R + 1, obj_rows(n, nn), o);
  {
    Scope sc(c, C_ACS, 0.0, 4.0 * nn * n->SD * 5.0);
    launch_acs(nn, n->bslots, n->pool, c->d_props, n->nd, n->GP, n->GPh, n->AP, g ? 1 : 0,
               n->acs_layer,
               n->acs_neuron, n->score, n->acs_fb, c->st);
  }
  d2h(c, layer_out, n->acs_layer, nn);
  d2h(c, neuron_out, n->acs_neuron, nn);
  if (score_out) d2h(c, score_out, n->score, nn);
  sync(c);
  API_END(c)
}

mnbab_status mnbab_bab_step(mnbab_ctx* c, mnbab_prop* const* props, int32_t n_props,
                            int32_t max_nodes, const mnbab_adam* cfg, mnbab_step_stats* out) {
  API_BEGIN(c)
  if (!props || !out) fail(MNBAB_E_INVALID_ARG, "null argument");
  const mnbab_adam a = cfg ? *cfg : default_adam();
  bab_step_impl(c, props, n_props, max_nodes, a, out);
  API_END(c)
}

mnbab_status mnbab_set_leaf_steps(mnbab_ctx* c, mnbab_prop* p, int32_t steps) {
  API_BEGIN(c)
  if (!p || steps < 0) fail(MNBAB_E_INVALID_ARG, "bad step count");
  p->leaf_steps = steps;
  API_END(c)
}

mnbab_status mnbab_set_budget(mnbab_ctx* c, mnbab_prop* p, int32_t max_nodes) {
  API_BEGIN(c)
  if (!p || max_nodes <= 0) fail(MNBAB_E_INVALID_ARG, "bad budget");
  p->budget = max_nodes;
  API_END(c)
}

mnbab_status mnbab_set_timeout(mnbab_ctx* c, mnbab_prop* p, double seconds) {
  API_BEGIN(c)
  if (!p || !(seconds >= 0.0)) fail(MNBAB_E_INVALID_ARG, "bad timeout");
  p->timeout_s = seconds;
  API_END(c)
}

mnbab_status mnbab_get_status(const mnbab_ctx* cc, const mnbab_prop* p, int32_t* bounded,
                              int32_t* timed_out, double* elapsed_s) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!p) fail(MNBAB_E_INVALID_ARG, "null property");
  if (bounded) *bounded = p->bounded;
  if (timed_out) *timed_out = p->timed_out ? 1 : 0;
  if (elapsed_s) *elapsed_s = p->t_start > 0.0 ? now_s() - p->t_start : 0.0;
  API_END(c)
}

mnbab_status mnbab_set_branching(mnbab_ctx* c, mnbab_prop* p, int32_t mode) {
  API_BEGIN(c)
  if (!p || mode < 0 || mode > 1) fail(MNBAB_E_INVALID_ARG, "bad branching mode");
  p->pd.cab = mode;
  upload_prop(c, p->index);
  sync(c);
  API_END(c)
}

mnbab_status mnbab_get_verdict(const mnbab_ctx* cc, const mnbab_prop* p, int32_t row,
                               int32_t* verdict, float* lb, float* x_cex) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!p || !verdict) fail(MNBAB_E_INVALID_ARG, "null argument");
  if (row >= p->n_rows) fail(MNBAB_E_INVALID_ARG, "bad row");
  if (row < 0) {
    *verdict = p->done ? p->verdict : MNBAB_UNKNOWN;
    if (lb) {
      float m = INFINITY;
      for (float v : p->row_lb) m = std::min(m, v);
      *lb = m;
    }
    if (x_cex && p->verdict == MNBAB_FALSIFIED)
      std::memcpy(x_cex, p->cex.data(), p->cex.size() * sizeof(float));
  } else {
    int v = MNBAB_UNKNOWN;
    if (p->row_fals[row]) v = MNBAB_FALSIFIED;
    else if (p->row_open[row] == 0 && !p->row_leaf[row] &&
             !(p->done && p->verdict != MNBAB_VERIFIED && p->row_lb[row] <= 0.f))
      v = MNBAB_VERIFIED;
    *verdict = v;
    if (lb) *lb = p->row_lb[row];
    if (x_cex && p->cex_row == row)
      std::memcpy(x_cex, p->cex.data(), p->cex.size() * sizeof(float));
  }
  API_END(c)
}

mnbab_status mnbab_get_trace(const mnbab_ctx* cc, const mnbab_prop* p, mnbab_trace_rec* recs,
                             int32_t max_recs, int32_t* n_out) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!p || !n_out) fail(MNBAB_E_INVALID_ARG, "null argument");
  const int nt = (int)p->trace.size();
  const int k = recs ? std::min(nt, std::max(0, (int)max_recs)) : 0;
  for (int i = 0; i < k; ++i) recs[i] = p->trace[i];
  *n_out = recs ? k : nt;
  API_END(c)
}

// HBM of one node slot of a network's pool: bounds, splits, slopes, split
// multipliers and their Adam moments per neuron, multi-neuron multipliers and
// moments per constraint row, the best minimiser and the slot's scalars
static uint64_t slot_bytes(const mnbab_net* n) {
  return (uint64_t)n->SD * (8 * sizeof(float) + 1) + (uint64_t)n->ctx->EC * 3 * sizeof(float) +
         (uint64_t)n->d0 * sizeof(float) + 3 * sizeof(int);
}

mnbab_status mnbab_submit(mnbab_ctx* c, mnbab_prop* p, double timeout_s, uint64_t* ticket) {
  API_BEGIN(c)
  if (!p || !ticket) fail(MNBAB_E_INVALID_ARG, "null argument");
  if (p->materialized || !p->admitted) fail(MNBAB_E_INVALID_ARG, "property already started or queued");
  mnbab_net* n = p->net;
  Request* r = new Request();
  r->ticket = c->requests.size() + 1;
  r->p = p;
  r->t_submit = now_s();
  r->deadline = timeout_s > 0 ? r->t_submit + timeout_s : 0.0;
  // live nodes never exceed the rows' roots plus two children per bounded node
  r->reserve = std::min(n->cap, p->n_rows + 1 + 2 * p->budget);
  r->bytes = (uint64_t)r->reserve * slot_bytes(n);
  p->admitted = false;
  c->requests.push_back(r);
  c->req_queue.push_back(r);
  *ticket = r->ticket;
  API_END(c)
}

mnbab_status mnbab_serve_step(mnbab_ctx* c, int32_t max_nodes, const mnbab_adam* cfg,
                              mnbab_serve_stats* out) {
  API_BEGIN(c)
  if (!out) fail(MNBAB_E_INVALID_ARG, "null argument");
  std::memset(out, 0, sizeof(*out));
  const mnbab_adam a = cfg ? *cfg : default_adam();
  if (c->reserved.size() < c->nets.size()) c->reserved.resize(c->nets.size(), 0);
  // admission, FIFO: a request starts once the HBM its node slots take fits
  // the serving budget next to the active requests of every network, and its
  // network's pool can hold the slots (the pools are allocated within the
  // context's HBM budget)
  const uint64_t hbm = c->serve_budget ? c->serve_budget : c->budget;
  while (!c->req_queue.empty()) {
    Request* r = c->req_queue.front();
    mnbab_net* n = r->p->net;
    const int avail = n->cap - 8;  // the pad slot and a small margin
    // a request larger than the room still runs once its network is idle, and
    // one larger than the budget once no request is active
    if (c->reserved[n->id] > 0 && c->reserved[n->id] + r->reserve > avail) break;
    if (c->serve_bytes > 0 && c->serve_bytes + r->bytes > hbm) break;
    c->reserved[n->id] += r->reserve;
    c->serve_bytes += r->bytes;
    r->p->admitted = true;
    r->state = 1;
    r->t_admit = now_s();
    c->req_queue.pop_front();
    out->admitted++;
  }
  // one BaB step per network over all its active requests: nodes of different
  // requests share the launches
  for (auto* n : c->nets) {
    std::vector<mnbab_prop*> props;
    for (auto* r : c->requests)
      if (r->state == 1 && r->p->net == n) props.push_back(r->p);
    if (props.empty()) continue;
    mnbab_step_stats st;
    bab_step_impl(c, props.data(), (int)props.size(), max_nodes, a, &st);
    out->step.nodes_bounded += st.nodes_bounded;
    out->step.nodes_verified += st.nodes_verified;
    out->step.nodes_falsified += st.nodes_falsified;
    out->step.nodes_branched += st.nodes_branched;
    out->step.nodes_leaf += st.nodes_leaf;
    out->step.rows_rebounded += st.rows_rebounded;
    out->step.h2d_bytes += st.h2d_bytes;
    out->step.d2h_bytes += st.d2h_bytes;
  }
  // retire: verdict, node budget, or timeout
  const double t = now_s();
  for (auto* r : c->requests) {
    if (r->state != 1) continue;
    mnbab_prop* p = r->p;
    mnbab_net* n = p->net;
    if (!p->done && r->deadline > 0 && t > r->deadline) {
      p->verdict = MNBAB_UNKNOWN;
      p->done = true;
      for (auto& q : p->queue) free_slot(n, q.slot);
      p->queue.clear();
      r->timed_out = 1;
    }
    if (p->done) {
      r->state = 2;
      r->t_done = t;
      c->reserved[n->id] -= r->reserve;
      c->serve_bytes -= r->bytes;
      out->finished++;
    }
  }
  for (auto* r : c->requests) {
    if (r->state == 0) out->queued++;
    if (r->state == 1) out->active++;
  }
  out->reserved_bytes = (int64_t)c->serve_bytes;
  API_END(c)
}

mnbab_status mnbab_set_serving_budget(mnbab_ctx* c, uint64_t bytes) {
  API_BEGIN(c)
  c->serve_budget = bytes;
  API_END(c)
}

mnbab_status mnbab_poll(mnbab_ctx* c, uint64_t ticket, int32_t* done) {
  API_BEGIN(c)
  if (!done || ticket == 0 || ticket > c->requests.size()) fail(MNBAB_E_INVALID_ARG, "bad ticket");
  *done = c->requests[ticket - 1]->state == 2 ? 1 : 0;
  API_END(c)
}

mnbab_status mnbab_request_result(mnbab_ctx* c, uint64_t ticket, int32_t* verdict, double* wait_s,
                                  double* total_s, int32_t* nodes) {
  API_BEGIN(c)
  if (ticket == 0 || ticket > c->requests.size()) fail(MNBAB_E_INVALID_ARG, "bad ticket");
  const Request* r = c->requests[ticket - 1];
  if (r->state != 2) fail(MNBAB_E_INVALID_ARG, "request not finished");
  if (verdict) *verdict = r->p->verdict;
  if (wait_s) *wait_s = r->t_admit - r->t_submit;
  if (total_s) *total_s = r->t_done - r->t_submit;
  if (nodes) *nodes = r->p->bounded;
  API_END(c)
}

mnbab_status mnbab_profile(mnbab_ctx* c, int32_t enable) {
  API_BEGIN(c)
  sync(c);
  if (enable) {
    for (int i = 0; i < 32; ++i) {
      c->acc_n[i] = 0;
      c->acc_ms[i] = c->acc_flops[i] = c->acc_bytes[i] = 0.0;
    }
  }
  c->prof = enable != 0;
  API_END(c)
}

mnbab_status mnbab_profile_mask(mnbab_ctx* c, uint64_t class_mask) {
  API_BEGIN(c)
  c->prof_mask = class_mask;
  API_END(c)
}

mnbab_status mnbab_profile_read(mnbab_ctx* c, mnbab_kernel_stat* stats, int32_t max_stats,
                                int32_t* n_out, int64_t* total_launches) {
  API_BEGIN(c)
  sync(c);
  const int k = stats ? std::min((int)NCAT, std::max(0, (int)max_stats)) : 0;
  for (int i = 0; i < k; ++i) {
    std::memset(stats[i].name, 0, sizeof(stats[i].name));
    std::strncpy(stats[i].name, CAT_NAMES[i], sizeof(stats[i].name) - 1);
    stats[i].launches = c->acc_n[i];
    stats[i].ms = c->acc_ms[i];
    stats[i].flops = c->acc_flops[i];
    stats[i].bytes = c->acc_bytes[i];
  }
  if (n_out) *n_out = stats ? k : (int)NCAT;
  if (total_launches) *total_launches = c->launches;
  API_END(c)
}

mnbab_status mnbab_attack(mnbab_ctx* c, const mnbab_prop* p, int32_t n_starts, int32_t steps,
                          const float* starts, float* best_out, float* x_out) {
  API_BEGIN(c)
  if (!p || n_starts <= 0 || steps < 1 || !starts || !best_out)
    fail(MNBAB_E_INVALID_ARG, "bad attack arguments");
  attack_impl(c, p, n_starts, steps, starts, best_out, x_out);
  API_END(c)
}

mnbab_status mnbab_autotune(mnbab_ctx* c, mnbab_net* n, int32_t max_rows, mnbab_tune_rec* recs,
                            int32_t max_recs, int32_t* n_out) {
  API_BEGIN(c)
  if (!n || n->ctx != c || max_rows < 1 || max_recs < 0 || (max_recs > 0 && !recs))
    fail(MNBAB_E_INVALID_ARG, "bad autotune arguments");
  std::vector<mnbab_tune_rec> all;
  autotune_impl(n, max_rows, all);
  const int k = std::min((int)all.size(), max_recs);
  if (k > 0) std::memcpy(recs, all.data(), (size_t)k * sizeof(mnbab_tune_rec));
  if (n_out) *n_out = (int)all.size();
  API_END(c)
}

mnbab_status mnbab_set_variant(mnbab_ctx* c, mnbab_net* n, int32_t node, int32_t edge, int32_t dir,
                               int32_t variant) {
  API_BEGIN(c)
  if (!n || n->ctx != c || node < 1 || node > n->R || edge < 0 || edge >= n->nd.n_edge[node] ||
      dir < 0 || dir > 1 || variant < 0 || variant >= NVARIANT)
    fail(MNBAB_E_INVALID_ARG, "bad variant arguments");
  LayerDev& L = edge == 0 ? n->nd.aff[node] : n->nd.aff2[node];
  for (int b = 0; b < 6; ++b) L.tune[dir][b] = (signed char)variant;
  API_END(c)
}

mnbab_status mnbab_set_attack_path(mnbab_ctx* c, int32_t path) {
  API_BEGIN(c)
  if (path < 0 || path > 2) fail(MNBAB_E_INVALID_ARG, "attack path is 0, 1 or 2");
  c->attack_path = path;
  API_END(c)
}

mnbab_status mnbab_set_attack(mnbab_ctx* c, mnbab_prop* p, int32_t n_starts, int32_t steps,
                              uint64_t seed) {
  API_BEGIN(c)
  if (!p || n_starts < 0 || (n_starts > 0 && steps < 1))
    fail(MNBAB_E_INVALID_ARG, "bad attack arguments");
  if (p->materialized) fail(MNBAB_E_INVALID_ARG, "property already started");
  p->atk_starts = n_starts;
  p->atk_steps = steps;
  p->atk_seed = seed;
  API_END(c)
}

mnbab_status mnbab_queue_size(const mnbab_ctx* cc, const mnbab_prop* p, int32_t* n_out) {
  mnbab_ctx* c = const_cast<mnbab_ctx*>(cc);
  API_BEGIN(c)
  if (!p || !n_out) fail(MNBAB_E_INVALID_ARG, "null argument");
  *n_out = (int)p->queue.size();
  API_END(c)
}

}  // extern "C"
