// Allocation-free DeepPoly bound for fully connected ReLU networks.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or allocator hooks, or embedded hosts whose device
// memory is partitioned up front.  For them, mnbab_deeppoly_fc_noalloc runs the same
// back-substitution kernels as mnbab_deeppoly_batch, but every scratch buffer
// (the two coefficient buffers, the per-row partial sums, the row tables and
// one property descriptor) is carved out of the file-scope array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mnbab.h"
#include "mnbab_internal.h"

using namespace mnbab;

namespace {

constexpr size_t kScratchBytes = MNBAB_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol: kernels must be given the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

__global__ void k_iota(int* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

// The property descriptor travels as a kernel argument and is stored by the
// device, so no host buffer has to outlive the call.
__global__ void k_store_prop(PropDev* dst, PropDev pd) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst = pd;
}

void set_err(char* buf, size_t len, const char* msg) {
  if (buf && len) {
    std::strncpy(buf, msg, len - 1);
    buf[len - 1] = 0;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" mnbab_status mnbab_deeppoly_fc_noalloc(int32_t n_affine, const int32_t* dims,
                                                  const float* const* W, const float* const* b,
                                                  const float* x_lo, const float* x_hi,
                                                  const float* l, const float* u,
                                                  const float* Wf, const float* bf,
                                                  int32_t n_rows, float* lb_out, void* stream,
                                                  char* err, size_t err_len) {
  if (n_affine < 1 || n_affine > MNBAB_MAXR + 1 || !dims || n_rows <= 0 || !x_lo || !x_hi ||
      !Wf || !bf || !lb_out || (n_affine > 1 && (!W || !b || !l || !u))) {
    set_err(err, err_len, "invalid argument");
    return MNBAB_E_INVALID_ARG;
  }
  for (int i = 0; i < n_affine; ++i)
    if (dims[i] <= 0) {
      set_err(err, err_len, "non-positive layer width");
      return MNBAB_E_INVALID_ARG;
    }
  const int R = n_affine - 1;
  // network description (hidden affine layers 1..R; the objective rows are Wf, bf)
  NetDev nd{};
  nd.R = R;
  nd.d[0] = dims[0];
  int off = 0, maxd = dims[0];
  for (int i = 1; i <= R; ++i) {
    LayerDev& Ld = nd.aff[i];
    Ld.kind = 1;
    Ld.d_in = dims[i - 1];
    Ld.d_out = dims[i];
    Ld.ci = Ld.d_in; Ld.co = Ld.d_out;
    Ld.hi = Ld.wi = Ld.ho = Ld.wo = Ld.k = Ld.s = 1;
    Ld.p = 0;
    Ld.W = W[i - 1];
    Ld.b = b[i - 1];
    if (!Ld.W || !Ld.b) {
      set_err(err, err_len, "null weight pointer");
      return MNBAB_E_INVALID_ARG;
    }
    nd.d[i] = dims[i];
    nd.n_edge[i] = 1;
    nd.src1[i] = i - 1;
    nd.off[i] = off;
    off += dims[i];
    maxd = std::max(maxd, dims[i]);
  }
  nd.SD = off;
  nd.off[R + 1] = off;
  nd.n_edge[R + 1] = 1;
  nd.src1[R + 1] = R;
  int nslot = 1;
  for (int i = 1; i <= R; ++i) nslot += backsub_slots(nd.aff[i]);
  // scratch layout
  const size_t M = (size_t)n_rows;
  size_t at = 0;
  const size_t o_prop = at; at = align256(at + sizeof(PropDev));
  const size_t o_pidx = at; at = align256(at + sizeof(int));
  const size_t o_S = at; at = align256(at + std::max(1, off));
  const size_t o_node = at; at = align256(at + M * sizeof(int));
  const size_t o_j = at; at = align256(at + M * sizeof(int));
  const size_t o_A = at; at = align256(at + M * maxd * sizeof(float));
  const size_t o_B = at; at = align256(at + M * maxd * sizeof(float));
  const size_t o_part = at; at = align256(at + M * nslot * sizeof(float));
  if (at > kScratchBytes) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "needs %zu bytes of scratch, more than the %zu-byte static scratch; "
                  "bound fewer rows per call",
                  at, kScratchBytes);
    set_err(err, err_len, msg);
    return MNBAB_E_BUDGET;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "no current CUDA device");
    return MNBAB_E_DEVICE;
  }
  unsigned char* base = nullptr;
  {
    // once per device, with that device current: the device address of the scratch
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        set_err(err, err_len, cudaGetErrorString(e));
        return MNBAB_E_DEVICE;
      }
      g_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  PropDev pd{};
  pd.lo = x_lo;
  pd.hi = x_hi;
  pd.Wf = Wf;
  pd.bf = bf;
  pd.n_rows = n_rows;
  pd.E = 0;
  PropDev* d_prop = reinterpret_cast<PropDev*>(base + o_prop);
  int* d_pidx = reinterpret_cast<int*>(base + o_pidx);
  int8_t* d_S = reinterpret_cast<int8_t*>(base + o_S);
  int* d_node = reinterpret_cast<int*>(base + o_node);
  int* d_j = reinterpret_cast<int*>(base + o_j);
  float* d_A = reinterpret_cast<float*>(base + o_A);
  float* d_B = reinterpret_cast<float*>(base + o_B);
  float* d_part = reinterpret_cast<float*>(base + o_part);
  // the array keeps the previous call's contents: set everything that is read
  k_store_prop<<<1, 1, 0, st>>>(d_prop, pd);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(d_pidx, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_S, 0, std::max(1, off), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_node, 0, M * sizeof(int), st);
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return MNBAB_E_DEVICE;
  }
  k_iota<<<(n_rows + 255) / 256, 256, 0, st>>>(d_j, n_rows);
  // one node (slot 0) whose bounds are the caller's l, u and whose splits are none
  PoolDev pool{};
  pool.SD = off;
  pool.EC = 0;
  pool.d0 = dims[0];
  pool.L = const_cast<float*>(l);
  pool.U = const_cast<float*>(u);
  pool.S = d_S;
  pool.prop = d_pidx;
  auto epi_for = [&](int layer) {
    Epi ep{};
    ep.SD = off;
    ep.d0 = dims[0];
    ep.row_node = d_node;
    ep.pool = pool;
    ep.props = d_prop;
    ep.part = d_part;
    ep.nslot = nslot;
    ep.bias_div = 1;
    ep.gemm_path = 1;  // SIMT kernels: no error flag to report through
    if (layer >= 1) {
      ep.kind = EPI_RELU;
      ep.layer = layer;
      ep.off = nd.off[layer];
      ep.bias = nd.aff[layer].b;
    } else {
      ep.kind = EPI_CONC;
    }
    return ep;
  };
  // DeepPoly pass: heuristic slopes, no splits, no multipliers
  RowsDev rows{n_rows, d_node, d_j, nullptr};
  Epi e0 = epi_for(R);
  e0.slot_base = 0;
  float* cur = d_A;
  float* nxt = d_B;
  launch_init_rows(nd, R + 1, 0, rows, R >= 1 ? cur : nullptr, maxd, e0, st);
  int used = 1;
  for (int i = R; i >= 1; --i) {
    Epi ei = epi_for(i - 1);
    ei.slot_base = used;
    used += launch_backsub(nd.aff[i], n_rows, cur, maxd, i - 1 >= 1 ? nxt : nullptr, maxd, ei, st);
    std::swap(cur, nxt);
  }
  launch_reduce_lb(n_rows, d_part, nslot, used, nullptr, lb_out, false, d_node, pool, nullptr,
                   dims[0], st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return MNBAB_E_DEVICE;
  }
  set_err(err, err_len, "");
  return MNBAB_OK;
}
