// Tensor-core (tcgen05, sm_103a) GEMM with 3xTF32 split products and the
// fused back-substitution epilogues: the dense affine steps Lambda . W (Sec. 3.1,
// affine back-substitution) and G . W^T + b (adjoint / forward sweeps).
//
// C[M][N] = A[M][K] . B^T with A the coefficient rows (K contiguous) and B
// given as [N][K]; both operands are "K-major" for the MMA.  Every FP32 value
// x is split into hi = tf32(x) and lo = tf32(x - hi); the product uses
// hi.hi + hi.lo + lo.hi accumulated in FP32 in tensor memory, which keeps FP32
// accuracy (the dropped lo.lo term is below 2^-22 relative).
//
// Both operands reach shared memory by TMA only (cp.async.bulk.tensor):
//  - the weight operand of an FC layer is constant: it is split into hi / lo
//    once at load_network;
//  - the coefficient rows A are split by a streaming kernel right before the
//    GEMM into a workspace of the network;
// both in the core-matrix-major order [rows / 8][K / 4][8][4], so that a 3-D
// box of a tensor map lands in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices; along K 128 B apart, 8-row groups
// PBK / 4 x 128 B apart).
//
// A CTA computes a 128 x BN tile with warp-specialised roles over a ring of
// STAGES shared-memory stages (K = 16 per stage):
//  - one thread of warp 0 (producer) waits until a stage is free and issues
//    the four TMA loads (A hi / lo, B hi / lo) onto the stage's "full" barrier;
//  - one thread of warp 1 (MMA issuer) waits on "full", issues 2 k-steps x 3
//    tcgen05.mma (K = 8 each, accumulating in tensor memory) and commits them
//    to the stage's "empty" barrier, which frees the stage for the producer;
//    after the last stage it commits to the "done" barrier;
//  - all 16 warps then read the accumulator with tcgen05.ld (warp w: TMEM
//    lanes 32 (w mod 4) + 0..31 = tile rows, column group w / 4) into shared
//    memory, and apply the same epilogue functions as the SIMT kernels row by
//    row, lanes on consecutive columns (coalesced per-neuron loads and
//    stores; a row's offset partial is a fixed-order warp reduction).
// Every wait is bounded: a role that gives up records the failure, the MMA
// issuer still commits "done" (it arrives once the MMAs issued so far have
// completed), the producer waits (bounded) for the loads it issued that were
// never consumed, the kernel sets the device error flag and frees its tensor
// memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

#include "epilogue.cuh"
#include "mnbab.h"
#include "mnbab_internal.h"
#include "tc_common.cuh"

namespace mnbab {

namespace {

constexpr int TBM = 128;        // tile rows (TMEM lanes)
constexpr int PBK = 16;         // K per pipeline stage (2 MMAs of K = 8)
constexpr int P_THREADS = 512;  // 16 warps: roles in warps 0 / 1, all 16 in the epilogue
constexpr int SMEM_STAGES = 200 * 1024;

template <int BN>
struct Pipe {
  static constexpr int A_BYTES = TBM * PBK * 4;  // one part (hi or lo)
  static constexpr int B_BYTES = BN * PBK * 4;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int STAGES = SMEM_STAGES / STAGE < 8 ? SMEM_STAGES / STAGE : 8;
  static constexpr int CTS = BN + 1;  // epilogue tile row stride (floats)
  static constexpr int SMEM = 1024 + STAGES * STAGE + 8 * (2 * STAGES + 1) + 16;
  static_assert(TBM * CTS * 4 <= STAGES * STAGE, "epilogue tile exceeds the stage ring");
};

// stage s of the ring: A hi, A lo, B hi, B lo
template <int BN>
__device__ __forceinline__ unsigned char* stage_ptr(unsigned char* base, int s) {
  return base + s * Pipe<BN>::STAGE;
}

template <int BN>
__global__ void __launch_bounds__(P_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
              const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
              int M, int N, int K, const float* __restrict__ bias, int bias_div, float* C,
              int ldc, Epi e, int* err) {
  using P = Pipe<BN>;
  constexpr int S = P::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + S * P::STAGE);  // full[S], empty[S], done
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 2 * S + 1);
  __shared__ int s_fail, s_issued, s_consumed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
  const uint32_t full0 = tc::smem_u32(bar), empty0 = full0 + 8 * S, done = full0 + 16 * S;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(tmem_holder)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 2 * S + 1; ++i) tc::mbar_init(full0 + 8 * i, 1);
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const int nk = (K + PBK - 1) / PBK;
  volatile int* vfail = &s_fail;

  if (warp == 0) {
    if (lane == 0) {
      // producer: stage kb % S; its (kb / S)-th refill waits for the MMAs of
      // block kb - S (that stage's empty barrier, completion kb / S - 1)
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        if (kb >= S && !tc::mbar_wait(empty0 + 8 * s, (uint32_t)((kb / S - 1) & 1))) {
          *vfail = 1;
          break;
        }
        if (*vfail) break;
        const uint32_t fb = full0 + 8 * s;
        unsigned char* st = stage_ptr<BN>(base, s);
        tc::mbar_expect_tx(fb, (uint32_t)P::STAGE);
        const int kq = kb * (PBK / 4);
        tc::tma_load_3d(tc::smem_u32(st), &ta_hi, 0, kq, m0 / 8, fb);
        tc::tma_load_3d(tc::smem_u32(st + P::A_BYTES), &ta_lo, 0, kq, m0 / 8, fb);
        tc::tma_load_3d(tc::smem_u32(st + 2 * P::A_BYTES), &tb_hi, 0, kq, n0 / 8, fb);
        tc::tma_load_3d(tc::smem_u32(st + 2 * P::A_BYTES + P::B_BYTES), &tb_lo, 0, kq, n0 / 8, fb);
        issued = kb + 1;
      }
      s_issued = issued;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = tc::idesc_tf32_m128(BN);
      constexpr uint32_t SBO = (PBK / 4) * 128;  // 8-row groups
      int consumed = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % S;
        if (!tc::mbar_wait(full0 + 8 * s, (uint32_t)((kb / S) & 1))) {
          *vfail = 1;
          break;
        }
        if (*vfail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* st = stage_ptr<BN>(base, s);
        const uint32_t ah = tc::smem_u32(st), al = ah + P::A_BYTES;
        const uint32_t bh = ah + 2 * P::A_BYTES, bl = bh + P::B_BYTES;
#pragma unroll
        for (int ks = 0; ks < PBK / 8; ++ks) {
          const uint32_t o = ks * 256;  // two core matrices along K per MMA
          const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(tmem, tc::smem_desc(al + o, 128, SBO), tc::smem_desc(bh + o, 128, SBO),
                       idesc, first);
          tc::mma_tf32(tmem, tc::smem_desc(ah + o, 128, SBO), tc::smem_desc(bl + o, 128, SBO),
                       idesc, 1u);
          tc::mma_tf32(tmem, tc::smem_desc(ah + o, 128, SBO), tc::smem_desc(bh + o, 128, SBO),
                       idesc, 1u);
        }
        tc::mma_commit(empty0 + 8 * s);
        consumed = kb + 1;
      }
      // arrives once every MMA issued above has completed (at once if none)
      tc::mma_commit(done);
      s_consumed = consumed;
    }
    __syncwarp();
  }
  const bool mine = tc::mbar_wait(done, 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = __syncthreads_and(mine && *vfail == 0) != 0;
  if (!ok) {
    if (tid == 0) {
      // loads issued but never consumed still write this CTA's shared memory
      for (int i = s_consumed; i < s_issued; ++i)
        tc::mbar_wait(full0 + 8 * (i % S), (uint32_t)((i / S) & 1));
      atomicExch(err, 1);
    }
    __syncthreads();
  }
  if (ok) {
    // epilogue: every MMA has completed and every load landed, so the stage
    // ring holds the output tile.  First the accumulator goes to shared
    // memory (warp w: TMEM lanes 32 (w mod 4) + lane = tile rows, column
    // group w / 4); then each warp takes whole rows, lanes on consecutive columns,
    // so that the epilogue's per-neuron loads and the stores are coalesced.
    float* ctile = reinterpret_cast<float*>(base);
    {
      constexpr int NG = P_THREADS / 128, CW = BN / NG;  // column groups of the warps
      const int quarter = warp & 3, grp = warp >> 2;
      const int r = quarter * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = grp * CW; c0 < (grp + 1) * CW; c0 += 16) {
        float v[16];
        tc::tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) ctile[r * P::CTS + c0 + i] = v[i];
      }
    }
    __syncthreads();
    const bool has_part = epi_has_part(e);
    const bool per_node = e.kind == EPI_RELU || e.kind == EPI_ADJ || e.kind == EPI_CONC;
    constexpr int PER = BN / 32;                 // columns per lane of a row
    constexpr int RPW = TBM / (P_THREADS / 32);  // rows per warp
    // per-column inputs of this lane's columns, once per tile
    float cb[PER], gb[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int n = n0 + lane + 32 * i;
      cb[i] = n < N ? epi_colbias(e, n) : 0.f;
      gb[i] = (bias && n < N) ? bias[n / bias_div] : 0.f;
    }
    // the nodes of this warp's rows warp + 16 t: lane t loads row t's
    int my_nd = 0;
    if (per_node && lane < RPW && m0 + warp + 16 * lane < M)
      my_nd = e.row_node[m0 + warp + 16 * lane];
    // a warp's rows of one node (consecutive rows of a batch usually are) share
    // the node's per-column inputs: they are loaded when the node changes
    EpiIn in[PER];
    int have = -1;
#pragma unroll 1
    for (int t = 0; t < RPW; ++t) {
      const int rr = warp + 16 * t, m = m0 + rr;
      const int nd = __shfl_sync(0xffffffffu, my_nd, t);
      if (m >= M) break;  // rows ascend with t
      // every global load of the row's outputs in flight before the arithmetic
      if (nd != have || !per_node) {
        const PropDev* Pp = epi_prop(e, nd);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
          const int n = n0 + lane + 32 * i;
          if (n < N) epi_load_node(e, nd, Pp, n, in[i]);
          in[i].cb = cb[i];
        }
        have = nd;
      }
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int n = n0 + lane + 32 * i;
        if (n < N) epi_load_own(e, m, n, in[i]);
      }
      float part = 0.f;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int cc = lane + 32 * i, n = n0 + cc;
        if (n < N) {
          const float o = epi_finish(e, m, n, ctile[rr * P::CTS + cc] + gb[i], in[i], part);
          if (C) C[(size_t)m * ldc + n] = o;
        }
      }
      if (has_part) {
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = part;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN));
  }
}

// Rows of X [rows][K] (leading dimension ld) split into TF32 hi / lo in the
// core-matrix-major order [Rg / 8][Kp / 4][8][4]; rows >= rows and columns
// >= K are zero.  Thread q writes 16 bytes of each part (consecutive q,
// consecutive addresses).
__global__ void k_split_rows(const float* __restrict__ X, int ld, int rows, int K, int Rg, int Kp,
                             int vec, float* __restrict__ hi, float* __restrict__ lo) {
  const int kq4 = Kp / 4;
  const size_t total = (size_t)Rg * kq4;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int r8 = (int)(q & 7);
    const size_t gq = q >> 3;
    const int kq = (int)(gq % kq4);
    const int g = (int)(gq / kq4);
    const int r = g * 8 + r8, k = kq * 4;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < rows) {
      const float* src = X + (size_t)r * ld + k;
      if (vec && k + 3 < K) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(src));
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (k + i < K) x[i] = src[i];
      }
    }
    uint4 h, l;
    h.x = tc::to_tf32(x[0]);
    l.x = tc::to_tf32(x[0] - __uint_as_float(h.x));
    h.y = tc::to_tf32(x[1]);
    l.y = tc::to_tf32(x[1] - __uint_as_float(h.y));
    h.z = tc::to_tf32(x[2]);
    l.z = tc::to_tf32(x[2] - __uint_as_float(h.z));
    h.w = tc::to_tf32(x[3]);
    l.w = tc::to_tf32(x[3] - __uint_as_float(h.w));
    reinterpret_cast<uint4*>(hi)[q] = h;
    reinterpret_cast<uint4*>(lo)[q] = l;
  }
}

}  // namespace

// Pre-split weight operands of an FC layer: dir 0 B = W [d_out][d_in]
// (forward products), dir 1 B = W^T [d_in][d_out] (back-substitution), each as
// hi / lo arrays [Np / 8][Kp / 4][8][4] with their tensor maps, and the
// network's workspace for the split coefficient rows.
struct TcFc {
  bool ok[2] = {false, false};
  int N[2] = {0, 0}, K[2] = {0, 0}, Kp[2] = {0, 0};
  CUtensorMap hi[2], lo[2];
  float* ws = nullptr;
  size_t ws_floats = 0;
};

namespace {

__global__ void k_fc_split(const float* __restrict__ B, int N, int K, int Np, int Kp, float* hi,
                           float* lo) {
  const size_t total = (size_t)Np * Kp;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(q / Kp), k = (int)(q % Kp);
    const float w = (n < N && k < K) ? B[(size_t)n * K + k] : 0.f;
    const uint32_t h = tc::to_tf32(w);
    const uint32_t l = tc::to_tf32(w - __uint_as_float(h));
    const size_t o = (((size_t)(n >> 3) * (Kp / 4) + (k >> 2)) * 8 + (n & 7)) * 4 + (k & 3);
    hi[o] = __uint_as_float(h);
    lo[o] = __uint_as_float(l);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 fc_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int fc_np(int N) { return (N + 7) / 8 * 8; }
int fc_kp(int K) { return (K + PBK - 1) / PBK * PBK; }
int fc_bn(int N) { return N <= 64 ? 64 : (N <= 128 ? 128 : 256); }

// A [groups of 8 rows][Kp / 4][8][4] array as a 3-D tensor {32 floats = one
// core matrix, Kp / 4, groups}; a box is one K block (PBK / 4 core matrices
// along K) of `box_rows` / 8 row groups
bool encode_split(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, float* ptr, int groups,
                  int Kp, int box_rows) {
  const cuuint64_t gdim[3] = {32, (cuuint64_t)Kp / 4, (cuuint64_t)groups};
  const cuuint64_t gstr[2] = {128, (cuuint64_t)(Kp / 4) * 128};
  const cuuint32_t box[3] = {32, (cuuint32_t)PBK / 4, (cuuint32_t)box_rows / 8};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr, gdim, gstr, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_fc_floats(const LayerDev& L) {
  if (L.kind != MNBAB_FC) return 0;
  return 2 * ((size_t)fc_np(L.d_out) * fc_kp(L.d_in) + (size_t)fc_np(L.d_in) * fc_kp(L.d_out));
}

size_t tc_fc_workspace_floats(const LayerDev& L, int max_rows) {
  if (L.kind != MNBAB_FC) return 0;
  const size_t rg = (size_t)(max_rows + 7) / 8 * 8;
  return 2 * rg * (size_t)std::max(fc_kp(L.d_in), fc_kp(L.d_out));
}

TcFc* tc_fc_create(const LayerDev& L, float* buf, cudaStream_t st) {
  if (L.kind != MNBAB_FC || !buf || !L.W || !L.Wt) return nullptr;
  PFN_cuTensorMapEncodeTiled_v12000 enc = fc_encode_fn();
  if (!enc) return nullptr;
  TcFc* t = new TcFc();
  size_t at = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const float* B = dir == 0 ? L.W : L.Wt;
    const int N = dir == 0 ? L.d_out : L.d_in, K = dir == 0 ? L.d_in : L.d_out;
    const int Np = fc_np(N), Kp = fc_kp(K);
    float* hi = buf + at;
    float* lo = hi + (size_t)Np * Kp;
    at += 2 * (size_t)Np * Kp;
    const int blocks = (int)std::min<size_t>(4096, ((size_t)Np * Kp + 255) / 256);
    k_fc_split<<<blocks, 256, 0, st>>>(B, N, K, Np, Kp, hi, lo);
    // box height = the tile width launch_gemm_tc takes for this N
    const int BN = fc_bn(N);
    if (!encode_split(enc, &t->hi[dir], hi, Np / 8, Kp, BN) ||
        !encode_split(enc, &t->lo[dir], lo, Np / 8, Kp, BN))
      continue;
    t->ok[dir] = true;
    t->N[dir] = N;
    t->K[dir] = K;
    t->Kp[dir] = Kp;
  }
  return t;
}

void tc_fc_set_workspace(TcFc* t, float* ws, size_t floats) {
  if (!t) return;
  t->ws = ws;
  t->ws_floats = floats;
}

void tc_fc_destroy(TcFc* t) { delete t; }

template <int BN>
static int launch_bn(const TcFc* t, int dir, int M, int N, int K, const float* A, int lda,
                     const float* bias, int bias_div, float* C, int ldc, const Epi& e, int* err,
                     cudaStream_t st) {
  constexpr int smem = Pipe<BN>::SMEM;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  // split the coefficient rows into the workspace, then the GEMM
  const int Kp = t->Kp[dir];
  const int Rg = (M + 7) / 8 * 8;
  float* hi = t->ws;
  float* lo = hi + (size_t)Rg * Kp;
  const int vec = (lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
  const size_t quads = (size_t)Rg * (Kp / 4);
  const int blocks = (int)std::min<size_t>(152 * 16, (quads + 255) / 256);
  k_split_rows<<<blocks, 256, 0, st>>>(A, lda, M, K, Rg, Kp, vec, hi, lo);
  CUtensorMap ta_hi, ta_lo;
  PFN_cuTensorMapEncodeTiled_v12000 enc = fc_encode_fn();
  if (!encode_split(enc, &ta_hi, hi, Rg / 8, Kp, TBM) ||
      !encode_split(enc, &ta_lo, lo, Rg / 8, Kp, TBM))
    return -1;
  dim3 grid((N + BN - 1) / BN, (M + TBM - 1) / TBM);
  k_gemm_tc<BN><<<grid, P_THREADS, smem, st>>>(ta_hi, ta_lo, t->hi[dir], t->lo[dir], M, N, K,
                                               bias, bias_div, C, ldc, e, err);
  return grid.x;
}

int launch_gemm_tc(int M, int N, int K, const float* A, int lda, const float* bias, int bias_div,
                   float* C, int ldc, const Epi& e, int* err, cudaStream_t st, const void* pre,
                   int dir) {
  const TcFc* t = static_cast<const TcFc*>(pre);
  if (M <= 0 || !t || !t->ok[dir] || t->N[dir] != N || t->K[dir] != K || !t->ws) return -1;
  if (2 * (size_t)((M + 7) / 8 * 8) * t->Kp[dir] > t->ws_floats) return -1;
  switch (fc_bn(N)) {
    case 64: return launch_bn<64>(t, dir, M, N, K, A, lda, bias, bias_div, C, ldc, e, err, st);
    case 128: return launch_bn<128>(t, dir, M, N, K, A, lda, bias, bias_div, C, ldc, e, err, st);
    default: return launch_bn<256>(t, dir, M, N, K, A, lda, bias, bias_div, C, ldc, e, err, st);
  }
}

}  // namespace mnbab
