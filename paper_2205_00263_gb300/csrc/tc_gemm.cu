// Tensor-core (tcgen05, sm_103a) GEMM with 3xTF32 split products and the
// fused back-substitution epilogues: the dense affine steps Lambda . W (Sec. 3.1,
// affine back-substitution) and G . W^T + b (adjoint / forward sweeps).
//
// C[M][N] = A[M][K] . B^T with A row-major (K contiguous) and B given as
// [N][K] (K contiguous); both operands are "K-major" for the MMA.  Every FP32
// value x is split into hi = tf32(x) and lo = tf32(x - hi); the product uses
// hi.hi + hi.lo + lo.hi accumulated in FP32 in tensor memory, which keeps FP32
// accuracy (the dropped lo.lo term is below 2^-22 relative).
//
// One CTA = 16 warps computes a 128 x BN tile.  Per K block of 32, the threads
// load A and B, split them and store the four tiles in the no-swizzle
// canonical K-major layout (8-row x 16-byte core matrices; adjacent core
// matrices along K are LBO = 128 B apart, along M/N SBO = 1024 B apart); one
// thread issues 4 k-steps x 3 tcgen05.mma (K = 8 each) and commits them to the
// stage's mbarrier.  Two stages: the threads load and split block k + 1 while
// the tensor core works on block k.  The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31 = tile rows) and applies the same epilogue functions
// as the SIMT kernels; each thread owns one row, so the row partial sums of
// the offset need no cross-thread reduction.
//
// The weight operand of an FC layer is constant: it is split into hi / lo once
// at load_network, arranged as [N/8][K/4][8][4] (core-matrix-major) and loaded
// per block by TMA (cp.async.bulk.tensor, a 3-D tensor map whose box lands in
// exactly the canonical layout above); the staging threads then split only
// the coefficient rows A.  Without pre-split weights both operands are staged.
//
// Every wait on the mbarrier is bounded: on timeout the kernel records an
// error, waits once more (bounded) for its own MMAs, frees its tensor memory
// and returns.
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

constexpr int TBM = 128;  // tile rows (TMEM lanes)
constexpr int TBK = 32;   // K per staged block (4 MMAs of K = 8)
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// canonical no-swizzle K-major offset (bytes) of element (r, k) in a tile with
// TBK = 32 K-columns: 8 core matrices of 128 B along K per 8-row group
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 1024;
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, LBO mode 0, layout type 0 = no swizzle
  return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

template <int N>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// Loads the 128-or-BN-row x 32 K block of a K-major operand starting at
// (row0, k0), splits it into TF32 hi / lo and stores both in the canonical
// layout.  Vector path: a lane loads 4 consecutive K values (16 B) and stores 16 B
// per part; lanes 0-7 of each quarter-warp take 8 consecutive rows at the same
// K quad (conflict-free 16-byte shared stores), the quarter-warps 4 K quads
// (64 contiguous bytes per row in global memory).
constexpr int TC_THREADS = 512;  // 16 warps: loads in flight while staging

template <int ROWS>
__device__ __forceinline__ void tc_stage(const float* __restrict__ X, int ld, int nrows, int K,
                                         int row0, int k0, bool vec, unsigned char* hi,
                                         unsigned char* lo) {
  const int tid = threadIdx.x;
  if (vec) {
    constexpr int NQ = ROWS * TBK / 4;  // float4 per block
#pragma unroll 4
    for (int q = tid; q < NQ; q += TC_THREADS) {
      const int lane = q & 31, w = q >> 5;
      const int r = (w >> 1) * 8 + (lane & 7);
      const int k4 = (w & 1) * 4 + (lane >> 3);
      const int gr = row0 + r, gk = k0 + 4 * k4;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < nrows && gk < K) x = __ldg(reinterpret_cast<const float4*>(X + (size_t)gr * ld + gk));
      uint4 h, l;
      h.x = to_tf32(x.x);
      l.x = to_tf32(x.x - __uint_as_float(h.x));
      h.y = to_tf32(x.y);
      l.y = to_tf32(x.y - __uint_as_float(h.y));
      h.z = to_tf32(x.z);
      l.z = to_tf32(x.z - __uint_as_float(h.z));
      h.w = to_tf32(x.w);
      l.w = to_tf32(x.w - __uint_as_float(h.w));
      const uint32_t o = tile_off(r, 4 * k4);
      *reinterpret_cast<uint4*>(hi + o) = h;
      *reinterpret_cast<uint4*>(lo + o) = l;
    }
    return;
  }
  for (int q = tid; q < ROWS * TBK; q += TC_THREADS) {
    const int r = q >> 5, k = q & 31;
    const int gr = row0 + r, gk = k0 + k;
    const float x = (gr < nrows && gk < K) ? X[(size_t)gr * ld + gk] : 0.f;
    const uint32_t h = to_tf32(x);
    const uint32_t l = to_tf32(x - __uint_as_float(h));
    const uint32_t o = tile_off(r, k);
    *reinterpret_cast<uint32_t*>(hi + o) = h;
    *reinterpret_cast<uint32_t*>(lo + o) = l;
  }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const __grid_constant__ CUtensorMap tm_hi,
                                                 const __grid_constant__ CUtensorMap tm_lo,
                                                 int use_tma,
                                                 int M, int N, int K, const float* __restrict__ A,
                                                 int lda, const float* __restrict__ B, int ldb,
                                                 const float* __restrict__ bias, int bias_div,
                                                 float* C, int ldc, Epi e, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // two stages of 1024-aligned tiles: A_hi, A_lo (128 x 32), B_hi, B_lo (BN x 32)
  constexpr int STAGE = 2 * TBM * TBK * 4 + 2 * BN * TBK * 4;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * STAGE);  // mma[2], tma[2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 4);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
  const uint32_t bar0 = smem_u32(bar), bar1 = smem_u32(bar + 1);
  const bool vecA = (lda & 3) == 0 && (K & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const bool vecB = (ldb & 3) == 0 && (K & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t tma0 = smem_u32(bar + 2);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1));
    tc::mbar_init(tma0, 1);
    tc::mbar_init(tma0 + 8, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  constexpr uint32_t idesc = idesc_tf32(BN);

  // block kb uses stage kb & 1 and commits to that stage's barrier; before a
  // stage is refilled, the MMAs of the block that last used it (kb - 2) must be
  // done: that barrier's ((kb >> 1) - 1)-th completion
  const int nk = (K + TBK - 1) / TBK;
  bool ok = true;
  int last = -1;  // last committed block
  for (int kb = 0; kb < nk; ++kb) {
    const int st = kb & 1;
    const uint32_t bst = st ? bar1 : bar0;
    if (kb >= 2) {
      const bool mine = mbar_wait(bst, (uint32_t)(((kb >> 1) - 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      ok = __syncthreads_and(mine && s_fail == 0) != 0;  // uniform across the CTA
      if (!ok) break;
    }
    unsigned char* a_hi = base + st * STAGE;
    unsigned char* a_lo = a_hi + TBM * TBK * 4;
    unsigned char* b_hi = a_lo + TBM * TBK * 4;
    unsigned char* b_lo = b_hi + BN * TBK * 4;
    const int k0 = kb * TBK;
    const uint32_t tbar = tma0 + 8 * st;
    if (use_tma) {
      if (tid == 0) {
        // the pre-split weight block [n0 / 8 .. + BN / 8) x [k0 / 4 .. + 8) by TMA;
        // rows past N read as zeros
        tc::mbar_expect_tx(tbar, 2 * BN * TBK * 4);
        tc::tma_load_3d(smem_u32(b_hi), &tm_hi, 0, k0 / 4, n0 / 8, tbar);
        tc::tma_load_3d(smem_u32(b_lo), &tm_lo, 0, k0 / 4, n0 / 8, tbar);
      }
    } else {
      tc_stage<BN>(B, ldb, N, K, n0, k0, vecB, b_hi, b_lo);
    }
    tc_stage<TBM>(A, lda, M, K, m0, k0, vecA, a_hi, a_lo);
    // make the generic-proxy smem writes visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && use_tma && !tc::mbar_wait(tbar, (uint32_t)((kb >> 1) & 1))) s_fail = 1;
    if (tid == 0 && s_fail == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
      const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
      for (int ks = 0; ks < TBK / 8; ++ks) {
        const uint32_t off = ks * 256;  // two core matrices of K per MMA
        const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, smem_desc(al + off), smem_desc(bh + off), idesc, first);
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, 1u);
      }
    }
    if (tid == 0)  // also when nothing was issued: keeps the phases in step
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bst)
          : "memory");
    last = kb;
  }
  if (ok && last >= 0) {
    // the last commit covers every MMA issued before it
    const bool mine = mbar_wait(last & 1 ? bar1 : bar0, (uint32_t)((last >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(mine && s_fail == 0) != 0;
  }
  if (!ok) {
    // record the timeout, then give the MMAs in flight one more bounded wait
    // before the tensor memory they write is released
    if (tid == 0) {
      atomicExch(err, 1);
      if (last >= 0) mbar_wait(last & 1 ? bar1 : bar0, (uint32_t)((last >> 1) & 1));
    }
    __syncthreads();
  }
  __shared__ float cpart[4][TBM];  // row partials of the four column groups
  constexpr int CTS = BN + 1;       // output tile row stride (floats)
  float* ctile = reinterpret_cast<float*>(base);
  if (ok) {
    // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (tile rows, one
    // per thread) and column group w / 4 (BN / 4 columns)
    const int quarter = warp & 3, cg = warp >> 2;
    const int m = m0 + quarter * 32 + lane;
    float part = 0.f;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    // the finished tile goes through shared memory (the operand stages, idle now
    // that every MMA has completed) so that its global stores are coalesced
    for (int c0 = cg * (BN / 4); c0 < (cg + 1) * (BN / 4); c0 += 16) {
      float v[16];
      tmem_ld16<16>(trow + (uint32_t)c0, v);
      if (m < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = n0 + c0 + i;
          if (n < N) {
            float x = v[i];
            if (bias) x += bias[n / bias_div];
            const float o = epi_apply(e, m, n, x, part);
            if (C) ctile[(quarter * 32 + lane) * CTS + c0 + i] = o;
          }
        }
      }
    }
    cpart[cg][quarter * 32 + lane] = part;
  }
  __syncthreads();
  if (ok && C) {
    for (int q = tid; q < TBM * BN; q += TC_THREADS) {
      const int r = q / BN, c = q % BN;
      const int m = m0 + r, n = n0 + c;
      if (m < M && n < N) C[(size_t)m * ldc + n] = ctile[r * CTS + c];
    }
  }
  if (ok && warp < 4 && epi_has_part(e)) {
    const int r = warp * 32 + lane, m = m0 + r;
    if (m < M)
      e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] =
          ((cpart[0][r] + cpart[1][r]) + cpart[2][r]) + cpart[3][r];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)BN));
  }
}

template <int BN>
static constexpr int tc_smem_bytes() {
  return 1024 + 2 * (2 * TBM * TBK * 4 + 2 * BN * TBK * 4) + 64;
}

// Pre-split weight operands of an FC layer: dir 0 B = W [d_out][d_in]
// (forward), dir 1 B = W^T [d_in][d_out] (back-substitution), each as hi / lo
// arrays [Np / 8][Kp / 4][8][4] with their tensor maps.
struct TcFc {
  bool ok[2] = {false, false};
  int N[2] = {0, 0}, K[2] = {0, 0};
  CUtensorMap hi[2], lo[2];
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
int fc_kp(int K) { return (K + TBK - 1) / TBK * TBK; }

}  // namespace

size_t tc_fc_floats(const LayerDev& L) {
  if (L.kind != MNBAB_FC) return 0;
  return 2 * ((size_t)fc_np(L.d_out) * fc_kp(L.d_in) + (size_t)fc_np(L.d_in) * fc_kp(L.d_out));
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
    // {32 floats = one 8 x 4 core matrix, Kp / 4, Np / 8}; a box is one
    // K block (8 core matrices along K) of up to 32 row groups (BN <= 256)
    const cuuint64_t gdim[3] = {32, (cuuint64_t)Kp / 4, (cuuint64_t)Np / 8};
    const cuuint64_t gstr[2] = {128, (cuuint64_t)(Kp / 4) * 128};
    bool good = true;
    const cuuint32_t es[3] = {1, 1, 1};
    // box height = the tile width launch_gemm_tc takes for this N
    const int BN = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    const cuuint32_t box[3] = {32, (cuuint32_t)TBK / 4, (cuuint32_t)BN / 8};
    for (int part = 0; part < 2 && good; ++part)
      good = enc(part == 0 ? &t->hi[dir] : &t->lo[dir], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                 part == 0 ? hi : lo, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (!good) continue;
    t->ok[dir] = true;
    t->N[dir] = N;
    t->K[dir] = K;
  }
  return t;
}

void tc_fc_destroy(TcFc* t) { delete t; }

template <int BN>
static int launch_bn(const TcFc* pre, int dir, int M, int N, int K, const float* A, int lda,
                     const float* B, int ldb, const float* bias, int bias_div, float* C, int ldc,
                     const Epi& e, int* err, cudaStream_t st) {
  constexpr int smem = tc_smem_bytes<BN>();
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  dim3 grid((N + BN - 1) / BN, (M + TBM - 1) / TBM);
  // the maps are built for this tile width (N decides BN on both sides)
  const bool tma = pre && pre->ok[dir] && pre->N[dir] == N && pre->K[dir] == K;
  static CUtensorMap none{};
  k_gemm_tc<BN><<<grid, TC_THREADS, smem, st>>>(tma ? pre->hi[dir] : none,
                                                tma ? pre->lo[dir] : none, tma ? 1 : 0, M, N, K,
                                                A, lda, B, ldb, bias, bias_div, C, ldc, e, err);
  return grid.x;
}

// Tile width: the smallest of 64 / 128 / 256 that covers N in one tile, else 256.
int launch_gemm_tc(int M, int N, int K, const float* A, int lda, const float* Bnk, int ldb,
                   const float* bias, int bias_div, float* C, int ldc, const Epi& e, int* err,
                   cudaStream_t st, const void* pre, int dir) {
  const TcFc* p = static_cast<const TcFc*>(pre);
  if (N <= 64)
    return launch_bn<64>(p, dir, M, N, K, A, lda, Bnk, ldb, bias, bias_div, C, ldc, e, err, st);
  if (N <= 128)
    return launch_bn<128>(p, dir, M, N, K, A, lda, Bnk, ldb, bias, bias_div, C, ldc, e, err, st);
  return launch_bn<256>(p, dir, M, N, K, A, lda, Bnk, ldb, bias, bias_div, C, ldc, e, err, st);
}

}  // namespace mnbab
