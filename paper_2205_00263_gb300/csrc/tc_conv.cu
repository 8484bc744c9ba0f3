// Tensor-core (tcgen05) implicit-GEMM convolutions for the back-substitution
// sweeps (Sec. 3.1: the affine step through a convolution is its transposed
// convolution) and the adjoint / forward passes, with 3xTF32 split products
// and the fused epilogues of epilogue.cuh.
//
// Forward (dir 0): out[m, n, oy, ox] = sum over (ci, kh, kw) of
//   in[m, ci, oy s - p + kh, ox s - p + kw] W[n, ci, kh, kw] (+ b[n]).
// Transposed (dir 1), output positions with (y + p) mod s = ry and
// (x + p) mod s = rx (one stride class) take exactly the taps kh = ry + s a,
// kw = rx + s b: out[m, n, y, x] = sum over (o, a, b) of
//   in[m, o, (y + p - kh) / s, (x + p - kw) / s] W[o, n, kh, kw].
// Each class is a dense GEMM: rows = (objective row m, position), columns =
// channels n, reduction (ci, kh, kw) or (o, a, b).
//
// A CTA computes 128 GEMM rows = 4 objective rows x 32 positions of one class
// (warp w owns row m0 + w, lane = position), all N channels:
//  - B (weights) is pre-split into TF32 hi / lo once per layer, arranged per
//    class as [K / 4][N][4] in HBM and staged by TMA (a 3-D tiled tensor map,
//    cp.async.bulk.tensor), which lands it in the canonical no-swizzle K-major
//    layout (core matrices along K N x 16 B apart, along N 128 B apart);
//  - A is the implicit im2col operand: each thread gathers its position's 32
//    reduction values of a K block from the coefficient rows (L2), splits
//    them into hi / lo and stores them in the canonical layout;
//  - two stages: the threads gather block k + 1 while the tensor core runs
//    block k (3 MMAs of K = 8 per K step: hi.hi + hi.lo + lo.hi, FP32
//    accumulation in tensor memory);
//  - the epilogue reads each warp's 32 TMEM lanes (one objective row) with
//    tcgen05.ld and applies the same epilogue functions as the SIMT kernels;
//    a row's offset partial is a warp reduction in a fixed order, written to
//    slot (class, position chunk), so it does not depend on the other rows.
// Every wait is bounded; on timeout the kernel sets the device error flag,
// gives its MMAs one more bounded wait, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "epilogue.cuh"
#include "mnbab.h"
#include "mnbab_internal.h"
#include "tc_common.cuh"

namespace mnbab {

struct TcConv {
  bool ok[2] = {false, false};  // dir 0 forward, dir 1 transposed
  int N[2] = {0, 0}, NP[2] = {0, 0}, Kp[2] = {0, 0}, ncls[2] = {0, 0}, nchunk[2] = {0, 0};
  CUtensorMap hi[2], lo[2];
};

namespace {

constexpr int KC = 32;    // reduction values per staged block
constexpr int TROWS = 4;  // objective rows per CTA (one warp each)
constexpr int TC_KMAX = 1024;  // longest reduction (padded to KC) the kernel takes

struct ConvClass {
  int P, K;            // positions and reduction length of the class
  int y0, x0, nx;      // first output row / column of the class, columns of the class
  int ry, rx, na, nb;  // residues and tap counts (transposed)
};

__host__ __device__ inline ConvClass conv_class(const LayerDev& L, int dir, int cls) {
  ConvClass c;
  if (dir == 0) {
    c.P = L.ho * L.wo;
    c.K = L.ci * L.k * L.k;
    c.y0 = c.x0 = 0;
    c.nx = L.wo;
    c.ry = c.rx = 0;
    c.na = c.nb = L.k;
    return c;
  }
  const int s = L.s;
  c.ry = cls / s;
  c.rx = cls % s;
  c.y0 = ((c.ry - L.p) % s + s) % s;
  c.x0 = ((c.rx - L.p) % s + s) % s;
  const int ny = c.y0 < L.hi ? (L.hi - c.y0 + s - 1) / s : 0;
  c.nx = c.x0 < L.wi ? (L.wi - c.x0 + s - 1) / s : 0;
  c.na = c.ry < L.k ? (L.k - c.ry + s - 1) / s : 0;
  c.nb = c.rx < L.k ? (L.k - c.rx + s - 1) / s : 0;
  c.P = ny * c.nx;
  c.K = L.co * c.na * c.nb;
  return c;
}

// canonical no-swizzle K-major offset (bytes) of A element (r, k), KC = 32:
// core matrices along K 128 B apart, 8-row groups 1024 B apart
__device__ __forceinline__ uint32_t a_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// pre-split weights of one direction: buf_hi / buf_lo [ncls][Kp / 4][NP][4]
__global__ void k_tc_conv_split(LayerDev L, int dir, int Kp, int NP, float* hi, float* lo) {
  const int cls = blockIdx.y;
  const ConvClass c = conv_class(L, dir, cls);
  const int N = dir == 0 ? L.co : L.ci;
  const int total = Kp * NP;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int kk = q / NP, n = q % NP;
    float w = 0.f;
    if (n < N && kk < c.K) {
      if (dir == 0) {
        w = L.W[(size_t)n * c.K + kk];  // W [co][ci][kh][kw]: the reduction is contiguous
      } else {
        const int nab = c.na * c.nb;
        const int o = kk / nab, a = (kk / c.nb) % c.na, b = kk % c.nb;
        const int kh = c.ry + L.s * a, kw = c.rx + L.s * b;
        w = L.W[(((size_t)o * L.ci + n) * L.k + kh) * L.k + kw];
      }
    }
    const uint32_t h = tc::to_tf32(w);
    const uint32_t l = tc::to_tf32(w - __uint_as_float(h));
    const size_t o = (((size_t)cls * (Kp / 4) + kk / 4) * NP + n) * 4 + (kk & 3);
    hi[o] = __uint_as_float(h);
    lo[o] = __uint_as_float(l);
  }
}

constexpr int TC_THREADS = 256;  // 8 warps: two threads per GEMM row gather a K block

template <int NP>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const __grid_constant__ CUtensorMap tm_hi,
                                                        const __grid_constant__ CUtensorMap tm_lo,
                                                        LayerDev L, int dir, int M, int nchunk,
                                                        const float* __restrict__ in, int ld_in,
                                                        float* out, int ld_out, Epi e, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int A_BYTES = 128 * KC * 4;
  constexpr int B_BYTES = NP * KC * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t NCOLS = NP <= 32 ? 32 : 64;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * STAGE);  // tma[2], mma[2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 4);
  // reduction table of the whole K range, computed once: source offset
  // (channel plane + tap shift) and tap shifts for the bounds check
  // (dy = dx = -1000: padding past K)
  __shared__ int t_delta[TC_KMAX];
  __shared__ short2 t_dd[TC_KMAX];
  __shared__ int s_fail;
  __shared__ float s_part[2][TROWS];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rq = warp & 3;         // objective row of this warp (TMEM lane quarter)
  const int kh = warp >> 2;        // which half of a K block this warp gathers
  const int cls = blockIdx.x / nchunk, chunk = blockIdx.x % nchunk;
  const ConvClass c = conv_class(L, dir, cls);
  const int m = blockIdx.y * TROWS + rq;
  const int pos = chunk * 32 + lane;
  const bool rowv = m < M;
  const bool pv = rowv && pos < c.P;
  const int N = dir == 0 ? L.co : L.ci;
  const bool has_part = dir == 1 && epi_has_part(e);
  if (chunk * 32 >= c.P) {
    // no position of this class in the chunk: only the row partials (zero)
    if (has_part && kh == 0 && lane == 0 && rowv)
      e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = 0.f;
    return;
  }
  // this thread's position and the source plane of its gather
  const int iy = pv ? pos / c.nx : 0, ix = pv ? pos % c.nx : 0;
  int gy, gx;
  if (dir == 0) {
    gy = iy * L.s - L.p;
    gx = ix * L.s - L.p;
  } else {
    gy = (c.y0 + L.s * iy + L.p - c.ry) / L.s;
    gx = (c.x0 + L.s * ix + L.p - c.rx) / L.s;
  }
  const int Hs = dir == 0 ? L.hi : L.ho, Wsrc = dir == 0 ? L.wi : L.wo;
  const float* src = in + (size_t)(rowv ? m : 0) * ld_in + gy * Wsrc + gx;

  const uint32_t tma0 = tc::smem_u32(bar), mma0 = tc::smem_u32(bar + 2);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(tmem_holder)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(tma0 + 8 * i, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  constexpr uint32_t idesc = tc::idesc_tf32_m128(NP);

  const int nk = (c.K + KC - 1) / KC;
  for (int kidx = tid; kidx < nk * KC; kidx += TC_THREADS) {
    int delta = 0, dy = -1000, dx = -1000;
    if (kidx < c.K) {
      int off;
      if (dir == 0) {
        const int kk2 = L.k * L.k;
        off = (kidx / kk2) * L.hi * L.wi;
        dy = (kidx / L.k) % L.k;
        dx = kidx % L.k;
      } else {
        const int nab = c.na * c.nb;
        off = (kidx / nab) * L.ho * L.wo;
        dy = -((kidx / c.nb) % c.na);
        dx = -(kidx % c.nb);
      }
      delta = off + dy * Wsrc + dx;
    }
    t_delta[kidx] = delta;
    t_dd[kidx] = make_short2((short)dy, (short)dx);
  }
  __syncthreads();
  // implicit im2col: the 16 reduction values of this thread's GEMM row in K
  // block kb (half kh of the block)
  auto gather = [&](int kb, float (&v)[16]) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int kk = kb * KC + kh * 16 + u;
      const short2 dd = t_dd[kk];
      const int yy = gy + dd.x, xx = gx + dd.y;
      const bool in_b = pv && yy >= 0 && yy < Hs && xx >= 0 && xx < Wsrc;
      v[u] = in_b ? __ldg(src + t_delta[kk]) : 0.f;
    }
  };
  bool ok = true;
  int last = -1;
  float vn[16];
  if (nk > 0) gather(0, vn);
  for (int kb = 0; kb < nk; ++kb) {
    const int st = kb & 1;
    const uint32_t tbar = tma0 + 8 * st, mbar = mma0 + 8 * st;
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = vn[u];
    // the next block's loads are in flight while this block is staged and issued
    if (kb + 1 < nk) gather(kb + 1, vn);
    if (kb >= 2) {
      // the MMAs of block kb - 2 read this stage: wait for them
      const bool mine = tc::mbar_wait(mbar, (uint32_t)(((kb >> 1) - 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      ok = __syncthreads_and(mine && s_fail == 0) != 0;
    } else {
      ok = __syncthreads_and(s_fail == 0) != 0;
    }
    if (!ok) break;
    unsigned char* a_hi = base + st * STAGE;
    unsigned char* a_lo = a_hi + A_BYTES;
    unsigned char* b_hi = a_lo + A_BYTES;
    unsigned char* b_lo = b_hi + B_BYTES;
    if (tid == 0) {
      // weights of this K block (hi and lo) by TMA
      tc::mbar_expect_tx(tbar, 2 * B_BYTES);
      tc::tma_load_3d(tc::smem_u32(b_hi), &tm_hi, 0, kb * (KC / 4), cls, tbar);
      tc::tma_load_3d(tc::smem_u32(b_lo), &tm_lo, 0, kb * (KC / 4), cls, tbar);
    }
    const int r = rq * 32 + lane;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint4 h, l;
      h.x = tc::to_tf32(v[4 * q]);
      l.x = tc::to_tf32(v[4 * q] - __uint_as_float(h.x));
      h.y = tc::to_tf32(v[4 * q + 1]);
      l.y = tc::to_tf32(v[4 * q + 1] - __uint_as_float(h.y));
      h.z = tc::to_tf32(v[4 * q + 2]);
      l.z = tc::to_tf32(v[4 * q + 2] - __uint_as_float(h.z));
      h.w = tc::to_tf32(v[4 * q + 3]);
      l.w = tc::to_tf32(v[4 * q + 3] - __uint_as_float(h.w));
      const uint32_t o = a_off(r, kh * 16 + 4 * q);
      *reinterpret_cast<uint4*>(a_hi + o) = h;
      *reinterpret_cast<uint4*>(a_lo + o) = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (tc::mbar_wait(tbar, (uint32_t)((kb >> 1) & 1))) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = tc::smem_u32(a_hi), al = tc::smem_u32(a_lo);
        const uint32_t bh = tc::smem_u32(b_hi), bl = tc::smem_u32(b_lo);
        constexpr uint32_t BLBO = NP * 16;  // B: core matrices along K
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t ao = ks * 256, bo = ks * 2 * BLBO;
          const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
          tc::mma_tf32(tmem, tc::smem_desc(al + ao, 128, 1024), tc::smem_desc(bh + bo, BLBO, 128),
                       idesc, first);
          tc::mma_tf32(tmem, tc::smem_desc(ah + ao, 128, 1024), tc::smem_desc(bl + bo, BLBO, 128),
                       idesc, 1u);
          tc::mma_tf32(tmem, tc::smem_desc(ah + ao, 128, 1024), tc::smem_desc(bh + bo, BLBO, 128),
                       idesc, 1u);
        }
      } else {
        s_fail = 1;  // the weights never arrived: the next barrier stops the loop
      }
      tc::mma_commit(mbar);  // also when nothing was issued: keeps the phases in step
    }
    last = kb;
  }
  if (ok && last >= 0) {
    // the last commit covers every MMA issued before it
    const bool mine = tc::mbar_wait(mma0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(mine && s_fail == 0) != 0;
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(err, 1);
      if (last >= 0) tc::mbar_wait(mma0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1));
    }
    __syncthreads();
  }
  if (ok) {
    // epilogue: every warp reads its TMEM lane quarter (objective row rq); warp
    // group kh takes the 16-column chunks 16 (2 i + kh).  The inputs of four
    // outputs are loaded together before any of them is finished.
    float part = 0.f;
    const int y = dir == 0 ? iy : c.y0 + L.s * iy;
    const int x = dir == 0 ? ix : c.x0 + L.s * ix;
    const int plane = dir == 0 ? L.ho * L.wo : L.hi * L.wi;
    const int W2 = dir == 0 ? L.wo : L.wi;
    const int pj = y * W2 + x;
    const uint32_t trow = tmem + ((uint32_t)(rq * 32) << 16);
    const int nrow = pv ? e.row_node[m] : 0;
    const PropDev* Pp = pv ? epi_prop(e, nrow) : nullptr;
    for (int c0 = 16 * kh; c0 < NP; c0 += 32) {
      float v[16];
      if (nk > 0) {
        tc::tmem_ld16(trow + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;  // a class without taps
      }
      if (pv) {
#pragma unroll
        for (int g = 0; g < 16; g += 4) {
          EpiIn in[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int n = c0 + g + i;
            if (n < N) epi_load(e, nrow, Pp, m, n * plane + pj, in[i]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int n = c0 + g + i;
            if (n < N) {
              const int j = n * plane + pj;
              float val = v[g + i];
              if (dir == 0) val += L.b[n];
              const float o = epi_finish(e, m, j, val, in[i], part);
              if (out) out[(size_t)m * ld_out + j] = o;
            }
          }
        }
      }
    }
    if (has_part) {
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) s_part[kh][rq] = part;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // a row's offset partial: the two warp groups' sums, in that order
  if (ok && has_part && kh == 0 && lane == 0 && rowv)
    e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = s_part[0][rq] + s_part[1][rq];
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

template <int NP>
constexpr int conv_tc_smem() {
  return 1024 + 2 * (2 * 128 * KC * 4 + 2 * NP * KC * 4) + 64;
}

}  // namespace

size_t tc_conv_floats(const LayerDev& L) {
  if (L.kind != MNBAB_CONV2D) return 0;
  size_t tot = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int N = dir == 0 ? L.co : L.ci;
    const int NP = (N + 15) / 16 * 16;
    const int ncls = dir == 0 ? 1 : L.s * L.s;
    int K = 0;
    for (int cl = 0; cl < ncls; ++cl) K = std::max(K, conv_class(L, dir, cl).K);
    const int Kp = std::max(KC, (K + KC - 1) / KC * KC);
    if (N < 8 || NP > 64 || Kp > TC_KMAX) continue;
    tot += 2 * (size_t)ncls * Kp * NP;
  }
  return tot;
}

TcConv* tc_conv_create(const LayerDev& L, float* buf, cudaStream_t st) {
  if (L.kind != MNBAB_CONV2D || !buf) return nullptr;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return nullptr;
  TcConv* t = new TcConv();
  size_t at = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int N = dir == 0 ? L.co : L.ci;
    const int NP = (N + 15) / 16 * 16;
    const int ncls = dir == 0 ? 1 : L.s * L.s;
    int K = 0, pmax = 0;
    for (int cl = 0; cl < ncls; ++cl) {
      const ConvClass c = conv_class(L, dir, cl);
      K = std::max(K, c.K);
      pmax = std::max(pmax, c.P);
    }
    const int Kp = std::max(KC, (K + KC - 1) / KC * KC);
    // too few or too many channels for these tiles, or a reduction longer than the table
    if (N < 8 || NP > 64 || Kp > TC_KMAX) continue;
    float* hi = buf + at;
    float* lo = hi + (size_t)ncls * Kp * NP;
    at += 2 * (size_t)ncls * Kp * NP;
    dim3 grid((unsigned)std::min(1024, (Kp * NP + 255) / 256), ncls);
    k_tc_conv_split<<<grid, 256, 0, st>>>(L, dir, Kp, NP, hi, lo);
    // [ncls][Kp / 4][NP][4] floats as a 3-D tensor {4 NP, Kp / 4, ncls}; one box
    // = one K block of 32 of one class, all NP channels
    const cuuint64_t gdim[3] = {(cuuint64_t)4 * NP, (cuuint64_t)Kp / 4, (cuuint64_t)ncls};
    const cuuint64_t gstr[2] = {(cuuint64_t)4 * NP * 4, (cuuint64_t)(Kp / 4) * 4 * NP * 4};
    const cuuint32_t box[3] = {(cuuint32_t)4 * NP, (cuuint32_t)KC / 4, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    bool good = true;
    for (int part = 0; part < 2 && good; ++part)
      good = enc(part == 0 ? &t->hi[dir] : &t->lo[dir], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                 part == 0 ? hi : lo, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (!good) continue;
    t->ok[dir] = true;
    t->N[dir] = N;
    t->NP[dir] = NP;
    t->Kp[dir] = Kp;
    t->ncls[dir] = ncls;
    t->nchunk[dir] = (pmax + 31) / 32;
  }
  return t;
}

void tc_conv_destroy(TcConv* t) { delete t; }

bool tc_conv_usable(const LayerDev& L, int dir) {
  const TcConv* t = static_cast<const TcConv*>(L.tc);
  return t && t->ok[dir];
}

int tc_conv_slots(const LayerDev& L) {
  const TcConv* t = static_cast<const TcConv*>(L.tc);
  return t && t->ok[1] ? t->ncls[1] * t->nchunk[1] : 0;
}

int launch_tc_conv(const LayerDev& L, int dir, int M, const float* in, int ld_in, float* out,
                   int ld_out, const Epi& e, cudaStream_t st) {
  const TcConv* t = static_cast<const TcConv*>(L.tc);
  const dim3 grid(t->ncls[dir] * t->nchunk[dir], (M + TROWS - 1) / TROWS);
  static bool attr[4] = {false, false, false, false};
  auto go = [&](auto kern, int smem, int which) {
    if (!attr[which]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr[which] = true;
    }
    kern<<<grid, TC_THREADS, smem, st>>>(t->hi[dir], t->lo[dir], L, dir, M, t->nchunk[dir], in, ld_in,
                                  out, ld_out, e, e.err);
  };
  switch (t->NP[dir]) {
    case 16: go(k_conv_tc<16>, conv_tc_smem<16>(), 0); break;
    case 32: go(k_conv_tc<32>, conv_tc_smem<32>(), 1); break;
    case 48: go(k_conv_tc<48>, conv_tc_smem<48>(), 2); break;
    default: go(k_conv_tc<64>, conv_tc_smem<64>(), 3); break;
  }
  return grid.x;
}

}  // namespace mnbab
