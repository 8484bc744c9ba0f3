// Fused optimisation loop (Sec. 3.1) for chain networks without multi-neuron
// constraints: one CTA carries one objective row through all Adam iterations.
//
// Per iteration the CTA runs, on its row alone:
//   1. the back-substitution sweep at the node's current (alpha, beta): the
//      objective row a = (C W_L)_r, then for t = R .. 1 the ReLU step of layer t
//      (a' = a; D, blow by the sign of a'; ahat = a' D + beta S; offset
//      a' blow + ahat b_t) followed by the affine step through layer t, and the
//      concretisation over the input box (x*_k = lo_k if a0_k >= 0 else hi_k);
//   2. best-bound tracking: the node keeps the best bound and its minimiser;
//   3. the adjoint: the relaxed network evaluated forward at x* (h_t = W_t g +
//      b_t, g_t = h_t D_t + blow_t) gives d lb / d alpha_j = h_j a'_j on the
//      alpha branch and d lb / d beta_j = h_j S_j;
//   4. projected Adam on (alpha, beta) with the gradient-scaled eps.
// The coefficient rows, the a' checkpoints, the gradients and x* stay in shared
// memory; only the node's state (bounds, splits, parameters, moments) and the
// weights are read from global memory.  The arithmetic of each element is that
// of the unfused kernels; sums are accumulated in a different order.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdint>

#include "epilogue.cuh"
#include "mnbab.h"
#include "mnbab_internal.h"
#include "tc_common.cuh"

namespace mnbab {

namespace {

constexpr int FT = 512;  // threads per CTA (two CTAs per SM)
constexpr int FU = 3;    // neurons per thread whose node-state loads overlap (ReLU steps)
constexpr int FA = 4;    // parameters per thread whose loads overlap (Adam)

__device__ __forceinline__ float f_block_sum(float v, float* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int i = 0; i < FT / 32; ++i) r += red[i];
  return r;
}

__device__ __forceinline__ float f_block_max(float v, float* red) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float r = 0.f;
  for (int i = 0; i < FT / 32; ++i) r = fmaxf(r, red[i]);
  return r;
}

__device__ __forceinline__ void f_adam(float& th, float& mo, float& ve, float g, float lr,
                                       float b1, float b2, float eps, float bc1, float bc2) {
  mo = b1 * mo + (1.f - b1) * g;
  ve = b2 * ve + (1.f - b2) * g * g;
  const float mh = mo / bc1;
  const float vh = ve / bc2;
  th = th + lr * mh / (sqrtf(vh) + eps);
}

// Threads that share one output (a split of its reduction over adjacent
// lanes): the largest power of two <= 8 with items * KS <= FT.
__device__ __forceinline__ int f_split(int items) {
  int ks = 1;
  while (ks < 8 && items * ks * 2 <= FT) ks <<= 1;
  return ks;
}

__device__ __forceinline__ float f_group_sum(float v, int ks) {
  for (int o = ks >> 1; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Back-substitution through FC layer L: cur (d_out) -> nxt (d_in) = cur W.
__device__ void f_fc_back(const LayerDev& L, const float* cur, float* nxt) {
  const int din = L.d_in, dout = L.d_out;
  const bool vec = (din & 3) == 0 && (reinterpret_cast<uintptr_t>(L.W) & 15) == 0;
  const int CB = vec ? 4 : 1;
  const int items = din / CB;
  const int ks = f_split(items);
  const int rounds = (items * ks + FT - 1) / FT;
  for (int rr = 0; rr < rounds; ++rr) {
    const int b = rr * FT + threadIdx.x;
    const int it = b / ks, k0 = b % ks;
    const bool act = it < items;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (act) {
      if (vec) {
        const float4* w4 = reinterpret_cast<const float4*>(L.W) + it;
        const int n4 = din >> 2;
        int j = k0;
        for (; j + 3 * ks < dout; j += 4 * ks) {
          float4 w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) w[u] = __ldg(w4 + (size_t)(j + u * ks) * n4);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float a = cur[j + u * ks];
            a0 = fmaf(a, w[u].x, a0);
            a1 = fmaf(a, w[u].y, a1);
            a2 = fmaf(a, w[u].z, a2);
            a3 = fmaf(a, w[u].w, a3);
          }
        }
        for (; j < dout; j += ks) {
          const float4 w = __ldg(w4 + (size_t)j * n4);
          const float a = cur[j];
          a0 = fmaf(a, w.x, a0);
          a1 = fmaf(a, w.y, a1);
          a2 = fmaf(a, w.z, a2);
          a3 = fmaf(a, w.w, a3);
        }
      } else {
        for (int j = k0; j < dout; j += ks) a0 = fmaf(cur[j], __ldg(L.W + (size_t)j * din + it), a0);
      }
    }
    a0 = f_group_sum(a0, ks);
    if (vec) {
      a1 = f_group_sum(a1, ks);
      a2 = f_group_sum(a2, ks);
      a3 = f_group_sum(a3, ks);
    }
    if (act && k0 == 0) {
      if (vec) reinterpret_cast<float4*>(nxt)[it] = make_float4(a0, a1, a2, a3);
      else nxt[it] = a0;
    }
  }
}

// Forward through FC layer L: g (d_in) -> h (d_out) = W g + b; one warp per
// pair of outputs (each load of g serves both rows).
__device__ void f_fc_fwd(const LayerDev& L, const float* g, float* h) {
  const int din = L.d_in, dout = L.d_out;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool vec = (din & 3) == 0 && (reinterpret_cast<uintptr_t>(L.W) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(g) & 15) == 0;
  for (int i = 2 * warp; i < dout; i += FT / 16) {
    const bool two = i + 1 < dout;
    const int i1 = two ? i + 1 : i;
    float acc0 = 0.f, acc1 = 0.f;
    if (vec) {
      const float4* w0 = reinterpret_cast<const float4*>(L.W + (size_t)i * din);
      const float4* w1 = reinterpret_cast<const float4*>(L.W + (size_t)i1 * din);
      const float4* g4 = reinterpret_cast<const float4*>(g);
      const int n4 = din >> 2;
      for (int c0 = lane; c0 < n4; c0 += 32 * 2) {
        float4 a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = c0 + 32 * u;
          const bool in = c < n4;
          a[u] = in ? __ldg(w0 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
          b[u] = in ? __ldg(w1 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = c0 + 32 * u;
          if (c < n4) {
            const float4 x = g4[c];
            acc0 = fmaf(a[u].x, x.x, acc0);
            acc0 = fmaf(a[u].y, x.y, acc0);
            acc0 = fmaf(a[u].z, x.z, acc0);
            acc0 = fmaf(a[u].w, x.w, acc0);
            acc1 = fmaf(b[u].x, x.x, acc1);
            acc1 = fmaf(b[u].y, x.y, acc1);
            acc1 = fmaf(b[u].z, x.z, acc1);
            acc1 = fmaf(b[u].w, x.w, acc1);
          }
        }
      }
    } else {
      for (int j = lane; j < din; j += 32) {
        const float x = g[j];
        acc0 = fmaf(__ldg(L.W + (size_t)i * din + j), x, acc0);
        acc1 = fmaf(__ldg(L.W + (size_t)i1 * din + j), x, acc1);
      }
    }
    for (int o = 16; o; o >>= 1) {
      acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
      acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    }
    if (lane == 0) {
      h[i] = acc0 + L.b[i];
      if (two) h[i + 1] = acc1 + L.b[i + 1];
    }
  }
}

// Staged conv weights: one row per channel of the reduction-split dimension
// (Wb: a row per output channel co, Wf: a row per input channel ci).  Row
// strides are padded so that the lanes that split a reduction over channels
// (adjacent lanes, channels k0, k0 + ks, ...) fall in different shared-memory
// banks: stride = 4 mod 32 floats for float4 rows, 1 mod 32 for scalar rows.
__host__ __device__ inline int f_padw(int w, bool vec) {
  return vec ? w + ((36 - (w & 31)) & 31) : w + ((33 - (w & 31)) & 31);
}
__host__ __device__ inline int f_wb_stride(const LayerDev& L) {
  return f_padw(L.k * L.k * L.ci, (L.ci & 3) == 0);
}
__host__ __device__ inline int f_wf_stride(const LayerDev& L) {
  return f_padw(L.k * L.k * L.co, (L.co & 3) == 0);
}
__host__ __device__ inline int f_wb_floats(const LayerDev& L) {
  return (L.co * f_wb_stride(L) + 3) / 4 * 4;
}
__host__ __device__ inline int f_wf_floats(const LayerDev& L) {
  return (L.ci * f_wf_stride(L) + 3) / 4 * 4;
}
// shared-memory floats of a layer's staged weights (both layouts)
__host__ __device__ inline int f_conv_wfloats(const LayerDev& L) {
  return L.kind == MNBAB_CONV2D ? f_wb_floats(L) + f_wf_floats(L) : 0;
}
// copies rows of `w` floats from src (dense) to dst (stride `stride`)
__device__ inline void f_stage(float* dst, const float* src, int rows, int w, int stride,
                               int nthr) {
  for (int i = threadIdx.x; i < rows * w; i += nthr) dst[(i / w) * stride + i % w] = __ldg(src + i);
}

// Transposed convolution (back-substitution) through conv layer L with its
// weights in shared memory as Wb [co][kh][kw][ci]: cur [co][ho][wo] -> nxt
// [ci][hi][wi].  A thread group takes CB channels at two input positions of
// one row, s columns apart: both have the taps kh = (ih + p) mod s (+ s, ...),
// kw = (iw + p) mod s (+ s, ...), the second at ow + 1, so every staged
// weight load serves both positions.
__device__ void f_conv_back(const LayerDev& L, const float* cur, float* nxt, const float* Wb) {
  const int CB = (L.ci & 3) == 0 ? 4 : 1;
  const int S = L.s;
  const int W2 = (L.wi + 2 * S - 1) / (2 * S) * S;  // first positions per row (a few past the edge)
  const int ngr = L.ci / CB, P = L.hi * L.wi, hwo = L.ho * L.wo, PP = L.hi * W2;
  const int items = PP * ngr;
  const int ks = f_split(items);
  const int rounds = (items * ks + FT - 1) / FT;
  const size_t wco = (size_t)f_wb_stride(L);
  for (int rr = 0; rr < rounds; ++rr) {
    const int b = rr * FT + threadIdx.x;
    const int it = b / ks, k0 = b % ks;
    bool act = it < items;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
    int grp = 0, ih = 0, iw = 0;
    bool two = false;
    if (act) {
      grp = it / PP;
      const int q = it % PP;
      ih = q / W2;
      const int qw = q % W2;
      iw = (qw / S) * 2 * S + qw % S;
      act = iw < L.wi;
      two = iw + S < L.wi;
    }
    if (act) {
      const int kh0 = (ih + L.p) % S, kw0 = (iw + L.p) % S;
      const int oh0 = (ih + L.p - kh0) / S, ow0 = (iw + L.p - kw0) / S;
      for (int kh = kh0, oh = oh0; kh < L.k && oh >= 0; kh += S, --oh) {
        if (oh >= L.ho) continue;
        // the second position's ow is ow + 1, valid down to ow = -1
        for (int kw = kw0, ow = ow0; kw < L.k && ow >= -1; kw += S, --ow) {
          const bool ok0 = ow >= 0 && ow < L.wo;
          const bool ok1 = two && ow + 1 < L.wo;
          if (!ok0 && !ok1) continue;
          const float* ap = cur + oh * L.wo + ow;
          const float* wp = Wb + (size_t)(kh * L.k + kw) * L.ci + grp * CB;
          if (CB == 4) {
#pragma unroll 2
            for (int co = k0; co < L.co; co += ks) {
              const float v0 = ok0 ? ap[co * hwo] : 0.f;
              const float v1 = ok1 ? ap[co * hwo + 1] : 0.f;
              const float4 w = *reinterpret_cast<const float4*>(wp + co * wco);
              a0 = fmaf(v0, w.x, a0);
              a1 = fmaf(v0, w.y, a1);
              a2 = fmaf(v0, w.z, a2);
              a3 = fmaf(v0, w.w, a3);
              c0 = fmaf(v1, w.x, c0);
              c1 = fmaf(v1, w.y, c1);
              c2 = fmaf(v1, w.z, c2);
              c3 = fmaf(v1, w.w, c3);
            }
          } else {
#pragma unroll 2
            for (int co = k0; co < L.co; co += ks) {
              const float w = wp[co * wco];
              a0 = fmaf(ok0 ? ap[co * hwo] : 0.f, w, a0);
              c0 = fmaf(ok1 ? ap[co * hwo + 1] : 0.f, w, c0);
            }
          }
        }
      }
    }
    a0 = f_group_sum(a0, ks);
    c0 = f_group_sum(c0, ks);
    if (CB == 4) {
      a1 = f_group_sum(a1, ks);
      a2 = f_group_sum(a2, ks);
      a3 = f_group_sum(a3, ks);
      c1 = f_group_sum(c1, ks);
      c2 = f_group_sum(c2, ks);
      c3 = f_group_sum(c3, ks);
    }
    if (act && k0 == 0) {
      const int o = grp * CB * P + ih * L.wi + iw;
      nxt[o] = a0;
      if (CB == 4) {
        nxt[o + P] = a1;
        nxt[o + 2 * P] = a2;
        nxt[o + 3 * P] = a3;
      }
      if (two) {
        nxt[o + S] = c0;
        if (CB == 4) {
          nxt[o + S + P] = c1;
          nxt[o + S + 2 * P] = c2;
          nxt[o + S + 3 * P] = c3;
        }
      }
    }
  }
}

// Forward convolution through L (+ bias) with its weights in shared memory as
// Wf [ci][kh][kw][co]: g [ci][hi][wi] -> h [co][ho][wo].  A thread group takes
// CB output channels of one position: each input load serves CB channels (the
// weight loads of a warp are mostly broadcasts, the input loads are not).
template <int CB>
__device__ void f_conv_fwd_cb(const LayerDev& L, const float* g, float* h, const float* Wf) {
  const int ngr = L.co / CB, P = L.ho * L.wo, hwi = L.hi * L.wi;
  const int items = P * ngr;
  const int ks = f_split(items);
  const int rounds = (items * ks + FT - 1) / FT;
  for (int rr = 0; rr < rounds; ++rr) {
    const int b = rr * FT + threadIdx.x;
    const int it = b / ks, k0 = b % ks;
    const bool act = it < items;
    float a[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) a[u] = 0.f;
    int grp = 0, pos = 0;
    if (act) {
      grp = it / P;
      pos = it % P;
      const int oh = pos / L.wo, ow = pos % L.wo;
      const int ih0 = oh * L.s - L.p, iw0 = ow * L.s - L.p;
      const int kh_lo = max(0, -ih0), kh_hi = min(L.k, L.hi - ih0);
      const int kw_lo = max(0, -iw0), kw_hi = min(L.k, L.wi - iw0);
      for (int ci = k0; ci < L.ci; ci += ks) {
        const float* gp = g + ci * hwi;
        const float* wc = Wf + (size_t)ci * f_wf_stride(L) + grp * CB;
        for (int kh = kh_lo; kh < kh_hi; ++kh)
#pragma unroll 4
          for (int kw = kw_lo; kw < kw_hi; ++kw) {
            const float v = gp[(ih0 + kh) * L.wi + iw0 + kw];
            const float* wp = wc + (size_t)(kh * L.k + kw) * L.co;
            if (CB >= 4) {
#pragma unroll
              for (int q = 0; q < CB / 4; ++q) {
                const float4 w = *reinterpret_cast<const float4*>(wp + 4 * q);
                a[4 * q] = fmaf(v, w.x, a[4 * q]);
                a[4 * q + 1] = fmaf(v, w.y, a[4 * q + 1]);
                a[4 * q + 2] = fmaf(v, w.z, a[4 * q + 2]);
                a[4 * q + 3] = fmaf(v, w.w, a[4 * q + 3]);
              }
            } else {
              a[0] = fmaf(v, wp[0], a[0]);
            }
          }
      }
    }
#pragma unroll
    for (int u = 0; u < CB; ++u) a[u] = f_group_sum(a[u], ks);
    if (act && k0 == 0) {
      const int c = grp * CB;
#pragma unroll
      for (int u = 0; u < CB; ++u) h[(c + u) * P + pos] = a[u] + L.b[c + u];
    }
  }
}

__device__ void f_conv_fwd(const LayerDev& L, const float* g, float* h, const float* Wf) {
  if ((L.co & 7) == 0) f_conv_fwd_cb<8>(L, g, h, Wf);
  else if ((L.co & 3) == 0) f_conv_fwd_cb<4>(L, g, h, Wf);
  else f_conv_fwd_cb<1>(L, g, h, Wf);
}


// ---- transposed convolution of one conv layer on the tensor cores --------------
// The back-substitution step through conv layer T (Sec. 3.1: the affine step
// through a convolution is its transposed convolution) as one small GEMM per
// sweep plus a gather:
//   Z[(c, kh, kw), (oy, ox)] = sum over o of W[o, c, kh, kw] Lambda[o, oy, ox]
//   nxt[c, y, x] = sum over taps with y = oy s - p + kh, x = ox s - p + kw of Z.
// A = W viewed as [ci k k][co] stays in tensor memory for the whole launch
// (TF32 hi and lo parts, written once).  The layer's back-substitution weight
// region of shared memory (which the SIMT step no longer needs) holds, per
// sweep, first B = Lambda as [ho wo][co] (hi and lo) and then Z: D = Z
// accumulates in tensor memory with 3xTF32 split products (lo.hi + hi.lo +
// hi.hi, FP32 accumulation), is copied to that region once the MMAs are done
// and gathered into nxt in a fixed tap order.
constexpr int FTC_TAPS = 4;  // taps per dimension and stride class (k <= 4 s)

struct FusedTc {
  int t = 0;           // the layer (0: none)
  int RK = 0;          // rows of A: ci k k
  int P = 0;           // output positions ho wo
  int Mt = 0, Kp = 0, Np = 0;  // 128-row tiles, co padded to 8, P padded to 16
  int zs = 0;          // row stride of Z in shared memory (odd: no bank conflicts)
  int dcol = 0;        // first tensor-memory column of D
  uint32_t ncols = 0;  // tensor-memory columns allocated
};

// shared-memory floats of layer t's first weight region: the staged Wb, or
// for the tensor-core layer its B tile (hi and lo) and later its Z
__host__ __device__ inline int ftc_wb_region(const LayerDev& L, int t, const FusedTc& ft) {
  const int wb = f_wb_floats(L);
  if (t != ft.t) return wb;
  const int z = (ft.RK * ft.zs + 3) / 4 * 4, b = 2 * ft.Np * ft.Kp;
  const int m = z > b ? z : b;
  return wb > m ? wb : m;
}

// A (hi and lo) into tensor memory: warp w writes lanes 32 (w mod 4) .. + 31
// of 8-column chunks; called by every thread
__device__ void ftc_load_a(const FusedTc& ft, const LayerDev& L, uint32_t tmem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, g = warp >> 2;
  const int nch = ft.Kp / 8, ntask = ft.Mt * 2 * nch;
  for (int task = g; task < ntask; task += FT / 128) {
    const int i = task / (2 * nch), h = (task / nch) & 1, cc = task % nch;
    const int r = i * 128 + q * 32 + lane;
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int o = cc * 8 + j;
      const float w = (r < ft.RK && o < L.co) ? __ldg(L.W + (size_t)o * ft.RK + r) : 0.f;
      const uint32_t hi = tc::to_tf32(w);
      v[j] = h == 0 ? hi : tc::to_tf32(w - __uint_as_float(hi));
    }
    tc::tmem_st8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(i * 2 * ft.Kp + h * ft.Kp + cc * 8),
                 v);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// cur [co][ho][wo] -> nxt [ci][hi][wi]; the B tile and then Z in the region
// `Z` of shared memory.  Returns false (the same in every thread) when the MMAs
// did not complete within the bounded wait; the error flag is then set.
__device__ bool ftc_back(const FusedTc& ft, const LayerDev& L, const float* cur, float* nxt,
                         float* Z, uint32_t tmem, uint32_t bar, uint32_t& phase, int* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // B [Np][Kp] in the no-swizzle K-major canonical layout: core matrices of 8
  // positions x 4 channels, 128 B apart along K, Kp / 4 x 128 B apart along N
  const uint32_t sbo = (uint32_t)(ft.Kp / 4) * 128u;
  unsigned char* bhi = reinterpret_cast<unsigned char*>(Z);
  unsigned char* blo = bhi + (size_t)ft.Np * ft.Kp * 4;
  for (int o = warp; o < ft.Kp; o += FT / 32)
    for (int n = lane; n < ft.Np; n += 32) {
      const float v = (o < L.co && n < ft.P) ? cur[o * ft.P + n] : 0.f;
      const uint32_t h = tc::to_tf32(v);
      const uint32_t l = tc::to_tf32(v - __uint_as_float(h));
      const uint32_t off = (uint32_t)(n >> 3) * sbo + (uint32_t)(o >> 2) * 128u + (n & 7) * 16u +
                           (o & 3) * 4u;
      *reinterpret_cast<uint32_t*>(bhi + off) = h;
      *reinterpret_cast<uint32_t*>(blo + off) = l;
    }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = tc::idesc_tf32_m128(ft.Np);
    const uint32_t bh = tc::smem_u32(bhi), bl = tc::smem_u32(blo);
    for (int i = 0; i < ft.Mt; ++i) {
      const uint32_t d = tmem + (uint32_t)(ft.dcol + i * ft.Np);
      for (int ks = 0; ks < ft.Kp / 8; ++ks) {
        const uint32_t ah = tmem + (uint32_t)(i * 2 * ft.Kp + ks * 8);
        const uint32_t bo = (uint32_t)ks * 256u;
        tc::mma_tf32_tmem_a(d, ah + (uint32_t)ft.Kp, tc::smem_desc(bh + bo, 128, sbo), idesc,
                            ks > 0 ? 1u : 0u);
        tc::mma_tf32_tmem_a(d, ah, tc::smem_desc(bl + bo, 128, sbo), idesc, 1u);
        tc::mma_tf32_tmem_a(d, ah, tc::smem_desc(bh + bo, 128, sbo), idesc, 1u);
      }
    }
    tc::mma_commit(bar);
  }
  // every warp waits for the MMAs itself, then copies its lane quarter of D
  // (16-column chunks split over the four warps of a quarter) to Z
  const bool mine = __all_sync(0xffffffffu, tc::mbar_wait(bar, phase));
  if (mine) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int q = warp & 3, g = warp >> 2, nc = ft.Np / 16;
    for (int task = g; task < ft.Mt * nc; task += FT / 128) {
      const int i = task / nc, c = task % nc;
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ft.dcol + i * ft.Np + c * 16), v);
      const int r = i * 128 + q * 32 + lane;
      if (r < ft.RK) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c * 16 + j < ft.P) Z[r * ft.zs + c * 16 + j] = v[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if (!__syncthreads_and(mine)) {
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      tc::mbar_wait(bar, phase);  // one more bounded wait before the memory is released
    }
    return false;
  }
  phase ^= 1u;
  // gather: one item per (channel, input row, column residue mod s); its
  // columns share the row taps (kh, oy) and the column taps kw with ox = base + i
  // for the i-th column of the residue class.  Taps are summed in (kh, kw) order.
  const int S = L.s, HW = L.hi * L.wi, kk = L.k * L.k;
  const int items = L.ci * L.hi * S;
  for (int it = threadIdx.x; it < items; it += FT) {
    const int rx = it % S, y = (it / S) % L.hi, c = it / (S * L.hi);
    // row taps kh = kh0 + a s (valid: inside the kernel, oy in range) and
    // column taps kw = kw0 + b s
    const int kh0 = (y + L.p) % S, kw0 = (rx + L.p) % S;
    int zrow[FTC_TAPS], kwz[FTC_TAPS], base[FTC_TAPS];
    bool rv[FTC_TAPS], cv[FTC_TAPS];
#pragma unroll
    for (int a = 0; a < FTC_TAPS; ++a) {
      const int kh = kh0 + a * S, ty = y + L.p - kh;
      rv[a] = kh < L.k && ty >= 0 && ty / S < L.ho;
      zrow[a] = (c * kk + kh * L.k) * ft.zs + (rv[a] ? (ty / S) * L.wo : 0);
      const int kw = kw0 + a * S;
      cv[a] = kw < L.k;
      kwz[a] = kw * ft.zs;
      base[a] = (rx + L.p - kw) / S;  // exact: rx + p - kw is a multiple of s
    }
    float* out = nxt + c * HW + y * L.wi;
    for (int x = rx, i = 0; x < L.wi; x += S, ++i) {
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < FTC_TAPS; ++a) {
#pragma unroll
        for (int b = 0; b < FTC_TAPS; ++b) {
          const int ox = base[b] + i;
          if (rv[a] && cv[b] && ox >= 0 && ox < L.wo) acc += Z[zrow[a] + kwz[b] + ox];
        }
      }
      out[x] = acc;
    }
  }
  return true;
}

}  // namespace

// two CTAs per SM: at most 64 registers a thread
__global__ void __launch_bounds__(FT, 2) k_opt_chain(NetDev net, PoolDev pool, const PropDev* props,
                                                  const int* row_node, const int* row_j,
                                                  FusedHP hp, float* AP_out, float* GB_out,
                                                  int maxw, FusedTc ft, int* err,
                                                  const float* __restrict__ skip_lb) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ float red[32];
  __shared__ int improved;
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tc_holder;
  // a row whose DeepPoly bound (skip_lb, by batch row) already verifies its node
  // is not optimised: the node keeps its state and its DeepPoly best bound
  if (skip_lb && skip_lb[blockIdx.x] > 0.f) return;
  const int SD = pool.SD, d0 = pool.d0, R = net.R;
  // conv weights of every layer, staged once: Wb then Wf per conv layer (the
  // Wb region of the tensor-core layer holds its Z instead)
  int wtot = 0;
  for (int t = 1; t <= R; ++t) {
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_CONV2D) continue;
    const int wbr = ftc_wb_region(L, t, ft);
    if (t != ft.t) f_stage(fsm + wtot, L.Wb, L.co, L.k * L.k * L.ci, f_wb_stride(L), FT);
    f_stage(fsm + wtot + wbr, L.Wf, L.ci, L.k * L.k * L.co, f_wf_stride(L), FT);
    wtot += wbr + f_wf_floats(L);
  }
  uint32_t tmem = 0, phase = 0;
  const uint32_t bar = tc::smem_u32(&tc_bar);
  if (ft.t) {
    if ((threadIdx.x >> 5) == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       tc::smem_u32(&tc_holder)),
                   "r"(ft.ncols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
      tc::mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = tc_holder;
    ftc_load_a(ft, net.aff[ft.t], tmem);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  bool abort = false;
  const int SDp = (SD + 3) & ~3;  // 16-byte aligned sub-buffers
  float* B0 = fsm + wtot;
  float* B1 = B0 + maxw;
  float* APs = B1 + maxw;  // a' checkpoints, then d lb / d alpha
  float* Xs = APs + SDp;   // minimiser x*
  // case of each neuron, fixed during the optimisation (bounds and splits do not
  // change): 0 inactive, 1 active, 2 unstable and unsplit, 3 split with S = -1
  // (zhat >= 0), 4 split with S = +1 (zhat <= 0)
  unsigned char* code = reinterpret_cast<unsigned char*>(Xs + ((d0 + 3) & ~3));
  auto wsm = [&](int t) {  // staged weights of conv layer t
    int o = 0;
    for (int u = 1; u < t; ++u)
      if (net.aff[u].kind == MNBAB_CONV2D)
        o += ftc_wb_region(net.aff[u], u, ft) + f_wf_floats(net.aff[u]);
    return fsm + o;
  };
  const int m = blockIdx.x;
  const int n = row_node[m], r = row_j[m];
  const PropDev& P = props[pool.prop[n]];
  const size_t nb = (size_t)n * SD;
  float* GBs = GB_out + (size_t)m * SD;  // d lb / d beta
  // Adam moments restart per node
  for (int i = threadIdx.x; i < SD; i += FT) {
    pool.MA[nb + i] = 0.f;
    pool.VA[nb + i] = 0.f;
    pool.MB[nb + i] = 0.f;
    pool.VB[nb + i] = 0.f;
    const int sv = pool.S[nb + i];
    code[i] = sv == -1 ? 3 : sv == 1 ? 4 : pool.L[nb + i] >= 0.f ? 1 : pool.U[nb + i] <= 0.f ? 0 : 2;
  }
  const int dR = net.d[R];
  for (int step = 0; step <= hp.steps; ++step) {
    // ---- 1. back-substitution sweep at the current parameters
    __syncthreads();
    float part = 0.f;
    float* cur = B0;
    float* nxt = B1;
    for (int j = threadIdx.x; j < dR; j += FT) cur[j] = P.Wf[(size_t)r * dR + j];
    __syncthreads();
    for (int t = R; t >= 1; --t) {
      const int dt = net.d[t], off = net.off[t];
      const float* bias = net.bfull[t];
      // FU neurons per thread at a time: their node-state loads (slope, or
      // bounds, or beta) are all issued before the first is used
      for (int j0 = threadIdx.x; j0 < dt; j0 += FU * FT) {
        int cd[FU];
        float ap[FU], v0[FU], v1[FU];
#pragma unroll
        for (int k = 0; k < FU; ++k) {
          const int j = j0 + k * FT;
          cd[k] = j < dt ? code[off + j] : 0;
          ap[k] = j < dt ? cur[j] : 0.f;
          v0[k] = v1[k] = 0.f;
          const size_t q = nb + off + j;
          if (cd[k] == 2) {
            v0[k] = ap[k] >= 0.f ? pool.ALPHA[q] : pool.L[q];
            if (ap[k] < 0.f) v1[k] = pool.U[q];
          } else if (cd[k] >= 3) {
            v0[k] = pool.BETA[q];
          }
        }
#pragma unroll
        for (int k = 0; k < FU; ++k) {
          const int j = j0 + k * FT;
          if (j >= dt) break;
          float D, bl = 0.f, bt = 0.f;
          if (cd[k] == 2) {
            if (ap[k] >= 0.f) {
              D = v0[k];
            } else {
              const float l = v0[k], u = v1[k];
              const float den = u - l;
              D = u / den;
              bl = (-u * l) / den;
            }
          } else {
            D = (cd[k] == 1 || cd[k] == 3) ? 1.f : 0.f;
            if (cd[k] >= 3) bt = v0[k] * (cd[k] == 3 ? -1.f : 1.f);
          }
          const float ah = ap[k] * D + bt;
          APs[off + j] = ap[k];
          part += ap[k] * bl + ah * bias[j];
          cur[j] = ah;
        }
      }
      __syncthreads();
      const LayerDev& L = net.aff[t];
      if (L.kind == MNBAB_FC) {
        f_fc_back(L, cur, nxt);
      } else if (t == ft.t) {
        if (!ftc_back(ft, L, cur, nxt, wsm(t), tmem, bar, phase, err)) {
          abort = true;
          break;
        }
      } else {
        f_conv_back(L, cur, nxt, wsm(t));
      }
      __syncthreads();
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (abort) break;
    for (int j = threadIdx.x; j < d0; j += FT) {
      const float a = cur[j];
      const float x = a >= 0.f ? P.lo[j] : P.hi[j];
      part += a * x;
      Xs[j] = x;
    }
    const float lb = f_block_sum(part, red) + P.bf[r];
    // ---- 2. best bound and its minimiser
    if (threadIdx.x == 0) {
      improved = lb > pool.BEST[n];
      if (improved) pool.BEST[n] = lb;
    }
    __syncthreads();
    if (improved)
      for (int j = threadIdx.x; j < d0; j += FT) pool.BESTX[(size_t)n * d0 + j] = Xs[j];
    if (step == hp.steps) {
      // a' at the final parameters, for the branching scores
      for (int i = threadIdx.x; i < SD; i += FT) AP_out[(size_t)m * SD + i] = APs[i];
      break;
    }
    // ---- 3. adjoint: the relaxed network forward at x*
    const float* g = Xs;
    float gm = 0.f;
    for (int t = 1; t <= R; ++t) {
      float* h = (t & 1) ? B0 : B1;
      __syncthreads();
      const LayerDev& L = net.aff[t];
      if (L.kind == MNBAB_FC) f_fc_fwd(L, g, h);
      else f_conv_fwd(L, g, h, wsm(t) + ftc_wb_region(L, t, ft));
      __syncthreads();
      const int dt = net.d[t], off = net.off[t];
      for (int j0 = threadIdx.x; j0 < dt; j0 += FU * FT) {
        int cdk[FU];
        float apk[FU], v0[FU], v1[FU];
#pragma unroll
        for (int k = 0; k < FU; ++k) {
          const int j = j0 + k * FT;
          cdk[k] = j < dt ? code[off + j] : 0;
          apk[k] = j < dt ? APs[off + j] : 0.f;
          v0[k] = v1[k] = 0.f;
          if (cdk[k] == 2) {
            const size_t q = nb + off + j;
            v0[k] = apk[k] >= 0.f ? pool.ALPHA[q] : pool.L[q];
            if (apk[k] < 0.f) v1[k] = pool.U[q];
          }
        }
#pragma unroll
        for (int k = 0; k < FU; ++k) {
          const int j = j0 + k * FT;
          if (j >= dt) break;
          const int cd = cdk[k];
          const float ap = apk[k];
          const float hv = h[j];
          float D, bl = 0.f, ga = 0.f, gb = 0.f;
          if (cd == 2) {
            if (ap >= 0.f) {
              D = v0[k];
              ga = hv * ap;
            } else {
              const float l = v0[k], u = v1[k];
              const float den = u - l;
              D = u / den;
              bl = (-u * l) / den;
            }
          } else {
            D = (cd == 1 || cd == 3) ? 1.f : 0.f;
            if (cd >= 3) {
              gb = hv * (cd == 3 ? -1.f : 1.f);
              GBs[off + j] = gb;  // row scratch in global memory (L2-resident)
            }
          }
          APs[off + j] = ga;
          gm = fmaxf(gm, fmaxf(fabsf(ga), fabsf(gb)));
          h[j] = hv * D + bl;
        }
      }
      g = h;
    }
    // ---- 4. projected Adam
    const float gmax = f_block_max(gm, red);
    const float thr = hp.floor * gmax;
    const float eps = fmaxf(hp.eps_abs, hp.eps_rel * gmax);
    const float bc1 = hp.bc1[step], bc2 = hp.bc2[step];
    // the alpha of a stable or split neuron and the beta of an unsplit one have a
    // zero gradient at every step, so their (zero-moment) updates are identities
    // FA parameters per thread at a time: all their loads (parameter, both
    // moments, gradient) are issued before the first update
    for (int i0 = threadIdx.x; i0 < SD; i0 += FA * FT) {
      int cd[FA];
      float th[FA], mo[FA], ve[FA], gr[FA];
#pragma unroll
      for (int k = 0; k < FA; ++k) {
        const int i = i0 + k * FT;
        cd[k] = i < SD ? code[i] : 0;
        th[k] = mo[k] = ve[k] = gr[k] = 0.f;
        const size_t q = nb + i;
        if (cd[k] == 2) {
          th[k] = pool.ALPHA[q];
          mo[k] = pool.MA[q];
          ve[k] = pool.VA[q];
          gr[k] = APs[i];
        } else if (cd[k] >= 3) {
          th[k] = pool.BETA[q];
          mo[k] = pool.MB[q];
          ve[k] = pool.VB[q];
          gr[k] = GBs[i];
        }
      }
#pragma unroll
      for (int k = 0; k < FA; ++k) {
        if (cd[k] < 2) continue;
        const size_t q = nb + i0 + k * FT;
        float g = gr[k];
        if (fabsf(g) <= thr) g = 0.f;
        if (cd[k] == 2) {
          f_adam(th[k], mo[k], ve[k], g, hp.lr_a, hp.b1, hp.b2, eps, bc1, bc2);
          pool.ALPHA[q] = fminf(fmaxf(th[k], 0.f), 1.f);
          pool.MA[q] = mo[k];
          pool.VA[q] = ve[k];
        } else {
          f_adam(th[k], mo[k], ve[k], g, hp.lr_b, hp.b1, hp.b2, eps, bc1, bc2);
          pool.BETA[q] = fmaxf(th[k], 0.f);
          pool.MB[q] = mo[k];
          pool.VB[q] = ve[k];
        }
      }
    }
  }
  if (ft.t) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                   "r"(ft.ncols));
    }
  }
}

// Multi-row forms of the back-substitution helpers: RB rows in lockstep, row q's
// coefficients at cur + q * ps; each staged weight and each index computation
// serves all RB rows.
template <int RB>
__device__ void f_fc_back_rows(const LayerDev& L, const float* cur, float* nxt, int ps) {
  const int din = L.d_in, dout = L.d_out;
  const int items = din;
  const int ks = f_split(items);
  const int rounds = (items * ks + FT - 1) / FT;
  for (int rr = 0; rr < rounds; ++rr) {
    const int b = rr * FT + threadIdx.x;
    const int it = b / ks, k0 = b % ks;
    const bool act = it < items;
    float acc[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q] = 0.f;
    if (act)
      for (int j = k0; j < dout; j += ks) {
        const float w = __ldg(L.W + (size_t)j * din + it);
#pragma unroll
        for (int q = 0; q < RB; ++q) acc[q] = fmaf(cur[q * ps + j], w, acc[q]);
      }
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q] = f_group_sum(acc[q], ks);
    if (act && k0 == 0)
#pragma unroll
      for (int q = 0; q < RB; ++q) nxt[q * ps + it] = acc[q];
  }
}

template <int RB>
__device__ void f_conv_back_rows(const LayerDev& L, const float* cur, float* nxt, int ps,
                                 const float* Wb) {
  const int CB = (L.ci & 3) == 0 ? 4 : 1;
  const int ngr = L.ci / CB, P = L.hi * L.wi, hwo = L.ho * L.wo;
  const int items = P * ngr;
  const int ks = f_split(items);
  const int rounds = (items * ks + FT - 1) / FT;
  const size_t wco = (size_t)f_wb_stride(L);
  for (int rr = 0; rr < rounds; ++rr) {
    const int b = rr * FT + threadIdx.x;
    const int it = b / ks, k0 = b % ks;
    const bool act = it < items;
    float acc[RB][4];
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    int grp = 0, ih = 0, iw = 0;
    if (act) {
      grp = it / P;
      const int pos = it % P;
      ih = pos / L.wi;
      iw = pos % L.wi;
      const int kh0 = (ih + L.p) % L.s, kw0 = (iw + L.p) % L.s;
      const int oh0 = (ih + L.p - kh0) / L.s, ow0 = (iw + L.p - kw0) / L.s;
      for (int kh = kh0, oh = oh0; kh < L.k && oh >= 0; kh += L.s, --oh) {
        if (oh >= L.ho) continue;
        for (int kw = kw0, ow = ow0; kw < L.k && ow >= 0; kw += L.s, --ow) {
          if (ow >= L.wo) continue;
          const float* ap = cur + oh * L.wo + ow;
          const float* wp = Wb + (size_t)(kh * L.k + kw) * L.ci + grp * CB;
          if (CB == 4) {
#pragma unroll 4
            for (int co = k0; co < L.co; co += ks) {
              const float4 w = *reinterpret_cast<const float4*>(wp + co * wco);
#pragma unroll
              for (int q = 0; q < RB; ++q) {
                const float v = ap[q * ps + co * hwo];
                acc[q][0] = fmaf(v, w.x, acc[q][0]);
                acc[q][1] = fmaf(v, w.y, acc[q][1]);
                acc[q][2] = fmaf(v, w.z, acc[q][2]);
                acc[q][3] = fmaf(v, w.w, acc[q][3]);
              }
            }
          } else {
#pragma unroll 4
            for (int co = k0; co < L.co; co += ks) {
              const float w = wp[co * wco];
#pragma unroll
              for (int q = 0; q < RB; ++q) acc[q][0] = fmaf(ap[q * ps + co * hwo], w, acc[q][0]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      acc[q][0] = f_group_sum(acc[q][0], ks);
      if (CB == 4) {
        acc[q][1] = f_group_sum(acc[q][1], ks);
        acc[q][2] = f_group_sum(acc[q][2], ks);
        acc[q][3] = f_group_sum(acc[q][3], ks);
      }
    }
    if (act && k0 == 0) {
      const int o = grp * CB * P + ih * L.wi + iw;
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        nxt[q * ps + o] = acc[q][0];
        if (CB == 4) {
          nxt[q * ps + o + P] = acc[q][1];
          nxt[q * ps + o + 2 * P] = acc[q][2];
          nxt[q * ps + o + 3 * P] = acc[q][3];
        }
      }
    }
  }
}

constexpr int SWEEP_RB = 4;  // rows per CTA pass

// Intermediate-bound rows (Sec. 3.2 re-bounding, DeepPoly slopes, beta = gamma =
// 0) that start at a fully connected neuron of zhat_t, above a chain: each CTA
// stages the transposed-conv weights once and carries groups of RB rows to the
// input in shared memory, in lockstep; row m's lower bound goes to lb[m].
template <int RB>
__global__ void __launch_bounds__(FT) k_sweep_chain(NetDev net, PoolDev pool,
                                                    const PropDev* props, RowsDev rows, int t0,
                                                    float* lb, int maxw) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ float red[32];
  int wtot = 0;
  for (int t = 1; t < t0; ++t) {
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_CONV2D) continue;
    f_stage(fsm + wtot, L.Wb, L.co, L.k * L.k * L.ci, f_wb_stride(L), FT);
    wtot += f_wb_floats(L);
  }
  const int ps = maxw;  // plane stride of a row's coefficients
  float* B0 = fsm + wtot;
  float* B1 = B0 + RB * ps;
  const int SD = pool.SD;
  const LayerDev& Lt = net.aff[t0];
  const int ngroups = (rows.M + RB - 1) / RB;
  for (int gI = blockIdx.x; gI < ngroups; gI += gridDim.x) {
    const int m0 = gI * RB;
    int nq[RB], jq[RB];
    float sq[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const bool in = m0 + q < rows.M;
      nq[q] = in ? rows.node[m0 + q] : rows.node[m0];
      jq[q] = in ? rows.j[m0 + q] : 0;
      sq[q] = in ? (rows.sign ? rows.sign[m0 + q] : 1.f) : 0.f;  // absent rows are zero
    }
    const int dprev = Lt.d_in;
    __syncthreads();
    float* cur = B0;
    float* nxt = B1;
#pragma unroll
    for (int q = 0; q < RB; ++q)
      for (int k = threadIdx.x; k < dprev; k += FT)
        cur[q * ps + k] = sq[q] * __ldg(Lt.W + (size_t)jq[q] * dprev + k);
    __syncthreads();
    float part[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) part[q] = 0.f;
    int wo = wtot;
    for (int t = t0 - 1; t >= 1; --t) {
      const int dt = net.d[t], off = net.off[t];
      const float* bias = net.bfull[t];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const size_t nb = (size_t)nq[q] * SD;
        for (int k = threadIdx.x; k < dt; k += FT) {
          const size_t qq = nb + off + k;
          const float l = pool.L[qq], u = pool.U[qq];
          const int s = pool.S[qq];
          const float ap = cur[q * ps + k];
          float D, bl = 0.f;
          if (s == -1) D = 1.f;
          else if (s == 1) D = 0.f;
          else if (l >= 0.f) D = 1.f;
          else if (u <= 0.f) D = 0.f;
          else if (ap >= 0.f) D = u >= -l ? 1.f : 0.f;
          else {
            const float den = u - l;
            D = u / den;
            bl = (-u * l) / den;
          }
          const float ah = ap * D;
          part[q] += ap * bl + ah * bias[k];
          cur[q * ps + k] = ah;
        }
      }
      __syncthreads();
      const LayerDev& L = net.aff[t];
      if (L.kind == MNBAB_FC) {
        f_fc_back_rows<RB>(L, cur, nxt, ps);
      } else {
        wo -= f_wb_floats(L);
        f_conv_back_rows<RB>(L, cur, nxt, ps, fsm + wo);
      }
      __syncthreads();
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const PropDev& P = props[pool.prop[nq[q]]];
      for (int k = threadIdx.x; k < pool.d0; k += FT) {
        const float a = cur[q * ps + k];
        part[q] += a * (a >= 0.f ? P.lo[k] : P.hi[k]);
      }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      const float tot = f_block_sum(part[q], red);
      if (threadIdx.x == 0 && m0 + q < rows.M) {
        const float bj = net.bfull[t0] ? net.bfull[t0][jq[q]] : Lt.b[jq[q]];
        lb[m0 + q] = tot + sq[q] * bj;
      }
    }
  }
}

static int sweep_wfloats(const NetDev& net, int t0) {
  int w = 0;
  for (int t = 1; t < t0; ++t)
    if (net.aff[t].kind == MNBAB_CONV2D) w += f_wb_floats(net.aff[t]);
  return w;
}

// Adversarial pre-attack (Sec. 4): sign-step projected gradient descent on the
// margin f_r(x) = (C f(x) + d)_r of one property row from one starting point;
// one CTA per (row, start).  Per iterate: the forward pass (pre-activations kept
// for the ReLU derivatives, ReLU'(0) = 1), the margin, best tracking (first
// minimiser), the gradient by the backward pass, and x <- clip(x - alpha sign(g)).
__global__ void __launch_bounds__(FT) k_attack_chain(NetDev net, const PropDev* props, int prop,
                                                     const float* starts, int n_starts,
                                                     int steps, float* best_out,
                                                     float* bx_out, int maxw) {
  extern __shared__ __align__(16) float fsm[];
  __shared__ float red[32];
  __shared__ int improved;
  const int R = net.R, d0 = net.d[0];
  int wtot = 0;
  for (int t = 1; t <= R; ++t) {
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_CONV2D) continue;
    f_stage(fsm + wtot, L.Wb, L.co, L.k * L.k * L.ci, f_wb_stride(L), FT);
    f_stage(fsm + wtot + f_wb_floats(L), L.Wf, L.ci, L.k * L.k * L.co, f_wf_stride(L), FT);
    wtot += f_conv_wfloats(L);
  }
  int SD = 0;
  for (int t = 1; t <= R; ++t) SD += net.d[t];
  const int d0p = (d0 + 3) & ~3;
  float* B0 = fsm + wtot;
  float* B1 = B0 + maxw;
  float* Z = B1 + maxw;                  // pre-activations of every ReLU layer
  float* X = Z + ((SD + 3) & ~3);        // current iterate
  auto wsm = [&](int t) {
    int o = 0;
    for (int u = 1; u < t; ++u) o += f_conv_wfloats(net.aff[u]);
    return fsm + o;
  };
  const int r = blockIdx.x / n_starts, sidx = blockIdx.x % n_starts;
  const PropDev& P = props[prop];
  const int dR = net.d[R];
  const float* wf = P.Wf + (size_t)r * dR;
  float* bx = bx_out + (size_t)blockIdx.x * d0;
  for (int j = threadIdx.x; j < d0; j += FT)
    X[j] = fminf(fmaxf(starts[(size_t)sidx * d0 + j], P.lo[j]), P.hi[j]);
  float best = INFINITY;
  for (int k = 0; k <= steps; ++k) {
    // forward pass
    __syncthreads();
    const float* g = X;
    for (int t = 1; t <= R; ++t) {
      float* h = (t & 1) ? B0 : B1;
      const LayerDev& L = net.aff[t];
      if (L.kind == MNBAB_FC) f_fc_fwd(L, g, h);
      else f_conv_fwd(L, g, h, wsm(t) + f_wb_floats(L));
      __syncthreads();
      const int off = net.off[t];
      for (int j = threadIdx.x; j < net.d[t]; j += FT) {
        const float z = h[j];
        Z[off + j] = z;
        h[j] = fmaxf(z, 0.f);
      }
      __syncthreads();
      g = h;
    }
    float part = 0.f;
    for (int j = threadIdx.x; j < dR; j += FT) part = fmaf(wf[j], g[j], part);
    const float f = f_block_sum(part, red) + P.bf[r];
    if (threadIdx.x == 0) improved = f < best;
    __syncthreads();
    if (improved) {
      best = f;
      for (int j = threadIdx.x; j < d0; j += FT) bx[j] = X[j];
    }
    if (k == steps) break;
    // backward pass: d f / d x through the ReLU derivatives at the pre-activations
    float* cur = (R & 1) ? B1 : B0;  // not the buffer holding g_R
    __syncthreads();
    for (int j = threadIdx.x; j < dR; j += FT) cur[j] = Z[net.off[R] + j] >= 0.f ? wf[j] : 0.f;
    __syncthreads();
    float* nxt = (cur == B0) ? B1 : B0;
    for (int t = R; t >= 1; --t) {
      const LayerDev& L = net.aff[t];
      if (L.kind == MNBAB_FC) f_fc_back(L, cur, nxt);
      else f_conv_back(L, cur, nxt, wsm(t));
      __syncthreads();
      if (t > 1) {
        const int off = net.off[t - 1];
        for (int j = threadIdx.x; j < net.d[t - 1]; j += FT)
          nxt[j] = Z[off + j] >= 0.f ? nxt[j] : 0.f;
        __syncthreads();
      }
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    // sign step and projection onto the box
    for (int j = threadIdx.x; j < d0; j += FT) {
      const float gj = cur[j];
      const float sg = gj > 0.f ? 1.f : (gj < 0.f ? -1.f : 0.f);
      const float alpha = 2.5f * (P.hi[j] - P.lo[j]) / (2.0f * (float)steps);
      X[j] = fminf(fmaxf(X[j] - alpha * sg, P.lo[j]), P.hi[j]);
    }
  }
  if (threadIdx.x == 0) best_out[blockIdx.x] = best;
}

static int fused_maxw(const NetDev& net, int d0) {
  int maxw = d0;
  for (int t = 1; t <= net.R; ++t) maxw = std::max(maxw, net.d[t]);
  return (maxw + 3) / 4 * 4;
}

static int fused_smem_floats(const NetDev& net, int SD, int d0, const FusedTc& ft = FusedTc()) {
  int w = 0;
  for (int t = 1; t <= net.R; ++t)
    if (net.aff[t].kind == MNBAB_CONV2D)
      w += ftc_wb_region(net.aff[t], t, ft) + f_wf_floats(net.aff[t]);
  return w + 2 * fused_maxw(net, d0) + (SD + 3) / 4 * 4 + (d0 + 3) / 4 * 4 + (SD + 3) / 4;
}

bool fused_supported(const NetDev& net, int SD, int d0, int steps) {
  if (steps < 0 || steps > FUSED_MAX_STEPS || net.R < 1) return false;
  for (int t = 1; t <= net.R + 1; ++t)
    if (net.n_edge[t] != 1 || net.src1[t] != t - 1) return false;
  for (int t = 1; t <= net.R; ++t) {
    const LayerDev& L = net.aff[t];
    if (!net.bfull[t] || (L.kind != MNBAB_FC && L.kind != MNBAB_CONV2D)) return false;
    if (L.kind == MNBAB_CONV2D && (!L.Wb || !L.Wf)) return false;
  }
  return fused_smem_floats(net, SD, d0) * (int)sizeof(float) <= 200 * 1024;
}

// The conv layer whose transposed convolution runs on the tensor cores: the one
// with the most multiply-adds among those whose operands fit (A and D in 256
// tensor-memory columns, the whole shared-memory layout with B and Z within the
// fused kernel's limit); t = 0 when none fits.
static FusedTc fused_tc_plan(const NetDev& net, int SD, int d0) {
  constexpr int kTwoPerSm = 112 * 1024;  // dynamic shared memory of two CTAs per SM
  const int simt = fused_smem_floats(net, SD, d0) * (int)sizeof(float);
  FusedTc best;
  double best_macs = 0.0;
  for (int t = 1; t <= net.R; ++t) {
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_CONV2D || !L.W || L.k > FTC_TAPS * L.s) continue;
    FusedTc f;
    f.t = t;
    f.RK = L.ci * L.k * L.k;
    f.P = L.ho * L.wo;
    f.Mt = (f.RK + 127) / 128;
    f.Kp = (L.co + 7) / 8 * 8;
    f.Np = std::max(16, (f.P + 15) / 16 * 16);
    f.zs = f.P | 1;
    f.dcol = f.Mt * 2 * f.Kp;
    const int cols = f.dcol + f.Mt * f.Np;
    // a larger Z region must not cost the second CTA per SM
    const int bytes = fused_smem_floats(net, SD, d0, f) * (int)sizeof(float);
    if (f.Np > 256 || cols > 256 || bytes > 200 * 1024 ||
        (simt <= kTwoPerSm && bytes > kTwoPerSm))
      continue;
    f.ncols = 32;
    while ((int)f.ncols < cols) f.ncols <<= 1;
    const double macs = (double)L.co * f.P * f.RK;
    if (macs > best_macs) {
      best_macs = macs;
      best = f;
    }
  }
  return best;
}

int fused_tc_layer(const NetDev& net, int SD, int d0) { return fused_tc_plan(net, SD, d0).t; }

void launch_opt_chain(int M, const NetDev& net, const PoolDev& pool, const PropDev* props,
                      const int* row_node, const int* row_j, const FusedHP& hp, float* AP_out,
                      float* GB_out, bool allow_tc, int* err, cudaStream_t st,
                      const float* skip_lb) {
  if (M <= 0) return;
  const FusedTc ft = allow_tc && err ? fused_tc_plan(net, pool.SD, pool.d0) : FusedTc();
  const int smem = fused_smem_floats(net, pool.SD, pool.d0, ft) * (int)sizeof(float);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_opt_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int maxw = fused_maxw(net, pool.d0);
  k_opt_chain<<<M, FT, smem, st>>>(net, pool, props, row_node, row_j, hp, AP_out, GB_out, maxw, ft,
                                  err, skip_lb);
}

bool sweep_chain_supported(const NetDev& net, int t0) {
  if (t0 < 2 || t0 > net.R || net.aff[t0].kind != MNBAB_FC) return false;
  for (int t = 1; t <= t0; ++t) {
    if (net.n_edge[t] != 1 || net.src1[t] != t - 1 || !net.bfull[t]) return false;
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_FC && L.kind != MNBAB_CONV2D) return false;
    if (L.kind == MNBAB_CONV2D && !L.Wb) return false;
  }
  int maxw = net.d[0];
  for (int t = 1; t < t0; ++t) maxw = std::max(maxw, net.d[t]);
  maxw = (maxw + 3) / 4 * 4;
  return (sweep_wfloats(net, t0) + 2 * SWEEP_RB * maxw) * (int)sizeof(float) <= 200 * 1024;
}

void launch_sweep_chain(const NetDev& net, const PoolDev& pool, const PropDev* props,
                        const RowsDev& rows, int t0, float* lb, cudaStream_t st) {
  if (rows.M <= 0) return;
  int maxw = net.d[0];
  for (int t = 1; t < t0; ++t) maxw = std::max(maxw, net.d[t]);
  maxw = (maxw + 3) / 4 * 4;
  const int smem = (sweep_wfloats(net, t0) + 2 * SWEEP_RB * maxw) * (int)sizeof(float);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_sweep_chain<SWEEP_RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
  static int sms = 0;
  if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess)
    sms = 152;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_chain<SWEEP_RB>, FT, smem) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int grid = std::min((rows.M + SWEEP_RB - 1) / SWEEP_RB, sms * per_sm);
  k_sweep_chain<SWEEP_RB><<<grid, FT, smem, st>>>(net, pool, props, rows, t0, lb, maxw);
}

int attack_smem_bytes(const NetDev& net) {
  int w = 0, SD = 0;
  for (int t = 1; t <= net.R; ++t) {
    w += f_conv_wfloats(net.aff[t]);
    SD += net.d[t];
  }
  return (w + 2 * fused_maxw(net, net.d[0]) + (SD + 3) / 4 * 4 + (net.d[0] + 3) / 4 * 4) *
         (int)sizeof(float);
}

bool attack_supported(const NetDev& net) {
  if (net.R < 1) return false;
  for (int t = 1; t <= net.R + 1; ++t)
    if (net.n_edge[t] != 1 || net.src1[t] != t - 1) return false;
  for (int t = 1; t <= net.R; ++t) {
    const LayerDev& L = net.aff[t];
    if (L.kind != MNBAB_FC && L.kind != MNBAB_CONV2D) return false;
    if (L.kind == MNBAB_CONV2D && (!L.Wb || !L.Wf)) return false;
  }
  return attack_smem_bytes(net) <= 200 * 1024;
}

void launch_attack_chain(const NetDev& net, const PropDev* props, int prop, int n_rows,
                         const float* starts, int n_starts, int steps, float* best_out,
                         float* bx_out, cudaStream_t st) {
  if (n_rows <= 0 || n_starts <= 0) return;
  const int smem = attack_smem_bytes(net);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_attack_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_attack_chain<<<n_rows * n_starts, FT, smem, st>>>(net, props, prop, starts, n_starts, steps,
                                                      best_out, bx_out, fused_maxw(net, net.d[0]));
}

}  // namespace mnbab
