// Device kernels of libmnbab: back-substitution through affine and ReLU layers
// with fused relaxation epilogues (Sec. 3.1), concretisation over the input box
// (Eq. minimum), the adjoint sweep for d lb / d (alpha, beta, gamma), projected
// Adam, ACS scoring (Sec. 3.2) and the BaB node bookkeeping (Sec. 3.2, enforcing
// splits).  All arithmetic is IEEE FP32 with FMA accumulation.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stdint.h>

#include "epilogue.cuh"
#include "mnbab.h"
#include "mnbab_internal.h"

namespace mnbab {

// block-wide sum; every thread gets the result
__device__ float block_sum(float v) {
  __shared__ float sh[32];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  float r = 0.f;
  for (int i = 0; i < nw; ++i) r += sh[i];
  return r;
}

template <typename F>
static void set_smem(F f, int bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------------------
// starting rows
// ---------------------------------------------------------------------------
// Starting rows through one affine edge into node t: a = sign * A[j, :] on the
// edge's source (the folded objective rows Wf for t = R + 1), c0 = sign * (sum
// of the edge biases at j) on the first edge; the partial goes to slot_base.
__global__ void k_init_rows(NetDev net, int t, int edge, RowsDev rows, float* out, int ld, Epi e) {
  const int m = blockIdx.x;
  if (m >= rows.M) return;
  const int n = rows.node[m];
  const int j = rows.j ? rows.j[m] : 0;
  const float sg = rows.sign ? rows.sign[m] : 1.f;
  const int src = edge == 0 ? net.src1[t] : net.src2[t];
  const int width = net.d[src];
  // a = 0 contributes nothing and maps to 0 through an intermediate ReLU step
  // (no beta / gamma terms), through concretisation (x* not kept) and as a raw
  // contribution, unless an earlier edge's contribution must be added
  const bool zero_passes = !e.acc_in &&
                           ((e.kind == EPI_RELU && !e.final_mode && !e.GP && !e.GPh && !e.AP) ||
                            (e.kind == EPI_CONC && !e.X) || e.kind == EPI_STORE);
  float c0 = 0.f;
  float part = 0.f;
  if (rows.cidx) {
    // combination of three neurons of zhat_t: a = sum_k c_k W_t[j_k, :]
    const LayerDev& L = edge == 0 ? net.aff[t] : net.aff2[t];
    int jk[3];
    float ck[3];
    for (int k = 0; k < 3; ++k) {
      jk[k] = rows.cidx[3 * m + k];
      ck[k] = rows.ccoef[3 * m + k];
      if (edge == 0) {
        const float bj = net.bfull[t] ? net.bfull[t][jk[k]]
                                      : (L.kind == 1 ? L.b[jk[k]] : L.b[jk[k] / (L.ho * L.wo)]);
        c0 += ck[k] * bj;
      }
    }
    const int hw = L.ho * L.wo, ihw = L.hi * L.wi;
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
      float a = 0.f;
      for (int k = 0; k < 3; ++k) {
        if (ck[k] == 0.f) continue;
        if (L.kind == 1) {
          a += ck[k] * L.W[(size_t)jk[k] * width + col];
        } else {
          const int co = jk[k] / hw, oh = (jk[k] % hw) / L.wo, ow = jk[k] % L.wo;
          const int ci = col / ihw, kh = (col % ihw) / L.wi - (oh * L.s - L.p);
          const int kw = col % L.wi - (ow * L.s - L.p);
          if (kh >= 0 && kh < L.k && kw >= 0 && kw < L.k)
            a += ck[k] * L.W[(((size_t)co * L.ci + ci) * L.k + kh) * L.k + kw];
        }
      }
      const float o = epi_apply(e, m, col, a, part);
      if (out) out[(size_t)m * ld + col] = o;
    }
  } else if (t == net.R + 1) {
    const PropDev& P = e.props[e.pool.prop[n]];
    const float* w = P.Wf + (size_t)j * width;
    c0 = P.bf[j];
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
      const float o = epi_apply(e, m, col, w[col], part);
      if (out) out[(size_t)m * ld + col] = o;
    }
  } else {
    const LayerDev& L = edge == 0 ? net.aff[t] : net.aff2[t];
    if (edge == 0) {
      const float bj = net.bfull[t] ? net.bfull[t][j]
                                    : (L.kind == 1 ? L.b[j] : L.b[j / (L.ho * L.wo)]);
      c0 = sg * bj;
    }
    if (L.kind == 1) {
      const float* w = L.W + (size_t)j * width;
      for (int col = threadIdx.x; col < width; col += blockDim.x) {
        const float o = epi_apply(e, m, col, sg * w[col], part);
        if (out) out[(size_t)m * ld + col] = o;
      }
    } else if (!out && zero_passes) {
      // only the kernel window of neuron j = (co, oh, ow) is nonzero and
      // nothing is stored: walk the window
      const int hw = L.ho * L.wo;
      const int co = j / hw, oh = (j % hw) / L.wo, ow = j % L.wo;
      const int h0 = oh * L.s - L.p, w0 = ow * L.s - L.p;
      const int kk = L.k * L.k;
      for (int q = threadIdx.x; q < L.ci * kk; q += blockDim.x) {
        const int ci = q / kk, kh = (q % kk) / L.k, kw = q % L.k;
        const int ih = h0 + kh, iw = w0 + kw;
        if (ih < 0 || ih >= L.hi || iw < 0 || iw >= L.wi) continue;
        const float a = sg * L.W[(((size_t)co * L.ci + ci) * L.k + kh) * L.k + kw];
        epi_apply(e, m, (ci * L.hi + ih) * L.wi + iw, a, part);
      }
    } else {
      // row j = (co, oh, ow) of the convolution's Toeplitz matrix
      const int hw = L.ho * L.wo;
      const int co = j / hw, oh = (j % hw) / L.wo, ow = j % L.wo;
      const int h0 = oh * L.s - L.p, w0 = ow * L.s - L.p;
      const int ihw = L.hi * L.wi;
      for (int col = threadIdx.x; col < width; col += blockDim.x) {
        const int ci = col / ihw, ih = (col % ihw) / L.wi, iw = col % L.wi;
        const int kh = ih - h0, kw = iw - w0;
        if (kh >= 0 && kh < L.k && kw >= 0 && kw < L.k) {
          const float a = sg * L.W[(((size_t)co * L.ci + ci) * L.k + kh) * L.k + kw];
          const float o = epi_apply(e, m, col, a, part);
          if (out) out[(size_t)m * ld + col] = o;
        } else if (zero_passes) {
          // outside the receptive field a = 0 and, without beta or gamma terms,
          // the ReLU step maps it to 0 with no offset contribution
          if (out) out[(size_t)m * ld + col] = 0.f;
        } else {
          const float o = epi_apply(e, m, col, 0.f, part);
          if (out) out[(size_t)m * ld + col] = o;
        }
      }
    }
  }
  const float tot = block_sum(part);
  if (threadIdx.x == 0 && e.part) e.part[(size_t)m * e.nslot + e.slot_base] = tot + c0;
}

void launch_init_rows(const NetDev& net, int t, int edge, const RowsDev& rows, float* out, int ld,
                      const Epi& e, cudaStream_t st) {
  if (rows.M <= 0) return;
  k_init_rows<<<rows.M, 128, 0, st>>>(net, t, edge, rows, out, ld, e);
}

// ---------------------------------------------------------------------------
// rows of layer 1: one affine step from the input box, then concretisation
// ---------------------------------------------------------------------------
// lb = sign * b_j + sum_k min(a_k lo_k, a_k hi_k), a = sign * W_1[j, :]; a conv
// neuron touches only its k x k x ci patch (one thread per row), an FC neuron
// its whole weight row (one warp per row).
__global__ void k_first_rows_conv(NetDev net, PoolDev pool, const PropDev* props, RowsDev rows,
                                  float* lb) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= rows.M) return;
  const LayerDev& L = net.aff[1];
  const int j = rows.j[m];
  const float sg = rows.sign ? rows.sign[m] : 1.f;
  const PropDev& P = props[pool.prop[rows.node[m]]];
  const int hw = L.ho * L.wo;
  const int co = j / hw, oh = (j % hw) / L.wo, ow = j % L.wo;
  const int h0 = oh * L.s - L.p, w0 = ow * L.s - L.p;
  const float* w = L.W + (size_t)co * L.ci * L.k * L.k;
  float acc = 0.f;
  for (int ci = 0; ci < L.ci; ++ci)
    for (int kh = 0; kh < L.k; ++kh) {
      const int ih = h0 + kh;
      if (ih < 0 || ih >= L.hi) continue;
      for (int kw = 0; kw < L.k; ++kw) {
        const int iw = w0 + kw;
        if (iw < 0 || iw >= L.wi) continue;
        const float a = sg * __ldg(w + (ci * L.k + kh) * L.k + kw);
        const int x = (ci * L.hi + ih) * L.wi + iw;
        acc += a * (a >= 0.f ? P.lo[x] : P.hi[x]);
      }
    }
  lb[m] = acc + sg * (net.bfull[1] ? net.bfull[1][j] : L.b[co]);
}

__global__ void k_first_rows_fc(NetDev net, PoolDev pool, const PropDev* props, RowsDev rows,
                                float* lb) {
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= rows.M) return;
  const LayerDev& L = net.aff[1];
  const int j = rows.j[m];
  const float sg = rows.sign ? rows.sign[m] : 1.f;
  const PropDev& P = props[pool.prop[rows.node[m]]];
  const float* w = L.W + (size_t)j * L.d_in;
  float acc = 0.f;
  for (int k = lane; k < L.d_in; k += 32) {
    const float a = sg * __ldg(w + k);
    acc += a * (a >= 0.f ? P.lo[k] : P.hi[k]);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lb[m] = acc + sg * (net.bfull[1] ? net.bfull[1][j] : L.b[j]);
}

void launch_first_rows(const NetDev& net, const PoolDev& pool, const PropDev* props,
                       const RowsDev& rows, float* lb, cudaStream_t st) {
  if (rows.M <= 0) return;
  if (net.aff[1].kind == MNBAB_CONV2D)
    k_first_rows_conv<<<(rows.M + 127) / 128, 128, 0, st>>>(net, pool, props, rows, lb);
  else
    k_first_rows_fc<<<(rows.M + 7) / 8, 256, 0, st>>>(net, pool, props, rows, lb);
}

// ---------------------------------------------------------------------------
// windowed rows (intermediate bounds of convolution neurons)
// ---------------------------------------------------------------------------
// A row at neuron (co, oh, ow) of zhat_t starts, after its first step, as the
// k x k kernel patch of output channel co with origin (oh s - p, ow s - p) at
// layer t-1.  A convolution (stride s, kernel k, padding p) maps coefficients
// on an h x w window with origin (y0, x0) to a ((h-1)s + k) x ((w-1)s + k)
// window with origin (y0 s - p, x0 s - p); relative output position yy takes
// input position Y = (yy - kh) / s wherever that is an integer in [0, h).
// Positions outside the layer (padding) carry no coefficient.
constexpr int WIN_MAX_FLOATS = 12288;  // per buffer: two buffers = 96 KB

bool win_plan(const NetDev& net, int t, WinPlan& wp) {
  if (t < 2 || t > net.R) return false;  // rows at layer 1 are direct in k_init_rows
  for (int i = 1; i <= t; ++i)
    if (net.n_edge[i] != 1 || net.src1[i] != i - 1 || net.aff[i].kind != MNBAB_CONV2D)
      return false;
  wp.t = t;
  int h = net.aff[t].k, w = net.aff[t].k;
  wp.h[t - 1] = h;
  wp.w[t - 1] = w;
  int mx = net.aff[t].ci * h * w;
  for (int i = t - 1; i >= 1; --i) {
    const LayerDev& L = net.aff[i];
    h = (h - 1) * L.s + L.k;
    w = (w - 1) * L.s + L.k;
    wp.h[i - 1] = h;
    wp.w[i - 1] = w;
    mx = std::max(mx, L.ci * h * w);
  }
  wp.maxw = mx;
  return mx <= WIN_MAX_FLOATS;
}

__global__ void k_win_rows(NetDev net, WinPlan wp, RowsDev rows, Epi e) {
  extern __shared__ __align__(16) float wsm[];
  float* A = wsm;
  float* B = wsm + wp.maxw;
  const int m = blockIdx.x;
  const int t = wp.t;
  const int j = rows.j[m];
  const float sg = rows.sign ? rows.sign[m] : 1.f;
  const LayerDev& Lt = net.aff[t];
  const int hwt = Lt.ho * Lt.wo;
  const int co = j / hwt, oh = (j % hwt) / Lt.wo, ow = j % Lt.wo;
  int y0 = oh * Lt.s - Lt.p, x0 = ow * Lt.s - Lt.p;
  {
    const int n0 = Lt.ci * Lt.k * Lt.k;
    for (int q = threadIdx.x; q < n0; q += blockDim.x) A[q] = sg * __ldg(Lt.W + (size_t)co * n0 + q);
  }
  const float c0 = sg * (net.bfull[t] ? net.bfull[t][j] : Lt.b[co]);
  float part = 0.f;
  int h = Lt.k, w = Lt.k;
  for (int i = t - 1; i >= 0; --i) {
    const LayerDev& Ln = net.aff[i + 1];  // layer i is this edge's input
    const int C = Ln.ci, H = Ln.hi, W = Ln.wi, hw = h * w;
    __syncthreads();
    if (i == 0) {
      // concretisation over the input box
      const PropDev& P = e.props[e.pool.prop[rows.node[m]]];
      for (int q = threadIdx.x; q < C * hw; q += blockDim.x) {
        const int c = q / hw, r = q % hw, y = y0 + r / w, x = x0 + r % w;
        if (y < 0 || y >= H || x < 0 || x >= W) continue;
        const int jx = (c * H + y) * W + x;
        const float a = A[q];
        part += a * (a >= 0.f ? P.lo[jx] : P.hi[jx]);
      }
      break;
    }
    // ReLU step of layer i (DeepPoly slopes, splits enforced)
    Epi el = e;
    el.kind = EPI_RELU;
    el.off = net.off[i];
    el.bias = net.bfull[i];
    el.bias_div = 1;
    for (int q = threadIdx.x; q < C * hw; q += blockDim.x) {
      const int c = q / hw, r = q % hw, y = y0 + r / w, x = x0 + r % w;
      if (y < 0 || y >= H || x < 0 || x >= W) {
        A[q] = 0.f;
        continue;
      }
      A[q] = epi_relu(el, m, (c * H + y) * W + x, A[q], part);
    }
    __syncthreads();
    // transposed convolution through layer i's edge
    const LayerDev& Li = net.aff[i];
    const int s = Li.s, k = Li.k, kk = k * k;
    const int h2 = (h - 1) * s + k, w2 = (w - 1) * s + k, hw2 = h2 * w2;
    const int y2 = y0 * s - Li.p, x2 = x0 * s - Li.p;
    const size_t wco = (size_t)Li.ci * kk;  // stride of W over output channels
    for (int q = threadIdx.x; q < Li.ci * hw2; q += blockDim.x) {
      const int c = q / hw2, r = q % hw2, yy = r / w2, xx = r % w2;
      const int ya = y2 + yy, xa = x2 + xx;
      float acc = 0.f;
      if (ya >= 0 && ya < Li.hi && xa >= 0 && xa < Li.wi) {
        for (int kh = yy % s; kh < k && kh <= yy; kh += s) {
          const int Y = (yy - kh) / s;
          if (Y >= h) continue;
          for (int kw = xx % s; kw < k && kw <= xx; kw += s) {
            const int X = (xx - kw) / s;
            if (X >= w) continue;
            const float* ap = A + Y * w + X;
            const float* wp2 = Li.W + (size_t)c * kk + kh * k + kw;
            for (int o = 0; o < Li.co; ++o) acc = fmaf(ap[o * hw], __ldg(wp2 + o * wco), acc);
          }
        }
      }
      B[q] = acc;
    }
    float* tmp = A;
    A = B;
    B = tmp;
    h = h2;
    w = w2;
    y0 = y2;
    x0 = x2;
  }
  const float tot = block_sum(part);
  if (threadIdx.x == 0) e.part[(size_t)m * e.nslot + e.slot_base] = tot + c0;
}

// The same windowed rows, RB rows per CTA in lockstep (small windows): every
// phase covers the RB rows' windows, so each barrier and index computation
// serves RB rows; row q keeps its own window origin, node and partial sum.
template <int RB>
__global__ void k_win_rows_rb(NetDev net, WinPlan wp, RowsDev rows, Epi e) {
  extern __shared__ __align__(16) float wsm[];
  const int t = wp.t;
  const LayerDev& Lt = net.aff[t];
  const int m0 = blockIdx.x * RB;
  float* A = wsm;                   // RB planes of wp.maxw
  float* B = wsm + RB * wp.maxw;
  int y0[RB], x0[RB], mq[RB];
  float part[RB], c0[RB];
  const int hwt = Lt.ho * Lt.wo;
  const int n0 = Lt.ci * Lt.k * Lt.k;
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    const bool in = m0 + q < rows.M;
    mq[q] = in ? m0 + q : m0;  // absent rows repeat the first (results dropped)
    const int j = rows.j[mq[q]];
    const float sg = rows.sign ? rows.sign[mq[q]] : 1.f;
    const int co = j / hwt, oh = (j % hwt) / Lt.wo, ow = j % Lt.wo;
    y0[q] = oh * Lt.s - Lt.p;
    x0[q] = ow * Lt.s - Lt.p;
    c0[q] = sg * (net.bfull[t] ? net.bfull[t][j] : Lt.b[co]);
    part[q] = 0.f;
    for (int i = threadIdx.x; i < n0; i += blockDim.x)
      A[q * wp.maxw + i] = sg * __ldg(Lt.W + (size_t)co * n0 + i);
  }
  int h = Lt.k, w = Lt.k;
  for (int i = t - 1; i >= 0; --i) {
    const LayerDev& Ln = net.aff[i + 1];
    const int C = Ln.ci, H = Ln.hi, W = Ln.wi, hw = h * w;
    __syncthreads();
    if (i == 0) {
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const PropDev& P = e.props[e.pool.prop[rows.node[mq[q]]]];
        for (int r0 = threadIdx.x; r0 < C * hw; r0 += blockDim.x) {
          const int c = r0 / hw, r = r0 % hw, y = y0[q] + r / w, x = x0[q] + r % w;
          if (y < 0 || y >= H || x < 0 || x >= W) continue;
          const int jx = (c * H + y) * W + x;
          const float a = A[q * wp.maxw + r0];
          part[q] += a * (a >= 0.f ? P.lo[jx] : P.hi[jx]);
        }
      }
      break;
    }
    Epi el = e;
    el.kind = EPI_RELU;
    el.off = net.off[i];
    el.bias = net.bfull[i];
    el.bias_div = 1;
#pragma unroll
    for (int q = 0; q < RB; ++q)
      for (int r0 = threadIdx.x; r0 < C * hw; r0 += blockDim.x) {
        const int c = r0 / hw, r = r0 % hw, y = y0[q] + r / w, x = x0[q] + r % w;
        float* a = A + q * wp.maxw + r0;
        if (y < 0 || y >= H || x < 0 || x >= W) {
          *a = 0.f;
          continue;
        }
        *a = epi_relu(el, mq[q], (c * H + y) * W + x, *a, part[q]);
      }
    __syncthreads();
    const LayerDev& Li = net.aff[i];
    const int s = Li.s, k = Li.k, kk = k * k;
    const int h2 = (h - 1) * s + k, w2 = (w - 1) * s + k, hw2 = h2 * w2;
    const size_t wco = (size_t)Li.ci * kk;
    for (int r0 = threadIdx.x; r0 < Li.ci * hw2; r0 += blockDim.x) {
      const int c = r0 / hw2, r = r0 % hw2, yy = r / w2, xx = r % w2;
      float acc[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) acc[q] = 0.f;
      for (int kh = yy % s; kh < k && kh <= yy; kh += s) {
        const int Y = (yy - kh) / s;
        if (Y >= h) continue;
        for (int kw = xx % s; kw < k && kw <= xx; kw += s) {
          const int X = (xx - kw) / s;
          if (X >= w) continue;
          const float* ap = A + Y * w + X;
          const float* wp2 = Li.W + (size_t)c * kk + kh * k + kw;
          for (int o = 0; o < Li.co; ++o) {
            const float wv = __ldg(wp2 + o * wco);
#pragma unroll
            for (int q = 0; q < RB; ++q) acc[q] = fmaf(ap[q * wp.maxw + o * hw], wv, acc[q]);
          }
        }
      }
      // positions outside the layer (padding) carry no coefficient
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int ya = y0[q] * s - Li.p + yy, xa = x0[q] * s - Li.p + xx;
        B[q * wp.maxw + r0] = (ya >= 0 && ya < Li.hi && xa >= 0 && xa < Li.wi) ? acc[q] : 0.f;
      }
    }
    float* tmp = A;
    A = B;
    B = tmp;
    h = h2;
    w = w2;
#pragma unroll
    for (int q = 0; q < RB; ++q) {
      y0[q] = y0[q] * s - Li.p;
      x0[q] = x0[q] * s - Li.p;
    }
  }
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    const float tot = block_sum(part[q]);
    if (threadIdx.x == 0 && m0 + q < rows.M)
      e.part[(size_t)(m0 + q) * e.nslot + e.slot_base] = tot + c0[q];
  }
}

void launch_win_rows(const NetDev& net, const WinPlan& wp, const RowsDev& rows, const Epi& e,
                     cudaStream_t st) {
  if (rows.M <= 0) return;
  if (wp.maxw <= 1024) {
    constexpr int RB = 4;
    const int smem = 2 * RB * wp.maxw * (int)sizeof(float);
    k_win_rows_rb<RB><<<(rows.M + RB - 1) / RB, 128, smem, st>>>(net, wp, rows, e);
    return;
  }
  const int threads = wp.maxw >= 1024 ? 256 : 128;
  const int smem = 2 * wp.maxw * (int)sizeof(float);
  set_smem(k_win_rows, smem);
  k_win_rows<<<rows.M, threads, smem, st>>>(net, wp, rows, e);
}

// ---------------------------------------------------------------------------
// dense GEMM C = A B (+ bias) with a fused epilogue; SIMT FP32, 64x64x16 tiles
// ---------------------------------------------------------------------------
constexpr int GBK = 16;

// BM x BN tile, 256 threads as 16 x 16, each thread (BM/16) x (BN/16) outputs.
template <int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A,
                                              int lda, const float* __restrict__ B, int ldb,
                                              const float* __restrict__ bias, int bias_div,
                                              float* C, int ldc, Epi e) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ float As[GBK][BM + 4];
  __shared__ float Bs[GBK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    for (int q = tid; q < BM * GBK; q += 256) {
      const int r = q >> 4, cc = q & 15;
      const int gm = m0 + r, gk = k0 + cc;
      As[cc][r] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.f;
    }
    for (int q = tid; q < BN * GBK; q += 256) {
      const int r = q / BN, cc = q % BN;
      const int gk = k0 + r, gn = n0 + cc;
      Bs[r][cc] = (gk < K && gn < N) ? B[(size_t)gk * ldb + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float part[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) part[i] = 0.f;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[n / bias_div];
      const float o = epi_apply(e, m, n, v, part[i]);
      if (C) C[(size_t)m * ldc + n] = o;
    }
  }
  if (epi_has_part(e)) {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      float p = part[i];
      for (int o = 8; o; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o, 16);
      const int m = m0 + ty + 16 * i;
      if (tx == 0 && m < M) e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = p;
    }
  }
}

// Split-K partial products: CTA z computes K range [z*kc, (z+1)*kc) of a
// 32 x 32 tile into ws[z][m][n] (no epilogue).
__global__ void __launch_bounds__(256) k_gemm_splitk(int M, int N, int K, int kc,
                                                     const float* __restrict__ A, int lda,
                                                     const float* __restrict__ B, int ldb,
                                                     float* __restrict__ ws) {
  __shared__ float As[GBK][32 + 4];
  __shared__ float Bs[GBK][32 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = kb; k0 < ke; k0 += GBK) {
    for (int q = tid; q < 32 * GBK; q += 256) {
      const int r = q >> 4, cc = q & 15;
      const int gm = m0 + r, gk = k0 + cc;
      As[cc][r] = (gm < M && gk < ke) ? A[(size_t)gm * lda + gk] : 0.f;
    }
    for (int q = tid; q < 32 * GBK; q += 256) {
      const int r = q >> 5, cc = q & 31;
      const int gk = k0 + r, gn = n0 + cc;
      Bs[r][cc] = (gk < ke && gn < N) ? B[(size_t)gk * ldb + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      const float a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  float* w = ws + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) w[(size_t)m * N + n] = acc[i][j];
    }
}

// Sum of the split-K partials (fixed order) + bias, then the epilogue; a CTA
// covers 8 rows x 32 columns, one warp per row, and writes one offset partial
// per (row, 32-column tile).
__global__ void __launch_bounds__(256) k_splitk_epi(int M, int N, int S, const float* __restrict__ ws,
                                                    const float* __restrict__ bias, int bias_div,
                                                    float* C, int ldc, Epi e) {
  const int m = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int n = blockIdx.x * 32 + (threadIdx.x & 31);
  float part = 0.f;
  if (m < M && n < N) {
    float v = 0.f;
    for (int z = 0; z < S; ++z) v += ws[((size_t)z * M + m) * N + n];
    if (bias) v += bias[n / bias_div];
    const float o = epi_apply(e, m, n, v, part);
    if (C) C[(size_t)m * ldc + n] = o;
  }
  if (epi_has_part(e)) {
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && m < M)
      e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = part;
  }
}

// 64 x 64 tiles unless that grid would leave most of the 152 SMs idle; then
// 32 x 32 tiles, split along K when the K loop is long and the workspace fits.
// SIMT GEMM variants: V_SPLITK (reduction split over up to 16 CTAs per tile
// so that small products fill the SMs; -1 when no split is possible), V_G64,
// V_G32.
static int gemm_variant(int v, int M, int N, int K, const float* A, int lda, const float* B,
                        int ldb, const float* bias, int bias_div, float* C, int ldc, const Epi& e,
                        cudaStream_t st) {
  if (v == V_SPLITK) {
    if (K < 256 || !e.ws) return -1;
    const long small = (long)((N + 31) / 32) * ((M + 31) / 32);
    int S = (int)std::min<long>(16, std::max<long>(2, (2 * 152 + small - 1) / small));
    S = std::min(S, K / 64);
    while (S > 1 && (size_t)S * M * N > e.ws_floats) --S;
    if (S <= 1) return -1;
    const int kc = ((K + S - 1) / S + GBK - 1) / GBK * GBK;
    S = (K + kc - 1) / kc;
    dim3 g1((N + 31) / 32, (M + 31) / 32, S);
    k_gemm_splitk<<<g1, 256, 0, st>>>(M, N, K, kc, A, lda, B, ldb, e.ws);
    dim3 g2((N + 31) / 32, (M + 7) / 8);
    k_splitk_epi<<<g2, 256, 0, st>>>(M, N, S, e.ws, bias, bias_div, C, ldc, e);
    return g2.x;
  }
  if (v == V_G64) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<64, 64><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, bias, bias_div, C, ldc, e);
    return grid.x;
  }
  if (v == V_G32) {
    dim3 grid((N + 31) / 32, (M + 31) / 32);
    k_gemm<32, 32><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, bias, bias_div, C, ldc, e);
    return grid.x;
  }
  return -1;
}

// built-in choice: split-K when neither tiling fills two waves, else 64 x 64
// tiles when they do, else 32 x 32
static int gemm_launch(int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                       const float* bias, int bias_div, float* C, int ldc, const Epi& e,
                       cudaStream_t st) {
  const long big = (long)((N + 63) / 64) * ((M + 63) / 64);
  const long small = (long)((N + 31) / 32) * ((M + 31) / 32);
  if (big < 2 * 152 && small < 2 * 152) {
    const int r = gemm_variant(V_SPLITK, M, N, K, A, lda, B, ldb, bias, bias_div, C, ldc, e, st);
    if (r >= 0) return r;
  }
  return gemm_variant(big >= 2 * 152 ? V_G64 : V_G32, M, N, K, A, lda, B, ldb, bias, bias_div, C,
                      ldc, e, st);
}

// ---------------------------------------------------------------------------
// convolution: transposed (back-substitution) and forward (adjoint / forward)
// ---------------------------------------------------------------------------
// Input positions are enumerated phase-major (ih mod s, iw mod s) so that the
// threads of a warp share kernel taps and read the weights from shared memory
// as broadcasts.
__device__ __forceinline__ void decode_phase(int pidx, int hi, int wi, int s, int& ih, int& iw) {
  for (int ph = 0; ph < s; ++ph) {
    const int nh = (hi - ph + s - 1) / s;
    for (int pw = 0; pw < s; ++pw) {
      const int nw = (wi - pw + s - 1) / s;
      const int cnt = nh * nw;
      if (pidx < cnt) {
        ih = ph + s * (pidx / nw);
        iw = pw + s * (pidx % nw);
        return;
      }
      pidx -= cnt;
    }
  }
  ih = iw = -1;
}

template <int CB>
__global__ void __launch_bounds__(128) k_convT(int M, const float* __restrict__ in, int ld_in,
                                               float* out, int ld_out, LayerDev L, Epi e) {
  extern __shared__ float Ws[];
  const int nW = L.co * L.ci * L.k * L.k;
  for (int i = threadIdx.x; i < nW; i += blockDim.x) Ws[i] = L.W[i];
  __syncthreads();
  const int m = blockIdx.y;
  const int Pin = L.hi * L.wi;
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  float part = 0.f;
  if (pidx < Pin) {
    int ih, iw;
    decode_phase(pidx, L.hi, L.wi, L.s, ih, iw);
    const float* lam = in + (size_t)m * ld_in;
    const int kk = L.k * L.k;
    const int hwo = L.ho * L.wo;
    const int kh0 = (ih + L.p) % L.s, kw0 = (iw + L.p) % L.s;
    for (int cb = 0; cb < L.ci; cb += CB) {
      float acc[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) acc[c] = 0.f;
      for (int kh = kh0; kh < L.k; kh += L.s) {
        const int th = ih + L.p - kh;
        if (th < 0) break;
        const int oh = th / L.s;
        if (oh >= L.ho) continue;
        for (int kw = kw0; kw < L.k; kw += L.s) {
          const int tw = iw + L.p - kw;
          if (tw < 0) break;
          const int ow = tw / L.s;
          if (ow >= L.wo) continue;
          const float* lp = lam + oh * L.wo + ow;
          const float* wp = Ws + (size_t)cb * kk + kh * L.k + kw;
          for (int co = 0; co < L.co; ++co) {
            const float v = lp[(size_t)co * hwo];
            const float* w = wp + (size_t)co * L.ci * kk;
#pragma unroll
            for (int c = 0; c < CB; ++c)
              if (CB == 1 || cb + c < L.ci) acc[c] = fmaf(v, w[c * kk], acc[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int ci = cb + c;
        if (ci >= L.ci) break;
        const int j = ci * Pin + ih * L.wi + iw;
        const float o = epi_apply(e, m, j, acc[c], part);
        if (out) out[(size_t)m * ld_out + j] = o;
      }
    }
  }
  if (epi_has_part(e)) {
    const float tot = block_sum(part);
    if (threadIdx.x == 0) e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = tot;
  }
}

template <int CB>
__global__ void __launch_bounds__(128) k_conv_fwd(int M, const float* __restrict__ in, int ld_in,
                                                  float* out, int ld_out, LayerDev L, Epi e) {
  extern __shared__ float Ws[];
  const int nW = L.co * L.ci * L.k * L.k;
  for (int i = threadIdx.x; i < nW; i += blockDim.x) Ws[i] = L.W[i];
  __syncthreads();
  // rows_per: rows sharing one CTA (output planes smaller than the CTA)
  const int Pout = L.ho * L.wo;
  const int rows_per = Pout >= (int)blockDim.x ? 1 : (int)blockDim.x / Pout;
  const int m = rows_per == 1 ? (int)blockIdx.y : (int)blockIdx.y * rows_per + (int)threadIdx.x / Pout;
  const int pos = rows_per == 1 ? (int)(blockIdx.x * blockDim.x + threadIdx.x) : (int)threadIdx.x % Pout;
  float part = 0.f;
  if (pos < Pout && m < M && (rows_per == 1 || (int)threadIdx.x < rows_per * Pout)) {
    const int oh = pos / L.wo, ow = pos % L.wo;
    const float* x = in + (size_t)m * ld_in;
    const int kk = L.k * L.k;
    const int hwi = L.hi * L.wi;
    for (int cb = 0; cb < L.co; cb += CB) {
      float acc[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) acc[c] = 0.f;
      for (int ci = 0; ci < L.ci; ++ci) {
        for (int kh = 0; kh < L.k; ++kh) {
          const int ih = oh * L.s - L.p + kh;
          if (ih < 0 || ih >= L.hi) continue;
          for (int kw = 0; kw < L.k; ++kw) {
            const int iw = ow * L.s - L.p + kw;
            if (iw < 0 || iw >= L.wi) continue;
            const float v = x[(size_t)ci * hwi + ih * L.wi + iw];
            const float* w = Ws + ((size_t)cb * L.ci + ci) * kk + kh * L.k + kw;
#pragma unroll
            for (int c = 0; c < CB; ++c)
              if (CB == 1 || cb + c < L.co) acc[c] = fmaf(v, w[(size_t)c * L.ci * kk], acc[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        const int co = cb + c;
        if (co >= L.co) break;
        const int j = co * Pout + pos;
        const float o = epi_apply(e, m, j, acc[c] + L.b[co], part);
        if (out) out[(size_t)m * ld_out + j] = o;
      }
    }
  }
  // forward epilogues (adjoint, ReLU) produce no offset partials; the partial
  // slot layout below assumes one row per CTA
  if (epi_has_part(e) && rows_per == 1) {
    const float tot = block_sum(part);
    if (threadIdx.x == 0) e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = tot;
  }
}

// Staging into shared memory with all of a thread's loads in flight: rows of
// `width` floats taken at src + r * stride (r < nrows), written densely.  float4
// loads when every row start is 16-byte aligned, 4 per thread per round.
__device__ __forceinline__ void stage_rows(float* __restrict__ dst, const float* __restrict__ src,
                                           int nrows, int width, size_t stride, int valid) {
  const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                     (stride * 4)) & 15) == 0 &&
                   (width & 3) == 0 && (valid & 3) == 0;
  if (vec) {
    const int w4 = width >> 2, n4 = nrows * w4;
    float4* d4 = reinterpret_cast<float4*>(dst);
    int i = threadIdx.x;
    const int bd = blockDim.x;
    for (; i + 3 * bd < n4; i += 4 * bd) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ii = i + u * bd, r = ii / w4, c = (ii % w4) * 4;
        v[u] = c < valid ? __ldg(reinterpret_cast<const float4*>(src + r * stride + c))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) d4[i + u * bd] = v[u];
    }
    for (; i < n4; i += bd) {
      const int r = i / w4, c = (i % w4) * 4;
      d4[i] = c < valid ? __ldg(reinterpret_cast<const float4*>(src + r * stride + c))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  const int n = nrows * width;
  int i = threadIdx.x;
  const int bd = blockDim.x;
  for (; i + 3 * bd < n; i += 4 * bd) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ii = i + u * bd, r = ii / width, c = ii % width;
      v[u] = c < valid ? __ldg(src + r * stride + c) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) dst[i + u * bd] = v[u];
  }
  for (; i < n; i += bd) {
    const int r = i / width, c = i % width;
    dst[i] = c < valid ? __ldg(src + r * stride + c) : 0.f;
  }
}

// Row-resident convolution kernels.  A CTA takes one row, one chunk of output
// positions and one group of channel blocks.  It stages the row's input and
// its slice of the weights (pre-arranged in global memory so that a channel
// block is contiguous, float4 loads) in shared memory; each thread computes
// CB channels of one output position.  Few rows are spread over more CTAs
// (position chunks x channel groups) so that a launch fills the GPU.
struct ConvSplit {
  int ppc;   // positions per chunk
  int npc;   // position chunks
  int bpg;   // channel blocks per group
  int ngrp;  // channel groups
};

// smem_of(channel width) gives the staged floats for a slice of that width;
// groups are added until the slice fits in `limit` floats.
template <typename F>
static ConvSplit conv_split(int M, int P, int nblk, int CB, F smem_of, int limit) {
  const int per_row = std::max(1, std::min(32, (4 * 152 + M - 1) / M));
  ConvSplit cs;
  int min_grp = 1;
  while (min_grp < nblk && smem_of(((nblk + min_grp - 1) / min_grp) * CB) > limit) ++min_grp;
  cs.ngrp = std::max(min_grp, std::min(nblk, per_row));
  cs.bpg = (nblk + cs.ngrp - 1) / cs.ngrp;
  cs.ngrp = (nblk + cs.bpg - 1) / cs.bpg;
  cs.npc = std::max(1, std::min((per_row + cs.ngrp - 1) / cs.ngrp, (P + 31) / 32));
  cs.npc = std::max(cs.npc, (P + 1023) / 1024);
  cs.ppc = (P + cs.npc - 1) / cs.npc;
  cs.npc = (P + cs.ppc - 1) / cs.ppc;
  return cs;
}

static int convT_row_smem(const LayerDev& L, int cwidth) {
  return L.co * L.ho * L.wo + L.co * L.k * L.k * cwidth;
}

template <int CB>
__global__ void __launch_bounds__(128) k_convT_row(int M, const float* __restrict__ in, int ld_in,
                                                   float* out, int ld_out, LayerDev L, Epi e,
                                                   ConvSplit cs) {
  extern __shared__ __align__(16) float sm[];
  const int kk = L.k * L.k;
  const int nIn = L.co * L.ho * L.wo;
  const int chunk = blockIdx.x % cs.npc, grp = blockIdx.x / cs.npc;
  const int nblk = (L.ci + CB - 1) / CB;
  const int b0 = grp * cs.bpg, b1 = min(nblk, b0 + cs.bpg);
  const int c0 = b0 * CB, c1 = min(L.ci, b1 * CB);
  const int cw = cs.bpg * CB;       // stride of the staged channel slice
  float* Ws = sm;                   // [co][kh][kw][cw]
  float* Ls = sm + L.co * kk * cw;  // input row
  const int m = blockIdx.y;
  // weight slice: rows (co, kh, kw) of Wb [co][kh][kw][ci], channels c0 .. c0 + cw
  stage_rows(Ws, L.Wb + c0, L.co * kk, cw, (size_t)L.ci, c1 - c0);
  const float* lam = in + (size_t)m * ld_in;
  // bounding box (over all channels) of the row's nonzero coefficients: rows
  // that start at a convolution neuron are nonzero only in its receptive field
  __shared__ int box[4];
  if (threadIdx.x == 0) { box[0] = L.ho; box[1] = -1; box[2] = L.wo; box[3] = -1; }
  __syncthreads();
  int bh0 = L.ho, bh1 = -1, bw0 = L.wo, bw1 = -1;
  stage_rows(Ls, lam, 1, nIn, 0, nIn);
  __syncthreads();
  // (dense rows: the whole plane)
  if (!e.sparse_rows) {
    bh0 = bw0 = 0;
    bh1 = L.ho - 1;
    bw1 = L.wo - 1;
  }
  for (int i = threadIdx.x; e.sparse_rows && i < nIn; i += blockDim.x) {
    if (Ls[i] != 0.f) {
      const int r = i % (L.ho * L.wo), oh = r / L.wo, ow = r % L.wo;
      bh0 = min(bh0, oh); bh1 = max(bh1, oh); bw0 = min(bw0, ow); bw1 = max(bw1, ow);
    }
  }
  atomicMin(&box[0], bh0); atomicMax(&box[1], bh1); atomicMin(&box[2], bw0); atomicMax(&box[3], bw1);
  __syncthreads();
  // output positions that can be nonzero: ih in [oh0*s - p, oh1*s - p + k - 1]
  const int ih_lo = box[0] * L.s - L.p, ih_hi = box[1] * L.s - L.p + L.k - 1;
  const int iw_lo = box[2] * L.s - L.p, iw_hi = box[3] * L.s - L.p + L.k - 1;
  // a zero coefficient maps to 0 with no offset contribution through these
  // epilogues, so positions outside the window are written as 0 directly
  const bool zero_passes = !e.acc_in &&
                           ((e.kind == EPI_RELU && !e.final_mode && !e.GP && !e.GPh && !e.AP) ||
                            (e.kind == EPI_CONC && !e.X) || e.kind == EPI_STORE);
  const int Pin = L.hi * L.wi;
  const int p0 = chunk * cs.ppc;
  const int np = min(cs.ppc, Pin - p0);
  const int hwo = L.ho * L.wo;
  const int rn = e.row_node[m];
  const PropDev* rp = epi_prop(e, rn);
  float part = 0.f;
  for (int item = threadIdx.x; item < np * (b1 - b0); item += blockDim.x) {
    const int cb = b0 + item / np, pidx = p0 + item % np;
    int ih, iw;
    decode_phase(pidx, L.hi, L.wi, L.s, ih, iw);
    if (zero_passes && (ih < ih_lo || ih > ih_hi || iw < iw_lo || iw > iw_hi)) {
      if (out)
        for (int c = 0; c < CB && cb * CB + c < L.ci; ++c)
          out[(size_t)m * ld_out + (cb * CB + c) * Pin + ih * L.wi + iw] = 0.f;
      continue;
    }
    float acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = 0.f;
    const int kh0 = (ih + L.p) % L.s, kw0 = (iw + L.p) % L.s;
    const int coff = (cb - b0) * CB;
    for (int kh = kh0; kh < L.k; kh += L.s) {
      const int th = ih + L.p - kh;
      if (th < 0) break;
      const int oh = th / L.s;
      if (oh >= L.ho) continue;
      for (int kw = kw0; kw < L.k; kw += L.s) {
        const int tw = iw + L.p - kw;
        if (tw < 0) break;
        const int ow = tw / L.s;
        if (ow >= L.wo) continue;
        const float* lp = Ls + oh * L.wo + ow;
        const float* wp = Ws + (size_t)(kh * L.k + kw) * cw + coff;
        for (int co = 0; co < L.co; ++co) {
          const float v = lp[co * hwo];
          const float* w = wp + (size_t)co * kk * cw;
          if (CB % 4 == 0) {
#pragma unroll
            for (int c = 0; c < CB; c += 4) {
              const float4 w4 = *reinterpret_cast<const float4*>(w + c);
              acc[c] = fmaf(v, w4.x, acc[c]);
              acc[c + 1] = fmaf(v, w4.y, acc[c + 1]);
              acc[c + 2] = fmaf(v, w4.z, acc[c + 2]);
              acc[c + 3] = fmaf(v, w4.w, acc[c + 3]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[c] = fmaf(v, w[c], acc[c]);
          }
        }
      }
    }
    EpiIn pin[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (cb * CB + c < L.ci) epi_load(e, rn, rp, m, (cb * CB + c) * Pin + ih * L.wi + iw, pin[c]);
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int ci = cb * CB + c;
      if (ci >= L.ci) break;
      const int j = ci * Pin + ih * L.wi + iw;
      const float o = epi_finish(e, m, j, acc[c], pin[c], part);
      if (out) out[(size_t)m * ld_out + j] = o;
    }
  }
  if (epi_has_part(e)) {
    const float tot = block_sum(part);
    if (threadIdx.x == 0) e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = tot;
  }
}

static int conv_fwd_row_smem(const LayerDev& L, int cwidth) {
  return L.ci * L.hi * L.wi + L.ci * L.k * L.k * cwidth;
}

template <int CB>
__global__ void __launch_bounds__(128) k_conv_fwd_row(int M, const float* __restrict__ in,
                                                      int ld_in, float* out, int ld_out,
                                                      LayerDev L, Epi e, ConvSplit cs) {
  extern __shared__ __align__(16) float sm[];
  const int kk = L.k * L.k;
  const int nIn = L.ci * L.hi * L.wi;
  const int chunk = blockIdx.x % cs.npc, grp = blockIdx.x / cs.npc;
  const int nblk = (L.co + CB - 1) / CB;
  const int b0 = grp * cs.bpg, b1 = min(nblk, b0 + cs.bpg);
  const int c0 = b0 * CB, c1 = min(L.co, b1 * CB);
  const int cw = cs.bpg * CB;
  float* Ws = sm;                   // [ci][kh][kw][cw]
  float* Xs = sm + L.ci * kk * cw;  // input row
  const int m = blockIdx.y;
  // weight slice: rows (ci, kh, kw) of Wf [ci][kh][kw][co], channels c0 .. c0 + cw
  stage_rows(Ws, L.Wf + c0, L.ci * kk, cw, (size_t)L.co, c1 - c0);
  stage_rows(Xs, in + (size_t)m * ld_in, 1, nIn, 0, nIn);
  __syncthreads();
  const int P = L.ho * L.wo;
  const int p0 = chunk * cs.ppc;
  const int np = min(cs.ppc, P - p0);
  const int hwi = L.hi * L.wi;
  const int rn = (e.kind == EPI_RELU || e.kind == EPI_ADJ) ? e.row_node[m] : 0;
  float part = 0.f;
  for (int item = threadIdx.x; item < np * (b1 - b0); item += blockDim.x) {
    const int cb = b0 + item / np, pos = p0 + item % np;
    const int oh = pos / L.wo, ow = pos % L.wo;
    const int coff = (cb - b0) * CB;
    float acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = 0.f;
    for (int ci = 0; ci < L.ci; ++ci) {
      for (int kh = 0; kh < L.k; ++kh) {
        const int ih = oh * L.s - L.p + kh;
        if (ih < 0 || ih >= L.hi) continue;
        for (int kw = 0; kw < L.k; ++kw) {
          const int iw = ow * L.s - L.p + kw;
          if (iw < 0 || iw >= L.wi) continue;
          const float v = Xs[ci * hwi + ih * L.wi + iw];
          const float* w = Ws + (size_t)((ci * L.k + kh) * L.k + kw) * cw + coff;
          if (CB % 4 == 0) {
#pragma unroll
            for (int c = 0; c < CB; c += 4) {
              const float4 w4 = *reinterpret_cast<const float4*>(w + c);
              acc[c] = fmaf(v, w4.x, acc[c]);
              acc[c + 1] = fmaf(v, w4.y, acc[c + 1]);
              acc[c + 2] = fmaf(v, w4.z, acc[c + 2]);
              acc[c + 3] = fmaf(v, w4.w, acc[c + 3]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[c] = fmaf(v, w[c], acc[c]);
          }
        }
      }
    }
    EpiIn pin[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c)
      if (cb * CB + c < L.co) epi_load(e, rn, nullptr, m, (cb * CB + c) * P + pos, pin[c]);
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      const int co = cb * CB + c;
      if (co >= L.co) break;
      const int j = co * P + pos;
      const float o = epi_finish(e, m, j, acc[c] + L.b[co], pin[c], part);
      if (out) out[(size_t)m * ld_out + j] = o;
    }
  }
  (void)part;  // forward epilogues (adjoint, ReLU) produce no offset partials
}



// ---------------------------------------------------------------------------
// implicit-GEMM convolutions for dense rows
// ---------------------------------------------------------------------------
// Forward: out[m, n, oy, ox] = sum over (ci, kh, kw) of
//   in[m, ci, oy s - p + kh, ox s - p + kw] W[n, ci, kh, kw]  (+ b[n]);
// GEMM rows (m, oy, ox), columns n = co, reduction (ci, kh, kw), weights Wf.
// Transposed (back-substitution): out[m, n, y, x] = sum over (o, kh, kw) with
//   (y + p - kh) and (x + p - kw) divisible by s of
//   in[m, o, (y + p - kh) / s, (x + p - kw) / s] W[o, n, kh, kw].
// Output positions with (y + p) mod s = ry, (x + p) mod s = rx (a parity
// class) take exactly the taps kh = ry + s a, kw = rx + s b, so each class is
// a dense GEMM with reduction (o, a, b) and weights Wb; no masked taps.
// A CTA computes RB rows x one chunk of pc positions of one class x tn
// channels; each row has its own group of tpr threads, so a row's outputs and
// its partial sum do not depend on which rows share the CTA.
struct IgCfg {
  int dir;     // 0 forward, 1 transposed
  int N;       // output channels (co forward, ci transposed)
  int RB, tpr, pc, nchunk, ncls, tn, ngrp, KC;
};

struct IgClass {
  int P, K;             // positions and reduction length of the class
  int y0, x0, ny, nx;   // first output row / column of the class and their counts
  int ry, rx, na, nb;   // residues and tap counts (transposed)
};

__device__ __forceinline__ IgClass ig_class(const LayerDev& L, int dir, int cls) {
  IgClass c;
  if (dir == 0) {
    c.P = L.ho * L.wo;
    c.K = L.ci * L.k * L.k;
    c.y0 = c.x0 = 0;
    c.ny = L.ho;
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
  c.ny = c.y0 < L.hi ? (L.hi - c.y0 + s - 1) / s : 0;
  c.nx = c.x0 < L.wi ? (L.wi - c.x0 + s - 1) / s : 0;
  c.na = c.ry < L.k ? (L.k - c.ry + s - 1) / s : 0;
  c.nb = c.rx < L.k ? (L.k - c.rx + s - 1) / s : 0;
  c.P = c.ny * c.nx;
  c.K = L.co * c.na * c.nb;
  return c;
}

template <int TN>
__global__ void __launch_bounds__(256) k_conv_igemm(int M, const float* __restrict__ in, int ld_in,
                                                    float* out, int ld_out, LayerDev L, Epi e,
                                                    IgCfg g) {
  extern __shared__ __align__(16) float ism[];
  constexpr int TM = 4;
  constexpr int PPT = 4;  // (row, position) pairs a thread gathers: RB pc <= 4 RB tpr
  __shared__ int t_off[32], t_dy[32], t_dx[32], t_row[32];
  const int nthr = blockDim.x;
  float* As = ism;                              // [KC][RB][pc]
  float* Bs = ism + (size_t)g.KC * g.RB * g.pc;  // [KC][tn]
  const int bx = blockIdx.x;
  const int grp = bx % g.ngrp;
  const int chunk = (bx / g.ngrp) % g.nchunk;
  const int cls = bx / (g.ngrp * g.nchunk);
  const IgClass c = ig_class(L, g.dir, cls);
  const int m0 = blockIdx.y * g.RB;
  const int p0 = chunk * g.pc;
  const int np = max(0, min(g.pc, c.P - p0));
  const int n0 = grp * g.tn;
  const int nn = min(g.tn, g.N - n0);
  const int q = threadIdx.x / g.tpr, tl = threadIdx.x % g.tpr;
  const int npg = g.pc / TM, nng = g.tn / TN;
  const int pg = tl % npg, ng = tl / npg;
  const bool act = q < g.RB && ng < nng;
  const int rpc = g.RB * g.pc;
  const float* Wsrc = g.dir == 0 ? L.Wf : L.Wb;
  // source plane of the gather (input of the forward conv, coefficients of the
  // transposed one) and this thread's gather pairs, decoded once
  const int Hs = g.dir == 0 ? L.hi : L.ho, Ws_ = g.dir == 0 ? L.wi : L.wo;
  int pr_base[PPT], pr_y[PPT], pr_x[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int pr = threadIdx.x + i * nthr;
    const int qq = pr / g.pc, pos = pr % g.pc;
    pr_base[i] = -1;
    pr_y[i] = pr_x[i] = 0;
    if (pr < rpc && m0 + qq < M && pos < np) {
      const int pi = p0 + pos;
      const int iy = pi / c.nx, ix = pi % c.nx;
      int y, x;
      if (g.dir == 0) {
        y = iy * L.s - L.p;
        x = ix * L.s - L.p;
      } else {
        y = (c.y0 + L.s * iy + L.p - c.ry) / L.s;
        x = (c.x0 + L.s * ix + L.p - c.rx) / L.s;
      }
      pr_y[i] = y;
      pr_x[i] = x;
      pr_base[i] = 0;  // valid pair; the row offset is added at the load
    }
  }
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int jn = 0; jn < TN; ++jn) acc[i][jn] = 0.f;
  const int Kc = np > 0 ? c.K : 0;
  const int KC = min(g.KC, 32);
  for (int k0 = 0; k0 < Kc; k0 += KC) {
    const int kcn = min(KC, Kc - k0);
    __syncthreads();
    // reduction-index table of this chunk: channel-plane offset, tap shifts, weight row
    if (threadIdx.x < kcn) {
      const int kidx = k0 + threadIdx.x;
      if (g.dir == 0) {
        const int kk2 = L.k * L.k;
        const int ci = kidx / kk2, kh = (kidx / L.k) % L.k, kw = kidx % L.k;
        t_dy[threadIdx.x] = kh;
        t_dx[threadIdx.x] = kw;
        t_off[threadIdx.x] = ci * L.hi * L.wi;
        t_row[threadIdx.x] = kidx;  // Wf [ci][kh][kw][co]
      } else {
        const int nab = c.na * c.nb;
        const int o = kidx / nab, a = (kidx / c.nb) % c.na, b = kidx % c.nb;
        t_dy[threadIdx.x] = -a;
        t_dx[threadIdx.x] = -b;
        t_off[threadIdx.x] = o * L.ho * L.wo;
        t_row[threadIdx.x] = (o * L.k + c.ry + L.s * a) * L.k + c.rx + L.s * b;  // Wb [co][kh][kw][ci]
      }
    }
    __syncthreads();
    // gather the A chunk: consecutive threads take consecutive positions
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int pr = threadIdx.x + i * nthr;
      if (pr >= rpc) break;
      const float* src = in + (size_t)(m0 + pr / g.pc) * ld_in;
      for (int kk = 0; kk < kcn; ++kk) {
        float v = 0.f;
        if (pr_base[i] == 0) {
          const int yy = pr_y[i] + t_dy[kk], xx = pr_x[i] + t_dx[kk];
          if (yy >= 0 && yy < Hs && xx >= 0 && xx < Ws_) v = __ldg(src + t_off[kk] + yy * Ws_ + xx);
        }
        As[kk * rpc + pr] = v;
      }
    }
    // the B chunk: weight rows of the reduction indices, channels n0 .. n0 + tn
    for (int el = threadIdx.x; el < kcn * g.tn; el += nthr) {
      const int kk = el / g.tn, n = el % g.tn;
      Bs[kk * g.tn + n] = n < nn ? __ldg(Wsrc + (size_t)t_row[kk] * g.N + n0 + n) : 0.f;
    }
    __syncthreads();
    if (act) {
      const float* ap = As + q * g.pc + pg * TM;
      const float* bp = Bs + ng * TN;
#pragma unroll 4
      for (int kk = 0; kk < kcn; ++kk) {
        const float4 a4 = *reinterpret_cast<const float4*>(ap + (size_t)kk * rpc);
        float bv[TN];
        if constexpr (TN == 4) {
          const float4 b4 = *reinterpret_cast<const float4*>(bp + kk * g.tn);
          bv[0] = b4.x;
          bv[1] = b4.y;
          bv[2] = b4.z;
          bv[3] = b4.w;
        } else {
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) bv[jn] = bp[kk * g.tn + jn];
        }
        const float av[TM] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) acc[i][jn] = fmaf(av[i], bv[jn], acc[i][jn]);
      }
    }
  }
  // epilogue
  float part = 0.f;
  const int m = m0 + q;
  if (act && m < M) {
    const int plane = g.dir == 0 ? L.ho * L.wo : L.hi * L.wi;
    const int W2 = g.dir == 0 ? L.wo : L.wi;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int pos = pg * TM + i;
      if (pos >= np) break;
      const int pi = p0 + pos;
      const int iy = pi / c.nx, ix = pi % c.nx;
      const int y = g.dir == 0 ? iy : c.y0 + L.s * iy;
      const int x = g.dir == 0 ? ix : c.x0 + L.s * ix;
#pragma unroll
      for (int jn = 0; jn < TN; ++jn) {
        const int n = ng * TN + jn;
        if (n >= nn) break;
        const int j = (n0 + n) * plane + y * W2 + x;
        float v = acc[i][jn];
        if (g.dir == 0) v += L.b[n0 + n];
        const float o = epi_apply(e, m, j, v, part);
        if (out) out[(size_t)m * ld_out + j] = o;
      }
    }
  }
  if (g.dir == 1 && epi_has_part(e)) {
    // per-row sum in a fixed order: warps of the row group, then their sums
    __shared__ float wsum[32];
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = part;
    __syncthreads();
    const int wpr = g.tpr >> 5;
    if (tl == 0 && q < g.RB && m < M) {
      float tot = 0.f;
      for (int w = 0; w < wpr; ++w) tot += wsum[q * wpr + w];
      e.part[(size_t)m * e.nslot + e.slot_base + blockIdx.x] = tot;
    }
  }
}

static IgCfg ig_plan(const LayerDev& L, int dir, int M) {
  IgCfg g;
  g.dir = dir;
  g.N = dir == 0 ? L.co : L.ci;
  const int TN = g.N % 4 == 0 ? 4 : 1;
  g.tn = TN == 4 ? std::min(g.N, 64) : std::min(g.N, 8);
  g.ncls = dir == 0 ? 1 : L.s * L.s;
  int pmax = 0;
  if (dir == 0) {
    pmax = L.ho * L.wo;
  } else {
    for (int r = 0; r < L.s; ++r) {
      const int y0 = ((r - L.p) % L.s + L.s) % L.s;
      const int ny = y0 < L.hi ? (L.hi - y0 + L.s - 1) / L.s : 0;
      for (int r2 = 0; r2 < L.s; ++r2) {
        const int x0 = ((r2 - L.p) % L.s + L.s) % L.s;
        const int nx = x0 < L.wi ? (L.wi - x0 + L.s - 1) / L.s : 0;
        pmax = std::max(pmax, ny * nx);
      }
    }
  }
  const int cap = TN == 4 ? 64 : 128;
  g.pc = std::max(4, std::min((pmax + 3) / 4 * 4, cap));
  // few rows: fewer rows per CTA, then narrower channel groups and shorter
  // position chunks, so that the grid covers the SMs (at most the ig_slots blocks)
  g.RB = 8;
  for (;;) {
    g.ngrp = (g.N + g.tn - 1) / g.tn;
    g.nchunk = std::max(1, (pmax + g.pc - 1) / g.pc);
    g.tpr = ((g.pc / 4) * (g.tn / TN) + 31) / 32 * 32;
    g.RB = std::max(1, std::min(g.RB, 256 / g.tpr));
    const long blocks = (long)((M + g.RB - 1) / g.RB) * g.ncls * g.nchunk * g.ngrp;
    if (blocks >= 2 * 152) break;
    if (g.RB > 1) g.RB >>= 1;
    else if (TN == 4 && g.tn > 16) g.tn = (g.tn / 2 + 3) / 4 * 4;
    else if (g.pc > 16) g.pc = std::max(16, (g.pc / 2 + 3) / 4 * 4);
    else break;
  }
  g.KC = g.RB * g.pc <= 512 ? 32 : 16;  // at most 32 (reduction-index table)
  return g;
}

static int ig_smem(const IgCfg& g) { return g.KC * (g.RB * g.pc + g.tn) * (int)sizeof(float); }

static bool ig_supported(const LayerDev& L, int dir) {
  const IgCfg g = ig_plan(L, dir, 1 << 20);
  return g.tpr <= 256 && ig_smem(g) <= 96 * 1024 && (dir == 0 ? L.Wf : L.Wb) != nullptr;
}

static int ig_slots(const LayerDev& L) {
  // the finest split of ig_plan (one row: position chunks of 16, channel groups of 16)
  const IgCfg g = ig_plan(L, 1, 1);
  return g.ncls * g.nchunk * g.ngrp;
}

// Per-row work above which the implicit GEMM beats the row-resident kernels
// (whose per-row CTAs then serialise too much work)
static bool ig_preferred(const LayerDev& L) {
  return (double)L.co * L.ho * L.wo * L.ci * L.k * L.k >= 512.0 * 1024.0;
}

// launches the implicit-GEMM kernel; returns the partial-sum slots (transposed)
static int launch_ig(const LayerDev& L, int dir, int M, const float* in, int ld_in, float* out,
                     int ld_out, const Epi& e, cudaStream_t st) {
  const IgCfg g = ig_plan(L, dir, M);
  const int smem = ig_smem(g);
  dim3 grid(g.ncls * g.nchunk * g.ngrp, (M + g.RB - 1) / g.RB);
  const int thr = g.RB * g.tpr;
  if (g.N % 4 == 0) {
    set_smem(k_conv_igemm<4>, smem);
    k_conv_igemm<4><<<grid, thr, smem, st>>>(M, in, ld_in, out, ld_out, L, e, g);
  } else {
    set_smem(k_conv_igemm<1>, smem);
    k_conv_igemm<1><<<grid, thr, smem, st>>>(M, in, ld_in, out, ld_out, L, e, g);
  }
  return grid.x;
}

// Tensor-core path: always when forced, and automatically when the problem
// fills at least two waves of 128 x BN tiles on the 152 SMs.
static bool use_tc(const Epi& e, int M, int N) {
  if (e.gemm_path == 2) return true;
  if (e.gemm_path != 0 || !e.err) return false;
  const int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  return (long)((M + 127) / 128) * ((N + bn - 1) / bn) >= 2 * 152;
}

// Whether the row-resident conv kernels can stage this layer (input row plus the
// narrowest weight slice within 40 K floats = 160 KB of shared memory).
bool conv_supported(const LayerDev& L) {
  const int cbT = L.ci <= 1 ? 1 : (L.ci <= 4 ? 4 : 8);
  return convT_row_smem(L, cbT) <= 40 * 1024 && conv_fwd_row_smem(L, 4) <= 40 * 1024;
}

// Tensor-core convolutions: always with gemm_path 2, never with 1, and with 0
// where the SIMT kernels would take the implicit GEMM (large per-row work);
// dense rows only (rows started at one neuron skip their zero region in the
// row-resident kernels)
static bool use_tc_conv(const LayerDev& L, int dir, const Epi& e) {
  if (e.gemm_path == 1 || !tc_conv_usable(L, dir)) return false;
  if (dir == 1 && e.sparse_rows) return false;
  return e.gemm_path == 2 || (double)L.co * L.ho * L.wo * L.ci * L.k * L.k >= 512.0 * 1024.0;
}

static int tuned_variant(const LayerDev& L, int dir, int M, const Epi& e);

bool conv_tc_chosen(const LayerDev& L, int dir, const Epi& e, int M) {
  if (L.kind != MNBAB_CONV2D) return false;
  const int tv = tuned_variant(L, dir, M, e);
  if (tv > 0) return tv == V_TC && tc_conv_usable(L, dir);
  return use_tc_conv(L, dir, e);
}

int backsub_slots(const LayerDev& L) {
  if (L.kind == 1) return (L.d_in + 31) / 32;  // upper bound over the tile shapes
  // upper bound over the implicit-GEMM blocks, the row-resident splits (<= 32
  // CTAs per row, more for large planes) and the fallback tiling (128 positions
  // per CTA)
  const int P = L.hi * L.wi;
  return std::max(std::max(std::max(32 * ((P + 1023) / 1024), (P + 127) / 128), ig_slots(L)),
                  tc_conv_slots(L));
}

// One variant of the transposed convolution (back-substitution, dir 1) or the
// convolution (forward, dir 0); -1 when it does not take this layer.
static int conv_variant(int v, int dir, const LayerDev& L, int M, const float* in, int ld_in,
                        float* out, int ld_out, const Epi& e, cudaStream_t st) {
  if (v == V_TC) {
    if (!tc_conv_usable(L, dir) || (dir == 1 && e.sparse_rows)) return -1;
    const int slots = launch_tc_conv(L, dir, M, in, ld_in, out, ld_out, e, st);
    return dir == 1 ? slots : 0;
  }
  if (v == V_IG) {
    if (!ig_supported(L, dir) || (dir == 1 && e.sparse_rows)) return -1;
    const int slots = launch_ig(L, dir, M, in, ld_in, out, ld_out, e, st);
    return dir == 1 ? slots : 0;
  }
  if (v == V_ROW && dir == 1) {
    const int CBv = L.ci <= 1 ? 1 : (L.ci <= 4 ? 4 : 8);
    const ConvSplit cs = conv_split(M, L.hi * L.wi, (L.ci + CBv - 1) / CBv, CBv,
                                    [&](int cw) { return convT_row_smem(L, cw); }, 40 * 1024);
    const int rsm = convT_row_smem(L, cs.bpg * CBv) * 4;
    if (rsm > 160 * 1024 || !L.Wb || cs.npc * cs.ngrp > backsub_slots(L)) return -1;
    dim3 grid(cs.npc * cs.ngrp, M);
    if (CBv == 1) {
      set_smem(k_convT_row<1>, rsm);
      k_convT_row<1><<<grid, 128, rsm, st>>>(M, in, ld_in, out, ld_out, L, e, cs);
    } else if (CBv == 4) {
      set_smem(k_convT_row<4>, rsm);
      k_convT_row<4><<<grid, 128, rsm, st>>>(M, in, ld_in, out, ld_out, L, e, cs);
    } else {
      set_smem(k_convT_row<8>, rsm);
      k_convT_row<8><<<grid, 128, rsm, st>>>(M, in, ld_in, out, ld_out, L, e, cs);
    }
    return grid.x;
  }
  if (v == V_ROW && dir == 0) {
    const int CBv = (L.co % 8 == 0 && L.ho * L.wo >= 64) ? 8 : 4;
    const ConvSplit cs = conv_split(M, L.ho * L.wo, (L.co + CBv - 1) / CBv, CBv,
                                    [&](int cw) { return conv_fwd_row_smem(L, cw); }, 40 * 1024);
    const int rsm = conv_fwd_row_smem(L, cs.bpg * CBv) * 4;
    if (rsm > 160 * 1024 || !L.Wf) return -1;
    dim3 grid(cs.npc * cs.ngrp, M);
    if (CBv == 8) {
      set_smem(k_conv_fwd_row<8>, rsm);
      k_conv_fwd_row<8><<<grid, 128, rsm, st>>>(M, in, ld_in, out, ld_out, L, e, cs);
    } else {
      set_smem(k_conv_fwd_row<4>, rsm);
      k_conv_fwd_row<4><<<grid, 128, rsm, st>>>(M, in, ld_in, out, ld_out, L, e, cs);
    }
    return 0;
  }
  if (v == V_PLAIN) {
    const int smem = L.co * L.ci * L.k * L.k * 4;
    if (smem > 200 * 1024) return -1;
    if (dir == 1) {
      dim3 grid((L.hi * L.wi + 127) / 128, M);
      if (L.ci <= 1) {
        set_smem(k_convT<1>, smem);
        k_convT<1><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
      } else if (L.ci <= 4) {
        set_smem(k_convT<4>, smem);
        k_convT<4><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
      } else if (L.ci <= 16) {
        set_smem(k_convT<16>, smem);
        k_convT<16><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
      } else {
        set_smem(k_convT<32>, smem);
        k_convT<32><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
      }
      return grid.x;
    }
    const int Pout = L.ho * L.wo;
    const int rows_per = Pout >= 128 ? 1 : 128 / Pout;
    dim3 grid(rows_per == 1 ? (Pout + 127) / 128 : 1, (M + rows_per - 1) / rows_per);
    if (L.co <= 16) {
      set_smem(k_conv_fwd<16>, smem);
      k_conv_fwd<16><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
    } else {
      set_smem(k_conv_fwd<32>, smem);
      k_conv_fwd<32><<<grid, 128, smem, st>>>(M, in, ld_in, out, ld_out, L, e);
    }
    return 0;
  }
  return -1;
}

int launch_affine_variant(int v, int dir, const LayerDev& L, int M, const float* in, int ld_in,
                          float* out, int ld_out, const Epi& e, cudaStream_t st) {
  if (M <= 0) return -1;
  if (L.kind == 1) {
    if (v == V_TC) {
      const int slots =
          dir == 1 ? launch_gemm_tc(M, L.d_in, L.d_out, in, ld_in, nullptr, 1, out, ld_out, e,
                                    e.err, st, L.tc, 1)
                   : launch_gemm_tc(M, L.d_out, L.d_in, in, ld_in, L.b, 1, out, ld_out, e, e.err,
                                    st, L.tc, 0);
      return slots < 0 ? -1 : (dir == 1 ? slots : 0);
    }
    // back-substitution Lambda [M][d_out] x W [d_out][d_in]; forward G [M][d_in] x W^T + b
    const int slots =
        dir == 1 ? gemm_variant(v, M, L.d_in, L.d_out, in, ld_in, L.W, L.d_in, nullptr, 1, out,
                                ld_out, e, st)
                 : gemm_variant(v, M, L.d_out, L.d_in, in, ld_in, L.Wt, L.d_out, L.b, 1, out,
                                ld_out, e, st);
    return slots < 0 ? -1 : (dir == 1 ? slots : 0);
  }
  return conv_variant(v, dir, L, M, in, ld_in, out, ld_out, e, st);
}

// the autotuner's variant for this launch, if it applies: not under a forced
// GEMM path, and not for rows that the built-in choice serves with the
// sparse-row kernels
static int tuned_variant(const LayerDev& L, int dir, int M, const Epi& e) {
  if (e.gemm_path != 0 || (dir == 1 && e.sparse_rows && L.kind != 1)) return 0;
  return L.tune[dir][tune_bucket(M)];
}

int launch_backsub(const LayerDev& L, int M, const float* in, int ld_in, float* out, int ld_out,
                   const Epi& e, cudaStream_t st) {
  if (M <= 0) return backsub_slots(L);
  const int tv = tuned_variant(L, 1, M, e);
  if (tv > 0) {
    const int slots = launch_affine_variant(tv, 1, L, M, in, ld_in, out, ld_out, e, st);
    if (slots >= 0) return slots;
  }
  if (L.kind == 1) {
    // Lambda [M][d_out] x W [d_out][d_in]; the tensor-core kernel takes W as [d_in][d_out] = W^T
    if (use_tc(e, M, L.d_in)) {
      const int slots = launch_affine_variant(V_TC, 1, L, M, in, ld_in, out, ld_out, e, st);
      if (slots >= 0) return slots;
    }
    return gemm_launch(M, L.d_in, L.d_out, in, ld_in, L.W, L.d_in, nullptr, 1, out, ld_out, e, st);
  }
  if (use_tc_conv(L, 1, e)) return launch_tc_conv(L, 1, M, in, ld_in, out, ld_out, e, st);
  // dense rows: implicit GEMM per parity class; rows that start at a neuron
  // (nonzero only near it) skip the zero region in the row-resident kernel
  if (!e.sparse_rows && ig_supported(L, 1) && (ig_preferred(L) || !conv_supported(L)))
    return launch_ig(L, 1, M, in, ld_in, out, ld_out, e, st);
  const int slots = conv_variant(V_ROW, 1, L, M, in, ld_in, out, ld_out, e, st);
  if (slots >= 0) return slots;
  return conv_variant(V_PLAIN, 1, L, M, in, ld_in, out, ld_out, e, st);
}

void launch_forward(const LayerDev& L, int M, const float* in, int ld_in, float* out, int ld_out,
                    const Epi& e, cudaStream_t st) {
  if (M <= 0) return;
  const int tv = tuned_variant(L, 0, M, e);
  if (tv > 0 && launch_affine_variant(tv, 0, L, M, in, ld_in, out, ld_out, e, st) >= 0) return;
  if (L.kind == 1) {
    // G [M][d_in] x W^T + b; the tensor-core kernel takes W [d_out][d_in] as is
    if (use_tc(e, M, L.d_out) &&
        launch_affine_variant(V_TC, 0, L, M, in, ld_in, out, ld_out, e, st) >= 0)
      return;
    gemm_launch(M, L.d_out, L.d_in, in, ld_in, L.Wt, L.d_out, L.b, 1, out, ld_out, e, st);
    return;
  }
  if (use_tc_conv(L, 0, e)) {
    launch_tc_conv(L, 0, M, in, ld_in, out, ld_out, e, st);
    return;
  }
  if (ig_supported(L, 0) && (ig_preferred(L) || !conv_supported(L))) {
    launch_ig(L, 0, M, in, ld_in, out, ld_out, e, st);
    return;
  }
  if (conv_variant(V_ROW, 0, L, M, in, ld_in, out, ld_out, e, st) >= 0) return;
  conv_variant(V_PLAIN, 0, L, M, in, ld_in, out, ld_out, e, st);
}

// ---------------------------------------------------------------------------
// reductions and bookkeeping
// ---------------------------------------------------------------------------
__global__ void k_reduce_lb(int M, const float* part, int nslot, int used, const float* gp0,
                            float* lb, int track, const int* row_node, PoolDev pool,
                            const float* X, int d0) {
  const int m = blockIdx.x;
  __shared__ int imp;
  __shared__ int node;
  if (threadIdx.x == 0) {
    float acc = 0.f;
    const float* p = part + (size_t)m * nslot;
    for (int i = 0; i < used; ++i) acc += p[i];
    if (gp0) acc -= gp0[m];
    lb[m] = acc;
    imp = 0;
    node = row_node ? row_node[m] : 0;
    if (track && acc > pool.BEST[node]) {
      pool.BEST[node] = acc;
      imp = 1;
    }
  }
  __syncthreads();
  if (imp)
    for (int k = threadIdx.x; k < d0; k += blockDim.x)
      pool.BESTX[(size_t)node * d0 + k] = X[(size_t)m * d0 + k];
}

void launch_reduce_lb(int M, const float* part, int nslot, int used, const float* gp0, float* lb,
                      bool track, const int* row_node, PoolDev pool, const float* X, int d0,
                      cudaStream_t st) {
  if (M <= 0) return;
  k_reduce_lb<<<M, 128, 0, st>>>(M, part, nslot, used, gp0, lb, track ? 1 : 0, row_node, pool,
                                  X, d0);
}

// Rows (+e_j, -e_j) for every unstable (l < 0 < u) unsplit neuron of a layer,
// ascending j within a node.
__global__ void k_collect_rows(const int* nodes, PoolDev pool, int off, int d, int* counter,
                               int* row_node, int* row_j, float* row_sign) {
  const int n = nodes[blockIdx.x];
  const size_t base = (size_t)n * pool.SD + off;
  int cnt = 0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const float l = pool.L[base + j], u = pool.U[base + j];
    cnt += (l < 0.f && u > 0.f && pool.S[base + j] == 0) ? 1 : 0;
  }
  const int tot = (int)block_sum((float)cnt);
  __shared__ int start;
  if (threadIdx.x == 0) start = atomicAdd(counter, 2 * tot);
  __syncthreads();
  __shared__ int wsum[32];
  int run = 0;  // rows emitted before this chunk
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j0 = 0; j0 < d; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool f = false;
    if (j < d) {
      const float l = pool.L[base + j], u = pool.U[base + j];
      f = l < 0.f && u > 0.f && pool.S[base + j] == 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int before_lane = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int before_warp = 0, chunk = 0;
    for (int i = 0; i < nw; ++i) {
      if (i < w) before_warp += wsum[i];
      chunk += wsum[i];
    }
    if (f) {
      const int r = start + 2 * (run + before_warp + before_lane);
      row_node[r] = n; row_j[r] = j; row_sign[r] = 1.f;
      row_node[r + 1] = n; row_j[r + 1] = j; row_sign[r + 1] = -1.f;
    }
    run += chunk;
    __syncthreads();
  }
}

void launch_collect_rows(int nb, const int* nodes, PoolDev pool, int off, int d, int* counter,
                         int* row_node, int* row_j, float* row_sign, cudaStream_t st) {
  if (nb <= 0) return;
  k_collect_rows<<<nb, 256, 0, st>>>(nodes, pool, off, d, counter, row_node, row_j, row_sign);
}

__global__ void k_update_bounds(int npairs, const int* row_node, const int* row_j,
                                const float* lb, PoolDev pool, int off) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npairs) return;
  const int n = row_node[2 * q], j = row_j[2 * q];
  const size_t i = (size_t)n * pool.SD + off + j;
  pool.L[i] = fmaxf(pool.L[i], lb[2 * q]);
  pool.U[i] = fminf(pool.U[i], -lb[2 * q + 1]);
}

void launch_update_bounds(int npairs, const int* row_node, const int* row_j, const float* lb,
                          PoolDev pool, int off, cudaStream_t st) {
  if (npairs <= 0) return;
  k_update_bounds<<<(npairs + 255) / 256, 256, 0, st>>>(npairs, row_node, row_j, lb, pool, off);
}

__device__ __forceinline__ int layer_of(const NetDev& net, int f) {
  int i = 1;
  while (i < net.R && f >= net.off[i + 1]) ++i;
  return i;
}

// gamma^T P and gamma^T Phat per neuron (CSR by neuron), gamma^T p per row.
// A CTA serves one row: its node and its property's per-layer CSR pointers are
// looked up once into shared memory; a thread takes one neuron and keeps eight
// of its entries' loads in flight at a time (the sums keep entry order).
struct MncCsr {
  const int* cptr;
  const int* ce;
  const float* cP;
  const float* cPh;
  int goff, e;
};

__global__ void k_gamma_proj(int M, const int* __restrict__ row_node, PoolDev pool,
                             const PropDev* __restrict__ props, NetDev net, float* __restrict__ GP,
                             float* __restrict__ GPh) {
  const int m = blockIdx.y;
  __shared__ int s_n;
  __shared__ MncCsr s_mc[MNBAB_MAXR + 1];
  if (threadIdx.x == 0) s_n = row_node[m];
  __syncthreads();
  const int n = s_n;
  if (threadIdx.x >= 1 && threadIdx.x <= net.R) {
    const MncDev& mc = props[pool.prop[n]].mnc[threadIdx.x];
    s_mc[threadIdx.x] = MncCsr{mc.cptr, mc.ce, mc.cP, mc.cPh, mc.goff, mc.e};
  }
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= net.SD) return;
  const int i = layer_of(net, f);
  const MncCsr& mc = s_mc[i];
  float gp = 0.f, gph = 0.f;
  if (mc.e > 0) {
    const int j = f - net.off[i];
    const float* gam = pool.GAM + (size_t)n * pool.EC + mc.goff;
    const int q1 = mc.cptr[j + 1];
    int q = mc.cptr[j];
    for (; q + 8 <= q1; q += 8) {
      int ce[8];
      float g[8], cp[8], cph[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ce[k] = mc.ce[q + k];
        cp[k] = mc.cP[q + k];
        cph[k] = mc.cPh[q + k];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) g[k] = gam[ce[k]];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gp = fmaf(g[k], cp[k], gp);
        gph = fmaf(g[k], cph[k], gph);
      }
    }
    for (; q < q1; ++q) {
      const float g = gam[mc.ce[q]];
      gp = fmaf(g, mc.cP[q], gp);
      gph = fmaf(g, mc.cPh[q], gph);
    }
  }
  GP[(size_t)m * net.SD + f] = gp;
  GPh[(size_t)m * net.SD + f] = gph;
}

// gamma^T p of one row: GP_THREADS threads, four independent partial sums a
// thread (fixed order, so the value does not depend on the launch)
constexpr int GP_THREADS = 512;

__global__ void __launch_bounds__(GP_THREADS) k_gamma_p(int M, const int* row_node, PoolDev pool,
                                                        const PropDev* props, NetDev net,
                                                        float* gp0) {
  const int m = blockIdx.x;
  const int n = row_node[m];
  const PropDev& P = props[pool.prop[n]];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = 1; i <= net.R; ++i) {
    const MncDev& mc = P.mnc[i];
    const float* gam = pool.GAM + (size_t)n * pool.EC + mc.goff;
    const int e1 = mc.e;
    int e = threadIdx.x;
    for (; e + 3 * GP_THREADS < e1; e += 4 * GP_THREADS) {
      float g[4], p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        g[u] = gam[e + u * GP_THREADS];
        p[u] = mc.p[e + u * GP_THREADS];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(g[u], p[u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < 3; ++u, e += GP_THREADS)
      if (e < e1) acc[u] = fmaf(gam[e], mc.p[e], acc[u]);
  }
  const float tot = block_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
  if (threadIdx.x == 0) gp0[m] = tot;
}

void launch_gamma_proj(int M, const int* row_node, PoolDev pool, const PropDev* props,
                       const NetDev& net, float* GP, float* GPh, float* gp0, cudaStream_t st) {
  if (M <= 0) return;
  dim3 grid((net.SD + 255) / 256, M);
  k_gamma_proj<<<grid, 256, 0, st>>>(M, row_node, pool, props, net, GP, GPh);
  k_gamma_p<<<M, GP_THREADS, 0, st>>>(M, row_node, pool, props, net, gp0);
}

// d lb / d gamma_e = sum_k P_ek (d lb / d a')_idx + Phat_ek (d lb / d ahat)_idx - p_e.
constexpr int GAMMA_NPT = 4;
// A CTA serves one row (node and property looked up once); each thread takes
// GAMMA_NPT constraint rows, loading every row's entries before the gathers.
__global__ void k_gamma_grad(int M, const int* __restrict__ row_node, PoolDev pool,
                             const PropDev* __restrict__ props, NetDev net,
                             const float* __restrict__ Gz, const float* __restrict__ Hz,
                             float* __restrict__ GG) {
  const int m = blockIdx.y;
  __shared__ const PropDev* s_P;
  __shared__ int s_goff[MNBAB_MAXR + 1], s_e[MNBAB_MAXR + 1];
  if (threadIdx.x == 0) s_P = props + pool.prop[row_node[m]];
  __syncthreads();
  const PropDev& P = *s_P;
  if (threadIdx.x <= net.R) {
    s_goff[threadIdx.x] = threadIdx.x >= 1 ? P.mnc[threadIdx.x].goff : 0;
    s_e[threadIdx.x] = threadIdx.x >= 1 ? P.mnc[threadIdx.x].e : 0;
  }
  __syncthreads();
  const int E = P.E;
  const int e0 = blockIdx.x * (blockDim.x * GAMMA_NPT) + threadIdx.x;
#pragma unroll
  for (int u = 0; u < GAMMA_NPT; ++u) {
    const int ef = e0 + u * blockDim.x;
    if (ef >= E) break;
    int i = 0;
    for (int t = 1; t <= net.R; ++t)
      if (s_e[t] > 0 && ef >= s_goff[t] && ef < s_goff[t] + s_e[t]) i = t;
    if (i == 0) continue;
    const MncDev& mc = P.mnc[i];
    const int e = ef - s_goff[i];
    const float* gz = Gz + (size_t)m * net.SD + net.off[i];
    const float* hz = Hz + (size_t)m * net.SD + net.off[i];
    const int k = mc.k;
    float g = -mc.p[e];
    if (k == 3) {
      const int j0 = mc.idx[(size_t)e * 3], j1 = mc.idx[(size_t)e * 3 + 1],
                j2 = mc.idx[(size_t)e * 3 + 2];
      const float p0 = mc.P[(size_t)e * 3], p1 = mc.P[(size_t)e * 3 + 1],
                  p2 = mc.P[(size_t)e * 3 + 2];
      const float h0 = mc.Ph[(size_t)e * 3], h1 = mc.Ph[(size_t)e * 3 + 1],
                  h2 = mc.Ph[(size_t)e * 3 + 2];
      const float z0 = gz[j0], z1 = gz[j1], z2 = gz[j2];
      const float y0 = hz[j0], y1 = hz[j1], y2 = hz[j2];
      g = fmaf(p0, z0, g);
      g = fmaf(h0, y0, g);
      g = fmaf(p1, z1, g);
      g = fmaf(h1, y1, g);
      g = fmaf(p2, z2, g);
      g = fmaf(h2, y2, g);
    } else {
      for (int kk = 0; kk < k; ++kk) {
        const int j = mc.idx[(size_t)e * k + kk];
        g = fmaf(mc.P[(size_t)e * k + kk], gz[j], g);
        g = fmaf(mc.Ph[(size_t)e * k + kk], hz[j], g);
      }
    }
    GG[(size_t)m * pool.EC + ef] = g;
  }
}

void launch_gamma_grad(int M, const int* row_node, PoolDev pool, const PropDev* props,
                       const NetDev& net, const float* Gz, const float* Hz, float* GG,
                       cudaStream_t st) {
  if (M <= 0 || pool.EC <= 0) return;
  dim3 grid((pool.EC + 256 * GAMMA_NPT - 1) / (256 * GAMMA_NPT), M);
  k_gamma_grad<<<grid, 256, 0, st>>>(M, row_node, pool, props, net, Gz, Hz, GG);
}

// Projected Adam ascent step (Sec. 3.1): alpha in [0, 1], beta, gamma >= 0.
__device__ __forceinline__ void adam1(float& th, float& mo, float& ve, float g, float lr, float b1,
                                      float b2, float eps, float bc1, float bc2) {
  mo = b1 * mo + (1.f - b1) * g;
  ve = b2 * ve + (1.f - b2) * g * g;
  const float mh = mo / bc1;
  const float vh = ve / bc2;
  th = th + lr * mh / (sqrtf(vh) + eps);
}

// largest |gradient component| of each row over alpha, beta and gamma
__global__ void k_grad_max(int SD, int EC, const int* row_node, const PoolDev pool,
                           const PropDev* props, const float* GA, const float* GB,
                           const float* GG, float* gmax) {
  const int m = blockIdx.x;
  const int E = props[pool.prop[row_node[m]]].E;
  float mx = 0.f;
  for (int i = threadIdx.x; i < SD; i += blockDim.x)
    mx = fmaxf(mx, fmaxf(fabsf(GA[(size_t)m * SD + i]), fabsf(GB[(size_t)m * SD + i])));
  for (int e = threadIdx.x; e < E; e += blockDim.x) mx = fmaxf(mx, fabsf(GG[(size_t)m * EC + e]));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, sh[i]);
    gmax[m] = r;
  }
}

// The alpha of a neuron that is not unstable and unsplit, and the beta of an
// unsplit one, have a zero gradient at every step of an optimisation (its
// bounds and splits are fixed), and their moments start at zero: their
// updates are identities and are skipped.  gmax is read only when the
// dead-zone or the gradient-scaled eps is on (use_gmax).
__global__ void k_adam(int M, const int* __restrict__ row_node, PoolDev pool,
                       const PropDev* __restrict__ props, int SD, const float* __restrict__ GA,
                       const float* __restrict__ GB, const float* __restrict__ GG,
                       const float* __restrict__ gmax, int use_gmax, float floor, float lr_a,
                       float lr_b, float lr_g, float b1, float b2, float eps_abs, float eps_rel,
                       float bc1, float bc2) {
  const int m = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = row_node[m];
  const float gm = use_gmax ? gmax[m] : 0.f;
  const float thr = floor * gm;
  const float eps = fmaxf(eps_abs, eps_rel * gm);
  auto dz = [thr](float g) { return fabsf(g) <= thr ? 0.f : g; };
  if (idx < SD) {
    const size_t q = (size_t)n * SD + idx;
    if (pool.S[q] != 0 || !(pool.L[q] < 0.f) || !(pool.U[q] > 0.f)) return;
    float th = pool.ALPHA[q], mo = pool.MA[q], ve = pool.VA[q];
    adam1(th, mo, ve, dz(GA[(size_t)m * SD + idx]), lr_a, b1, b2, eps, bc1, bc2);
    pool.ALPHA[q] = fminf(fmaxf(th, 0.f), 1.f);
    pool.MA[q] = mo; pool.VA[q] = ve;
  } else if (idx < 2 * SD) {
    const int f = idx - SD;
    const size_t q = (size_t)n * SD + f;
    if (pool.S[q] == 0) return;
    float th = pool.BETA[q], mo = pool.MB[q], ve = pool.VB[q];
    adam1(th, mo, ve, dz(GB[(size_t)m * SD + f]), lr_b, b1, b2, eps, bc1, bc2);
    pool.BETA[q] = fmaxf(th, 0.f);
    pool.MB[q] = mo; pool.VB[q] = ve;
  } else {
    const int e = idx - 2 * SD;
    if (e >= props[pool.prop[n]].E) return;
    const size_t q = (size_t)n * pool.EC + e;
    float th = pool.GAM[q], mo = pool.MG[q], ve = pool.VG[q];
    adam1(th, mo, ve, dz(GG[(size_t)m * pool.EC + e]), lr_g, b1, b2, eps, bc1, bc2);
    pool.GAM[q] = fmaxf(th, 0.f);
    pool.MG[q] = mo; pool.VG[q] = ve;
  }
}

void launch_adam(int M, const int* row_node, PoolDev pool, const PropDev* props, int SD,
                 const float* GA, const float* GB, const float* GG, float* gmax, float floor,
                 float lr_a, float lr_b, float lr_g, float b1, float b2, float eps, float eps_rel,
                 float bc1, float bc2, cudaStream_t st) {
  if (M <= 0) return;
  const int use_gmax = (floor != 0.f || eps_rel != 0.f) ? 1 : 0;
  if (use_gmax)
    k_grad_max<<<M, 256, 0, st>>>(SD, pool.EC, row_node, pool, props, GA, GB, GG, gmax);
  const int tot = 2 * SD + pool.EC;
  dim3 grid((tot + 255) / 256, M);
  k_adam<<<grid, 256, 0, st>>>(M, row_node, pool, props, SD, GA, GB, GG, gmax, use_gmax, floor,
                               lr_a, lr_b, lr_g, b1, b2, eps, eps_rel, bc1, bc2);
}

__global__ void k_zero_adam(const int* row_node, PoolDev pool) {
  const int n = row_node[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < pool.SD) {
    const size_t q = (size_t)n * pool.SD + idx;
    pool.MA[q] = 0.f; pool.VA[q] = 0.f; pool.MB[q] = 0.f; pool.VB[q] = 0.f;
  } else if (idx < pool.SD + pool.EC) {
    const size_t q = (size_t)n * pool.EC + idx - pool.SD;
    pool.MG[q] = 0.f; pool.VG[q] = 0.f;
  }
}

void launch_zero_adam(int M, const int* row_node, PoolDev pool, cudaStream_t st) {
  if (M <= 0) return;
  dim3 grid((pool.SD + pool.EC + 255) / 256, M);
  k_zero_adam<<<grid, 256, 0, st>>>(row_node, pool);
}

__global__ void k_set_best(int M, const int* row_node, PoolDev pool, float v) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) pool.BEST[row_node[m]] = v;
}

void launch_set_best(int M, const int* row_node, PoolDev pool, float v, cudaStream_t st) {
  if (M <= 0) return;
  k_set_best<<<(M + 255) / 256, 256, 0, st>>>(M, row_node, pool, v);
}

// ACS (Sec. 3.2) with the intercept fallback; with CAB the score is divided by
// the cost of a split in the neuron's layer (the fallback decision is taken on
// the raw scores).  Ties within 1e-5 of the maximum go to the lowest
// (layer, neuron).
__global__ void k_acs(int M, const int* row_node, PoolDev pool, const PropDev* props, NetDev net,
                      const float* GP, const float* GPh, const float* AP, int has_gamma,
                      int* out_layer, int* out_neuron, float* out_score, int* out_fallback) {
  const int m = blockIdx.x;
  const int n = row_node[m];
  const PropDev& P = props[pool.prop[n]];
  const size_t nb = (size_t)n * pool.SD, mb = (size_t)m * net.SD;
  __shared__ float smax[32];
  __shared__ int sany[32];
  __shared__ int smin[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto bmax = [&](float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) smax[w] = v;
    __syncthreads();
    float r = -INFINITY;
    for (int i = 0; i < nw; ++i) r = fmaxf(r, smax[i]);
    return r;
  };
  // candidates and whether any active-constraint score is positive
  float raw = -INFINITY;
  int any = 0;
  for (int f = threadIdx.x; f < net.SD; f += blockDim.x) {
    const float l = pool.L[nb + f], u = pool.U[nb + f];
    if (l < 0.f && u > 0.f && pool.S[nb + f] == 0) {
      any = 1;
      const float sc = has_gamma ? fabsf(GP[mb + f]) + fabsf(GPh[mb + f]) : 0.f;
      raw = fmaxf(raw, sc);
    }
  }
  raw = bmax(raw);
  for (int o = 16; o; o >>= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
  if (lane == 0) sany[w] = any;
  __syncthreads();
  any = 0;
  for (int i = 0; i < nw; ++i) any |= sany[i];
  if (!any) {
    if (threadIdx.x == 0) {
      out_layer[m] = 0; out_neuron[m] = -1; out_score[m] = 0.f; out_fallback[m] = 0;
    }
    return;
  }
  const int fallback = !(raw > 0.f);
  auto score = [&](int f, float l, float u) {
    float sc = fallback ? fabsf(AP[mb + f]) * ((-l * u) / (u - l))
                        : fabsf(GP[mb + f]) + fabsf(GPh[mb + f]);
    if (P.cab) sc *= P.cab_inv[layer_of(net, f)];
    return sc;
  };
  float mx = -INFINITY;
  for (int f = threadIdx.x; f < net.SD; f += blockDim.x) {
    const float l = pool.L[nb + f], u = pool.U[nb + f];
    if (l < 0.f && u > 0.f && pool.S[nb + f] == 0) mx = fmaxf(mx, score(f, l, u));
  }
  mx = bmax(mx);
  const float thr = mx - 1e-5f * fabsf(mx);
  int best = 0x7fffffff;
  for (int f = threadIdx.x; f < net.SD; f += blockDim.x) {
    const float l = pool.L[nb + f], u = pool.U[nb + f];
    if (l < 0.f && u > 0.f && pool.S[nb + f] == 0 && score(f, l, u) >= thr && f < best) best = f;
  }
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  __syncthreads();
  if (lane == 0) smin[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int b = 0x7fffffff;
    for (int i = 0; i < nw; ++i) b = min(b, smin[i]);
    const int i = layer_of(net, b);
    out_layer[m] = i;
    out_neuron[m] = b - net.off[i];
    out_score[m] = mx;
    out_fallback[m] = fallback;
  }
}

void launch_acs(int M, const int* row_node, PoolDev pool, const PropDev* props, const NetDev& net,
                const float* GP, const float* GPh, const float* AP, int has_gamma, int* out_layer,
                int* out_neuron, float* out_score, int* out_fallback, cudaStream_t st) {
  if (M <= 0) return;
  k_acs<<<M, 256, 0, st>>>(M, row_node, pool, props, net, GP, GPh, AP, has_gamma, out_layer,
                            out_neuron, out_score, out_fallback);
}

// Children of a split (Sec. 3.2, enforcing splits): copies of the parent with
// S = +1 (zhat <= 0, u <- min(u, 0)) for the first child and S = -1 (zhat >= 0,
// l <- max(l, 0)) for the second; the split neuron's beta starts at 0.
__global__ void k_children(const int* parents, const int* kids, const int* layer,
                           const int* neuron, PoolDev pool, NetDev net) {
  const int b = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int par = parents[b];
  const int f_split = net.off[layer[b]] + neuron[b];
  for (int c = 0; c < 2; ++c) {
    const int kid = kids[2 * b + c];
    if (idx < pool.SD) {
      const size_t qs = (size_t)par * pool.SD + idx, qd = (size_t)kid * pool.SD + idx;
      float l = pool.L[qs], u = pool.U[qs];
      int8_t s = pool.S[qs];
      float be = pool.BETA[qs];
      if (idx == f_split) {
        be = 0.f;
        if (c == 0) { s = 1; u = fminf(u, 0.f); }
        else { s = -1; l = fmaxf(l, 0.f); }
      }
      pool.L[qd] = l; pool.U[qd] = u; pool.S[qd] = s;
      pool.ALPHA[qd] = pool.ALPHA[qs];
      pool.BETA[qd] = be;
    } else if (idx < pool.SD + pool.EC) {
      const int e = idx - pool.SD;
      pool.GAM[(size_t)kid * pool.EC + e] = pool.GAM[(size_t)par * pool.EC + e];
    }
    if (idx == 0) {
      pool.prop[kid] = pool.prop[par];
      pool.row[kid] = pool.row[par];
    }
  }
}

void launch_children(int nb, const int* parents, const int* kids, const int* layer,
                     const int* neuron, PoolDev pool, const NetDev& net, cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid((pool.SD + pool.EC + 255) / 256, nb);
  k_children<<<grid, 256, 0, st>>>(parents, kids, layer, neuron, pool, net);
}

// ---------------------------------------------------------------------------
// Optimised intermediate bounds (Sec. 3.1, parameter sharing): the parameter
// set of one (node, target layer, side) lives in a scratch pool slot.
// ---------------------------------------------------------------------------
// Set slot dst[b] from node src[b]: bounds and splits, DeepPoly slopes
// (alpha = 1 if u >= -l else 0), beta = 0, gamma = 0, zero Adam moments.
__global__ void k_set_init(const int* src, const int* dst, PoolDev pool) {
  const int b = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = src[b], d = dst[b];
  if (i < pool.SD) {
    const size_t qs = (size_t)s * pool.SD + i, qd = (size_t)d * pool.SD + i;
    const float l = pool.L[qs], u = pool.U[qs];
    pool.L[qd] = l;
    pool.U[qd] = u;
    pool.S[qd] = pool.S[qs];
    pool.ALPHA[qd] = u >= -l ? 1.f : 0.f;
    pool.BETA[qd] = 0.f;
    pool.MA[qd] = 0.f;
    pool.VA[qd] = 0.f;
    pool.MB[qd] = 0.f;
    pool.VB[qd] = 0.f;
  }
  if (i < pool.EC) {
    // multi-neuron multipliers start at 0 with zero moments
    const size_t qd = (size_t)d * pool.EC + i;
    pool.GAM[qd] = 0.f;
    pool.MG[qd] = 0.f;
    pool.VG[qd] = 0.f;
  }
  if (i == 0) {
    pool.prop[d] = pool.prop[s];
    pool.row[d] = pool.row[s];
  }
}

void launch_set_init(int nsets, const int* src, const int* dst, PoolDev pool, cudaStream_t st) {
  if (nsets <= 0) return;
  dim3 grid((std::max(pool.SD, pool.EC) + 255) / 256, nsets);
  k_set_init<<<grid, 256, 0, st>>>(src, dst, pool);
}

// best[m] = lb[m] on the first iterate, max(best[m], lb[m]) after.
__global__ void k_rows_best(int M, const float* lb, float* best, int first) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) best[m] = first ? lb[m] : fmaxf(best[m], lb[m]);
}

void launch_rows_best(int M, const float* lb, float* best, int first, cudaStream_t st) {
  if (M <= 0) return;
  k_rows_best<<<(M + 255) / 256, 256, 0, st>>>(M, lb, best, first);
}

// Adds the per-row gradients GA, GB ([row][SD], rows of one chunk) of each
// set's rows to the set's gradients IGA, IGB ([set][SD]), entries k < lim.
// seg holds (set, first row, end row) per block row, rows relative to the
// chunk; the rows of a set are summed in order.
__global__ void k_set_grad(const int* seg, int SD, int lim, const float* GA, const float* GB,
                           float* IGA, float* IGB) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= lim) return;
  const int s = seg[3 * blockIdx.y], r0 = seg[3 * blockIdx.y + 1], r1 = seg[3 * blockIdx.y + 2];
  float ga = 0.f, gb = 0.f;
  for (int m = r0; m < r1; ++m) {
    ga += GA[(size_t)m * SD + k];
    gb += GB[(size_t)m * SD + k];
  }
  IGA[(size_t)s * SD + k] += ga;
  IGB[(size_t)s * SD + k] += gb;
}

void launch_set_grad(int nseg, const int* seg, int SD, int lim, const float* GA, const float* GB,
                     float* IGA, float* IGB, cudaStream_t st) {
  if (nseg <= 0 || lim <= 0) return;
  dim3 grid((lim + 255) / 256, nseg);
  k_set_grad<<<grid, 256, 0, st>>>(seg, SD, lim, GA, GB, IGA, IGB);
}

// Adds the per-row gradients GG ([row][EC]) w.r.t. the multi-neuron
// multipliers of each set's rows to the set's gradient IGG ([set][EC]), rows
// in order; only constraints of ReLU layers below t (the layers the rows pass)
// get a gradient, every other entry stays 0 (those multipliers stay 0).
__global__ void k_set_grad_gamma(const int* seg, const int* set_slot, PoolDev pool,
                                 const PropDev* props, int t, const float* GG, float* IGG) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = seg[3 * blockIdx.y], r0 = seg[3 * blockIdx.y + 1], r1 = seg[3 * blockIdx.y + 2];
  const PropDev& P = props[pool.prop[set_slot[s]]];
  if (e >= P.E) return;
  bool below = false;
  for (int i = 1; i < t && i <= MNBAB_MAXR; ++i)
    if (e >= P.mnc[i].goff && e < P.mnc[i].goff + P.mnc[i].e) below = true;
  if (!below) return;
  float g = 0.f;
  for (int m = r0; m < r1; ++m) g += GG[(size_t)m * pool.EC + e];
  IGG[(size_t)s * pool.EC + e] += g;
}

void launch_set_grad_gamma(int nseg, const int* seg, const int* set_slot, PoolDev pool,
                           const PropDev* props, int t, const float* GG, float* IGG,
                           cudaStream_t st) {
  if (nseg <= 0 || pool.EC <= 0) return;
  dim3 grid((pool.EC + 255) / 256, nseg);
  k_set_grad_gamma<<<grid, 256, 0, st>>>(seg, set_slot, pool, props, t, GG, IGG);
}

// Intersects the bounds of neuron j[m] of the layer at offset off of node
// orig[m] with row m's best bound: sign +1 bounds zhat_j from below, -1 is
// the lower bound of -zhat_j, so -best bounds it from above.
__global__ void k_set_update(int M, const int* orig, const int* j, const float* sign,
                             const float* best, PoolDev pool, int off) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const size_t q = (size_t)orig[m] * pool.SD + off + j[m];
  if (sign[m] > 0.f) pool.L[q] = fmaxf(pool.L[q], best[m]);
  else pool.U[q] = fminf(pool.U[q], -best[m]);
}

void launch_set_update(int M, const int* orig, const int* j, const float* sign, const float* best,
                       PoolDev pool, int off, cudaStream_t st) {
  if (M <= 0) return;
  k_set_update<<<(M + 255) / 256, 256, 0, st>>>(M, orig, j, sign, best, pool, off);
}

// Root nodes from their property's root-bound slot: DeepPoly slopes
// (alpha = 1 if u >= -l else 0), beta = gamma = 0, no splits.
__global__ void k_root_init(const int* slots, const int* srcs, const int* rows, PoolDev pool) {
  const int dst = slots[blockIdx.y];
  const int src = srcs[blockIdx.y];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < pool.SD) {
    const size_t qs = (size_t)src * pool.SD + idx, qd = (size_t)dst * pool.SD + idx;
    const float l = pool.L[qs], u = pool.U[qs];
    pool.L[qd] = l; pool.U[qd] = u; pool.S[qd] = 0;
    pool.ALPHA[qd] = (u >= -l) ? 1.f : 0.f;
    pool.BETA[qd] = 0.f;
  } else if (idx < pool.SD + pool.EC) {
    pool.GAM[(size_t)dst * pool.EC + idx - pool.SD] = 0.f;
  }
  if (idx == 0) {
    pool.prop[dst] = pool.prop[src];
    pool.row[dst] = rows[blockIdx.y];
  }
}

void launch_root_init(int nb, const int* slots, const int* srcs, const int* rows, PoolDev pool,
                      cudaStream_t st) {
  if (nb <= 0) return;
  dim3 grid((pool.SD + pool.EC + 255) / 256, nb);
  k_root_init<<<grid, 256, 0, st>>>(slots, srcs, rows, pool);
}

// f_r(z_R) through the property's folded last layer, one warp per row.
__global__ void k_final_dot(int M, const int* row_node, PoolDev pool, const PropDev* props,
                            const float* z, int ld, int dR, float* f) {
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= M) return;
  const int n = row_node[m];
  const PropDev& P = props[pool.prop[n]];
  const int r = pool.row[n];
  const float* w = P.Wf + (size_t)r * dR;
  const float* x = z + (size_t)m * ld;
  float acc = 0.f;
  for (int k = lane; k < dR; k += 32) acc = fmaf(w[k], x[k], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) f[m] = acc + P.bf[r];
}

void launch_final_dot(int M, const int* row_node, PoolDev pool, const PropDev* props,
                      const float* z, int ld, int dR, float* f, cudaStream_t st) {
  if (M <= 0) return;
  k_final_dot<<<(M + 7) / 8, 256, 0, st>>>(M, row_node, pool, props, z, ld, dR, f);
}

// Concrete forward pass f_r(x) in FP64 (one CTA per row), used to confirm
// counterexamples: the sign of f_r at x* decides FALSIFIED (Sec. 2.2), so it is
// evaluated in double precision from the FP32 weights.  The row buffer holds
// x and every ReLU output (layer t at offset d0 + off[t]), so residual edges
// can read any earlier layer.
__device__ double f64_edge(const LayerDev& L, const double* z, int o) {
  if (L.kind == 1) {
    double acc = (double)L.b[o];
    const float* w = L.W + (size_t)o * L.d_in;
    for (int k = 0; k < L.d_in; ++k) acc = fma((double)w[k], z[k], acc);
    return acc;
  }
  const int hw = L.ho * L.wo;
  const int co = o / hw, oh = (o % hw) / L.wo, ow = o % L.wo;
  double acc = (double)L.b[co];
  for (int ci = 0; ci < L.ci; ++ci)
    for (int kh = 0; kh < L.k; ++kh) {
      const int ih = oh * L.s - L.p + kh;
      if (ih < 0 || ih >= L.hi) continue;
      for (int kw = 0; kw < L.k; ++kw) {
        const int iw = ow * L.s - L.p + kw;
        if (iw < 0 || iw >= L.wi) continue;
        acc = fma((double)L.W[(((size_t)co * L.ci + ci) * L.k + kh) * L.k + kw],
                  z[((size_t)ci * L.hi + ih) * L.wi + iw], acc);
      }
    }
  return acc;
}

// FP64 forward pass of counterexample candidates (Sec. 3.1, upper bounding):
// one launch per layer, one thread per (candidate, neuron), then the objective
// row per candidate.
// With dcount set, only the first *dcount of the M rows are live (a count the
// device computed; the grid covers M).
__global__ void k_f64_input(int M, const int* dcount, const float* X, int ldx, double* buf, int ldb,
                            int d0) {
  const int m = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (dcount && m >= *dcount) return;
  if (m < M && k < d0) buf[(size_t)m * ldb + k] = (double)X[(size_t)m * ldx + k];
}

__global__ void k_f64_layer(int M, const int* dcount, NetDev net, int t, double* buf, int ldb) {
  const int m = blockIdx.y;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M || o >= net.d[t] || (dcount && m >= *dcount)) return;
  double* z = buf + (size_t)m * ldb;
  const int d0 = net.d[0];
  auto seg = [&](int s) { return s == 0 ? z : z + d0 + net.off[s]; };
  double v = f64_edge(net.aff[t], seg(net.src1[t]), o);
  if (net.n_edge[t] > 1) v += f64_edge(net.aff2[t], seg(net.src2[t]), o);
  seg(t)[o] = v > 0.0 ? v : 0.0;
}

__global__ void k_f64_objective(int M, const int* dcount, const int* row_node, PoolDev pool,
                                const PropDev* props, NetDev net, const double* buf, int ldb,
                                double* fout) {
  const int m = blockIdx.x;
  if (dcount && m >= *dcount) return;
  const double* z = buf + (size_t)m * ldb;
  const int n = row_node[m];
  const PropDev& P = props[pool.prop[n]];
  const int r = pool.row[n];
  const int sR = net.src1[net.R + 1];
  const int dR = net.d[sR];
  const double* h = sR == 0 ? z : z + net.d[0] + net.off[sR];
  double acc = 0.0;
  for (int k = threadIdx.x; k < dR; k += blockDim.x) acc = fma((double)P.Wf[(size_t)r * dR + k], h[k], acc);
  __shared__ double sh[32];
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tt = (double)P.bf[r];
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tt += sh[i];
    fout[m] = tt;
  }
}

void launch_forward_f64(int M, const int* row_node, PoolDev pool, const PropDev* props,
                        const NetDev& net, const float* X, int ldx, double* buf, int ldb,
                        double* fout, cudaStream_t st, const int* dcount) {
  if (M <= 0) return;
  k_f64_input<<<dim3((net.d[0] + 255) / 256, M), 256, 0, st>>>(M, dcount, X, ldx, buf, ldb,
                                                                net.d[0]);
  for (int t = 1; t <= net.R; ++t)
    k_f64_layer<<<dim3((net.d[t] + 127) / 128, M), 128, 0, st>>>(M, dcount, net, t, buf, ldb);
  k_f64_objective<<<M, 256, 0, st>>>(M, dcount, row_node, pool, props, net, buf, ldb, fout);
}

// Counterexample candidates of a batch (Sec. 3.1, upper bounding), in batch
// order: rows m < M whose FP32 objective at the node's best minimiser is
// negative and whose best bound is not positive.  One CTA of up to 1024
// threads, a thread per row and rounds of 1024 rows; writes the rows' batch
// indices and slots and their count.
__global__ void __launch_bounds__(1024) k_select_cand(int M, const float* __restrict__ fout,
                                                      const int* __restrict__ slots,
                                                      const float* __restrict__ best,
                                                      int* cand_idx, int* cand_slot, int* count) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m0 = 0; m0 < M; m0 += blockDim.x) {
    const int m = m0 + threadIdx.x;
    bool c = false;
    if (m < M) c = fout[m] < 0.f && !(best[slots[m]] > 0.f);
    const unsigned bal = __ballot_sync(0xffffffffu, c);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = base;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    before += __popc(bal & ((1u << lane) - 1u));
    if (c) {
      cand_idx[before] = m;
      cand_slot[before] = slots[m];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < nw; ++w) base += warp_tot[w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

void launch_select_cand(int M, const float* fout, const int* slots, const float* best,
                        int* cand_idx, int* cand_slot, int* count, cudaStream_t st) {
  const int thr = std::max(32, std::min(1024, (M + 31) / 32 * 32));
  k_select_cand<<<1, thr, 0, st>>>(M, fout, slots, best, cand_idx, cand_slot, count);
}

__global__ void k_fill(float* p, size_t n, float v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Root-bound slots of newly started properties: l = -inf, u = +inf, no splits,
// and the slot's property index.
__global__ void k_root_slot_init(int nb, const int* slots, const int* prop, PoolDev pool) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  const size_t o = (size_t)slots[b] * pool.SD;
  for (int j = threadIdx.x; j < pool.SD; j += blockDim.x) {
    pool.L[o + j] = -INFINITY;
    pool.U[o + j] = INFINITY;
    pool.S[o + j] = 0;
  }
  if (threadIdx.x == 0) pool.prop[slots[b]] = prop[b];
}

void launch_root_slot_init(int nb, const int* slots, const int* prop, PoolDev pool,
                           cudaStream_t st) {
  if (nb > 0) k_root_slot_init<<<nb, 256, 0, st>>>(nb, slots, prop, pool);
}

void launch_fill(float* p, size_t n, float v, cudaStream_t st) {
  if (n == 0) return;
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, v);
}

// ---------------------------------------------------------------------------
// Pre-attack in the per-layer form (Sec. 4, experimental setup): candidate m
// is a scratch node slot whose bounds hold the pre-activations at its point
// (l = u = zhat), so that a DeepPoly back-substitution of the objective row
// through it is the gradient of the margin (ReLU' = 1 where zhat >= 0).
// ---------------------------------------------------------------------------
// Slot m of the chunk: no splits, zero parameters, property `prop`, row
// (q0 + m) / n_starts; its point, start (q0 + m) mod n_starts clipped to the
// box (starts null: left as is); best margin +inf.
__global__ void k_attack_init(int M, int q0, int n_starts, const int* slots, PoolDev pool,
                              int prop, const PropDev* props, const float* starts, float* X,
                              float* best) {
  const int m = blockIdx.y;
  const int slot = slots[m];
  const int q = q0 + m;
  const PropDev& P = props[prop];
  const int lim = max(pool.SD, pool.d0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += gridDim.x * blockDim.x) {
    if (i < pool.SD) {
      const size_t o = (size_t)slot * pool.SD + i;
      pool.L[o] = 0.f;
      pool.U[o] = 0.f;
      pool.S[o] = 0;
      pool.ALPHA[o] = 0.f;
      pool.BETA[o] = 0.f;
    }
    if (starts && i < pool.d0)
      X[(size_t)m * pool.d0 + i] =
          fminf(fmaxf(starts[(size_t)(q % n_starts) * pool.d0 + i], P.lo[i]), P.hi[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pool.prop[slot] = prop;
    pool.row[slot] = q / n_starts;
    if (best) best[m] = INFINITY;
  }
}

void launch_attack_init(int M, int q0, int n_starts, const int* slots, PoolDev pool, int prop,
                        const PropDev* props, const float* starts, float* X, float* best,
                        cudaStream_t st) {
  if (M <= 0) return;
  const int lim = std::max(pool.SD, pool.d0);
  dim3 grid((unsigned)std::min(64, (lim + 255) / 256), (unsigned)M);
  k_attack_init<<<grid, 256, 0, st>>>(M, q0, n_starts, slots, pool, prop, props, starts, X, best);
}

// z [M][d] holds the pre-activations zhat of ReLU layer (offset off): they go
// to the bounds of each row's slot (l = u = zhat) and z becomes max(zhat, 0)
__global__ void k_pattern_relu(int M, const int* slots, PoolDev pool, int off, int d, float* z) {
  const size_t total = (size_t)M * d;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / d), j = (int)(i % d);
    const float v = z[i];
    const size_t q = (size_t)slots[m] * pool.SD + off + j;
    pool.L[q] = v;
    pool.U[q] = v;
    z[i] = fmaxf(v, 0.f);
  }
}

void launch_pattern_relu(int M, const int* slots, PoolDev pool, int off, int d, float* z,
                         cudaStream_t st) {
  if (M <= 0 || d <= 0) return;
  const size_t total = (size_t)M * d;
  const int blocks = (int)std::min<size_t>(152 * 8, (total + 255) / 256);
  k_pattern_relu<<<blocks, 256, 0, st>>>(M, slots, pool, off, d, z);
}

// best[m] and its point bx[m] <- f[m] and X[m] when f[m] is smaller (the
// first minimiser is kept on ties; NaN never replaces it)
__global__ void k_attack_best(const float* f, const float* X, int d0, float* best, float* bx) {
  const int m = blockIdx.x;
  const bool better = f[m] < best[m];
  if (better)
    for (int j = threadIdx.x; j < d0; j += blockDim.x) bx[(size_t)m * d0 + j] = X[(size_t)m * d0 + j];
  __syncthreads();
  if (better && threadIdx.x == 0) best[m] = f[m];
}

void launch_attack_best(int M, const float* f, const float* X, int d0, float* best, float* bx,
                        cudaStream_t st) {
  if (M <= 0) return;
  k_attack_best<<<M, 128, 0, st>>>(f, X, d0, best, bx);
}

// x <- clip(x - alpha sign(g), lo, hi), alpha_j = 2.5 (hi_j - lo_j) / (2 steps),
// sign(0) = 0, with g [M][ld] the margin's gradient
__global__ void k_attack_step(int M, const float* g, int ld, float* X, int d0,
                              const PropDev* props, int prop, int steps) {
  const PropDev& P = props[prop];
  const size_t total = (size_t)M * d0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / d0), j = (int)(i % d0);
    const float gj = g[(size_t)m * ld + j];
    const float sg = gj > 0.f ? 1.f : (gj < 0.f ? -1.f : 0.f);
    const float alpha = 2.5f * (P.hi[j] - P.lo[j]) / (2.0f * (float)steps);
    X[i] = fminf(fmaxf(X[i] - alpha * sg, P.lo[j]), P.hi[j]);
  }
}

void launch_attack_step(int M, const float* g, int ld, float* X, int d0, const PropDev* props,
                        int prop, int steps, cudaStream_t st) {
  if (M <= 0) return;
  const size_t total = (size_t)M * d0;
  const int blocks = (int)std::min<size_t>(152 * 8, (total + 255) / 256);
  k_attack_step<<<blocks, 256, 0, st>>>(M, g, ld, X, d0, props, prop, steps);
}

}  // namespace mnbab
