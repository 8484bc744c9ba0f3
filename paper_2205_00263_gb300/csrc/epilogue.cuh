// Fused back-substitution epilogues shared by the SIMT and tensor-core kernels.
#pragma once
#include <cuda_runtime.h>

#include "mnbab_internal.h"

namespace mnbab {

// ---------------------------------------------------------------------------
// epilogues
// ---------------------------------------------------------------------------
// ReLU back-substitution of one coefficient a on z_j (Sec. 3.1, combined ReLU
// step): a' = a + (gamma^T P)_j, D / blow from the single-neuron table with
// split precedence, ahat = a' D + beta S + (gamma^T Phat)_j.  The offset
// contribution a' blow + ahat b_j (bias of the consuming affine layer) goes to
// the row partial sum.
__device__ __forceinline__ float epi_relu(const Epi& e, int m, int j, float a, float& part) {
  const int n = e.row_node[m];
  const size_t q = (size_t)n * e.SD + e.off + j;
  const size_t qm = (size_t)m * e.SD + e.off + j;
  const float l = e.pool.L[q], u = e.pool.U[q];
  const int s = e.pool.S[q];
  float ap = a;
  if (e.GP) ap += e.GP[qm];
  float D, bl = 0.f;
  if (s == -1) D = 1.f;
  else if (s == 1) D = 0.f;
  else if (l >= 0.f) D = 1.f;
  else if (u <= 0.f) D = 0.f;
  else if (ap >= 0.f) D = e.final_mode ? e.pool.ALPHA[q] : (u >= -l ? 1.f : 0.f);
  else {
    const float den = u - l;
    D = u / den;
    bl = (-u * l) / den;
  }
  float ah = ap * D;
  if (e.final_mode) ah += e.pool.BETA[q] * (float)s;
  if (e.GPh) ah += e.GPh[qm];
  if (e.AP) e.AP[qm] = ap;
  part += ap * bl + ah * e.bias[j / e.bias_div];
  return ah;
}

// Concretisation of a coefficient on input x_j over [lo, hi] (Eq. minimum):
// x*_j = lo_j if a >= 0 else hi_j, contribution a x*_j.
__device__ __forceinline__ float epi_conc(const Epi& e, int m, int j, float a, float& part) {
  const int n = e.row_node[m];
  const PropDev& P = e.props[e.pool.prop[n]];
  const float x = a >= 0.f ? P.lo[j] : P.hi[j];
  part += a * x;
  if (e.X) e.X[(size_t)m * e.d0 + j] = x;
  return a;
}

// Adjoint of the ReLU step at pre-activation adjoint h = d lb / d ahat_j:
// d lb / d alpha_j = h a'_j on the alpha branch, d lb / d beta_j = h S_j,
// and d lb / d a'_j = h D_j + blow_j flows to the next layer.
__device__ __forceinline__ float epi_adj(const Epi& e, int m, int j, float h) {
  const int n = e.row_node[m];
  const size_t q = (size_t)n * e.SD + e.off + j;
  const size_t qm = (size_t)m * e.SD + e.off + j;
  const float l = e.pool.L[q], u = e.pool.U[q];
  const int s = e.pool.S[q];
  const float ap = e.AP[qm];
  float D, bl = 0.f;
  bool abr = false;
  if (s == -1) D = 1.f;
  else if (s == 1) D = 0.f;
  else if (l >= 0.f) D = 1.f;
  else if (u <= 0.f) D = 0.f;
  else if (ap >= 0.f) { D = e.pool.ALPHA[q]; abr = true; }
  else {
    const float den = u - l;
    D = u / den;
    bl = (-u * l) / den;
  }
  e.GA[qm] = abr ? h * ap : 0.f;
  e.GB[qm] = h * (float)s;
  const float g = h * D + bl;
  if (e.Hz) {
    e.Hz[qm] = h;
    e.Gz[qm] = g;
  }
  return g;
}

__device__ __forceinline__ float epi_apply(const Epi& e, int m, int j, float v, float& part) {
  // a node that sums two affine edges: the first edge's contribution is added
  // before the epilogue of the second
  if (e.acc_in) v += e.acc_in[(size_t)m * e.acc_ld + j];
  switch (e.kind) {
    case EPI_RELU: return epi_relu(e, m, j, v, part);
    case EPI_CONC: return epi_conc(e, m, j, v, part);
    case EPI_ADJ: return epi_adj(e, m, j, v);
    case EPI_FWD_RELU: return fmaxf(v, 0.f);
    default: return v;
  }
}

// Two-phase form of epi_apply for kernels that finish several outputs per
// thread: epi_load issues every global load an output's epilogue needs (so the
// loads of all of a thread's outputs are in flight together), epi_finish does
// the same arithmetic as epi_apply on the loaded values.
struct EpiIn {
  float acc, l, u, al, be, gp, gph;
  float cb;  // bias of the consuming affine layer at j (ReLU step)
  int s;
};

__device__ __forceinline__ const PropDev* epi_prop(const Epi& e, int n) {
  return e.kind == EPI_CONC ? &e.props[e.pool.prop[n]] : nullptr;
}

// the part of an output's inputs that depends on its column j only
__device__ __forceinline__ float epi_colbias(const Epi& e, int j) {
  return e.kind == EPI_RELU ? e.bias[j / e.bias_div] : 0.f;
}

// every input of output (m, j) except the column bias (in.cb)
__device__ __forceinline__ void epi_load_row(const Epi& e, int n, const PropDev* P, int m, int j,
                                             EpiIn& in) {
  in.acc = e.acc_in ? e.acc_in[(size_t)m * e.acc_ld + j] : 0.f;
  in.al = in.be = in.gp = in.gph = 0.f;
  in.s = 0;
  if (e.kind == EPI_RELU || e.kind == EPI_ADJ) {
    const size_t q = (size_t)n * e.SD + e.off + j;
    const size_t qm = (size_t)m * e.SD + e.off + j;
    in.l = e.pool.L[q];
    in.u = e.pool.U[q];
    in.s = e.pool.S[q];
    if (e.kind == EPI_RELU) {
      if (e.final_mode) {
        in.al = e.pool.ALPHA[q];
        in.be = e.pool.BETA[q];
      }
      if (e.GP) in.gp = e.GP[qm];
      if (e.GPh) in.gph = e.GPh[qm];
    } else {
      in.al = e.pool.ALPHA[q];
      in.gp = e.AP[qm];
    }
  } else if (e.kind == EPI_CONC) {
    in.l = P->lo[j];
    in.u = P->hi[j];
  }
}

// epi_load_row in two parts: the inputs that depend on the node and column only
// (bounds, split, slope, multiplier; the input box), which rows of one node can
// share, and those of the row itself
__device__ __forceinline__ void epi_load_node(const Epi& e, int n, const PropDev* P, int j,
                                              EpiIn& in) {
  in.al = in.be = 0.f;
  in.s = 0;
  if (e.kind == EPI_RELU || e.kind == EPI_ADJ) {
    const size_t q = (size_t)n * e.SD + e.off + j;
    in.l = e.pool.L[q];
    in.u = e.pool.U[q];
    in.s = e.pool.S[q];
    if (e.kind == EPI_ADJ || e.final_mode) in.al = e.pool.ALPHA[q];
    if (e.kind == EPI_RELU && e.final_mode) in.be = e.pool.BETA[q];
  } else if (e.kind == EPI_CONC) {
    in.l = P->lo[j];
    in.u = P->hi[j];
  }
}

__device__ __forceinline__ void epi_load_own(const Epi& e, int m, int j, EpiIn& in) {
  in.acc = e.acc_in ? e.acc_in[(size_t)m * e.acc_ld + j] : 0.f;
  in.gp = in.gph = 0.f;
  const size_t qm = (size_t)m * e.SD + e.off + j;
  if (e.kind == EPI_RELU) {
    if (e.GP) in.gp = e.GP[qm];
    if (e.GPh) in.gph = e.GPh[qm];
  } else if (e.kind == EPI_ADJ) {
    in.gp = e.AP[qm];
  }
}

__device__ __forceinline__ void epi_load(const Epi& e, int n, const PropDev* P, int m, int j,
                                         EpiIn& in) {
  epi_load_row(e, n, P, m, j, in);
  in.cb = epi_colbias(e, j);
}

__device__ __forceinline__ float epi_finish(const Epi& e, int m, int j, float v, const EpiIn& in,
                                            float& part) {
  if (e.acc_in) v += in.acc;
  switch (e.kind) {
    case EPI_RELU: {
      const size_t qm = (size_t)m * e.SD + e.off + j;
      const float l = in.l, u = in.u;
      const int s = in.s;
      float ap = v;
      if (e.GP) ap += in.gp;
      float D, bl = 0.f;
      if (s == -1) D = 1.f;
      else if (s == 1) D = 0.f;
      else if (l >= 0.f) D = 1.f;
      else if (u <= 0.f) D = 0.f;
      else if (ap >= 0.f) D = e.final_mode ? in.al : (u >= -l ? 1.f : 0.f);
      else {
        const float den = u - l;
        D = u / den;
        bl = (-u * l) / den;
      }
      float ah = ap * D;
      if (e.final_mode) ah += in.be * (float)s;
      if (e.GPh) ah += in.gph;
      if (e.AP) e.AP[qm] = ap;
      part += ap * bl + ah * in.cb;
      return ah;
    }
    case EPI_CONC: {
      const float x = v >= 0.f ? in.l : in.u;
      part += v * x;
      if (e.X) e.X[(size_t)m * e.d0 + j] = x;
      return v;
    }
    case EPI_ADJ: {
      const size_t qm = (size_t)m * e.SD + e.off + j;
      const float l = in.l, u = in.u, ap = in.gp, h = v;
      const int s = in.s;
      float D, bl = 0.f;
      bool abr = false;
      if (s == -1) D = 1.f;
      else if (s == 1) D = 0.f;
      else if (l >= 0.f) D = 1.f;
      else if (u <= 0.f) D = 0.f;
      else if (ap >= 0.f) { D = in.al; abr = true; }
      else {
        const float den = u - l;
        D = u / den;
        bl = (-u * l) / den;
      }
      e.GA[qm] = abr ? h * ap : 0.f;
      e.GB[qm] = h * (float)s;
      const float g = h * D + bl;
      if (e.Hz) {
        e.Hz[qm] = h;
        e.Gz[qm] = g;
      }
      return g;
    }
    case EPI_FWD_RELU: return fmaxf(v, 0.f);
    default: return v;
  }
}

__device__ __forceinline__ bool epi_has_part(const Epi& e) {
  return e.part != nullptr && (e.kind == EPI_RELU || e.kind == EPI_CONC);
}

}  // namespace mnbab
