// Internal device data layout and kernel launchers of libmnbab.
//
// Per-node state lives in a structure-of-arrays pool in HBM: every array has
// one row of SD = sum_i d_i floats per node slot (ReLU layers concatenated,
// layer i at offset off[i]), so an epilogue that walks a back-substitution
// row j of layer i reads l, u, S, alpha, beta of its node contiguously.
// Scratch arrays of a launch are indexed by the launch's row m instead.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#define MNBAB_MAXR 16

namespace mnbab {

struct LayerDev {
  int kind;  // 1 fc, 2 conv
  int d_in, d_out;
  int ci, hi, wi, co, ho, wo, k, s, p;
  const float* W;   // fc [d_out][d_in]; conv [co][ci][k][k]
  const float* Wt;  // fc only: [d_in][d_out]
  const float* b;   // [d_out] (fc) or [co] (conv)
  const float* Wb;  // conv only: [co][kh][kw][ci] (back-substitution layout)
  const float* Wf;  // conv only: [ci][kh][kw][co] (forward layout)
  const void* tc;   // host-side tensor-core operands (TcConv for conv, TcFc for FC), or null
  // kernel variant per direction (0 forward, 1 back-substitution) and row
  // bucket (tune_bucket), set by the autotuner; 0 = the built-in choice
  signed char tune[2][6];
};

// Kernel variants of an affine step (the autotuner times them).
enum KernelVariant {
  V_AUTO = 0,    // built-in choice
  V_TC = 1,      // tensor cores (tcgen05, 3xTF32)
  V_IG = 2,      // SIMT implicit GEMM per stride class (conv)
  V_ROW = 3,     // SIMT row-resident kernels (conv)
  V_PLAIN = 4,   // SIMT kernels with the whole weight tensor in shared memory (conv)
  V_G32 = 5,     // SIMT GEMM, 32 x 32 tiles (FC)
  V_G64 = 6,     // SIMT GEMM, 64 x 64 tiles (FC)
  V_SPLITK = 7,  // SIMT split-K GEMM (FC)
  NVARIANT = 8
};
// row bucket of a launch of M rows: <= 32, 128, 512, 2048, 8192, more
inline int tune_bucket(int M) {
  int b = 0;
  for (int lim = 32; b < 5 && M > lim; lim *= 4) ++b;
  return b;
}
constexpr int TUNE_ROWS[6] = {32, 128, 512, 2048, 8192, 32768};

// The network as a DAG: node t = 1..R (ReLU layers) and R + 1 (output) sums
// one or two affine edges, zhat_t = A1(z_src1) + A2(z_src2) (+ biases), with
// z_0 = x.  A chain has one edge (t - 1, aff[t]) per node.
struct NetDev {
  int R;                          // ReLU layers
  int d[MNBAB_MAXR + 2];          // d[0] input, d[i] ReLU layer i
  int off[MNBAB_MAXR + 2];        // offset of ReLU layer i in a node row
  int SD;                         // sum of d[1..R]
  int n_out;                      // logits
  LayerDev aff[MNBAB_MAXR + 2];   // first edge into node t = 1..R+1
  LayerDev aff2[MNBAB_MAXR + 2];  // second edge (residual sum), if n_edge[t] == 2
  int src1[MNBAB_MAXR + 2];       // source node of the first edge
  int src2[MNBAB_MAXR + 2];       // source node of the second edge
  int n_edge[MNBAB_MAXR + 2];
  const float* bfull[MNBAB_MAXR + 2];  // per-neuron sum of the edge biases into t (may be null)
};

// Multi-neuron constraints of one property and ReLU layer.  Row form
// (idx, P, Ph, p) for gradients, CSR by neuron for gamma^T P and gamma^T Phat.
struct MncDev {
  int e;          // rows
  int k;          // neurons per row
  int goff;       // offset of this layer's gamma entries in a node's gamma row
  const int* idx; const float* P; const float* Ph; const float* p;
  const int* cptr; const int* ce; const float* cP; const float* cPh;
};

struct PropDev {
  const float* lo;
  const float* hi;
  const float* Wf;   // folded last layer [n_rows][d_R]
  const float* bf;   // [n_rows]
  int n_rows;
  int E;             // gamma entries per node
  int cab;           // 1: branching scores are divided by the split cost (CAB)
  float cab_inv[MNBAB_MAXR + 1];  // 1 / cost of a split in ReLU layer i
  MncDev mnc[MNBAB_MAXR + 1];  // 1..R
};

struct PoolDev {
  int SD, EC, d0;
  float *L, *U, *ALPHA, *BETA;
  int8_t* S;
  float *MA, *VA, *MB, *VB;
  float *GAM, *MG, *VG;
  float* BESTX;  // [cap][d0]
  float* BEST;   // [cap]
  int* prop;     // property index of each slot
  int* row;      // objective row of each slot
};

// Rows of one back-substitution launch.
struct RowsDev {
  int M;
  const int* node;    // pool slot per row
  const int* j;       // start neuron (intermediate rows) or property row (objective rows)
  const float* sign;  // +1 / -1 (intermediate rows); null for objective rows
  // combination rows (multi-neuron constraint generation): row m starts at
  // sum_k ccoef[3 m + k] zhat_{cidx[3 m + k]} instead of sign * zhat_j
  const int* cidx;
  const float* ccoef;
};

// One multi-neuron constraint row of a group of three neurons:
// P . z_G + Ph . zhat_G <= p.
struct MncRow {
  double P[3], Ph[3], p;
};
// Rows of one group from the 26 lower bounds of d . zhat_G, d in {-1, 0, 1}^3
// without 0 in lexicographic order (csrc/mnc_hull.cu); false: no rows.
bool mnc_group_rows(const double* oct_lb, std::vector<MncRow>& rows);

enum EpiKind { EPI_RELU = 0, EPI_CONC = 1, EPI_ADJ = 2, EPI_FWD_RELU = 3, EPI_STORE = 4 };

// Everything an epilogue may need; unused pointers are null.
struct Epi {
  int kind;
  int layer;         // ReLU layer index (EPI_RELU / EPI_ADJ)
  int off, SD, d0;
  const int* row_node;
  PoolDev pool;
  const PropDev* props;
  bool final_mode;   // objective rows: use alpha/beta of the node, store a'
  const float* GP;   // [M][SD] gamma^T P
  const float* GPh;  // [M][SD] gamma^T Phat
  float* AP;         // [M][SD] a' checkpoints (written in EPI_RELU, read in EPI_ADJ)
  const float* bias; // bias of the consuming affine layer (EPI_RELU)
  int bias_div;      // neuron j uses bias[j / bias_div]
  float* X;          // [M][d0] minimiser (EPI_CONC)
  float* GA;         // [M][SD] d lb / d alpha (EPI_ADJ)
  float* GB;         // [M][SD] d lb / d beta
  float* Gz;         // [M][SD] d lb / d a' (for gamma gradients)
  float* Hz;         // [M][SD] d lb / d ahat
  float* part;       // [M][nslot] row partial sums of the offset c
  int nslot;
  int slot_base;
  int gemm_path;     // 0 auto, 1 SIMT, 2 tensor cores (dense FC steps)
  int* err;          // device error flag (bounded waits of the tensor-core kernel)
  float* ws;         // split-K workspace (may be null: no split)
  size_t ws_floats;
  const float* acc_in;  // earlier edge's contribution added before the epilogue (may alias out)
  int acc_ld;
  int sparse_rows;   // rows started at one neuron and met only convolutions since:
                     // nonzero near it, so conv steps skip the zero region
};

// ---- tensor-core convolutions (tc_conv.cu) --------------------------------
// Pre-split TF32 hi / lo weights per stride class with their TMA tensor maps.
struct TcConv;
// device floats the layer's pre-split weights take (both directions)
size_t tc_conv_floats(const LayerDev& L);
// splits L.W into buf (tc_conv_floats(L) floats, on `st`) and encodes the
// tensor maps; null when the layer or the driver does not support it
TcConv* tc_conv_create(const LayerDev& L, float* buf, cudaStream_t st);
void tc_conv_destroy(TcConv* t);
// dir 0 forward (channels co), dir 1 transposed (channels ci)
bool tc_conv_usable(const LayerDev& L, int dir);
int tc_conv_slots(const LayerDev& L);
// whether launch_backsub (dir 1) / launch_forward (dir 0) take the tensor-core
// kernel for this layer and epilogue (kernels.cu)
bool conv_tc_chosen(const LayerDev& L, int dir, const Epi& e, int M);
// launches the implicit GEMM; returns the partial-sum slots written (dir 1)
int launch_tc_conv(const LayerDev& L, int dir, int M, const float* in, int ld_in, float* out,
                   int ld_out, const Epi& e, cudaStream_t st);

// ---- launchers (kernels.cu, tc_gemm.cu) ----------------------------------
// Tensor-core 3xTF32 GEMM C = A . B^T (+ bias) with the fused epilogue, B the
// pre-split weight operand of direction `dir` of the layer's TcFc `pre` (0: W
// for forward products, 1: W^T for back-substitution); A is split into the
// TcFc's workspace first.  Returns the number of column tiles (partial-sum
// slots written), or -1 without launching anything when the TcFc cannot serve
// this product (no tensor maps, other shape, workspace too small).
int launch_gemm_tc(int M, int N, int K, const float* A, int lda, const float* bias, int bias_div,
                   float* C, int ldc, const Epi& e, int* err, cudaStream_t st, const void* pre,
                   int dir);
// Pre-split TF32 weights of an FC layer for the tensor-core GEMM (tc_gemm.cu).
struct TcFc;
size_t tc_fc_floats(const LayerDev& L);
// workspace floats for coefficient-row products of up to max_rows rows
size_t tc_fc_workspace_floats(const LayerDev& L, int max_rows);
TcFc* tc_fc_create(const LayerDev& L, float* buf, cudaStream_t st);
void tc_fc_set_workspace(TcFc* t, float* ws, size_t floats);
void tc_fc_destroy(TcFc* t);
// Starting rows: a = sign * W_t[j, :] (t <= R) or Wf[row, :] (t = R + 1) on
// z^(t-1), with c = sign * b_t[j] into slot 0, through epilogue `e`.
void launch_init_rows(const NetDev& net, int t, int edge, const RowsDev& rows, float* out, int ld,
                      const Epi& e, cudaStream_t st);
// Intermediate-bound rows of ReLU layer 1 (one affine step from the input box):
// lower bounds straight to lb[m].
void launch_first_rows(const NetDev& net, const PoolDev& pool, const PropDev* props,
                       const RowsDev& rows, float* lb, cudaStream_t st);
// Windowed back-substitution of intermediate-bound rows that start at a
// convolution neuron of zhat_t and meet only convolutions below it: after each
// step the row is nonzero only within its receptive-field window, so one CTA
// carries it to the input in shared memory.  h[i] x w[i] is the window at
// layer i (all of the layer's channels); maxw the largest window in floats.
struct WinPlan {
  int t;
  int h[MNBAB_MAXR + 2], w[MNBAB_MAXR + 2];
  int maxw;
};
// Plan for rows at zhat_t with the DeepPoly epilogue, or false where the layers
// below t are not a single chain of convolutions or the windows do not fit.
bool win_plan(const NetDev& net, int t, WinPlan& wp);
// Bounds of rows.M rows through plan wp: the whole lower bound of row m (offset
// terms, concretisation and sign * b_t[j]) goes to partial slot e.slot_base.
void launch_win_rows(const NetDev& net, const WinPlan& wp, const RowsDev& rows, const Epi& e,
                     cudaStream_t st);
// Fused optimisation loop for chain networks without multi-neuron constraints
// (csrc/fused.cu): one CTA per objective row runs all sweeps, adjoints and Adam
// steps.  bc1[s] / bc2[s] are Adam's bias corrections 1 - beta^(s+1).
constexpr int FUSED_MAX_STEPS = 64;
struct FusedHP {
  int steps;
  float lr_a, lr_b, b1, b2, eps_abs, eps_rel, floor;
  float bc1[FUSED_MAX_STEPS], bc2[FUSED_MAX_STEPS];
};
bool fused_supported(const NetDev& net, int SD, int d0, int steps);
// rows m < M: node row_node[m], objective row row_j[m]; a' of the final sweep
// goes to AP_out [M][SD]; GB_out [M][SD] is row scratch for d lb / d beta;
// BEST / BESTX of the node track the best iterate.
// allow_tc: the largest conv layer whose operands fit takes its transposed
// convolution on the tensor cores (3xTF32); err is the device error flag of
// its bounded waits (null: SIMT only).  skip_lb (optional, by row): rows whose
// value is positive (verified by the DeepPoly pass) are not optimised.
void launch_opt_chain(int M, const NetDev& net, const PoolDev& pool, const PropDev* props,
                      const int* row_node, const int* row_j, const FusedHP& hp, float* AP_out,
                      float* GB_out, bool allow_tc, int* err, cudaStream_t st,
                      const float* skip_lb = nullptr);
// the layer launch_opt_chain(allow_tc = true) runs on the tensor cores (0: none)
int fused_tc_layer(const NetDev& net, int SD, int d0);
// Intermediate-bound rows that start at a fully connected neuron of zhat_t0
// above a chain of FC / conv layers: one persistent CTA loop, each row carried
// to the input in shared memory with DeepPoly epilogues; lower bounds to lb[m].
bool sweep_chain_supported(const NetDev& net, int t0);
void launch_sweep_chain(const NetDev& net, const PoolDev& pool, const PropDev* props,
                        const RowsDev& rows, int t0, float* lb, cudaStream_t st);
// Adversarial pre-attack of property `prop` (chain networks): CTA b = r *
// n_starts + s runs sign-step PGD on row r from start s; best_out[b] is its
// smallest margin, bx_out [b][d0] the first minimiser.
bool attack_supported(const NetDev& net);
void launch_attack_chain(const NetDev& net, const PropDev* props, int prop, int n_rows,
                         const float* starts, int n_starts, int steps, float* best_out,
                         float* bx_out, cudaStream_t st);
// Back-substitution through affine layer i: in [M][d_i] -> out [M][d_{i-1}].
// Returns the number of partial-sum slots used.
// One kernel variant of the back-substitution (dir 1) or forward (dir 0) step
// through layer L: the partial-sum slots written (back-substitution) or 0, or
// -1 without launching when the variant does not take this layer.
int launch_affine_variant(int variant, int dir, const LayerDev& L, int M, const float* in,
                          int ld_in, float* out, int ld_out, const Epi& e, cudaStream_t st);
int launch_backsub(const LayerDev& L, int M, const float* in, int ld_in, float* out, int ld_out,
                   const Epi& e, cudaStream_t st);
int backsub_slots(const LayerDev& L);
// Whether the conv kernels can stage the layer in shared memory.
bool conv_supported(const LayerDev& L);
// Forward through affine layer i (+ bias): in [M][d_{i-1}] -> out [M][d_i].
void launch_forward(const LayerDev& L, int M, const float* in, int ld_in, float* out, int ld_out,
                    const Epi& e, cudaStream_t st);
// lb[m] = sum of partial slots - gp0[m]; with track, keep the best bound and
// its minimiser per node.
void launch_reduce_lb(int M, const float* part, int nslot, int used, const float* gp0,
                      float* lb, bool track, const int* row_node, PoolDev pool, const float* X,
                      int d0, cudaStream_t st);
// Unstable unsplit neurons of layer t for each node -> rows (+, -).
void launch_collect_rows(int nb, const int* nodes, PoolDev pool, int off, int d, int* counter,
                         int* row_node, int* row_j, float* row_sign, cudaStream_t st);
void launch_update_bounds(int npairs, const int* row_node, const int* row_j, const float* lb,
                          PoolDev pool, int off, cudaStream_t st);
void launch_gamma_proj(int M, const int* row_node, PoolDev pool, const PropDev* props,
                       const NetDev& net, float* GP, float* GPh, float* gp0, cudaStream_t st);
void launch_gamma_grad(int M, const int* row_node, PoolDev pool, const PropDev* props,
                       const NetDev& net, const float* Gz, const float* Hz, float* GG,
                       cudaStream_t st);
// Adam step; with G = max|g| of the row: dead-zone |g| <= floor * G and
// denominator eps max(eps, eps_rel * G).
void launch_adam(int M, const int* row_node, PoolDev pool, const PropDev* props, int SD,
                 const float* GA, const float* GB, const float* GG, float* gmax, float floor,
                 float lr_a, float lr_b, float lr_g, float b1, float b2, float eps, float eps_rel,
                 float bc1, float bc2, cudaStream_t st);
void launch_zero_adam(int M, const int* row_node, PoolDev pool, cudaStream_t st);
void launch_set_best(int M, const int* row_node, PoolDev pool, float v, cudaStream_t st);
void launch_acs(int M, const int* row_node, PoolDev pool, const PropDev* props, const NetDev& net,
                const float* GP, const float* GPh, const float* AP, int has_gamma, int* out_layer,
                int* out_neuron, float* out_score, int* out_fallback, cudaStream_t st);
void launch_children(int nb, const int* parents, const int* kids, const int* layer,
                     const int* neuron, PoolDev pool, const NetDev& net, cudaStream_t st);
// Optimised intermediate bounds (Sec. 3.1, parameter sharing): set slots
// dst[b] start from node src[b] with DeepPoly slopes, beta = 0, zero moments;
// per-row best bounds; per-set gradient sums over segments (set, first row,
// end row) of a chunk's rows; the nodes' bounds intersected with the best.
void launch_set_init(int nsets, const int* src, const int* dst, PoolDev pool, cudaStream_t st);
void launch_rows_best(int M, const float* lb, float* best, int first, cudaStream_t st);
void launch_set_grad(int nseg, const int* seg, int SD, int lim, const float* GA, const float* GB,
                     float* IGA, float* IGB, cudaStream_t st);
// per-set gradient of the multipliers of constraints in ReLU layers below t
void launch_set_grad_gamma(int nseg, const int* seg, const int* set_slot, PoolDev pool,
                           const PropDev* props, int t, const float* GG, float* IGG,
                           cudaStream_t st);
void launch_set_update(int M, const int* orig, const int* j, const float* sign, const float* best,
                       PoolDev pool, int off, cudaStream_t st);
// Root nodes: slots[i] initialised from root-bound slot srcs[i] for row rows[i].
void launch_root_init(int nb, const int* slots, const int* srcs, const int* rows, PoolDev pool,
                      cudaStream_t st);
// Pre-attack in the per-layer form: candidate slots (no splits, zero
// parameters, property and row, points clipped from the starts), the
// pre-activation capture (slot bounds l = u = zhat, z <- max(zhat, 0)), best
// tracking and the clipped sign step.
void launch_attack_init(int M, int q0, int n_starts, const int* slots, PoolDev pool, int prop,
                        const PropDev* props, const float* starts, float* X, float* best,
                        cudaStream_t st);
void launch_pattern_relu(int M, const int* slots, PoolDev pool, int off, int d, float* z,
                         cudaStream_t st);
void launch_attack_best(int M, const float* f, const float* X, int d0, float* best, float* bx,
                        cudaStream_t st);
void launch_attack_step(int M, const float* g, int ld, float* X, int d0, const PropDev* props,
                        int prop, int steps, cudaStream_t st);
void launch_final_dot(int M, const int* row_node, PoolDev pool, const PropDev* props,
                      const float* z, int ld, int dR, float* f, cudaStream_t st);
// Counterexample confirmation in FP64 needs a per-row buffer of d0 + SD doubles.

void launch_fill(float* p, size_t n, float v, cudaStream_t st);
// slots[b]: l = -inf, u = +inf, S = 0, prop = prop[b] (b < nb)
void launch_root_slot_init(int nb, const int* slots, const int* prop, PoolDev pool,
                           cudaStream_t st);
// FP64 forward pass f_r(x) of rows of X (counterexample confirmation).
void launch_forward_f64(int M, const int* row_node, PoolDev pool, const PropDev* props,
                        const NetDev& net, const float* X, int ldx, double* buf, int ldb,
                        double* fout, cudaStream_t st, const int* dcount = nullptr);
// batch rows with a negative FP32 objective and a non-positive best bound, in
// batch order: cand_idx / cand_slot [count], count on the device
void launch_select_cand(int M, const float* fout, const int* slots, const float* best,
                        int* cand_idx, int* cand_slot, int* count, cudaStream_t st);

}  // namespace mnbab
