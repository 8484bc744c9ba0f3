/*
 * mnbab.h -- C ABI of the GB300 library for batched MN-BaB bounding.
 *
 * The library bounds branch-and-bound (BaB) subproblems of the neural-network
 * verification problem min_{x in D} f(x) (Sec. 2.1, Eq. 1), with the linear
 * property folded into a final affine layer so that the goal is f(x) > 0, by
 * back-substitution through affine and ReLU layers with optimisable slopes
 * alpha, split multipliers beta and multi-neuron-constraint multipliers gamma
 * (Sec. 3.1), projected Adam ascent on those parameters (Sec. 3.1), Active
 * Constraint Score branching (Sec. 3.2) and a FIFO BaB queue (Sec. 2.2).
 *
 * Conventions
 *  - Every call returns an mnbab_status; nothing throws across the ABI.
 *  - Host pointers passed in are read before the call returns and stay owned
 *    by the caller; outputs go to caller-allocated host memory.
 *  - Handles are opaque.  Device memory is owned by the context, allocated with
 *    cudaMalloc within the context's HBM budget, and freed by mnbab_destroy.
 *  - All work of a context runs on its stream (mnbab_options.stream, or a
 *    stream the library creates); calls are synchronous with respect to the
 *    host unless stated otherwise.  One context per host thread.
 *  - Floating point is IEEE FP32 on the device; the library re-checks every
 *    counterexample with an FP64 forward pass (device kernel) before reporting it.
 *  - Errors: MNBAB_E_INVALID_ARG for bad handles, sizes or shapes;
 *    MNBAB_E_BUDGET when the HBM budget or a pool capacity would be exceeded;
 *    MNBAB_E_DEVICE for CUDA errors; MNBAB_E_UNSUPPORTED for layer kinds or
 *    shapes the library does not handle.  mnbab_last_error() gives the text.
 */
#ifndef MNBAB_H
#define MNBAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mnbab_status;
#define MNBAB_OK 0
#define MNBAB_E_INVALID_ARG (-1)
#define MNBAB_E_BUDGET (-2)
#define MNBAB_E_DEVICE (-3)
#define MNBAB_E_TIMEOUT (-4)
#define MNBAB_E_UNSUPPORTED (-5)

/* verdicts (Sec. 2.2): a lower bound > 0 on every subdomain verifies, an
 * input with f_r(x) < 0 falsifies */
#define MNBAB_UNKNOWN 0
#define MNBAB_VERIFIED 1
#define MNBAB_FALSIFIED (-1)

typedef struct mnbab_ctx mnbab_ctx;
typedef struct mnbab_net mnbab_net;
typedef struct mnbab_prop mnbab_prop;

/* A node id names one BaB subproblem held in the context's device node pool. */
typedef int64_t mnbab_node_id;

typedef struct {
  int32_t device;              /* CUDA device ordinal */
  uint64_t hbm_budget_bytes;   /* cap on the context's device allocations; 0 = 64 GiB */
  void* stream;                /* cudaStream_t to run on; NULL = a stream of the library */
  int32_t node_capacity;       /* node slots per network pool; 0 = 65536 */
  int32_t max_mnc_rows;        /* gamma entries per node (sum over layers); 0 = none */
  int32_t row_chunk;           /* max back-substitution rows per launch; 0 = 32768, at most 65534 */
  int32_t gemm_path;           /* dense FC steps: 0 = auto (tcgen05 3xTF32 when a launch fills
                                  two waves of 128-row tiles, else SIMT FP32), 1 = SIMT FP32
                                  only, 2 = tcgen05 3xTF32 always.  It also picks the form of
                                  the optimisation loop of chain networks without multi-neuron
                                  constraints: 0 = one fused launch per batch whose largest
                                  conv layer's transposed convolution runs on tcgen05, 1 = the
                                  fused launch in SIMT FP32 only, 2 = per-layer launches */
  int32_t use_graphs;          /* 1 = replay the optimisation loop from captured CUDA graphs
                                  (rows padded to multiples of 64, one graph per padded size);
                                  0 = launch it kernel by kernel (default) */
} mnbab_options;

/* Layer kinds.  A network is a list of ops; an FC or CONV2D op reads the
 * previous op unless src_a names another (1-based op index, or -1 for the
 * network input); a RELU reads the previous op, which must be an FC / CONV2D
 * op or an ADD; an ADD sums the outputs of the FC / CONV2D / ADD ops src_a and
 * src_b (1-based), as in residual blocks (ResAdd).  Every affine op must read
 * a RELU output or the input, at most two affine ops may sum into one RELU,
 * and the last op must be an FC layer. */
#define MNBAB_FC 1
#define MNBAB_CONV2D 2
#define MNBAB_RELU 3
#define MNBAB_ADD 4

typedef struct {
  int32_t kind;
  /* FC: in_c = in features, out_c = out features, spatial sizes 1.
   * CONV2D: input in_c x in_h x in_w, output out_c x out_h x out_w,
   *         square kernel k, stride, zero padding pad (all sides). */
  int32_t in_c, in_h, in_w;
  int32_t out_c, out_h, out_w;
  int32_t k, stride, pad;
  const float* W; /* FC [out_c][in_c]; CONV2D [out_c][in_c][k][k]; row-major */
  const float* b; /* [out_c] */
  int32_t src_a, src_b; /* see the layer kinds above; 0 = the previous op */
} mnbab_layer_desc;

/* Projected Adam ascent on (alpha, beta, gamma) (Sec. 3.1). */
typedef struct {
  int32_t steps;   /* gradient steps; the bound is evaluated steps + 1 times */
  float lr_alpha, lr_beta, lr_gamma;
  float beta1, beta2, eps;
  /* Optional, off by default (0 gives standard projected Adam):
   * grad_floor: components with |g| <= grad_floor * G count as zero;
   * eps_rel: Adam's denominator uses max(eps, eps_rel * G) instead of eps;
   * with G = max_j |g_j| over all of a node's parameters.  Constraints that
   * are tight at the relaxed point have gradients at rounding level; with the
   * fixed eps, Adam's per-component normalisation turns that noise into steps
   * of full size and random sign, so FP32 and FP64 runs of the same
   * optimisation can part by more than 1e-3.  eps_rel = 1e-3 keeps the update
   * continuous in the gradient (the runs then agree to about 1e-6); it is not
   * the paper's optimiser, which names only projected gradient ascent. */
  float grad_floor;
  float eps_rel;
} mnbab_adam;

typedef struct {
  int32_t nodes_bounded;   /* subproblems bounded in this step */
  int32_t nodes_verified;  /* closed with lower bound > 0 */
  int32_t nodes_falsified; /* closed with an FP64-confirmed counterexample */
  int32_t nodes_branched;  /* split into two children */
  int32_t nodes_leaf;      /* open but nothing left to split */
  int32_t props_done;      /* properties with a final verdict after this step */
  int64_t rows_rebounded;  /* intermediate-bound rows back-substituted */
  int64_t h2d_bytes;       /* host-to-device bytes copied by the step */
  int64_t d2h_bytes;       /* device-to-host bytes copied by the step */
} mnbab_step_stats;

/* Per-kernel-class timing (CUDA events on the context's stream around every
 * launch of the class) and the algorithmic work those launches did. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;     /* summed launch durations */
  double flops;  /* algorithmic floating-point operations (1 FMA = 2) */
  double bytes;  /* algorithmic HBM bytes (each operand read or written once) */
} mnbab_kernel_stat;

/* One record per bounded node, in bounding order (for traces and tests). */
typedef struct {
  int64_t seq;           /* FIFO node number within the property */
  int32_t row;           /* property row */
  int32_t depth;
  float lb;              /* node lower bound (best of DeepPoly pass and Adam iterates) */
  float lb_deeppoly;
  float f_xstar;         /* f_r at the minimiser x* (FP64 host value) */
  int32_t verdict;       /* MNBAB_VERIFIED / _FALSIFIED / _UNKNOWN (branched or leaf) */
  int32_t split_layer;   /* ReLU layer (1-based) of the chosen split, 0 if none */
  int32_t split_neuron;
  int32_t fallback;      /* 1 if the split came from the intercept fallback score */
  int32_t leaf;          /* 1 if the node had no unstable unsplit neuron left (a leaf) */
} mnbab_trace_rec;

/* ---- context ---------------------------------------------------------- */
/* Creates a context on opt->device.  opt may be NULL for defaults. */
mnbab_status mnbab_create(const mnbab_options* opt, mnbab_ctx** out);
/* Frees every device allocation, network and property of the context. */
void mnbab_destroy(mnbab_ctx* ctx);
/* Text of the last error of this context; valid until its next call. */
const char* mnbab_last_error(const mnbab_ctx* ctx);

/* ---- network and property (Sec. 2.1, Eq. 1) --------------------------- */
/* Copies a chain network to the device.  The last layer must be FC; its
 * outputs are the logits that properties fold into (Sec. 2.1). */
mnbab_status mnbab_load_network(mnbab_ctx* ctx, const mnbab_layer_desc* layers, int32_t n_layers,
                                mnbab_net** out);

/* Sets a property: input box x_lo <= x <= x_hi (d0 floats each, the clipped
 * L-inf ball of Sec. 2.1) and rows C f(x) + d > 0 (C [n_rows][n_out]
 * row-major, d [n_rows]).  Folds C into the last layer and uploads the box
 * and the folded layer.  When the property starts (its first mnbab_bab_step,
 * or the first call that reads roots), the DeepPoly intermediate bounds of
 * every ReLU layer are computed on the device (Sec. 3.1, one
 * back-substitution per neuron and side) and one root node per row is
 * queued.  *out stays valid until mnbab_destroy. */
mnbab_status mnbab_set_property(mnbab_ctx* ctx, const mnbab_net* net, const float* x_lo,
                                const float* x_hi, const float* C, const float* d,
                                int32_t n_rows, mnbab_prop** out);

/* Root bounds l, u of ReLU layer relu_layer (1-based), d_i floats each: the
 * intermediate bounds of Sec. 3.1 at the property's root. */
mnbab_status mnbab_get_root_bounds(const mnbab_ctx* ctx, const mnbab_prop* prop,
                                   int32_t relu_layer, float* l_out, float* u_out);

/* Uploads the multi-neuron constraints P z + Phat zhat - p <= 0 of one ReLU
 * layer (Sec. 3.1, enforcing multi-neuron constraints), n_rows rows over k
 * neurons each: idx [n_rows][k] neuron indices, P and Phat [n_rows][k], p
 * [n_rows].  Called once per layer after mnbab_set_property and before any
 * bounding; gamma of existing nodes starts at 0. */
mnbab_status mnbab_set_mnc(mnbab_ctx* ctx, mnbab_prop* prop, int32_t relu_layer, int32_t n_rows,
                           int32_t k, const int32_t* idx, const float* P, const float* Phat,
                           const float* p);

/* Generates and uploads the multi-neuron constraints of every ReLU layer of a
 * property (Sec. 3.1, enforcing multi-neuron constraints; the paper takes them
 * from PRIMA and gives no generator).  This library's construction, from the
 * property's root bounds (the property is started if it was not; DeepPoly
 * bounds, or the optimised ones when mnbab_set_intermediate_steps asked for
 * them, whose sets then hold no constraints):
 *  - groups: the unstable neurons of the layer in the order of decreasing
 *    -l u / (u - l) (ties by index), taken as sliding triples (j0, j1, j2),
 *    (j1, j2, j3), ..., at most max_groups per layer;
 *  - per group, the DeepPoly lower bounds of d . zhat_G for the 26 directions
 *    d in {-1, 0, 1}^3 \ {0}, back-substituted on the device;
 *  - per group, on the host in FP64 (threads over groups), the facets of the
 *    convex hull of the ReLU graph over that octahedron (mnbab_mnc_group),
 *    uploaded as with mnbab_set_mnc.
 * Every layer counts as set afterwards (mnbab_set_mnc then refuses it); call
 * before bounding any node of the property.  A property that its pre-attack
 * (mnbab_set_attack) falsified when it started gets no rows.  *rows_out (nullable) receives
 * the number of constraint rows.  MNBAB_E_BUDGET when the rows exceed
 * mnbab_options.max_mnc_rows (the exact hull gives about 100 to 250 rows per
 * group). */
mnbab_status mnbab_generate_mnc(mnbab_ctx* ctx, mnbab_prop* prop, int32_t max_groups,
                                int64_t* rows_out);

/* Reads back the constraint rows of one ReLU layer of a property (as set by
 * mnbab_set_mnc or mnbab_generate_mnc, k = 3 neurons a row): idx and P, Phat
 * [max_rows][3], p [max_rows] (host); *n_out = the number of rows
 * (MNBAB_E_BUDGET, with *n_out set, when it exceeds max_rows). */
mnbab_status mnbab_get_mnc(mnbab_ctx* ctx, const mnbab_prop* prop, int32_t relu_layer,
                           int32_t max_rows, int32_t* idx, float* P, float* Phat, float* p,
                           int32_t* n_out);

/* The constraint rows of one group of three neurons from its octahedron, on
 * the host only (no device, no context): oct_lb[26] are lower bounds of
 * d . zhat_G for d in {-1, 0, 1}^3 \ {0} in lexicographic order of
 * (d0, d1, d2) (d0 slowest).  Rows are P . relu(zhat_G) + Phat . zhat_G <= p:
 * the facets of the convex hull of {(relu(x), x) : x in the octahedron} with
 * unit normals (|(P, Phat)| = 1), offsets at the exact support, and without
 * facets that involve one neuron only.  P, Phat [max_rows][3] and p
 * [max_rows] (host, FP64) receive the rows, *n_out their number (0 when the
 * octahedron is degenerate); MNBAB_E_BUDGET (with *n_out set) when more than
 * max_rows rows exist. */
mnbab_status mnbab_mnc_group(const double* oct_lb, int32_t max_rows, double* P, double* Phat,
                             double* p, int32_t* n_out);

/* ---- nodes ------------------------------------------------------------- */
/* A fresh root node of property row `row` outside the property's BaB queue
 * (the root subproblem of Sec. 2.2: root bounds, DeepPoly slopes,
 * beta = gamma = 0). */
mnbab_status mnbab_node_root(mnbab_ctx* ctx, mnbab_prop* prop, int32_t row, mnbab_node_id* out);
mnbab_status mnbab_node_free(mnbab_ctx* ctx, mnbab_node_id node);

/* Parameter block of a node, little-endian, in this order:
 *   int32 split_layer (0..R; layers > split_layer are re-bounded by the next
 *         mnbab_bound_batch), int32 R, int32 SD = sum_i d_i, int32 E,
 *   float l[SD], float u[SD], int8 S[SD], float alpha[SD], float beta[SD],
 *   float gamma[E]
 * where per-neuron arrays concatenate ReLU layers 1..R and S uses the split
 * encoding of Sec. 3.1 (-1 positive split, +1 negative split, 0 none).
 * With host_buf NULL, *bytes receives the size. */
mnbab_status mnbab_export_params(const mnbab_ctx* ctx, mnbab_node_id node, void* host_buf,
                                 size_t* bytes);
mnbab_status mnbab_import_params(mnbab_ctx* ctx, mnbab_node_id node, const void* host_buf,
                                 size_t bytes);

/* ---- bounding (Sec. 3.1) --------------------------------------------- */
/* For each node: re-bound the ReLU layers after its split layer (only its
 * unstable, unsplit neurons, with DeepPoly slopes and beta = gamma = 0,
 * intersected with its current bounds; Sec. 3.2 enforcing splits), then bound
 * its objective row at its current (alpha, beta, gamma).  lb_out[i] gets the
 * lower bound, ub_out[i] (nullable) f_r(x*) at the minimiser x* (FP32). */
mnbab_status mnbab_bound_batch(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                               float* lb_out, float* ub_out);

/* The DeepPoly pass of each node's objective (Sec. 4, experimental setup:
 * DeepPoly before the optimisation; slopes from the area heuristic,
 * beta = gamma = 0); nodes must already be re-bounded. */
mnbab_status mnbab_deeppoly_batch(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                                  float* lb_out);

/* The objective bound at the node's parameters and its gradient w.r.t.
 * (alpha, beta, gamma) from the adjoint back-substitution (Sec. 3.1: the bound
 * is optimised by gradient ascent in these parameters): grad_out holds
 * n * (2 * SD + E) floats, per node alpha[SD], beta[SD], gamma[E]. */
mnbab_status mnbab_bound_grad(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                              float* lb_out, float* grad_out);

/* Sets the parameters of each node from params, laid out as grad_out of
 * mnbab_bound_grad: per node alpha[SD], beta[SD], gamma[E] (host floats).  The
 * values are taken as given: a bound is sound only for 0 <= alpha <= 1 and
 * beta, gamma >= 0 (Sec. 3.1), so callers that step the parameters project
 * them.  Bounds and splits of the nodes are unchanged. */
mnbab_status mnbab_set_params(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                              const float* params);

/* cfg->steps projected Adam steps (Sec. 3.1, projected gradient ascent) from
 * each node's current parameters (alpha clamped to [0, 1], beta, gamma >= 0).  best_lb_out[i] = the best
 * bound over the steps + 1 evaluated iterates; the node keeps the last
 * iterate's parameters.  Nodes must already be re-bounded.  For a chain of
 * FC / CONV2D layers without multi-neuron constraints the whole loop runs in
 * one launch, one CTA per node (see mnbab_options.gemm_path). */
mnbab_status mnbab_optimize(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                            const mnbab_adam* cfg, float* best_lb_out);

/* Optimised intermediate bounds (Sec. 3.1, parameter sharing).  For ReLU
 * layers t = max(2, first_layer) .. R in order: the rows are the unstable,
 * unsplit neurons j of layer t of each node, once as lower bounds (+e_j) and
 * once as upper bounds (-e_j).  Each (node, side) has one parameter set
 * (alpha and beta over the ReLU layers below t) shared by its rows, started at
 * DeepPoly slopes (alpha = 1 if u >= -l else 0) and beta = 0; cfg->steps
 * projected Adam steps ascend the sum of the rows' bounds (cfg NULL: 20 steps,
 * default rates).  Each row keeps the best bound of the steps + 1 iterates,
 * and the node's bounds of layer t are intersected with them before layer
 * t + 1.  Works on each node's current bounds (re-bound split nodes first,
 * e.g. with mnbab_bound_batch); the nodes' own parameters are unchanged.
 * With multi-neuron constraints a set also holds gamma (Sec. 3.1: gamma is a
 * parameter like alpha and beta) for the constraints of the layers below t,
 * started at 0 and stepped at lr_gamma; the other multipliers stay 0.
 * At most half the context's batch capacity of nodes per call, each listed
 * once (a repeated node is MNBAB_E_INVALID_ARG).  *rows_out (nullable) receives the
 * number of rows bounded.  Scratch node slots are taken from the pool for the
 * duration of the call (MNBAB_E_BUDGET if it is full).  The rows of one layer
 * (2 x unstable neurons x nodes) must fit the network's row scratch
 * (min(2^26, 2 * SD * batch capacity) rows, at least row_chunk and 2 * SD);
 * more is MNBAB_E_BUDGET with both counts in the message: pass fewer nodes. */
mnbab_status mnbab_optimize_intermediate(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                                         int32_t first_layer, const mnbab_adam* cfg,
                                         int64_t* rows_out);

/* Optimised intermediate bounds at the root of a property, as
 * mnbab_optimize_intermediate with `steps` Adam steps at the default rates:
 * run when the property starts, after its DeepPoly root bounds and before its
 * root nodes take them; 0 (the default) keeps the DeepPoly root bounds.  Call
 * before the property starts (MNBAB_E_INVALID_ARG after), on a context whose
 * batch capacity is at least 2 (node_capacity >= 4; MNBAB_E_INVALID_ARG
 * otherwise).  The root's sets use the constraints uploaded by then (none when
 * mnbab_generate_mnc starts the property: it generates from the optimised
 * root bounds). */
mnbab_status mnbab_set_intermediate_steps(mnbab_ctx* ctx, mnbab_prop* prop, int32_t steps);

/* ACS branching score (Sec. 3.2) at each node's current parameters:
 * s_j = |(gamma^T P)_j| + |(gamma^T Phat)_j| over unstable unsplit neurons,
 * or, when every candidate scores 0, the intercept score
 * |a'_j| (-l_j u_j / (u_j - l_j)).  Picks the lowest (layer, neuron) among
 * scores within 1e-5 (relative) of the maximum.  layer_out is 0 when the
 * node has no candidate. */
mnbab_status mnbab_score_branches(mnbab_ctx* ctx, const mnbab_node_id* nodes, int32_t n,
                                  int32_t* layer_out, int32_t* neuron_out, float* score_out);

/* ---- branch and bound (Sec. 2.2, Sec. 3.2) ----------------------------- */
/* One BaB step over the given properties (all of one network): pops up to
 * max_nodes open nodes in FIFO order from their queues (within each
 * property's node budget), re-bounds, runs the DeepPoly pass, optimises the
 * nodes it does not verify, checks the minimiser for a counterexample,
 * branches the rest by ACS and queues their two children.  This call starts
 * (creates and bounds the root nodes of) only the properties passed to it;
 * calls that read roots (get_root_bounds, node_root, bound_batch ...) start
 * every property set on the network.  A caller can so upload many properties
 * ahead of time and step a window of them.  cfg may be
 * NULL (20 steps, default rates).  max_nodes is clamped to the context's batch
 * capacity. */
mnbab_status mnbab_bab_step(mnbab_ctx* ctx, mnbab_prop* const* props, int32_t n_props,
                            int32_t max_nodes, const mnbab_adam* cfg, mnbab_step_stats* out);

/* Exact completion of fully split leaves (Sec. 3.3: with every unstable
 * neuron split, the network is affine on the node's region, and the bound
 * maximised over beta, gamma reaches the region's exact minimum by LP duality).
 * A node that has no unstable unsplit neuron left and whose bound does not
 * verify it takes `steps` more projected Adam steps from its parameters: every
 * iterate's bound is a certified lower bound (> 0 verifies the node), and the
 * average of the iterates' minimisers over the second half of the steps is
 * checked in FP64 as a counterexample (< 0 falsifies the property).  A leaf
 * decided by neither stays UNKNOWN.  0 turns completion off; default 256. */
mnbab_status mnbab_set_leaf_steps(mnbab_ctx* ctx, mnbab_prop* prop, int32_t steps);

/* Per-property node budget (bounded nodes including roots); default 256. */
mnbab_status mnbab_set_budget(mnbab_ctx* ctx, mnbab_prop* prop, int32_t max_nodes);

/* Per-property wall-clock limit (Sec. 4: each property has a timeout; a
 * property not decided within it counts as unknown).  The clock starts at the
 * property's first mnbab_bab_step; a step that ends after the limit with the
 * property still open sets its verdict to MNBAB_UNKNOWN and frees its queue.
 * 0 (the default) sets no limit; negative values are MNBAB_E_INVALID_ARG. */
mnbab_status mnbab_set_timeout(mnbab_ctx* ctx, mnbab_prop* prop, double seconds);

/* Progress of a property: nodes bounded so far, whether its timeout ended it
 * (1) or not (0), and the seconds since its first BaB step (0 before it);
 * every output is nullable. */
mnbab_status mnbab_get_status(const mnbab_ctx* ctx, const mnbab_prop* prop, int32_t* bounded,
                              int32_t* timed_out, double* elapsed_s);

/* Branching score of a property (Sec. 3.2): mode 0 = ACS; mode 1 = ACS + CAB,
 * the score divided by the cost of the split (App. B): with per-layer costs
 * (affine: weight entries, or d_out k^2 for a convolution; ReLU: d + number
 * of multi-neuron constraints) and C_t the cost of back-substituting from
 * zhat_t, a split in ReLU layer k costs sum_{t>k} 2 d_t C_t plus one
 * objective back-substitution (this library's addition, so that the last
 * layer's cost is positive). */
mnbab_status mnbab_set_branching(mnbab_ctx* ctx, mnbab_prop* prop, int32_t mode);

/* Verdict of a property (row < 0) or of one row (Sec. 2.2: VERIFIED when every
 * subproblem's lower bound is positive, FALSIFIED by a concrete input with a
 * negative margin).  lb (nullable) = the lowest
 * open or leaf lower bound seen (+inf if verified).  x_cex (nullable, d0
 * floats) receives the counterexample when FALSIFIED. */
mnbab_status mnbab_get_verdict(const mnbab_ctx* ctx, const mnbab_prop* prop, int32_t row,
                               int32_t* verdict, float* lb, float* x_cex);

/* Copies up to max_recs trace records of the property's bounded nodes. */
mnbab_status mnbab_get_trace(const mnbab_ctx* ctx, const mnbab_prop* prop, mnbab_trace_rec* recs,
                             int32_t max_recs, int32_t* n_out);

/* enable = 1 clears the per-kernel statistics and starts timing every launch
 * with CUDA events (adds a little launch overhead); enable = 0 stops. */
mnbab_status mnbab_profile(mnbab_ctx* ctx, int32_t enable);

/* Restricts CUDA-event timing to the kernel classes whose bit is set (bit i =
 * the i-th statistic of mnbab_profile_read); launches and algorithmic work are
 * still counted for every class.  All classes are timed by default.  Timing
 * few classes keeps the per-launch event overhead out of a measured region. */
mnbab_status mnbab_profile_mask(mnbab_ctx* ctx, uint64_t class_mask);

/* Reads up to max_stats kernel-class statistics (synchronises the stream) and
 * the number of kernels the context has launched since it was created. */
mnbab_status mnbab_profile_read(mnbab_ctx* ctx, mnbab_kernel_stat* stats, int32_t max_stats,
                                int32_t* n_out, int64_t* total_launches);

/* ---- serving: continuous batching of verification requests ------------ */
typedef struct {
  int32_t admitted;        /* requests admitted in this pass */
  int32_t finished;        /* requests that got their final verdict in this pass */
  int32_t active;          /* admitted, not finished */
  int32_t queued;          /* waiting for admission */
  mnbab_step_stats step;   /* summed over the networks' BaB steps */
  int64_t reserved_bytes;  /* HBM held by the active requests' node slots after the pass */
} mnbab_serve_stats;

/* Queues a property (created by mnbab_set_property and not yet used) as a
 * request of the context's request loop; timeout_s > 0 limits its time from
 * this call to its verdict (UNKNOWN when exceeded).  A finished request's
 * record stays in the context, readable by its ticket, until mnbab_destroy;
 * its node slots and HBM reservation are released when it finishes. */
mnbab_status mnbab_submit(mnbab_ctx* ctx, mnbab_prop* prop, double timeout_s, uint64_t* ticket);

/* HBM bytes that the active requests' node slots may hold together, over all
 * networks of the context; 0 (the default) means the context's HBM budget. */
mnbab_status mnbab_set_serving_budget(mnbab_ctx* ctx, uint64_t bytes);

/* One pass of the request loop: admits queued requests in FIFO order while
 * the HBM of their reservation (n_rows + 1 + 2 * node budget slots, each slot
 * the per-neuron state, parameters and moments of a node) fits the serving
 * budget next to the active requests of every network, and their network's
 * node pool (allocated within the HBM budget) can hold the slots (a request
 * larger than the pool runs once its network is idle, one larger than the
 * serving budget once no request is active), runs one BaB step per
 * network over all of its active requests (nodes of different requests share
 * the launches, so requests that arrive while others run join the next
 * batch), and retires requests that reached a verdict, their node budget or
 * their timeout.  A request's results do not depend on the others it ran
 * with, except when its root bounds were computed in one pass with other
 * requests' roots: kernel shapes and reduction splits follow the number of
 * rows of a launch, so its bounds may then differ at rounding level (and a
 * branching choice only where two scores tie at that level). */
mnbab_status mnbab_serve_step(mnbab_ctx* ctx, int32_t max_nodes, const mnbab_adam* cfg,
                              mnbab_serve_stats* out);

/* done = 1 once the request has its final verdict. */
mnbab_status mnbab_poll(mnbab_ctx* ctx, uint64_t ticket, int32_t* done);

/* Verdict, queueing time, time to verdict (from submission, seconds) and
 * bounded nodes of a finished request. */
mnbab_status mnbab_request_result(mnbab_ctx* ctx, uint64_t ticket, int32_t* verdict, double* wait_s,
                                  double* total_s, int32_t* nodes);

/* Adversarial pre-attack (Sec. 4, experimental setup: counterexamples are
 * searched before branch-and-bound).  For every row r of the property,
 * projected gradient descent with sign steps on the margin (C f(x) + d)_r:
 *   x_{k+1} = clip(x_k - alpha sign(grad), lo, hi), alpha = 2.5 (hi - lo) / (2 steps),
 * k = 0 .. steps - 1, from each of n_starts starting points (host, [n_starts][d0],
 * clipped to the box; the caller draws them).  best_out[r] (host, n_rows) is the
 * smallest FP32 margin over all iterates of all starts; x_out (host,
 * [n_rows][d0], nullable) its first minimiser (starts in order).  A negative
 * margin is a counterexample candidate: confirm it in higher precision before
 * using it.  Any network the library loads.  Two forms compute it (chosen by
 * mnbab_set_attack_path): one kernel per (row, start) that keeps the weights
 * and the iterate in shared memory (chain networks whose weights fit), and
 * the per-layer form, which runs the bounding path's forward and
 * back-substitution kernels on scratch node slots whose bounds hold the
 * iterate's pre-activations (l = u = zhat: the DeepPoly back-substitution of
 * the objective row is then the margin's gradient, ReLU' = 1 where zhat >= 0);
 * it takes a node slot per candidate, in chunks of the batch capacity. */
mnbab_status mnbab_attack(mnbab_ctx* ctx, const mnbab_prop* prop, int32_t n_starts, int32_t steps,
                          const float* starts, float* best_out, float* x_out);

/* The pre-attack run when the property starts (Sec. 4, experimental setup:
 * counterexamples are searched before branch-and-bound): mnbab_attack's sign
 * steps (`steps` of them) from n_starts starting points, the box centre and
 * n_starts - 1 points lo + (hi - lo) u with u_{k,j} = the top 53 bits of the
 * SplitMix64 output at state seed + (i + 1) 0x9E3779B97F4A7C15,
 * i = (k - 1) d0 + j, over [0, 1).  A row whose best point has a negative
 * margin in FP64 (a forward pass on the host for the one-kernel form, on the
 * device for the per-layer form) falsifies the property before any node is
 * bounded; otherwise branch-and-bound proceeds as usual.  n_starts = 0
 * (the default) turns it off.  Call before the property starts. */
mnbab_status mnbab_set_attack(mnbab_ctx* ctx, mnbab_prop* prop, int32_t n_starts, int32_t steps,
                              uint64_t seed);

/* Form of the attack for the whole context: 0 (default) the one-kernel form
 * where the network allows it, else the per-layer form; 1 the one-kernel form
 * only (MNBAB_E_UNSUPPORTED on other networks); 2 the per-layer form always. */
mnbab_status mnbab_set_attack_path(mnbab_ctx* ctx, int32_t path);

/* ---- kernel variants and the autotuner --------------------------------- */
/* Kernel variants of an affine step (back-substitution through a layer, or
 * the forward step of the adjoint): */
#define MNBAB_VARIANT_AUTO 0   /* the built-in choice */
#define MNBAB_VARIANT_TC 1     /* tensor cores (tcgen05, 3xTF32, TMA-staged weights) */
#define MNBAB_VARIANT_IGEMM 2  /* SIMT implicit GEMM per stride class (convolutions) */
#define MNBAB_VARIANT_ROW 3    /* SIMT row-resident kernels (convolutions) */
#define MNBAB_VARIANT_PLAIN 4  /* SIMT, whole weight tensor in shared memory (convolutions) */
#define MNBAB_VARIANT_G32 5    /* SIMT GEMM, 32 x 32 tiles (FC) */
#define MNBAB_VARIANT_G64 6    /* SIMT GEMM, 64 x 64 tiles (FC) */
#define MNBAB_VARIANT_SPLITK 7 /* SIMT split-K GEMM (FC) */

typedef struct {
  int32_t node;    /* ReLU layer (1..R) that the affine edge feeds */
  int32_t edge;    /* 0, or 1 for the second edge of a residual sum */
  int32_t dir;     /* 0 forward step, 1 back-substitution */
  int32_t rows;    /* rows of the timed launches */
  int32_t variant; /* the fastest: the layer's choice for this row bucket */
  float ms[8];     /* time per launch of each variant (index = variant), -1 if it does not apply */
} mnbab_tune_rec;

/* Autotuner (a GB300 addition; the paper has no counterpart): for every affine
 * edge of the network, both directions and the row buckets <= 32, 128, 512,
 * 2048, 8192 and more (up to min(max_rows, the row scratch)), times each
 * variant that takes the layer (one untimed and three timed launches with
 * CUDA events on the context's stream, the fastest counts) with a plain store
 * epilogue, and makes the fastest the layer's choice for that bucket; larger
 * buckets take the largest one timed.  Later launches of the network use the
 * choices (except under a forced mnbab_options.gemm_path, and for
 * back-substitution rows that the built-in choice sends to the sparse-row
 * kernels).  The variants compute the same products, with sums in different
 * orders.  recs (nullable when max_recs = 0) receives up to max_recs records;
 * *n_out (nullable) their total.  Call between BaB steps. */
mnbab_status mnbab_autotune(mnbab_ctx* ctx, mnbab_net* net, int32_t max_rows,
                            mnbab_tune_rec* recs, int32_t max_recs, int32_t* n_out);

/* Fixes the variant of one affine edge and direction for every row bucket
 * (MNBAB_VARIANT_AUTO restores the built-in choice); a variant that does not
 * take the layer falls back to the built-in choice at launch. */
mnbab_status mnbab_set_variant(mnbab_ctx* ctx, mnbab_net* net, int32_t node, int32_t edge,
                               int32_t dir, int32_t variant);

/* Number of open nodes queued for the property. */
mnbab_status mnbab_queue_size(const mnbab_ctx* ctx, const mnbab_prop* prop, int32_t* n_out);

/* ---- allocation-free variant ----------------------------------------------- */
/* Size of the device scratch array that mnbab_deeppoly_fc_noalloc uses. */
#define MNBAB_NOALLOC_SCRATCH_BYTES (16u << 20)

/* DeepPoly lower bounds of query rows of a fully connected ReLU network, for
 * callers that cannot allocate device memory (code running inside another
 * framework's memory pool or allocator hooks, hosts whose device memory is
 * partitioned up front).  The paper has no counterpart: this is a deployment variant of
 * the back-substitution sweep of mnbab_deeppoly_batch, with every scratch
 * buffer taken from a static device array of MNBAB_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that each GPU loading the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Arguments (all arrays are DEVICE pointers owned by the caller, FP32,
 * row-major, except dims, W and b, which are host arrays):
 *   n_affine    affine layers in the chain affine, ReLU, ..., affine (>= 1);
 *   dims        host [n_affine]: dims[0] input width, dims[i] width of the
 *               ReLU layer after hidden affine layer i (i = 1..n_affine-1);
 *   W, b        host arrays of n_affine - 1 device pointers: hidden layer i
 *               has W[i-1] [dims[i]][dims[i-1]] and b[i-1] [dims[i]];
 *   x_lo, x_hi  input box [dims[0]];
 *   l, u        pre-activation bounds of the ReLU layers, concatenated
 *               [dims[1] + ... + dims[n_affine-1]];
 *   Wf, bf      the query rows on the last ReLU layer's output (a property
 *               folded into the last affine layer): Wf [n_rows][dims[n_affine-1]]
 *               (dims[0] when n_affine == 1), bf [n_rows];
 *   lb_out      [n_rows] lower bounds, written on `stream`;
 *   stream      cudaStream_t (NULL = the legacy default stream);
 *   err, err_len  optional buffer for a message.
 * Returns MNBAB_E_BUDGET (with a message) when n_rows rows need more scratch
 * than the static array holds (about 4 * n_rows * (2 * max_width + 20)
 * bytes); split the rows over several calls then.  The first call on a device
 * looks up the array's device address with that device current (done once per
 * device); make that first call before any stream capture.  Each device has
 * its own copy of the array; every call on a device uses that copy, which keeps
 * the last call's contents.  Two calls whose GPU work overlaps on one device
 * (for example on two streams) race on it: issue them one after another on one
 * stream. */
mnbab_status mnbab_deeppoly_fc_noalloc(int32_t n_affine, const int32_t* dims,
                                       const float* const* W, const float* const* b,
                                       const float* x_lo, const float* x_hi, const float* l,
                                       const float* u, const float* Wf, const float* bf,
                                       int32_t n_rows, float* lb_out, void* stream, char* err,
                                       size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* MNBAB_H */
