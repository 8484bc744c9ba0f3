"""Shared set-up for the GPU-vs-oracle parity tests."""
from __future__ import annotations

import numpy as np
import torch

import synth
from oracle import bab, core, mnc
from oracle.core import DT

TOL = 1e-4  # bound tolerance: |gpu - oracle| <= TOL * (1 + |oracle|)


def close(g, o, tol=TOL):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    both_inf = np.isinf(g) & np.isinf(o) & (np.sign(g) == np.sign(o))
    ok = both_inf | (np.abs(g - o) <= tol * (1.0 + np.abs(o)))
    return ok


def f32(t):
    return torch.as_tensor(np.asarray(t, np.float32).astype(np.float64), dtype=DT)


def fc_case(seed, dims, eps, with_mnc=False, x_seed=None):
    layers = synth.tiny_fc_net(seed, list(dims))
    rng = np.random.default_rng(seed + 100 if x_seed is None else x_seed)
    x0 = rng.uniform(0.2, 0.8, dims[0]).astype(np.float32)
    y = synth.net_forward(layers, x0)
    C, d = synth.property_rows(int(np.argmax(y)), dims[-1])
    lo, hi = synth.input_box(x0, eps)
    prep = bab.prepare(layers, C, d, lo, hi, mnc.mnc_fn() if with_mnc else None)
    return layers, C, d, lo, hi, prep


def conv_spec(seed):
    """Small conv chain with ragged sizes (stride 2, padding, odd widths)."""
    return dict(seed=seed, in_shape=(2, 11, 11),
                layers=[("conv", 5, 3, 2, 1), ("relu",), ("conv", 7, 4, 2, 1), ("relu",),
                        ("fc", 13), ("relu",), ("fc", 4)])


def conv_small_spec(seed):
    """The conv_small_28 layer pattern: 1x28x28 -> conv16 4x4 s2 -> conv32 4x4 s2
    -> FC100 -> FC10."""
    return dict(seed=seed, in_shape=(1, 28, 28),
                layers=[("conv", 16, 4, 2, 0), ("relu",), ("conv", 32, 4, 2, 0), ("relu",),
                        ("fc", 100), ("relu",), ("fc", 10)])


def convbig_spec(seed):
    """The conv-big layer pattern (3x3 s1 p1, 4x4 s2 p1; 32 and 64 channels) on
    a 3x12x12 input: the 64 -> 64 4x4 layer's weights (256 KB) exceed shared
    memory, so the kernels must stage them in channel slices."""
    return dict(seed=seed, in_shape=(3, 12, 12),
                layers=[("conv", 32, 3, 1, 1), ("relu",), ("conv", 32, 4, 2, 1), ("relu",),
                        ("conv", 64, 3, 1, 1), ("relu",), ("conv", 64, 4, 2, 1), ("relu",),
                        ("fc", 50), ("relu",), ("fc", 10)])


def resnet_spec(seed):
    """Two residual blocks (ResAdd of a 3x3 main branch and a 1x1 shortcut, the
    second with stride 2) on a 3x10x10 input."""
    return dict(seed=seed, in_shape=(3, 10, 10),
                layers=[("conv", 8, 3, 1, 1), ("relu",),
                        ("conv", 8, 3, 1, 1, 1), ("relu",), ("conv", 8, 3, 1, 1, 3, 0.5),
                        ("conv", 8, 1, 1, 0, 1), ("add", 4, 5), ("relu",),
                        ("conv", 16, 3, 2, 1, 7), ("relu",), ("conv", 16, 3, 1, 1, 9, 0.5),
                        ("conv", 16, 1, 2, 0, 7), ("add", 10, 11), ("relu",),
                        ("fc", 20), ("relu",), ("fc", 5)])


def conv_case(seed, eps, spec_fn=None):
    spec = (spec_fn or conv_spec)(seed)
    layers = synth.make_network(spec)
    x0 = synth.make_image(seed + 7, spec["in_shape"]).reshape(-1)
    y = synth.net_forward(layers, x0)
    C, d = synth.property_rows(int(np.argmax(y)), y.shape[0])
    lo, hi = synth.input_box(x0, eps)
    prep = bab.prepare(layers, C, d, lo, hi)
    return layers, C, d, lo, hi, prep


def gpu_property(ctx, layers, lo, hi, C, d, mncs=None, net=None):
    """A property on `net` (a new copy of `layers` when None) with its
    multi-neuron constraints."""
    if net is None:
        net = ctx.load_network(layers)
    prop = ctx.set_property(net, lo, hi, C, d)
    if mncs:
        for i in sorted(mncs):
            m = mncs[i]
            ctx.set_mnc(prop, i, m.idx, m.P, m.Ph, m.p)
    return net, prop


def random_node(prep, rng, n_splits, row=0, gamma_scale=0.2):
    """Oracle node with random splits (clamped, not yet re-bounded) and random
    parameters, all rounded to float32 so both sides start from the same values."""
    net, lo, hi, l, u, S, m, dense = prep
    node = bab.root_node(net, row, l, u, S, m)
    cands = [(i, j) for i in l for j in range(l[i].numel()) if l[i][j] < 0 < u[i][j]]
    k = min(n_splits, len(cands))
    picks = [cands[t] for t in rng.choice(len(cands), size=k, replace=False)] if k else []
    for (i, j) in picks:
        sgn = int(rng.choice([1, -1]))
        node.S[i][j] = sgn
        if sgn == 1:
            node.u[i][j] = min(float(node.u[i][j]), 0.0)
        else:
            node.l[i][j] = max(float(node.l[i][j]), 0.0)
    node.split_layer = max([p[0] for p in picks], default=net.R) if picks else net.R
    if picks and rng.random() < 0.5:
        node.split_layer = min(p[0] for p in picks)
    for i in l:
        node.l[i] = f32(node.l[i].numpy())
        node.u[i] = f32(node.u[i].numpy())
        node.alpha[i] = f32(rng.uniform(0, 1, l[i].numel()))
        node.beta[i] = f32(rng.uniform(0, 1, l[i].numel()) * (node.S[i].numpy() != 0))
        node.gamma[i] = f32(rng.uniform(0, gamma_scale, node.gamma[i].numel()))
    return node


def to_params(node, R):
    from paper_2205_00263_gb300 import NodeParams
    ks = range(1, R + 1)
    cat = lambda D, dt: np.concatenate([np.asarray(D[i].numpy(), dt) for i in ks])
    gam = [node.gamma[i].numpy() for i in ks if node.gamma[i].numel()]
    return NodeParams(node.split_layer, R, cat(node.l, np.float32), cat(node.u, np.float32),
                      cat(node.S, np.int8), cat(node.alpha, np.float32), cat(node.beta, np.float32),
                      np.concatenate(gam).astype(np.float32) if gam else np.zeros(0, np.float32))


def concat(D, R):
    return np.concatenate([D[i].numpy() for i in range(1, R + 1)])


def run_gpu_bab(ctx, props, max_nodes, steps=20):
    for _ in range(10000):
        st = ctx.bab_step(props, max_nodes=max_nodes, steps=steps)
        if st["nodes_bounded"] == 0:
            break


ACS_TIE = 1e-5  # branching ties: scores within this relative band of the maximum
# A node's optimised bound counts as not determined at FP32 precision when
# rounding-level perturbations of its gradients (core.noise_sensitivity) move
# it by more than this fraction of the tolerance band.
COND = 0.1


def _acs_tie(o, layer, neuron):
    """Whether the oracle's own scores at node o put (layer, neuron) within
    ACS_TIE (relative) of their maximum."""
    sc = o.scores
    if not sc or layer not in sc or neuron >= sc[layer].numel():
        return False
    mx = max(float(v.max()) for v in sc.values() if v.numel())
    s = float(sc[layer][neuron])
    return s >= mx - ACS_TIE * abs(mx)


def compare_trace(gtr, ores, max_cmp=None, recompute=None, sensitivity=None):
    """Node-by-node agreement of a GPU BaB trace with the oracle's
    (bab.verify(record=True)).

    Every compared node has the same FIFO number, row, DeepPoly bound (within
    TOL), node bound (within TOL), verdict and split.  The comparison of the
    property ends (its trees may part from there on) only at:

    * "margin": the oracle's node bound lies inside the band
      |lb| <= TOL (1 + |lb|), so the verdict may differ;
    * "tie": the splits differ and the oracle's own branching scores put the
      GPU's choice within ACS_TIE (relative) of their maximum (checked here);
    * "inherited": the GPU, given the oracle's exact starting state of the node
      (``recompute(o)`` -> (bound, split) on the GPU), reproduces the oracle's
      bound within TOL and its split (or a tie): the GPU's own node differs
      only through the FP32 parameters it inherited from its parent;
    * "conditioning": otherwise, the oracle's own probe (``sensitivity(o)``,
      core.noise_sensitivity at the node's starting state) shows that
      rounding-level gradient perturbations move the node's optimised bound by
      more than COND x TOL: projected Adam amplifies rounding there, so the
      bound is not determined at FP32 precision.

    At the last two the GPU node must still be valid: node bound no lower than
    its own DeepPoly bound, a FALSIFIED verdict only with f(x*) < 0.
    Returns (nodes compared, reason the comparison ended or None).
    """
    n = min(len(gtr), len(ores.nodes))
    if max_cmp is not None:
        n = min(n, max_cmp)
    for k in range(n):
        g, o = gtr[k], ores.nodes[k]
        assert g["seq"] == o.node_id and g["row"] == o.row, (k, g, o)
        dp_band = TOL * (1 + abs(o.lb_dp))
        assert abs(g["lb_deeppoly"] - o.lb_dp) <= dp_band, ("DeepPoly bound", k, g, o.lb_dp)
        band = TOL * (1 + abs(o.lb))
        gs = (g["split_layer"], g["split_neuron"]) if g["split_layer"] > 0 else None
        if o.leaf:
            # a fully split leaf: the oracle's exact LP minimum, the GPU's
            # certified dual bound below it; the verdicts agree
            assert g["leaf"] == 1 and g["lb"] <= o.lb + band, (k, g, o.lb)
            if abs(o.lb) <= band:
                return k, "margin"
            assert g["verdict"] == o.verdict, (k, g, o.verdict)
            continue
        bound_ok = abs(g["lb"] - o.lb) <= band
        if bound_ok and abs(o.lb) <= band:
            return k, "margin"
        split_ok = gs == o.split or (gs is not None and o.split is not None
                                     and _acs_tie(o, gs[0], gs[1]))
        if bound_ok and g["verdict"] == o.verdict and split_ok:
            if gs != o.split:
                return k, "tie"
            continue
        # the GPU's node differs from the oracle's: explain it or fail
        assert g["lb"] >= g["lb_deeppoly"] - 1e-6 * (1 + abs(g["lb"])), (k, g)
        if g["verdict"] == -1:
            assert g["f_xstar"] < 0, (k, g)
        assert recompute is not None and o.start is not None, (
            "node differs", k, g["lb"], o.lb, gs, o.split)
        r_lb, r_split = recompute(o)
        same = abs(r_lb - o.lb) <= band and (
            o.split is None or r_split == o.split or _acs_tie(o, r_split[0], r_split[1]))
        if same:
            return k, "inherited"
        sens = sensitivity(o) if sensitivity is not None else 0.0
        assert sens > COND * band, ("node differs from the oracle's own state", k, r_lb, o.lb,
                                    r_split, o.split, sens)
        return k, "conditioning"
    return n, None


def oracle_sensitivity(prep, hp=None):
    """sensitivity(o) for compare_trace from the oracle's prepared problem."""
    net, lo_t, hi_t, l, u, S, m, dense = prep
    hp = hp or core.AdamHP()
    return lambda o: core.noise_sensitivity(net, o.start, dense, lo_t, hi_t, hp)


def gpu_recompute(ctx, prop, R, steps=20, adam=None):
    """recompute(o) for compare_trace: the node bounded on the GPU from the
    oracle's starting state o.start (re-bounding, DeepPoly pass, steps Adam
    steps, ACS at the final parameters) -> (node bound, (layer, neuron))."""
    adam = adam or {}

    def f(o):
        gid = ctx.node_root(prop, o.start.row)
        try:
            ctx.import_params(gid, to_params(o.start, R))
            ctx.bound_batch([gid])
            dp = float(ctx.deeppoly_batch([gid])[0])
            best = dp
            if not dp > 0:
                best = max(dp, float(ctx.optimize([gid], steps=steps, **adam)[0]))
            lay, neu, _ = ctx.score_branches([gid])
            return best, (int(lay[0]), int(neu[0]))
        finally:
            ctx.node_free(gid)
    return f


def verdicts_consistent(v_gpu, v_oracle):
    """Both sides are sound: one may be UNKNOWN (budget, parted trees), but a
    VERIFIED property is never FALSIFIED by the other."""
    return {v_gpu, v_oracle} != {1, -1}


# --------------------------------------------------------------------------
# oracle jobs for a spawn process pool (started before or beside GPU work:
# a pool forked after the first CUDA call would hang)
# --------------------------------------------------------------------------
def oracle_root_bounds_job(cfg, prop=0, threads=4):
    """FP64 DeepPoly root bounds of every ReLU layer of one property of a
    config's full-size network: {layer: (l, u)} as numpy arrays."""
    torch.set_num_threads(threads)
    layers = synth.make_network(cfg)
    pr = synth.make_properties(cfg, layers, n=prop + 1, eps=synth.load_eps(cfg))[prop]
    net = core.fold_property(core.load_net(layers), pr.C, pr.d)
    l, u, _ = core.root_bounds(net, torch.as_tensor(pr.lo, dtype=DT),
                               torch.as_tensor(pr.hi, dtype=DT))
    return {i: (l[i].numpy(), u[i].numpy()) for i in l}


def oracle_verify_job(cfg, prop, budget, with_mnc, threads=2):
    """(verdict, bounded nodes) of the oracle's BaB on one property."""
    torch.set_num_threads(threads)
    layers = synth.make_network(cfg)
    pr = synth.make_properties(cfg, layers, n=prop + 1, eps=synth.load_eps(cfg))[prop]
    r = bab.verify(layers, pr.C, pr.d, pr.lo, pr.hi, max_nodes=budget,
                   mnc_fn=mnc.mnc_fn() if with_mnc else None)
    return r.verdict, len(r.nodes)


def spawn_pool(n):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(n)
