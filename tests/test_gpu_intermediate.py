"""GPU parity of the optimised intermediate bounds (Sec. 3.1, parameter
sharing: one set per layer and side, shared by the layer's neurons) against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from helpers import (TOL, close, compare_trace, concat, conv_case, fc_case, gpu_property,
                     gpu_recompute, oracle_sensitivity, verdicts_consistent,
                     random_node, run_gpu_bab, to_params)
from oracle import bab, core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context as Ctx
    return Ctx


def _case(kind):
    if kind == "fc":
        return fc_case(21, (37, 53, 41, 29, 7), 0.1)
    return conv_case(5, 0.05)


@pytest.mark.parametrize("row_chunk", [0, 38])
@pytest.mark.parametrize("kind", ["fc", "conv"])
def test_optimized_intermediate_bounds_match_oracle(Context, kind, row_chunk):
    """Root and split nodes (float32 start values shared by both sides): after
    20 Adam steps per set, every neuron's bounds match the oracle's within
    1e-4 (1 + |b|), the row counts agree exactly, and the nodes' own
    parameters are left as they were.  With row_chunk = 38 the rows run in
    chunks of 38, so sets span chunk boundaries and the last chunk is ragged."""
    layers, C, d, lo, hi, prep = _case(kind)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    R = net.R
    assert R >= 3
    rng = np.random.default_rng(21)
    with Context(node_capacity=64, row_chunk=row_chunk) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d)
        onodes, gids = [], []
        for k in range(4):
            on = random_node(prep, rng, n_splits=k, row=k % C.shape[0], gamma_scale=0.0)
            on.split_layer = R
            gid = ctx.node_root(prop, on.row)
            ctx.import_params(gid, to_params(on, R))
            onodes.append(on)
            gids.append(gid)
        before = [ctx.export_params(g) for g in gids]
        rows = ctx.optimize_intermediate(gids, first_layer=2, steps=20)
        ref_rows = 0
        for k, on in enumerate(onodes):
            ref_rows += core.optimize_intermediate(net, on, lo_t, hi_t, core.AdamHP())
            got = ctx.export_params(gids[k])
            for name, g_, o_ in (("l", got.l, concat(on.l, R)), ("u", got.u, concat(on.u, R))):
                ok = close(g_, o_)
                assert ok.all(), (f"node {k} {name}: {int((~ok).sum())} of {ok.size} off, worst "
                                  f"{np.max(np.abs(g_ - o_) / (1 + np.abs(o_)))}")
            assert np.array_equal(got.alpha, before[k].alpha)
            assert np.array_equal(got.beta, before[k].beta)
            assert np.all(got.l >= before[k].l) and np.all(got.u <= before[k].u)
        assert rows == ref_rows


def test_optimized_intermediate_bounds_sound_on_samples(Context):
    """Root node of the conv case: the GPU's optimised bounds contain every
    pre-activation of 10^4 sampled inputs, and tighten some neuron."""
    layers, C, d, lo, hi, prep = _case("conv")
    net = prep[0]
    with Context(node_capacity=64) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d)
        gid = ctx.node_root(prop, 0)
        before = ctx.export_params(gid)
        ctx.optimize_intermediate([gid], steps=20)
        got = ctx.export_params(gid)
    gain = float(np.sum(got.l - before.l) + np.sum(before.u - got.u))
    assert gain > 1e-4
    import torch
    X = np.random.default_rng(3).uniform(lo, hi, size=(10000, lo.size))
    h = torch.as_tensor(X, dtype=torch.float64)
    off = 0
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h).numpy()
        di = zh.shape[1]
        li, ui = got.l[off:off + di], got.u[off:off + di]
        slack = TOL * (1.0 + np.abs(zh))
        assert np.all(zh >= li - slack), f"layer {i}: lower bound above a sample"
        assert np.all(zh <= ui + slack), f"layer {i}: upper bound below a sample"
        h = torch.clamp(torch.as_tensor(zh), min=0)
        off += di


@pytest.mark.parametrize("row_chunk", [0, 40])
def test_optimized_intermediate_with_constraints_match_oracle(Context, row_chunk):
    """Properties with multi-neuron constraints: each shared set carries
    gamma_i for the constraints of the layers below t (Sec. 3.1).  Under the
    eps_rel option (Adam's denominator relative to the largest gradient
    component, so rounding-level gradients of tight constraints take no step)
    the bounds match the oracle's within 1e-4 (1 + |b|) and the row counts
    agree; the nodes' own parameters are left as they were.  row_chunk = 40
    caps the sets bounded together."""
    layers, C, d, lo, hi, prep = fc_case(8, (37, 53, 29, 7), 0.12, with_mnc=True)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    R = net.R
    E = sum(v.idx.shape[0] for v in m.values())
    assert E > 0
    hp = core.AdamHP(eps_rel=1e-3)
    rng = np.random.default_rng(8)
    with Context(node_capacity=64, max_mnc_rows=E, row_chunk=row_chunk) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d, m)
        onodes, gids = [], []
        for k in range(3):
            on = random_node(prep, rng, n_splits=k, row=k % C.shape[0], gamma_scale=0.2)
            on.split_layer = R
            gid = ctx.node_root(prop, on.row)
            ctx.import_params(gid, to_params(on, R))
            onodes.append(on)
            gids.append(gid)
        before = [ctx.export_params(g) for g in gids]
        rows = ctx.optimize_intermediate(gids, first_layer=2, steps=20, eps_rel=1e-3)
        ref_rows = 0
        for k, on in enumerate(onodes):
            ref_rows += core.optimize_intermediate(net, on, lo_t, hi_t, hp, dense_mnc=dense)
            got = ctx.export_params(gids[k])
            for name, g_, o_ in (("l", got.l, concat(on.l, R)), ("u", got.u, concat(on.u, R))):
                ok = close(g_, o_)
                assert ok.all(), (f"node {k} {name}: {int((~ok).sum())} of {ok.size} off, worst "
                                  f"{np.max(np.abs(g_ - o_) / (1 + np.abs(o_)))}")
            assert np.array_equal(got.alpha, before[k].alpha)
            assert np.array_equal(got.gamma, before[k].gamma)
            assert np.all(got.l >= before[k].l) and np.all(got.u <= before[k].u)
        assert rows == ref_rows


def test_optimized_intermediate_with_constraints_sound_standard_adam(Context):
    """Standard Adam with gamma in the sets: the root's optimised bounds contain
    every pre-activation of 10^4 sampled inputs and are never looser than
    DeepPoly.  Per-bound parity is not asked for here (standard Adam's steps
    on rounding-level gradients of tight constraints differ between FP32 and
    FP64); the summed tightening over all neurons agrees with the oracle's
    within 2 %."""
    layers, C, d, lo, hi, prep = fc_case(8, (37, 53, 29, 7), 0.12, with_mnc=True)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    E = sum(v.idx.shape[0] for v in m.values())
    with Context(node_capacity=64, max_mnc_rows=E) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d, m)
        gid = ctx.node_root(prop, 0)
        before = ctx.export_params(gid)
        ctx.optimize_intermediate([gid], steps=20)
        got = ctx.export_params(gid)
    assert np.all(got.l >= before.l) and np.all(got.u <= before.u)
    gain = float(np.sum(got.l - before.l) + np.sum(before.u - got.u))
    assert gain > 1e-4
    import torch
    X = np.random.default_rng(3).uniform(lo, hi, size=(10000, lo.size))
    h = torch.as_tensor(X, dtype=torch.float64)
    off = 0
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h).numpy()
        di = zh.shape[1]
        li, ui = got.l[off:off + di], got.u[off:off + di]
        slack = TOL * (1.0 + np.abs(zh))
        assert np.all(zh >= li - slack), f"layer {i}: lower bound above a sample"
        assert np.all(zh <= ui + slack), f"layer {i}: upper bound below a sample"
        h = torch.clamp(torch.as_tensor(zh), min=0)
        off += di
    root = bab.root_node(net, 0, l, u, S, m)
    core.optimize_intermediate(net, root, lo_t, hi_t, core.AdamHP(), dense_mnc=dense)
    ogain = sum(float((root.l[i] - l[i]).sum() + (u[i] - root.u[i]).sum()) for i in l)
    assert abs(gain - ogain) <= 2e-2 * (1 + abs(ogain)), (gain, ogain)


def test_root_intermediate_steps_in_bab_match_oracle(Context):
    """Properties set to optimise their root's intermediate bounds: the GPU's
    root bounds match the oracle's optimised root bounds, and the BaB trace
    matches the oracle's verify(inter_steps=20) node by node, under the same
    trace rules as the plain BaB parity test."""
    layers = synth.make_network(0)
    eps = synth.load_eps(0)
    prs = synth.make_properties(0, layers, n=2, eps=eps, start=50)
    budget = 16
    matched = 0
    with Context(node_capacity=4096) as ctx:
        for pr in prs:
            prep = bab.prepare(layers, pr.C, pr.d, pr.lo, pr.hi)
            net, lo_t, hi_t, l, u, S, m, dense = prep
            root = bab.root_node(net, 0, l, u, S, None)
            core.optimize_intermediate(net, root, lo_t, hi_t, core.AdamHP())
            gnet, prop = gpu_property(ctx, layers, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_intermediate_steps(prop, 20)
            ctx.set_budget(prop, budget)
            for i in range(1, net.R + 1):
                gl, gu = ctx.root_bounds(prop, i)
                assert close(gl, root.l[i].numpy()).all(), f"layer {i} lower root bounds"
                assert close(gu, root.u[i].numpy()).all(), f"layer {i} upper root bounds"
            ores = bab.verify(layers, pr.C, pr.d, pr.lo, pr.hi, max_nodes=budget, prepared=prep,
                              inter_steps=20, record=True)
            run_gpu_bab(ctx, [prop], max_nodes=1)
            k, why = compare_trace(ctx.trace(prop), ores,
                                   recompute=gpu_recompute(ctx, prop, net.R),
                                   sensitivity=oracle_sensitivity(prep))
            matched += k
            v, _, _ = ctx.verdict(prop)
            if why is None and k == len(ores.nodes):
                assert v == ores.verdict
            assert verdicts_consistent(v, ores.verdict)
        with pytest.raises(Exception):
            ctx.set_intermediate_steps(prop, 5)   # already started
    assert matched >= 16


def test_small_pool_refuses_intermediate_steps(Context):
    """A batch capacity of 1 (node_capacity 2) cannot hold a node's two
    parameter sets: the root option is refused with an error (it used to loop),
    and a node listed twice in one call is refused as well."""
    from paper_2205_00263_gb300 import MnbabError
    layers, C, d, lo, hi, prep = fc_case(31, (12, 9, 8, 4), 0.1)
    with Context(node_capacity=2) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d)
        with pytest.raises(MnbabError):
            ctx.set_intermediate_steps(prop, 5)
    with Context(node_capacity=64) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d)
        n0 = ctx.node_root(prop, 0)
        with pytest.raises(MnbabError):
            ctx.optimize_intermediate([n0, n0], steps=2)
