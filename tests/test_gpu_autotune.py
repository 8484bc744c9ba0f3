"""Kernel variants of the affine steps and the autotuner (mnbab_autotune,
mnbab_set_variant).  Every variant, forced on every edge and direction of a
network, must give the oracle's bounds and gradients at fixed parameters (so
each kernel of the back-substitution and of the adjoint's forward pass is
checked on its own, not only the one the built-in choice picks); the
autotuner must keep, per edge, direction and row bucket, the fastest variant
it timed, and bounds after tuning must still match the oracle."""
import numpy as np
import pytest

from helpers import (close, concat, conv_case, convbig_spec, fc_case, gpu_property, random_node,
                     resnet_spec, to_params)
from oracle import core

pytestmark = pytest.mark.gpu

VARIANTS = ("tc", "igemm", "row", "plain", "g32", "g64", "splitk")


@pytest.fixture(scope="module")
def Context():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context as Ctx
    return Ctx


def _case(case):
    if case == "fc_mnc":
        return fc_case(3, (37, 53, 29, 7), 0.12, with_mnc=True)
    if case == "conv":
        return conv_case(4, 0.08)
    if case == "convbig":
        return conv_case(5, 0.01, convbig_spec)
    return conv_case(6, 0.02, resnet_spec)


def _edges(net):
    return [(t, k) for t in range(1, net.R + 1) for k in range(len(net.edges[t]))]


def _assert(got, ref, what):
    ok = close(np.atleast_1d(got), np.atleast_1d(ref))
    assert ok.all(), (what, np.max(np.abs(np.atleast_1d(got) - np.atleast_1d(ref))))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", ["fc_mnc", "conv", "convbig", "resnet"])
def test_every_variant_matches_oracle(Context, case, variant):
    """All edges and both directions forced to one variant (layers it does not
    take use the built-in choice): re-bounded intermediate bounds, the
    objective bound and its gradient match the oracle at fixed parameters."""
    layers, C, d, lo, hi, prep = _case(case)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    E = sum(v.idx.shape[0] for v in m.values()) if m else 0
    SD = sum(l[i].numel() for i in l)
    rng = np.random.default_rng(17)
    with Context(node_capacity=128, max_mnc_rows=max(E, 1)) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d, m)
        for t, k in _edges(net):
            for direction in (0, 1):
                ctx.set_variant(gnet, t, k, direction, variant)
        onodes, gids = [], []
        for q in range(8):
            on = random_node(prep, rng, n_splits=q % 4, row=q % C.shape[0])
            gid = ctx.node_root(prop, on.row)
            ctx.import_params(gid, to_params(on, net.R))
            onodes.append(on)
            gids.append(gid)
        lb, _ = ctx.bound_batch(gids)
        for q, (on, gid) in enumerate(zip(onodes, gids)):
            core.rebound_node(net, on, lo_t, hi_t)
            p = ctx.export_params(gid)
            _assert(p.l, concat(on.l, net.R), f"node {q} l")
            _assert(p.u, concat(on.u, net.R), f"node {q} u")
            ref, _, _ = core.final_bound(net, on, on.alpha, on.beta, on.gamma, dense, lo_t, hi_t)
            _assert(lb[q], float(ref), f"node {q} lb")
        for on in onodes:
            on.split_layer = net.R
        lbg, ga, gb, gg = ctx.bound_grad(gids, SD, E)
        for q, on in enumerate(onodes):
            ref, _, oa, ob, og = core.bound_and_grad(net, on, on.alpha, on.beta, on.gamma,
                                                     dense, lo_t, hi_t)
            _assert(lbg[q], float(ref), f"node {q} lb (gradient call)")
            for name, g, o in (("alpha", ga[q], concat(oa, net.R)),
                               ("beta", gb[q], concat(ob, net.R))):
                assert np.abs(g - o).max() <= 1e-4 * (1 + np.abs(o).max()), (name, q)


def test_autotune_keeps_the_fastest_and_bounds_match(Context):
    """conv_big-shaped net: one record per edge, direction and row bucket up to
    512 rows; each record's choice is its fastest timed variant; bounds after
    tuning match the oracle."""
    layers, C, d, lo, hi, prep = _case("convbig")
    net, lo_t, hi_t, l, u, S, m, dense = prep
    rng = np.random.default_rng(19)
    with Context(node_capacity=128) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d)
        recs = ctx.autotune(gnet, max_rows=512)
        n_edges = len(_edges(net))
        assert len(recs) == n_edges * 2 * 3     # buckets 32, 128, 512
        for r in recs:
            assert r["ms"], r
            assert r["variant"] == min(r["ms"], key=r["ms"].get), r
            assert all(v > 0 for v in r["ms"].values())
        onodes, gids = [], []
        for q in range(8):
            on = random_node(prep, rng, n_splits=q % 4, row=q % C.shape[0])
            gid = ctx.node_root(prop, on.row)
            ctx.import_params(gid, to_params(on, net.R))
            onodes.append(on)
            gids.append(gid)
        lb, _ = ctx.bound_batch(gids)
        for q, (on, gid) in enumerate(zip(onodes, gids)):
            core.rebound_node(net, on, lo_t, hi_t)
            p = ctx.export_params(gid)
            _assert(p.l, concat(on.l, net.R), f"node {q} l")
            _assert(p.u, concat(on.u, net.R), f"node {q} u")
            ref, _, _ = core.final_bound(net, on, on.alpha, on.beta, on.gamma, dense, lo_t, hi_t)
            _assert(lb[q], float(ref), f"node {q} lb")
