"""Request loop (continuous batching): a request's verdict and BaB trace are the
same whether it runs alone or mixed with requests of other properties and
networks that arrive while it runs; admission waits for node-pool room;
timeouts end a request with UNKNOWN."""
import numpy as np
import pytest
import torch

import synth
from helpers import conv_case, resnet_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    return Context


def _drain(ctx, tickets, max_nodes=512, steps=5, limit=500):
    for _ in range(limit):
        if all(ctx.poll(t) for t in tickets):
            return
        ctx.serve_step(max_nodes, steps=steps)
    raise AssertionError("requests did not finish")


def _key(tr):
    return [(r["seq"], r["row"], r["verdict"], r["split_layer"], r["split_neuron"], r["lb"])
            for r in tr]


def test_results_alone_equal_results_in_the_mix(Context):
    layers = synth.make_network(1)
    eps = synth.load_eps(1)
    prs = synth.make_properties(1, layers, n=5, eps=eps)
    rl, rC, rd, rlo, rhi, _ = conv_case(11, 0.03, resnet_spec)
    rspec = synth.make_network(resnet_spec(11))
    alone = []
    for pr in prs:
        with Context(node_capacity=2048) as ctx:
            net = ctx.load_network(layers)
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_budget(p, 24)
            t = ctx.submit(p)
            _drain(ctx, [t])
            alone.append((ctx.request_result(t)["verdict"], _key(ctx.trace(p))))
    with Context(node_capacity=2048) as ctx:
        res_alone = ctx.load_network(rl)
        rp = ctx.set_property(res_alone, rlo, rhi, rC, rd)
        ctx.set_budget(rp, 12)
        rt = ctx.submit(rp)
        _drain(ctx, [rt])
        r_alone = (ctx.request_result(rt)["verdict"], _key(ctx.trace(rp)))
    with Context(node_capacity=2048) as ctx:
        net = ctx.load_network(layers)
        rnet = ctx.load_network(rl)
        tickets, props = [], []
        for k, pr in enumerate(prs):
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_budget(p, 24)
            tickets.append(ctx.submit(p))
            props.append(p)
            if k == 2:   # a request of another network arrives mid-way
                rp = ctx.set_property(rnet, rlo, rhi, rC, rd)
                ctx.set_budget(rp, 12)
                rt = ctx.submit(rp)
            ctx.serve_step(512, steps=5)   # arrivals while earlier requests run
        _drain(ctx, tickets + [rt])
        for t, p, (v, key) in zip(tickets, props, alone):
            assert ctx.request_result(t)["verdict"] == v
            assert _key(ctx.trace(p)) == key
        assert (ctx.request_result(rt)["verdict"], _key(ctx.trace(rp))) == r_alone


def test_admission_waits_for_pool_room_and_timeouts(Context):
    layers = synth.make_network(1)
    eps = synth.load_eps(1)
    prs = synth.make_properties(1, layers, n=4, eps=eps, start=50)
    # room for one request of budget 40 at a time (reservation 9 + 1 + 80 slots)
    with Context(node_capacity=150) as ctx:
        net = ctx.load_network(layers)
        tickets = []
        for pr in prs:
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_budget(p, 40)
            tickets.append(ctx.submit(p))
        st = ctx.serve_step(512, steps=5)
        assert st["admitted"] == 1 and st["queued"] == 3
        _drain(ctx, tickets, limit=2000)
        waits = [ctx.request_result(t)["wait_s"] for t in tickets]
        assert waits[-1] > waits[0]
        # a request that times out ends UNKNOWN
        pr = synth.make_properties(1, layers, n=1, eps=eps * 3, start=90)[0]
        p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
        ctx.set_budget(p, 40)
        t = ctx.submit(p, timeout_s=1e-9)
        _drain(ctx, [t])
        r = ctx.request_result(t)
        assert r["verdict"] in (0, -1)


def test_admission_by_hbm_bytes_across_networks(Context):
    """Admission by HBM: the active requests' node slots (per-neuron state,
    parameters and moments of each reserved node) must fit the serving budget
    together, over all networks.  With room for about one and a half requests,
    one runs at a time (a request of another network waits as well); the
    verdicts and tree shapes equal those of the unconstrained loop and the
    bounds agree within the tolerance."""
    layers = synth.make_network(1)
    eps = synth.load_eps(1)
    prs = synth.make_properties(1, layers, n=3, eps=eps, start=60)
    rl, rC, rd, rlo, rhi, _ = conv_case(11, 0.03, resnet_spec)

    def run(budget_bytes):
        with Context(node_capacity=2048) as ctx:
            net = ctx.load_network(layers)
            rnet = ctx.load_network(rl)
            if budget_bytes:
                ctx.set_serving_budget(budget_bytes)
            tickets, props = [], []
            for pr in prs:
                p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
                ctx.set_budget(p, 24)
                tickets.append(ctx.submit(p))
                props.append(p)
            rp = ctx.set_property(rnet, rlo, rhi, rC, rd)
            ctx.set_budget(rp, 12)
            tickets.append(ctx.submit(rp))
            props.append(rp)
            first = ctx.serve_step(512, steps=5)
            peak = first["reserved_bytes"]
            for _ in range(2000):
                if all(ctx.poll(t) for t in tickets):
                    break
                st = ctx.serve_step(512, steps=5)
                peak = max(peak, st["reserved_bytes"])
            assert all(ctx.poll(t) for t in tickets)
            assert ctx.serve_step(512, steps=5)["reserved_bytes"] == 0
            res = [(ctx.request_result(t)["verdict"], _key(ctx.trace(p)))
                   for t, p in zip(tickets, props)]
            return first, peak, res

    first, peak, res_free = run(0)
    assert first["admitted"] == 4 and first["queued"] == 0
    # one request of the conv net: 9 rows + 1 + 2 x 24 slots of
    # SD = 2704 + 800 + 100 neurons x (8 floats + 1 byte) + 784 input floats + 12 B
    one = (9 + 1 + 2 * 24) * (3604 * 33 + 784 * 4 + 12)
    budget = int(1.5 * one)
    first_b, peak_b, res_b = run(budget)
    assert first_b["admitted"] == 1 and first_b["queued"] == 3
    assert 0 < peak_b <= budget
    # roots bounded together with other requests' roots take kernels sized for
    # the larger batch, so bounds may differ at rounding level (tolerance 1e-4)
    for (vb, kb), (vf, kf) in zip(res_b, res_free):
        assert vb == vf and len(kb) == len(kf)
        for a, b in zip(kb, kf):
            assert a[:5] == b[:5]
            assert abs(a[5] - b[5]) <= 1e-4 * (1 + abs(b[5]))
