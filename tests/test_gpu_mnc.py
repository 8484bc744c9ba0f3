"""The library's multi-neuron constraint generator end to end on the GPU
(mnbab_generate_mnc): groups and octahedral bounds from the device's DeepPoly
root bounds, hulls on the host, rows uploaded to the property.

Against the oracle (mnc.generate on the FP64 root bounds) for a property of
the 784-100-100-10 network: the same groups (the sliding triples of the
unstable neurons), and per shared group rows that match the oracle's within
the FP32 tolerance of the octahedral bounds; then the constraints are used:
a BaB run with ACS on them gives a sound verdict.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import close
from oracle import bab, mnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    return Context


def _by_group(idx, P, Ph, p):
    out = {}
    for r in range(len(p)):
        out.setdefault(tuple(int(v) for v in idx[r]), []).append(
            np.concatenate([P[r], Ph[r], [p[r]]]).astype(np.float64))
    return {k: np.array(v) for k, v in out.items()}


def test_generated_constraints_match_oracle_and_run(Context):
    layers = synth.make_network(0)
    pr = synth.make_properties(0, layers, n=2, eps=synth.load_eps(0))[1]
    prep = bab.prepare(layers, pr.C, pr.d, pr.lo, pr.hi, mnc.mnc_fn())
    ref = prep[6]
    with Context(node_capacity=2048, max_mnc_rows=65536) as ctx:
        net = ctx.load_network(layers)
        prop = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
        rows = ctx.generate_mnc(prop)
        assert rows > 0
        got_total, shared, matched, compared = 0, 0, 0, 0
        for t in range(1, net.R + 1):
            idx, P, Ph, p = ctx.get_mnc(prop, t)
            got_total += len(p)
            g = _by_group(idx, P, Ph, p)
            o = _by_group(ref[t].idx, ref[t].P, ref[t].Ph, ref[t].p) if t in ref else {}
            assert len(set(g) ^ set(o)) <= 0.1 * max(1, len(o)), (t, len(g), len(o))
            for key in set(g) & set(o):
                shared += 1
                A, B = g[key], o[key]
                # every generated row is (to FP32 rounding of the bounds) an oracle facet
                d = np.abs(A[:, None, :] - B[None, :, :]).max(-1).min(1)
                compared += len(d)
                matched += int((d <= 1e-4 * (1 + np.abs(A[:, 6]))).sum())
        assert got_total == rows
        assert shared >= 40
        assert matched >= 0.95 * compared, (matched, compared)
        # the constraints in use: BaB with ACS over them
        ctx.set_budget(prop, 64)
        for _ in range(100):
            if ctx.bab_step([prop], max_nodes=32, steps=20)["nodes_bounded"] == 0:
                break
        v, _, xc = ctx.verdict(prop)
        if v == -1:
            assert np.all(xc >= pr.lo) and np.all(xc <= pr.hi)
            assert (pr.C @ synth.net_forward(layers, xc) + pr.d).min() < 0
        ores = bab.verify(layers, pr.C, pr.d, pr.lo, pr.hi, max_nodes=64, prepared=prep)
        assert {v, ores.verdict} != {1, -1}
        assert any(rec["fallback"] == 0 for rec in ctx.trace(prop) if rec["split_layer"] > 0)
