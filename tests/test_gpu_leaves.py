"""Exact completion of fully split leaves on the GPU (Sec. 3.3, completeness).

On tiny 2-8-8-2 networks at radii within 5% of a critical radius, unlimited
branch-and-bound with leaf completion (mnbab_set_leaf_steps) reproduces the
sign of the exact minimum over the input box (pattern enumeration with one
LP per pattern, oracle/exact.py): VERIFIED when it is positive, FALSIFIED
(with a counterexample that holds in FP64) when negative.  The nodes are
bounded by the DeepPoly pass alone (0 Adam steps) so that the trees reach
fully split leaves, and once more with 20 Adam steps.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import exact
from test_oracle_pins import TINY_CASES, _tiny_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    return Context


@pytest.mark.parametrize("steps", [0, 20])
def test_unlimited_bab_with_leaf_completion_is_complete(Context, steps):
    leaves_seen = 0
    for seed, eps in TINY_CASES:
        layers, C, d, lo, hi = _tiny_problem(seed, eps)
        m = min(exact.exact_min(layers, C, d, r, lo, hi)[0] for r in range(C.shape[0]))
        with Context(node_capacity=8192) as ctx:
            net = ctx.load_network(layers)
            prop = ctx.set_property(net, lo, hi, C, d)
            ctx.set_budget(prop, 4000)
            ctx.set_leaf_steps(prop, 256)
            for _ in range(10000):
                st = ctx.bab_step([prop], max_nodes=64, steps=steps)
                if st["nodes_bounded"] == 0:
                    break
            v, _, xc = ctx.verdict(prop)
            tr = ctx.trace(prop)
        leaves_seen += sum(1 for r in tr if r["leaf"] and r["verdict"] != 0)  # decided leaves
        assert v == (1 if m > 0 else -1), (seed, eps, m, v)
        if v == -1:
            assert np.all(xc >= lo) and np.all(xc <= hi)
            assert (C @ synth.net_forward(layers, xc.astype(np.float64)) + d).min() < 0
    if steps == 0:
        assert leaves_seen > 0
