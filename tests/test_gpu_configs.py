"""The configurations at their specified sizes against the FP64 oracle.

* Conv-big (3x32x32, seven ReLU layers) and the ResNet (3x32x32, two residual
  blocks): the DeepPoly root bounds of every layer -- convolution and fully
  connected -- element by element (Sec. 3.1 back-substitution through
  convolutions and residual sums), for one property each.  The oracle takes
  about a minute per network, in a spawn process pool beside the GPU work.
* The 784-100-100-10 net with k = 3 multi-neuron constraints, one subproblem
  per launch, 256-node budget: the verdicts of all 16 properties.  The trees
  may part where a node's optimised bound is not determined at FP32
  precision (see helpers.compare_trace), so verdicts must be consistent
  (never VERIFIED against FALSIFIED), identical for most properties, and every
  counterexample must hold in FP64.
"""
import numpy as np
import pytest
import torch

import synth
from helpers import (TOL, close, gpu_property, oracle_root_bounds_job, oracle_verify_job,
                     spawn_pool, verdicts_consistent)
from oracle import mnc as omnc
from oracle import bab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    return Context


def test_full_size_root_bounds_match_oracle(Context):
    pool = spawn_pool(2)
    try:
        jobs = {cfg: pool.apply_async(oracle_root_bounds_job, (cfg, 0, 6)) for cfg in (2, 3)}
        gpu = {}
        for cfg in (2, 3):
            layers = synth.make_network(cfg)
            pr = synth.make_properties(cfg, layers, n=1, eps=synth.load_eps(cfg))[0]
            with Context(node_capacity=64) as ctx:
                net = ctx.load_network(layers)
                p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
                gpu[cfg] = [ctx.root_bounds(p, i) for i in range(1, net.R + 1)]
        for cfg in (2, 3):
            ref = jobs[cfg].get(timeout=1800)
            assert len(ref) == len(gpu[cfg])
            for i, (gl, gu) in enumerate(gpu[cfg], start=1):
                ol, ou = ref[i]
                for name, g, o in (("l", gl, ol), ("u", gu, ou)):
                    ok = close(g, o)
                    assert ok.all(), (cfg, f"{name}{i}", int((~ok).sum()), g[~ok][:4], o[~ok][:4])
    finally:
        pool.close()
        pool.join()


def test_fc_mnc_verdicts_at_budget(Context):
    budget = 256
    layers = synth.make_network(0)
    prs = synth.make_properties(0, layers, eps=synth.load_eps(0))
    pool = spawn_pool(8)
    try:
        jobs = [pool.apply_async(oracle_verify_job, (0, k, budget, True, 2)) for k in range(len(prs))]
        got = []
        with Context(node_capacity=4096, max_mnc_rows=65536) as ctx:
            gnet = ctx.load_network(layers)
            for pr in prs:
                prep = bab.prepare(layers, pr.C, pr.d, pr.lo, pr.hi, omnc.mnc_fn())
                _, prop = gpu_property(ctx, layers, pr.lo, pr.hi, pr.C, pr.d, prep[6], net=gnet)
                ctx.set_budget(prop, budget)
                for _ in range(100000):
                    if ctx.bab_step([prop], max_nodes=1, steps=20)["nodes_bounded"] == 0:
                        break
                v, _, xc = ctx.verdict(prop)
                if v == -1:
                    assert np.all(xc >= pr.lo) and np.all(xc <= pr.hi)
                    assert (pr.C @ synth.net_forward(layers, xc) + pr.d).min() < 0
                got.append((v, len(ctx.trace(prop))))
        ref = [j.get(timeout=3600) for j in jobs]
    finally:
        pool.close()
        pool.join()
    same = sum(g[0] == o[0] for g, o in zip(got, ref))
    print("config 0 verdicts (gpu, oracle):", [(g[0], o[0]) for g, o in zip(got, ref)])
    for g, o in zip(got, ref):
        assert verdicts_consistent(g[0], o[0]), (g, o)
    assert same >= 12, (same, got, ref)
