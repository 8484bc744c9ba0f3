"""The allocation-free entry point against the ordinary one.

mnbab_deeppoly_fc_noalloc exists for callers that cannot allocate device
memory themselves (code inside another framework's memory pool or allocator
hooks, hosts with device memory partitioned up front).  It takes device pointers the caller already
owns and keeps its scratch in a static device array.  This test computes the
DeepPoly bounds of every property row once through a context
(mnbab_deeppoly_batch on root nodes) and twice in a row through the
allocation-free call, and requires the same bounds within the tolerance of
the other parity tests.  The file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from helpers import TOL, close

pytestmark = pytest.mark.gpu


def _case(seed, dims, eps):
    layers = synth.tiny_fc_net(seed, list(dims))
    x0 = np.random.default_rng(seed + 100).uniform(0.2, 0.8, dims[0]).astype(np.float32)
    y = synth.net_forward(layers, x0)
    Cm, d = synth.property_rows(int(np.argmax(y)), dims[-1])
    lo, hi = synth.input_box(x0, eps)
    return layers, Cm, d, lo, hi


def _reference(ctx, layers, Cm, d, lo, hi, R):
    net = ctx.load_network(layers)
    prop = ctx.set_property(net, lo, hi, Cm, d)
    nodes = [ctx.node_root(prop, r) for r in range(Cm.shape[0])]
    lb = ctx.deeppoly_batch(nodes)
    bounds = [ctx.root_bounds(prop, i) for i in range(1, R + 1)]
    return lb, bounds


def _noalloc(lib, layers, Cm, d, lo, hi, bounds):
    dev = torch.device("cuda", 0)
    fcs = [L for L in layers if L["kind"] == "fc"]
    dims = [fcs[0]["W"].shape[1]] + [L["W"].shape[0] for L in fcs[:-1]]
    Wd = [torch.as_tensor(L["W"], device=dev).contiguous() for L in fcs[:-1]]
    bd = [torch.as_tensor(L["b"], device=dev).contiguous() for L in fcs[:-1]]
    # the property folded into the last layer, in FP64 then rounded (as the library does)
    last = fcs[-1]
    Wf = (Cm.astype(np.float64) @ last["W"].astype(np.float64)).astype(np.float32)
    bf = (Cm.astype(np.float64) @ last["b"].astype(np.float64) + d).astype(np.float32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=dev)
    lo_d, hi_d, Wf_d, bf_d = t(lo), t(hi), t(Wf), t(bf)
    l_d = t(np.concatenate([b[0] for b in bounds]))
    u_d = t(np.concatenate([b[1] for b in bounds]))
    out = torch.full((Cm.shape[0],), float("nan"), device=dev)
    dims_c = (C.c_int32 * len(dims))(*dims)
    W_c = (C.c_void_p * max(1, len(Wd)))(*[w.data_ptr() for w in Wd])
    b_c = (C.c_void_p * max(1, len(bd)))(*[x.data_ptr() for x in bd])
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev)
    st = lib.mnbab_deeppoly_fc_noalloc(len(dims), dims_c, W_c, b_c, lo_d.data_ptr(),
                                       hi_d.data_ptr(), l_d.data_ptr(), u_d.data_ptr(),
                                       Wf_d.data_ptr(), bf_d.data_ptr(), Cm.shape[0],
                                       out.data_ptr(), C.c_void_p(stream.cuda_stream), err, 256)
    assert st == 0, err.value.decode()
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_context_path_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context, _lib
    lib = _lib.load()
    cases = [(21, (37, 53, 29, 7), 0.1), (22, (784, 100, 100, 10), 0.02)]
    with Context(device=0, node_capacity=64) as ctx:
        refs = []
        for seed, dims, eps in cases:
            layers, Cm, d, lo, hi = _case(seed, dims, eps)
            lb, bounds = _reference(ctx, layers, Cm, d, lo, hi, len(dims) - 2)
            refs.append((layers, Cm, d, lo, hi, lb, bounds))
    # two calls in a row, different networks and row counts: the second call must
    # not see anything the first one left in the shared scratch
    for layers, Cm, d, lo, hi, lb, bounds in refs:
        got = _noalloc(lib, layers, Cm, d, lo, hi, bounds)
        ok = close(got, lb, TOL)
        assert ok.all(), (got, lb)
    # rows beyond the static scratch are rejected with a message, not run
    layers, Cm, d, lo, hi, lb, bounds = refs[1]
    big = np.tile(Cm, (2000, 1))
    dims = (C.c_int32 * 3)(784, 100, 100)
    err = C.create_string_buffer(256)
    st = lib.mnbab_deeppoly_fc_noalloc(3, dims, (C.c_void_p * 2)(1, 1), (C.c_void_p * 2)(1, 1),
                                       1, 1, 1, 1, 1, 1, big.shape[0], 1, None, err, 256)
    assert st == -2 and b"static scratch" in err.value
