"""GPU adversarial pre-attack (mnbab_attack) against the oracle (oracle/attack.py),
in both forms: one kernel per (row, start) (path 1) and the per-layer kernels
on scratch node slots (path 2, and the only form for residual networks and
networks whose weights exceed shared memory)."""
import numpy as np
import pytest

import synth
from helpers import TOL, conv_case, resnet_spec
from oracle import attack, core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context as C
    return C


def _margin64(layers, C, d, r, x):
    return float(C[r] @ synth.net_forward(layers, np.asarray(x, np.float64)) + d[r])


@pytest.mark.parametrize("path", [1, 2])
def test_affine_region_reaches_the_closed_form_minimum(Context, path):
    """Every ReLU active on the box: the margin is affine and the sign steps end at
    the minimising corner, so the attack must return the exact minimum."""
    layers = synth.tiny_fc_net(5, [5, 8, 6, 3])
    layers[0]["b"] = (layers[0]["b"] + 50.0).astype(np.float32)
    layers[2]["W"] = np.abs(layers[2]["W"]).astype(np.float32)
    layers[2]["b"] = (layers[2]["b"] + 50.0).astype(np.float32)
    C, d = synth.property_rows(0, 3)
    lo, hi = np.full(5, -0.3, np.float32), np.full(5, 0.4, np.float32)
    starts = (lo + (hi - lo) * np.random.default_rng(1).uniform(size=(2, 5))).astype(np.float32)
    ref = attack.attack(layers, C, d, lo, hi, starts.astype(np.float64), steps=6)
    with Context(node_capacity=64) as ctx:
        ctx.set_attack_path(path)
        net = ctx.load_network(layers)
        p = ctx.set_property(net, lo, hi, C, d)
        best, x = ctx.attack(p, starts, steps=6)
    for r, (rb, _) in enumerate(ref):
        assert abs(best[r] - rb) <= TOL * (1 + abs(rb)), (r, best[r], rb)
        assert abs(_margin64(layers, C, d, r, x[r]) - rb) <= TOL * (1 + abs(rb))


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("case", ["fc", "conv"])
def test_one_step_matches_oracle(Context, case, path):
    """From identical starting points, one sign step gives the oracle's iterate and
    margin wherever no gradient component is near zero (there FP32 and FP64 may
    take different signs, so such samples are skipped)."""
    if case == "fc":
        layers = synth.tiny_fc_net(11, [12, 16, 9, 4])
        x0 = np.random.default_rng(12).uniform(0.2, 0.8, 12).astype(np.float32)
        y = synth.net_forward(layers, x0)
        C, d = synth.property_rows(int(np.argmax(y)), 4)
        lo, hi = synth.input_box(x0, 0.1)
    else:
        layers, C, d, lo, hi, _ = conv_case(6, 0.05)
    net64 = core.fold_property(core.load_net(layers), C, d)
    rng = np.random.default_rng(13)
    checked = 0
    with Context(node_capacity=64) as ctx:
        ctx.set_attack_path(path)
        net = ctx.load_network(layers)
        p = ctx.set_property(net, lo, hi, C, d)
        for _ in range(6):
            s = (lo + (hi - lo) * rng.uniform(size=lo.size)).astype(np.float32)
            best, x = ctx.attack(p, s[None, :], steps=1)
            for r in range(C.shape[0]):
                f0, g = attack.margin_and_grad(net64, s.astype(np.float64), r)
                if np.abs(g).min() <= 1e-3 * np.abs(g).max():
                    continue
                rb, rx, _ = attack.pgd_row(net64, lo, hi, r, s[None, :].astype(np.float64), 1)
                f1 = _margin64(layers, C, d, r, np.clip(s - attack.step_size(lo, hi, 1) * np.sign(g),
                                                        lo, hi))
                if abs(f1 - f0) <= 1e-3 * (1 + abs(f0)):
                    continue  # argmin of two nearly equal margins
                assert abs(best[r] - rb) <= TOL * (1 + abs(rb)), (r, best[r], rb)
                assert np.allclose(x[r], rx, rtol=0, atol=1e-5)
                checked += 1
    assert checked >= 5


def test_full_attack_on_the_conv_net_is_sound(Context):
    """The 28x28 conv net, 5 starts x 50 steps: every minimiser lies in the box, its
    FP64 margin is the reported one, and it is no worse than the starts; negative
    margins are counterexamples."""
    layers = synth.make_network(1)
    pr = synth.make_properties(1, layers, n=1, eps=synth.load_eps(1))[0]
    rng = np.random.default_rng(14)
    starts = (pr.lo + (pr.hi - pr.lo) * rng.uniform(size=(5, pr.lo.size))).astype(np.float32)
    with Context(node_capacity=64) as ctx:
        net = ctx.load_network(layers)
        p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
        best, x = ctx.attack(p, starts, steps=50)
    for r in range(pr.C.shape[0]):
        assert (x[r] >= pr.lo).all() and (x[r] <= pr.hi).all()
        m = _margin64(layers, pr.C, pr.d, r, x[r])
        assert abs(m - best[r]) <= TOL * (1 + abs(m))
        f_starts = min(_margin64(layers, pr.C, pr.d, r, s) for s in starts)
        assert best[r] <= f_starts + TOL * (1 + abs(f_starts))


def test_one_kernel_form_refuses_residual_networks(Context):
    """Path 1 (one kernel per row and start) takes chain networks only; the
    default path runs residual networks in the per-layer form."""
    from paper_2205_00263_gb300 import MnbabError
    layers, C, d, lo, hi, _ = conv_case(4, 0.02, resnet_spec)
    with Context(node_capacity=64) as ctx:
        net = ctx.load_network(layers)
        p = ctx.set_property(net, lo, hi, C, d)
        ctx.set_attack_path(1)
        with pytest.raises(MnbabError):
            ctx.attack(p, lo[None, :], steps=2)
        ctx.set_attack_path(0)
        best, x = ctx.attack(p, lo[None, :], steps=2)
        assert np.all(np.isfinite(best))


def _well_conditioned(net64, lo, hi, r, start, steps, rel=1e-4):
    """Whether the FP64 sign-step trajectory of row r from `start` stays away
    from decisions FP32 could take differently: every gradient component is
    exactly 0 (no path reaches it, in any precision) or at least rel of the
    largest, and no iterate at another point has a margin within 1e-4 of the
    running minimum (the first minimiser is then determined)."""
    x = np.clip(np.asarray(start, np.float64), lo, hi)
    alpha = attack.step_size(lo, hi, steps)
    best, bx = np.inf, None
    for k in range(steps + 1):
        f, g = attack.margin_and_grad(net64, x, r)
        if bx is not None and not np.array_equal(x, bx) and abs(f - best) <= 1e-4 * (1 + abs(best)):
            return False
        if f < best:
            best, bx = f, x.copy()
        if k == steps:
            return True
        ga = np.abs(g)
        if np.any((ga > 0) & (ga <= rel * ga.max())):
            return False
        x = np.clip(x - alpha * np.sign(g), lo, hi)


@pytest.mark.parametrize("case,path", [("fc", 1), ("fc", 2), ("conv", 1), ("conv", 2),
                                       ("resnet", 0)])
def test_multi_step_attack_matches_oracle(Context, case, path):
    """Six sign steps from identical starts give the oracle's best margin and
    minimiser on every row whose FP64 trajectory is well conditioned (the
    residual network in the per-layer form)."""
    if case == "resnet":
        layers, C, d, lo, hi, _ = conv_case(4, 0.02, resnet_spec)
    elif case == "fc":
        layers = synth.tiny_fc_net(11, [12, 16, 9, 4])
        x0 = np.random.default_rng(12).uniform(0.2, 0.8, 12).astype(np.float32)
        y = synth.net_forward(layers, x0)
        C, d = synth.property_rows(int(np.argmax(y)), 4)
        lo, hi = synth.input_box(x0, 0.1)
    else:
        layers, C, d, lo, hi, _ = conv_case(6, 0.05)
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    net64 = core.fold_property(core.load_net(layers), C, d)
    rng = np.random.default_rng(21)
    checked = 0
    with Context(node_capacity=64) as ctx:
        ctx.set_attack_path(path)
        net = ctx.load_network(layers)
        p = ctx.set_property(net, lo, hi, C, d)
        for _ in range(16):
            s = (lo + (hi - lo) * rng.uniform(size=lo.size)).astype(np.float32)
            best, x = ctx.attack(p, s[None, :], steps=6)
            for r in range(C.shape[0]):
                if not _well_conditioned(net64, lo64, hi64, r, s.astype(np.float64), 6):
                    continue
                rb, rx, _ = attack.pgd_row(net64, lo64, hi64, r, s[None, :].astype(np.float64), 6)
                assert abs(best[r] - rb) <= TOL * (1 + abs(rb)), (r, best[r], rb)
                assert np.allclose(x[r], rx, rtol=0, atol=1e-5)
                checked += 1
    assert checked >= 4


def test_pre_attack_in_bab_falsifies_before_any_node(Context):
    """mnbab_set_attack: when the property starts, the attack from the box
    centre and SplitMix64 starts runs first; a property the oracle's attack
    (same starts) falsifies is FALSIFIED with no node bounded and a
    counterexample that holds in FP64; one it does not falsify goes on to
    branch-and-bound."""
    layers = synth.make_network(1)
    prs = synth.make_properties(1, layers, n=6, eps=synth.load_eps(1))
    seen = {True: 0, False: 0}
    with Context(node_capacity=4096) as ctx:
        net = ctx.load_network(layers)
        for k, pr in enumerate(prs):
            starts = attack.attack_starts(pr.lo, pr.hi, 4, seed=100 + k)
            ref = attack.attack(layers, pr.C, pr.d, pr.lo, pr.hi, starts, steps=20)
            o_fals = min(b for b, _ in ref) < -1e-4
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_attack(p, 4, 20, seed=100 + k)
            ctx.set_budget(p, 16)
            ctx.bab_step([p], max_nodes=64, steps=20)
            v, _, xc = ctx.verdict(p)
            if o_fals:
                assert v == -1 and len(ctx.trace(p)) == 0, k
                assert np.all(xc >= pr.lo) and np.all(xc <= pr.hi)
                assert (pr.C @ synth.net_forward(layers, xc.astype(np.float64)) + pr.d).min() < 0
            elif min(b for b, _ in ref) > 1e-4:
                assert len(ctx.trace(p)) > 0
            seen[o_fals] += 1
        with pytest.raises(Exception):
            ctx.set_attack(p, 4, 20)   # already started
    assert seen[True] >= 1


def test_per_layer_attack_on_conv_big_is_sound(Context):
    """conv_big_32 (weights beyond shared memory: the per-layer form), 3 starts
    x 8 steps: every minimiser lies in the box, its FP64 margin is the reported
    one within the tolerance, and it is no worse than its start."""
    layers = synth.make_network(2)
    pr = synth.make_properties(2, layers, n=1, eps=synth.load_eps(2))[0]
    rng = np.random.default_rng(15)
    starts = (pr.lo + (pr.hi - pr.lo) * rng.uniform(size=(3, pr.lo.size))).astype(np.float32)
    with Context(node_capacity=64) as ctx:
        net = ctx.load_network(layers)
        p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
        best, x = ctx.attack(p, starts, steps=8)
    for r in range(pr.C.shape[0]):
        assert (x[r] >= pr.lo).all() and (x[r] <= pr.hi).all()
        m = _margin64(layers, pr.C, pr.d, r, x[r])
        assert abs(m - best[r]) <= TOL * (1 + abs(m))
        f_starts = min(_margin64(layers, pr.C, pr.d, r, s) for s in starts)
        assert best[r] <= f_starts + TOL * (1 + abs(f_starts))


def test_pre_attack_in_bab_on_a_residual_network(Context):
    """mnbab_set_attack on a residual network (per-layer form, FP64 check on the
    device): a property the oracle's attack (same starts) falsifies is
    FALSIFIED before any node with a counterexample that holds in FP64; one
    it does not falsify goes on to branch-and-bound."""
    seen = 0
    with Context(node_capacity=256) as ctx:
        for k, (seed, eps) in enumerate(((4, 0.06), (5, 0.06), (6, 0.06), (5, 0.004))):
            layers, C, d, lo, hi, _ = conv_case(seed, eps, resnet_spec)
            starts = attack.attack_starts(lo, hi, 3, seed=200 + k)
            ref = attack.attack(layers, C, d, lo, hi, starts, steps=10)
            o_best = min(b for b, _ in ref)
            net = ctx.load_network(layers)
            p = ctx.set_property(net, lo, hi, C, d)
            ctx.set_attack(p, 3, 10, seed=200 + k)
            ctx.set_budget(p, 8)
            ctx.bab_step([p], max_nodes=64, steps=5)
            v, _, xc = ctx.verdict(p)
            if o_best < -1e-4:
                assert v == -1 and len(ctx.trace(p)) == 0, k
                assert np.all(xc >= lo) and np.all(xc <= hi)
                assert (C @ synth.net_forward(layers, xc.astype(np.float64)) + d).min() < 0
                seen += 1
            elif o_best > 1e-4:
                assert len(ctx.trace(p)) > 0
    assert seen >= 1
