"""Pins of the oracle's adversarial pre-attack (oracle/attack.py) by facts that
do not come from the oracle itself: finite differences, a closed-form minimum,
and the network's own forward pass."""
import numpy as np
import pytest
import torch

import synth
from oracle import attack, core


def _net(seed, dims, shift=0.0):
    layers = synth.tiny_fc_net(seed, list(dims))
    for L in layers:
        if L["kind"] == "fc" and shift:
            L["b"] = (L["b"] + shift).astype(np.float32)
    return layers


def _folded(layers, C, d):
    return core.fold_property(core.load_net(layers), C, d)


def _preacts(layers, x):
    pre = []
    synth.net_forward(layers, x, collect=pre)
    return pre


def test_gradient_matches_central_differences():
    layers = _net(3, (6, 9, 7, 4))
    C, d = synth.property_rows(1, 4)
    net = _folded(layers, C, d)
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(40):
        x = rng.uniform(-1, 1, 6)
        if min(np.abs(z).min() for z in _preacts(layers, x)) < 1e-3:
            continue  # too close to a ReLU kink for a difference quotient
        for r in range(C.shape[0]):
            _, g = attack.margin_and_grad(net, x, r)
            h = 1e-6
            fd = np.array([(attack.margin_and_grad(net, x + h * e, r)[0] -
                            attack.margin_and_grad(net, x - h * e, r)[0]) / (2 * h)
                           for e in np.eye(6)])
            assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)
        checked += 1
    assert checked >= 10


def test_affine_region_reaches_the_closed_form_minimum():
    """With every ReLU active on the box the margin is affine, g . x + c; sign
    steps of total length 1.25 (hi - lo) end at the minimising corner."""
    layers = _net(5, (5, 8, 6, 3), shift=50.0)
    layers[2]["W"] = np.abs(layers[2]["W"])  # nonnegative weights keep layer 2 active
    C, d = synth.property_rows(0, 3)
    lo, hi = np.full(5, -0.3), np.full(5, 0.4)
    W1, b1 = layers[0]["W"].astype(np.float64), layers[0]["b"].astype(np.float64)
    W2, b2 = layers[2]["W"].astype(np.float64), layers[2]["b"].astype(np.float64)
    W3, b3 = layers[4]["W"].astype(np.float64), layers[4]["b"].astype(np.float64)
    rng = np.random.default_rng(1)
    starts = lo + (hi - lo) * rng.uniform(size=(2, 5))
    assert all(min(z.min() for z in _preacts(layers, x)) > 0 for x in (lo, hi, *starts))
    res = attack.attack(layers, C, d, lo, hi, starts, steps=6)
    for r, (best, bx) in enumerate(res):
        g = C[r] @ W3 @ W2 @ W1
        c = C[r] @ (W3 @ (W2 @ b1 + b2) + b3) + d[r]
        exact = np.minimum(g * lo, g * hi).sum() + c
        assert best == pytest.approx(exact, abs=1e-9)
        assert bx is not None


def test_results_are_forward_margins_in_the_box_and_no_worse_than_starts():
    layers = _net(7, (8, 12, 10, 5))
    C, d = synth.property_rows(2, 5)
    x0 = np.random.default_rng(2).uniform(0.2, 0.8, 8)
    lo, hi = synth.input_box(x0.astype(np.float32), 0.1)
    starts = lo + (hi - lo) * np.random.default_rng(3).uniform(size=(3, 8))
    net = _folded(layers, C, d)
    for r, (best, bx) in enumerate(attack.attack(layers, C, d, lo, hi, starts, steps=10)):
        assert (bx >= lo - 1e-12).all() and (bx <= hi + 1e-12).all()
        y = C[r] @ synth.net_forward(layers, bx) + d[r]
        assert best == pytest.approx(y, abs=1e-9)
        f_starts = [attack.margin_and_grad(net, s, r)[0] for s in starts]
        assert best <= min(f_starts) + 1e-12


def test_splitmix_starts_follow_the_published_generator():
    """SplitMix64's first outputs from state 0 are the reference code's
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f; the counter form
    takes the (i + 1)-th output; starts are the box centre then box points."""
    s, outs = 0, []
    for _ in range(3):
        o, s = attack.splitmix64(s)
        outs.append(o)
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert attack.splitmix_uniform(0, 1) == (0x6E789E6AA1B965F4 >> 11) / 2.0 ** 53
    lo, hi = np.array([0.1, -1.0, 2.0]), np.array([0.3, 1.0, 2.5])
    st = attack.attack_starts(lo, hi, 4, seed=7)
    assert np.allclose(st[0], 0.5 * (lo + hi))
    assert np.all(st >= lo) and np.all(st < hi)
    assert len({tuple(r) for r in st}) == 4
