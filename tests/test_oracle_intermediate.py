"""Pins of the oracle's optimised intermediate bounds (Sec. 3.1, parameter
sharing: one parameter set per layer shared by its neurons, separate sets for
lower and upper bounds).

Plausible mistakes these catch: an unsound update of the node's bounds (a
dropped intersection, lower and upper rows swapped), a set objective whose
gradient is not the sum of the rows' gradients, an optimiser that does not
reach the optimum of a linear objective on [0, 1], and a best bound that
exceeds what any parameter value gives.  None of these tests calls the GPU
library.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import bab, core
from oracle.core import DT

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def _fc(W, b):
    return dict(kind="fc", W=np.asarray(W, np.float32), b=np.asarray(b, np.float32))


RELU = dict(kind="relu")


def _case(seed, dims=(10, 14, 12, 10, 3), eps=0.12):
    L = synth.tiny_fc_net(seed, list(dims))
    rng = np.random.default_rng(seed + 100)
    x0 = rng.uniform(0.2, 0.8, dims[0]).astype(np.float32)
    y = synth.net_forward(L, x0)
    C, d = synth.property_rows(int(np.argmax(y)), dims[-1])
    lo, hi = synth.input_box(x0, eps)
    return bab.prepare(L, C, d, lo, hi, None), lo, hi


def _split_node(prep, rng, n_splits):
    """A root node with n_splits layer-1 splits, re-bounded (Sec. 3.2)."""
    net, lo, hi, l, u, S, m, dense = prep
    node = bab.root_node(net, 0, l, u, S, m)
    cands = [j for j in range(l[1].numel()) if l[1][j] < 0 < u[1][j]]
    for j in rng.choice(cands, size=min(n_splits, len(cands)), replace=False):
        sgn = int(rng.choice([1, -1]))
        node.S[1][j] = sgn
        if sgn == 1:
            node.u[1][j] = 0.0
        else:
            node.l[1][j] = 0.0
    node.split_layer = 1
    core.rebound_node(net, node, lo, hi)
    return node


def _in_subdomain(net, node, X):
    keep = np.ones(X.shape[0], bool)
    h = _t(X)
    for i in range(1, net.R + 1):
        z = net.aff[i].forward(h).numpy()
        S = node.S[i].numpy()
        keep &= np.all((S[None, :] != 1) | (z <= 0), axis=1)
        keep &= np.all((S[None, :] != -1) | (z >= 0), axis=1)
        h = torch.clamp(_t(z), min=0)
    return keep


@pytest.mark.parametrize("seed,n_splits", [(0, 0), (1, 0), (2, 3)])
def test_optimised_bounds_sound_and_never_looser(seed, n_splits):
    """The optimised bounds contain every sampled pre-activation of the node's
    subdomain, are never looser than the DeepPoly bounds they start from (the
    first iterate is DeepPoly), and at the root they tighten some neuron."""
    prep, lo, hi = _case(seed)
    net, lo_t, hi_t = prep[0], prep[1], prep[2]
    rng = np.random.default_rng(seed)
    node = _split_node(prep, rng, n_splits)
    l0 = {i: node.l[i].clone() for i in node.l}
    u0 = {i: node.u[i].clone() for i in node.u}
    hp = core.AdamHP(steps=20)
    rows = core.optimize_intermediate(net, node, lo_t, hi_t, hp)
    assert rows > 0
    gain = 0.0
    for i in node.l:
        assert bool((node.l[i] >= l0[i]).all()) and bool((node.u[i] <= u0[i]).all())
        gain += float((node.l[i] - l0[i]).sum() + (u0[i] - node.u[i]).sum())
    assert bool((node.l[1] == l0[1]).all()) and bool((node.u[1] == u0[1]).all())
    if n_splits == 0:
        assert gain > 1e-6, "optimisation never tightened a bound"
    X = rng.uniform(lo, hi, size=(10000, lo.size))
    X = X[_in_subdomain(net, node, X)]
    h = _t(X)
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h)
        assert bool((zh >= node.l[i] - 1e-9).all()), f"layer {i}: lower bound above a sample"
        assert bool((zh <= node.u[i] + 1e-9).all()), f"layer {i}: upper bound below a sample"
        h = torch.clamp(zh, min=0)


@pytest.mark.parametrize("t,side", [(2, 1), (3, -1), (3, 1)])
def test_set_gradient_matches_finite_differences(t, side):
    """The gradient that the shared set ascends is the derivative of the summed
    row bounds: autograd against central differences at an interior point."""
    prep, lo, hi = _case(4)
    net, lo_t, hi_t = prep[0], prep[1], prep[2]
    rng = np.random.default_rng(4)
    node = _split_node(prep, rng, 2)
    idx = torch.nonzero((node.l[t] < 0) & (node.u[t] > 0) & (node.S[t] == 0)).reshape(-1)
    assert idx.numel() > 0
    alpha = {i: _t(rng.uniform(0.2, 0.8, node.l[i].numel())) for i in range(1, t)}
    beta = {i: _t(rng.uniform(0.1, 0.5, node.l[i].numel())) * (node.S[i] != 0)
            for i in range(1, t)}
    _, ga, gb = core.intermediate_objective_grad(net, node, t, idx, side, alpha, beta, lo_t, hi_t)

    def f(a, b):
        return float(core.intermediate_objective(net, node, t, idx, side, a, b, lo_t, hi_t).sum())

    h = 1e-6
    checked = 0
    for i in range(1, t):
        for j in range(node.l[i].numel()):
            if not (node.l[i][j] < 0 < node.u[i][j]) or node.S[i][j] != 0:
                continue
            ap = {k: v.clone() for k, v in alpha.items()}
            am = {k: v.clone() for k, v in alpha.items()}
            ap[i][j] += h
            am[i][j] -= h
            fd = (f(ap, beta) - f(am, beta)) / (2 * h)
            assert abs(fd - float(ga[i][j])) <= 1e-6 * (1 + abs(fd)), (i, j, fd, float(ga[i][j]))
            checked += 1
        for j in torch.nonzero(node.S[i] != 0).reshape(-1).tolist():
            bp = {k: v.clone() for k, v in beta.items()}
            bm = {k: v.clone() for k, v in beta.items()}
            bp[i][j] += h
            bm[i][j] -= h
            fd = (f(alpha, bp) - f(alpha, bm)) / (2 * h)
            assert abs(fd - float(gb[i][j])) <= 1e-6 * (1 + abs(fd))
            checked += 1
    assert checked > 3


def _one_unstable_net():
    """2 -> 2 -> 2 -> 1 over [-1, 1]^2: layer-1 neuron 0 ranges over [-1.5, 1.5]
    (unstable) and is the only path from the input; neuron 1 is the constant 1.
    A row's input coefficients are then alpha (or the fixed lower slope) times
    one weight row, so their signs, and the minimising corner of the box, do
    not change with alpha."""
    layers = [_fc([[1.0, 0.5], [0.0, 0.0]], [0.0, 1.0]), RELU,
              _fc([[1.0, -1.0], [-2.0, 0.5]], [0.1, 0.3]), RELU,
              _fc([[1.0, 1.0]], [0.0])]
    net = core.load_net(layers)
    lo, hi = _t([-1.0, -1.0]), _t([1.0, 1.0])
    l, u, S = core.root_bounds(net, lo, hi)
    return net, lo, hi, l, u, S


def test_each_row_keeps_its_best_iterate():
    """Every iterate of a set gives valid bounds, so each row keeps the best it
    reached (Sec. 3.1).  x in [-1, 1]; layer 1 is x and x + 2 (stable), and
    z2 = relu(x) - 0.375 (x + 2) + 0.75 = relu(x) - 0.375 x.  Its lower bound
    with the first neuron's shared slope alpha is -|alpha - 0.375| (DeepPoly,
    alpha = 1: -0.625).  From alpha = 1 Adam's first steps are lr = 0.1 long and
    reach alpha = 0.4 (-0.025) before momentum carries alpha past the optimum,
    so the optimised lower bound is at least -0.025 and at most the exact
    minimum 0."""
    L = [_fc([[1.0], [1.0]], [0.0, 2.0]), RELU, _fc([[1.0, -0.375]], [0.75]), RELU,
         _fc([[1.0]], [0.0])]
    net, lo, hi, l, u, S, _, _ = bab.prepare(L, [[1.0]], [0.0], [-1.0], [1.0])
    assert float(l[2][0]) == pytest.approx(-0.625, abs=1e-12)
    assert float(u[2][0]) == pytest.approx(0.625, abs=1e-12)
    node = bab.root_node(net, 0, l, u, S, None)
    core.optimize_intermediate(net, node, lo, hi, core.AdamHP(steps=20))
    assert float(node.l[2][0]) >= -0.025 - 1e-7
    assert float(node.l[2][0]) <= 1e-12


def test_linear_set_objective_reaches_its_corner():
    """With one unstable neuron below the target layer, every row bound is
    linear in that neuron's shared slope, so the set objective is maximised at
    alpha = 0 or 1: the optimised bounds reach the better corner's sum, and no
    row's best bound exceeds the larger of its two corner values."""
    net, lo, hi, l, u, S = _one_unstable_net()
    assert float(l[1][0]) < 0 < float(u[1][0]) and float(l[1][1]) > 0
    idx = torch.nonzero((l[2] < 0) & (u[2] > 0)).reshape(-1)
    assert idx.numel() == 2
    node = bab.root_node(net, 0, l, u, S, None)
    beta = {1: torch.zeros(2, dtype=DT)}

    def rows(a, side):
        return core.intermediate_objective(net, node, 2, idx, side, {1: _t([a, 1.0])}, beta, lo, hi)

    best = {}
    for side in (1, -1):
        r0, r1, rh = rows(0.0, side), rows(1.0, side), rows(0.5, side)
        assert torch.allclose(rh, 0.5 * (r0 + r1), atol=1e-12), "row bounds not linear in alpha"
        best[side] = (r0, r1)
    node2 = bab.root_node(net, 0, l, u, S, None)
    core.optimize_intermediate(net, node2, lo, hi, core.AdamHP(steps=20))
    lb_opt = node2.l[2][idx]
    ub_opt = node2.u[2][idx]
    for side, got in ((1, lb_opt), (-1, -ub_opt)):
        r0, r1 = best[side]
        assert float(got.sum()) >= max(float(r0.sum()), float(r1.sum())) - 1e-12
        assert bool((got <= torch.maximum(r0, r1) + 1e-12).all())
    # the corner values differ, so the optimum is a real choice
    assert not torch.allclose(best[1][0].sum(), best[1][1].sum())


@pytest.mark.parametrize("seed", [5, 6])
def test_zero_steps_reproduce_deeppoly_root_bounds(seed):
    """With no Adam step the only iterate is the start point, DeepPoly slopes
    and beta = 0 (Sec. 3.1 start point), so the root's bounds must stay the
    DeepPoly root bounds (same rows, same relaxation) to rounding."""
    prep, lo, hi = _case(seed)
    net, lo_t, hi_t, l, u, S = prep[0], prep[1], prep[2], prep[3], prep[4], prep[5]
    node = bab.root_node(net, 0, l, u, S, None)
    # widen the unstable neurons' bounds of layers >= 2 (they stay unstable), so
    # that only a recomputation equal to DeepPoly's restores them
    for i in range(2, net.R + 1):
        unst = (l[i] < 0) & (u[i] > 0)
        span = (u[i] - l[i]) + 1.0
        node.l[i] = torch.where(unst, l[i] - span, l[i])
        node.u[i] = torch.where(unst, u[i] + span, u[i])
    rows = core.optimize_intermediate(net, node, lo_t, hi_t, core.AdamHP(steps=0))
    assert rows > 0
    for i in range(1, net.R + 1):
        assert torch.allclose(node.l[i], l[i], rtol=0, atol=1e-12), f"layer {i} lower"
        assert torch.allclose(node.u[i], u[i], rtol=0, atol=1e-12), f"layer {i} upper"


def _mnc_case(seed, dims=(10, 14, 12, 10, 3), eps=0.15):
    """A case whose layers carry multi-neuron constraints (Sec. 2.3)."""
    from oracle import mnc
    L = synth.tiny_fc_net(seed, list(dims))
    rng = np.random.default_rng(seed + 100)
    x0 = rng.uniform(0.2, 0.8, dims[0]).astype(np.float32)
    y = synth.net_forward(L, x0)
    C, d = synth.property_rows(int(np.argmax(y)), dims[-1])
    lo, hi = synth.input_box(x0, eps)
    prep = bab.prepare(L, C, d, lo, hi, mnc.mnc_fn(40))
    assert prep[7] and any(prep[7][i][2].numel() > 0 for i in prep[7] if i < prep[0].R)
    return prep, lo, hi


@pytest.mark.parametrize("seed", [7, 8])
def test_gamma_sets_sound_and_zero_steps_give_deeppoly(seed):
    """With multi-neuron constraints in the shared sets (gamma_i of the layers
    below t, started at 0), zero Adam steps still give the DeepPoly bounds (the
    start point has gamma = 0), and optimised bounds contain every sampled
    pre-activation and are never looser than DeepPoly."""
    prep, lo, hi = _mnc_case(seed)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    node = bab.root_node(net, 0, l, u, S, m)
    core.optimize_intermediate(net, node, lo_t, hi_t, core.AdamHP(steps=0), dense_mnc=dense)
    for i in range(1, net.R + 1):
        assert torch.allclose(node.l[i], l[i], rtol=0, atol=1e-12)
        assert torch.allclose(node.u[i], u[i], rtol=0, atol=1e-12)
    node = bab.root_node(net, 0, l, u, S, m)
    rows = core.optimize_intermediate(net, node, lo_t, hi_t, core.AdamHP(steps=20), dense_mnc=dense)
    assert rows > 0
    for i in node.l:
        assert bool((node.l[i] >= l[i]).all()) and bool((node.u[i] <= u[i]).all())
    rng = np.random.default_rng(seed)
    X = rng.uniform(lo, hi, size=(20000, lo.size))
    h = _t(X)
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h)
        assert bool((zh >= node.l[i] - 1e-9).all()), f"layer {i}: lower bound above a sample"
        assert bool((zh <= node.u[i] + 1e-9).all()), f"layer {i}: upper bound below a sample"
        h = torch.clamp(zh, min=0)


@pytest.mark.parametrize("side", [1, -1])
def test_gamma_gradient_matches_finite_differences(side):
    """The shared set's gradient w.r.t. gamma_i (constraint multipliers of layer
    i < t) is the derivative of the summed row bounds: autograd against
    central differences at an interior point (gamma > 0)."""
    prep, lo, hi = _mnc_case(7)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    node = bab.root_node(net, 0, l, u, S, m)
    t = net.R
    idx = torch.nonzero((l[t] < 0) & (u[t] > 0)).reshape(-1)
    if idx.numel() == 0:
        idx = torch.arange(l[t].numel())
    rng = np.random.default_rng(3)
    alpha = {i: _t(rng.uniform(0.2, 0.8, l[i].numel())) for i in range(1, t)}
    beta = {i: torch.zeros(l[i].numel(), dtype=DT) for i in range(1, t)}
    gamma = {i: _t(rng.uniform(0.05, 0.3, dense[i][2].numel() if i in dense else 0))
             for i in range(1, t)}
    _, _, _, gg = core.intermediate_objective_grad(net, node, t, idx, side, alpha, beta,
                                                   lo_t, hi_t, gamma, dense)

    def f(g):
        return float(core.intermediate_objective(net, node, t, idx, side, alpha, beta,
                                                 lo_t, hi_t, g, dense).sum())

    h = 1e-6
    checked = nonzero = 0
    for i in range(1, t):
        for k in range(0, gamma[i].numel(), max(1, gamma[i].numel() // 12)):
            gp = {a: v.clone() for a, v in gamma.items()}
            gm = {a: v.clone() for a, v in gamma.items()}
            gp[i][k] += h
            gm[i][k] -= h
            fd = (f(gp) - f(gm)) / (2 * h)
            assert abs(fd - float(gg[i][k])) <= 1e-6 * (1 + abs(fd)), (i, k, fd, float(gg[i][k]))
            checked += 1
            nonzero += abs(fd) > 1e-9
    assert checked > 5 and nonzero > 0
