"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test targets a plausible mistake: a dropped or mis-signed term of the
ReLU back-substitution (Sec. 3.1), a transposed or mis-padded convolution, a
wrong concretisation (Eq. minimum), a wrong x* (Sec. 3.1 upper bounding), an
unsound multi-neuron constraint, a wrong gradient, or a wrong ACS formula
(Sec. 3.2).  None of these tests calls the GPU library.
"""
import itertools
import math

import numpy as np
import pytest
import torch
from scipy.optimize import linprog

import synth
from oracle import bab, core, exact, mnc
from oracle.core import DT

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def _fc(W, b):
    return dict(kind="fc", W=np.asarray(W, np.float32), b=np.asarray(b, np.float32))


RELU = dict(kind="relu")


# --------------------------------------------------------------------------
# affine layers and concretisation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ci,h,co,k,s,p", [(1, 28, 16, 4, 2, 0), (16, 13, 32, 4, 2, 0),
                                           (3, 9, 5, 3, 1, 1), (4, 8, 6, 4, 2, 1)])
def test_conv_forward_and_adjoint(ci, h, co, k, s, p):
    """Conv forward equals the direct definition (synth's numpy loops), and the
    back-substitution is its exact adjoint: <L, conv x> = <conv^T L, x>."""
    rng = np.random.default_rng(5)
    ho = (h + 2 * p - k) // s + 1
    L = dict(kind="conv", W=rng.standard_normal((co, ci, k, k)).astype(np.float32),
             b=rng.standard_normal(co).astype(np.float32), stride=s, pad=p,
             in_shape=(ci, h, h), out_shape=(co, ho, ho))
    net = core.load_net([L])
    A = net.aff[1]
    x = rng.standard_normal(ci * h * h)
    ref = synth.net_forward([L], x)
    got = A.forward(_t(x)[None])[0].numpy()
    assert np.allclose(got, ref, atol=1e-10)
    lam = _t(rng.standard_normal((3, co * ho * ho)))
    lin = A.forward(_t(x)[None]) - A.forward(torch.zeros(1, ci * h * h, dtype=DT))
    lhs = (lam * lin).sum(1)
    rhs = A.backsub(lam) @ _t(x)
    assert torch.allclose(lhs, rhs, atol=1e-9)
    bias_full = A.forward(torch.zeros(1, ci * h * h, dtype=DT))[0]
    assert torch.allclose(A.bias_dot(lam), lam @ bias_full, atol=1e-10)


def test_affine_only_is_exact_and_hoelder():
    """One affine layer: the bound is the exact minimum over the box, and without
    clipping it is the Hoelder form a x0 - ||a||_1 eps + c (Eq. minimum)."""
    rng = np.random.default_rng(1)
    W = rng.standard_normal((4, 6))
    b = rng.standard_normal(4)
    net = core.load_net([_fc(W, b)])
    x0 = rng.uniform(0.3, 0.7, 6)
    eps = 0.1
    lo, hi = synth.input_box(x0, eps)
    lb, xs, _ = core.backsub_rows(net, 1, torch.eye(4, dtype=DT), {}, _t(lo), _t(hi))
    Wf, bf = W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    corners = np.array(list(itertools.product(*zip(lo, hi))), dtype=np.float64)
    brute = (corners @ Wf.T + bf).min(0)
    assert np.allclose(lb.numpy(), brute, atol=1e-12)
    x0f = x0.astype(np.float32).astype(np.float64)
    hoelder = Wf @ x0f - np.abs(Wf).sum(1) * np.float64(np.float32(eps)) + bf
    assert np.allclose(lb.numpy(), hoelder, atol=1e-6)
    # x* attains the bound
    assert np.allclose((xs.numpy() * Wf).sum(1) + bf, lb.numpy(), atol=1e-12)


# --------------------------------------------------------------------------
# the single-neuron table by hand (Sec. 3.1)
# --------------------------------------------------------------------------
def _one_neuron(w, c):
    return [_fc([[1.0]], [0.0]), RELU, _fc([[w]], [c])]


def test_relu_table_positive_coefficient():
    """f = 3 relu(x) + 1, x in [-1, 2]: DeepPoly slope 1 gives -2; the alpha
    bound is 1 - 3 alpha, so Adam drives alpha to 0 and reaches the exact 1."""
    L = _one_neuron(3.0, 1.0)
    net, lo, hi, l, u, S, m, dense = bab.prepare(L, [[1.0]], [0.0], [-1.0], [2.0])
    assert float(l[1][0]) == -1.0 and float(u[1][0]) == 2.0
    node = bab.root_node(net, 0, l, u, S, None)
    lb_dp, _ = core.deeppoly_final(net, node, lo, hi)
    assert float(lb_dp) == pytest.approx(-2.0, abs=1e-12)
    for a in (0.0, 0.25, 0.6):
        lb, _, _ = core.final_bound(net, node, {1: _t([a])}, {1: _t([0.0])},
                                    {1: torch.zeros(0, dtype=DT)}, None, lo, hi)
        assert float(lb) == pytest.approx(1.0 - 3.0 * a, abs=1e-12)
    best, _, a, _, _ = core.optimize(net, node, None, lo, hi, core.AdamHP())
    assert best == pytest.approx(1.0, abs=1e-12)
    assert float(a[1][0]) == 0.0


@pytest.mark.parametrize("sign", [1, -1])
def test_standard_adam_closed_form(sign):
    """Projected Adam (Sec. 3.1, projected gradient ascent) on a split neuron.

    f = relu(x), x in [0.5, 1]; the neuron is split with S = sign.  Then
    ahat = D + beta S (D = 0 for S = +1, 1 for S = -1) and
    lb(beta) = min_x (D + beta S) x, whose gradient is constant in beta >= 0:
    +lo = 0.5 for S = +1 (x* = lo) and -lo for S = -1.
    With a constant gradient g, bias-corrected Adam has m_hat = g and
    v_hat = g^2 at every step, so each step is exactly lr g / (|g| + eps):
    three steps give beta = 3 lr g / (|g| + 1e-8) for S = +1 (the gradient-
    scaled eps option would give 3 lr / 1.001; no bias correction a first step
    3x larger), and for S = -1 the projection keeps beta at 0."""
    L = _one_neuron(1.0, 0.0)
    net, lo, hi, l, u, S, m, dense = bab.prepare(L, [[1.0]], [0.0], [0.5], [1.0])
    node = bab.root_node(net, 0, l, u, S, None)
    node.S[1][0] = sign
    if sign == 1:
        node.u[1][0] = 0.0
    hp = core.AdamHP(steps=3)
    best, _, _, beta, _ = core.optimize(net, node, None, lo, hi, hp)
    if sign == 1:
        g = 0.5
        expect = 3 * hp.lr_beta * g / (g + 1e-8)
        assert float(beta[1][0]) == pytest.approx(expect, rel=1e-14)
        assert best == pytest.approx(0.5 * expect, rel=1e-14)
        assert abs(float(beta[1][0]) - 3 * hp.lr_beta / 1.001) > 1e-4
    else:
        assert float(beta[1][0]) == 0.0
        assert best == pytest.approx(0.5, abs=1e-15)
    # the named option changes exactly the denominator
    _, _, _, beta_r, _ = core.optimize(net, node, None, lo, hi, core.AdamHP(steps=3, eps_rel=1e-3))
    if sign == 1:
        assert float(beta_r[1][0]) == pytest.approx(3 * hp.lr_beta * 0.5 / (0.5 + 0.5e-3),
                                                    rel=1e-12)


def test_adam_returns_the_best_iterate():
    """The optimiser reports the best bound over its iterates (Sec. 3.1: every
    parameter setting gives a valid bound).  f = relu(x) - 0.375 x on [-1, 1],
    the linear part through a stable neuron z2 = x + 2:
    lb(alpha) = -|alpha - 0.375|, maximal inside (0, 1).  From alpha = 1
    Adam's first steps have a constant gradient, so each is lr = 0.1 long;
    the sixth reaches alpha = 0.4 (lb = -0.025) and momentum then carries
    alpha past the optimum.  The reported bound is at least -0.025, longer
    runs never report less, and none exceeds the exact minimum 0."""
    L = [_fc([[1.0], [1.0]], [0.0, 2.0]), RELU, _fc([[1.0, -0.375]], [0.75])]
    net, lo, hi, l, u, S, _, _ = bab.prepare(L, [[1.0]], [0.0], [-1.0], [1.0])
    assert float(l[1][1]) > 0 and float(l[1][0]) < 0 < float(u[1][0])
    node = bab.root_node(net, 0, l, u, S, None)
    for a in (0.0, 0.375, 0.8):
        lb, _, _ = core.final_bound(net, node, {1: _t([a, 1.0])}, {1: _t([0.0, 0.0])},
                                    {1: torch.zeros(0, dtype=DT)}, None, lo, hi)
        assert float(lb) == pytest.approx(-abs(a - 0.375), abs=1e-12)
    prev = -math.inf
    for steps in (6, 12, 20, 30):
        best, *_ = core.optimize(net, node, None, lo, hi, core.AdamHP(steps=steps))
        assert best >= -0.025 - 1e-7  # steps are lr / (1 + eps / |g|) long
        assert best <= 1e-12
        assert best >= prev
        prev = best


def test_multi_neuron_terms_by_hand():
    """The gamma terms of the ReLU step (Sec. 3.1, enforcing multi-neuron
    constraints) by hand.  x in [-1, 1], zhat = x, y = relu(x), f = w y, one
    constraint y - 0.5 zhat - 0.5 <= 0 (the triangle's upper facet) with
    multiplier g.  The bound adds g (y - 0.5 zhat - 0.5) to f, so the
    coefficient on y is a' = w + g, the one on zhat gains -0.5 g and the offset
    -0.5 g.  With a' >= 0 the lower slope alpha applies:
    lb = -|a' alpha - 0.5 g| - 0.5 g; with a' < 0 the upper line (slope 1/2,
    intercept 1/2) applies: lb = -|0.5 a' - 0.5 g| + 0.5 a' - 0.5 g."""
    m = core.MNC(np.array([[0]]), np.array([[1.0]]), np.array([[-0.5]]), np.array([0.5]))
    dense = {1: m.dense(1)}
    for w in (1.0, -1.0):
        net, lo, hi, l, u, S, _, _ = bab.prepare(_one_neuron(w, 0.0), [[1.0]], [0.0], [-1.0], [1.0])
        node = bab.root_node(net, 0, l, u, S, None)
        for a, g in ((0.5, 1.0), (0.25, 2.0), (0.8, 0.3), (0.1, 0.0)):
            lb, _, _ = core.final_bound(net, node, {1: _t([a])}, {1: _t([0.0])}, {1: _t([g])},
                                        dense, lo, hi)
            ap = w + g
            if ap >= 0:
                ref = -abs(ap * a - 0.5 * g) - 0.5 * g
            else:
                ref = -abs(0.5 * ap - 0.5 * g) + 0.5 * ap - 0.5 * g
            assert float(lb) == pytest.approx(ref, abs=1e-12), (w, a, g)


def test_relu_table_negative_coefficient():
    """f = -2 relu(x) + 5, x in [-1, 2]: the upper line u/(u-l)(x - l) with
    intercept -ul/(u-l) = 2/3 gives the exact minimum 1."""
    L = _one_neuron(-2.0, 5.0)
    net, lo, hi, l, u, S, _, _ = bab.prepare(L, [[1.0]], [0.0], [-1.0], [2.0])
    node = bab.root_node(net, 0, l, u, S, None)
    lb, xs = core.deeppoly_final(net, node, lo, hi)
    assert float(lb) == pytest.approx(1.0, abs=1e-12)
    assert float(xs[0]) == 2.0


def test_relu_table_two_neurons_and_splits():
    """f = relu(x1+x2) + relu(x1-x2) on [-1,1]^2 has bound -2 max(alpha); the
    negative objective -relu(x1+x2) is exact (-2); a negative split (S=+1)
    gives -2 beta (best 0) and a positive split gives -2 (1 + beta)."""
    W1 = [[1.0, 1.0], [1.0, -1.0]]
    L = [_fc(W1, [0, 0]), RELU, _fc([[1.0, 1.0]], [0.0])]
    net, lo, hi, l, u, S, _, _ = bab.prepare(L, [[1.0]], [0.0], [-1, -1], [1, 1])
    node = bab.root_node(net, 0, l, u, S, None)
    for a1, a2 in ((1, 1), (0.3, 0.7), (0, 0), (0.9, 0.1)):
        lb, _, _ = core.final_bound(net, node, {1: _t([a1, a2])}, {1: _t([0, 0])},
                                    {1: torch.zeros(0, dtype=DT)}, None, lo, hi)
        assert float(lb) == pytest.approx(-2 * max(a1, a2), abs=1e-12)
    L2 = [_fc(W1, [0, 0]), RELU, _fc([[-1.0, 0.0]], [0.0])]
    net, lo, hi, l, u, S, _, _ = bab.prepare(L2, [[1.0]], [0.0], [-1, -1], [1, 1])
    node = bab.root_node(net, 0, l, u, S, None)
    lb, _ = core.deeppoly_final(net, node, lo, hi)
    assert float(lb) == pytest.approx(-2.0, abs=1e-12)
    for sgn, f_beta in ((1, lambda b: -2 * b), (-1, lambda b: -2 * (1 + b))):
        n2 = bab.root_node(net, 0, l, u, S, None)
        n2.S[1] = torch.tensor([sgn, 0], dtype=torch.int8)
        if sgn == 1:
            n2.u[1] = torch.minimum(n2.u[1], _t([0.0, 1e9]))
        else:
            n2.l[1] = torch.maximum(n2.l[1], _t([0.0, -1e9]))
        for bval in (0.0, 0.5, 2.0):
            lb, _, _ = core.final_bound(net, n2, {1: _t([0.5, 0.5])}, {1: _t([bval, 0])},
                                        {1: torch.zeros(0, dtype=DT)}, None, lo, hi)
            assert float(lb) == pytest.approx(f_beta(bval), abs=1e-12)


# --------------------------------------------------------------------------
# soundness, exactness and gradients on small nets
# --------------------------------------------------------------------------
def _small_case(seed, dims=(12, 10, 10, 3), eps=0.08, with_mnc=True):
    L = synth.tiny_fc_net(seed, list(dims))
    rng = np.random.default_rng(seed + 100)
    x0 = rng.uniform(0.2, 0.8, dims[0]).astype(np.float32)
    y = synth.net_forward(L, x0)
    C, d = synth.property_rows(int(np.argmax(y)), dims[-1])
    lo, hi = synth.input_box(x0, eps)
    fn = mnc.mnc_fn() if with_mnc else None
    prep = bab.prepare(L, C, d, lo, hi, fn)
    return L, C, d, lo, hi, prep


def _random_node(prep, rng, n_splits=2, row=0):
    net, lo, hi, l, u, S, m, dense = prep
    node = bab.root_node(net, row, l, u, S, m)
    cands = [(i, j) for i in l for j in range(l[i].numel()) if l[i][j] < 0 < u[i][j]]
    picks = [cands[k] for k in rng.choice(len(cands), size=min(n_splits, len(cands)), replace=False)]
    low = min(p[0] for p in picks) if picks else net.R
    for (i, j) in picks:
        sgn = int(rng.choice([1, -1]))
        node.S[i][j] = sgn
        if sgn == 1:
            node.u[i][j] = 0.0
        else:
            node.l[i][j] = 0.0
    node.split_layer = low
    core.rebound_node(net, node, lo, hi)
    node.alpha = {i: _t(rng.uniform(0, 1, l[i].numel())) for i in l}
    node.beta = {i: _t(rng.uniform(0, 1, l[i].numel())) * (node.S[i] != 0) for i in l}
    node.gamma = {i: _t(rng.uniform(0, 0.2, node.gamma[i].numel())) for i in l}
    return node


def _in_subdomain(net, node, X):
    """Rows of X satisfying the node's split signs."""
    keep = np.ones(X.shape[0], bool)
    h = _t(X)
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h)
        S = node.S[i].numpy()
        z = zh.numpy()
        keep &= np.all((S[None, :] != 1) | (z <= 0), axis=1)
        keep &= np.all((S[None, :] != -1) | (z >= 0), axis=1)
        h = torch.clamp(zh, min=0)
    return keep


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_soundness_random_parameters(seed):
    """Every 0 <= alpha <= 1, beta, gamma >= 0 gives a sound bound (Sec. 3.1):
    lb <= f_r at 10^4 samples of the subdomain and at x*; root bounds contain
    every sampled pre-activation."""
    L, C, d, lo, hi, prep = _small_case(seed, eps=0.15)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    assert m, "expected multi-neuron constraints on this case"
    rng = np.random.default_rng(seed)
    X = rng.uniform(lo, hi, size=(10000, lo.size))
    h = _t(X)
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h)
        assert bool((zh >= l[i] - 1e-9).all()) and bool((zh <= u[i] + 1e-9).all())
        h = torch.clamp(zh, min=0)
    for trial in range(4):
        node = _random_node(prep, rng, n_splits=trial)
        lb, xs, _ = core.final_bound(net, node, node.alpha, node.beta, node.gamma, dense, lo_t, hi_t)
        keep = _in_subdomain(net, node, X)
        f = net.forward(_t(X[keep]))[:, node.row].numpy()
        if f.size:
            assert float(lb) <= f.min() + 1e-9
        # intermediate bounds of the node contain the subdomain's pre-activations
        h = _t(X[keep])
        for i in range(1, net.R + 1):
            zh = net.aff[i].forward(h)
            assert bool((zh >= node.l[i] - 1e-9).all()) and bool((zh <= node.u[i] + 1e-9).all())
            h = torch.clamp(zh, min=0)


@pytest.mark.parametrize("seed", [3, 4])
def test_lower_bounds_below_exact_minimum(seed):
    """2->8->8->2: DeepPoly and optimised bounds never exceed the exact minimum
    from activation-pattern enumeration with an LP per pattern."""
    L, C, d, lo, hi, prep = _small_case(seed, dims=(2, 8, 8, 2), eps=0.15)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    ex, xarg = exact.exact_min(L, C, d, 0, lo, hi)
    node = bab.root_node(net, 0, l, u, S, m)
    lb_dp, _ = core.deeppoly_final(net, node, lo_t, hi_t)
    best, bx, *_ = core.optimize(net, node, dense, lo_t, hi_t, core.AdamHP(steps=40))
    assert float(lb_dp) <= ex + 1e-9
    assert best <= ex + 1e-9
    assert best >= float(lb_dp) - 1e-12


@pytest.mark.parametrize("seed", [5, 6])
def test_fully_split_leaf_reaches_lp_optimum(seed):
    """Completeness limit (Sec. 3.3): once every unstable neuron is split the
    relaxation is exact and optimising beta approaches the LP optimum of the
    subproblem from below."""
    L, C, d, lo, hi, prep = _small_case(seed, dims=(2, 6, 6, 2), eps=0.2, with_mnc=False)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    rng = np.random.default_rng(seed)
    X = rng.uniform(lo, hi, size=(1, 2))
    # split every unstable neuron by the pattern of a sampled point (feasible leaf)
    node = bab.root_node(net, 0, l, u, S, None)
    h = _t(X)
    splits = {}
    for i in range(1, net.R + 1):
        zh = net.aff[i].forward(h)[0]
        for j in range(zh.numel()):
            if node.l[i][j] < 0 < node.u[i][j]:
                sgn = 1 if zh[j] <= 0 else -1
                node.S[i][j] = sgn
                splits[(i, j)] = sgn
                if sgn == 1:
                    node.u[i][j] = 0.0
                else:
                    node.l[i][j] = 0.0
        h = torch.clamp(zh[None], min=0)
    ex, _ = exact.exact_min(L, C, d, 0, lo, hi, splits=splits)
    best, *_ = core.optimize(net, node, None, lo_t, hi_t, core.AdamHP(steps=600, lr_beta=0.02))
    assert best <= ex + 1e-9
    assert best >= ex - 2e-2 * (1 + abs(ex))


def test_gradient_matches_finite_differences():
    """Reverse-mode gradient of the bound w.r.t. alpha, beta, gamma equals
    central finite differences (FP64, h = 1e-6) away from case switches."""
    L, C, d, lo, hi, prep = _small_case(7)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    rng = np.random.default_rng(7)
    node = _random_node(prep, rng, n_splits=2)
    lb, _, ga, gb, gg = core.bound_and_grad(net, node, node.alpha, node.beta, node.gamma,
                                            dense, lo_t, hi_t)

    def f(al, be, gm):
        v, _, _ = core.final_bound(net, node, al, be, gm, dense, lo_t, hi_t)
        return float(v)

    h = 1e-6
    checked = 0
    for grp, G in (("a", ga), ("b", gb), ("g", gg)):
        for i in G:
            nz = torch.nonzero(G[i]).reshape(-1)
            for j in nz[:6].tolist():
                P = [{k: v.clone() for k, v in D.items()} for D in (node.alpha, node.beta, node.gamma)]
                M = [{k: v.clone() for k, v in D.items()} for D in (node.alpha, node.beta, node.gamma)]
                gi = "abg".index(grp)
                P[gi][i][j] += h
                M[gi][i][j] -= h
                fd = (f(*P) - f(*M)) / (2 * h)
                # FP64 central differences carry a rounding error of about
                # eps |f| / h = 2e-16 * 10 / 1e-6 = 2e-9 on this net's bounds
                assert fd == pytest.approx(float(G[i][j]), rel=1e-6, abs=1e-8)
                checked += 1
    assert checked >= 10


# --------------------------------------------------------------------------
# multi-neuron constraints
# --------------------------------------------------------------------------
def test_mnc_rows_are_sound_per_orthant():
    """Every constraint row holds on {octahedron and orthant} (LP per orthant)
    and at sampled network activations."""
    L, C, d, lo, hi, prep = _small_case(8)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    t = sorted(m)[0]
    rows = m[t]
    groups = sorted(set(map(tuple, rows.idx.tolist())))[:3]
    ob = mnc.octahedron_bounds(net, t, groups, l, u, S, lo_t, hi_t)
    for G, lbs in zip(groups, ob):
        sel = np.nonzero((rows.idx == np.array(G)).all(1))[0]
        for e in sel[:40]:
            for sig in itertools.product((-1.0, 1.0), repeat=3):
                sig = np.array(sig)
                # variables x (3); y = x on positive coordinates, 0 otherwise
                cy = np.where(sig > 0, rows.P[e], 0.0)
                obj = -(cy + rows.Ph[e])
                A_ub = np.concatenate([-mnc.DIRS, -np.diag(sig)])
                b_ub = np.concatenate([-lbs, np.zeros(3)])
                r = linprog(obj, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * 3, method="highs")
                if r.status == 0:
                    assert -r.fun <= rows.p[e] + 1e-9
    rng = np.random.default_rng(8)
    X = _t(rng.uniform(lo, hi, size=(5000, lo.size)))
    h = X
    for i in range(1, t + 1):
        zh = net.aff[i].forward(h)
        h = torch.clamp(zh, min=0)
    z, zh = h.numpy(), zh.numpy()
    viol = (rows.P * z[:, rows.idx]).sum(-1) + (rows.Ph * zh[:, rows.idx]).sum(-1) - rows.p
    assert viol.max() <= 1e-9


# --------------------------------------------------------------------------
# branching and counterexamples
# --------------------------------------------------------------------------
def test_acs_scores_by_hand():
    """s_j = |(gamma^T P)_j| + |(gamma^T Phat)_j| over unstable unsplit neurons
    (Sec. 3.2); ties go to the lowest (layer, index)."""
    l = {1: _t([-1, -1, -1, 1]), 2: _t([-1, -1])}
    u = {1: _t([1, 1, 1, 2]), 2: _t([1, 1])}
    S = {1: torch.zeros(4, dtype=torch.int8), 2: torch.tensor([0, -1], dtype=torch.int8)}
    m1 = core.MNC(np.array([[0, 1, 2], [0, 1, 2]]), np.array([[1.0, 0, 0], [0, -2.0, 0]]),
                  np.array([[0, 0, 1.0], [0, 0, 0]]), np.array([0.0, 0.0]))
    m2 = core.MNC(np.array([[0, 1, 0]]), np.array([[0.0, 3.0, 0]]), np.array([[0.1, 0, 0]]),
                  np.array([0.0]))
    dense = {1: m1.dense(4), 2: m2.dense(2)}
    node = core.Node(0, l, u, S, {}, {}, {}, split_layer=2)
    gamma = {1: _t([0.5, 0.3]), 2: _t([2.0])}
    sc, fb = core.acs_scores(node, gamma, dense, None)
    assert not fb
    assert np.allclose(sc[1].numpy()[:3], [0.5, 0.6, 0.5])
    assert sc[1][3] == -math.inf and sc[2][1] == -math.inf   # stable / split
    assert float(sc[2][0]) == pytest.approx(0.2)
    assert core.pick_split(sc)[:2] == (1, 1)
    gamma = {1: _t([0.5, 0.25]), 2: _t([0.0])}
    sc, _ = core.acs_scores(node, gamma, dense, None)
    assert core.pick_split(sc)[:2] == (1, 0)    # three-way tie at 0.5
    # no active constraint: intercept fallback |a'_j| (-l u / (u - l))
    gamma = {1: _t([0.0, 0.0]), 2: _t([0.0])}
    aps = {1: _t([[1.0, -3.0, 0.5, 9.0]]), 2: _t([[0.1, 5.0]])}
    sc, fb = core.acs_scores(node, gamma, dense, aps)
    assert fb and np.allclose(sc[1].numpy()[:3], [0.5, 1.5, 0.25])
    assert core.pick_split(sc)[:2] == (1, 1)
    # the fallback's intercept -l u / (u - l) with l != -1: 2/3, 3/4, 3/4
    node3 = core.Node(0, {1: _t([-2, -1, -3, 1]), 2: _t([-1, -1])},
                      {1: _t([1, 3, 1, 2]), 2: _t([1, 1])}, S, {}, {}, {}, split_layer=2)
    sc, fb = core.acs_scores(node3, gamma, dense, aps)
    assert fb and np.allclose(sc[1].numpy()[:3], [2.0 / 3.0, 2.25, 0.375])
    # ties: within 1e-5 (relative) of the maximum the lowest (layer, index)
    # wins; beyond the band the maximum does
    assert core.pick_split({1: _t([0.5, 0.5 * (1 + 1e-6)])})[:2] == (1, 0)
    assert core.pick_split({1: _t([0.5, 0.5 * (1 + 1e-4)])})[:2] == (1, 1)
    assert core.pick_split({1: _t([0.1]), 2: _t([0.1 * (1 + 1e-6)])})[:2] == (1, 0)


def test_folded_property_is_the_margin():
    """Folding C f(x) + d into the last affine layer (Sec. 2.1) gives a network
    whose outputs are the margins, by the generator's own numpy forward pass;
    the last layer's bias is large here so that a dropped C b shows."""
    L = synth.tiny_fc_net(12, [5, 7, 4])
    L[-1]["b"] = np.array([1.0, -2.0, 0.5, 3.0], np.float32)
    C, d = synth.property_rows(2, 4)
    d = d + np.array([0.25, -0.5, 1.0], np.float32)
    folded = core.fold_property(core.load_net(L), C, d)
    X = np.random.default_rng(12).uniform(-1, 1, size=(20, 5))
    got = folded.forward(_t(X)).numpy()
    ref = np.stack([C.astype(np.float64) @ synth.net_forward(L, x) + d for x in X])
    assert np.allclose(got, ref, atol=1e-10)


def test_bab_root_verdict_uses_the_optimised_bound():
    """f = 3 relu(x) + 1 on [-1, 2]: DeepPoly gives -2 and the optimised slope 0
    the exact 1 > 0, so BaB verifies at the root with one node bounded; it
    branches only when the optimised bound does not decide (Sec. 3.1, then
    Sec. 3.2)."""
    res = bab.verify(_one_neuron(3.0, 1.0), np.array([[1.0]]), np.array([0.0]),
                     np.array([-1.0]), np.array([2.0]), max_nodes=10)
    assert res.verdict == bab.VERIFIED and res.n_bounded == 1
    assert res.nodes[0].lb_dp == pytest.approx(-2.0, abs=1e-12)
    assert res.nodes[0].lb == pytest.approx(1.0, abs=1e-12)


def test_counterexamples_are_real():
    """Every FALSIFIED verdict carries x* in the box with f_r(x*) < 0 under an
    independent float64 forward pass (Sec. 3.1, upper bounding)."""
    L = synth.tiny_fc_net(11, [16, 12, 12, 4])
    n_fals = 0
    for p in range(6):
        x0 = np.random.default_rng(200 + p).uniform(0.2, 0.8, 16).astype(np.float32)
        y = synth.net_forward(L, x0)
        C, d = synth.property_rows(int(np.argmax(y)), 4)
        lo, hi = synth.input_box(x0, 0.25)
        r = bab.verify(L, C, d, lo, hi, max_nodes=20, hp=core.AdamHP(steps=5))
        # every node's f(x*) is its own row's margin at its x*
        for nd in r.nodes:
            m = C.astype(np.float64) @ synth.net_forward(L, nd.xstar) + d
            assert nd.f_xstar == pytest.approx(m[nd.row], abs=1e-6 * (1 + abs(m[nd.row])))
        if r.verdict == bab.FALSIFIED:
            n_fals += 1
            nr = r.nodes[-1]
            assert np.all(nr.xstar >= lo - 1e-12) and np.all(nr.xstar <= hi + 1e-12)
            m = C @ synth.net_forward(L, nr.xstar) + d
            assert m[nr.row] < 0
    assert n_fals >= 1
    # the check at x* uses the node's own row, on every row of a property
    x0 = np.random.default_rng(210).uniform(0.2, 0.8, 16).astype(np.float32)
    C, d = synth.property_rows(int(np.argmax(synth.net_forward(L, x0))), 4)
    lo, hi = synth.input_box(x0, 0.05)
    net, lo_t, hi_t, l, u, S, m_, dense = bab.prepare(L, C, d, lo, hi)
    for row in range(C.shape[0]):
        nr, _ = bab.bound_node(net, bab.root_node(net, row, l, u, S, None), None, lo_t, hi_t,
                               core.AdamHP(steps=2))
        m = C.astype(np.float64) @ synth.net_forward(L, nr.xstar) + d
        assert nr.row == row
        assert nr.f_xstar == pytest.approx(m[row], abs=1e-6 * (1 + abs(m[row])))


def test_children_keep_earlier_bounds():
    """Bounds of layers up to and including the split layer are not recomputed
    (Sec. 3.2, enforcing splits); later layers only tighten."""
    L, C, d, lo, hi, prep = _small_case(9, with_mnc=False)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    node = bab.root_node(net, 0, l, u, S, None)
    j = int(torch.nonzero((l[1] < 0) & (u[1] > 0))[0])
    kids = bab.children(node, (node.alpha, node.beta, node.gamma), (1, j, 0.0), 1)
    for ch in kids:
        core.rebound_node(net, ch, lo_t, hi_t)
        assert torch.equal(ch.l[1][torch.arange(l[1].numel()) != j], l[1][torch.arange(l[1].numel()) != j])
        assert bool((ch.l[2] >= l[2] - 1e-12).all()) and bool((ch.u[2] <= u[2] + 1e-12).all())
    assert float(kids[0].u[1][j]) == 0.0 and int(kids[0].S[1][j]) == 1
    assert float(kids[1].l[1][j]) == 0.0 and int(kids[1].S[1][j]) == -1


def test_rebound_after_split_is_exact_on_single_neurons():
    """Re-bounding after a split (Sec. 3.2) by hand: x in [-1, 1], z1 = x,
    z2 = relu(z1) - 0.5, f = relu(z2).  At the root DeepPoly gives
    z2 in [-1.5, 0.5] (lower slope 1 since u1 = -l1; upper line (x + 1) / 2).
    Splitting z1 <= 0 makes relu(z1) = 0, so the re-bounded z2 is exactly
    -0.5; splitting z1 >= 0 makes the ReLU the identity, and with beta = 0
    the re-bounding sees z1 = x over the whole box: z2 in [-1.5, 0.5]."""
    L = [_fc([[1.0]], [0.0]), RELU, _fc([[1.0]], [-0.5]), RELU, _fc([[1.0]], [0.0])]
    net, lo, hi, l, u, S, _, _ = bab.prepare(L, [[1.0]], [0.0], [-1.0], [1.0])
    assert (float(l[1][0]), float(u[1][0])) == (-1.0, 1.0)
    assert float(l[2][0]) == pytest.approx(-1.5, abs=1e-12)
    assert float(u[2][0]) == pytest.approx(0.5, abs=1e-12)
    node = bab.root_node(net, 0, l, u, S, None)
    neg, pos = bab.children(node, (node.alpha, node.beta, node.gamma), (1, 0, 0.0), 1)
    for ch in (neg, pos):
        core.rebound_node(net, ch, lo, hi)
    assert float(neg.l[2][0]) == pytest.approx(-0.5, abs=1e-12)
    assert float(neg.u[2][0]) == pytest.approx(-0.5, abs=1e-12)
    assert float(pos.l[2][0]) == pytest.approx(-1.5, abs=1e-12)
    assert float(pos.u[2][0]) == pytest.approx(0.5, abs=1e-12)


def test_cab_costs_by_hand():
    """CAB costs (App. B): 2 -> 3 -> 4 -> 2 net with 5 and 7 constraint rows.
    Layer costs: aff1 = 6, relu1 = 3 + 5, aff2 = 12, relu2 = 4 + 7; C_1 = 6,
    C_2 = 6 + 8 + 12 = 26; objective row: 26 + 11 + 4 = 41.  Split at layer 1
    recomputes layer 2: 41 + 2 * 4 * 26 = 249; split at layer 2: 41."""
    L = [_fc(np.ones((3, 2)), np.zeros(3)), RELU, _fc(np.ones((4, 3)), np.zeros(4)), RELU,
         _fc(np.ones((2, 4)), np.zeros(2))]
    net = core.load_net(L)
    costs = core.cab_costs(net, {1: 5, 2: 7})
    assert costs == {1: 249.0, 2: 41.0}
    # conv layers count d_out k^2
    Lc = [dict(kind="conv", W=np.ones((2, 1, 3, 3), np.float32), b=np.zeros(2, np.float32),
               stride=1, pad=0, in_shape=(1, 5, 5), out_shape=(2, 3, 3)), RELU,
          _fc(np.ones((4, 18)), np.zeros(4)), RELU, _fc(np.ones((2, 4)), np.zeros(2))]
    c2 = core.cab_costs(core.load_net(Lc))
    # aff1 = 18 * 9 = 162, relu1 = 18, aff2 = 72 -> C_2 = 252; objective 252 + 4 + 4 = 260
    assert c2 == {1: 260.0 + 2 * 4 * 252, 2: 260.0}
    sc = {1: torch.tensor([1.0, 2.0]), 2: torch.tensor([0.5, 0.1])}
    cab = core.cab_scores(sc, {1: 10.0, 2: 1.0})
    assert core.pick_split(cab)[:2] == (2, 0)


# --------------------------------------------------------------------------
# residual (ResAdd) networks
# --------------------------------------------------------------------------
def _tiny_resnet(seed, bias=0.1):
    """x(6) -> fc8 -> relu -> fc8 -> relu -> fc8 (+ fc8 shortcut from the first
    relu) -> relu -> fc3."""
    rng = np.random.default_rng(seed)
    def fc(o, i, src=None):
        d = _fc(rng.standard_normal((o, i)) * 0.6, rng.standard_normal(o) * 0.1 + bias)
        if src is not None:
            d["src"] = src
        return d
    return [fc(8, 6), RELU, fc(8, 8), RELU, fc(8, 8, 3), fc(8, 8, 1),
            dict(kind="add", src=(4, 5)), RELU, fc(3, 8)]


def test_resnet_forward_matches_definition():
    L = _tiny_resnet(0)
    net = core.load_net(L)
    assert net.R == 3 and len(net.edges[3]) == 2
    x = np.random.default_rng(1).uniform(0, 1, 6)
    assert np.allclose(net.forward(_t(x)[None])[0].numpy(), synth.net_forward(L, x), atol=1e-12)


def test_resnet_bound_is_exact_when_linear():
    """With every ReLU stable (large biases, small box) the network is affine
    on the box and the back-substituted bound through both edges of the
    residual sum equals the exact minimum of that affine map."""
    L = _tiny_resnet(5, bias=20.0)
    x0 = np.full(6, 0.5)
    lo, hi = synth.input_box(x0, 0.002)
    C, d = np.array([[1.0, -1.0, 0.0]], np.float32), np.zeros(1, np.float32)
    net, lo_t, hi_t, l, u, S, _, _ = bab.prepare(L, C, d, lo, hi)
    assert all(bool(((l[i] >= 0) | (u[i] <= 0)).all()) for i in l)
    assert any(bool((l[i] >= 0).any()) for i in l)
    node = bab.root_node(net, 0, l, u, S, None)
    lb, _ = core.deeppoly_final(net, node, lo_t, hi_t)
    # affine map by evaluating the net at the box centre and along the axes
    f = lambda x: float((C @ synth.net_forward(L, x) + d)[0])
    c0 = f(np.zeros(6))
    g = np.array([f(np.eye(6)[k]) - c0 for k in range(6)])
    exact = c0 + np.minimum(g * lo, g * hi).sum()
    assert float(lb) == pytest.approx(exact, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("seed", [3, 4])
def test_resnet_soundness_random_parameters(seed):
    L = _tiny_resnet(seed, bias=0.0)
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.2, 0.8, 6)
    y = synth.net_forward(L, x0)
    C, d = synth.property_rows(int(np.argmax(y)), 3)
    lo, hi = synth.input_box(x0, 0.3)
    net, lo_t, hi_t, l, u, S, _, _ = bab.prepare(L, C, d, lo, hi)
    X = rng.uniform(lo, hi, size=(20000, 6))
    F = np.stack([C @ synth.net_forward(L, x) + d for x in X[:4000]])
    # root bounds contain every sampled pre-activation (the residual sum included)
    z = {0: _t(X)}
    for t in range(1, net.R + 1):
        h = sum(A.forward(z[s]) for s, A in net.edges[t])
        assert bool((h >= l[t] - 1e-9).all()) and bool((h <= u[t] + 1e-9).all())
        z[t] = torch.clamp(h, min=0)
    for trial in range(3):
        node = bab.root_node(net, trial % C.shape[0], l, u, S, None)
        node.alpha = {i: _t(rng.uniform(0, 1, l[i].numel())) for i in l}
        lb, _, _ = core.final_bound(net, node, node.alpha, node.beta, node.gamma, None, lo_t, hi_t)
        assert float(lb) <= F[:, node.row].min() + 1e-9


def test_bab_without_leaf_completion_never_verifies_an_undecided_leaf():
    """With exact leaf completion off, a fully split leaf that its bound does
    not decide stays UNKNOWN, and so does its property (Sec. 3.3: only a
    decided leaf closes a branch).  On a near-critical 2-8-8-2 problem whose
    exact minimum is negative, DeepPoly-only BaB ends with undecided leaves
    and never reports VERIFIED."""
    layers, C, d, lo, hi = _tiny_problem(2, 0.34159)
    m = min(exact.exact_min(layers, C, d, r, lo, hi)[0] for r in range(C.shape[0]))
    assert m < 0
    res = bab.verify(layers, C, d, lo, hi, max_nodes=100000, hp=core.AdamHP(steps=0),
                     leaf_lp=False)
    assert any(n.split is None and n.verdict == bab.UNKNOWN for n in res.nodes)
    assert res.verdict != bab.VERIFIED


def _tiny_problem(seed, eps):
    layers = synth.tiny_fc_net(seed, [2, 8, 8, 2])
    x0 = np.random.default_rng(seed + 50).uniform(0.3, 0.7, 2).astype(np.float32)
    y = synth.net_forward(layers, x0)
    C, d = synth.property_rows(int(np.argmax(y)), 2)
    lo, hi = synth.input_box(x0, eps)
    return layers, C, d, lo, hi


# radii within 5% of a critical radius (bisection on the exact minimum), where
# the DeepPoly bound needs branching down to fully split leaves
TINY_CASES = [(2, 0.30906), (2, 0.34159), (9, 0.42384), (1, 0.30496), (11, 0.11772)]


@pytest.mark.parametrize("seed,eps", TINY_CASES)
def test_unlimited_bab_with_exact_leaves_is_complete(seed, eps):
    """Sec. 3.3 completeness: BaB with fully split leaves resolved exactly
    reproduces the sign of the exact minimum of every property row (pattern
    enumeration with one LP per pattern), here from the DeepPoly bound alone
    (no Adam steps) so that leaves are reached."""
    layers, C, d, lo, hi = _tiny_problem(seed, eps)
    m = min(exact.exact_min(layers, C, d, r, lo, hi)[0] for r in range(C.shape[0]))
    assert abs(m) > 1e-3
    res = bab.verify(layers, C, d, lo, hi, max_nodes=100000, hp=core.AdamHP(steps=0))
    assert res.verdict == (bab.VERIFIED if m > 0 else bab.FALSIFIED), (m, res.verdict)
    if seed in (2, 9):
        assert any(n.leaf for n in res.nodes)
