"""FP64 restatement of MN-BaB bounding (Sec. 3.1) -- test infrastructure only.

Notation follows the paper.  A network is a chain of affine layers
``aff[1..R+1]`` (fully connected or convolutional) with a ReLU after each of
the first R; ``aff[i]`` maps z^(i-1) to the pre-activation zhat^(i), z^(0) = x.
The linear property is folded into the last affine layer (Sec. 2.1), so each
property row r asks for min_x zhat^(R+1)_r(x) > 0.

A bound is a row vector ``a`` over some layer's neurons plus an offset ``c``
(Sec. 3.1).  Back-substitution pushes it down to the input:

* affine layer (Sec. 3.1, affine back-substitution equation):
  a^(i-1) = ahat^(i) W^(i),  c^(i-1) = ahat^(i) . b^(i) + chat^(i);
* ReLU layer (Sec. 3.1, combined ReLU back-substitution equation):
  a' = a + gamma^T P,
  ahat = a' D + beta^T S + gamma^T Phat,
  chat = a' . blow - gamma^T p + c,
  with D and blow from the single-neuron table and S from the split encoding;
* concretisation over the box [lo, hi] (Eq. minimum, here in its clipped-box
  form): lb = sum_k min(a0_k lo_k, a0_k hi_k) + c, minimiser x*_k = lo_k if
  a0_k >= 0 else hi_k (Sec. 3.1, upper bounding the minimum objective).

Readings of the paper taken here (each also listed in the design notes):

* the D / blow case split uses the sign of a' = a + gamma^T P (the primes are
  dropped "for readability" in the table); a'_j = 0 on an unstable neuron takes
  the alpha branch;
* split neurons take precedence: a positive split (S = -1, zhat >= 0) gives
  D = 1, a negative split (S = +1, zhat <= 0) gives D = 0; then l >= 0 gives 1,
  u <= 0 gives 0, and only l < 0 < u is unstable;
* the garbled offset term "(a + gamma^T P)' blow" is read as a' . blow;
* the input region is the L-inf ball clipped to [0, 1]; with no clipping the
  concretisation equals the Hoelder form a x0 - ||a||_1 eps + c exactly;
* DeepPoly's initial slope is alpha = 1 if u >= -l else 0 (area heuristic);
* intermediate bounds of a subproblem are recomputed only for layers after
  the split layer (Sec. 3.2, enforcing splits), only for neurons unstable in
  the parent, with DeepPoly slopes, beta = gamma = 0, and intersected with the
  parent's bounds; the split neuron is clamped (u <= 0 or l >= 0).

Parity: pinned by the closed forms, sampling, exact-enumeration and finite
difference tests in tests/test_oracle_*.py (see each function).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch
import torch.nn.functional as F

DT = torch.float64


# ----------------------------------------------------------------------------
# Networks
# ----------------------------------------------------------------------------
@dataclass
class Affine:
    kind: str                   # "fc" | "conv"
    W: torch.Tensor             # fc: [out, in]; conv: [Co, Ci, k, k]
    b: torch.Tensor             # fc: [out]; conv: [Co]
    stride: int = 1
    pad: int = 0
    in_shape: tuple = ()
    out_shape: tuple = ()

    @property
    def d_in(self) -> int:
        return self.W.shape[1] if self.kind == "fc" else int(np.prod(self.in_shape))

    @property
    def d_out(self) -> int:
        return self.W.shape[0] if self.kind == "fc" else int(np.prod(self.out_shape))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """zhat = W z + b for rows of x ([Q, d_in] -> [Q, d_out])."""
        if self.kind == "fc":
            return x @ self.W.T + self.b
        q = x.shape[0]
        y = F.conv2d(x.reshape(q, *self.in_shape), self.W, self.b,
                     stride=self.stride, padding=self.pad)
        return y.reshape(q, -1)

    def backsub(self, A: torch.Tensor) -> torch.Tensor:
        """A W: coefficients on zhat -> coefficients on z^(i-1)."""
        if self.kind == "fc":
            return A @ self.W
        q = A.shape[0]
        co, ho, wo = self.out_shape
        ci, hi, wi = self.in_shape
        k = self.W.shape[2]
        oph = hi - ((ho - 1) * self.stride - 2 * self.pad + k)
        opw = wi - ((wo - 1) * self.stride - 2 * self.pad + k)
        y = F.conv_transpose2d(A.reshape(q, co, ho, wo), self.W, None, stride=self.stride,
                               padding=self.pad, output_padding=(oph, opw))
        return y.reshape(q, -1)

    def bias_dot(self, A: torch.Tensor) -> torch.Tensor:
        """A . b with b broadcast over output positions ([Q, d_out] -> [Q])."""
        if self.kind == "fc":
            return A @ self.b
        co, ho, wo = self.out_shape
        return A.reshape(A.shape[0], co, ho * wo).sum(-1) @ self.b


@dataclass
class Net:
    """ReLU network as a DAG of affine edges: zhat^(t) = sum over the edges
    (s, A) into t of A(z^(s)), with z^(0) = x; ReLU layers t = 1..R, the output
    is node R + 1.  A chain has one edge (t - 1, aff[t]) per node; residual
    networks (ResAdd) have two edges into the sum after a block."""
    edges: list          # edges[t] = [(s, Affine), ...], t = 1..R+1 (edges[0] unused)

    @property
    def R(self) -> int:
        return len(self.edges) - 2

    @property
    def aff(self) -> list:
        """First edge of every node (the whole network for a chain)."""
        return [None] + [self.edges[t][0][1] for t in range(1, len(self.edges))]

    def width(self, t: int) -> int:
        return self.edges[t][0][1].d_out

    def dims(self) -> list[int]:
        """d_i of each ReLU layer i = 1..R (index 0 is the input)."""
        d0 = [A.d_in for (s, A) in self.edges[1] if s == 0][0]
        return [d0] + [self.width(i) for i in range(1, self.R + 1)]

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """Exact network output f(x) for rows of x (Eq. 1 constraints)."""
        z = {0: x}
        for t in range(1, self.R + 2):
            h = sum(A.forward(z[s]) for s, A in self.edges[t])
            z[t] = torch.clamp(h, min=0.0) if t <= self.R else h
        return z[self.R + 1]


def _affine(L) -> Affine:
    W = torch.as_tensor(np.asarray(L["W"]), dtype=DT)
    b = torch.as_tensor(np.asarray(L["b"]), dtype=DT)
    if L["kind"] == "fc":
        return Affine("fc", W, b)
    return Affine("conv", W, b, L["stride"], L["pad"], tuple(L["in_shape"]), tuple(L["out_shape"]))


def load_net(layers: list[dict]) -> Net:
    """Layer list from ``synth`` -> oracle Net in float64.

    Every op reads the previous op unless it names ``src`` (an op index);
    ``add`` sums the affine ops (or adds) listed in ``src``.  A ReLU's input is
    an affine op or a sum of them; affine ops read a ReLU output or the input.
    """
    relu_of = {}        # op index of a ReLU -> ReLU layer number
    feed = {}           # op index of an affine / add -> [(source ReLU layer, Affine)]
    edges = [[]]
    for i, L in enumerate(layers):
        k = L["kind"]
        if k == "relu":
            src = L.get("src", i - 1)
            assert src in feed, "a ReLU must read an affine layer or a sum"
            edges.append(list(feed[src]))
            relu_of[i] = len(edges) - 1
        elif k == "add":
            parts = []
            for a in L["src"]:
                assert a in feed, "add sums affine layers"
                parts += feed[a]
            feed[i] = parts
        else:
            src = L.get("src", i - 1)
            if src < 0:   # the network input
                s = 0
            else:
                assert src in relu_of, "an affine layer must read a ReLU output or the input"
                s = relu_of[src]
            feed[i] = [(s, _affine(L))]
    last = len(layers) - 1
    assert last in feed, "the network must end with an affine layer"
    edges.append(list(feed[last]))
    return Net(edges)


def fold_property(net: Net, C: np.ndarray, d: np.ndarray) -> Net:
    """Fold the linear property C f(x) + d > 0 into the last affine layer (Sec. 2.1)."""
    assert len(net.edges[-1]) == 1
    s, last = net.edges[-1][0]
    assert last.kind == "fc"
    Ct = torch.as_tensor(np.asarray(C), dtype=DT)
    dt = torch.as_tensor(np.asarray(d), dtype=DT)
    new = Affine("fc", Ct @ last.W, Ct @ last.b + dt)
    return Net(net.edges[:-1] + [[(s, new)]])


# ----------------------------------------------------------------------------
# ReLU relaxation and back-substitution
# ----------------------------------------------------------------------------
def deeppoly_alpha(l: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """DeepPoly's initial lower slope: 1 if u >= -l else 0 (reading, see header)."""
    return (u >= -l).to(DT)


def relu_cases(l, u, S):
    """Masks of the single-neuron table with split precedence (Sec. 3.1)."""
    pos_split = S == -1
    neg_split = S == 1
    one = pos_split | (~neg_split & (l >= 0))
    zero = neg_split | (~pos_split & ~(l >= 0) & (u <= 0))
    unst = ~(one | zero)
    return one, zero, unst


def relu_backsub(a, l, u, S, alpha, beta, GP=None, GPh=None, gp0=None):
    """One ReLU layer: (a on z) -> (ahat on zhat, offset increment).

    Implements ahat = (a + gamma^T P) D + beta^T S + gamma^T Phat and
    dc = (a + gamma^T P) . blow - gamma^T p (Sec. 3.1, combined ReLU step).
    ``GP = gamma^T P``, ``GPh = gamma^T Phat``, ``gp0 = gamma^T p`` per row.
    """
    ap = a if GP is None else a + GP
    one, zero, unst = relu_cases(l, u, S)
    den = torch.where(unst, u - l, torch.ones_like(u))
    slope = torch.where(unst, u / den, torch.zeros_like(u))
    icpt = torch.where(unst, -u * l / den, torch.zeros_like(u))
    neg = unst & (ap < 0)
    D = torch.where(one, torch.ones_like(ap),
                    torch.where(zero, torch.zeros_like(ap),
                                torch.where(neg, slope.expand_as(ap), alpha.expand_as(ap))))
    blow = torch.where(neg, icpt.expand_as(ap), torch.zeros_like(ap))
    ahat = ap * D + beta * S.to(DT)
    if GPh is not None:
        ahat = ahat + GPh
    dc = (ap * blow).sum(-1)
    if gp0 is not None:
        dc = dc - gp0
    return ahat, dc, ap


def concretize(A0, c, lo, hi):
    """lb = sum_k min(a0_k lo_k, a0_k hi_k) + c and x* (Eq. minimum, Sec. 3.1)."""
    xstar = torch.where(A0 >= 0, lo, hi)
    # a0 . x* equals sum_k min(a0_k lo_k, a0_k hi_k); written this way its
    # gradient w.r.t. a0 is x* itself, including the tie a0_k = 0 -> lo_k
    lb = (A0 * xstar).sum(-1) + c
    return lb, xstar


@dataclass
class Relax:
    """Parameters of one ReLU layer for a set of rows (broadcast over rows)."""
    l: torch.Tensor
    u: torch.Tensor
    S: torch.Tensor
    alpha: torch.Tensor
    beta: torch.Tensor
    GP: torch.Tensor | None = None
    GPh: torch.Tensor | None = None
    gp0: torch.Tensor | None = None


def backsub_rows(net: Net, t: int, E: torch.Tensor, relax: dict, lo, hi, keep_ap=False):
    """Lower bounds of the rows E (coefficients on zhat^(t)) over the box.

    Pushes E through the affine edges into t, then through ReLU t-1, its edges,
    ..., down to the input (coefficients reaching one z^(s) from several edges
    add up) and concretises.  ``relax[i]`` gives the relaxation of ReLU layer i.
    Returns (lb, x*, {i: a'_i} if keep_ap).
    """
    lam = {}
    c = torch.zeros(E.shape[0], dtype=DT)

    def push(u, Ahat):
        nonlocal c
        for s, A in net.edges[u]:
            lam[s] = lam[s] + A.backsub(Ahat) if s in lam else A.backsub(Ahat)
            c = c + A.bias_dot(Ahat)

    push(t, E)
    aps = {}
    for i in range(t - 1, 0, -1):
        if i not in lam:
            continue
        r = relax[i]
        A, dc, ap = relu_backsub(lam.pop(i), r.l, r.u, r.S, r.alpha, r.beta, r.GP, r.GPh, r.gp0)
        if keep_ap:
            aps[i] = ap
        c = c + dc
        push(i, A)
    d0 = net.dims()[0]
    A0 = lam.get(0, torch.zeros(E.shape[0], d0, dtype=DT))
    lb, xstar = concretize(A0, c, lo, hi)
    return lb, xstar, aps


def deeppoly_relax(l, u, S) -> Relax:
    z = torch.zeros_like(l)
    return Relax(l, u, S, deeppoly_alpha(l, u), z)


def _unit_rows(d: int, idx: torch.Tensor) -> torch.Tensor:
    """Rows +e_j for j in idx followed by rows -e_j (lower, then upper bounds)."""
    n = idx.numel()
    E = torch.zeros(2 * n, d, dtype=DT)
    ar = torch.arange(n)
    E[ar, idx] = 1.0
    E[n + ar, idx] = -1.0
    return E


def root_bounds(net: Net, lo, hi, chunk: int = 4096):
    """DeepPoly bounds l^(t), u^(t) of every ReLU layer at the root (Sec. 3.1).

    Layer t is bounded by back-substituting +-e_j from zhat^(t) with DeepPoly
    slopes on layers < t (beta = gamma = 0, no splits).
    """
    R = net.R
    dims = net.dims()
    l, u, S = {}, {}, {}
    for t in range(1, R + 1):
        relax = {i: deeppoly_relax(l[i], u[i], S[i]) for i in range(1, t)}
        idx = torch.arange(dims[t])
        lbs = []
        for s in range(0, dims[t], chunk):
            E = _unit_rows(dims[t], idx[s:s + chunk])
            lb, _, _ = backsub_rows(net, t, E, relax, lo, hi)
            lbs.append(lb)
        # rows come as [+ chunk, - chunk] per chunk
        low, up = [], []
        for s, lb in zip(range(0, dims[t], chunk), lbs):
            n = min(chunk, dims[t] - s)
            low.append(lb[:n])
            up.append(-lb[n:])
        l[t] = torch.cat(low)
        u[t] = torch.cat(up)
        S[t] = torch.zeros(dims[t], dtype=torch.int8)
    return l, u, S


# ----------------------------------------------------------------------------
# Subproblems
# ----------------------------------------------------------------------------
@dataclass
class MNC:
    """Multi-neuron constraints of one ReLU layer: P z + Phat zhat - p <= 0."""
    idx: np.ndarray     # [e, k] neuron indices
    P: np.ndarray       # [e, k]
    Ph: np.ndarray      # [e, k]
    p: np.ndarray       # [e]

    def dense(self, d: int):
        e = self.idx.shape[0]
        Pd = torch.zeros(e, d, dtype=DT)
        Phd = torch.zeros(e, d, dtype=DT)
        rows = np.repeat(np.arange(e), self.idx.shape[1])
        Pd.index_put_((torch.as_tensor(rows), torch.as_tensor(self.idx.reshape(-1))),
                      torch.as_tensor(self.P.reshape(-1), dtype=DT), accumulate=True)
        Phd.index_put_((torch.as_tensor(rows), torch.as_tensor(self.idx.reshape(-1))),
                       torch.as_tensor(self.Ph.reshape(-1), dtype=DT), accumulate=True)
        return Pd, Phd, torch.as_tensor(self.p, dtype=DT)


@dataclass
class Node:
    """One BaB subproblem of one property row."""
    row: int
    l: dict
    u: dict
    S: dict
    alpha: dict
    beta: dict
    gamma: dict
    split_layer: int            # ReLU layer of the newest split; R for a root
    depth: int = 0
    node_id: int = 0
    parent: int = -1            # node id of the parent (-1 for a root)


def init_params(net: Net, l, u, mnc: dict | None):
    """Root parameters: DeepPoly slopes, beta = gamma = 0 (Sec. 3.1 start point)."""
    alpha = {i: deeppoly_alpha(l[i], u[i]) for i in l}
    beta = {i: torch.zeros_like(l[i]) for i in l}
    gamma = {i: torch.zeros(0 if not mnc or i not in mnc else mnc[i].idx.shape[0], dtype=DT)
             for i in l}
    return alpha, beta, gamma


def rebound_node(net: Net, node: Node, lo, hi):
    """Recompute bounds of layers after the split layer (Sec. 3.2, enforcing splits).

    Only neurons unstable (l < 0 < u) and unsplit in the node are re-bounded;
    new bounds are intersected with the node's current ones.
    """
    R = net.R
    for t in range(node.split_layer + 1, R + 1):
        l, u, S = node.l[t], node.u[t], node.S[t]
        idx = torch.nonzero((l < 0) & (u > 0) & (S == 0)).reshape(-1)
        if idx.numel() == 0:
            continue
        relax = {i: deeppoly_relax(node.l[i], node.u[i], node.S[i]) for i in range(1, t)}
        E = _unit_rows(l.numel(), idx)
        lb, _, _ = backsub_rows(net, t, E, relax, lo, hi)
        n = idx.numel()
        l = l.clone()
        u = u.clone()
        l[idx] = torch.maximum(l[idx], lb[:n])
        u[idx] = torch.minimum(u[idx], -lb[n:])
        node.l[t], node.u[t] = l, u


def final_relax(node: Node, alpha, beta, gamma, dense_mnc: dict | None):
    relax = {}
    for i in node.l:
        GP = GPh = gp0 = None
        if dense_mnc and i in dense_mnc and gamma[i].numel() > 0:
            Pd, Phd, pv = dense_mnc[i]
            GP = gamma[i] @ Pd
            GPh = gamma[i] @ Phd
            gp0 = gamma[i] @ pv
        relax[i] = Relax(node.l[i], node.u[i], node.S[i], alpha[i], beta[i], GP, GPh, gp0)
    return relax


def final_bound(net: Net, node: Node, alpha, beta, gamma, dense_mnc, lo, hi, keep_ap=False):
    """Lower bound of property row ``node.row`` at parameters (alpha, beta, gamma)."""
    R = net.R
    E = torch.zeros(1, net.width(R + 1), dtype=DT)
    E[0, node.row] = 1.0
    relax = final_relax(node, alpha, beta, gamma, dense_mnc)
    lb, xstar, aps = backsub_rows(net, R + 1, E, relax, lo, hi, keep_ap)
    return lb[0], xstar[0], aps


def deeppoly_final(net: Net, node: Node, lo, hi):
    """DeepPoly pass of the objective: heuristic alpha, beta = gamma = 0 (Sec. 4 setup)."""
    alpha = {i: deeppoly_alpha(node.l[i], node.u[i]) for i in node.l}
    beta = {i: torch.zeros_like(node.l[i]) for i in node.l}
    gamma = {i: torch.zeros(0, dtype=DT) for i in node.l}
    lb, xs, _ = final_bound(net, node, alpha, beta, gamma, None, lo, hi)
    return lb, xs


@dataclass
class AdamHP:
    """Projected Adam ascent (Sec. 3.1, projected gradient ascent).  The paper
    names no optimiser or step sizes: parity unpinned, values are this
    project's choice.  The defaults are standard Adam (eps = 1e-8 in the
    denominator) with a projection after every step."""
    steps: int = 20
    lr_alpha: float = 0.1
    lr_beta: float = 0.05
    lr_gamma: float = 0.05
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    # Two named options, both off by default.  With G the node's largest
    # |gradient component|: eps_rel > 0 makes the denominator use
    # max(eps, eps_rel * G); grad_floor > 0 counts components with
    # |g| <= grad_floor * G as zero.  Constraints that are tight at the relaxed
    # point have gradients at rounding level, which standard Adam's
    # per-component normalisation turns into full steps of arbitrary sign;
    # eps_rel keeps the update continuous in the gradient instead.
    eps_rel: float = 0.0
    grad_floor: float = 0.0


def bound_and_grad(net, node, alpha, beta, gamma, dense_mnc, lo, hi):
    """Objective bound and its exact reverse-mode gradient (D cases held fixed)."""
    a = {i: alpha[i].detach().clone().requires_grad_(True) for i in alpha}
    b = {i: beta[i].detach().clone().requires_grad_(True) for i in beta}
    g = {i: gamma[i].detach().clone().requires_grad_(True) for i in gamma}
    lb, xs, _ = final_bound(net, node, a, b, g, dense_mnc, lo, hi)
    leaves = list(a.values()) + list(b.values()) + list(g.values())
    grads = torch.autograd.grad(lb, leaves, allow_unused=True)
    n = len(a)
    keys = list(a.keys())
    ga = {k: (gr if gr is not None else torch.zeros_like(a[k])) for k, gr in zip(keys, grads[:n])}
    gb = {k: (gr if gr is not None else torch.zeros_like(b[k])) for k, gr in zip(keys, grads[n:2 * n])}
    gg = {k: (gr if gr is not None else torch.zeros_like(g[k])) for k, gr in zip(keys, grads[2 * n:])}
    return lb.detach(), xs.detach(), ga, gb, gg


def optimize(net, node: Node, dense_mnc, lo, hi, hp: AdamHP, noise=None):
    """hp.steps projected Adam ascent steps from the node's inherited parameters.

    Evaluates the bound at theta_0 .. theta_N (N = hp.steps) and returns the
    best bound (first maximiser), its x*, and the final parameters theta_N.

    ``noise = (seed, rel)`` is a test probe, not part of the method: every
    gradient component that is computed as a sum (alpha of unstable unsplit
    neurons, beta of split neurons, every gamma) gets an independent uniform
    perturbation in [-rel G, rel G], G = the node's largest |component|, before
    the Adam update -- a model of the rounding of an FP32 implementation.
    """
    alpha = {i: node.alpha[i].clone() for i in node.alpha}
    beta = {i: node.beta[i].clone() for i in node.beta}
    gamma = {i: node.gamma[i].clone() for i in node.gamma}
    state = {}
    for grp, P in (("a", alpha), ("b", beta), ("g", gamma)):
        for i in P:
            state[(grp, i)] = (torch.zeros_like(P[i]), torch.zeros_like(P[i]))
    best, best_x = -math.inf, None
    lr = {"a": hp.lr_alpha, "b": hp.lr_beta, "g": hp.lr_gamma}
    for step in range(hp.steps + 1):
        lb, xs, ga, gb, gg = bound_and_grad(net, node, alpha, beta, gamma, dense_mnc, lo, hi)
        if float(lb) > best:
            best, best_x = float(lb), xs
        if step == hp.steps:
            break
        t = step + 1
        gmax = max([float(G[i].abs().max()) for G in (ga, gb, gg) for i in G if G[i].numel()] + [0.0])
        if noise is not None:
            gen = torch.Generator().manual_seed(noise[0] * 1000 + step)
            for grp, G in (("a", ga), ("b", gb), ("g", gg)):
                for i in G:
                    if grp == "a":
                        live = (node.l[i] < 0) & (node.u[i] > 0) & (node.S[i] == 0)
                    elif grp == "b":
                        live = node.S[i] != 0
                    else:
                        live = torch.ones_like(G[i], dtype=torch.bool)
                    e = (torch.rand(G[i].shape, generator=gen, dtype=DT) * 2 - 1) * noise[1] * gmax
                    G[i] = G[i] + torch.where(live, e, torch.zeros_like(e))
        floor = hp.grad_floor * gmax
        eps = max(hp.eps, hp.eps_rel * gmax)
        for G in (ga, gb, gg):
            for i in G:
                G[i] = torch.where(G[i].abs() <= floor, torch.zeros_like(G[i]), G[i])
        for grp, P, G in (("a", alpha, ga), ("b", beta, gb), ("g", gamma, gg)):
            for i in P:
                m, v = state[(grp, i)]
                m = hp.b1 * m + (1 - hp.b1) * G[i]
                v = hp.b2 * v + (1 - hp.b2) * G[i] * G[i]
                state[(grp, i)] = (m, v)
                mh = m / (1 - hp.b1 ** t)
                vh = v / (1 - hp.b2 ** t)
                P[i] = P[i] + lr[grp] * mh / (torch.sqrt(vh) + eps)
                if grp == "a":
                    P[i] = torch.clamp(P[i], 0.0, 1.0)
                else:
                    P[i] = torch.clamp(P[i], min=0.0)
    return best, best_x, alpha, beta, gamma


def noise_sensitivity(net, node: Node, dense_mnc, lo, hi, hp: AdamHP, seeds=(1, 2, 3),
                      rel=1e-6, always=False) -> float:
    """How far the node's optimised bound moves when its gradients carry
    rounding-level perturbations (``optimize(noise=...)``): the largest
    |best_perturbed - best| over the seeds, 0 for a node its DeepPoly pass
    verifies (no optimisation in BaB) unless ``always``.  ``node`` is the node as queued; it is not
    changed.  A test probe: a bound that moves by more than a small part of the
    parity tolerance is not determined at FP32 precision."""
    nd = Node(node.row, {i: node.l[i].clone() for i in node.l},
              {i: node.u[i].clone() for i in node.u}, {i: node.S[i].clone() for i in node.S},
              node.alpha, node.beta, node.gamma, node.split_layer, node.depth, node.node_id)
    rebound_node(net, nd, lo, hi)
    lb_dp, _ = deeppoly_final(net, nd, lo, hi)
    if float(lb_dp) > 0 and not always:
        return 0.0
    best, *_ = optimize(net, nd, dense_mnc, lo, hi, hp)
    best = max(best, float(lb_dp))
    dev = 0.0
    for sd in seeds:
        b, *_ = optimize(net, nd, dense_mnc, lo, hi, hp, noise=(sd, rel))
        dev = max(dev, abs(max(b, float(lb_dp)) - best))
    return dev


# ----------------------------------------------------------------------------
# Optimised intermediate bounds (Sec. 3.1, parameter sharing)
# ----------------------------------------------------------------------------
def intermediate_objective(net: Net, node: Node, t: int, idx, side: int, alpha, beta, lo, hi,
                           gamma=None, dense_mnc=None):
    """Lower bounds of the rows side * e_j (j in idx) of zhat^(t) with one
    parameter set (alpha_i, beta_i and, with multi-neuron constraints, gamma_i
    for i < t) shared by every row.

    side = +1 gives lower bounds of zhat_j, side = -1 lower bounds of -zhat_j
    (the upper bounds, negated).  Returns the per-row bounds; their sum is the
    objective that the set ascends.
    """
    E = torch.zeros(idx.numel(), node.l[t].numel(), dtype=DT)
    E[torch.arange(idx.numel()), idx] = float(side)
    relax = {}
    for i in range(1, t):
        GP = GPh = gp0 = None
        if gamma is not None and dense_mnc and i in dense_mnc and gamma[i].numel() > 0:
            Pd, Phd, pv = dense_mnc[i]
            GP, GPh, gp0 = gamma[i] @ Pd, gamma[i] @ Phd, gamma[i] @ pv
        relax[i] = Relax(node.l[i], node.u[i], node.S[i], alpha[i], beta[i], GP, GPh, gp0)
    lb, _, _ = backsub_rows(net, t, E, relax, lo, hi)
    return lb


def intermediate_objective_grad(net: Net, node: Node, t: int, idx, side: int, alpha, beta, lo, hi,
                                gamma=None, dense_mnc=None):
    """Per-row bounds and the gradient of their sum w.r.t. the shared set
    (alpha, beta, and gamma when given)."""
    a = {i: alpha[i].detach().clone().requires_grad_(True) for i in alpha}
    b = {i: beta[i].detach().clone().requires_grad_(True) for i in beta}
    g = ({i: gamma[i].detach().clone().requires_grad_(True) for i in gamma}
         if gamma is not None else None)
    lb = intermediate_objective(net, node, t, idx, side, a, b, lo, hi, g, dense_mnc)
    keys = list(a.keys())
    leaves = [a[k] for k in keys] + [b[k] for k in keys] + ([g[k] for k in keys] if g else [])
    grads = torch.autograd.grad(lb.sum(), leaves, allow_unused=True)
    n = len(keys)
    ga = {k: (x if x is not None else torch.zeros_like(a[k])) for k, x in zip(keys, grads[:n])}
    gb = {k: (x if x is not None else torch.zeros_like(b[k])) for k, x in zip(keys, grads[n:2 * n])}
    if g is None:
        return lb.detach(), ga, gb
    gg = {k: (x if x is not None else torch.zeros_like(g[k])) for k, x in zip(keys, grads[2 * n:])}
    return lb.detach(), ga, gb, gg


def optimize_intermediate(net: Net, node: Node, lo, hi, hp: AdamHP, first_layer: int = 2,
                          dense_mnc=None):
    """Optimised intermediate bounds of a node (Sec. 3.1: intermediate bounds
    come from the same bounding procedure; each layer's neurons share one
    parameter set, with separate sets for lower and upper bounds).

    For t = max(2, first_layer) .. R in order (layer 1 bounds over the box are
    exact already): the rows are the unstable, unsplit neurons j of layer t,
    once with side +1 (lower bounds) and once with side -1 (upper bounds).  Each
    side has one set (alpha_i, beta_i for the ReLU layers i < t, and with
    multi-neuron constraints gamma_i of those layers' constraints) shared by
    all its rows, started at DeepPoly slopes, beta = 0 and gamma = 0, and takes
    hp.steps projected Adam steps (as in ``optimize``) ascending sum_j lb_j.
    Every iterate gives valid bounds, so each row keeps the best bound it
    reached (the first iterate is the DeepPoly bound); the node's bounds of
    layer t are intersected with them before layer t + 1 is bounded.  Returns
    the number of rows bounded.
    """
    R = net.R
    total = 0
    lr = {"a": hp.lr_alpha, "b": hp.lr_beta, "g": hp.lr_gamma}
    for t in range(max(2, first_layer), R + 1):
        l, u, S = node.l[t], node.u[t], node.S[t]
        idx = torch.nonzero((l < 0) & (u > 0) & (S == 0)).reshape(-1)
        if idx.numel() == 0:
            continue
        best = {}
        for side in (1, -1):
            alpha = {i: deeppoly_alpha(node.l[i], node.u[i]) for i in range(1, t)}
            beta = {i: torch.zeros_like(node.l[i]) for i in range(1, t)}
            gamma = None
            if dense_mnc:
                gamma = {i: torch.zeros(dense_mnc[i][2].numel() if i in dense_mnc else 0, dtype=DT)
                         for i in range(1, t)}
            groups = {"a": alpha, "b": beta}
            if gamma is not None:
                groups["g"] = gamma
            state = {(g, i): (torch.zeros_like(P[i]), torch.zeros_like(P[i]))
                     for g, P in groups.items() for i in P}
            bs = torch.full((idx.numel(),), -math.inf, dtype=DT)
            for step in range(hp.steps + 1):
                out = intermediate_objective_grad(net, node, t, idx, side, alpha, beta, lo, hi,
                                                  gamma, dense_mnc)
                lb, grads = out[0], {"a": out[1], "b": out[2]}
                if gamma is not None:
                    grads["g"] = out[3]
                bs = torch.maximum(bs, lb)
                if step == hp.steps:
                    break
                k = step + 1
                gmax = max([float(G[i].abs().max()) for G in grads.values() for i in G
                            if G[i].numel()] + [0.0])
                floor = hp.grad_floor * gmax
                eps = max(hp.eps, hp.eps_rel * gmax)
                for grp, P in groups.items():
                    for i in P:
                        g = grads[grp][i]
                        g = torch.where(g.abs() <= floor, torch.zeros_like(g), g)
                        m, v = state[(grp, i)]
                        m = hp.b1 * m + (1 - hp.b1) * g
                        v = hp.b2 * v + (1 - hp.b2) * g * g
                        state[(grp, i)] = (m, v)
                        mh = m / (1 - hp.b1 ** k)
                        vh = v / (1 - hp.b2 ** k)
                        P[i] = P[i] + lr[grp] * mh / (torch.sqrt(vh) + eps)
                        P[i] = torch.clamp(P[i], 0.0, 1.0) if grp == "a" else torch.clamp(P[i], min=0.0)
            best[side] = bs
        l = l.clone()
        u = u.clone()
        l[idx] = torch.maximum(l[idx], best[1])
        u[idx] = torch.minimum(u[idx], -best[-1])
        node.l[t], node.u[t] = l, u
        total += 2 * idx.numel()
    return total


# ----------------------------------------------------------------------------
# Branching (Sec. 3.2)
# ----------------------------------------------------------------------------
ACS_TIE = 1e-5


def acs_scores(node: Node, gamma, dense_mnc, aps: dict):
    """Active Constraint Score s_j = |(gamma^T P)_j| + |(gamma^T Phat)_j| (Sec. 3.2).

    Candidates are unstable, unsplit neurons of every ReLU layer.  If every
    candidate scores 0 (e.g. no multi-neuron constraints), the fallback score
    |a'_j| * (-l_j u_j / (u_j - l_j)) is used (paper silent; this project's
    reading).  Returns ({i: scores with -inf on non-candidates}, used_fallback).
    """
    scores = {}
    any_pos = False
    for i in node.l:
        l, u, S = node.l[i], node.u[i], node.S[i]
        cand = (l < 0) & (u > 0) & (S == 0)
        s = torch.zeros_like(l)
        if dense_mnc and i in dense_mnc and gamma[i].numel() > 0:
            Pd, Phd, _ = dense_mnc[i]
            s = torch.abs(gamma[i] @ Pd) + torch.abs(gamma[i] @ Phd)
        if bool((s[cand] > 0).any()):
            any_pos = True
        scores[i] = torch.where(cand, s, torch.full_like(s, -math.inf))
    if any_pos:
        return scores, False
    fb = {}
    for i in node.l:
        l, u, S = node.l[i], node.u[i], node.S[i]
        cand = (l < 0) & (u > 0) & (S == 0)
        den = torch.where(cand, u - l, torch.ones_like(u))
        icpt = torch.where(cand, -l * u / den, torch.zeros_like(u))
        s = torch.abs(aps[i].reshape(-1)) * icpt
        fb[i] = torch.where(cand, s, torch.full_like(s, -math.inf))
    return fb, True


def cab_costs(net: Net, n_mnc: dict | None = None) -> dict:
    """Cost of splitting a neuron of ReLU layer k (App. B, cost-adjusted branching).

    Per-layer costs: affine layer = number of weight entries (FC) or d_out k^2
    (conv); ReLU layer = d + (number of multi-neuron constraints).  C_t = sum of
    the costs of every layer below zhat_t; a split at layer k recomputes both
    bounds of every neuron of the later ReLU layers: sum_{t>k} 2 d_t C_t.
    Reading (the paper is silent): the cost of one objective back-substitution
    C_obj (a single row, d_R weight entries in the last layer) is added so that
    splits in the last ReLU layer have a positive cost.
    """
    n_mnc = n_mnc or {}
    R = net.R

    def aff_cost(A: Affine) -> float:
        if A.kind == "fc":
            return float(A.W.numel())
        return float(A.d_out * A.W.shape[2] * A.W.shape[3])

    C = {}
    acc = 0.0
    for t in range(1, R + 1):
        acc += sum(aff_cost(A) for _, A in net.edges[t])
        C[t] = acc                                   # all layers below zhat_t
        acc += net.width(t) + n_mnc.get(t, 0)        # relu_t
    c_obj = acc + net.width(R) if R >= 1 else acc    # one objective row through the last layer
    costs = {}
    for k in range(1, R + 1):
        costs[k] = c_obj + sum(2.0 * net.width(t) * C[t] for t in range(k + 1, R + 1))
    return costs


def cab_scores(scores: dict, costs: dict) -> dict:
    """ACS (or fallback) score divided by the cost of the split (Sec. 3.2, CAB)."""
    return {i: scores[i] / costs[i] for i in scores}


def pick_split(scores: dict):
    """Argmax with ties |s - max| <= 1e-5 * max broken by lowest (layer, index)."""
    mx = -math.inf
    for i in sorted(scores):
        if scores[i].numel():
            mx = max(mx, float(scores[i].max()))
    if mx == -math.inf:
        return None
    thr = mx - ACS_TIE * abs(mx)
    for i in sorted(scores):
        hit = torch.nonzero(scores[i] >= thr).reshape(-1)
        if hit.numel():
            return i, int(hit[0]), mx
    return None
