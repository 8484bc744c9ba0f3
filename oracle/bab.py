"""Branch-and-bound driver of the oracle (Sec. 2.2; Sec. 3.2) -- test infrastructure only.

Each property row r (margin y_t - y_j) is its own BaB problem on the scalar
objective zhat^(R+1)_r (Sec. 2.1).  Per node:

1. recompute the intermediate bounds of layers after its split layer
   (Sec. 3.2, enforcing splits);
2. the DeepPoly pass of the objective (Sec. 4, experimental setup): if its
   bound is > 0 the node is verified;
3. otherwise projected Adam on (alpha, beta, gamma) (Sec. 3.1); the node bound
   is the best of the DeepPoly pass and the iterates;
4. the minimiser x* is pushed through the network: f_r(x*) < 0 is a
   counterexample (Sec. 2.2, Sec. 3.1 upper bounding);
5. otherwise the ACS score picks the split (Sec. 3.2) and two children are
   queued: S = +1 (negative split, zhat <= 0, u <- min(u, 0)) first, then
   S = -1 (positive split, zhat >= 0, l <- max(l, 0)).  Children inherit the
   parent's final parameters; the new split's beta starts at 0.

Queue order is FIFO by node id over all rows of a property (the paper is
silent; FIFO makes the tree independent of batch size and of bound values at
rounding level), and the node budget counts bounded nodes including roots.
Parity status: the queue policy is parity unpinned (a definition of this
project); every node bound is pinned through ``core``.
"""
from __future__ import annotations

import copy
import math
from collections import deque
from dataclasses import dataclass, field, replace

import numpy as np
import torch

from . import core
from .core import DT, AdamHP, Node

VERIFIED, FALSIFIED, UNKNOWN = 1, -1, 0


@dataclass
class NodeResult:
    node_id: int
    row: int
    lb: float
    lb_dp: float
    f_xstar: float
    xstar: np.ndarray
    verdict: int                    # VERIFIED / FALSIFIED / UNKNOWN (branched or leaf)
    split: tuple | None = None      # (layer, neuron)
    fallback: bool = False
    split_layer: int = 0
    depth: int = 0
    parent: int = -1
    # with verify(..., record=True): the branching scores {layer: tensor} the
    # split was chosen from, and the node as queued (before step 1)
    scores: dict | None = None
    start: Node | None = None
    leaf: bool = False              # resolved as a fully split leaf (exact LP)


@dataclass
class PropResult:
    verdict: int
    nodes: list = field(default_factory=list)
    n_bounded: int = 0


def prepare(layers, C, d, lo, hi, mnc_fn=None):
    """Fold the property, compute root bounds, optional constraints and root nodes."""
    net = core.fold_property(core.load_net(layers), C, d)
    lo_t = torch.as_tensor(np.asarray(lo), dtype=DT)
    hi_t = torch.as_tensor(np.asarray(hi), dtype=DT)
    l, u, S = core.root_bounds(net, lo_t, hi_t)
    mnc = mnc_fn(net, l, u, lo_t, hi_t) if mnc_fn is not None else None
    dense = {i: m.dense(l[i].numel()) for i, m in mnc.items()} if mnc else None
    return net, lo_t, hi_t, l, u, S, mnc, dense


def root_node(net, row, l, u, S, mnc, node_id=0) -> Node:
    alpha, beta, gamma = core.init_params(net, l, u, mnc)
    return Node(row=row, l={i: l[i].clone() for i in l}, u={i: u[i].clone() for i in u},
                S={i: S[i].clone() for i in S}, alpha=alpha, beta=beta, gamma=gamma,
                split_layer=net.R, depth=0, node_id=node_id)


def bound_node(net, node: Node, dense, lo, hi, hp: AdamHP):
    """Steps 1-4 above; returns (NodeResult, final params)."""
    core.rebound_node(net, node, lo, hi)
    lb_dp, xs_dp = core.deeppoly_final(net, node, lo, hi)
    lb_dp = float(lb_dp)
    params = (node.alpha, node.beta, node.gamma)
    if lb_dp > 0:
        lb, xs = lb_dp, xs_dp
    else:
        best, bx, a, b, g = core.optimize(net, node, dense, lo, hi, hp)
        params = (a, b, g)
        if best > lb_dp:
            lb, xs = best, bx
        else:
            lb, xs = lb_dp, xs_dp
    f = float(net.forward(xs.reshape(1, -1))[0, node.row])
    if lb > 0:
        verdict = VERIFIED
    elif f < 0:
        verdict = FALSIFIED
    else:
        verdict = UNKNOWN
    res = NodeResult(node.node_id, node.row, lb, lb_dp, f, xs.numpy(), verdict,
                     split_layer=node.split_layer, depth=node.depth, parent=node.parent)
    return res, params


def branch(net, node: Node, params, dense, lo, hi, cab=None):
    """ACS split choice; with ``cab`` (layer costs from core.cab_costs) the
    cost-adjusted score (Sec. 3.2) is used instead."""
    a, b, g = params
    _, _, aps = core.final_bound(net, node, a, b, g, dense, lo, hi, keep_ap=True)
    scores, fb = core.acs_scores(node, g, dense, aps)
    if cab is not None:
        scores = core.cab_scores(scores, cab)
    return core.pick_split(scores), fb, scores


def children(node: Node, params, split, next_id: int):
    layer, j, _ = split
    a, b, g = params
    out = []
    for k, sgn in enumerate((1, -1)):
        S = {i: node.S[i].clone() for i in node.S}
        l = {i: node.l[i].clone() for i in node.l}
        u = {i: node.u[i].clone() for i in node.u}
        S[layer][j] = sgn
        if sgn == 1:
            u[layer][j] = min(float(u[layer][j]), 0.0)
        else:
            l[layer][j] = max(float(l[layer][j]), 0.0)
        beta = {i: b[i].clone() for i in b}
        beta[layer][j] = 0.0
        out.append(Node(row=node.row, l=l, u=u, S=S,
                        alpha={i: a[i].clone() for i in a}, beta=beta,
                        gamma={i: g[i].clone() for i in g},
                        split_layer=layer, depth=node.depth + 1, node_id=next_id + k,
                        parent=node.node_id))
    return out


def leaf_exact(layers, C, d, node: Node, lo, hi):
    """Exact minimum of a fully split leaf (Sec. 3.3: with every unstable neuron
    split the network is affine on the leaf, so its minimum is a linear
    program; the optimal-beta bound equals it).  Returns (value, argmin) from
    exact.exact_min over the leaf's splits, FC networks only."""
    from . import exact
    splits = {(i, j): int(node.S[i][j]) for i in node.S
              for j in torch.nonzero(node.S[i]).reshape(-1).tolist()}
    return exact.exact_min(layers, C, d, node.row, np.asarray(lo), np.asarray(hi),
                           splits=splits)


def verify(layers, C, d, lo, hi, max_nodes=256, hp: AdamHP | None = None, mnc_fn=None,
           rows=None, prepared=None, cab=False, inter_steps=0, record=False,
           leaf_lp=None) -> PropResult:
    """BaB on every row of one property; verdict VERIFIED / FALSIFIED / UNKNOWN.
    With ``cab`` the split is chosen by the cost-adjusted ACS score.  With
    ``inter_steps`` > 0 the root's intermediate bounds are first optimised
    (``core.optimize_intermediate``, Sec. 3.1 parameter sharing, that many Adam
    steps at hp's rates) and shared by every row's root node.  With ``record``
    every node result also carries its starting state and its branching
    scores (for the parity tests).  A fully split leaf whose bound does not
    decide it is resolved by its exact LP (``leaf_exact``) when the network is
    fully connected (``leaf_lp`` None: whenever it is), else it stays an
    UNKNOWN leaf."""
    hp = hp or AdamHP()
    net, lo_t, hi_t, l, u, S, mnc, dense = prepared or prepare(layers, C, d, lo, hi, mnc_fn)
    if inter_steps > 0:
        root = root_node(net, 0, l, u, S, mnc)
        core.optimize_intermediate(net, root, lo_t, hi_t, replace(hp, steps=inter_steps),
                                   dense_mnc=dense)
        l, u = root.l, root.u
    costs = core.cab_costs(net, {i: m.idx.shape[0] for i, m in mnc.items()} if mnc else None) \
        if cab else None
    rows = list(range(net.width(net.R + 1))) if rows is None else rows
    q = deque()
    nid = 0
    for r in rows:
        q.append(root_node(net, r, l, u, S, mnc, nid))
        nid += 1
    res = PropResult(UNKNOWN)
    unknown_leaf = False
    while q and res.n_bounded < max_nodes:
        node = q.popleft()
        start = copy.deepcopy(node) if record else None
        nr, params = bound_node(net, node, dense, lo_t, hi_t, hp)
        nr.start = start
        res.n_bounded += 1
        if nr.verdict == UNKNOWN:
            split, fb, scores = branch(net, node, params, dense, lo_t, hi_t, costs)
            nr.fallback = fb
            if record:
                nr.scores = scores
            if split is None:
                if leaf_lp is None:
                    leaf_lp = all(L["kind"] in ("fc", "relu") for L in layers)
                if leaf_lp:
                    v, xa = leaf_exact(layers, C, d, node, lo_t, hi_t)
                    nr.leaf = True
                    nr.lb = float(v)
                    if v > 0:
                        nr.verdict = VERIFIED
                    else:
                        fx = float(net.forward(torch.as_tensor(xa, dtype=DT)[None])[0, node.row])
                        nr.f_xstar = fx
                        nr.xstar = np.asarray(xa)
                        nr.verdict = FALSIFIED if fx < 0 else UNKNOWN
                        unknown_leaf = unknown_leaf or nr.verdict == UNKNOWN
                else:
                    unknown_leaf = True
            else:
                nr.split = (split[0], split[1])
                for ch in children(node, params, split, nid):
                    q.append(ch)
                nid += 2
        res.nodes.append(nr)
        if nr.verdict == FALSIFIED:
            res.verdict = FALSIFIED
            return res
    if not q and not unknown_leaf:
        res.verdict = VERIFIED
    return res
