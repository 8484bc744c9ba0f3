"""Multi-neuron constraint generator over k=3 neuron groups -- test infrastructure only.

The paper takes its constraints from PRIMA (Sec. 2.3 and Sec. 3.1, enforcing
multi-neuron constraints) and gives no generator; any linear constraints valid
on the joint (z, zhat) space of a ReLU layer are admissible.  This is the
project's reading (parity unpinned against the paper's own constraint sets;
soundness is pinned by LP per orthant in the tests):

1. unstable neurons of the layer, sorted by -l u / (u - l) descending (ties by
   index), grouped as sliding triples (j0, j1, j2), (j1, j2, j3), ...,
   at most ``max_groups`` groups;
2. for each group, DeepPoly lower bounds of d . zhat_G for the 26 directions
   d in {-1, 0, 1}^3 \\ {0}: an octahedral over-approximation of zhat_G;
3. per orthant, every vertex of {octahedron and orthant} (all triples of
   bounding planes, feasibility tolerance 1e-9), lifted to (relu(x), x);
4. the 6-D convex hull of all lifted vertices (Qhull via scipy); each facet
   n_y . y + n_x . x <= p is re-tightened to p = max over the lifted points;
5. facets that involve a single neuron are dropped (the single-neuron
   relaxation already holds them); rows are written as [P = n_y, Phat = n_x, p].
"""
from __future__ import annotations

import itertools

import numpy as np
import torch
from scipy.spatial import ConvexHull

from . import core
from .core import DT


DIRS = np.array([d for d in itertools.product((-1, 0, 1), repeat=3) if any(d)], dtype=np.float64)


def octahedron_bounds(net, t, groups, l, u, S, lo, hi, chunk=2048):
    """Lower bounds of d . zhat^(t)_G for all 26 directions (rows [g, 26])."""
    relax = {i: core.deeppoly_relax(l[i], u[i], S[i]) for i in range(1, t)}
    d = l[t].numel()
    out = np.zeros((len(groups), len(DIRS)))
    for s in range(0, len(groups), chunk):
        gs = groups[s:s + chunk]
        E = torch.zeros(len(gs) * len(DIRS), d, dtype=DT)
        for gi, G in enumerate(gs):
            for di, dv in enumerate(DIRS):
                for k in range(3):
                    E[gi * len(DIRS) + di, G[k]] += dv[k]
        lb, _, _ = core.backsub_rows(net, t, E, relax, lo, hi)
        out[s:s + len(gs)] = lb.numpy().reshape(len(gs), len(DIRS))
    return out


def _vertices(planes_n, planes_b, tol=1e-9):
    """Vertices of {x : n . x >= b} in 3-D by all plane triples."""
    m = planes_n.shape[0]
    tri = np.array(list(itertools.combinations(range(m), 3)))
    A = planes_n[tri]                       # [T, 3, 3]
    rhs = planes_b[tri]                     # [T, 3]
    det = np.linalg.det(A)
    ok = np.abs(det) > 1e-12
    A, rhs = A[ok], rhs[ok]
    X = np.linalg.solve(A, rhs[..., None])[..., 0]
    slack = X @ planes_n.T - planes_b[None, :]
    feas = (slack >= -tol * (1.0 + np.abs(planes_b[None, :]))).all(axis=1)
    X = X[feas]
    if X.shape[0] == 0:
        return X
    return np.unique(np.round(X, 12), axis=0)


def group_constraints(oct_lb):
    """Constraint rows (P [e,3], Phat [e,3], p [e]) for one group."""
    pts = []
    for sig in itertools.product((-1.0, 1.0), repeat=3):
        sig = np.array(sig)
        n = np.concatenate([DIRS, np.diag(sig)])
        b = np.concatenate([oct_lb, np.zeros(3)])
        V = _vertices(n, b)
        if V.shape[0] == 0:
            continue
        Y = np.where(sig[None, :] > 0, V, 0.0)   # relu is linear in the orthant
        Y = np.maximum(Y, 0.0)
        pts.append(np.concatenate([Y, V], axis=1))
    if not pts:
        return None
    pts = np.unique(np.concatenate(pts), axis=0)
    if pts.shape[0] < 7:
        return None
    try:
        hull = ConvexHull(pts)
    except Exception:
        try:
            hull = ConvexHull(pts, qhull_options="QJ")
        except Exception:
            return None
    eq = hull.equations[:, :6]
    eq = np.unique(np.round(eq, 10), axis=0)
    rows_P, rows_Ph, rows_p = [], [], []
    for nvec in eq:
        ny, nx = nvec[:3], nvec[3:]
        support = (np.abs(ny) > 1e-9) | (np.abs(nx) > 1e-9)
        if support.sum() <= 1:
            continue
        p = float((pts @ nvec).max())
        rows_P.append(ny)
        rows_Ph.append(nx)
        rows_p.append(p)
    if not rows_P:
        return None
    return np.array(rows_P), np.array(rows_Ph), np.array(rows_p)


def unstable_groups(l, u, max_groups):
    l = l.numpy()
    u = u.numpy()
    idx = np.nonzero((l < 0) & (u > 0))[0]
    if idx.size < 3:
        return []
    key = -l[idx] * u[idx] / (u[idx] - l[idx])
    order = idx[np.lexsort((idx, -key))]
    groups = [tuple(int(v) for v in order[s:s + 3]) for s in range(order.size - 2)]
    return groups[:max_groups]


def generate(net, l, u, lo, hi, max_groups=2000, layers=None):
    """Constraints of every ReLU layer at the root: {layer: core.MNC}."""
    S = {i: torch.zeros(l[i].numel(), dtype=torch.int8) for i in l}
    out = {}
    for t in (layers or sorted(l)):
        groups = unstable_groups(l[t], u[t], max_groups)
        if not groups:
            continue
        ob = octahedron_bounds(net, t, groups, l, u, S, lo, hi)
        idx, P, Ph, p = [], [], [], []
        for G, lbs in zip(groups, ob):
            r = group_constraints(lbs)
            if r is None:
                continue
            P.append(r[0]); Ph.append(r[1]); p.append(r[2])
            idx.append(np.tile(np.array(G), (r[0].shape[0], 1)))
        if idx:
            out[t] = core.MNC(np.concatenate(idx).astype(np.int32), np.concatenate(P),
                              np.concatenate(Ph), np.concatenate(p))
    return out


def mnc_fn(max_groups=2000):
    def fn(net, l, u, lo, hi):
        return generate(net, l, u, lo, hi, max_groups)
    return fn
