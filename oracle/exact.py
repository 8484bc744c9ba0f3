"""Exact minima of tiny ReLU networks -- test infrastructure only.

min_{x in box, splits} f_r(x) is found by enumerating the activation patterns
of every neuron that interval arithmetic cannot prove stable, and solving one
LP per pattern (the network is affine in x once the pattern is fixed; the
pattern adds the sign constraints zhat_j >= 0 or <= 0).  Interval arithmetic
is used instead of the oracle's own bounds so that this check does not rest on
the code it pins.  Used to pin the completeness limit (Sec. 3.3): a fully split
subproblem is linear and its optimal-beta bound equals the LP optimum.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import linprog


def _fc_layers(layers):
    Ws, bs = [], []
    for L in layers:
        if L["kind"] == "fc":
            Ws.append(np.asarray(L["W"], dtype=np.float64))
            bs.append(np.asarray(L["b"], dtype=np.float64))
        elif L["kind"] != "relu":
            raise ValueError("exact enumeration supports fully connected nets only")
    return Ws, bs


def interval_bounds(Ws, bs, lo, hi):
    """Interval-arithmetic pre-activation bounds of every hidden layer."""
    l, u = np.asarray(lo, float), np.asarray(hi, float)
    out = []
    for i, (W, b) in enumerate(zip(Ws, bs)):
        Wp, Wn = np.maximum(W, 0), np.minimum(W, 0)
        zl = Wp @ l + Wn @ u + b
        zu = Wp @ u + Wn @ l + b
        if i < len(Ws) - 1:
            out.append((zl, zu))
            l, u = np.maximum(zl, 0), np.maximum(zu, 0)
    return out


def exact_min(layers, C, d, row, lo, hi, splits=None, max_patterns=1 << 14):
    """Exact min of (C f(x) + d)_row over the box and split signs.

    ``splits``: {(layer, neuron): +1 (zhat <= 0) or -1 (zhat >= 0)}, layers
    counted from 1.  Returns (value, argmin) or (inf, None) if infeasible.
    """
    Ws, bs = _fc_layers(layers)
    Ws = [W.copy() for W in Ws]
    bs = [b.copy() for b in bs]
    C = np.asarray(C, np.float64)
    Ws[-1] = C @ Ws[-1]
    bs[-1] = C @ bs[-1] + np.asarray(d, np.float64)
    ib = interval_bounds(Ws, bs, lo, hi)
    splits = splits or {}
    free = []
    fixed = {}
    for i, (zl, zu) in enumerate(ib, start=1):
        for j in range(zl.size):
            if (i, j) in splits:
                fixed[(i, j)] = 1 if splits[(i, j)] == -1 else 0
            elif zl[j] >= 0:
                fixed[(i, j)] = 1
            elif zu[j] <= 0:
                fixed[(i, j)] = 0
            else:
                free.append((i, j))
    if 2 ** len(free) > max_patterns:
        raise ValueError(f"{len(free)} free neurons: too many patterns")
    n = len(lo)
    bounds = list(zip(np.asarray(lo, float), np.asarray(hi, float)))
    best, arg = np.inf, None
    for bits in itertools.product((0, 1), repeat=len(free)):
        act = dict(fixed)
        act.update({f: b for f, b in zip(free, bits)})
        A = np.eye(n)
        c = np.zeros(n)
        A_ub, b_ub = [], []
        for i in range(1, len(Ws)):
            Z = Ws[i - 1] @ A
            zc = Ws[i - 1] @ c + bs[i - 1]
            m = np.array([act[(i, j)] for j in range(Z.shape[0])], dtype=float)
            for j in range(Z.shape[0]):
                # active: zhat >= 0  ->  -Z x <= zc ; inactive: Z x <= -zc
                if m[j] == 1:
                    A_ub.append(-Z[j]); b_ub.append(zc[j])
                else:
                    A_ub.append(Z[j]); b_ub.append(-zc[j])
            A = m[:, None] * Z
            c = m * zc
        obj = (Ws[-1] @ A)[row]
        off = (Ws[-1] @ c + bs[-1])[row]
        r = linprog(obj, A_ub=np.array(A_ub), b_ub=np.array(b_ub), bounds=bounds, method="highs")
        if r.status == 0 and r.fun + off < best:
            best, arg = r.fun + off, r.x
    return best, arg
