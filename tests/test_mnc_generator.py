"""The library's multi-neuron constraint generator on the host (mnbab_mnc_group).

The paper takes its constraints from PRIMA (Sec. 2.3, Sec. 3.1) and gives no
generator; both sides implement this project's reading: the facets of the
convex hull of the ReLU graph over a group's octahedron, with unit normals,
offsets at the exact support, single-neuron facets dropped.  The library
finds the facets by the double-description method (C++), the oracle with
Qhull; these tests need no GPU:

* soundness: for every row and orthant, the LP maximum of the row over the
  octahedron in that orthant is at most its offset (scipy linprog);
* facets: every row touches the lifted vertex set in 6 affinely independent
  points;
* independent neurons (a box): the hull is the product of single-neuron
  triangles, so no row is left;
* against the oracle (mnc.group_constraints) on the octahedra of the
  784-100-100-10 network's groups: the same rows as a set (Qhull's
  triangulated output repeats a non-simplicial facet as several rows equal to
  about 1e-10; they count once).
"""
import itertools

import numpy as np
import pytest
from scipy.optimize import linprog

import synth
from oracle import bab, mnc

DIRS = np.array([d for d in itertools.product((-1, 0, 1), repeat=3) if any(d)], dtype=np.float64)


@pytest.fixture(scope="module")
def group():
    from paper_2205_00263_gb300 import build
    build.build()
    from paper_2205_00263_gb300.api import mnc_group
    return mnc_group


def _random_octahedron(rng):
    """Lower bounds of d . x over a random affine image of a box (a valid,
    correlated octahedron around a point that straddles the origin)."""
    c = rng.uniform(-0.5, 0.5, 3)
    A = rng.normal(size=(3, 3)) * 0.6
    corners = np.array(list(itertools.product((-1.0, 1.0), repeat=3)))
    X = c + corners @ A.T
    return (DIRS @ X.T).min(1) - 1e-3


def _lifted_points(oct_lb):
    pts = []
    for sig in itertools.product((-1.0, 1.0), repeat=3):
        for tri in itertools.combinations(range(29), 3):
            n = np.concatenate([DIRS, np.diag(sig)])
            b = np.concatenate([oct_lb, np.zeros(3)])
            M = n[list(tri)]
            if abs(np.linalg.det(M)) < 1e-12:
                continue
            x = np.linalg.solve(M, b[list(tri)])
            if np.all(n @ x - b >= -1e-9 * (1 + np.abs(b))):
                y = np.where(np.array(sig) > 0, np.maximum(x, 0), 0.0)
                pts.append(np.concatenate([y, x]))
    return np.unique(np.round(np.array(pts), 12), axis=0)


@pytest.mark.parametrize("seed", range(6))
def test_rows_are_sound_per_orthant_and_facets(group, seed):
    oct_lb = _random_octahedron(np.random.default_rng(seed))
    P, Ph, p = group(oct_lb)
    assert P.shape[0] > 0
    assert np.allclose(np.linalg.norm(np.concatenate([P, Ph], 1), axis=1), 1.0)
    pts = _lifted_points(oct_lb)
    for r in range(P.shape[0]):
        # soundness: LP over each orthant piece, relu linear there
        for sig in itertools.product((-1.0, 1.0), repeat=3):
            sig = np.array(sig)
            c = -(Ph[r] + np.where(sig > 0, P[r], 0.0))      # maximise
            A_ub = np.concatenate([-DIRS, -np.diag(sig)])
            b_ub = np.concatenate([-oct_lb, np.zeros(3)])
            res = linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * 3, method="highs")
            if res.status == 0:
                assert -res.fun <= p[r] + 1e-8, (r, sig, -res.fun, p[r])
        # a facet: 6 affinely independent lifted points on it
        n6 = np.concatenate([P[r], Ph[r]])
        on = pts[np.abs(pts @ n6 - p[r]) < 1e-8]
        assert len(on) >= 6 and np.linalg.matrix_rank(on[1:] - on[0], tol=1e-9) == 5


def test_independent_neurons_give_no_rows(group):
    l = np.array([-1.0, -0.5, -2.0])
    u = np.array([2.0, 1.5, 0.5])
    oct_lb = np.array([np.minimum(d * l, d * u).sum() for d in DIRS])
    P, Ph, p = group(oct_lb)
    assert P.shape[0] == 0


def test_rows_match_the_oracle_on_network_octahedra(group):
    layers = synth.make_network(0)
    pr = synth.make_properties(0, layers, n=1, eps=synth.load_eps(0))[0]
    net, lo, hi, l, u, S, _, _ = bab.prepare(layers, pr.C, pr.d, pr.lo, pr.hi)
    n_rows = 0
    for t in (1, 2):
        groups = mnc.unstable_groups(l[t], u[t], 12)
        for lbs in mnc.octahedron_bounds(net, t, groups, l, u, S, lo, hi):
            ref = mnc.group_constraints(lbs)
            P, Ph, p = group(lbs)
            A = np.concatenate([P, Ph, p[:, None]], 1)
            if ref is None:
                assert A.shape[0] == 0
                continue
            B = np.concatenate([ref[0], ref[1], ref[2][:, None]], 1)
            # every oracle row is one of ours, and ours are distinct oracle rows
            dAB = np.abs(A[:, None, :] - B[None, :, :]).max(-1)
            assert dAB.min(0).max() <= 1e-7
            assert dAB.min(1).max() <= 1e-7
            assert np.abs(A[:, None, :] - A[None, :, :]).max(-1)[~np.eye(len(A), dtype=bool)].min() > 1e-7
            n_rows += A.shape[0]
    assert n_rows > 500
