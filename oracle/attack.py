"""Adversarial pre-attack of the oracle (Sec. 4, experimental setup) -- test
infrastructure only: the GPU library and its tests compare against it; no
product path imports it.

Before branch-and-bound, MN-BaB searches for counterexamples with an
adversarial attack.  Reading (the paper defers the attack to cited work):
projected gradient descent with sign steps on the margin of one property row,

    f_r(x) = (C f(x) + d)_r,
    x_{k+1} = clip(x_k - alpha * sign(grad f_r(x_k)), lo, hi),   k = 0 .. steps-1,
    alpha_j = 2.5 * (hi_j - lo_j) / (2 * steps),

from caller-given starting points x_0 (one per restart; random numbers are
inputs, not drawn here), and the result of a row is the smallest margin over all
iterates of all restarts with its first minimiser (restarts in order, iterates in
order).  ReLU'(0) = 1 (the derivative autograd gives the forward pass's clamp)
and sign(0) = 0.  A negative margin is a counterexample.

Gradients are exact reverse-mode derivatives of the FP64 forward pass (torch
autograd as a library step); they are pinned by central finite differences.
"""
from __future__ import annotations

import numpy as np
import torch

from . import core
from .core import DT


def margin_and_grad(net: core.Net, x: np.ndarray, row: int) -> tuple[float, np.ndarray]:
    """f_r(x) and its gradient (net is the property-folded network)."""
    xt = torch.as_tensor(np.asarray(x, np.float64), dtype=DT).reshape(1, -1).clone()
    xt.requires_grad_(True)
    y = net.forward(xt)[0, row]
    y.backward()
    return float(y.detach()), xt.grad.detach().numpy().reshape(-1).copy()


def step_size(lo: np.ndarray, hi: np.ndarray, steps: int) -> np.ndarray:
    return 2.5 * (np.asarray(hi, np.float64) - np.asarray(lo, np.float64)) / (2.0 * steps)


def pgd_row(net: core.Net, lo, hi, row: int, starts: np.ndarray, steps: int):
    """Smallest margin of row `row` over all iterates, its first minimiser, and
    the last iterate of the last restart."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    alpha = step_size(lo, hi, steps)
    best, bx, last = np.inf, None, None
    for x0 in np.asarray(starts, np.float64):
        x = np.clip(x0, lo, hi)
        for k in range(steps + 1):
            f, g = margin_and_grad(net, x, row)
            if f < best:
                best, bx = f, x.copy()
            if k == steps:
                break
            x = np.clip(x - alpha * np.sign(g), lo, hi)
        last = x
    return best, bx, last


def attack(layers, C, d, lo, hi, starts: np.ndarray, steps: int):
    """Per property row: (smallest margin, minimiser) over all restarts."""
    net = core.fold_property(core.load_net(layers), np.asarray(C), np.asarray(d))
    out = []
    for r in range(np.asarray(C).shape[0]):
        best, bx, _ = pgd_row(net, lo, hi, r, starts, steps)
        out.append((best, bx))
    return out


def splitmix64(state: int) -> tuple[int, int]:
    """One output of SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference
    code): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds and a
    final xor-shift.  Returns (output, new state)."""
    m = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & m
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31), state


def splitmix_uniform(seed: int, index: int) -> float:
    """Counter-based uniform in [0, 1): the top 53 bits of the SplitMix64
    output at state seed + index * 0x9E3779B97F4A7C15 (its (index + 1)-th
    output from state seed)."""
    m = (1 << 64) - 1
    out, _ = splitmix64((seed + index * 0x9E3779B97F4A7C15) & m)
    return (out >> 11) * (1.0 / (1 << 53))


def attack_starts(lo, hi, n_starts: int, seed: int) -> np.ndarray:
    """Starting points of the pre-attack run inside branch-and-bound: the box
    centre, then points lo + (hi - lo) u with u = splitmix_uniform(seed,
    (k - 1) d0 + j) for start k >= 1 and coordinate j."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d0 = lo.size
    out = np.empty((n_starts, d0))
    out[0] = 0.5 * (lo + hi)
    for k in range(1, n_starts):
        u = np.array([splitmix_uniform(seed, (k - 1) * d0 + j) for j in range(d0)])
        out[k] = lo + (hi - lo) * u
    return out
