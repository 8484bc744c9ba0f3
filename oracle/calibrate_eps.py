"""Calibrate the L-inf radius of each synthetic workload (writes synth/eps.json)
-- test infrastructure only: the stored radii are inputs of the tests and the
bench; the product path never runs this script.

For every property the largest radius eps_p at which a single DeepPoly pass
(root intermediate bounds, DeepPoly objective bound of every margin row, no
branching, no slope optimisation) verifies it is found by bisection on
[0, 0.5]; the workload radius is the largest eps at which at least 30% of the
properties verify, i.e. the ceil(0.3 n)-th largest eps_p, times 1.5.  Only the
FP64 oracle is used.  Run: ``python -m oracle.calibrate_eps 0 1``; the large
convolutional networks use a sample of properties and a narrower bracket
(``python -m oracle.calibrate_eps 3 2 --n 6 --iters 7 --hi 0.02``: DeepPoly
fails for every sampled property at 0.02).
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np
import torch

import synth
from . import core
from .core import DT


def deeppoly_verifies(net, lo, hi) -> bool:
    lo_t = torch.as_tensor(lo, dtype=DT)
    hi_t = torch.as_tensor(hi, dtype=DT)
    l, u, S = core.root_bounds(net, lo_t, hi_t)
    relax = {i: core.deeppoly_relax(l[i], u[i], S[i]) for i in l}
    R = net.R
    E = torch.eye(net.width(R + 1), dtype=DT)
    lb, _, _ = core.backsub_rows(net, R + 1, E, relax, lo_t, hi_t)
    return bool((lb > 0).all())


def critical_eps(net, x0, iters=20, hi_eps=0.5) -> float:
    a, b = 0.0, hi_eps
    for _ in range(iters):
        m = 0.5 * (a + b)
        lo, hi = synth.input_box(x0, m)
        if deeppoly_verifies(net, lo, hi):
            a = m
        else:
            b = m
    return a


def calibrate(cfg: int, n_props: int | None = None, iters: int = 20, frac: float = 0.3,
              factor: float = 1.5, hi_eps: float = 0.5) -> dict:
    layers = synth.make_network(cfg)
    props = synth.make_properties(cfg, layers, n=n_props)
    crit = []
    for pr in props:
        net = core.fold_property(core.load_net(layers), pr.C, pr.d)
        crit.append(critical_eps(net, pr.x0, iters, hi_eps))
        print(cfg, "property", pr.index, "critical eps", crit[-1], flush=True)
    s = sorted(crit, reverse=True)
    k = max(1, math.ceil(frac * len(s)))
    eps0 = s[k - 1]
    return dict(eps=eps0 * factor, eps_deeppoly_30pct=eps0, n_props=len(props),
                bisection_iters=iters, bracket=[0.0, hi_eps], critical=crit)


def main(argv):
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("cfgs", nargs="*", type=int, default=[0, 1])
    ap.add_argument("--n", type=int, default=None, help="properties (default: the config's)")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--hi", type=float, default=0.5, help="upper end of the bisection bracket")
    a = ap.parse_args(argv)
    cfgs = a.cfgs
    try:
        with open(synth.EPS_FILE) as f:
            data = json.load(f)
    except FileNotFoundError:
        data = {}
    for c in cfgs:
        t = time.time()
        r = calibrate(c, n_props=a.n, iters=a.iters, hi_eps=a.hi)
        r["seconds"] = round(time.time() - t, 1)
        data[str(c)] = r
        print(c, r["eps"], r["seconds"], flush=True)
        with open(synth.EPS_FILE) as f:   # other calibrations may have finished meanwhile
            data.update({k: v for k, v in json.load(f).items() if k != str(c)})
        with open(synth.EPS_FILE, "w") as f:
            json.dump(data, f, indent=1)


if __name__ == "__main__":
    torch.set_num_threads(max(1, torch.get_num_threads()))
    main(sys.argv[1:])
