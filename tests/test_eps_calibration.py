"""The stored workload radii (synth/eps.json) are the oracle calibration's
output, reproduced here on the CPU.

The radius of a workload is 1.5 x the largest eps at which a single DeepPoly
pass verifies at least 30% of its properties (per-property critical radii by
bisection).  Config 0 is recomputed in full; config 1 on two of its
properties; for every config the stored radius follows from its stored
critical radii by that rule.
"""
import json
import math

import pytest

import synth
from oracle import calibrate_eps, core


def _stored():
    with open(synth.EPS_FILE) as f:
        return json.load(f)


def test_rule_from_the_stored_critical_radii():
    for cfg, r in _stored().items():
        s = sorted(r["critical"], reverse=True)
        k = max(1, math.ceil(0.3 * len(s)))
        assert r["eps_deeppoly_30pct"] == s[k - 1], cfg
        assert r["eps"] == pytest.approx(1.5 * s[k - 1], rel=1e-15), cfg
        assert synth.load_eps(int(cfg)) == r["eps"]


def test_config0_recomputed():
    r = calibrate_eps.calibrate(0)
    st = _stored()["0"]
    # bisection on a 2^-20 grid of [0, 0.5]: equal up to a grid step where
    # rounding flips a decision at the verification boundary
    assert r["critical"] == pytest.approx(st["critical"], abs=1e-6)
    assert r["eps"] == pytest.approx(st["eps"], abs=1.5e-6)


@pytest.mark.parametrize("p", [1, 4])
def test_config1_sampled_properties_recomputed(p):
    layers = synth.make_network(1)
    pr = synth.make_properties(1, layers, n=1, start=p)[0]
    net = core.fold_property(core.load_net(layers), pr.C, pr.d)
    assert calibrate_eps.critical_eps(net, pr.x0) == pytest.approx(
        _stored()["1"]["critical"][p], abs=1e-6)
