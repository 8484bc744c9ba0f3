"""The synthetic workloads follow their stated recipe (CPU only).

The seeded networks, images, properties and request stream stand in for the
paper's MNIST / CIFAR10 networks and test images (Sec. 4, Tables 4 and 5), so
their shapes and statistics are pinned here against the configuration specs:
layer shapes, He-normal weights (std sqrt(2 / fan_in), residual-branch convs
scaled by 0.5), N(0, 0.01) biases, blurred uniform images, margin rows, input
boxes clipped to [0, 1], and the Poisson request stream.
"""
import numpy as np
import pytest

import synth


def _affine(layers):
    return [L for L in layers if L["kind"] in ("fc", "conv")]


@pytest.mark.parametrize("cfg,shapes", [
    (0, [(100, 784), (100, 100), (10, 100)]),
    (1, [(16, 1, 4, 4), (32, 16, 4, 4), (100, 800), (10, 100)]),
    (2, [(32, 3, 3, 3), (32, 32, 4, 4), (64, 32, 3, 3), (64, 64, 4, 4), (512, 4096),
         (512, 512), (10, 512)]),
    (3, [(16, 3, 3, 3), (32, 16, 3, 3), (32, 32, 3, 3), (32, 16, 1, 1), (64, 32, 3, 3),
         (64, 64, 3, 3), (64, 32, 1, 1), (100, 4096), (10, 100)]),
])
def test_layer_shapes(cfg, shapes):
    layers = synth.make_network(cfg)
    assert [L["W"].shape for L in _affine(layers)] == shapes
    assert all(L["W"].dtype == np.float32 and L["b"].dtype == np.float32 for L in _affine(layers))


def test_conv_output_shapes():
    """conv16 4x4 s2 on 28x28 gives 13x13, conv32 4x4 s2 then 5x5; conv-big
    keeps 32x32 at stride 1 (pad 1) and halves it at the 4x4 s2 (pad 1) layers."""
    c1 = [L["out_shape"] for L in synth.make_network(1) if L["kind"] == "conv"]
    assert c1 == [(16, 13, 13), (32, 5, 5)]
    c2 = [L["out_shape"] for L in synth.make_network(2) if L["kind"] == "conv"]
    assert c2 == [(32, 32, 32), (32, 16, 16), (64, 16, 16), (64, 8, 8)]
    c3 = [L["out_shape"] for L in synth.make_network(3) if L["kind"] == "conv"]
    assert c3 == [(16, 32, 32), (32, 16, 16), (32, 16, 16), (32, 16, 16), (64, 8, 8),
                  (64, 8, 8), (64, 8, 8)]


def test_he_normal_statistics():
    """Sample std of every large weight tensor within 5% of sqrt(2 / fan_in)
    (times 0.5 on the residual branches' second convs); bias std about 0.01."""
    for cfg in (0, 1, 2, 3):
        scaled = {2, 5} if cfg == 3 else set()   # second conv of each basic block
        biases = []
        for k, L in enumerate(_affine(synth.make_network(cfg))):
            W = L["W"].astype(np.float64)
            fan_in = W.shape[1] * (W.shape[2] * W.shape[3] if W.ndim == 4 else 1)
            want = np.sqrt(2.0 / fan_in) * (0.5 if k in scaled else 1.0)
            if W.size >= 2000:
                assert abs(W.std() / want - 1.0) < 0.05, (cfg, k)
                assert abs(W.mean()) < 0.1 * want, (cfg, k)
            biases.append(L["b"].astype(np.float64))
        b = np.concatenate(biases)
        assert 0.007 < b.std() < 0.013


def test_images_properties_and_boxes():
    """Images are blurred uniform[0, 1] pixels (in [0, 1], smoother than raw
    uniform noise); each property's rows are the margins y_t - y_j, j != t,
    with t the network's argmax; the box is the eps ball clipped to [0, 1]."""
    layers = synth.make_network(1)
    props = synth.make_properties(1, layers, n=5, eps=0.1)
    for p in props:
        x = p.x0.reshape(28, 28)
        assert x.min() >= 0.0 and x.max() <= 1.0
        # a 3x3 mean of uniform[0, 1] has variance (1/12) / 9 in the interior
        assert x[1:-1, 1:-1].std() < 0.15
        y = synth.net_forward(layers, p.x0)
        assert p.label == int(np.argmax(y))
        assert p.C.shape == (9, 10) and np.all(p.d == 0)
        m = p.C.astype(np.float64) @ y
        others = [j for j in range(10) if j != p.label]
        assert np.allclose(m, y[p.label] - y[others])
        assert np.all(p.lo == np.maximum(0.0, p.x0 - np.float32(0.1)))
        assert np.all(p.hi == np.minimum(1.0, p.x0 + np.float32(0.1)))
        assert np.all(p.lo >= 0.0) and np.all(p.hi <= 1.0)
    # property p of config s uses image seed s + 1000 + p
    assert np.array_equal(props[3].x0, synth.make_image(1 + 1000 + 3, (1, 28, 28)).reshape(-1))


def test_poisson_stream():
    """Rate 4/s, 400 requests, seed 4: mean gap near 1/4 s, arrivals increasing,
    networks drawn from those given, input seeds 4e6 + index."""
    s = synth.poisson_stream(rate=4.0, n=400, seed=4, nets=(1, 2, 3))
    t = np.array([r["arrival_s"] for r in s])
    assert len(s) == 400 and np.all(np.diff(t) > 0)
    assert abs(np.diff(np.concatenate([[0.0], t])).mean() - 0.25) < 0.05
    assert {r["cfg"] for r in s} == {1, 2, 3}
    assert [r["input_seed"] for r in s[:3]] == [4_000_000, 4_000_001, 4_000_002]
