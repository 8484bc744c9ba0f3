"""Seeded synthetic workloads shared by the FP64 oracle and the GPU library.

This module only draws inputs: network weights, input images, property rows,
input boxes and request streams.  It holds none of the verification method's
arithmetic (no bounding, relaxation, optimisation or branching); both sides
read the same arrays from here and each computes everything else itself.

The recipe follows the workload descriptions used throughout the project:

* weights are He-normal, std = sqrt(2 / fan_in) with fan_in = in_features or
  Ci*kh*kw, biases N(0, 0.01) (0.01 read as the standard deviation), drawn
  with ``numpy.random.default_rng(seed)`` in layer order, W before b, and
  stored as float32;
* images are uniform[0, 1] per pixel and channel followed by a 3x3 box blur
  that averages over the in-bounds neighbours only;
* property p of a network with seed s uses image seed s + 1000 + p, its true
  label is the argmax of the network output at the image, and its rows are
  the margins y_t - y_j for every j != t (the linear property folded into a
  final affine layer, Sec. 2.1);
* the input region is the L-inf ball of radius eps clipped to [0, 1].

These synthetic nets and images stand in for the MNIST / CIFAR10 networks and
test images of the paper's evaluation (Sec. 4, Tables 4 and 5), keeping their
input shapes and layer arithmetic; neither the datasets nor trained weights
are used.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CONFIGS", "make_network", "make_image", "make_properties", "input_box",
    "property_rows", "tiny_fc_net", "poisson_stream", "load_eps", "net_forward",
    "Property",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
EPS_FILE = os.path.join(_HERE, "eps.json")


def _conv_out(n: int, k: int, s: int, p: int) -> int:
    return (n + 2 * p - k) // s + 1


# Layer specs: ("fc", out[, src]) | ("conv", Co, k, stride, pad[, src[, scale]]) | ("relu",)
#              | ("add", a, b).
# Every op reads the previous op unless it names ``src`` (an op index, -1 for
# the network input); ``add`` sums two affine ops (residual sum).  ``scale``
# multiplies the drawn He-normal weights (residual branches).
CONFIGS = {
    0: dict(name="fc_784_100_100_10", seed=0, in_shape=(1, 28, 28), n_props=16,
            layers=[("fc", 100), ("relu",), ("fc", 100), ("relu",), ("fc", 10)],
            mnc_k=3, adam_steps=20, max_nodes=256, batch=1),
    1: dict(name="conv_small_28", seed=1, in_shape=(1, 28, 28), n_props=100,
            layers=[("conv", 16, 4, 2, 0), ("relu",), ("conv", 32, 4, 2, 0), ("relu",),
                    ("fc", 100), ("relu",), ("fc", 10)],
            mnc_k=0, adam_steps=20, max_nodes=256, batch=512),
    2: dict(name="conv_big_32", seed=2, in_shape=(3, 32, 32), n_props=100,
            layers=[("conv", 32, 3, 1, 1), ("relu",), ("conv", 32, 4, 2, 1), ("relu",),
                    ("conv", 64, 3, 1, 1), ("relu",), ("conv", 64, 4, 2, 1), ("relu",),
                    ("fc", 512), ("relu",), ("fc", 512), ("relu",), ("fc", 10)],
            mnc_k=3, adam_steps=20, max_nodes=256, batch=256, timeout_s=60.0),
    # ResNet6-like: stem, two basic blocks (3x3 s2 + 3x3 s1 main branch whose
    # second conv is scaled by 0.5, 1x1 s2 shortcut), FC100, FC10
    3: dict(name="resnet_32", seed=3, in_shape=(3, 32, 32), n_props=50,
            layers=[("conv", 16, 3, 1, 1), ("relu",),
                    ("conv", 32, 3, 2, 1, 1), ("relu",), ("conv", 32, 3, 1, 1, 3, 0.5),
                    ("conv", 32, 1, 2, 0, 1), ("add", 4, 5), ("relu",),
                    ("conv", 64, 3, 2, 1, 7), ("relu",), ("conv", 64, 3, 1, 1, 9, 0.5),
                    ("conv", 64, 1, 2, 0, 7), ("add", 10, 11), ("relu",),
                    ("fc", 100), ("relu",), ("fc", 10)],
            mnc_k=3, adam_steps=20, max_nodes=256, batch=128, timeout_s=120.0),
}


def make_network(cfg: int | dict) -> list[dict]:
    """Seeded He-normal network of a config (float32 arrays)."""
    spec = CONFIGS[cfg] if isinstance(cfg, int) else cfg
    rng = np.random.default_rng(spec["seed"])
    shapes = {-1: tuple(spec["in_shape"])}
    layers: list[dict] = []
    for i, L in enumerate(spec["layers"]):
        prev = i - 1
        if L[0] == "relu":
            layers.append(dict(kind="relu"))
            shapes[i] = shapes[prev]
            continue
        if L[0] == "add":
            layers.append(dict(kind="add", src=(L[1], L[2])))
            shapes[i] = shapes[L[1]]
            continue
        if L[0] == "fc":
            src = L[2] if len(L) > 2 else prev
            shape = shapes[src]
            fan_in = int(np.prod(shape))
            out = L[1]
            W = rng.standard_normal((out, fan_in)) * np.sqrt(2.0 / fan_in)
            b = rng.standard_normal(out) * 0.01
            d = dict(kind="fc", W=W.astype(np.float32), b=b.astype(np.float32))
            if len(L) > 2:
                d["src"] = src
            layers.append(d)
            shapes[i] = (out,)
        else:
            co, k, s, p = L[1:5]
            src = L[5] if len(L) > 5 else prev
            scale = L[6] if len(L) > 6 else 1.0
            ci, hi, wi = shapes[src]
            fan_in = ci * k * k
            W = rng.standard_normal((co, ci, k, k)) * np.sqrt(2.0 / fan_in) * scale
            b = rng.standard_normal(co) * 0.01
            ho, wo = _conv_out(hi, k, s, p), _conv_out(wi, k, s, p)
            d = dict(kind="conv", W=W.astype(np.float32), b=b.astype(np.float32),
                     stride=s, pad=p, in_shape=(ci, hi, wi), out_shape=(co, ho, wo))
            if len(L) > 5:
                d["src"] = src
            layers.append(d)
            shapes[i] = (co, ho, wo)
    return layers


def tiny_fc_net(seed: int, dims: list[int], scale: float = 1.0) -> list[dict]:
    """Small fully connected ReLU net (He-normal, seeded) for exact checks."""
    rng = np.random.default_rng(seed)
    layers: list[dict] = []
    for i in range(len(dims) - 1):
        W = rng.standard_normal((dims[i + 1], dims[i])) * np.sqrt(2.0 / dims[i]) * scale
        b = rng.standard_normal(dims[i + 1]) * 0.1
        layers.append(dict(kind="fc", W=W.astype(np.float32), b=b.astype(np.float32)))
        if i < len(dims) - 2:
            layers.append(dict(kind="relu"))
    return layers


def _blur3(img: np.ndarray) -> np.ndarray:
    """3x3 box blur per channel, averaging the in-bounds neighbours only."""
    c, h, w = img.shape
    acc = np.zeros_like(img)
    cnt = np.zeros((h, w))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ys0, ys1 = max(0, dy), h + min(0, dy)
            xs0, xs1 = max(0, dx), w + min(0, dx)
            acc[:, ys0 - dy:ys1 - dy, xs0 - dx:xs1 - dx] += img[:, ys0:ys1, xs0:xs1]
            cnt[ys0 - dy:ys1 - dy, xs0 - dx:xs1 - dx] += 1
    return acc / cnt


def make_image(seed: int, in_shape) -> np.ndarray:
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 1.0, size=tuple(in_shape))
    return _blur3(img).astype(np.float32)


def net_forward(layers: list[dict], x: np.ndarray, collect: list | None = None) -> np.ndarray:
    """Plain float64 network evaluation (labels the images; with `collect`, the
    input of every ReLU is appended to it in layer order)."""
    out = {-1: np.asarray(x, dtype=np.float64).reshape(-1)}
    for i, L in enumerate(layers):
        k = L["kind"]
        if k == "add":
            out[i] = out[L["src"][0]] + out[L["src"][1]]
            continue
        h = out[L.get("src", i - 1)]
        if k == "relu":
            if collect is not None:
                collect.append(h)
            out[i] = np.maximum(h, 0.0)
        elif k == "fc":
            out[i] = L["W"].astype(np.float64) @ h + L["b"].astype(np.float64)
        else:
            ci, hi, wi = L["in_shape"]
            co, ho, wo = L["out_shape"]
            s, p = L["stride"], L["pad"]
            W = L["W"].astype(np.float64)
            kk = W.shape[2]
            xi = np.zeros((ci, hi + 2 * p, wi + 2 * p))
            xi[:, p:p + hi, p:p + wi] = h.reshape(ci, hi, wi)
            o = np.zeros((co, ho, wo))
            for kh in range(kk):
                for kw in range(kk):
                    patch = xi[:, kh:kh + s * (ho - 1) + 1:s, kw:kw + s * (wo - 1) + 1:s]
                    o += np.einsum("oc,chw->ohw", W[:, :, kh, kw], patch)
            out[i] = (o + L["b"].astype(np.float64)[:, None, None]).reshape(-1)
    return out[len(layers) - 1]


def property_rows(label: int, n_classes: int) -> tuple[np.ndarray, np.ndarray]:
    """Margin rows e_t - e_j (j != t) and zero offsets: goal C f(x) + d > 0."""
    rows = [j for j in range(n_classes) if j != label]
    C = np.zeros((len(rows), n_classes), dtype=np.float32)
    for r, j in enumerate(rows):
        C[r, label] = 1.0
        C[r, j] = -1.0
    return C, np.zeros(len(rows), dtype=np.float32)


def input_box(x0: np.ndarray, eps: float) -> tuple[np.ndarray, np.ndarray]:
    """L-inf ball of radius eps around x0, clipped to the pixel range [0, 1]."""
    x0 = np.asarray(x0, dtype=np.float32).reshape(-1)
    lo = np.maximum(0.0, x0 - np.float32(eps)).astype(np.float32)
    hi = np.minimum(1.0, x0 + np.float32(eps)).astype(np.float32)
    return lo, hi


@dataclass
class Property:
    index: int
    x0: np.ndarray
    label: int
    C: np.ndarray
    d: np.ndarray
    lo: np.ndarray = field(default=None)
    hi: np.ndarray = field(default=None)


def make_properties(cfg: int, layers: list[dict] | None = None, n: int | None = None,
                    eps: float | None = None, start: int = 0) -> list[Property]:
    spec = CONFIGS[cfg]
    layers = layers if layers is not None else make_network(cfg)
    n = spec["n_props"] if n is None else n
    props = []
    for p in range(start, start + n):
        x0 = make_image(spec["seed"] + 1000 + p, spec["in_shape"]).reshape(-1)
        y = net_forward(layers, x0)
        t = int(np.argmax(y))
        C, d = property_rows(t, y.shape[0])
        pr = Property(index=p, x0=x0, label=t, C=C, d=d)
        if eps is not None:
            pr.lo, pr.hi = input_box(x0, eps)
        props.append(pr)
    return props


def load_eps(cfg: int) -> float:
    """Calibrated radius of a config, written by the oracle's calibration script."""
    with open(EPS_FILE) as f:
        return float(json.load(f)[str(cfg)]["eps"])


def poisson_stream(rate: float = 4.0, n: int = 400, seed: int = 4,
                   nets=(1, 2)) -> list[dict]:
    """Request stream: exponential inter-arrivals, network drawn uniformly."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    which = rng.integers(0, len(nets), size=n)
    t = np.cumsum(gaps)
    return [dict(arrival_s=float(t[i]), cfg=int(nets[which[i]]), input_seed=4_000_000 + i)
            for i in range(n)]
