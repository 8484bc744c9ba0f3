"""Thin Python binding of libmnbab: argument marshalling only.

Every step of the bounding path runs in the library's CUDA kernels; this
module converts numpy arrays to C pointers, checks status codes and raises
``MnbabError`` with the library's message.  The library owns its device
memory; the optional torch stream handle is only passed through.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib as L


class MnbabError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libmnbab error {code}: {msg}")
        self.code = code


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fp(a: np.ndarray):
    return a.ctypes.data_as(L.FP)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(L.IP)


@dataclass
class NodeParams:
    """Parameter block of one node (mnbab_export_params layout)."""
    split_layer: int
    R: int
    l: np.ndarray
    u: np.ndarray
    S: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    gamma: np.ndarray

    def pack(self) -> bytes:
        SD = self.l.size
        hdr = np.array([self.split_layer, self.R, SD, self.gamma.size], dtype=np.int32)
        return b"".join([hdr.tobytes(), _f32(self.l).tobytes(), _f32(self.u).tobytes(),
                         np.asarray(self.S, np.int8).tobytes(), _f32(self.alpha).tobytes(),
                         _f32(self.beta).tobytes(), _f32(self.gamma).tobytes()])

    @staticmethod
    def unpack(buf: bytes) -> "NodeParams":
        hdr = np.frombuffer(buf[:16], dtype=np.int32)
        split, R, SD, E = (int(v) for v in hdr)
        o = 16
        def take(dt, n, size):
            nonlocal o
            a = np.frombuffer(buf[o:o + n * size], dtype=dt).copy()
            o += n * size
            return a
        l = take(np.float32, SD, 4)
        u = take(np.float32, SD, 4)
        S = take(np.int8, SD, 1)
        al = take(np.float32, SD, 4)
        be = take(np.float32, SD, 4)
        ga = take(np.float32, E, 4)
        return NodeParams(split, R, l, u, S, al, be, ga)


class Net:
    def __init__(self, ctx: "Context", handle, layers):
        self.ctx, self.h = ctx, handle
        out_dim = {}
        self.d0 = None
        self.relu_dims = []
        for i, Ly in enumerate(layers):
            k = Ly["kind"]
            if k == "relu":
                out_dim[i] = out_dim[i - 1]
                self.relu_dims.append(out_dim[i])
            elif k == "add":
                out_dim[i] = out_dim[Ly["src"][0]]
            else:
                if self.d0 is None and Ly.get("src", i - 1) < 0:   # reads the network input
                    self.d0 = (int(np.prod(Ly["W"].shape[1:])) if k == "fc"
                               else int(np.prod(Ly["in_shape"])))
                out_dim[i] = Ly["W"].shape[0] if k == "fc" else int(np.prod(Ly["out_shape"]))
        self.R = len(self.relu_dims)
        self.SD = int(sum(self.relu_dims))


class Prop:
    def __init__(self, ctx: "Context", handle, net: Net, n_rows: int):
        self.ctx, self.h, self.net, self.n_rows = ctx, handle, net, n_rows


class Context:
    """One libmnbab context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None,
                 node_capacity: int = 0, max_mnc_rows: int = 0, row_chunk: int = 0,
                 gemm_path: int = 0, graphs: bool = False):
        self.lib = L.load()
        o = L.Options(device, hbm_budget_bytes, stream, node_capacity, max_mnc_rows, row_chunk,
                      gemm_path, 1 if graphs else 0)
        h = C.c_void_p()
        st = self.lib.mnbab_create(C.byref(o), C.byref(h))
        if st != 0:
            raise MnbabError(st, "mnbab_create failed (no CUDA device?)")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.mnbab_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st != 0:
            msg = self.lib.mnbab_last_error(self.h)
            raise MnbabError(st, msg.decode() if msg else "")

    # ---- network / property ------------------------------------------------
    def load_network(self, layers: list[dict]) -> Net:
        descs = (L.LayerDesc * len(layers))()
        keep = []
        for i, Ly in enumerate(layers):
            d = descs[i]
            if Ly["kind"] == "relu":
                d.kind = L.RELU
                continue
            if Ly["kind"] == "add":
                d.kind = L.ADD
                d.src_a, d.src_b = Ly["src"][0] + 1, Ly["src"][1] + 1
                continue
            if "src" in Ly:   # op index it reads; -1 = the network input
                d.src_a = Ly["src"] + 1 if Ly["src"] >= 0 else -1
            W = _f32(Ly["W"])
            b = _f32(Ly["b"])
            keep += [W, b]
            d.W, d.b = _fp(W), _fp(b)
            if Ly["kind"] == "fc":
                d.kind = L.FC
                d.in_c, d.in_h, d.in_w = W.shape[1], 1, 1
                d.out_c, d.out_h, d.out_w = W.shape[0], 1, 1
                d.k, d.stride, d.pad = 1, 1, 0
            else:
                d.kind = L.CONV2D
                d.in_c, d.in_h, d.in_w = Ly["in_shape"]
                d.out_c, d.out_h, d.out_w = Ly["out_shape"]
                d.k, d.stride, d.pad = W.shape[2], Ly["stride"], Ly["pad"]
        h = C.c_void_p()
        self._ck(self.lib.mnbab_load_network(self.h, descs, len(layers), C.byref(h)))
        return Net(self, h, layers)

    def set_property(self, net: Net, lo, hi, Cm, d=None) -> Prop:
        lo, hi, Cm = _f32(lo).reshape(-1), _f32(hi).reshape(-1), _f32(Cm)
        d = np.zeros(Cm.shape[0], np.float32) if d is None else _f32(d)
        h = C.c_void_p()
        self._ck(self.lib.mnbab_set_property(self.h, net.h, _fp(lo), _fp(hi), _fp(Cm), _fp(d),
                                             Cm.shape[0], C.byref(h)))
        return Prop(self, h, net, Cm.shape[0])

    def root_bounds(self, prop: Prop, layer: int):
        d = prop.net.relu_dims[layer - 1]
        l = np.empty(d, np.float32)
        u = np.empty(d, np.float32)
        self._ck(self.lib.mnbab_get_root_bounds(self.h, prop.h, layer, _fp(l), _fp(u)))
        return l, u

    def set_mnc(self, prop: Prop, layer: int, idx, P, Ph, p):
        idx = np.ascontiguousarray(np.asarray(idx, np.int32))
        P, Ph, p = _f32(P), _f32(Ph), _f32(p)
        n_rows = idx.shape[0]
        k = idx.shape[1] if idx.ndim == 2 else 3
        self._ck(self.lib.mnbab_set_mnc(self.h, prop.h, layer, n_rows, k, _ip(idx), _fp(P),
                                        _fp(Ph), _fp(p)))

    def generate_mnc(self, prop: Prop, max_groups: int = 2000) -> int:
        """Generates and uploads the multi-neuron constraints of every ReLU layer
        from the property's root bounds (mnbab_generate_mnc); returns the rows."""
        n = C.c_int64()
        self._ck(self.lib.mnbab_generate_mnc(self.h, prop.h, max_groups, C.byref(n)))
        return n.value

    def get_mnc(self, prop: Prop, layer: int):
        """(idx [e, 3], P [e, 3], Phat [e, 3], p [e]) of one ReLU layer."""
        n = C.c_int32()
        st = self.lib.mnbab_get_mnc(self.h, prop.h, layer, 0, None, None, None, None, C.byref(n))
        if st not in (0, -2):
            self._ck(st)
        e = n.value
        idx = np.zeros((e, 3), np.int32)
        P = np.zeros((e, 3), np.float32)
        Ph = np.zeros((e, 3), np.float32)
        p = np.zeros(e, np.float32)
        if e:
            self._ck(self.lib.mnbab_get_mnc(self.h, prop.h, layer, e, _ip(idx), _fp(P), _fp(Ph),
                                            _fp(p), C.byref(n)))
        return idx, P, Ph, p

    def set_leaf_steps(self, prop: Prop, steps: int):
        """Adam steps of the exact completion of fully split leaves (0: off)."""
        self._ck(self.lib.mnbab_set_leaf_steps(self.h, prop.h, steps))

    def set_budget(self, prop: Prop, n: int):
        self._ck(self.lib.mnbab_set_budget(self.h, prop.h, n))

    def set_timeout(self, prop: Prop, seconds: float):
        """Wall-clock limit of the property from its first BaB step (0: none)."""
        self._ck(self.lib.mnbab_set_timeout(self.h, prop.h, float(seconds)))

    def status(self, prop: Prop):
        """(nodes bounded, ended by its timeout, seconds since its first step)."""
        b, t, e = C.c_int32(), C.c_int32(), C.c_double()
        self._ck(self.lib.mnbab_get_status(self.h, prop.h, C.byref(b), C.byref(t), C.byref(e)))
        return b.value, bool(t.value), e.value

    def set_branching(self, prop: Prop, cab: bool):
        """ACS (cab=False) or cost-adjusted ACS (cab=True) for this property."""
        self._ck(self.lib.mnbab_set_branching(self.h, prop.h, 1 if cab else 0))

    # ---- nodes ------------------------------------------------------------
    def node_root(self, prop: Prop, row: int) -> int:
        out = L.node_id()
        self._ck(self.lib.mnbab_node_root(self.h, prop.h, row, C.byref(out)))
        return out.value

    def node_free(self, node: int):
        self._ck(self.lib.mnbab_node_free(self.h, node))

    def export_params(self, node: int) -> NodeParams:
        n = C.c_size_t()
        self._ck(self.lib.mnbab_export_params(self.h, node, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._ck(self.lib.mnbab_export_params(self.h, node, buf, C.byref(n)))
        return NodeParams.unpack(buf.raw)

    def import_params(self, node: int, p: NodeParams):
        b = p.pack()
        self._ck(self.lib.mnbab_import_params(self.h, node, b, len(b)))

    @staticmethod
    def _ids(nodes):
        a = (L.node_id * len(nodes))(*nodes)
        return a, len(nodes)

    def bound_batch(self, nodes, with_ub=True):
        ids, n = self._ids(nodes)
        lb = np.empty(n, np.float32)
        ub = np.empty(n, np.float32) if with_ub else None
        self._ck(self.lib.mnbab_bound_batch(self.h, ids, n, _fp(lb), _fp(ub) if with_ub else None))
        return (lb, ub) if with_ub else lb

    def deeppoly_batch(self, nodes):
        ids, n = self._ids(nodes)
        lb = np.empty(n, np.float32)
        self._ck(self.lib.mnbab_deeppoly_batch(self.h, ids, n, _fp(lb)))
        return lb

    def bound_grad(self, nodes, SD: int, E: int):
        ids, n = self._ids(nodes)
        lb = np.empty(n, np.float32)
        g = np.empty(n * (2 * SD + E), np.float32)
        self._ck(self.lib.mnbab_bound_grad(self.h, ids, n, _fp(lb), _fp(g)))
        g = g.reshape(n, 2 * SD + E)
        return lb, g[:, :SD], g[:, SD:2 * SD], g[:, 2 * SD:]

    def set_params(self, nodes, params):
        """Writes each node's (alpha, beta, gamma) from one flat float array laid
        out per node as alpha[SD], beta[SD], gamma[E] (mnbab_set_params)."""
        ids, n = self._ids(nodes)
        p = _f32(params).reshape(-1)
        self._ck(self.lib.mnbab_set_params(self.h, ids, n, _fp(p)))

    def optimize(self, nodes, steps=20, lr_alpha=0.1, lr_beta=0.05, lr_gamma=0.05, beta1=0.9,
                 beta2=0.999, eps=1e-8, grad_floor=0.0, eps_rel=0.0):
        ids, n = self._ids(nodes)
        a = L.Adam(steps, lr_alpha, lr_beta, lr_gamma, beta1, beta2, eps, grad_floor, eps_rel)
        best = np.empty(n, np.float32)
        self._ck(self.lib.mnbab_optimize(self.h, ids, n, C.byref(a), _fp(best)))
        return best

    def set_intermediate_steps(self, prop: Prop, steps: int):
        """Optimised intermediate bounds at the property's root when it starts."""
        self._ck(self.lib.mnbab_set_intermediate_steps(self.h, prop.h, steps))

    def optimize_intermediate(self, nodes, first_layer=2, steps=20, lr_alpha=0.1, lr_beta=0.05,
                              beta1=0.9, beta2=0.999, eps=1e-8, grad_floor=0.0, eps_rel=0.0,
                              lr_gamma=0.05):
        """Optimised intermediate bounds of the nodes (shared per-layer sets of
        alpha, beta and, with multi-neuron constraints, gamma); returns the
        number of rows bounded."""
        ids, n = self._ids(nodes)
        a = L.Adam(steps, lr_alpha, lr_beta, lr_gamma, beta1, beta2, eps, grad_floor, eps_rel)
        rows = C.c_int64()
        self._ck(self.lib.mnbab_optimize_intermediate(self.h, ids, n, first_layer, C.byref(a),
                                                      C.byref(rows)))
        return rows.value

    def score_branches(self, nodes):
        ids, n = self._ids(nodes)
        lay = np.empty(n, np.int32)
        neu = np.empty(n, np.int32)
        sc = np.empty(n, np.float32)
        self._ck(self.lib.mnbab_score_branches(self.h, ids, n, _ip(lay), _ip(neu), _fp(sc)))
        return lay, neu, sc

    # ---- branch and bound ----------------------------------------------------
    def bab_step(self, props, max_nodes: int, steps: int = 20, adam: dict | None = None):
        arr = (C.c_void_p * len(props))(*[p.h.value for p in props])
        a = L.Adam(steps, *(adam or {}).get("rates", (0.1, 0.05, 0.05, 0.9, 0.999, 1e-8, 0.0,
                                                       0.0)))
        st = L.StepStats()
        self._ck(self.lib.mnbab_bab_step(self.h, arr, len(props), max_nodes, C.byref(a),
                                         C.byref(st)))
        return {k: getattr(st, k) for k, _ in L.StepStats._fields_}

    def verdict(self, prop: Prop, row: int = -1):
        v = C.c_int32()
        lb = C.c_float()
        x = np.zeros(prop.net.d0, np.float32)
        self._ck(self.lib.mnbab_get_verdict(self.h, prop.h, row, C.byref(v), C.byref(lb), _fp(x)))
        return v.value, lb.value, x

    def trace(self, prop: Prop):
        n = C.c_int32()
        self._ck(self.lib.mnbab_get_trace(self.h, prop.h, None, 0, C.byref(n)))
        recs = (L.TraceRec * max(1, n.value))()
        self._ck(self.lib.mnbab_get_trace(self.h, prop.h, recs, n.value, C.byref(n)))
        return [{k: getattr(recs[i], k) for k, _ in L.TraceRec._fields_} for i in range(n.value)]

    def queue_size(self, prop: Prop) -> int:
        n = C.c_int32()
        self._ck(self.lib.mnbab_queue_size(self.h, prop.h, C.byref(n)))
        return n.value

    VARIANTS = ("auto", "tc", "igemm", "row", "plain", "g32", "g64", "splitk")

    def autotune(self, net: Net, max_rows: int = 4096):
        """Times the kernel variants of every affine edge, direction and row
        bucket and keeps the fastest; returns one dict per (edge, dir, bucket)."""
        n = C.c_int32()
        self._ck(self.lib.mnbab_autotune(self.h, net.h, max_rows, None, 0, C.byref(n)))
        arr = (L.TuneRec * max(1, n.value))()
        self._ck(self.lib.mnbab_autotune(self.h, net.h, max_rows, arr, n.value, C.byref(n)))
        out = []
        for i in range(n.value):
            r = arr[i]
            out.append(dict(node=r.node, edge=r.edge, dir=r.dir, rows=r.rows,
                            variant=self.VARIANTS[r.variant],
                            ms={self.VARIANTS[v]: r.ms[v] for v in range(8) if r.ms[v] >= 0}))
        return out

    def set_variant(self, net: Net, node: int, edge: int, direction: int, variant: str):
        """Fixes the kernel variant of one affine edge and direction ("auto" restores)."""
        self._ck(self.lib.mnbab_set_variant(self.h, net.h, node, edge, direction,
                                            self.VARIANTS.index(variant)))

    def set_attack_path(self, path: int):
        """0 auto, 1 one kernel per (row, start), 2 per-layer kernels."""
        self._ck(self.lib.mnbab_set_attack_path(self.h, path))

    def set_attack(self, prop: Prop, n_starts: int, steps: int, seed: int = 0):
        """Pre-attack when the property starts (box centre plus SplitMix64 starts)."""
        self._ck(self.lib.mnbab_set_attack(self.h, prop.h, n_starts, steps, seed))

    def attack(self, prop: Prop, starts, steps: int):
        """Adversarial pre-attack (sign-step PGD per property row from the given
        starting points [n_starts][d0]); returns (best margin per row, minimisers)."""
        st = _f32(np.asarray(starts).reshape(-1, prop.net.d0))
        best = np.empty(prop.n_rows, np.float32)
        x = np.empty((prop.n_rows, prop.net.d0), np.float32)
        self._ck(self.lib.mnbab_attack(self.h, prop.h, st.shape[0], int(steps), _fp(st),
                                       _fp(best), _fp(x)))
        return best, x

    # ---- profiling --------------------------------------------------------
    def profile(self, enable: bool):
        self._ck(self.lib.mnbab_profile(self.h, 1 if enable else 0))

    def profile_mask(self, classes=None):
        """Time only the named kernel classes with CUDA events (None: all)."""
        if classes is None:
            mask = (1 << 64) - 1
        else:
            stats, _ = self.profile_read()
            names = list(stats)
            mask = 0
            for c in classes:
                mask |= 1 << names.index(c)
        self._ck(self.lib.mnbab_profile_mask(self.h, mask))

    def profile_read(self):
        """({kernel class: {launches, ms, flops, bytes}}, total launches)."""
        arr = (L.KernelStat * 32)()
        n = C.c_int32()
        tot = C.c_int64()
        self._ck(self.lib.mnbab_profile_read(self.h, arr, 32, C.byref(n), C.byref(tot)))
        out = {}
        for i in range(n.value):
            k = arr[i]
            out[k.name.decode()] = dict(launches=k.launches, ms=k.ms, flops=k.flops, bytes=k.bytes)
        return out, tot.value

    # ---- serving ------------------------------------------------------------
    def submit(self, prop: Prop, timeout_s: float = 0.0) -> int:
        t = C.c_uint64()
        self._ck(self.lib.mnbab_submit(self.h, prop.h, timeout_s, C.byref(t)))
        return t.value

    def set_serving_budget(self, nbytes: int):
        """HBM bytes the active requests' node slots may hold (0: the context's budget)."""
        self._ck(self.lib.mnbab_set_serving_budget(self.h, int(nbytes)))

    def serve_step(self, max_nodes: int, steps: int = 20):
        a = L.Adam(steps, 0.1, 0.05, 0.05, 0.9, 0.999, 1e-8, 0.0, 0.0)
        st = L.ServeStats()
        self._ck(self.lib.mnbab_serve_step(self.h, max_nodes, C.byref(a), C.byref(st)))
        out = {k: getattr(st, k) for k, _ in L.ServeStats._fields_ if k != "step"}
        out["step"] = {k: getattr(st.step, k) for k, _ in L.StepStats._fields_}
        return out

    def poll(self, ticket: int) -> bool:
        d = C.c_int32()
        self._ck(self.lib.mnbab_poll(self.h, ticket, C.byref(d)))
        return bool(d.value)

    def request_result(self, ticket: int):
        v, n = C.c_int32(), C.c_int32()
        w, t = C.c_double(), C.c_double()
        self._ck(self.lib.mnbab_request_result(self.h, ticket, C.byref(v), C.byref(w), C.byref(t),
                                               C.byref(n)))
        return dict(verdict=v.value, wait_s=w.value, total_s=t.value, nodes=n.value)


def mnc_group(oct_lb, max_rows: int = 4096):
    """Constraint rows (P [e, 3], Phat [e, 3], p [e]) of one group of three
    neurons from its 26 octahedral lower bounds (mnbab_mnc_group; host only)."""
    lib = L.load()
    ob = np.ascontiguousarray(np.asarray(oct_lb, np.float64).reshape(26))
    P = np.empty((max_rows, 3))
    Ph = np.empty((max_rows, 3))
    p = np.empty(max_rows)
    n = C.c_int32()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    st = lib.mnbab_mnc_group(dp(ob), max_rows, dp(P), dp(Ph), dp(p), C.byref(n))
    if st != 0:
        raise MnbabError(st, "mnbab_mnc_group failed")
    k = n.value
    return P[:k].copy(), Ph[:k].copy(), p[:k].copy()
