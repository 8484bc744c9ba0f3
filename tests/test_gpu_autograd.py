"""The adjoint kernels behind torch.autograd (paper_2205_00263_gb300.autograd).

The gradient that NodeBound's backward returns is checked two ways:

* against central differences of the library's own bound
  (mnbab_bound_batch at parameters theta +- h e_k, differenced in FP64 on the
  host).  The bound is piecewise linear in every parameter (Sec. 3.1: the
  back-substitution is linear in alpha, beta, gamma for fixed D cases), so a
  coordinate is used only where the differences at h and h / 2 agree, i.e. no
  D-case switch lies within +-h;
* against the FP64 oracle's reverse-mode gradient (core.bound_and_grad).
"""
import numpy as np
import pytest
import torch

from helpers import TOL, concat, conv_case, fc_case, gpu_property, random_node, to_params
from oracle import core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    return Context


@pytest.mark.parametrize("case", ["fc_mnc", "conv"])
def test_node_bound_gradient_fd_and_oracle(Context, case):
    from paper_2205_00263_gb300.autograd import NodeBound
    if case == "fc_mnc":
        layers, C, d, lo, hi, prep = fc_case(16, (37, 53, 29, 7), 0.12, with_mnc=True)
    else:
        layers, C, d, lo, hi, prep = conv_case(17, 0.06)
    net, lo_t, hi_t, l, u, S, m, dense = prep
    E = sum(v.idx.shape[0] for v in m.values()) if m else 0
    SD = sum(l[i].numel() for i in l)
    rng = np.random.default_rng(16)
    dev = torch.device("cuda", 0)
    with Context(node_capacity=128, max_mnc_rows=max(E, 1)) as ctx:
        gnet, prop = gpu_property(ctx, layers, lo, hi, C, d, m)
        onodes, gids = [], []
        for k in range(4):
            on = random_node(prep, rng, n_splits=2 + k % 2, row=k % C.shape[0])
            on.split_layer = net.R          # bounds as given: nothing to re-bound
            gid = ctx.node_root(prop, on.row)
            ctx.import_params(gid, to_params(on, net.R))
            onodes.append(on)
            gids.append(gid)
        alpha = torch.tensor(np.stack([concat(o.alpha, net.R) for o in onodes]), dtype=torch.float32,
                             device=dev, requires_grad=True)
        beta = torch.tensor(np.stack([concat(o.beta, net.R) for o in onodes]), dtype=torch.float32,
                            device=dev, requires_grad=True)
        gam = np.stack([np.concatenate([o.gamma[i].numpy() for i in sorted(o.gamma)
                                        if o.gamma[i].numel()] or [np.zeros(0)]) for o in onodes])
        gamma = torch.tensor(gam, dtype=torch.float32, device=dev, requires_grad=True)
        lb = NodeBound.apply(alpha, beta, gamma, ctx, gids)
        assert lb.device == dev and lb.shape == (len(gids),)
        (lb * torch.arange(1, len(gids) + 1, device=dev)).sum().backward()
        G = torch.cat([alpha.grad, beta.grad, gamma.grad], dim=1).cpu().numpy().astype(np.float64)
        theta = torch.cat([alpha, beta, gamma], dim=1).detach().cpu().numpy()

        # 1. the FP64 oracle's gradient at the same parameters (weights 1..n)
        for k, on in enumerate(onodes):
            ref, _, oa, ob, og = core.bound_and_grad(net, on, on.alpha, on.beta, on.gamma, dense,
                                                     lo_t, hi_t)
            assert abs(float(lb[k].detach()) - float(ref)) <= TOL * (1 + abs(float(ref)))
            o = np.concatenate([concat(oa, net.R), concat(ob, net.R)]
                               + ([np.concatenate([og[i].numpy() for i in sorted(og)
                                                   if og[i].numel()])] if E else []))
            assert np.abs(G[k] / (k + 1) - o).max() <= 1e-4 * (1 + np.abs(o).max())

        # 2. central differences of mnbab_bound_batch, away from case switches
        def bound_at(th):
            ctx.set_params(gids, th)
            return ctx.bound_batch(gids, with_ub=False).astype(np.float64)

        h = 2e-2
        used = 0
        lb0 = lb.detach().cpu().numpy()
        for k in range(len(gids)):
            # FP32 bounds resolve differences down to their spacing: use
            # coordinates whose bound change over +-h spans >= 2000 spacings
            ulp = float(np.spacing(np.float32(abs(lb0[k]) + 1.0)))
            cand = np.nonzero(np.abs(G[k]) / (k + 1) * h >= 2000 * ulp)[0]
            for j in rng.choice(cand, size=min(12, cand.size), replace=False):
                diffs = []
                for hh in (h, h / 2):
                    tp, tm = theta.copy(), theta.copy()
                    tp[k, j] += hh
                    tm[k, j] -= hh
                    diffs.append((bound_at(tp)[k] - bound_at(tm)[k]) / (2 * hh))
                if abs(diffs[0] - diffs[1]) > 1e-3 * (1 + abs(diffs[1])):
                    continue    # a D-case switch within +-h: not a linear piece
                g = G[k, j] / (k + 1)
                assert abs(diffs[1] - g) <= 2e-3 * (1 + abs(g)), (k, j, diffs, g)
                used += 1
        assert used >= 12
        # the nodes keep the parameters last set
        ctx.set_params(gids, theta)
        lb2 = ctx.bound_batch(gids, with_ub=False)
        assert np.allclose(lb2, lb.detach().cpu().numpy(), rtol=0, atol=1e-6)
