"""Planted mistakes in the oracle fail its pins.

The oracle is the reference the GPU path is compared with, so it is trusted
only as far as its pins would catch a plausible mistake in it.  Each case
below plants one such mistake (a dropped term, a wrong sign, a swapped operand
or index, a missing projection) by editing the source text of one oracle
function in memory for the duration of the test, and runs the pins that target
that function: at least one of them must fail (an assertion, or an error the
mistake provokes).  The edit is checked to apply exactly once, so a case
cannot silently stop planting anything when the oracle changes.  Everything here runs on the CPU; nothing
calls the GPU library.
"""
import __future__
import inspect
import sys
import textwrap

import pytest

from oracle import attack, bab, core, exact, mnc

import test_attack_pins as apins
import test_oracle_intermediate as ipins
import test_oracle_pins as pins


def _mutant(owner, name, old, new):
    """The function `owner.name` recompiled from its source with `old`
    replaced by `new` (exactly one occurrence), in its module's namespace."""
    fn = inspect.getattr_static(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, f"{name}: the edit must apply exactly once: {old!r}"
    ns = dict(vars(sys.modules[fn.__module__]))
    code = compile(src.replace(old, new), f"<planted mistake in {name}>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    exec(code, ns)
    return ns[name]


# pins, by what they target
CONV_ADJOINT = (pins.test_conv_forward_and_adjoint, (16, 13, 32, 4, 2, 0))
AFFINE_EXACT = (pins.test_affine_only_is_exact_and_hoelder, ())
RELU_POS = (pins.test_relu_table_positive_coefficient, ())
RELU_NEG = (pins.test_relu_table_negative_coefficient, ())
RELU_SPLITS = (pins.test_relu_table_two_neurons_and_splits, ())
ADAM_POS = (pins.test_standard_adam_closed_form, (1,))
ADAM_NEG = (pins.test_standard_adam_closed_form, (-1,))
SOUND = (pins.test_soundness_random_parameters, (0,))
SOUND_1 = (pins.test_soundness_random_parameters, (1,))
BELOW_EXACT = (pins.test_lower_bounds_below_exact_minimum, (3,))
BELOW_EXACT_4 = (pins.test_lower_bounds_below_exact_minimum, (4,))
REBOUND_EXACT = (pins.test_rebound_after_split_is_exact_on_single_neurons, ())
ADAM_BEST = (pins.test_adam_returns_the_best_iterate, ())
MNC_TERMS = (pins.test_multi_neuron_terms_by_hand, ())
FOLD = (pins.test_folded_property_is_the_margin, ())
BAB_ROOT = (pins.test_bab_root_verdict_uses_the_optimised_bound, ())
LEAF_LP = (pins.test_fully_split_leaf_reaches_lp_optimum, (5,))
COMPLETE = (pins.test_unlimited_bab_with_exact_leaves_is_complete, (2, 0.30906))
UNDECIDED_LEAF = (pins.test_bab_without_leaf_completion_never_verifies_an_undecided_leaf, ())
INTER_GAMMA = (ipins.test_gamma_sets_sound_and_zero_steps_give_deeppoly, (7,))
INTER_GAMMA_FD = (ipins.test_gamma_gradient_matches_finite_differences, (1,))
INTER_LOOSER = (ipins.test_optimised_bounds_sound_and_never_looser, (1, 0))
INTER_BEST = (ipins.test_each_row_keeps_its_best_iterate, ())
MNC_SOUND = (pins.test_mnc_rows_are_sound_per_orthant, ())
ACS = (pins.test_acs_scores_by_hand, ())
CEX = (pins.test_counterexamples_are_real, ())
CHILDREN = (pins.test_children_keep_earlier_bounds, ())
CAB = (pins.test_cab_costs_by_hand, ())
RES_FWD = (pins.test_resnet_forward_matches_definition, ())
RES_EXACT = (pins.test_resnet_bound_is_exact_when_linear, ())
INTER_SOUND = (ipins.test_optimised_bounds_sound_and_never_looser, (0, 0))
INTER_CORNER = (ipins.test_linear_set_objective_reaches_its_corner, ())
INTER_ZERO = (ipins.test_zero_steps_reproduce_deeppoly_root_bounds, (5,))
ATTACK_MIN = (apins.test_affine_region_reaches_the_closed_form_minimum, ())
SPLITMIX = (apins.test_splitmix_starts_follow_the_published_generator, ())

# (case, owner, function, text, planted text, pins)
CASES = [
    # affine layers (Sec. 3.1: the affine step of a back-substitution)
    ("conv_backsub_flipped_kernel", core.Affine, "backsub",
     "self.W, None, stride=self.stride,", "self.W.flip(2, 3), None, stride=self.stride,",
     [CONV_ADJOINT]),
    ("conv_bias_wrong_axis", core.Affine, "bias_dot",
     "A.reshape(A.shape[0], co, ho * wo).sum(-1)", "A.reshape(A.shape[0], ho * wo, co).sum(1)",
     [CONV_ADJOINT]),
    ("fc_forward_without_bias", core.Affine, "forward",
     "return x @ self.W.T + self.b", "return x @ self.W.T", [AFFINE_EXACT, RES_FWD]),
    ("bias_term_dropped", core, "backsub_rows",
     "c = c + A.bias_dot(Ahat)", "c = c + 0.0 * A.bias_dot(Ahat)", [AFFINE_EXACT]),
    ("residual_edges_overwrite", core, "backsub_rows",
     "lam[s] = lam[s] + A.backsub(Ahat) if s in lam else A.backsub(Ahat)",
     "lam[s] = A.backsub(Ahat)", [RES_EXACT]),
    ("forward_without_relu", core.Net, "forward",
     "torch.clamp(h, min=0.0) if t <= self.R else h", "h", [RES_FWD]),
    # concretisation (Sec. 3.1, minimum over the input box)
    ("concretize_lo_hi_swapped", core, "concretize",
     "torch.where(A0 >= 0, lo, hi)", "torch.where(A0 >= 0, hi, lo)", [AFFINE_EXACT]),
    # ReLU relaxation and split handling (Sec. 3.1)
    ("deeppoly_slope_reversed", core, "deeppoly_alpha", "(u >= -l)", "(u <= -l)", [RELU_POS]),
    ("inactive_taken_as_unstable", core, "relu_cases",
     "zero = neg_split | (~pos_split & ~(l >= 0) & (u <= 0))", "zero = neg_split",
     [SOUND, SOUND_1]),
    ("upper_intercept_dropped", core, "relu_backsub",
     "dc = (ap * blow).sum(-1)", "dc = 0.0 * (ap * blow).sum(-1)", [RELU_NEG]),
    ("upper_slope_uses_l", core, "relu_backsub",
     "torch.where(unst, u / den, torch.zeros_like(u))",
     "torch.where(unst, -l / den, torch.zeros_like(u))", [RELU_NEG]),
    ("lower_upper_case_reversed", core, "relu_backsub",
     "neg = unst & (ap < 0)", "neg = unst & (ap > 0)", [RELU_POS, RELU_NEG]),
    ("beta_term_wrong_sign", core, "relu_backsub",
     "ahat = ap * D + beta * S.to(DT)", "ahat = ap * D - beta * S.to(DT)", [RELU_SPLITS]),
    ("gamma_P_dropped", core, "relu_backsub",
     "ap = a if GP is None else a + GP", "ap = a", [MNC_TERMS]),
    ("gamma_Phat_dropped", core, "relu_backsub",
     "ahat = ahat + GPh", "ahat = ahat + 0.0 * GPh", [MNC_TERMS]),
    ("gamma_p_wrong_sign", core, "relu_backsub",
     "dc = dc - gp0", "dc = dc + gp0", [MNC_TERMS]),
    # intermediate bounds (Sec. 3.1 root bounds, Sec. 3.2 re-bounding after a split)
    ("root_upper_bound_not_negated", core, "root_bounds",
     "up.append(-lb[n:])", "up.append(lb[n:])", [SOUND]),
    ("rebound_upper_not_negated", core, "rebound_node",
     "u[idx] = torch.minimum(u[idx], -lb[n:])", "u[idx] = torch.minimum(u[idx], lb[n:])",
     [REBOUND_EXACT]),
    ("rebound_skips_next_layer", core, "rebound_node",
     "range(node.split_layer + 1, R + 1)", "range(node.split_layer + 2, R + 1)",
     [REBOUND_EXACT]),
    ("split_bound_not_applied", bab, "children",
     "u[layer][j] = min(float(u[layer][j]), 0.0)", "u[layer][j] = float(u[layer][j])",
     [CHILDREN]),
    # projected Adam (Sec. 3.1, projected gradient ascent)
    ("adam_no_bias_correction", core, "optimize",
     "mh = m / (1 - hp.b1 ** t)", "mh = m", [ADAM_POS]),
    ("adam_descends", core, "optimize",
     "P[i] = P[i] + lr[grp] * mh", "P[i] = P[i] - lr[grp] * mh", [ADAM_POS, RELU_POS]),
    ("beta_not_projected", core, "optimize",
     "P[i] = torch.clamp(P[i], min=0.0)", "P[i] = P[i]", [ADAM_NEG]),
    ("alpha_beta_gradients_swapped", core, "optimize",
     '(("a", alpha, ga), ("b", beta, gb)', '(("a", alpha, gb), ("b", beta, ga)',
     [ADAM_POS, RELU_POS]),
    ("last_iterate_not_best", core, "optimize",
     "if float(lb) > best:", "if True:", [ADAM_BEST]),
    # optimised intermediate bounds (Sec. 3.1, parameter sets per layer)
    ("inter_upper_not_negated", core, "optimize_intermediate",
     "u[idx] = torch.minimum(u[idx], -best[-1])", "u[idx] = torch.minimum(u[idx], best[-1])",
     [INTER_SOUND]),
    ("inter_sets_start_at_one", core, "optimize_intermediate",
     "alpha = {i: deeppoly_alpha(node.l[i], node.u[i]) for i in range(1, t)}",
     "alpha = {i: torch.ones_like(node.l[i]) for i in range(1, t)}", [INTER_ZERO]),
    ("inter_descends", core, "optimize_intermediate",
     "P[i] = P[i] + lr[grp] * mh", "P[i] = P[i] - lr[grp] * mh", [INTER_CORNER]),
    ("inter_last_iterate_kept", core, "optimize_intermediate",
     "bs = torch.maximum(bs, lb)", "bs = lb", [INTER_BEST]),
    ("inter_gamma_dropped", core, "intermediate_objective",
     "GP, GPh, gp0 = gamma[i] @ Pd, gamma[i] @ Phd, gamma[i] @ pv",
     "GP, GPh, gp0 = None, None, None", [INTER_GAMMA, INTER_GAMMA_FD]),
    ("undecided_leaf_closes_the_property", bab, "verify",
     "if not q and not unknown_leaf:", "if not q:", [UNDECIDED_LEAF]),
    ("inter_side_ignored", core, "intermediate_objective",
     "= float(side)", "= 1.0", [INTER_SOUND]),
    # multi-neuron constraints (Sec. 2.3, Sec. 3.1)
    ("mnc_offset_not_the_support", mnc, "group_constraints",
     "p = float((pts @ nvec).max())", "p = float((pts @ nvec).mean())", [MNC_SOUND]),
    ("mnc_relu_not_applied", mnc, "group_constraints",
     "Y = np.maximum(Y, 0.0)", "Y = V", [MNC_SOUND]),
    # branching (Sec. 3.2, App. B)
    ("acs_abs_dropped", core, "acs_scores",
     "s = torch.abs(gamma[i] @ Pd) + torch.abs(gamma[i] @ Phd)",
     "s = (gamma[i] @ Pd) + (gamma[i] @ Phd)", [ACS]),
    ("acs_fallback_intercept_wrong", core, "acs_scores",
     "icpt = torch.where(cand, -l * u / den, torch.zeros_like(u))",
     "icpt = torch.where(cand, u / den, torch.zeros_like(u))", [ACS]),
    ("tie_goes_to_highest_index", core, "pick_split",
     "return i, int(hit[0]), mx", "return i, int(hit[-1]), mx", [ACS]),
    ("tie_band_dropped", core, "pick_split",
     "thr = mx - ACS_TIE * abs(mx)", "thr = mx", [ACS]),
    ("cab_recompute_factor_dropped", core, "cab_costs",
     "2.0 * net.width(t) * C[t]", "net.width(t) * C[t]", [CAB]),
    ("cab_conv_cost_as_weights", core, "cab_costs",
     "A.d_out * A.W.shape[2] * A.W.shape[3]", "A.W.numel()", [CAB]),
    ("octahedron_direction_negated", mnc, "octahedron_bounds",
     "E[gi * len(DIRS) + di, G[k]] += dv[k]", "E[gi * len(DIRS) + di, G[k]] -= dv[k]",
     [MNC_SOUND]),
    # the BaB step (Sec. 3.2, Sec. 3.3)
    ("optimised_bound_ignored", bab, "bound_node",
     "if best > lb_dp:", "if False:", [BAB_ROOT]),
    ("counterexample_checked_on_row_0", bab, "bound_node",
     "[0, node.row])", "[0, 0])", [CEX]),
    ("exact_minimum_active_sign_flipped", exact, "exact_min",
     "A_ub.append(-Z[j]); b_ub.append(zc[j])", "A_ub.append(Z[j]); b_ub.append(-zc[j])",
     [BELOW_EXACT, BELOW_EXACT_4, LEAF_LP, COMPLETE]),
    # the property and counterexamples (Sec. 2.1, Sec. 4)
    ("property_offset_dropped", core, "fold_property",
     "Ct @ last.b + dt", "dt", [FOLD]),
    ("attack_ascends", attack, "pgd_row",
     "x - alpha * np.sign(g)", "x + alpha * np.sign(g)", [ATTACK_MIN]),
    ("splitmix_shift_changed", attack, "splitmix64",
     "(z ^ (z >> 27))", "(z ^ (z >> 28))", [SPLITMIX]),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    cid, owner, name, old, new, checks = case
    monkeypatch.setattr(owner, name, _mutant(owner, name, old, new))
    for fn, args in checks:
        try:
            fn(*args)
        except Exception:  # an assertion, or an error the mistake provokes
            return
    pytest.fail(f"no pin caught the planted mistake {cid} in {name}")


def test_unplanted_sources_recompile_to_the_same_results(monkeypatch):
    """The recompiling itself changes nothing: a no-op edit of every planted
    function leaves the pins green."""
    seen = set()
    for cid, owner, name, old, new, checks in CASES:
        if (owner, name) in seen:
            continue
        seen.add((owner, name))
        monkeypatch.setattr(owner, name, _mutant(owner, name, old, old))
    for fn, args in (AFFINE_EXACT, RELU_SPLITS, ADAM_POS, ACS, CAB, RES_EXACT, CHILDREN):
        fn(*args)
