"""The pins reject plausible mistakes in the oracle.

Each case plants one known-wrong step in the oracle (a dropped term, a wrong
sign, index, order or operand; ``oracle.planted``) and runs the pins that
should see it: at least one of them must fail.  Together they show that the
pins in ``test_oracle_pins.py`` constrain every step the oracle takes, not
only its output on the cases it was written for.  CPU only.
"""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import mlp as om
from tests import test_oracle_mlp as mpins
from tests import test_oracle_pins as pins

# mistake -> the pins (function, arguments) expected to reject it
MUTANTS = {
    "prescale_off": [(pins.test_setup_matches_dense_lstsq, dict(dim=2, n=7, bs=1, kind="additive", nu=3)),
                     (pins.test_scale_invariance_of_setup, {})],
    "update_sign": [(pins.test_setup_matches_dense_lstsq, dict(dim=2, n=7, bs=1, kind="additive", nu=3))],
    "lambda_t": [(pins.test_setup_matches_dense_lstsq, dict(dim=2, n=6, bs=2, kind="additive", nu=2))],
    "smooth_t": [(pins.test_smoother_propagators, dict(kind="additive", bs=2))],
    "colour_order": [(pins.test_smoother_propagators, dict(kind="multiplicative", bs=1))],
    "reverse_order": [(pins.test_smoother_propagators, dict(kind="additive", bs=1))],
    "smooth_sign": [(pins.test_damped_jacobi_and_redblack_gs, {})],
    "interp_one_sided": [(pins.test_galerkin_matches_dense_rap, dict(dim=2, n=8)),
                         (pins.test_galerkin_poisson_stencil_closed_form, dict(dim=2))],
    "restrict_unscaled": [(pins.test_restriction_scale_invariance, {})],
    "coarse_chol": [(pins.test_coarse_solve_is_direct_nonsymmetric, dict(n=4))],
    "trunc_smallest": [(pins.test_truncation_matches_dense, {})],
    "minnorm_off": [(pins.test_setup_matches_dense_lstsq, dict(dim=2, n=7, bs=3, kind="additive", nu=2))],
    "overlap_sum": [(pins.test_overlapping_additive_cascade_matches_dense_definition, dict(singletons=0)),
                    (pins.test_overlapping_additive_cascade_matches_dense_definition, dict(singletons=3))],
    "stokes_q2": [(pins.test_stokes_prescaling_has_its_defining_properties, dict(q=2, mode="stokes2"))],
    "spd_no_upper": [(pins.test_spd_projection_is_bounded_by_block_jacobi, {})],
    "pcg_beta": [(pins.test_pcg_matches_a_plain_pcg_around_the_oracle_cycle, dict(blocks="points"))],
    "greedy_ascending": [(pins.test_csr_hierarchy_galerkin_and_greedy_colouring, {})],
    "sketch_stale": [(pins.test_sketched_setup_matches_dense_lstsq,
                      dict(kind="additive", bs=1, exact_first=False, s=6, prob="sym"))],
    "prescale_power": [(pins.test_scale_invariance_of_setup, {})],
    "overlap_smooth_sum": [(pins.test_overlapping_additive_cascade_matches_dense_definition, dict(singletons=0))],
    "galerkin_rscale": [(pins.test_csr_hierarchy_galerkin_and_greedy_colouring, {})],
    "parity": [(pins.test_setup_matches_dense_lstsq, dict(dim=2, n=7, bs=1, kind="multiplicative", nu=3))],
    "givens_sign": [(pins.test_gmres_residuals_are_minimal, dict(method="gmres"))],
    "right_update_v": [(pins.test_manufactured_convergence,
                        dict(dim=2, n=31, kind="additive", method="gmres_right")),
                       (pins.test_gmres_residuals_are_minimal, dict(method="gmres_right"))],
    "inplace_colour": [(pins.test_coarse_level_setup_matches_dense_lstsq,
                        dict(dim=2, n=14, bs=1, kind="multiplicative"))],
    "sketch_first_t": [(pins.test_sketched_setup_matches_dense_lstsq,
                        dict(kind="multiplicative", bs=2, exact_first=True, s=16, prob="nonsym"))],
    "boundary_wrap": [(pins.test_couplings_to_boundary_nodes_are_ignored, {}),
                      (pins.test_galerkin_matches_dense_rap, dict(dim=2, n=8))],
    "prolong_sign": [(pins.test_manufactured_convergence, dict(dim=2, n=31, kind="additive", method="stationary"))],
    "rf_forward": [(pins.test_vcycle_symmetry_rf, dict(kind="additive"))],
    "stokes_vel_l1": [(pins.test_stokes_prescaling_has_its_defining_properties, dict(q=1, mode="stokes1"))],
    "sketch_z_once": [(pins.test_sketched_setup_matches_dense_lstsq,
                       dict(kind="multiplicative", bs=1, exact_first=False, s=5, prob="sym"))],
    "spd_unweighted": [(pins.test_spd_projection_is_bounded_by_block_jacobi, {})],
}


def test_every_planted_mistake_has_a_case():
    """The binding's names follow the C enum of planted mistakes one to one."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "cs_oracle.c")).read()
    body = re.search(r"enum \{\s*PL_NONE = 0,(.*?)\};", src, re.S).group(1)
    ids = [m.lower() for m in re.findall(r"PL_(\w+),", body)]
    assert tuple(ids) == oracle.PLANTS
    assert set(MUTANTS) == set(oracle.PLANTS)


@pytest.mark.parametrize("mistake", list(MUTANTS))
def test_pins_reject_the_planted_mistake(mistake):
    failed = []
    with oracle.planted(mistake):
        for fn, kw in MUTANTS[mistake]:
            try:
                with np.errstate(all="ignore"):
                    fn(**kw)
            except (AssertionError, np.linalg.LinAlgError, ValueError, RuntimeError):
                failed.append(fn.__name__)
    assert failed, f"no pin rejects the planted mistake '{mistake}'"
    # and without the mistake the same pins pass
    for fn, kw in MUTANTS[mistake]:
        fn(**kw)


# the network's oracle (oracle/mlp.py): mistake -> the pins expected to reject it
MLP_MUTANTS = {
    "weights_unrounded": [(mpins.test_forward_rounds_the_weights_to_bf16, {})],
    "loss_sum": [(mpins.test_loss_is_the_mean_squared_error, {})],
    "relu_grad_open": [(mpins.test_backprop_matches_finite_differences, {})],
    "window_mirror": [(mpins.test_features_are_the_prescaled_rows_over_every_window, dict(n=10, bs=3))],
    "target_unscaled": [(mpins.test_targets_are_the_prescaled_blocks_of_every_block, dict(n=10, bs=3))],
}


def test_every_planted_network_mistake_has_a_case():
    assert set(MLP_MUTANTS) == set(om.PLANTS)


@pytest.mark.parametrize("mistake", list(MLP_MUTANTS))
def test_network_pins_reject_the_planted_mistake(mistake):
    failed = []
    with om.planted(mistake):
        for fn, kw in MLP_MUTANTS[mistake]:
            try:
                fn(**kw)
            except AssertionError:
                failed.append(fn.__name__)
    assert failed, f"no pin rejects the planted network mistake '{mistake}'"
    for fn, kw in MLP_MUTANTS[mistake]:
        fn(**kw)
