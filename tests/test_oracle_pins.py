"""The oracle against its pins (no GPU): closed forms, invariants, library routines,
brute force and equivalent evaluations, each check citing the passage it pins."""
import pytest

import oracle
from tests import oracle_checks as C

L, CO = oracle.LANDAU, oracle.COULOMB
F1, EX = oracle.OR_FIRST_ORDER, oracle.OR_EXACT

CASES = [
    (C.check_unit_field_closed_form, (L,)),
    (C.check_unit_field_closed_form, (CO,)),
    (C.check_constant_diagonal_field_closed_form, ()),
    *[(C.check_single_link_excitation_closed_form, (nu,)) for nu in range(4)],
    (C.check_delta_properties_and_two_theta_evaluations, ()),
    (C.check_gradient_identity, (L,)),
    (C.check_gradient_identity, (CO,)),
    (C.check_global_rotation_invariance, ()),
    (C.check_su2_maximiser_matches_brute_force_on_2x4_lattice, ()),
    (C.check_su2_maximiser_value_and_degenerate_case, ()),
    (C.check_overrelaxation_exact_form_is_matrix_power, ()),
    (C.check_overrelaxation_first_order_form, ()),
    *[(C.check_relaxation_omega1_never_decreases_F, (f, g)) for f in (F1, EX) for g in (L, CO)],
    (C.check_sweeps_are_gauge_transformations, (L,)),
    (C.check_sweeps_are_gauge_transformations, (CO,)),
    (C.check_half_sweep_touches_only_its_parity, ()),
    (C.check_subgroup_fixed_point_after_site_update, (L,)),
    (C.check_subgroup_fixed_point_after_site_update, (CO,)),
    (C.check_updated_site_delta_from_GK, (L,)),
    (C.check_updated_site_delta_from_GK, (CO,)),
    (C.check_even_translation_covariance_is_exact, ()),
    (C.check_reunit_is_gram_schmidt_projection, ()),
    (C.check_fix_stop_rule_and_bookkeeping, ()),
    *[(C.check_pure_gauge_reaches_unit_field, (s,)) for s in (21, 22, 23)],
    (C.check_smooth_field_recovered_functional, ()),
    (C.check_coulomb_slices_fix_independently, ()),
    (C.check_coulomb_per_slice_masks_freeze_converged_slices, ()),
    (C.check_fasd_filter_inverts_laplacian, (L,)),
    (C.check_fasd_filter_inverts_laplacian, (CO,)),
    (C.check_fasd_unit_filter_is_naive_descent, (L,)),
    (C.check_fasd_unit_filter_is_naive_descent, (CO,)),
    (C.check_fasd_ascends_and_is_gauge_transformation, (L,)),
    (C.check_fasd_ascends_and_is_gauge_transformation, (CO,)),
    (C.check_fasd_coulomb_slices_independent, ()),
    (C.check_fasd_converges_faster_than_or, ()),
]


@pytest.mark.parametrize("check,args", CASES, ids=[f"{c.__name__[6:]}{list(a)}" for c, a in CASES])
def test_oracle_pin(check, args):
    check(oracle, *args)
