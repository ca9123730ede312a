"""The pins are sensitive: each planted mistake in a copy of the oracle (built
on the CPU with -DORACLE_MUTANT=k) fails at least one pin of
test_oracle_pins.py or test_oracle_q.py.  Mutants:
1 derivative from the wrong orbit index,
2 wrong sign in Re(z^2),
3 s_{l,n} built with p_l instead of p_{l-1},
4 level line walked the wrong way,
5 missing conjugate fold,
6 q_{l,n} built with p_{l-1} instead of p_l (its level line and values),
7 q_{l,n} as the union of its factors with the product of eq. polySimple
  taken from s_{1,n} = p_n as well (p_n three times),
8 the real-root rule |Im| < eps/2 -> Im = 0 missing,
9 the exact period taken as the largest vanishing divisor, not the smallest,
10 no finishing steps to the working precision,
11 q_{l,n} as the union with p_n counted once (q_{0,n} without s_{1,n}),
12 s_{l,n} types with Mis(l,k) tested before Hyp(k)."""
from __future__ import annotations

import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_q as qpins

# (mutant, pin function, its arguments)
CASES = [
    (1, pins.test_orbit_at_minus_two, (5,)),
    (2, pins.test_period3_cardano, ()),
    (2, pins.test_orbit_off_axis_against_integer_polynomial, ()),
    (3, pins.test_tiny_misiurewicz, ()),
    (3, pins.test_s_2_4_example, ()),
    (3, pins.test_level_line_iso_angle_zero_misiurewicz, (2, 3)),
    (4, pins.test_level_line_iso_angle_zero, (4,)),
    (5, pins.test_counts_and_exact_periods, (8,)),
    (6, qpins.test_level_line_iso_angle_zero_q, (2, 2)),
    (6, qpins.test_q_roots_are_roots_of_q, ()),
    (7, qpins.test_types_and_multiplicities_follow_thm_fact_mis, (4, 2)),
    (7, qpins.test_worked_factorisation_q_2_4, ()),
    (7, qpins.test_q_1_n_is_p_n_squared, (5,)),
    (8, pins.test_counts_and_exact_periods, (6,)),
    (8, pins.test_real_root_count_sturm, (6,)),
    (9, pins.test_counts_and_exact_periods, (6,)),
    (9, pins.test_hyp_1_and_2, ()),
    (10, pins.test_counts_and_exact_periods, (8,)),
    (10, pins.test_vieta_power_sums, (8,)),
    (11, qpins.test_types_and_multiplicities_follow_thm_fact_mis, (3, 4)),
    (11, qpins.test_worked_factorisation_q_2_4, ()),
    (11, qpins.test_library_roots_of_exact_coefficients, (2, 2)),
    (12, pins.test_s_2_4_example, ()),
    (12, pins.test_tiny_misiurewicz, ()),
]


@pytest.mark.parametrize("k,pin,args", CASES, ids=[f"mutant{k}-{p.__name__}" for k, p, _ in CASES])
def test_pin_catches_planted_mistake(tmp_path, k, pin, args):
    path = oracle.build_mutant(k, str(tmp_path))
    with oracle.use_library(path):
        with pytest.raises(Exception):
            pin(*args)
    pin(*args)  # and the real oracle still passes
