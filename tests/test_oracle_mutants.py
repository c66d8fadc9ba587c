"""Planted mistakes in the oracle must each fail at least one pin.

The oracle source carries compile-time hooks (RBD_ORACLE_MUTANT = k) that plant one plausible
mistake each; the default build has none.  This shows the pins are strong enough to catch a
dropped re-orthogonalisation sweep, a wrong sign, a wrong tie-break, an ignored start column,
a squared indicator, a missing normalisation, T taken from the unnormalised vector, a strict
comparison in step 2.4, a squared Frobenius test, an off-by-one Gram-Schmidt loop, and under a
diagonal A-norm the weights dropped from the indicator or from the step 2.2 test.
"""
import functools

import pytest

import pins

MUTANTS = {
    1: "single Gram-Schmidt sweep (no re-orthogonalisation)",
    2: "wrong sign of the projection coefficient",
    3: "argmax ties go to the highest index",
    4: "start column ignored",
    5: "indicator squared",
    6: "basis vector not normalised",
    7: "T row computed from the unnormalised vector",
    8: "step 2.4 uses a strict comparison",
    9: "Frobenius stop test on the squared norm",
    10: "Gram-Schmidt loop skips the last basis",
    14: "A-norm indicator takes the Euclidean norm (weights dropped)",
    15: "step 2.2 break test on the Euclidean norm under an A-norm",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS), ids=lambda k: f"mut{k}")
def test_mutant_is_caught(oracle_mod, mutant):
    oracle_mod.build(mutant)
    c = functools.partial(oracle_mod.compress, mutant=mutant)
    failed = []
    for pin in pins.FAST_PINS + [pins.pin_paper_rank_functions] + pins.W_PINS:
        try:
            pin(c)
        except (AssertionError, ValueError, IndexError, FloatingPointError) as e:
            failed.append((pin.__name__, str(e)[:80]))
    assert failed, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
