"""The CPU oracle against what the paper and mathematics fix (no GPU).

Pins: hand-worked examples (tests/golden/hand_examples.txt), brute force
over every start position on tiny inputs, alternative characterisations of
the RAM and AE rules, closed forms (constant, ramp, spike, uniform-byte
statistics), invariants (tiling, size bounds, AE-Min/AE-Max mirror) and edit
locality. See tests/pins.py for the statements and their sources.
"""
import pytest

import pins


def test_hand_examples(orc):
    pins.check_hand_examples(orc)


def test_brute_force_every_start(orc):
    pins.check_brute_small(orc, trials=400)


def test_alternative_characterisations(orc):
    pins.check_alternative_forms(orc, trials=150)


def test_closed_forms(orc):
    pins.check_closed_forms(orc)


def test_uniform_statistics(orc):
    pins.check_uniform_statistics(orc)


def test_invariants(orc):
    pins.check_invariants(orc)


def test_edit_locality(orc):
    pins.check_edit_locality(orc)


def test_empty_input(orc):
    import numpy as np
    for alg in pins.ALGS:
        assert orc.chunk(alg, np.zeros(0, dtype=np.uint8), 4, 1, 10).size == 0
