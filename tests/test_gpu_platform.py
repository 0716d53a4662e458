"""Runs with the GPU suite, i.e. on the machine that measures: the seeded
generators give the same inputs there as where the CPU suite runs."""
import pytest

import test_graphgen


@pytest.mark.gpu
def test_generator_outputs_are_stable_here():
    test_graphgen.test_generator_outputs_are_stable()
