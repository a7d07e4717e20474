"""The mixed form's FP32 <-> FP64 conversions (integer-pipe widening of the
FP32 increments and round-to-nearest-even narrowing of the FP64 registers)
against the GPU's own conversion instructions, bit for bit."""
import pytest

import paper_2408_16509_gb300 as fr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2])
def test_conversions_match_hardware(seed):
    fr.build()
    assert fr.check_conversions(1 << 24, seed=seed) == 0
