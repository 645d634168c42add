"""The device ALU rates that the ALU-bound rooflines divide by
(qpfrg_alu_rates): results per SM per clock within the range any recent part
gives (MUFU 8-128, FP32 FMA 32-256), the same on a second call to 5 %."""
import pytest

from paper_2005_00827_gb300 import api

pytestmark = pytest.mark.gpu


def test_alu_rates_are_plausible_and_repeatable():
    a = api.qpfrg_alu_rates()
    b = api.qpfrg_alu_rates()
    for k, lo, hi in (("ex2", 8, 128), ("rcp", 8, 128), ("ffma", 32, 256)):
        assert lo <= a[k] <= hi
        assert abs(a[k] - b[k]) <= 0.05 * a[k]
