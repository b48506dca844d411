"""The int32 issue-rate measurement that backs the roofline (trioseq_alu_rate), through the C ABI."""
import pytest

from paper_2605_28400_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_alu_rates_are_plausible():
    for op, name in enumerate(B.ALU_FORMS):
        rate, mhz = B.trioseq_alu_rate(op)
        # thread-level instructions per SM per clock: forms with a maximum run on the ALU pipe
        # alone (at most its 128 lanes); adds may also issue on the FMA pipe
        bound = 130.0 if name in ("max", "add_max", "max3") else 260.0
        assert 16.0 < rate <= bound, (name, rate)
        assert 300.0 < mhz < 3000.0, (name, mhz)
    with pytest.raises(B.TrioseqError):
        B.trioseq_alu_rate(5)
