"""The engine's integer FP64 routines (row reciprocal of the Hines elimination,
float-to-double widening of the mixed path's synaptic sums) against the GPU's
own IEEE operations, bit for bit, through pa_check_arith."""
import pytest

from paper_2411_16445_b300 import engine as E


@pytest.mark.gpu
def test_integer_reciprocal_and_widening_match_ieee():
    r = E.check_arith(device=0, seed=20241125, n_random=1 << 31)
    # 2^23 x 8 seed-sweep inputs + the random ones + all 2^32 floats
    assert r["checked"] == (1 << 26) + (1 << 31) + (1 << 32)
    assert r["rcp_mismatch"] == 0, hex(r["first_bad_rcp_bits"])
    assert r["widen_mismatch"] == 0
