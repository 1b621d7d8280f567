"""The packed two-lane float-float arithmetic that the float-float step and adjoint use for two
velocity pairs at a time (B300's f32x2 add, sub and mul, scalar FMAs): every packed operation
reproduces, in each lane, the bits of its scalar form on seeded operands of both signs and
many binades (lbm_test_packed_ff)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [1, 2, 0xC0FFEE])
def test_packed_ops_equal_scalar_ops_bit_for_bit(seed):
    from paper_1405_1253_b300 import lbm
    assert lbm.test_packed_ff(1 << 18, seed) == 0


def test_packed_selftest_rejects_bad_arguments():
    from paper_1405_1253_b300 import lbm
    with pytest.raises(lbm.LBMError) as e:
        lbm.test_packed_ff(0, 1)
    assert e.value.code == lbm.LBM_EINVAL
