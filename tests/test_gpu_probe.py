"""The FP64-pipe probe (lbm_probe_fp64_rate), the second roof that the bench states beside the
HBM roof of the FP64-storage kernels: a plausible rate for a B300 (its FP64 units run at about
1/64 of the FP32 rate: ~2 FMAs per SM per clock, ~0.6e12 per second on 148 SMs at 2 GHz),
the same rate for twice the work, and the argument checks."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_rate_is_plausible_and_stable():
    from paper_1405_1253_b300 import lbm
    r1 = lbm.probe_fp64_rate(1024)
    r2 = lbm.probe_fp64_rate(2048)
    print("FP64 FMA per second", r1, r2)
    for r in (r1, r2):
        assert 5e10 < r < 5e12
    assert abs(r1 - r2) / r2 < 0.2


@pytest.mark.parametrize("iters", [0, -1, (1 << 18) + 1])
def test_probe_rejects_bad_arguments(iters):
    from paper_1405_1253_b300 import lbm
    with pytest.raises(lbm.LBMError) as e:
        lbm.probe_fp64_rate(iters)
    assert e.value.code == lbm.LBM_EINVAL
