"""The FP64 rate probe (qsim_fp64_rate) returns a plausible rate: above the
rate of one SM and below the nominal 1.25 TFLOP/s of the part (0.625e12
FMA/s) with some margin for a faster clock."""
import pytest

from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def test_fp64_rate_is_plausible():
    r = qsim.fp64_rate(0)
    assert 1e10 < r < 1.0e12
    with pytest.raises(qsim.QsimError):
        qsim.fp64_rate(1 << 20)                   # no such device
