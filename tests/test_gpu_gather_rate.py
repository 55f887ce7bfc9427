"""The gather-rate measurement behind the kernels' roofline: it runs, gives
a plausible rate for independent and dependent gathers, and checks its
arguments."""
import pytest

from paper_1505_04086_gb300 import gc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dependent", [False, True])
def test_gather_rate_is_plausible(dependent):
    rc, rate = gc.gc_measure_gather_rate(0, 8 << 20, 2, dependent)
    assert rc == gc.GC_OK, gc.gc_strerror(rc)
    # an L2-resident array: between 10 and 5000 G loads/s on any sm_103a GPU
    assert 10.0 < rate < 5000.0, rate


def test_gather_rate_odd_sizes_round_down():
    rc, rate = gc.gc_measure_gather_rate(0, (8 << 20) + 12345, 1, True)
    assert rc == gc.GC_OK and rate > 0.0
    rc, rate = gc.gc_measure_gather_rate(0, 4096, 1, False)
    assert rc == gc.GC_OK and rate > 0.0
