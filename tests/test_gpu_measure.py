"""The FP64 FMA rate probe (a measurement helper beside the FP64 roofline):
positive and below the derived nominal peak of 2 DFMA per clock per SM."""
import pytest

from gpu_util import ad, need_gpu

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible():
    need_gpu()
    r = ad().fp64_fma_rate(2, 1 << 14)
    assert 0.2 < r < 152 * 2 * 2 * 2.07e9 / 1e12 * 1.02, r
    with pytest.raises(ad().AdError):
        ad().fp64_fma_rate(0, 1 << 14)
