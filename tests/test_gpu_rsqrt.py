"""The FP64 reciprocal square root of the pivot-block Cholesky (an FP32
estimate refined by one second-order Newton step) against CUDA's correctly
rounded 1.0 / sqrt(x), on the GPU through the C ABI (bipm_check_rsqrt)."""

import pytest

pytestmark = pytest.mark.gpu


def test_reciprocal_square_root_within_two_ulp_of_cuda():
    import torch

    assert torch.cuda.is_available()
    from paper_2606_26341_gb300 import bipm

    # log-spaced over [1e-40, 1e40]: inside the refined range and both fallbacks
    worst = bipm.check_rsqrt(1 << 20)
    assert worst <= 2.0, worst


def test_reciprocal_square_root_check_rejects_bad_arguments():
    from paper_2606_26341_gb300 import bipm

    with pytest.raises(bipm.BipmError) as e:
        bipm.check_rsqrt(0)
    assert e.value.code == bipm.EINVAL
