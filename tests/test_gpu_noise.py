"""GPU noise against the oracle: Philox words bit-exact, Box-Muller to FP32 accuracy."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_common import np_

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (64, 32), (16, 8, 32), (256, 256), (8, 4096)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("seed,field", [(0, 0), (0xDEADBEEF12345678, 7), (12345, 63)])
def test_noise_bits_exact(hf, shape, seed, field):
    plan = hf.Plan(shape)
    N = int(np.prod(shape))
    bits = torch.empty(N, dtype=torch.int32, device="cuda")
    z = torch.empty(N, dtype=torch.float32, device="cuda")
    hf.hufield_noise(plan, seed, field, bits=bits, z=z)
    torch.cuda.synchronize()
    got = np_(bits).view(np.uint32).reshape(shape)
    np.testing.assert_array_equal(got, oracle.noise_bits(shape, seed, field))
    want = oracle.noise(shape, seed, field)
    err = np.abs(np_(z).reshape(shape).astype(np.float64) - want)
    # FP32 Box-Muller: a few ulp of the radius and < 1e-7 rad of angle
    assert err.max() < 2e-6 * max(1.0, np.abs(want).max())
    assert np.sqrt(np.mean(err * err)) < 2e-7


def test_noise_single_output(hf):
    plan = hf.Plan((32, 32))
    z = torch.empty(1024, dtype=torch.float32, device="cuda")
    hf.hufield_noise(plan, 5, 1, z=z)
    torch.cuda.synchronize()
    np.testing.assert_allclose(np_(z), oracle.noise((1024,), 5, 1), atol=2e-6)
