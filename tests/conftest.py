import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def hf():
    """The CUDA library's binding, built in-tree if needed (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    from paper_2509_08675_gb300 import builder

    builder.build()
    from paper_2509_08675_gb300 import hufield

    return hufield


CANARY = 4096  # guard bytes on each side of every workspace a GPU test takes from Plan.workspace
CANARY_LO, CANARY_HI = 0xA5, 0x5A


@pytest.fixture(autouse=True)
def workspace_canaries(request):
    """In GPU tests, every workspace from Plan.workspace sits between two guard
    bands of known bytes, checked after the test: a kernel or a layout that
    writes past either end of its workspace fails the test that made it (the
    stand-in for a memory checker, which this pool does not offer)."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    hf_mod = request.getfixturevalue("hf")
    import torch

    orig = hf_mod.Plan.workspace
    guards = []

    def guarded(self, *args, **kwargs):
        ws = orig(self, *args, **kwargs)
        n = ws.numel()
        buf = torch.empty(n + 2 * CANARY, dtype=torch.uint8, device=ws.device)
        buf[:CANARY].fill_(CANARY_LO)
        buf[CANARY + n:].fill_(CANARY_HI)
        del ws
        guards.append((buf, n))
        return buf[CANARY:CANARY + n]

    hf_mod.Plan.workspace = guarded
    try:
        yield
    finally:
        hf_mod.Plan.workspace = orig
    torch.cuda.synchronize()
    for buf, n in guards:
        lo, hi = buf[:CANARY], buf[CANARY + n:]
        assert bool((lo == CANARY_LO).all()), "a write landed in the guard band below a workspace"
        assert bool((hi == CANARY_HI).all()), "a write landed in the guard band above a workspace"
