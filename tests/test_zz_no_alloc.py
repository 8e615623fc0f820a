"""hufield_spectrum_noalloc: the allocation-free spectrum call (static device
scratch instead of a plan and workspace) gives the same bins as
hufield_spectrum, call after call.  Some callers cannot allocate device memory
(a plugin that may only use buffers handed to it, a host-managed memory budget,
a latency-critical loop that cannot take cudaMalloc's device synchronisation);
this entry point serves them.  Collected last so that a stop-at-first-failure
run has already run every other test."""
import numpy as np
import pytest
import torch

from tests import inputs
from tests.gpu_common import check_bins, dev_zeros, np_

pytestmark = pytest.mark.gpu

CASES = [((256, 256), 64, 6), ((1024, 1024), 128, 1), ((16, 32, 64), 16, 1), ((128, 128, 64), 32, 1)]


def _with_plan(hf, shape, y, nr, nt):
    plan = hf.Plan(shape)
    ws = plan.workspace(1, nr * nt)
    s, c = dev_zeros(nr * nt, torch.float64), dev_zeros(nr * nt, torch.int64)
    hf.hufield_spectrum(plan, y, nr, nt, False, s, c, ws)
    torch.cuda.synchronize()
    return np_(s), np_(c)


@pytest.mark.parametrize("shape,nr,nt", CASES)
def test_noalloc_matches_workspace_call_twice(hf, shape, nr, nt):
    y1 = torch.from_numpy(inputs.random_field(shape, 31, np.float32)).cuda()
    y2 = torch.from_numpy(np.where(inputs.random_field(shape, 32) >= 0.3, 1, -1).astype(np.int8)).cuda()
    want1 = _with_plan(hf, shape, y1, nr, nt)
    want2 = _with_plan(hf, shape, y2, nr, nt)
    for y, (ws_, wc) in ((y1, want1), (y1, want1), (y2, want2)):  # two calls in a row, then new data
        s, c = dev_zeros(nr * nt, torch.float64), dev_zeros(nr * nt, torch.int64)
        hf.hufield_spectrum_noalloc(shape, y, nr, nt, False, s, c)
        torch.cuda.synchronize()
        assert hf.hufield_spectrum_noalloc_status() == hf.OK
        check_bins(np_(s), ws_, np_(c), wc)


def test_noalloc_allocates_nothing(hf):
    # after the first call on the device (the set-up, and the first use of the
    # kernels), further calls leave both torch's pool and the device's free
    # memory exactly as they were
    shape, nr = (128, 128), 32
    y = torch.from_numpy(inputs.random_field(shape, 34, np.float32)).cuda()
    s, c = dev_zeros(nr, torch.float64), dev_zeros(nr, torch.int64)
    hf.hufield_spectrum_noalloc(shape, y, nr, 1, False, s, c)
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        hf.hufield_spectrum_noalloc(shape, y, nr, 1, True, s, c)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert after == before
    assert hf.hufield_spectrum_noalloc_status() == hf.OK


def test_noalloc_accumulates_and_rejects_too_large(hf):
    shape = (64, 64)
    y = torch.from_numpy(inputs.random_field(shape, 33, np.float32)).cuda()
    s, c = dev_zeros(16, torch.float64), dev_zeros(16, torch.int64)
    hf.hufield_spectrum_noalloc(shape, y, 16, 1, False, s, c)
    hf.hufield_spectrum_noalloc(shape, y, 16, 1, True, s, c)
    torch.cuda.synchronize()
    ws_, wc = _with_plan(hf, shape, y, 16, 1)
    check_bins(np_(s) / 2, ws_, np_(c) // 2, wc)
    big = torch.zeros((2048, 1024), device="cuda")
    with pytest.raises(hf.HufieldError) as e:
        hf.hufield_spectrum_noalloc((2048, 1024), big, 16, 1, False, s, c)
    assert e.value.status == hf.ERR_TOO_LARGE
    # buffers that do not match the lattice or the bins are refused before any launch
    for args in (((64, 128), y, 16, 1), (shape, y, 32, 1), (shape, y, 4, 8)):
        with pytest.raises(hf.HufieldError) as e:
            hf.hufield_spectrum_noalloc(*args, False, s, c)
        assert e.value.status == hf.ERR_INVALID_ARG
