"""Failure detection without a GPU fault: the strided passes bound every wait
on their bulk copies.  A test-hook plan never issues one load, so its waits
run out (~2 ms); the call must report the timeout through the workspace
status word, and the context must stay usable for correct work afterwards."""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs
from tests.gpu_common import check_field, filters, np_

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(256, 256), (32, 16, 64)])
def test_timeout_is_reported_and_context_survives(hf, shape):
    fk = dict(p=3.0, axes=(1.0, 0.8, 1.2), k0=0.3, width=0.1, supp=2.0)
    gf, of = filters(hf, **fk)
    bad = hf.Plan(shape, inject_timeout=True)
    ws = bad.workspace(0, 0)
    out = torch.empty(shape, device="cuda")
    hf.hufield_generate(bad, gf, 0, 0, out, ws)  # enqueued: the failure is on the device
    assert hf.hufield_workspace_status(ws) == hf.ERR_TIMEOUT
    good = hf.Plan(shape)
    hf.hufield_generate(good, gf, 0, 0, out, ws)  # same workspace: the new call clears the word
    assert hf.hufield_workspace_status(ws) == hf.OK
    torch.cuda.synchronize()
    check_field(np_(out), oracle.generate(shape, of, 0, 0))


def test_status_ok_after_spectrum_and_pipeline(hf):
    shape = (64, 64)
    plan = hf.Plan(shape)
    ws = plan.workspace(1, 16)
    y = torch.from_numpy(inputs.random_field(shape, 4, np.float32)).cuda()
    s = torch.zeros(16, dtype=torch.float64, device="cuda")
    c = torch.zeros(16, dtype=torch.int64, device="cuda")
    hf.hufield_spectrum(plan, y, 16, 1, False, s, c, ws)
    assert hf.hufield_workspace_status(ws) == hf.OK
