"""A bounded device wait that runs out, and a GPU that stays usable after it.

Every wait in which a CTA of a merge waits for another CTA (the exchange levels'
"reads done" flags and step joins, the fused merge's group barrier) gives up after the
call's wait limit, records IPM_ERR_TIMEOUT in the workspace status word and leaves; the
call's later kernels then skip their work.  Here the limit is set to 1 ns, so the first
such wait that needs more than a few polls expires during an ordinary multi-level merge.
No trap, no fault and no unbounded wait is involved.  Afterwards the default limit is
restored and the same workspace merges a fresh buffer exactly.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu

TIMEOUT = 6


def test_expired_wait_is_reported_and_the_gpu_stays_usable(ipm, dev, orc):
    import torch

    la = lb = 1 << 24  # int32: two exchange levels, then 4 groups of the fused merge
    _, levels = ipm.ipm_merge_fused_plan(la, lb, "int32")
    assert levels > 0
    host = W.make_buffer("uniform", np.int32, la, lb, seed=17)
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "int32"), dev)
    statuses = []
    ipm.ipm_set_wait_limit_ns(1)
    try:
        for _ in range(3):
            buf = to_dev(host, dev)
            ipm.ipm_merge_inplace(buf, la, lb, "int32", ws)
            statuses.append(ipm.ipm_read_device_status(ws))
            if statuses[-1] == TIMEOUT:
                break
    finally:
        ipm.ipm_set_wait_limit_ns(0)
    assert statuses[-1] == TIMEOUT, statuses
    assert set(statuses) <= {0, TIMEOUT}
    torch.cuda.synchronize()

    # default limit again: the same workspace, a fresh copy of the input
    assert ipm.ipm_get_wait_limit_ns() == 2_000_000_000
    buf = to_dev(host, dev)
    ipm.ipm_merge_inplace(buf, la, lb, "int32", ws)
    assert ipm.ipm_read_device_status(ws) == 0
    want = orc.merge(host[:la], host[la:])
    assert np.array_equal(from_dev(buf, np.int32), want)
