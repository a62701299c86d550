"""The merge entry point for callers that cannot allocate device memory.

ipm_merge_inplace_noalloc takes no workspace: its scratch is a fixed array inside
the library.  It exists for callers that cannot call cudaMalloc (memory held by
another framework's pool, allocation-free latency-critical paths, plain C callers
without an allocator).  These tests call it through the C ABI twice in a row (the
second call finds the first call's leftovers in the shared array) and compare each
result, bit for bit, with the allocating entry point ipm_merge_inplace on the same
input.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_equals_the_allocating_merge_on_two_calls_in_a_row(ipm, dev):
    import torch

    cases = [("uniform", 3_000_001, 2_500_000, 1), ("dup16", 1_000_003, 4_200_000, 2)]
    for dist, la, lb, seed in cases:
        host = W.make_buffer(dist, np.int32, la, lb, seed)
        ref = torch.from_numpy(host.copy()).to(dev)
        ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "int32"), dev)
        ipm.ipm_merge_inplace(ref, la, lb, "int32", ws)
        got = torch.from_numpy(host.copy()).to(dev)
        ipm.ipm_merge_inplace_noalloc(got, la, lb, "int32")
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (dist, la, lb)


def test_noalloc_rejects_inputs_beyond_its_scratch(ipm):
    # 2^31 int32 keys need 2^16 pairs, more than the fixed scratch serves; the call
    # is refused on the host before any device work.
    with pytest.raises(ipm.IpmError) as e:
        ipm.ipm_merge_inplace_noalloc(0x1000, 1 << 30, 1 << 30, "int32")
    assert e.value.code == 1
