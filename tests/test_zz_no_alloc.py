"""The merge entry point for callers that cannot allocate device memory.

ipm_merge_inplace_noalloc takes no workspace: its scratch is a fixed array inside the
library.  It exists for callers that cannot call cudaMalloc: code running while another
framework's pool holds nearly all device memory, latency-critical paths that cannot
afford an allocation (and the synchronisation a later cudaFree brings), and plain C
callers without an allocator.  These tests call it through the C ABI twice in a row (the
second call finds the first call's leftovers in the shared array), compare each result
bit for bit with the allocating entry point ipm_merge_inplace on the same input and with
the CPU oracle, read the call's device status from the array, and check that a buffer
that is not memory of the current device is refused before anything runs.  This file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.int32, np.uint64])
def test_noalloc_equals_the_allocating_merge_on_two_calls_in_a_row(ipm, dev, orc, dtype):
    import torch

    name = {np.int32: "int32", np.uint64: "uint64"}[dtype]
    cases = [("uniform", 3_000_001, 2_500_000, 1), ("dup16", 1_000_003, 4_200_000, 2)]
    for dist, la, lb, seed in cases:
        host = W.make_buffer(dist, dtype, la, lb, seed)
        ref = to_dev(host, dev)
        ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, name), dev)
        ipm.ipm_merge_inplace(ref, la, lb, name, ws)
        got = to_dev(host, dev)
        ipm.ipm_merge_inplace_noalloc(got, la, lb, name)
        assert ipm.ipm_read_noalloc_status() == 0
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (dist, la, lb)
        want = orc.merge(host[:la], host[la:])
        assert np.array_equal(from_dev(got, dtype), want), (dist, la, lb)


def test_noalloc_at_its_largest_size(ipm, dev):
    """2^15 full tiles of int32 keys, the most the fixed scratch serves (~1.1e9 keys):
    accepted, and equal to the allocating merge.  The runs are drawn on the device."""
    import torch

    _, tile = ipm.ipm_merge_plan(1, 1, "int32")
    n = (1 << 15) * tile
    la, lb = n // 2, n - n // 2
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    a = torch.randint(0, 2**31 - 1, (la,), device=dev, dtype=torch.int32, generator=g)
    b = torch.randint(0, 2**31 - 1, (lb,), device=dev, dtype=torch.int32, generator=g)
    buf = torch.cat([a.sort().values, b.sort().values])
    del a, b
    ref = buf.clone()
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, "int32"), dev)
    ipm.ipm_merge_inplace(ref, la, lb, "int32", ws)
    ipm.ipm_merge_inplace_noalloc(buf, la, lb, "int32")
    assert ipm.ipm_read_noalloc_status() == 0
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)
    assert bool((ref[1:] >= ref[:-1]).all())


def test_noalloc_refuses_memory_that_is_not_on_the_current_device(ipm, dev):
    import torch

    host = np.arange(2000, dtype=np.int32)[::-1].copy()
    pinned = torch.from_numpy(host.copy()).pin_memory()
    for ptr in (pinned.data_ptr(), host.ctypes.data):
        with pytest.raises(ipm.IpmError) as e:
            ipm.ipm_merge_inplace_noalloc(ptr, 1000, 1000, "int32")
        assert e.value.code == 7  # IPM_ERR_DEVICE, nothing launched
    assert np.array_equal(pinned.numpy(), host)
    assert np.array_equal(host, np.arange(2000, dtype=np.int32)[::-1])


def test_noalloc_rejects_inputs_beyond_its_scratch(ipm):
    # 2^31 int32 keys need 2^16 pairs, more than the fixed scratch serves; the call
    # is refused on the host before any device work.
    with pytest.raises(ipm.IpmError) as e:
        ipm.ipm_merge_inplace_noalloc(0x1000, 1 << 30, 1 << 30, "int32")
    assert e.value.code == 1
