"""GPU parity at the full workload sizes, in the launch configuration bench.py times
(automatic pair count), element by element against the oracle's merge."""
import numpy as np
import pytest

import workloads as W
from gpu_util import NAME, first_diff, from_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _run(ipm, dev, orc, dist, dt, la, lb, seed=0):
    import torch

    buf = W.make_buffer_torch(torch, dist, dt, la, lb, seed, dev)
    host = W.as_numpy_keys(buf, dt)
    a, b = host[:la], host[la:]
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, NAME[np.dtype(dt)]), dev)
    ipm.ipm_merge_inplace(buf, la, lb, NAME[np.dtype(dt)], ws)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    got = from_dev(buf, dt)
    del buf
    want = orc.merge(a, b)
    assert first_diff(got, want) is None


@pytest.mark.parametrize("dist", ["uniform", "dup16", "alternation", "disjoint",
                                  "revdisjoint"])
def test_int32_2p28_plus_2p28(ipm, dev, orc, dist):
    _run(ipm, dev, orc, dist, np.int32, 1 << 28, 1 << 28)


def test_int32_unbalanced_2p29_2p20(ipm, dev, orc):
    _run(ipm, dev, orc, "uniform", np.int32, 1 << 29, 1 << 20)


@pytest.mark.parametrize("dist", ["uniform", "alternation"])
def test_uint64_2p28_plus_2p28(ipm, dev, orc, dist):
    _run(ipm, dev, orc, dist, np.uint64, 1 << 28, 1 << 28)


def test_kv_zipf_2p26_plus_2p26(ipm, dev, orc):
    import torch

    la = lb = 1 << 26
    keys = W.make_buffer_torch(torch, "zipf", np.uint32, la, lb, 0, dev)
    host = W.as_numpy_keys(keys, np.uint32)
    vals = torch.arange(la + lb, dtype=torch.int32, device=dev)
    ipm.merge_inplace_kv(keys, vals, la, lb, "uint32")
    torch.cuda.synchronize()
    wk, wv = orc.merge_kv(host[:la], np.arange(la, dtype=np.uint32), host[la:],
                          np.arange(la, la + lb, dtype=np.uint32))
    assert first_diff(from_dev(keys, np.uint32), wk) is None
    assert np.array_equal(from_dev(vals, np.uint32), wv)


def test_int64_2p28_plus_2p28(ipm, dev, orc):
    _run(ipm, dev, orc, "uniform", np.int64, 1 << 28, 1 << 28)


def test_kv8_uint64_2p27_plus_2p27(ipm, dev, orc):
    """uint64 keys with uint64 payloads (payload = original index, high bits set)."""
    import torch

    la = lb = 1 << 27
    keys = W.make_buffer_torch(torch, "uniform", np.uint64, la, lb, 0, dev)
    host = W.as_numpy_keys(keys, np.uint64)
    pay = np.arange(la + lb, dtype=np.uint64) | np.uint64(0xABCD000000000000)
    vals = torch.from_numpy(pay.view(np.int64).copy()).to(dev)
    ipm.merge_inplace_kv(keys, vals, la, lb, "uint64", val_dtype="uint64")
    torch.cuda.synchronize()
    wk, wv = orc.merge_kvw(host[:la], pay[:la], host[la:], pay[la:])
    assert first_diff(from_dev(keys, np.uint64), wk) is None
    assert np.array_equal(vals.cpu().numpy().view(np.uint64), wv)
