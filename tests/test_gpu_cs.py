"""GPU parity of the circular-shifting exchange (Sec. 3.4) against the oracle's CS.

Sizes cover both execution modes of the kernel: every cycle handled whole by one
worker (short cycles, including more cycles than workers), and long cycles cut into
segments (one cycle, a few cycles, >= 32 cycles), for 4- and 8-byte elements.
"""
import numpy as np
import pytest

from gpu_util import first_diff, from_dev, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    (1, 1), (1, 2), (2, 1), (3, 5), (7, 7), (6, 9),
    (1000, 9),                        # one cycle of 1009, segmented
    (1000, 1000),                     # 1000 cycles of 2, whole
    (4096, 12288),                    # 4096 cycles of 4
    (1, 100_003), (100_003, 1),       # one cycle
    (999_983, 7919),                  # coprime: one long cycle, many segments
    (64 * 100_003, 64 * 77_777),      # 64 cycles of 177,780, segmented, coalesced
    (1 << 21, 1 << 21),               # 2^21 cycles of 2: more cycles than workers
    (3 << 20, 1 << 21),               # 2^20 cycles of 5
    ((1 << 22) + 1, (1 << 22) - 1),   # gcd 1
    (12 * 65_537, 18 * 65_537),       # 6 * 65,537 cycles of 5
]


def _data(n, dt, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, np.iinfo(dt).max, n, dtype=dt, endpoint=True)


@pytest.mark.parametrize("elem", [4, 8])
def test_cs_rotate_matches_oracle(ipm, dev, orc, elem):
    import torch

    dt = np.uint32 if elem == 4 else np.uint64
    for lx, ly in CASES:
        x = _data(lx + ly, dt, lx ^ ly)
        t = to_dev(x, dev)
        ws = ipm.workspace(ipm.ipm_rotate_cs_workspace_bytes(lx, ly, elem), dev)
        ipm.ipm_rotate_cs(t, lx, ly, elem, ws)
        torch.cuda.synchronize()
        assert ipm.ipm_read_device_status(ws) == 0
        got = from_dev(t, dt)
        if lx + ly <= 1 << 22:
            want, cycles, moves = orc.cs_rotate(x, lx)
            assert cycles == np.gcd(lx, ly) and moves == lx + ly
        else:
            want = np.roll(x, -lx)
        assert first_diff(got, want) is None, (lx, ly)


def test_cs_rotate_empty_sides_are_no_ops(ipm, dev):
    import torch

    x = _data(1000, np.uint32, 3)
    t = to_dev(x, dev)
    ws = ipm.workspace(4096, dev)
    ipm.ipm_rotate_cs(t, 0, 1000, 4, ws)
    ipm.ipm_rotate_cs(t, 1000, 0, 4, ws)
    torch.cuda.synchronize()
    assert first_diff(from_dev(t, np.uint32), x) is None


def test_cs_and_ls_agree_on_a_misaligned_range(ipm, dev):
    """Both exchanges on the same sub-range that starts at an odd element offset."""
    import torch

    dt = np.uint32
    x = _data(3_000_001, dt, 5)
    off, lx, ly = 3, 1_234_567, 1_000_003
    res = []
    for rot, wsq in ((ipm.ipm_rotate, ipm.ipm_rotate_workspace_bytes),
                     (ipm.ipm_rotate_cs, ipm.ipm_rotate_cs_workspace_bytes)):
        t = to_dev(x, dev)
        ws = ipm.workspace(wsq(lx, ly, 4), dev)
        rot(t[off:], lx, ly, 4, ws)
        torch.cuda.synchronize()
        res.append(from_dev(t, dt))
    want = x.copy()
    want[off:off + lx + ly] = np.roll(x[off:off + lx + ly], -lx)
    assert first_diff(res[0], want) is None
    assert first_diff(res[1], want) is None


@pytest.mark.slow
@pytest.mark.parametrize("lx", [1 << 28, (1 << 28) + 64, (1 << 28) + 1])
def test_cs_rotate_fullsize(ipm, dev, lx):
    """2^29 uint32 elements (2 GiB) at the three split points the bench times."""
    import torch

    n = 1 << 29
    t = torch.randint(0, 1 << 31, (n,), dtype=torch.int64, device=dev).to(torch.int32)
    want = torch.roll(t, -lx)
    ws = ipm.workspace(ipm.ipm_rotate_cs_workspace_bytes(lx, n - lx, 4), dev)
    ipm.ipm_rotate_cs(t, lx, n - lx, 4, ws)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    assert torch.equal(t, want)
