"""Host side of the batched autotuner: the workload signature and the cache file.

A cache hit with a host copy of the segment table answers without any CUDA call, so
these run without a GPU (the device pointers passed are never touched).
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def m():
    from paper_2005_12648_gb300 import build_ext

    build_ext.build_library()
    import paper_2005_12648_gb300 as ipm

    ipm.load()
    return ipm


def _table(lengths_a, lengths_b):
    la, lb = np.asarray(lengths_a, np.int64), np.asarray(lengths_b, np.int64)
    off = np.concatenate([[0], np.cumsum(la + lb)[:-1]])
    return np.stack([off, la, lb], axis=1)


def test_signature_depends_on_the_coarse_statistics_only(m):
    rng = np.random.default_rng(3)
    la = rng.integers(16, 5000, 1000)
    lb = rng.integers(16, 5000, 1000)
    t = _table(la, lb)
    s = m.ipm_batched_tune_signature(t, "int32")
    # order of the table and small changes of the lengths leave it unchanged
    perm = rng.permutation(1000)
    assert m.ipm_batched_tune_signature(_table(la[perm], lb[perm]), "int32") == s
    assert m.ipm_batched_tune_signature(_table(la + (la % 2 == 0), lb), "int32") in (s,)
    # key type, payload, segment count and longest segment enter it
    assert m.ipm_batched_tune_signature(t, "uint64") != s
    assert m.ipm_batched_tune_signature(t, "int32", with_values=True) != s
    assert m.ipm_batched_tune_signature(t[:300], "int32") != s
    big = t.copy()
    big[0, 1] = 1 << 20
    assert m.ipm_batched_tune_signature(big, "int32") != s


def test_cache_hit_answers_without_timing(m, tmp_path):
    L = m.load()
    t = _table([100, 2000, 30], [50, 4000, 7])
    sig = m.ipm_batched_tune_signature(t, "int32")
    path = tmp_path / "tune.txt"
    path.write_text("garbage line\n"
                    f"ipmtune2 {sig} 1 0 0 1 9.0\n"
                    "ipmtune2 0123456789abcdef 2 1 1 2 1.0\n"
                    f"ipmtune1 {sig} 2 0 0 0.1\n"  # an older format: ignored
                    f"ipmtune2 {sig} 3 2 1 2 0.5\n")  # the last matching line wins
    hs = np.ascontiguousarray(t.view(np.uint64))
    res = m.IpmBatchedTuneResult()
    fake = 0x1000  # never dereferenced on a cache hit
    rc = L.ipm_merge_batched_tune(fake, None, int(t[:, 1:].sum()), fake, hs.ctypes.data, 3, 0,
                                  1, fake, None, fake, 1 << 20, 5, str(path).encode(),
                                  ctypes.addressof(res), None)
    assert rc == 0
    d = res.as_dict()
    assert d["from_cache"] and d["candidates"] == 0 and d["signature"] == sig
    assert d["best"] == {"tile": 3, "ctas_per_sm": 2, "order": 1, "form": 2}
    assert d["best_ms"] == pytest.approx(0.5)


def test_tune_argument_errors(m):
    L = m.load()
    res = m.IpmBatchedTuneResult()
    hs = np.zeros((1, 3), np.uint64)
    # reps out of range, NULL result, payload type other than uint32
    assert L.ipm_merge_batched_tune(0x1000, None, 10, 0x2000, hs.ctypes.data, 1, 0, 1, 0x3000,
                                    None, 0x4000, 1 << 20, 0, b"", ctypes.addressof(res),
                                    None) == 1
    assert L.ipm_merge_batched_tune(0x1000, None, 10, 0x2000, hs.ctypes.data, 1, 0, 1, 0x3000,
                                    None, 0x4000, 1 << 20, 5, b"", None, None) == 1
    assert L.ipm_merge_batched_tune(0x1000, 0x5000, 10, 0x2000, hs.ctypes.data, 1, 0, 2,
                                    0x3000, 0x6000, 0x4000, 1 << 20, 5, b"",
                                    ctypes.addressof(res), None) == 2
    # scratch payload buffer missing while payloads are given
    assert L.ipm_merge_batched_tune(0x1000, 0x5000, 10, 0x2000, hs.ctypes.data, 1, 0, 1,
                                    0x3000, None, 0x4000, 1 << 20, 5, b"",
                                    ctypes.addressof(res), None) == 1
    # tuning workspace: the largest of the three tiles' workspaces
    ws = m.ipm_merge_batched_tune_workspace_bytes(1 << 20, 100, "int32")
    for tile in (1, 2, 3):
        assert ws >= m.ipm_merge_batched_workspace_bytes(1 << 20, 100, "int32",
                                                         options={"tile": tile})
