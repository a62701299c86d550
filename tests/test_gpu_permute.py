"""GPU parity of the division stage by one permutation (sOptMov, Alg. 2, Sec. 3.2).

The arranged layout A_0 B_0 A_1 B_1 ... of a split table has a plain definition (the
oracle's arrange), so the permutation must reproduce it bit for bit: from exact merge
splits and from arbitrary valid tables, with and without payloads, on sizes that leave
cycles for the sampled rounds and for the out-of-place last round, and on the
degenerate tables (one pair, empty runs, more pairs than elements).
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import NAME, first_diff, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _random_table(rng, la, lb, G):
    """A valid table that is not a merge's: i_k drawn between the bounds the layout
    allows (both parts of every pair inside A and B)."""
    n, P = la + lb, 1 << G
    d = [(k * n) >> G for k in range(P + 1)]
    i = [0] * (P + 1)
    i[P] = la
    for k in range(1, P):
        lo = max(i[k - 1], d[k] - lb, la - (n - d[k]))
        hi = min(la, d[k], i[k - 1] + (d[k] - d[k - 1]))
        i[k] = int(rng.integers(lo, hi + 1)) if hi > lo else lo
    return np.array(i, dtype=np.uint64)


def _payload(n, vb):
    idx = np.arange(n, dtype=np.uint64)
    if vb == 8:
        return (idx << np.uint64(32)) | ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF))
    return ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def _permute(ipm, dev, a, b, split_np, G, dt, vb):
    import torch

    la, lb = a.size, b.size
    name = NAME[np.dtype(dt)]
    buf = to_dev(np.concatenate([a, b]), dev)
    vals = None
    if vb:
        pay = _payload(la + lb, vb)
        vals = torch.from_numpy(pay.view(np.int64 if vb == 8 else np.int32).copy()).to(dev)
    split = torch.from_numpy(split_np.astype(np.int64)).to(dev)
    ws = ipm.workspace(ipm.ipm_rearrange_permute_workspace_bytes(la, lb, name, vb), dev)
    ipm.ipm_rearrange_permute(buf, vals, la, lb, name, split, G, ws, with_values=vb)
    torch.cuda.synchronize()
    got_v = None
    if vb:
        got_v = vals.cpu().numpy().view(np.uint64 if vb == 8 else np.uint32)
    return from_dev(buf, dt), got_v


CASES = [(50_000, 43_211, "uniform", 4), (30_001, 30_000, "dup16", 7),
         (20_000, 20_000, "revdisjoint", 3), (90_000, 77, "uniform", 6),
         (77, 90_000, "uniform", 6), (1_000_003, 700_001, "uniform", 10),
         (123_457, 98_765, "alternation", 9), (5, 3, "uniform", 4), (0, 1000, "uniform", 2),
         (1000, 0, "uniform", 2), (4096, 4096, "uniform", 0), (1, 1, "uniform", 1)]


@pytest.mark.parametrize("dt,vb", [(np.int32, 0), (np.uint32, 4), (np.float32, 8),
                                   (np.uint64, 0), (np.int64, 4), (np.uint64, 8)])
def test_permute_merge_splits_match_oracle_layout(ipm, dev, orc, dt, vb):
    for la, lb, dist, G in CASES:
        if dist == "alternation" and dt == np.float32:
            dist = "dup16"
        a, b = W.make_pair(dist, dt, la, lb, seed=la + 7 * lb + G)
        d = orc.diagonals(la + lb, 1 << G)
        i = orc.splits_replay(a, b, d)
        got, got_v = _permute(ipm, dev, a, b, i, G, dt, vb)
        assert first_diff(got, orc.arrange(a, b, d, i)) is None, (la, lb, dist, G)
        if vb:
            pay = _payload(la + lb, vb)
            assert np.array_equal(got_v, orc.arrange(pay[:la], pay[la:], d, i)), (la, lb, G)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_permute_random_tables_match_oracle_layout(ipm, dev, orc, seed):
    """Tables that are no merge's: the cycle structure differs (short cycles, many
    fixed points), which exercises the later rounds and the out-of-place round."""
    rng = np.random.default_rng(seed)
    for la, lb, G in [(4096, 4096, 5), (9999, 3, 7), (7, 9999, 7), (200_000, 200_000, 10),
                      (1_000_000, 777_777, 12), (3, 5, 4)]:
        a, b = W.make_pair("uniform", np.uint32, la, lb, seed=seed + la)
        i = _random_table(rng, la, lb, G)
        d = orc.diagonals(la + lb, 1 << G)
        got, got_v = _permute(ipm, dev, a, b, i, G, np.uint32, 4)
        assert first_diff(got, orc.arrange(a, b, d, i)) is None, (la, lb, G)
        pay = _payload(la + lb, 4)
        assert np.array_equal(got_v, orc.arrange(pay[:la], pay[la:], d, i)), (la, lb, G)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
def test_merge_through_permutation_matches_oracle(ipm, dev, orc, dt):
    """The whole merge with the permutation as its division stage: device splits, one
    permutation, the pair merge."""
    import torch

    name = NAME[np.dtype(dt)]
    for la, lb, dist in [(3_000_017, 2_900_011, "uniform"), (1_000_003, 700_001, "dup16"),
                         (2_000_001, 17, "uniform")]:
        a, b = W.make_pair(dist, dt, la, lb, seed=la - lb)
        G = ipm.ipm_merge_plan(la, lb, name)[0]
        buf = to_dev(np.concatenate([a, b]), dev)
        split = torch.empty((1 << G) + 1, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits(buf, la, lb, name, 1 << G, split)
        ws = ipm.workspace(ipm.ipm_rearrange_permute_workspace_bytes(la, lb, name), dev)
        ipm.ipm_rearrange_permute(buf, None, la, lb, name, split, G, ws)
        ipm.ipm_merge_pairs(buf, None, la, lb, name, split, G)
        torch.cuda.synchronize()
        assert first_diff(from_dev(buf, dt), orc.merge(a, b)) is None, (la, lb, dist)


def test_permute_rejects_a_table_that_is_not_a_layout(ipm, dev):
    """A table whose pair would take more A elements than its diagonal allows is
    reported as an invalid argument before any element moves."""
    import torch

    la, lb, G = 1000, 1000, 3
    a, b = W.make_pair("uniform", np.int32, la, lb, seed=5)
    x = np.concatenate([a, b])
    buf = to_dev(x, dev)
    bad = np.array([((k * 2000) >> G) // 2 for k in range(9)], dtype=np.int64)  # valid
    bad[4] = 800  # pair 3 would take 425 A elements on a diagonal step of 250
    split = torch.from_numpy(bad).to(dev)
    ws = ipm.workspace(ipm.ipm_rearrange_permute_workspace_bytes(la, lb, "int32"), dev)
    with pytest.raises(ipm.IpmError) as e:
        ipm.ipm_rearrange_permute(buf, None, la, lb, "int32", split, G, ws)
    assert e.value.code == 1
    torch.cuda.synchronize()
    assert first_diff(from_dev(buf, np.int32), x) is None
