"""GPU parity: every step of the hot path, through the C ABI, against the CPU oracle.

Integer, byte and index work, so the bar is bit-exact equality everywhere.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import NAME, bits, first_diff, from_dev, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.uint64, np.float32, np.int64]


def _merge_dev(ipm, dev, a, b, log2_pairs=0):
    import torch

    buf = to_dev(np.concatenate([a, b]), dev)
    ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(a.size, b.size, NAME[a.dtype], False,
                                                     log2_pairs), dev)
    ipm.ipm_merge_inplace(buf, a.size, b.size, NAME[a.dtype], ws, log2_pairs)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    return from_dev(buf, a.dtype)


# ----------------------------------------------------------------------- step a1

@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("dist", ["uniform", "dup16", "alternation", "revdisjoint"])
def test_splits_match_oracle(ipm, dev, orc, dt, dist):
    import torch

    if dist == "alternation" and dt == np.float32:
        pytest.skip("alternation is an integer layout")
    for la, lb, P in [(0, 0, 1), (0, 17, 4), (17, 0, 4), (1, 1, 2), (1000, 1, 7),
                      (70_001, 65_537, 64), (123_457, 98_765, 1000), (5000, 5000, 10_000)]:
        if dist == "alternation" and dt == np.float32:
            continue
        a, b = W.make_pair(dist, dt, la, lb, seed=la + lb)
        buf = to_dev(np.concatenate([a, b]), dev)
        out = torch.empty(P + 1, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits(buf, la, lb, NAME[np.dtype(dt)], P, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.uint64)
        want = orc.splits_replay(a, b, orc.diagonals(la + lb, P))
        assert np.array_equal(got, want), (la, lb, P)


@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32, np.int64])
@pytest.mark.parametrize("dist", ["uniform", "dup16", "zipf", "disjoint", "revdisjoint"])
def test_two_pass_splits_match_oracle(ipm, dev, orc, dt, dist):
    """Many diagonals (P >= 2048, a multiple of 32) take two passes: every 32nd diagonal
    over its whole range, then the others inside the brackets their coarse neighbours
    give; every entry equals the oracle's replayed split, including runs of equal keys
    across the brackets, one-sided regions and unbalanced runs."""
    import torch

    if dist == "zipf" and dt == np.float32:
        dist = "dup16"
    for la, lb, P in [(1_500_007, 1_400_011, 2048), (3_000_017, 41, 4096),
                      (37, 2_200_003, 8192), (600_001, 600_001, 16_384), (5000, 7000, 2048)]:
        a, b = W.make_pair(dist, dt, la, lb, seed=la + 3 * lb)
        buf = to_dev(np.concatenate([a, b]), dev)
        out = torch.empty(P + 1, dtype=torch.int64, device=dev)
        ipm.ipm_merge_splits(buf, la, lb, NAME[np.dtype(dt)], P, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.uint64)
        want = orc.splits_replay(a, b, orc.diagonals(la + lb, P))
        assert np.array_equal(got, want), (la, lb, P, dist)


# ----------------------------------------------------------------------- step a2

@pytest.mark.parametrize("elem", [4, 8])
def test_rotate_matches_roll(ipm, dev, elem):
    import torch

    dt = np.uint32 if elem == 4 else np.uint64
    cases = [(1, 1), (1, 2), (2, 1), (3, 5), (100, 100), (4097, 4095), (1, 100_003),
             (100_003, 1), (65_536, 131_071), (1 << 20, (1 << 20) + 77), (999_983, 7919),
             # both the size difference and the smaller block exceed the on-chip stash:
             # linear-shifting block swaps first, then the closed-form pass
             (3_000_017, 260_001), (260_001, 2_900_011), (1_000_003, 700_001),
             (700_001, 1_000_003), (4_000_037, 3_700_019)]
    for lx, ly in cases:
        x = np.arange(lx + ly, dtype=dt) * 2654435761 % (1 << 31)
        t = to_dev(x, dev)
        ws = ipm.workspace(ipm.ipm_rotate_workspace_bytes(lx, ly, elem), dev)
        ipm.ipm_rotate(t, lx, ly, elem, ws)
        torch.cuda.synchronize()
        got = from_dev(t, dt)
        assert first_diff(got, np.roll(x, -lx)) is None, (lx, ly)


@pytest.mark.parametrize("dt", [np.int32, np.uint64])
@pytest.mark.parametrize("G", [1, 2, 3, 5, 8])
def test_rearrange_matches_oracle_layout(ipm, dev, orc, dt, G):
    import torch

    for dist, la, lb in [("uniform", 50_000, 43_211), ("dup16", 30_001, 30_000),
                         ("revdisjoint", 20_000, 20_000), ("uniform", 90_000, 77)]:
        a, b = W.make_pair(dist, dt, la, lb, seed=G)
        P = 1 << G
        d = orc.diagonals(la + lb, P)
        i = orc.splits_replay(a, b, d)
        buf = to_dev(np.concatenate([a, b]), dev)
        split = torch.from_numpy(i.astype(np.int64)).to(dev)
        # workspace size grows with G; the merge query needs pairs that fit a tile
        wsG = max(G, ipm.ipm_merge_plan(la, lb, NAME[np.dtype(dt)])[0])
        ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, NAME[np.dtype(dt)], False,
                                                         wsG), dev)
        ipm.ipm_merge_rearrange(buf, None, la, lb, NAME[np.dtype(dt)], split, G, ws)
        torch.cuda.synchronize()
        want = orc.arrange(a, b, d, i)
        assert first_diff(from_dev(buf, dt), want) is None, (dist, la, lb)


# ----------------------------------------------------------------------- step a3

@pytest.mark.parametrize("dt", DTYPES)
def test_pair_merge_of_arranged_buffer(ipm, dev, orc, dt):
    import torch

    for dist, la, lb, G in [("uniform", 40_000, 39_999, 2), ("dup16", 5, 70_000, 3),
                            ("uniform", 3, 3, 0), ("uniform", 60_000, 60_001, 4)]:
        a, b = W.make_pair(dist, dt, la, lb, seed=11)
        G = max(G, ipm.ipm_merge_plan(la, lb, NAME[np.dtype(dt)])[0])
        P = 1 << G
        d = orc.diagonals(la + lb, P)
        i = orc.splits_replay(a, b, d)
        buf = to_dev(orc.arrange(a, b, d, i), dev)
        split = torch.from_numpy(i.astype(np.int64)).to(dev)
        ipm.ipm_merge_pairs(buf, None, la, lb, NAME[np.dtype(dt)], split, G)
        torch.cuda.synchronize()
        assert first_diff(from_dev(buf, dt), orc.merge(a, b)) is None, (dist, la, lb)


# ----------------------------------------------------------------------- whole path

@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("dist", ["uniform", "dup16", "disjoint", "revdisjoint",
                                  "alternation"])
def test_merge_inplace_matches_oracle(ipm, dev, orc, dt, dist):
    if dist == "alternation" and dt == np.float32:
        pytest.skip("alternation is an integer layout")
    _, tile = ipm.ipm_merge_plan(1, 1, NAME[np.dtype(dt)])
    sizes = [(1, 1), (1, 0), (0, 1), (5, 3), (tile // 2, tile // 2),
             (tile // 2 + 1, tile // 2), (int(1.7 * tile), int(2.1 * tile) + 3),
             (3 * tile + 11, 29), (29, 3 * tile + 11), (5 * tile + 1, 4 * tile + 2)]
    for la, lb in sizes:
        a, b = W.make_pair(dist, dt, la, lb, seed=la * 7 + lb)
        got = _merge_dev(ipm, dev, a, b)
        want = orc.merge(a, b)
        assert first_diff(got, want) is None, (dist, la, lb)


@pytest.mark.parametrize("G", [1, 2, 4, 6, 9])
def test_merge_inplace_forced_pair_counts(ipm, dev, orc, G):
    for dt in (np.int32, np.uint64):
        for dist in ("uniform", "dup16", "paper"):
            a, b = W.make_pair(dist, dt, 20_011, 17_003, seed=G)
            if G < ipm.ipm_merge_plan(a.size, b.size, NAME[np.dtype(dt)])[0]:
                continue  # pairs would not fit one tile
            got = _merge_dev(ipm, dev, a, b, log2_pairs=G)
            assert first_diff(got, orc.merge(a, b)) is None, (dt, dist, G)


def test_float_signed_zero_bits(ipm, dev, orc):
    rng = np.random.default_rng(0)
    a = np.sort(rng.choice(np.array([-1.0, -0.0, 0.0, 1.0], np.float32), 50_000))
    b = np.sort(rng.choice(np.array([-0.0, 0.0, 2.0], np.float32), 60_000))
    got = _merge_dev(ipm, dev, a, b)
    assert np.array_equal(bits(got), bits(orc.merge(a, b)))


@pytest.mark.parametrize("dt", DTYPES)
def test_merge_inplace_kv_stable(ipm, dev, orc, dt):
    import torch

    _, tile = ipm.ipm_merge_plan(1, 1, NAME[np.dtype(dt)], with_values=True)
    dist = "zipf" if dt != np.float32 else "dup16"
    for la, lb in [(1, 1), (7, 0), (tile // 3, tile // 2), (3 * tile + 5, 2 * tile + 1),
                   (4 * tile, 17)]:
        a, b = W.make_pair(dist, dt, la, lb, seed=la + 3 * lb)
        keys = to_dev(np.concatenate([a, b]), dev)
        vals = torch.arange(la + lb, dtype=torch.int32, device=dev)
        ipm.merge_inplace_kv(keys, vals, la, lb, NAME[np.dtype(dt)])
        torch.cuda.synchronize()
        wk, wv = orc.merge_kv(a, np.arange(la, dtype=np.uint32), b,
                              np.arange(la, la + lb, dtype=np.uint32))
        assert first_diff(from_dev(keys, dt), wk) is None
        assert np.array_equal(from_dev(vals, np.uint32), wv)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("dist", ["zipf", "uniform", "dup16"])
def test_merge_inplace_kv8_matches_oracle(ipm, dev, orc, dt, dist):
    """8-byte payloads (every bit pattern: index in the high word, a hash in the low
    word) move with their keys exactly as the oracle's wide-payload merge moves them."""
    import torch

    if dist == "zipf" and dt == np.float32:
        dist = "dup16"
    _, tile = ipm.ipm_merge_plan(1, 1, NAME[np.dtype(dt)], with_values=8)
    for la, lb in [(1, 1), (0, 9), (9, 0), (tile // 3, tile // 2), (3 * tile + 5, 2 * tile + 1),
                   (5 * tile + 3, 7 * tile + 11), (4 * tile, 17)]:
        a, b = W.make_pair(dist, dt, la, lb, seed=la + 5 * lb)
        n = la + lb
        idx = np.arange(n, dtype=np.uint64)
        pay = (idx << np.uint64(32)) | ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF))
        pay[::7] |= np.uint64(1 << 63)
        keys = to_dev(np.concatenate([a, b]), dev)
        vals = torch.from_numpy(pay.view(np.int64).copy()).to(dev)
        ipm.merge_inplace_kv(keys, vals, la, lb, NAME[np.dtype(dt)], val_dtype="uint64")
        torch.cuda.synchronize()
        wk, wv = orc.merge_kvw(a, pay[:la], b, pay[la:])
        assert first_diff(from_dev(keys, dt), wk) is None, (la, lb)
        assert np.array_equal(vals.cpu().numpy().view(np.uint64), wv), (la, lb)


@pytest.mark.parametrize("engine,fused", [(1, 0), (1, 2), (1, 5), (1, 8), (0, 4), (2, 1),
                                          (2, 9)])
@pytest.mark.parametrize("dt", [np.uint32, np.int64])
def test_kv8_fused_levels_match_oracle(ipm, dev, orc, engine, fused, dt):
    """8-byte payloads through every fused-level setting (the cluster engine hands
    8-byte payloads to the group barrier)."""
    import torch

    la, lb = 700_001, 655_357
    a, b = W.make_pair("uniform", dt, la, lb, seed=3)
    pay = np.arange(la + lb, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    try:
        ipm.ipm_set_fused_engine(engine)
        ipm.ipm_set_fused_levels(fused)
        keys = to_dev(np.concatenate([a, b]), dev)
        vals = torch.from_numpy(pay.view(np.int64).copy()).to(dev)
        ws = ipm.merge_inplace_kv(keys, vals, la, lb, NAME[np.dtype(dt)], val_dtype="uint64")
        torch.cuda.synchronize()
        assert ipm.ipm_read_device_status(ws) == 0
    finally:
        ipm.ipm_set_fused_engine(2)
        ipm.ipm_set_fused_levels(10)
    wk, wv = orc.merge_kvw(a, pay[:la], b, pay[la:])
    assert first_diff(from_dev(keys, dt), wk) is None
    assert np.array_equal(vals.cpu().numpy().view(np.uint64), wv)


@pytest.mark.parametrize("fused", [1, 2, 5, 9])
@pytest.mark.parametrize("dt,vb", [(np.uint32, 4), (np.float32, 8), (np.int64, 4),
                                   (np.uint64, 8)])
def test_kv_tensor_memory_engine_matches_oracle(ipm, dev, orc, fused, dt, vb):
    """Key-value merges through the two-pairs kernel (the first pair's keys and payloads
    parked in TMEM) for every key / payload width pair: fused depths from one level to
    the default, pair counts below the group size, empty runs, ties and ragged sizes."""
    import torch

    cases = [(3_000_017, 2_900_011, "uniform", 0), (123_457, 98_765, "dup16", 6),
             (1_000_000, 1, "uniform", 4), (50_000, 70_001, "zipf", 3),
             (333_333, 333_333, "revdisjoint", 5)]
    ipm.ipm_set_fused_levels(fused)
    try:
        for la, lb, dist, G in cases:
            if dist == "zipf" and dt == np.float32:
                dist = "dup16"
            a, b = W.make_pair(dist, dt, la, lb, seed=la + 3 * lb + fused)
            n = la + lb
            idx = np.arange(n, dtype=np.uint64)
            if vb == 8:
                pay = (idx << np.uint64(32)) | ((idx * np.uint64(2654435761)) &
                                               np.uint64(0xFFFFFFFF))
                vals = torch.from_numpy(pay.view(np.int64).copy()).to(dev)
            else:
                pay = (idx * np.uint64(2654435761) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
                vals = torch.from_numpy(pay.view(np.int32).copy()).to(dev)
            name = NAME[np.dtype(dt)]
            G = max(G, ipm.ipm_merge_plan(la, lb, name, with_values=vb)[0])
            assert ipm.ipm_merge_fused_plan(la, lb, name, with_values=vb)[0] == 2
            keys = to_dev(np.concatenate([a, b]), dev)
            ws = ipm.merge_inplace_kv(keys, vals, la, lb, name, log2_pairs=G)
            torch.cuda.synchronize()
            assert ipm.ipm_read_device_status(ws) == 0
            wk, wv = orc.merge_kvw(a, pay[:la], b, pay[la:])
            assert first_diff(from_dev(keys, dt), wk) is None, (la, lb, dist, G)
            got_v = vals.cpu().numpy().view(np.uint64 if vb == 8 else np.uint32)
            assert np.array_equal(got_v, wv), (la, lb, dist, G)
    finally:
        ipm.ipm_set_fused_levels(10)


def test_async_on_a_side_stream(ipm, dev, orc):
    import torch

    a, b = W.make_pair("uniform", np.int32, 300_000, 200_000, seed=1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        buf = to_dev(np.concatenate([a, b]), dev)
        ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(a.size, b.size, "int32"), dev)
        ipm.ipm_merge_inplace(buf, a.size, b.size, "int32", ws, stream=s)
    s.synchronize()
    assert first_diff(from_dev(buf, np.int32), orc.merge(a, b)) is None


@pytest.mark.parametrize("engine,fused", [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 1),
                                          (1, 3), (1, 5), (1, 6), (1, 7), (1, 8), (1, 10),
                                          (2, 1), (2, 2), (2, 5), (2, 8), (2, 9), (2, 10)])
@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.int64])
def test_fused_bottom_levels_match_oracle(ipm, dev, orc, engine, fused, dt):
    """The last `fused` levels done by groups of CTAs (each group stages its pairs, then
    writes them merged; groups synchronised by a thread-block cluster or by a barrier in
    global memory) give the oracle's merge for every depth, including pair counts below
    the group size, empty runs inside a group, ragged sizes and ties."""
    cases = [(3_000_017, 2_900_011, "uniform", 0), (1_000_003, 700_001, "dup16", 0),
             (50_000, 70_001, "uniform", 3), (123_457, 98_765, "alternation", 6),
             (1_000_000, 1, "uniform", 4), (333_333, 333_333, "revdisjoint", 5),
             (2_000_001, 17, "uniform", 0)]
    ipm.ipm_set_fused_levels(fused)
    ipm.ipm_set_fused_engine(engine)
    try:
        assert ipm.ipm_get_fused_levels() == fused
        for la, lb, dist, G in cases:
            if dist == "alternation" and dt == np.float32:
                continue
            a, b = W.make_pair(dist, dt, la, lb, seed=la + lb + fused)
            G = max(G, ipm.ipm_merge_plan(la, lb, NAME[np.dtype(dt)])[0])
            got = _merge_dev(ipm, dev, a, b, G)
            want = orc.merge(a, b)
            assert first_diff(got, want) is None, (la, lb, dist, G, first_diff(got, want))
    finally:
        ipm.ipm_set_fused_levels(10)
        ipm.ipm_set_fused_engine(2)


def test_default_fused_plan_uses_tensor_memory(ipm):
    """By default every key type, with or without a 4- or 8-byte payload, takes the
    two-pairs kernel that parks a merged pair in TMEM, fusing one level more than one
    pair per CTA."""
    n = 1 << 28
    e2, f2 = ipm.ipm_merge_fused_plan(n, n, "int32")
    try:
        ipm.ipm_set_fused_engine(1)
        e1, f1 = ipm.ipm_merge_fused_plan(n, n, "int32")
    finally:
        ipm.ipm_set_fused_engine(2)
    assert (e1, e2) == (1, 2) and f2 == f1 + 1
    for dt in ("uint64", "int64", "float32", "uint32"):
        assert ipm.ipm_merge_fused_plan(n, n, dt) == (2, f2), dt
    for dt in ("int32", "uint64"):
        for vb in (4, 8):
            assert ipm.ipm_merge_fused_plan(n, n, dt, with_values=vb) == (2, f2), (dt, vb)


@pytest.mark.parametrize("engine", [0, 1])
def test_exchange_engines_match_oracle(ipm, dev, orc, engine):
    """Both exchange executors (all threads in every role; producer warp + consumer
    warps) on rotations of every phase kind (SINGLE, SWAP, PAIR, SHIFT, LS steps) and on
    whole merges (keys and key-value), against the oracle."""
    import torch

    ipm.ipm_set_exchange_engine(engine)
    try:
        for elem, dt in [(4, np.uint32), (8, np.uint64)]:
            for lx, ly in [(1, 1), (5000, 4000), (65_536, 65_536), (1 << 20, (1 << 20) + 77),
                           (3_000_017, 260_001), (260_001, 2_900_011), (1_000_003, 700_001),
                           (700_001, 1_000_003), (4_000_037, 3_700_019), (999_983, 7919)]:
                x = W.make_pair("uniform", dt, lx + ly, 0, seed=lx ^ ly)[0]
                d = to_dev(x, dev)
                ws = ipm.workspace(ipm.ipm_rotate_workspace_bytes(lx, ly, elem), dev)
                ipm.ipm_rotate(d, lx, ly, elem, ws)
                torch.cuda.synchronize()
                assert ipm.ipm_read_device_status(ws) == 0
                assert np.array_equal(bits(from_dev(d, dt)), bits(np.roll(x, -lx))), (lx, ly)
        for dist, dt, la, lb in [("uniform", np.int32, 3_000_017, 2_900_011),
                                 ("dup16", np.uint32, 1_000_003, 700_001),
                                 ("revdisjoint", np.int32, 900_001, 1_200_007),
                                 ("uniform", np.uint64, 1_500_007, 1_400_011)]:
            for fused in (0, 4, 6):
                ipm.ipm_set_fused_levels(fused)
                a, b = W.make_pair(dist, dt, la, lb, seed=la)
                got = _merge_dev(ipm, dev, a, b)
                assert first_diff(got, orc.merge(a, b)) is None, (dist, la, lb, fused)
        ipm.ipm_set_fused_levels(10)
        ka, kb = W.make_pair("zipf", np.uint32, 2_000_003, 1_700_001, seed=3)
        keys = to_dev(np.concatenate([ka, kb]), dev)
        vals = torch.arange(ka.size + kb.size, dtype=torch.int32, device=dev)
        ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(ka.size, kb.size, "uint32", True), dev)
        ipm.ipm_merge_inplace_kv(keys, vals, ka.size, kb.size, "uint32", ws)
        torch.cuda.synchronize()
        assert ipm.ipm_read_device_status(ws) == 0
        wk, wv = orc.merge_kv(ka, np.arange(ka.size, dtype=np.uint32), kb,
                              np.arange(ka.size, ka.size + kb.size, dtype=np.uint32))
        assert np.array_equal(from_dev(keys, np.uint32), wk)
        assert np.array_equal(vals.cpu().numpy().view(np.uint32), wv)
    finally:
        ipm.ipm_set_exchange_engine(1)
        ipm.ipm_set_fused_levels(10)


@pytest.mark.parametrize("engine", [0, 1])
def test_exchange_stress_random_layouts(ipm, dev, orc, engine):
    """Random sizes, skews and pair counts (many small exchanges of every phase kind, in
    every interleaving of tickets across CTAs), both executors, against the oracle's
    arranged layout."""
    import torch

    rng = np.random.default_rng(1234 + engine)
    ipm.ipm_set_exchange_engine(engine)
    try:
        for it in range(24):
            dt = [np.int32, np.uint64][it % 2]
            dist = ["uniform", "dup16", "zipf", "alternation", "revdisjoint"][it % 5]
            if dist == "zipf" and dt == np.int32:
                dist = "uniform"
            la = int(rng.integers(1, 3_000_000))
            lb = int(rng.integers(1, 3_000_000))
            if it % 4 == 0:
                lb = int(rng.integers(1, 2000))  # very unbalanced
            G = int(rng.integers(1, 13))
            a, b = W.make_pair(dist, dt, la, lb, seed=it)
            P = 1 << G
            d = orc.diagonals(la + lb, P)
            i = orc.splits_replay(a, b, d)
            buf = to_dev(np.concatenate([a, b]), dev)
            split = torch.from_numpy(i.astype(np.int64)).to(dev)
            wsG = max(G, ipm.ipm_merge_plan(la, lb, NAME[np.dtype(dt)])[0])
            ws = ipm.workspace(ipm.ipm_merge_workspace_bytes(la, lb, NAME[np.dtype(dt)], False,
                                                             wsG), dev)
            ipm.ipm_merge_rearrange(buf, None, la, lb, NAME[np.dtype(dt)], split, G, ws)
            torch.cuda.synchronize()
            assert ipm.ipm_read_device_status(ws) == 0, (it, la, lb, G)
            want = orc.arrange(a, b, d, i)
            assert first_diff(from_dev(buf, dt), want) is None, (it, dist, la, lb, G)
    finally:
        ipm.ipm_set_exchange_engine(1)
