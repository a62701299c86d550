"""GPU parity of the batched segmented merge (one persistent launch over a segment
table) against the CPU oracle, segment by segment, bit-exact."""
import numpy as np
import pytest

import workloads as W
from gpu_util import NAME, first_diff, from_dev, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.uint64, np.float32, np.int64]
OPTIONS = [None, {"tile": 1}, {"tile": 3}, {"order": 1},
           {"tile": 2, "ctas_per_sm": 1, "order": 1},
           # the one-launch form (memset node + one persistent kernel)
           {"form": 2}, {"form": 2, "tile": 1}, {"form": 2, "tile": 3, "order": 1},
           {"form": 2, "tile": 2, "ctas_per_sm": 1}]


def _table(dt, tile, seed, kv=False):
    """Segments of every kind at odd offsets with untouched gaps between them:
    empty sides, tiny, one tile, just above one tile, several tiles, early exit
    (disjoint), reverse-disjoint, duplicates."""
    rng = np.random.default_rng(seed)
    dists = ["uniform", "dup16", "disjoint", "revdisjoint", "uniform", "dup16"]
    sizes = [(0, 0), (0, 5), (7, 0), (1, 1), (3, 2), (100, 37), (tile // 2, tile // 2),
             (tile // 2 + 1, tile // 2), (tile, 1), (1, tile), (tile + 3, tile - 5),
             (2 * tile + 11, tile + 2), (3 * tile, 2 * tile + 9), (5 * tile + 1, 17),
             (17, 4 * tile + 3)]
    sizes += [(int(x), int(y)) for x, y in rng.integers(0, 3 * tile, size=(12, 2))]
    parts, segs, want = [], [], []
    pos = 0
    for t, (la, lb) in enumerate(sizes):
        gap = int(rng.integers(0, 9))
        g = W.make_pair("uniform", dt, gap, 0, seed=900 + t)[0]
        parts.append(g)
        pos += gap
        a, b = W.make_pair(dists[t % len(dists)], dt, la, lb, seed=seed * 1000 + t)
        parts += [a, b]
        segs.append((pos, la, lb))
        pos += la + lb
    tail = W.make_pair("uniform", dt, 5, 0, seed=1)[0]
    parts.append(tail)
    buf = np.concatenate(parts)
    return buf, segs


def _expected(orc, buf, segs, vals=None):
    out = buf.copy()
    vout = None if vals is None else vals.copy()
    for off, la, lb in segs:
        a, b = buf[off:off + la], buf[off + la:off + la + lb]
        if vals is None:
            out[off:off + la + lb] = orc.merge(a, b)
        else:
            k, v = orc.merge_kv(a, vals[off:off + la], b, vals[off + la:off + la + lb])
            out[off:off + la + lb] = k
            vout[off:off + la + lb] = v
    return out, vout


def _run(ipm, dev, buf, segs, dt, vals=None, options=None):
    import torch

    d = to_dev(buf, dev)
    dv = None if vals is None else torch.from_numpy(vals.view(np.int32).copy()).to(dev)
    st = ipm.segment_table([s[0] for s in segs], [s[1] for s in segs], [s[2] for s in segs],
                           dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(
        buf.size, len(segs), NAME[np.dtype(dt)], vals is not None, options), dev)
    ipm.ipm_merge_batched(d, dv, buf.size, st, len(segs), NAME[np.dtype(dt)], ws,
                          options=options)
    torch.cuda.synchronize()
    status = ipm.ipm_read_device_status(ws)
    got = from_dev(d, dt)
    gv = None if dv is None else dv.cpu().numpy().view(np.uint32)
    return got, gv, status, ws


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("opt", range(len(OPTIONS)))
def test_batched_keys_match_oracle(ipm, dev, orc, dt, opt):
    options = OPTIONS[opt]
    tile = ipm.ipm_merge_plan(1, 1, NAME[np.dtype(dt)])[1]
    buf, segs = _table(dt, tile, seed=3 + opt)
    want, _ = _expected(orc, buf, segs)
    got, _, status, _ = _run(ipm, dev, buf, segs, dt, options=options)
    assert status == 0
    assert first_diff(got, want) is None, first_diff(got, want)


@pytest.mark.parametrize("dt", [np.uint32, np.uint64, np.float32, np.int64])
@pytest.mark.parametrize("opt", [0, 1, 2, 5, 7])
def test_batched_kv_stable(ipm, dev, orc, dt, opt):
    tile = ipm.ipm_merge_plan(1, 1, NAME[np.dtype(dt)], True)[1]
    buf, segs = _table(dt, tile, seed=11 + opt)
    vals = np.arange(buf.size, dtype=np.uint32)
    want, wv = _expected(orc, buf, segs, vals)
    got, gv, status, _ = _run(ipm, dev, buf, segs, dt, vals=vals, options=OPTIONS[opt])
    assert status == 0
    assert first_diff(got, want) is None
    assert np.array_equal(gv, wv)


@pytest.mark.parametrize("opt", range(len(OPTIONS)))
def test_batched_sizes_around_the_tile(ipm, dev, orc, opt):
    """Segment lengths straddling the merge tile in random order: the ones just above
    it need splits and an exchange level, the ones at or below it do not."""
    options = OPTIONS[opt]
    dt = np.int32
    tile = ipm.ipm_merge_batched_max_segment("int32", options=options) // 512
    rng = np.random.default_rng(40 + opt)
    parts, segs, pos = [], [], 0
    for t in range(300):
        n = int(tile + rng.integers(-40, 41))
        la = int(rng.integers(1, n))
        a, b = W.make_pair("uniform", dt, la, n - la, seed=7000 + t)
        parts += [a, b]
        segs.append((pos, la, n - la))
        pos += n
    buf = np.concatenate(parts)
    want, _ = _expected(orc, buf, segs)
    got, _, status, _ = _run(ipm, dev, buf, segs, dt, options=options)
    assert status == 0
    assert first_diff(got, want) is None


@pytest.mark.parametrize("form", [1, 2])
def test_batched_bad_segments_are_skipped(ipm, dev, orc, form):
    """A segment that leaves the buffer or exceeds the per-segment limit is left
    untouched and flagged; the valid segments are still merged."""
    dt = np.int32
    lim = ipm.ipm_merge_batched_max_segment("int32", options={"tile": 2})
    a, b = W.make_pair("uniform", dt, 1000, 999, seed=5)
    big_a, big_b = W.make_pair("uniform", dt, lim // 2 + 1, lim // 2 + 1, seed=6)
    buf = np.concatenate([a, b, big_a, big_b])
    n = buf.size
    segs = [(0, 1000, 999), (1999, big_a.size, big_b.size), (n - 10, 8, 8),
            (2**62, 1, 1), (0, 2**62, 2**62)]
    got, _, status, _ = _run(ipm, dev, buf, segs, dt, options={"tile": 2, "form": form})
    assert status == 1  # IPM_ERR_INVALID_ARG
    want = buf.copy()
    want[:1999] = orc.merge(a, b)
    assert first_diff(got, want) is None


@pytest.mark.parametrize("form", [1, 2])
def test_batched_merge_bytes(ipm, dev, orc, form):
    """Single-tile segments: a merged segment moves 2n elements, one whose runs are
    already in order is read once (n) and not written, one with an empty run is not
    touched."""
    dt = np.int32
    tile = ipm.ipm_merge_plan(1, 1, "int32")[1]
    buf, segs = _table(dt, tile, seed=21)
    segs = [s for s in segs if s[1] + s[2] <= tile]
    _, _, status, ws = _run(ipm, dev, buf, segs, dt, options={"form": form})
    assert status == 0
    want = 0
    for off, la, lb in segs:
        if la and lb:
            want += (2 if buf[off + la - 1] > buf[off + la] else 1) * (la + lb) * 4
    assert ipm.ipm_read_merge_bytes(ws) == want


@pytest.mark.parametrize("form", [1, 2])
def test_batched_graph_capture(ipm, dev, orc, form):
    """The call captures into a CUDA graph; replays merge the restored input again."""
    import torch

    opts = {"form": form}
    dt = np.int32
    tile = ipm.ipm_merge_plan(1, 1, "int32")[1]
    buf, segs = _table(dt, tile, seed=31)
    want, _ = _expected(orc, buf, segs)
    pristine = to_dev(buf, dev)
    d = pristine.clone()
    st = ipm.segment_table([s[0] for s in segs], [s[1] for s in segs], [s[2] for s in segs],
                           dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(buf.size, len(segs), "int32"), dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture (first-call attribute setup)
        ipm.ipm_merge_batched(d, None, buf.size, st, len(segs), "int32", ws, options=opts,
                              stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ipm.ipm_merge_batched(d, None, buf.size, st, len(segs), "int32", ws, options=opts,
                              stream=s)
    for _ in range(2):
        d.copy_(pristine)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert ipm.ipm_read_device_status(ws) == 0
        assert first_diff(from_dev(d, dt), want) is None


@pytest.mark.slow
@pytest.mark.parametrize("opt", [0, 1, 2, 5])
def test_batched_fullsize_20000_segments(ipm, dev, orc, opt):
    """20,000 uniform int32 segments, log-uniform side lengths, total <= 2^28."""
    import torch

    la, lb, _ = W.batched_lengths()
    d, offs = W.batched_buffer_torch(torch, la, lb, seed=0, device=dev)
    host = from_dev(d, np.int32)
    st = ipm.segment_table(offs.astype(np.int64), la, lb, dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(d.numel(), la.size, "int32",
                                                             False, OPTIONS[opt]), dev)
    ipm.ipm_merge_batched(d, None, d.numel(), st, la.size, "int32", ws, options=OPTIONS[opt])
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    got = from_dev(d, np.int32)
    for s in range(la.size):
        o, x, y = int(offs[s]), int(la[s]), int(lb[s])
        want = orc.merge(host[o:o + x], host[o + x:o + x + y])
        assert first_diff(got[o:o + x + y], want) is None, s


@pytest.mark.parametrize("kv", [False, True])
def test_autotuned_options_match_oracle(ipm, dev, orc, kv, tmp_path):
    """The autotuner times every candidate option set on a scratch copy (the input is
    only read), picks one, caches it; a merge with the pick equals the oracle segment
    by segment, and a second tuning call is answered from the cache."""
    import torch

    la, lb, _ = W.batched_lengths(nseg=600, total_cap=1 << 23, seed=4)
    buf, offs = W.batched_buffer(la, lb, seed=4)
    segs = list(zip(offs.tolist(), la.tolist(), lb.tolist()))
    vals = np.arange(buf.size, dtype=np.uint32) if kv else None
    d = to_dev(buf, dev)
    dv = None if vals is None else torch.from_numpy(vals.view(np.int32).copy()).to(dev)
    scratch = torch.empty_like(d)
    svals = None if dv is None else torch.empty_like(dv)
    st = ipm.segment_table(offs.astype(np.int64), la, lb, dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_tune_workspace_bytes(buf.size, len(segs), "int32",
                                                                  kv), dev)
    cache = str(tmp_path / "tune.txt")
    res = ipm.ipm_merge_batched_tune(d, dv, buf.size, st, len(segs), "int32", scratch, ws,
                                     scratch_vals=svals, reps=3, cache_path=cache)
    assert not res["from_cache"] and res["candidates"] >= 16
    assert {e["form"] for e in res["table"]} == {1, 2}
    assert res["best_ms"] > 0 and res["default_ms"] > 0
    assert res["best_ms"] <= min(e["ms"] for e in res["table"]) + 1e-6
    torch.cuda.synchronize()
    assert torch.equal(d, to_dev(buf, dev))  # the input was only read
    want, wv = _expected(orc, buf, segs, vals)
    # the scratch copy holds the last candidate's merge: already the right answer
    assert np.array_equal(from_dev(scratch, np.int32), want)
    got, gv, status, _ = _run(ipm, dev, buf, segs, np.int32, vals, options=res["best"])
    assert status == 0
    assert first_diff(got, want) is None
    if kv:
        assert np.array_equal(gv, wv)
    again = ipm.ipm_merge_batched_tune(d, dv, buf.size, st, len(segs), "int32", scratch, ws,
                                       scratch_vals=svals, reps=3, cache_path=cache)
    assert again["from_cache"] and again["best"] == res["best"]
    assert again["signature"] == res["signature"]


@pytest.mark.parametrize("form", [0, 2])
def test_batched_many_segments_prepare_in_many_chunks(ipm, dev, orc, form):
    """400,040 segments: the size-ordered queue is prepared in more chunks (of 2,048
    descriptors) than there are SMs, so every preparation CTA takes several chunks
    (bucket counts, then scatter), and the multi-tile segments scattered among them
    must still lead the queue.  Small segments with many equal keys, 40 segments of
    two to four tiles at random places in the table; every segment against the
    oracle."""
    import torch

    rng = np.random.default_rng(11)
    nsmall, nbig = 400_000, 40
    _, tile = ipm.ipm_merge_plan(1, 1, "int32")
    la = rng.integers(0, 49, nsmall + nbig)
    lb = rng.integers(0, 49, nsmall + nbig)
    big = rng.choice(nsmall + nbig, nbig, replace=False)
    la[big] = rng.integers(tile // 2, 2 * tile, nbig)
    lb[big] = rng.integers(tile // 2, 2 * tile, nbig)
    runs = np.stack([la, lb], 1).ravel()
    run_id = np.repeat(np.arange(runs.size), runs)
    keys = rng.integers(-1000, 1000, run_id.size).astype(np.int32)
    host = keys[np.lexsort((keys, run_id))]  # every run sorted, runs in table order
    offs = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.int64)
    d = to_dev(host, dev)
    opts = OPTIONS[5] if form == 2 else None
    st = ipm.segment_table(offs, la, lb, dev)
    ws = ipm.workspace(ipm.ipm_merge_batched_workspace_bytes(host.size, la.size, "int32",
                                                             False, opts), dev)
    ipm.ipm_merge_batched(d, None, host.size, st, la.size, "int32", ws, options=opts)
    torch.cuda.synchronize()
    assert ipm.ipm_read_device_status(ws) == 0
    got = from_dev(d, np.int32)
    for s in range(la.size):
        o, x, y = int(offs[s]), int(la[s]), int(lb[s])
        want = orc.merge(host[o:o + x], host[o + x:o + x + y])
        assert first_diff(got[o:o + x + y], want) is None, s
