"""The seeded generators: sorted runs, the promised shapes, numpy == torch bits."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("dist", ["uniform", "dup16", "disjoint", "revdisjoint",
                                  "alternation", "zipf", "paper"])
@pytest.mark.parametrize("dt", [np.int32, np.uint32, np.uint64])
def test_runs_sorted_and_deterministic(dist, dt):
    a, b = W.make_pair(dist, dt, 3000, 1717, seed=5)
    a2, b2 = W.make_pair(dist, dt, 3000, 1717, seed=5)
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert np.all(a[1:] >= a[:-1]) and np.all(b[1:] >= b[:-1])
    assert a.dtype == dt and b.dtype == dt


def test_shapes():
    a, b = W.make_pair("disjoint", np.int32, 5000, 5000, 1)
    assert a.max() < b.min() and a.min() >= 0 and b.max() < 2**31
    a, b = W.make_pair("revdisjoint", np.uint64, 5000, 5000, 1)
    assert b.max() < a.min()
    a, b = W.make_pair("alternation", np.int32, 10, 4, 0)
    assert a.tolist() == list(range(0, 20, 2)) and b.tolist() == [1, 3, 5, 7]
    a, b = W.make_pair("dup16", np.int32, 10000, 10, 0)
    assert set(np.unique(a).tolist()) == set(range(16))
    a, _ = W.make_pair("zipf", np.uint32, 200000, 0, 0)
    assert a.min() == 0 and a.max() < 2**20 and np.mean(a == 0) > 0.15
    a, _ = W.make_pair("gmm", np.float32, 100000, 0, 0)
    assert np.all(np.isfinite(a)) and not np.any(np.signbit(a) & (a == 0))
    a, _ = W.make_pair("paper", np.int32, 1000, 0, 0)
    assert a[0] == 0 and set(np.diff(a).tolist()) <= {0, 1, 2, 3, 4}


@pytest.mark.parametrize("dist,dt", [("uniform", np.int32), ("uniform", np.uint32),
                                     ("uniform", np.uint64), ("dup16", np.int32),
                                     ("disjoint", np.uint64), ("revdisjoint", np.int32),
                                     ("alternation", np.int32), ("uniform", np.float32)])
def test_numpy_and_torch_generators_give_the_same_bits(dist, dt):
    torch = pytest.importorskip("torch")
    ref = W.make_buffer(dist, dt, 4000, 2500, seed=3)
    t = W.make_buffer_torch(torch, dist, dt, 4000, 2500, 3, "cpu")
    assert np.array_equal(W.as_numpy_keys(t, dt).view(np.uint8), ref.view(np.uint8))


def test_batched_lengths_fit_the_cap():
    la, lb, e_max = W.batched_lengths()
    assert la.size == lb.size == 20000
    assert int(la.sum() + lb.sum()) <= 2**28
    assert 15.0 < e_max < 16.5 and la.min() >= 16
    small_a, small_b, _ = W.batched_lengths(nseg=50, total_cap=200000, seed=2)
    buf, offs = W.batched_buffer(small_a, small_b, seed=2)
    for s in range(50):
        o, x, y = int(offs[s]), int(small_a[s]), int(small_b[s])
        assert np.all(np.diff(buf[o:o + x]) >= 0) and np.all(np.diff(buf[o + x:o + x + y]) >= 0)
    torch = pytest.importorskip("torch")
    tb, toffs = W.batched_buffer_torch(torch, small_a, small_b, 2, "cpu")
    assert np.array_equal(tb.numpy(), buf) and np.array_equal(toffs, offs)


def test_split_training_diagonals():
    n = (1 << 29) + 12345
    d = W.split_training_diagonals(n, 4096, seed=0)
    assert d.dtype == np.uint64 and d.size == 4096
    assert np.all(np.diff(d.astype(np.int64)) >= 0) and int(d[-1]) <= n
    assert np.array_equal(d, W.split_training_diagonals(n, 4096, seed=0))
    # the stratified half covers every slice of the range
    hist = np.histogram(d.astype(np.float64), bins=64, range=(0, n))[0]
    assert hist.min() >= 4096 // 2 // 64
    assert W.split_training_diagonals(10, 7, seed=1).max() <= 10
