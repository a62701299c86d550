"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expectation comes from brute force
over all interleavings, a library routine that computes the same thing a different way
(Python's stable sort, numpy.roll, math.gcd, finite differences), a closed form stated
in the paper, or a hand-traced example.
"""
import itertools
import math
import random

import numpy as np
import pytest

import workloads

DTYPES = [np.int32, np.uint32, np.uint64, np.float32, np.int64]


def library_stable_merge(a, b):
    """Stable merge by sorting (key, origin, index) with Python's stable sort."""
    items = [(x, 0, i) for i, x in enumerate(a.tolist())] + \
            [(x, 1, j) for j, x in enumerate(b.tolist())]
    return sorted(items, key=lambda t: (t[0], t[1], t[2]))


def interleavings(c, la):
    """All ways to draw a sorted A of la elements from the sorted sequence c."""
    n = len(c)
    for pos in itertools.combinations(range(n), la):
        s = set(pos)
        yield c[list(pos)], c[[t for t in range(n) if t not in s]]


def _bits(x):
    return x.view({4: np.uint32, 8: np.uint64}[x.dtype.itemsize])


@pytest.mark.parametrize("alphabet", [1, 2, 4, None])
def test_merge_brute_force_all_interleavings(orc, alphabet):
    rng = np.random.default_rng(11)
    for n in range(0, 11):
        hi = alphabet if alphabet else 10_000
        c = np.sort(rng.integers(0, hi, n)).astype(np.int32)
        for la in range(n + 1):
            for a, b in interleavings(c, la):
                exp = library_stable_merge(a, b)
                got = orc.merge(a, b)
                assert got.tolist() == [t[0] for t in exp]
                va = np.arange(a.size, dtype=np.uint32)
                vb = np.arange(a.size, a.size + b.size, dtype=np.uint32)
                k, v = orc.merge_kv(a, va, b, vb)
                assert v.tolist() == [t[2] + (a.size if t[1] else 0) for t in exp]
                # split on every diagonal: number of A-origin items among the first d
                d = np.arange(n + 1, dtype=np.uint64)
                want = np.cumsum([0] + [1 - t[1] for t in exp])
                assert orc.splits_replay(a, b, d).tolist() == want.tolist()
                for dd in range(n + 1):
                    assert orc.split_bsearch(a, b, dd) == want[dd]


@pytest.mark.parametrize("dt", DTYPES)
def test_merge_random_all_dtypes(orc, dt):
    rng = random.Random(5)
    negatives = 0
    for _ in range(60):
        la, lb = rng.randint(0, 300), rng.randint(0, 300)
        for dist in ("uniform", "dup16"):
            a, b = workloads.make_pair(dist, dt, la, lb, seed=rng.randint(0, 10**6))
            negatives += int((a < 0).sum() + (b < 0).sum())
            exp = library_stable_merge(a, b)
            got = orc.merge(a, b)
            assert got.tolist() == [t[0] for t in exp]
    if dt == np.int64:
        # the signed instantiation must see keys on both sides of zero: an unsigned
        # comparison would order every negative key after the positive ones
        assert negatives > 1000


def test_merge_brute_force_int64_across_zero(orc):
    """Every interleaving of keys that straddle zero and both ends of the int64 range:
    the signed 64-bit instantiation must order them as Python's integers do."""
    c = np.array([-2**63, -2**40, -7, -1, -1, 0, 3, 2**40, 2**63 - 1], dtype=np.int64)
    for la in range(c.size + 1):
        for a, b in interleavings(c, la):
            exp = library_stable_merge(a, b)
            assert orc.merge(a, b).tolist() == [t[0] for t in exp]
            d = np.arange(c.size + 1, dtype=np.uint64)
            want = np.cumsum([0] + [1 - t[1] for t in exp])
            assert orc.splits_replay(a, b, d).tolist() == want.tolist()
            va = np.arange(a.size, dtype=np.uint32)
            vb = np.arange(a.size, a.size + b.size, dtype=np.uint32)
            _, v = orc.merge_kv(a, va, b, vb)
            assert v.tolist() == [t[2] + (a.size if t[1] else 0) for t in exp]


def test_float_signed_zero_ties_keep_input_order(orc):
    # -0.0 == +0.0 under "<=": stability decides, so bit patterns follow the origin
    a = np.array([-1.0, -0.0, 0.0, 2.0], dtype=np.float32)
    b = np.array([0.0, -0.0, 1.0], dtype=np.float32)
    got = orc.merge(a, b)
    want = np.array([-1.0, -0.0, 0.0, 0.0, -0.0, 1.0, 2.0], dtype=np.float32)
    assert np.array_equal(_bits(got), _bits(want))


def test_uint64_full_range(orc):
    a = np.array([0, 1, 2**63 - 1, 2**63, 2**64 - 1], dtype=np.uint64)
    b = np.array([2**63 - 2, 2**63, 2**64 - 2], dtype=np.uint64)
    assert orc.merge(a, b).tolist() == sorted(a.tolist() + b.tolist())


def test_split_forms_agree_and_balance(orc):
    rng = random.Random(9)
    for _ in range(40):
        la, lb = rng.randint(0, 2000), rng.randint(0, 2000)
        a, b = workloads.make_pair(rng.choice(["uniform", "dup16", "zipf"]), np.uint32, la,
                                   lb, seed=rng.randint(0, 999))
        P = rng.choice([1, 2, 3, 7, 16, 64])
        d = orc.diagonals(la + lb, P)
        rep = orc.splits_replay(a, b, d)
        for k in range(P + 1):
            assert orc.split_bsearch(a, b, int(d[k])) == rep[k]
        sizes = np.diff(d.astype(np.int64))
        n = la + lb
        assert set(sizes.tolist()) <= {n // P, -(-n // P)}
        # the pairs, merged one by one and concatenated, give the global merge
        out = []
        for k in range(P):
            i0, i1 = int(rep[k]), int(rep[k + 1])
            j0, j1 = int(d[k]) - i0, int(d[k + 1]) - i1
            out.append(orc.merge(a[i0:i1], b[j0:j1]))
        assert np.array_equal(np.concatenate(out) if out else a[:0], orc.merge(a, b))


def test_arrange_is_pairs_back_to_back(orc):
    a, b = workloads.make_pair("uniform", np.int32, 1000, 777, seed=1)
    d = orc.diagonals(1777, 8)
    i = orc.splits_replay(a, b, d)
    arr = orc.arrange(a, b, d, i)
    for k in range(8):
        i0, i1, j0, j1 = int(i[k]), int(i[k + 1]), int(d[k] - i[k]), int(d[k + 1] - i[k + 1])
        seg = arr[int(d[k]):int(d[k + 1])]
        assert np.array_equal(seg, np.concatenate([a[i0:i1], b[j0:j1]]))


def test_arrange_of_any_valid_table_is_a_permutation_into_pairs(orc):
    """The layout of an arbitrary table (not a merge's), for keys and 8-byte payloads:
    pair k holds A[i_k, i_{k+1}) then B[j_k, j_{k+1}), and the result is a permutation
    of A|B (every index appears once)."""
    rng = np.random.default_rng(4)
    for la, lb, P in [(1000, 777, 16), (5, 300, 8), (300, 5, 8), (64, 64, 32), (3, 2, 8)]:
        n = la + lb
        d = orc.diagonals(n, P)
        i = [0] * (P + 1)
        i[P] = la
        for k in range(1, P):
            dk, dp = int(d[k]), int(d[k - 1])
            lo = max(i[k - 1], dk - lb, la - (n - dk))
            hi = min(la, dk, i[k - 1] + (dk - dp))
            i[k] = int(rng.integers(lo, hi + 1)) if hi > lo else lo
        i = np.array(i, dtype=np.uint64)
        idx = np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        arr = orc.arrange(idx[:la], idx[la:], d, i)
        assert np.array_equal(np.sort(arr), np.sort(idx))
        for k in range(P):
            i0, i1 = int(i[k]), int(i[k + 1])
            j0, j1 = int(d[k]) - i0, int(d[k + 1]) - i1
            seg = arr[int(d[k]):int(d[k + 1])]
            assert np.array_equal(seg, np.concatenate([idx[i0:i1], idx[la + j0:la + j1]]))


def test_gallop_equals_bsearch_for_every_guess(orc):
    rng = random.Random(2)
    for _ in range(30):
        la, lb = rng.randint(0, 70), rng.randint(0, 70)
        a, b = workloads.make_pair(rng.choice(["uniform", "dup16"]), np.int32, la, lb,
                                   seed=rng.randint(0, 999))
        for d in range(la + lb + 1):
            want = orc.split_bsearch(a, b, d)
            for g in range(-2, la + 3):
                i, probes = orc.gallop_split(a, b, d, max(g, 0))
                assert i == want
                dist = abs(want - max(0, min(g, la)))
                # exponential bracket + bisection: O(log distance) probes
                assert probes <= 2 * math.ceil(math.log2(dist + 1)) + 3


def test_ls_rotate_equals_roll_and_paper_counts(orc):
    for lx in range(0, 14):
        for ly in range(0, 14):
            x = np.arange(lx + ly, dtype=np.int32)
            got, swaps = orc.ls_rotate(x, lx)
            assert np.array_equal(got, np.roll(x, -lx))
            if lx == ly:
                assert swaps == lx  # Sec. 3.5: exactly L_A swaps for equal blocks
            assert swaps <= 2 * (lx + ly)  # Sec. 3.5 bound
    x = np.arange(10**5 + 7, dtype=np.uint64)
    got, swaps = orc.ls_rotate(x, 7)
    assert np.array_equal(got, np.roll(x, -7))


def test_ls_hand_traced_example(orc):
    # Sec. 3.4 LS on X=[0,1], Y=[2,3,4,5,6], traced by hand:
    # swap X with Y's last 2 -> [5,6,2,3,4,0,1]; rotate [5,6|2,3,4]: swap [5,6] with
    # [3,4] -> [3,4,2,5,6]; rotate [3,4|2]: Y smaller, swap 2 with 3 -> [2,4,3];
    # rotate [4|3]: equal, swap -> [3,4].  6 elementary swaps.
    got, swaps = orc.ls_rotate(np.array([0, 1, 2, 3, 4, 5, 6], dtype=np.int32), 2)
    assert got.tolist() == [2, 3, 4, 5, 6, 0, 1]
    assert swaps == 6


def test_cs_rotate_gcd_cycles_and_exact_moves(orc):
    for la in range(0, 16):
        for lb in range(0, 16):
            x = np.arange(la + lb, dtype=np.int32)
            got, cycles, moves = orc.cs_rotate(x, la)
            assert np.array_equal(got, np.roll(x, -la))
            if la and lb:
                assert cycles == math.gcd(la, lb)  # proof of Sec. 3.4 (GCD, not LCM)
                assert moves == la + lb           # Sec. 3.5: exactly L_A + L_B moves
            else:
                assert cycles == 0 and moves == 0


def _valid_split(a, b, pa, pb):
    la, lb = len(a), len(b)
    return (pa == 0 or pb == lb or a[pa - 1] <= b[pb]) and \
        (pb == 0 or pa == la or b[pb - 1] <= a[pa])


def test_findmedian_corner_cases(orc):
    a = np.array([1, 2, 3], np.int32)
    b = np.array([3, 4], np.int32)
    assert orc.findmedian(a, b) == (3, 0)             # A <= B
    assert orc.findmedian(b + 10, a) == (0, 3)        # A > B
    assert orc.findmedian(a[:0], b) == (0, 0)         # |A| = 0
    assert orc.findmedian(a, b[:0]) == (3, 0)         # |B| = 0


def _findmedian_literal(A, B):
    """Alg. 1 taken literally: p_A, p_B start at the middles (the text's first step),
    the loop test uses the previous iteration's values, and the midpoints are
    recomputed after the loop."""
    la, lb = len(A), len(B)
    if la == 0 or lb == 0 or A[-1] <= B[0]:
        return la, 0
    if not A[0] <= B[-1]:
        return 0, lb
    lA, limA, lB, limB = 0, la, 0, lb
    pA, pB = la // 2, lb // 2
    while lA < limA and lB < limB and A[pA] != B[pB]:
        pA, pB = (limA - lA) // 2 + lA, (limB - lB) // 2 + lB
        if A[pA] < B[pB]:
            if pA + pB < (la - pA) + (lb - pB):
                lA = pA + 1
            else:
                limB = pB
        else:
            if pA + pB < (la - pA) + (lb - pB):
                lB = pB + 1
            else:
                limA = pA
    return (limA - lA) // 2 + lA, (limB - lB) // 2 + lB


def test_findmedian_reading_is_valid_where_literal_is_not(orc):
    # The literal listing returns an invalid split here (B0 holds 4 > A1[0] = 3);
    # the reading used by the oracle returns a valid one.
    A = [1, 3, 3, 4, 5, 7, 7, 9]
    B = [0, 0, 0, 1, 4, 5, 6, 7, 9]
    assert _findmedian_literal(A, B) == (2, 5)
    assert not _valid_split(A, B, 2, 5)
    pa, pb = orc.findmedian(np.array(A, np.int32), np.array(B, np.int32))
    assert _valid_split(A, B, pa, pb)
    rng = random.Random(1)
    for _ in range(20000):
        la, lb, m = rng.randint(0, 12), rng.randint(0, 12), rng.choice([3, 10, 1000])
        A = sorted(rng.randrange(m) for _ in range(la))
        B = sorted(rng.randrange(m) for _ in range(lb))
        pa, pb = orc.findmedian(np.array(A, np.int32), np.array(B, np.int32))
        assert 0 <= pa <= la and 0 <= pb <= lb
        assert _valid_split(A, B, pa, pb)


def test_findmedian_is_not_stable_under_ties(orc):
    # Even a valid FindMedian split can put a B key equal to A1[0] into B0, so equal
    # keys would interleave B-then-A across pairs; the hot path uses the stable split.
    a, b = np.array([3, 5, 5, 8], np.int32), np.array([1, 5, 5, 9], np.int32)
    pa, pb = orc.findmedian(a, b)
    assert (pa, pb) == (2, 2)
    assert b[pb - 1] == a[pa]  # B0 ends with 5 == A1[0]: not the stable split
    assert orc.split_bsearch(a, b, pa + pb) == 3


@pytest.mark.parametrize("shift", ["ls", "cs"])
@pytest.mark.parametrize("split", ["exact", "findmedian"])
def test_srecpar_gives_the_merge(orc, shift, split):
    rng = random.Random(3)
    for _ in range(80):
        la, lb = rng.randint(0, 400), rng.randint(0, 400)
        a, b = workloads.make_pair(rng.choice(["uniform", "dup16", "paper"]), np.int32, la,
                                   lb, seed=rng.randint(0, 999))
        buf = np.concatenate([a, b])
        depth = rng.randint(0, 5)
        got, moved = orc.srecpar(buf, la, depth, size_limit=rng.choice([1, 16]),
                                 split=split, shift=shift)
        assert np.array_equal(got, orc.merge(a, b))


def test_srecpar_exact_is_stable_with_payload_order(orc):
    # with exact splits the division stage keeps A before B on ties: check with keys
    # that carry their origin in the low bits
    rng = np.random.default_rng(4)
    k = np.sort(rng.integers(0, 8, 300)) * 1024
    a = np.sort(k[:170] + np.arange(170)).astype(np.int32)
    b = np.sort(k[170:] + 512 + np.arange(130)).astype(np.int32)
    got, _ = orc.srecpar(np.concatenate([a, b]), 170, 4)
    assert np.array_equal(got, np.sort(np.concatenate([a, b])))


def test_mlp_forward_closed_forms(orc):
    H = 4
    rng = np.random.default_rng(0)
    x = rng.random(9)
    p = rng.normal(size=3 * H + 1)
    p[:H] = 0.0  # w1 = 0: y = b2 + sum_h w2 tanh(b1)
    y = orc.mlp_forward(p, H, x)
    want = p[3 * H] + sum(p[2 * H + h] * math.tanh(p[H + h]) for h in range(H))
    assert np.allclose(y, want, rtol=0, atol=1e-14)
    q = np.array([0.7, -0.2, 1.5, 0.3])  # H = 1
    y = orc.mlp_forward(q, 1, x)
    assert np.allclose(y, [0.3 + 1.5 * math.tanh(0.7 * t - 0.2) for t in x], rtol=0,
                       atol=1e-14)


def test_mlp_gradient_matches_central_differences(orc):
    H = 32
    rng = np.random.default_rng(1)
    x, t = rng.random(50), rng.random(50)
    p = rng.normal(scale=0.7, size=3 * H + 1)
    loss, g = orc.mlp_loss_grad(p, H, x, t)
    y = orc.mlp_forward(p, H, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)
    h = 1e-6
    for q in range(3 * H + 1):
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (orc.mlp_loss_grad(pp, H, x, t)[0] - orc.mlp_loss_grad(pm, H, x, t)[0]) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # targets equal to the outputs: zero loss, zero gradient
    l0, g0 = orc.mlp_loss_grad(p, H, x, y)
    assert l0 < 1e-28 and np.abs(g0).max() < 1e-14


def test_adam_first_step_closed_form(orc):
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    lr, eps = 0.01, 1e-8
    p0 = p.copy()
    orc.adam_step(p, m, v, g, lr, 0.9, 0.999, eps, 1)
    # first step: mhat = g, vhat = g^2  ->  p - lr * g / (|g| + eps)
    assert np.allclose(p, p0 - lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)


def test_adam_three_steps_worked_by_hand(orc):
    """Steps 1-3 of Adam with beta1 = 1/2, beta2 = 3/4, lr = 1, eps = 0, worked out by
    hand.  Bias corrections: 1 - beta1^t = 1/2, 3/4, 7/8 and 1 - beta2^t = 1/4, 7/16,
    37/64.

    Coordinate 0, gradients 2, -2, 2:
      t=1  m = 1,    v = 1      mhat = 2,    vhat = 4  -> step  1
      t=2  m = -1/2, v = 7/4    mhat = -2/3, vhat = 4  -> step -1/3
      t=3  m = 3/4,  v = 37/16  mhat = 6/7,  vhat = 4  -> step  3/7
    Coordinate 1, gradients 1, 3, 0:
      t=1  m = 1/2,  v = 1/4    mhat = 1,    vhat = 1      -> step 1
      t=2  m = 7/4,  v = 39/16  mhat = 7/3,  vhat = 39/7   -> step (7/3) / sqrt(39/7)
      t=3  m = 7/8,  v = 117/64 mhat = 1,    vhat = 117/37 -> step 1 / sqrt(117/37)
    A first moment that forgets its history (m = (1 - beta1) g), a second moment that
    does, or a step count stuck at 1 changes every step after the first."""
    p = np.array([10.0, 10.0])
    m, v = np.zeros(2), np.zeros(2)
    grads = [np.array([2.0, 1.0]), np.array([-2.0, 3.0]), np.array([2.0, 0.0])]
    want = [np.array([9.0, 9.0]),
            np.array([9.0 + 1.0 / 3.0, 9.0 - (7.0 / 3.0) / math.sqrt(39.0 / 7.0)]),
            np.array([9.0 + 1.0 / 3.0 - 3.0 / 7.0,
                      9.0 - (7.0 / 3.0) / math.sqrt(39.0 / 7.0) - 1.0 / math.sqrt(117.0 / 37.0)])]
    want_m = [np.array([1.0, 0.5]), np.array([-0.5, 1.75]), np.array([0.75, 0.875])]
    want_v = [np.array([1.0, 0.25]), np.array([1.75, 39.0 / 16.0]),
              np.array([37.0 / 16.0, 117.0 / 64.0])]
    for t in range(3):
        orc.adam_step(p, m, v, grads[t], 1.0, 0.5, 0.75, 0.0, t + 1)
        assert np.allclose(m, want_m[t], rtol=1e-15, atol=0)
        assert np.allclose(v, want_v[t], rtol=1e-15, atol=0)
        assert np.allclose(p, want[t], rtol=1e-14, atol=0)


# ------------------------------------------------- division balance (Sec. 4, E1)

def _halving_sizes(n, depth):
    """Sizes after depth levels of cutting every region at floor(c/2)."""
    sizes = [n]
    for _ in range(depth):
        sizes = [s for c in sizes for s in (c // 2, c - c // 2)]
    return sizes


@pytest.mark.parametrize("depth", [1, 2, 3, 5])
def test_division_exact_halves_every_region(orc, depth):
    """When no region runs out of one side, the exact split cuts each region at its half
    diagonal: the pair sizes are the recursive floor / ceil halves of n."""
    for la, lb in [(1000, 1000), (1000, 999), (4096, 4095), (2048, 2049)]:
        a = np.arange(la, dtype=np.int64).astype(np.int32) * 2
        b = np.arange(lb, dtype=np.int64).astype(np.int32) * 2 + 1
        ia, jb = orc.division(a, b, depth, "exact")
        sizes = (np.diff(ia.astype(np.int64)) + np.diff(jb.astype(np.int64))).tolist()
        assert sizes == _halving_sizes(la + lb, depth)


@pytest.mark.parametrize("split", ["exact", "findmedian"])
def test_division_is_a_partition_of_the_merge(orc, split):
    """Brute force on small runs with many ties: every division yields pairs whose
    separate merges, concatenated, are the sorted whole (the exact split also keeps the
    stable order of equal keys)."""
    rng = random.Random(17)
    for _ in range(300):
        la, lb = rng.randint(0, 40), rng.randint(0, 40)
        a, b = workloads.make_pair(rng.choice(["dup16", "uniform", "paper"]), np.int32, la,
                                   lb, seed=rng.randint(0, 9999))
        depth = rng.randint(1, 4)
        ia, jb = orc.division(a, b, depth, split)
        assert ia[0] == 0 and jb[0] == 0 and ia[-1] == la and jb[-1] == lb
        assert np.all(np.diff(ia.astype(np.int64)) >= 0)
        assert np.all(np.diff(jb.astype(np.int64)) >= 0)
        # keys with their origin (0 = A, 1 = B) and index: the stable merge order
        ka = [(int(x), 0, i) for i, x in enumerate(a)]
        kb = [(int(x), 1, j) for j, x in enumerate(b)]
        out = []
        for k in range(len(ia) - 1):
            part = ka[int(ia[k]):int(ia[k + 1])] + kb[int(jb[k]):int(jb[k + 1])]
            out += sorted(part)  # (key, origin, index): a tie takes A, then index order
        keys = [t[0] for t in out]
        assert keys == sorted(keys)
        if split == "exact":
            assert out == sorted(ka + kb)


def test_division_stops_at_one_sided_regions(orc):
    # A entirely below B: FindMedian's first corner case gives (|A|, 0); each side is
    # then whole in one region and the deeper levels leave it as it is
    a = np.arange(10, dtype=np.int32)
    b = np.arange(10, 30, dtype=np.int32)
    ia, jb = orc.division(a, b, 3, "findmedian")
    na, nb = np.diff(ia.astype(np.int64)), np.diff(jb.astype(np.int64))
    assert sorted((na + nb).tolist(), reverse=True)[:2] == [20, 10]
    assert not np.any((na > 0) & (nb > 0))
    assert orc.division_balance(ia, jb) == (0, 20)
    # depth 1 is one call of FindMedian
    for seed in range(20):
        a, b = workloads.make_pair("paper", np.int32, 300 + seed, 500, seed=seed)
        ia, jb = orc.division(a, b, 1, "findmedian")
        assert (int(ia[1]), int(jb[1])) == orc.findmedian(a, b)


def test_division_findmedian_close_to_exact_on_the_paper_workload(orc):
    """Sec. 4 reports the FindMedian division as close to the optimal one on its
    workload, sometimes better (one-sided regions need no merge); under this reading the
    largest pair that needs a merge differs by a relative 5e-3 at most, either way, for
    T = 2..16 and the three split points."""
    n = 1 << 16
    for frac in (0.25, 0.5, 0.75):
        la = int(n * frac)
        a, b = workloads.make_pair("paper", np.int32, la, n - la, seed=4)
        for depth in (1, 2, 3, 4):
            fm = orc.division_balance(*orc.division(a, b, depth, "findmedian"))[0]
            ex = orc.division_balance(*orc.division(a, b, depth, "exact"))[0]
            assert ex > 0 and abs(fm - ex) / ex < 5e-3, (frac, depth, fm, ex)


def test_merge_kvw_moves_wide_payloads_as_the_4_byte_form(orc):
    """A payload of any width follows its key: an 8-byte payload's two halves each
    equal the 4-byte oracle's payload result, and a 16-byte record moves whole."""
    rng = random.Random(23)
    for _ in range(50):
        la, lb = rng.randint(0, 300), rng.randint(0, 300)
        a, b = workloads.make_pair(rng.choice(["dup16", "uniform", "zipf"]), np.int64, la,
                                   lb, seed=rng.randint(0, 9999))
        va = np.array([rng.getrandbits(64) for _ in range(la)], dtype=np.uint64)
        vb = np.array([rng.getrandbits(64) for _ in range(lb)], dtype=np.uint64)
        ko, vo = orc.merge_kvw(a, va, b, vb)
        for shift in (0, 32):
            lo_a = ((va >> np.uint64(shift)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            lo_b = ((vb >> np.uint64(shift)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            k4, v4 = orc.merge_kv(a, lo_a, b, lo_b)
            assert np.array_equal(ko, k4)
            assert np.array_equal(((vo >> np.uint64(shift)) & np.uint64(0xFFFFFFFF))
                                  .astype(np.uint32), v4)
        rec = np.dtype([("x", np.uint64), ("y", np.uint64)])
        ra = np.zeros(la, rec)
        rb = np.zeros(lb, rec)
        ra["x"], ra["y"] = va, np.arange(la, dtype=np.uint64)
        rb["x"], rb["y"] = vb, np.arange(la, la + lb, dtype=np.uint64)
        _, ro = orc.merge_kvw(a, ra, b, rb)
        assert np.array_equal(ro["x"], vo)
        # stability: the origin index rises within each run of equal keys
        same = ko[1:] == ko[:-1]
        assert np.all(ro["y"][1:][same] > ro["y"][:-1][same])
