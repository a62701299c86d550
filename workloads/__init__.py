"""Seeded synthetic inputs for the merge workloads.

This module is the only code that both the CPU oracle tests and the CUDA path use.
It holds none of the merge method's arithmetic: it draws values, sorts each run
(numpy or torch sort) and lays the runs out.  Raw values come from a counter-based
generator (SplitMix64 of seed, stream and index), so the numpy and the torch versions
produce identical integer inputs.

Distributions (per run, then sorted):
  uniform       int32 U[0,2^31), uint32 U[0,2^32), uint64 U[0,2^64), int64 the full
                signed range, float32 U[0,1)
                on a 2^-24 grid
  dup16         U{0..15} (heavy duplicates)
  disjoint      max(A) < min(B): A in [0,2^30), B in [2^30,2^31) (uint64: B >= 2^63;
                int64: A in [-2^62, 0), B in [0, 2^62))
  revdisjoint   the same ranges with A and B exchanged (B < A)
  alternation   A[i] = 2i, B[j] = 2j+1
  zipf          key = rank-1, rank ~ Zipf(s=1.2) on 1..2^20, inverse CDF
  gmm           float32 from an 8-component Gaussian mixture fixed by the seed
  paper         x[0] = 0, x[i] = x[i-1] + floor(5*U(0,1)) (the paper's workload, Sec. 4)
"""
from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB

DISTS = ("uniform", "dup16", "disjoint", "revdisjoint", "alternation", "zipf", "gmm",
         "paper")
DTYPES = {"int32": np.int32, "uint32": np.uint32, "uint64": np.uint64,
          "float32": np.float32, "int64": np.int64}


def _mix_seed(seed: int, stream: int) -> int:
    """Start of the counter sequence for (seed, stream)."""
    z = (seed * 0x100000001B3 + stream * 0xD6E8FEB86659FD93 + 0x2005_12648) & M64
    return z


def splitmix64_np(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 counters (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(GOLDEN)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(C2)
        return z ^ (z >> np.uint64(31))


def raw_np(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    base = np.uint64(_mix_seed(seed, stream))
    idx = np.arange(start, start + n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_np(idx + base)


def unit_np(h: np.ndarray) -> np.ndarray:
    """uint64 -> float64 in [0,1) on the 2^-53 grid (exact)."""
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def zipf_cdf(s: float = 1.2, nranks: int = 1 << 20) -> np.ndarray:
    w = 1.0 / np.power(np.arange(1, nranks + 1, dtype=np.float64), s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def gmm_params(seed: int, k: int = 8):
    """Mixture fixed by the seed: means U[-100,100], sigma log-uniform [0.5,10],
    weights Dirichlet(1) (normalised Exp(1) draws)."""
    u = unit_np(raw_np(seed, 900, 3 * k))
    means = -100.0 + 200.0 * u[:k]
    sig = np.exp(np.log(0.5) + (np.log(10.0) - np.log(0.5)) * u[k:2 * k])
    e = -np.log1p(-u[2 * k:3 * k])
    return means, sig, e / e.sum()


def _values_np(dist: str, dtype, side: int, n: int, seed: int) -> np.ndarray:
    dt = np.dtype(dtype)
    stream = 2 * DISTS.index(dist) + side
    if dist == "alternation":
        return (2 * np.arange(n, dtype=np.uint64) + side).astype(dt)
    if dist == "paper":
        u = unit_np(raw_np(seed, stream, n))
        inc = np.floor(u * 5.0).astype(np.int64)
        if n:
            inc[0] = 0
        return np.cumsum(inc).astype(dt)
    if dist == "gmm":
        if dt != np.float32:
            raise ValueError("gmm is a float32 distribution")
        means, sig, w = gmm_params(seed)
        h = raw_np(seed, stream, 3 * n).reshape(3, n) if n else np.zeros((3, 0), np.uint64)
        u0, u1, u2 = unit_np(h[0]), unit_np(h[1]), unit_np(h[2])
        comp = np.searchsorted(np.cumsum(w), u0, side="right").clip(0, len(w) - 1)
        g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
        x = (means[comp] + sig[comp] * g).astype(np.float32)
        x[x == 0] = np.float32(0.0)  # canonicalise -0.0 to +0.0
        return x
    h = raw_np(seed, stream, n)
    if dist == "zipf":
        return np.searchsorted(zipf_cdf(), unit_np(h), side="right").astype(dt)
    if dist == "dup16":
        return (h >> np.uint64(60)).astype(dt)
    if dist == "uniform":
        if dt == np.int32:
            return (h >> np.uint64(33)).astype(np.int32)
        if dt == np.uint32:
            return (h >> np.uint64(32)).astype(np.uint32)
        if dt == np.uint64:
            return h
        if dt == np.int64:
            return h.view(np.int64)  # the full signed range
        if dt == np.float32:
            return ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    if dist in ("disjoint", "revdisjoint"):
        low_side = 0 if dist == "disjoint" else 1
        hi = side != low_side
        if dt == np.uint64:
            v = h >> np.uint64(1)
            return v + np.uint64(1 << 63) if hi else v
        if dt == np.float32:
            v = (h >> np.uint64(41)).astype(np.float64) * 2.0 ** -23
            return (v + (1.0 if hi else 0.0)).astype(np.float32)
        if dt == np.int64:  # low side negative, high side non-negative
            v = (h >> np.uint64(2)).astype(np.int64)
            return v if hi else v - (1 << 62)
        v = (h >> np.uint64(34)).astype(np.int64) + ((1 << 30) if hi else 0)
        return v.astype(dt)
    raise ValueError(f"unknown distribution {dist!r} for {dt}")


def make_pair(dist: str, dtype, la: int, lb: int, seed: int = 0):
    """Sorted runs A (la keys) and B (lb keys) as numpy arrays."""
    a = np.sort(_values_np(dist, dtype, 0, la, seed), kind="stable")
    b = np.sort(_values_np(dist, dtype, 1, lb, seed), kind="stable")
    return a, b


def make_buffer(dist: str, dtype, la: int, lb: int, seed: int = 0) -> np.ndarray:
    """One contiguous buffer A|B."""
    a, b = make_pair(dist, dtype, la, lb, seed)
    return np.concatenate([a, b])


def payload(n: int) -> np.ndarray:
    """Key-value payload: the original buffer index of each key."""
    return np.arange(n, dtype=np.uint32)


# ----------------------------------------------------------------------------------
# torch (device) generation: identical integer values, sorted on the device.
# ----------------------------------------------------------------------------------

def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(torch, z, k: int):
    return (z >> k) & ((1 << (64 - k)) - 1)


def raw_torch(torch, seed: int, stream: int, n: int, device, start: int = 0):
    base = _i64(_mix_seed(seed, stream))
    z = torch.arange(start, start + n, dtype=torch.int64, device=device) + base
    z = z + _i64(GOLDEN)
    z = (z ^ _lsr(torch, z, 30)) * _i64(C1)
    z = (z ^ _lsr(torch, z, 27)) * _i64(C2)
    return z ^ _lsr(torch, z, 31)


def storage_dtype(torch, dtype):
    """torch storage dtype carrying the key bits (unsigned keys ride in signed ints)."""
    dt = np.dtype(dtype)
    return {np.dtype(np.int32): torch.int32, np.dtype(np.uint32): torch.int32,
            np.dtype(np.uint64): torch.int64, np.dtype(np.float32): torch.float32,
            np.dtype(np.int64): torch.int64}[dt]


def _sorted_side_torch(torch, dist, dtype, side, n, seed, device):
    dt = np.dtype(dtype)
    stream = 2 * DISTS.index(dist) + side
    if dist in ("gmm", "paper", "zipf"):
        v = _values_np(dist, dtype, side, n, seed)
        if dist != "paper":
            v = np.sort(v, kind="stable")
        t = torch.from_numpy(v.view({4: np.int32, 8: np.int64}[dt.itemsize])
                             if dt != np.float32 else v)
        return t.to(device)
    if dist == "alternation":
        v = 2 * torch.arange(n, dtype=torch.int64, device=device) + side
        return v.to(storage_dtype(torch, dtype))
    h = raw_torch(torch, seed, stream, n, device)
    if dist == "dup16":
        v = _lsr(torch, h, 60)
    elif dist == "uniform":
        if dt == np.int32:
            v = _lsr(torch, h, 33)
        elif dt == np.uint32:
            v = _lsr(torch, h, 32)
        elif dt == np.uint64:
            v = h ^ _i64(1 << 63)  # unsigned order as signed order
            v = torch.sort(v).values ^ _i64(1 << 63)
            return v
        elif dt == np.int64:
            return torch.sort(h).values
        else:
            v = _lsr(torch, h, 40).to(torch.float64) * 2.0 ** -24
            return torch.sort(v.to(torch.float32)).values
    elif dist in ("disjoint", "revdisjoint"):
        low_side = 0 if dist == "disjoint" else 1
        hi = side != low_side
        if dt == np.uint64:
            v = _lsr(torch, h, 1)
            v = torch.sort(v).values
            return v + _i64(1 << 63) if hi else v
        if dt == np.float32:
            v = _lsr(torch, h, 41).to(torch.float64) * 2.0 ** -23 + (1.0 if hi else 0.0)
            return torch.sort(v.to(torch.float32)).values
        if dt == np.int64:
            v = _lsr(torch, h, 2)
            return torch.sort(v if hi else v - (1 << 62)).values
        v = _lsr(torch, h, 34) + ((1 << 30) if hi else 0)
    else:
        raise ValueError(dist)
    v = torch.sort(v).values
    return v.to(storage_dtype(torch, dtype))


def make_buffer_torch(torch, dist: str, dtype, la: int, lb: int, seed: int, device):
    """A|B as one device tensor whose bits equal make_buffer(...) (integer dists)."""
    a = _sorted_side_torch(torch, dist, dtype, 0, la, seed, device)
    b = _sorted_side_torch(torch, dist, dtype, 1, lb, seed, device)
    return torch.cat([a, b])


def as_numpy_keys(t, dtype) -> np.ndarray:
    """Device/host tensor of key bits -> numpy array of the key dtype."""
    return t.cpu().numpy().view(np.dtype(dtype))


# ----------------------------------------------------------------------------------
# Batched segmented workload.
# ----------------------------------------------------------------------------------

def _seg_lengths(u: np.ndarray, e_lo: float, e_max: float) -> np.ndarray:
    return np.floor(np.exp2(e_lo + u * (e_max - e_lo))).astype(np.int64)


def batched_lengths(nseg: int = 20000, total_cap: int = 1 << 28, e_lo: float = 4.0,
                    e_hi: float = 22.0, seed: int = 0):
    """Per-side lengths, log-uniform shape, exponent range [e_lo, e_max] with e_max
    (<= e_hi) the largest value, found by bisection, whose total is <= total_cap.
    Returns (len_a, len_b, e_max)."""
    u = unit_np(raw_np(seed, 700, 2 * nseg)).reshape(2, nseg)
    if _seg_lengths(u, e_lo, e_hi).sum() <= total_cap:
        e_max = e_hi
    else:
        lo, hi = e_lo, e_hi
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if _seg_lengths(u, e_lo, mid).sum() <= total_cap:
                lo = mid
            else:
                hi = mid
        e_max = lo
    L = _seg_lengths(u, e_lo, e_max)
    return L[0], L[1], e_max


def batched_buffer(len_a: np.ndarray, len_b: np.ndarray, seed: int = 0):
    """int32 uniform segments laid out back to back (A_s|B_s for s = 0, 1, ...).
    Run r holds (SplitMix64(pos) >> 33) over its buffer positions, sorted.
    Returns (buffer, offsets)."""
    la = np.asarray(len_a, dtype=np.int64)
    lb = np.asarray(len_b, dtype=np.int64)
    runs = np.stack([la, lb], axis=1).reshape(-1)
    n = int(runs.sum())
    h = (raw_np(seed, 800, n) >> np.uint64(33))
    rid = np.repeat(np.arange(runs.size, dtype=np.uint64), runs)
    key = np.sort((rid << np.uint64(32)) | h)
    buf = (key & np.uint64(0xFFFFFFFF)).astype(np.int32)
    offs = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.uint64)
    return buf, offs


def batched_buffer_torch(torch, len_a, len_b, seed: int, device):
    """Device version of batched_buffer with identical values."""
    la = np.asarray(len_a, dtype=np.int64)
    lb = np.asarray(len_b, dtype=np.int64)
    runs = torch.from_numpy(np.stack([la, lb], axis=1).reshape(-1)).to(device)
    n = int(runs.sum().item())
    h = _lsr(torch, raw_torch(torch, seed, 800, n, device), 33)
    rid = torch.repeat_interleave(torch.arange(runs.numel(), device=device,
                                               dtype=torch.int64), runs)
    key = torch.sort((rid << 32) | h).values
    buf = (key & 0xFFFFFFFF).to(torch.int32)
    offs = np.concatenate([[0], np.cumsum(la + lb)[:-1]]).astype(np.uint64)
    return buf, offs


# ----------------------------------------------------------------------------------
# Training diagonals of the learned split proposer.
# ----------------------------------------------------------------------------------

def split_training_diagonals(n: int, nsamples: int = 4096, seed: int = 0) -> np.ndarray:
    """Diagonals in [0, n] for training: half uniform draws (SplitMix64 stream 900),
    half stratified (the centre of each of nsamples/2 equal slices), sorted, uint64."""
    half = nsamples // 2
    u = unit_np(raw_np(seed, 900, nsamples - half))
    uni = np.floor(u * (n + 1)).astype(np.uint64)
    strat = np.floor((np.arange(half, dtype=np.float64) + 0.5) * (n / max(half, 1))).astype(np.uint64)
    d = np.concatenate([uni, strat])
    return np.sort(np.minimum(d, np.uint64(n)))
