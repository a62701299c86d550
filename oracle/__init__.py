"""CPU oracle for the parallel in-place merge (arXiv 2005.12648).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The product
path (``paper_2005_12648_gb300``) never imports it, and the two share no code.

The arithmetic lives in plain sequential C (``ipm_oracle.c`` + ``oracle_typed.h``),
compiled with gcc on first use into ``oracle/_build/``; this module only marshals
numpy arrays through ctypes.  Each wrapper names the passage of the paper that the
C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libipm_oracle.so")
_SRCS = [os.path.join(_HERE, "ipm_oracle.c"), os.path.join(_HERE, "oracle_typed.h")]
_lock = threading.Lock()
_lib = None

SUFFIX = {np.dtype(np.int32): "i32", np.dtype(np.uint32): "u32",
          np.dtype(np.uint64): "u64", np.dtype(np.float32): "f32",
          np.dtype(np.int64): "i64"}

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march flags, so it builds on x86 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_SO) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in _SRCS)
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-Wall", "-Wextra", "-o", tmp, _SRCS[0], "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L: ctypes.CDLL) -> None:
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    for s in SUFFIX.values():
        getattr(L, f"orc_merge_{s}").argtypes = [vp, u64, vp, u64, vp]
        getattr(L, f"orc_merge_kv_{s}").argtypes = [vp, vp, u64, vp, vp, u64, vp, vp]
        getattr(L, f"orc_merge_kvw_{s}").argtypes = [vp, vp, u64, vp, vp, u64, u64, vp, vp]
        getattr(L, f"orc_splits_replay_{s}").argtypes = [vp, u64, vp, u64, vp, u64, vp]
        f = getattr(L, f"orc_split_bsearch_{s}")
        f.argtypes = [vp, u64, vp, u64, u64]
        f.restype = u64
        f = getattr(L, f"orc_gallop_split_{s}")
        f.argtypes = [vp, u64, vp, u64, u64, u64, _u64p]
        f.restype = u64
        getattr(L, f"orc_ls_rotate_{s}").argtypes = [vp, u64, u64, _u64p]
        getattr(L, f"orc_cs_rotate_{s}").argtypes = [vp, u64, u64, _u64p, _u64p]
        getattr(L, f"orc_findmedian_{s}").argtypes = [vp, u64, vp, u64, _u64p, _u64p]
        getattr(L, f"orc_srecpar_{s}").argtypes = [vp, u64, u64, ctypes.c_int, u64,
                                                   ctypes.c_int, ctypes.c_int, vp, _u64p]
        getattr(L, f"orc_arrange_{s}").argtypes = [vp, u64, vp, u64, vp, vp, u64, vp]
        getattr(L, f"orc_division_{s}").argtypes = [vp, u64, vp, u64, ctypes.c_int,
                                                    ctypes.c_int, vp, vp]
    L.orc_mlp_forward.argtypes = [vp, ctypes.c_int, vp, u64, vp]
    L.orc_mlp_loss_grad.argtypes = [vp, ctypes.c_int, vp, vp, u64, vp]
    L.orc_mlp_loss_grad.restype = ctypes.c_double
    L.orc_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int]


def _c(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x)


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def _sfx(*arrs: np.ndarray) -> str:
    dt = arrs[0].dtype
    for a in arrs[1:]:
        if a.dtype != dt:
            raise TypeError("A and B must have the same key dtype")
    if dt not in SUFFIX:
        raise TypeError(f"unsupported key dtype {dt}")
    return SUFFIX[dt]


def merge(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Stable merge of sorted A and B, ties taking A first (Sec. 1 problem statement)."""
    a, b = _c(a), _c(b)
    out = np.empty(a.size + b.size, dtype=a.dtype)
    getattr(lib(), f"orc_merge_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size, _p(out))
    return out


def merge_kv(ka, va, kb, vb):
    """Key-value stable merge: a uint32 payload rides with each key."""
    ka, kb = _c(ka), _c(kb)
    va, vb = _c(va).astype(np.uint32, copy=False), _c(vb).astype(np.uint32, copy=False)
    ko = np.empty(ka.size + kb.size, dtype=ka.dtype)
    vo = np.empty(ka.size + kb.size, dtype=np.uint32)
    getattr(lib(), f"orc_merge_kv_{_sfx(ka, kb)}")(_p(ka), _p(va), ka.size, _p(kb), _p(vb),
                                                   kb.size, _p(ko), _p(vo))
    return ko, vo


def merge_kvw(ka, va, kb, vb):
    """Key-value stable merge with payloads of any element size (va, vb: numpy arrays
    of one dtype, e.g. uint64 or a structured record); returns (keys, payloads)."""
    ka, kb, va, vb = _c(ka), _c(kb), _c(va), _c(vb)
    if va.dtype != vb.dtype or va.size != ka.size or vb.size != kb.size:
        raise ValueError("payloads must match their keys and share one dtype")
    ko = np.empty(ka.size + kb.size, dtype=ka.dtype)
    vo = np.empty(ka.size + kb.size, dtype=va.dtype)
    getattr(lib(), f"orc_merge_kvw_{_sfx(ka, kb)}")(_p(ka), _p(va), ka.size, _p(kb), _p(vb),
                                                    kb.size, va.dtype.itemsize, _p(ko),
                                                    _p(vo))
    return ko, vo


def diagonals(n: int, P: int) -> np.ndarray:
    """d_k = floor(k*n/P), k = 0..P (exact integer arithmetic)."""
    return np.array([(k * n) // P for k in range(P + 1)], dtype=np.uint64)


def splits_replay(a, b, d) -> np.ndarray:
    """Exact split i_k for each ascending diagonal d_k by replaying the plain merge."""
    a, b = _c(a), _c(b)
    d = _c(np.asarray(d, dtype=np.uint64))
    if d.size and (np.any(np.diff(d.astype(np.int64)) < 0) or int(d[-1]) > a.size + b.size):
        raise ValueError("diagonals must be ascending and <= len(A)+len(B)")
    out = np.empty(d.size, dtype=np.uint64)
    getattr(lib(), f"orc_splits_replay_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size, _p(d),
                                                      d.size, _p(out))
    return out


def split_bsearch(a, b, d: int) -> int:
    """Exact split on diagonal d by binary search (independent second form)."""
    a, b = _c(a), _c(b)
    return int(getattr(lib(), f"orc_split_bsearch_{_sfx(a, b)}")(_p(a), a.size, _p(b),
                                                                  b.size, int(d)))


def gallop_split(a, b, d: int, guess: int):
    """Exact split on diagonal d by galloping from a guess; returns (i, probes)."""
    a, b = _c(a), _c(b)
    pr = ctypes.c_uint64(0)
    i = getattr(lib(), f"orc_gallop_split_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size,
                                                          int(d), int(guess), ctypes.byref(pr))
    return int(i), int(pr.value)


def ls_rotate(x: np.ndarray, lx: int):
    """Linear shifting (Sec. 3.4): returns ([Y|X], elementary swaps)."""
    x = np.array(x, copy=True)
    ns = ctypes.c_uint64(0)
    getattr(lib(), f"orc_ls_rotate_{_sfx(x)}")(_p(x), int(lx), x.size - int(lx),
                                               ctypes.byref(ns))
    return x, int(ns.value)


def cs_rotate(x: np.ndarray, la: int):
    """Circular shifting (Sec. 3.4): returns ([B|A], cycles, moves)."""
    x = np.array(x, copy=True)
    nc, nm = ctypes.c_uint64(0), ctypes.c_uint64(0)
    getattr(lib(), f"orc_cs_rotate_{_sfx(x)}")(_p(x), int(la), x.size - int(la),
                                               ctypes.byref(nc), ctypes.byref(nm))
    return x, int(nc.value), int(nm.value)


def findmedian(a, b):
    """FindMedian (Alg. 1) in the corrected reading; returns (pA, pB)."""
    a, b = _c(a), _c(b)
    pa, pb = ctypes.c_uint64(0), ctypes.c_uint64(0)
    getattr(lib(), f"orc_findmedian_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size,
                                                   ctypes.byref(pa), ctypes.byref(pb))
    return int(pa.value), int(pb.value)


def srecpar(buf: np.ndarray, middle: int, depth_limit: int, size_limit: int = 1,
            split: str = "exact", shift: str = "ls"):
    """sRecPar (Alg. 3) run sequentially; returns (merged copy, element moves)."""
    x = np.array(buf, copy=True)
    tmp = np.empty_like(x)
    mv = ctypes.c_uint64(0)
    getattr(lib(), f"orc_srecpar_{_sfx(x)}")(
        _p(x), int(middle), x.size, int(depth_limit), int(size_limit),
        {"exact": 0, "findmedian": 1}[split], {"ls": 0, "cs": 1}[shift], _p(tmp),
        ctypes.byref(mv))
    return x, int(mv.value)


def division(a, b, depth: int, split: str = "findmedian"):
    """Pair boundaries of the division of Alg. 3 to 2^depth pairs (no data moved):
    (ia, jb), 2^depth + 1 entries each; pair k is A[ia[k], ia[k+1]) with
    B[jb[k], jb[k+1]).  split is "exact" (half-diagonal stable split) or "findmedian"."""
    a, b = _c(a), _c(b)
    P = 1 << int(depth)
    ia = np.zeros(P + 1, dtype=np.uint64)
    jb = np.zeros(P + 1, dtype=np.uint64)
    getattr(lib(), f"orc_division_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size, int(depth),
                                                 {"exact": 0, "findmedian": 1}[split],
                                                 _p(ia), _p(jb))
    return ia, jb


def division_balance(ia, jb):
    """Largest pair of a division: (over the pairs that need a merge, i.e. both sides
    non-empty; over all pairs).  The comparison metric of Sec. 4 is
    (Max_FindMedian - Max_optimal) / Max_optimal of these."""
    na = np.diff(ia.astype(np.int64))
    nb = np.diff(jb.astype(np.int64))
    c = na + nb
    need = (na > 0) & (nb > 0)
    return int(c[need].max()) if need.any() else 0, int(c.max())


def arrange(a, b, d, i) -> np.ndarray:
    """Layout after the division stage: A_0 B_0 A_1 B_1 ... (Sec. 3)."""
    a, b = _c(a), _c(b)
    d = _c(np.asarray(d, dtype=np.uint64))
    i = _c(np.asarray(i, dtype=np.uint64))
    out = np.empty(a.size + b.size, dtype=a.dtype)
    getattr(lib(), f"orc_arrange_{_sfx(a, b)}")(_p(a), a.size, _p(b), b.size, _p(d), _p(i),
                                                d.size - 1, _p(out))
    return out


def mlp_forward(params: np.ndarray, H: int, x: np.ndarray) -> np.ndarray:
    p = _c(np.asarray(params, dtype=np.float64))
    x = _c(np.asarray(x, dtype=np.float64))
    y = np.empty_like(x)
    lib().orc_mlp_forward(_p(p), H, _p(x), x.size, _p(y))
    return y


def mlp_loss_grad(params: np.ndarray, H: int, x: np.ndarray, t: np.ndarray):
    """MSE loss and its analytic gradient, float64."""
    p = _c(np.asarray(params, dtype=np.float64))
    x = _c(np.asarray(x, dtype=np.float64))
    t = _c(np.asarray(t, dtype=np.float64))
    g = np.empty(3 * H + 1, dtype=np.float64)
    loss = lib().orc_mlp_loss_grad(_p(p), H, _p(x), _p(t), x.size, _p(g))
    return float(loss), g


def adam_step(params, m, v, g, lr, beta1, beta2, eps, step):
    """One Adam step, in place on params, m and v (all float64 arrays)."""
    for arr in (params, m, v):
        if arr.dtype != np.float64 or not arr.flags.c_contiguous:
            raise TypeError("params, m, v must be contiguous float64")
    g = _c(np.asarray(g, dtype=np.float64))
    lib().orc_adam_step(_p(params), _p(m), _p(v), _p(g), params.size, lr, beta1, beta2,
                        eps, int(step))
