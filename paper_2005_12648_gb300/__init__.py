"""Python binding of the ipmerge C ABI (``include/ipmerge.h``).

GB300 (sm_103a) parallel in-place merge after Bramas & Bramas, arXiv 2005.12648.
Every function named ``ipm_*`` here calls the C function of the same name in
``_lib/libipmerge.so`` and only marshals arguments: tensors become device pointers,
dtype names become ``ipm_dtype`` codes, a torch stream becomes a ``cudaStream_t``,
and a non-OK status raises :class:`IpmError`.  Every step of the merge runs in the
library's CUDA kernels; there is no fallback.  PyTorch provides device memory
(workspaces come from its caching allocator) and streams only.

Importing this package does not need a GPU; calling an entry point does, and fails
loudly if the library has not been built (``build_ext.build_library()``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build_ext import LIB as _LIB_PATH

__all__ = [
    "IpmError", "DTYPES", "load", "ipm_status_string", "ipm_version", "ipm_merge_plan",
    "ipm_merge_workspace_bytes", "ipm_merge_inplace", "ipm_merge_inplace_kv",
    "ipm_merge_splits", "ipm_merge_rearrange", "ipm_merge_pairs",
    "ipm_rotate_workspace_bytes", "ipm_rotate", "ipm_rotate_cs_workspace_bytes",
    "ipm_rotate_cs", "ipm_division_splits", "SPLIT_KINDS", "division_splits",
    "ipm_read_device_status",
    "ipm_read_exchange_bytes",
    "ipm_timing_enable", "ipm_timing_read", "IpmTiming", "ipm_merge_inplace_noalloc",
    "ipm_read_noalloc_status", "ipm_set_wait_limit_ns", "ipm_get_wait_limit_ns",
    "workspace", "merge_inplace", "merge_inplace_kv",
    "IpmBatchedOptions", "ipm_merge_batched_workspace_bytes", "ipm_merge_batched_max_segment",
    "ipm_merge_batched", "ipm_read_merge_bytes", "segment_table", "merge_batched",
    "IpmBatchedTuneResult", "ipm_merge_batched_tune_workspace_bytes",
    "ipm_batched_tune_signature", "ipm_merge_batched_tune",
    "IpmSplitModel", "IpmSplitTrainOptions", "IpmSplitStats", "SPLIT_MODEL_HIDDEN",
    "ipm_split_model_train_workspace_bytes", "ipm_split_model_train", "ipm_split_model_forward",
    "ipm_split_model_loss_grad", "ipm_merge_splits_learned", "ipm_merge_inplace_learned",
    "split_model_initial_params", "split_model_to_device", "split_model_from_device",
    "train_split_model", "ipm_set_fused_levels", "ipm_get_fused_levels",
    "ipm_set_exchange_engine", "ipm_set_fused_engine", "ipm_merge_fused_plan",
]

DTYPES = {"int32": 0, "uint32": 1, "uint64": 2, "float32": 3, "int64": 4}
_ELEM = {0: 4, 1: 4, 2: 8, 3: 4, 4: 8}
STATUS = {0: "IPM_OK", 1: "IPM_ERR_INVALID_ARG", 2: "IPM_ERR_UNSUPPORTED_DTYPE",
          3: "IPM_ERR_ALIGNMENT", 4: "IPM_ERR_WORKSPACE", 5: "IPM_ERR_CUDA",
          6: "IPM_ERR_TIMEOUT", 7: "IPM_ERR_DEVICE"}


class IpmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(int(code), code)}")


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_vp, _u64, _u32, _i, _sz = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                            ctypes.c_size_t)
_SIGS = {
    "ipm_status_string": (ctypes.c_char_p, [_i]),
    "ipm_version": (_i, []),
    "ipm_merge_plan": (_i, [_u64, _u64, _i, _i, ctypes.POINTER(_u32),
                            ctypes.POINTER(_u64)]),
    "ipm_merge_workspace_bytes": (_i, [_u64, _u64, _i, _i, _u32, ctypes.POINTER(_sz)]),
    "ipm_merge_inplace": (_i, [_vp, _u64, _u64, _i, _u32, _vp, _sz, _vp]),
    "ipm_merge_inplace_kv": (_i, [_vp, _vp, _u64, _u64, _i, _i, _u32, _vp, _sz, _vp]),
    "ipm_merge_splits": (_i, [_vp, _u64, _u64, _i, _u64, _vp, _vp]),
    "ipm_merge_rearrange": (_i, [_vp, _vp, _u64, _u64, _i, _vp, _u32, _vp, _sz, _vp]),
    "ipm_merge_pairs": (_i, [_vp, _vp, _u64, _u64, _i, _vp, _u32, _vp]),
    "ipm_rearrange_permute_workspace_bytes": (_i, [_u64, _u64, _i, _i, ctypes.POINTER(_sz)]),
    "ipm_rearrange_permute": (_i, [_vp, _vp, _u64, _u64, _i, _i, _vp, _u32, _vp, _sz, _vp]),
    "ipm_rotate_workspace_bytes": (_i, [_u64, _u64, _u32, ctypes.POINTER(_sz)]),
    "ipm_read_exchange_bytes": (_i, [_vp, _vp, ctypes.POINTER(_u64)]),
    "ipm_rotate": (_i, [_vp, _u64, _u64, _u32, _vp, _sz, _vp]),
    "ipm_rotate_cs_workspace_bytes": (_i, [_u64, _u64, _u32, ctypes.POINTER(_sz)]),
    "ipm_rotate_cs": (_i, [_vp, _u64, _u64, _u32, _vp, _sz, _vp]),
    "ipm_division_splits": (_i, [_vp, _u64, _u64, _i, _u32, _u32, _vp, _vp, _vp]),
    "ipm_read_device_status": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "ipm_merge_inplace_noalloc": (_i, [_vp, _u64, _u64, _i, _vp]),
    "ipm_read_noalloc_status": (_i, [_vp, ctypes.POINTER(_i)]),
    "ipm_set_wait_limit_ns": (_i, [_u64]),
    "ipm_get_wait_limit_ns": (_i, [ctypes.POINTER(_u64)]),
    "ipm_timing_enable": (_i, [_i]),
    "ipm_timing_read": (_i, [ctypes.c_void_p]),
    "ipm_merge_batched_workspace_bytes": (_i, [_u64, _u32, _i, _i, _vp, ctypes.POINTER(_sz)]),
    "ipm_merge_batched_max_segment": (_i, [_i, _i, _vp, ctypes.POINTER(_u64)]),
    "ipm_merge_batched": (_i, [_vp, _vp, _u64, _vp, _u32, _i, _i, _vp, _vp, _sz, _vp]),
    "ipm_read_merge_bytes": (_i, [_vp, _vp, ctypes.POINTER(_u64)]),
    "ipm_merge_batched_tune_workspace_bytes": (_i, [_u64, _u32, _i, _i, ctypes.POINTER(_sz)]),
    "ipm_batched_tune_signature": (_i, [_vp, _u32, _i, _i, ctypes.POINTER(_u64)]),
    "ipm_merge_batched_tune": (_i, [_vp, _vp, _u64, _vp, _vp, _u32, _i, _i, _vp, _vp, _vp, _sz,
                                    _u32, ctypes.c_char_p, _vp, _vp]),
    "ipm_split_model_train_workspace_bytes": (_i, [_u32, ctypes.POINTER(_sz)]),
    "ipm_split_model_train": (_i, [_vp, _u64, _u64, _i, _vp, _u32, _vp, _vp, _vp, _sz, _vp]),
    "ipm_split_model_forward": (_i, [_vp, _vp, _u32, _vp, _vp]),
    "ipm_split_model_loss_grad": (_i, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "ipm_merge_splits_learned": (_i, [_vp, _u64, _u64, _i, _u64, _vp, _vp, _vp, _vp]),
    "ipm_merge_inplace_learned": (_i, [_vp, _u64, _u64, _i, _u32, _vp, _vp, _sz, _vp]),
    "ipm_set_fused_levels": (_i, [_u32]),
    "ipm_get_fused_levels": (_i, [ctypes.POINTER(_u32)]),
    "ipm_merge_fused_plan": (_i, [_u64, _u64, _i, _i, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "ipm_set_exchange_engine": (_i, [_u32]),
    "ipm_set_fused_engine": (_i, [_u32]),
}


TIMING_PHASES = 8


class IpmTiming(ctypes.Structure):
    """Mirror of ipm_timing: per-phase milliseconds and launch counts."""
    _fields_ = [("ms", ctypes.c_double * TIMING_PHASES),
                ("launches", ctypes.c_uint32 * TIMING_PHASES)]

    PHASES = ("split", "plan", "exchange", "merge", "batched", "train", "learned_split",
              "reserved")

    def as_dict(self):
        return {p: {"ms": self.ms[i], "launches": int(self.launches[i])}
                for i, p in enumerate(self.PHASES)}


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return list(_SIGS)


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libipmerge.so (once).  Raises if it is missing: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"ipmerge CUDA library not built ({p}); run "
                                   "paper_2005_12648_gb300.build_ext.build_library()")
            L = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(code: int, where: str) -> None:
    if code != 0:
        raise IpmError(code, where)


def _dt(dtype) -> int:
    if isinstance(dtype, int):
        if dtype not in _ELEM:
            raise ValueError(f"bad ipm_dtype {dtype}")
        return dtype
    if isinstance(dtype, str):
        return DTYPES[dtype]
    name = str(dtype).replace("torch.", "")
    if name in DTYPES:
        return DTYPES[name]
    raise ValueError(f"cannot map {dtype!r} to an ipm_dtype; pass 'int32', 'uint32', "
                     "'uint64', 'float32' or 'int64'")


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return x.data_ptr()
    raise TypeError(f"expected a tensor or an int pointer, got {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _nbytes(x) -> int:
    return x.numel() * x.element_size()


# ------------------------------------------------------------------ C ABI mirrors

def ipm_status_string(code: int) -> str:
    return load().ipm_status_string(int(code)).decode()


def ipm_version() -> int:
    return int(load().ipm_version())


def _payload(with_values) -> int:
    """The with_values argument of the merge queries: False / 0 keys only, True / 1 / 4 a
    4-byte payload, 8 an 8-byte payload; a dtype name gives its size."""
    if isinstance(with_values, bool):
        return int(with_values)
    if isinstance(with_values, str):
        return _ELEM[DTYPES[with_values]]
    return int(with_values)


def ipm_merge_plan(len_a: int, len_b: int, key_dtype, with_values=False):
    """Returns (log2_pairs, tile_capacity)."""
    g, t = _u32(0), _u64(0)
    _check(load().ipm_merge_plan(len_a, len_b, _dt(key_dtype), _payload(with_values),
                                 ctypes.byref(g), ctypes.byref(t)), "ipm_merge_plan")
    return int(g.value), int(t.value)


def ipm_merge_workspace_bytes(len_a: int, len_b: int, key_dtype, with_values=False,
                              log2_pairs: int = 0) -> int:
    out = _sz(0)
    _check(load().ipm_merge_workspace_bytes(len_a, len_b, _dt(key_dtype),
                                            _payload(with_values), log2_pairs,
                                            ctypes.byref(out)), "ipm_merge_workspace_bytes")
    return int(out.value)


def ipm_merge_inplace(buf, len_a: int, len_b: int, key_dtype, ws, log2_pairs: int = 0,
                      ws_bytes: int | None = None, stream=None) -> None:
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_merge_inplace(_ptr(buf), len_a, len_b, _dt(key_dtype), log2_pairs,
                                    _ptr(ws), wsb, _stream(stream)), "ipm_merge_inplace")


def ipm_merge_inplace_kv(keys, vals, len_a: int, len_b: int, key_dtype, ws,
                         val_dtype="uint32", log2_pairs: int = 0, ws_bytes: int | None = None,
                         stream=None) -> None:
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_merge_inplace_kv(_ptr(keys), _ptr(vals), len_a, len_b, _dt(key_dtype),
                                       _dt(val_dtype), log2_pairs, _ptr(ws), wsb,
                                       _stream(stream)), "ipm_merge_inplace_kv")


def ipm_merge_splits(buf, len_a: int, len_b: int, key_dtype, num_pairs: int, split_a,
                     stream=None) -> None:
    _check(load().ipm_merge_splits(_ptr(buf), len_a, len_b, _dt(key_dtype), num_pairs,
                                   _ptr(split_a), _stream(stream)), "ipm_merge_splits")


def ipm_merge_rearrange(buf, vals, len_a: int, len_b: int, key_dtype, split_a,
                        log2_pairs: int, ws, ws_bytes: int | None = None, stream=None):
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_merge_rearrange(_ptr(buf), _ptr(vals), len_a, len_b, _dt(key_dtype),
                                      _ptr(split_a), log2_pairs, _ptr(ws), wsb,
                                      _stream(stream)), "ipm_merge_rearrange")


def ipm_rearrange_permute_workspace_bytes(len_a: int, len_b: int, key_dtype,
                                          with_values=False) -> int:
    out = _sz(0)
    _check(load().ipm_rearrange_permute_workspace_bytes(len_a, len_b, _dt(key_dtype),
                                                        _payload(with_values),
                                                        ctypes.byref(out)),
           "ipm_rearrange_permute_workspace_bytes")
    return int(out.value)


def ipm_rearrange_permute(buf, vals, len_a: int, len_b: int, key_dtype, split_a,
                          log2_pairs: int, ws, ws_bytes: int | None = None, with_values=None,
                          stream=None) -> None:
    """The division stage as one permutation (sOptMov); with_values defaults to the
    payload tensor's element size (None: keys only)."""
    if with_values is None:
        with_values = 0 if vals is None else vals.element_size()
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_rearrange_permute(_ptr(buf), _ptr(vals), len_a, len_b, _dt(key_dtype),
                                        _payload(with_values), _ptr(split_a), log2_pairs,
                                        _ptr(ws), wsb, _stream(stream)),
           "ipm_rearrange_permute")


def ipm_merge_pairs(buf, vals, len_a: int, len_b: int, key_dtype, split_a,
                    log2_pairs: int, stream=None) -> None:
    _check(load().ipm_merge_pairs(_ptr(buf), _ptr(vals), len_a, len_b, _dt(key_dtype),
                                  _ptr(split_a), log2_pairs, _stream(stream)),
           "ipm_merge_pairs")


def ipm_rotate_workspace_bytes(len_x: int, len_y: int, elem_bytes: int) -> int:
    out = _sz(0)
    _check(load().ipm_rotate_workspace_bytes(len_x, len_y, elem_bytes, ctypes.byref(out)),
           "ipm_rotate_workspace_bytes")
    return int(out.value)


def ipm_read_exchange_bytes(ws, stream=None) -> int:
    out = _u64(0)
    _check(load().ipm_read_exchange_bytes(_ptr(ws), _stream(stream), ctypes.byref(out)),
           "ipm_read_exchange_bytes")
    return int(out.value)


def ipm_rotate(ptr, len_x: int, len_y: int, elem_bytes: int, ws,
               ws_bytes: int | None = None, stream=None) -> None:
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_rotate(_ptr(ptr), len_x, len_y, elem_bytes, _ptr(ws), wsb,
                             _stream(stream)), "ipm_rotate")


def ipm_rotate_cs_workspace_bytes(len_x: int, len_y: int, elem_bytes: int) -> int:
    out = _sz(0)
    _check(load().ipm_rotate_cs_workspace_bytes(len_x, len_y, elem_bytes, ctypes.byref(out)),
           "ipm_rotate_cs_workspace_bytes")
    return int(out.value)


def ipm_rotate_cs(ptr, len_x: int, len_y: int, elem_bytes: int, ws,
                  ws_bytes: int | None = None, stream=None) -> None:
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_rotate_cs(_ptr(ptr), len_x, len_y, elem_bytes, _ptr(ws), wsb,
                                _stream(stream)), "ipm_rotate_cs")


SPLIT_KINDS = {"exact": 0, "findmedian": 1}


def ipm_division_splits(buf, len_a: int, len_b: int, key_dtype, depth: int, split_kind,
                        ia, jb, stream=None) -> None:
    kind = SPLIT_KINDS[split_kind] if isinstance(split_kind, str) else int(split_kind)
    _check(load().ipm_division_splits(_ptr(buf), len_a, len_b, _dt(key_dtype), depth, kind,
                                      _ptr(ia), _ptr(jb), _stream(stream)),
           "ipm_division_splits")


def division_splits(buf, len_a: int, len_b: int, key_dtype, depth: int,
                    split_kind="findmedian", stream=None):
    """Pair boundaries of the division of Alg. 3 to 2^depth pairs, as two int64 device
    tensors (ia, jb) of 2^depth + 1 entries (pair k: A[ia[k], ia[k+1]) with
    B[jb[k], jb[k+1]))."""
    import torch

    ia = torch.empty((1 << depth) + 1, dtype=torch.int64, device=buf.device)
    jb = torch.empty_like(ia)
    ipm_division_splits(buf, len_a, len_b, key_dtype, depth, split_kind, ia, jb, stream)
    return ia, jb


def ipm_read_device_status(ws, stream=None) -> int:
    out = _i(0)
    _check(load().ipm_read_device_status(_ptr(ws), _stream(stream), ctypes.byref(out)),
           "ipm_read_device_status")
    return int(out.value)


def ipm_merge_inplace_noalloc(buf, len_a: int, len_b: int, key_dtype, stream=None) -> None:
    """The merge for callers that cannot allocate device memory: no workspace
    argument; the library's own fixed 8 MiB scratch array is used instead (at most
    2^15 pairs per call, keys only; calls that overlap on the GPU race on it)."""
    _check(load().ipm_merge_inplace_noalloc(_ptr(buf), len_a, len_b, _dt(key_dtype),
                                            _stream(stream)), "ipm_merge_inplace_noalloc")


def ipm_read_noalloc_status(stream=None) -> int:
    """Device status the last no-alloc merge on the current device left (0 = IPM_OK)."""
    out = _i(0)
    _check(load().ipm_read_noalloc_status(_stream(stream), ctypes.byref(out)),
           "ipm_read_noalloc_status")
    return int(out.value)


def ipm_set_wait_limit_ns(ns: int) -> None:
    """Limit of the merge calls' waits on other CTAs (0 = the default, 2 s)."""
    _check(load().ipm_set_wait_limit_ns(int(ns)), "ipm_set_wait_limit_ns")


def ipm_get_wait_limit_ns() -> int:
    out = _u64(0)
    _check(load().ipm_get_wait_limit_ns(ctypes.byref(out)), "ipm_get_wait_limit_ns")
    return int(out.value)


def ipm_timing_enable(enable: bool = True) -> None:
    _check(load().ipm_timing_enable(int(bool(enable))), "ipm_timing_enable")


def ipm_timing_read(into: "IpmTiming | None" = None) -> IpmTiming:
    t = into if into is not None else IpmTiming()
    _check(load().ipm_timing_read(ctypes.byref(t)), "ipm_timing_read")
    return t


class IpmBatchedOptions(ctypes.Structure):
    """Mirror of ipm_batched_options (tile 0 = default, 1 wide, 2 narrow, 3 quarter;
    order 0 = largest segment first, 1 = table order; ctas_per_sm 0 = as many as fit;
    form 0 = default, 1 = three launches, 2 = one launch)."""
    _fields_ = [("tile", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("order", ctypes.c_uint32), ("form", ctypes.c_uint32)]

    def as_dict(self):
        return {"tile": int(self.tile), "ctas_per_sm": int(self.ctas_per_sm),
                "order": int(self.order), "form": int(self.form)}


TUNE_MAX_CANDIDATES = 32


class IpmBatchedTuneEntry(ctypes.Structure):
    _fields_ = [("options", IpmBatchedOptions), ("ms", ctypes.c_float), ("pad", ctypes.c_uint32)]


class IpmBatchedTuneResult(ctypes.Structure):
    """Mirror of ipm_batched_tune_result."""
    _fields_ = [("best", IpmBatchedOptions), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float), ("candidates", ctypes.c_uint32),
                ("from_cache", ctypes.c_uint32), ("signature", ctypes.c_uint64),
                ("table", IpmBatchedTuneEntry * TUNE_MAX_CANDIDATES)]

    def as_dict(self):
        k = min(int(self.candidates), TUNE_MAX_CANDIDATES)
        return {"best": self.best.as_dict(), "best_ms": float(self.best_ms),
                "default_ms": float(self.default_ms), "candidates": int(self.candidates),
                "from_cache": bool(self.from_cache), "signature": f"{self.signature:016x}",
                "table": [{**self.table[i].options.as_dict(), "ms": float(self.table[i].ms)}
                          for i in range(k)]}


def _opts(options) -> "IpmBatchedOptions | None":
    if options is None or isinstance(options, IpmBatchedOptions):
        return options
    return IpmBatchedOptions(int(options.get("tile", 0)), int(options.get("ctas_per_sm", 0)),
                             int(options.get("order", 0)), int(options.get("form", 0)))


def ipm_merge_batched_workspace_bytes(buf_len: int, nseg: int, key_dtype,
                                      with_values: bool = False, options=None) -> int:
    out = _sz(0)
    o = _opts(options)
    _check(load().ipm_merge_batched_workspace_bytes(buf_len, nseg, _dt(key_dtype),
                                                    int(bool(with_values)),
                                                    ctypes.byref(o) if o is not None else None,
                                                    ctypes.byref(out)),
           "ipm_merge_batched_workspace_bytes")
    return int(out.value)


def ipm_merge_batched_max_segment(key_dtype, with_values: bool = False, options=None) -> int:
    out = _u64(0)
    o = _opts(options)
    _check(load().ipm_merge_batched_max_segment(_dt(key_dtype), int(bool(with_values)),
                                                ctypes.byref(o) if o is not None else None,
                                                ctypes.byref(out)),
           "ipm_merge_batched_max_segment")
    return int(out.value)


def ipm_merge_batched(buf, vals, buf_len: int, segs, nseg: int, key_dtype, ws,
                      val_dtype="uint32", options=None, ws_bytes: int | None = None,
                      stream=None) -> None:
    """segs: device array of nseg {offset, len_a, len_b} uint64 triples (e.g. an
    int64 tensor of shape [nseg, 3])."""
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    o = _opts(options)
    _check(load().ipm_merge_batched(_ptr(buf), _ptr(vals), buf_len, _ptr(segs), nseg,
                                    _dt(key_dtype), _dt(val_dtype),
                                    ctypes.byref(o) if o is not None else None, _ptr(ws), wsb,
                                    _stream(stream)), "ipm_merge_batched")


def ipm_read_merge_bytes(ws, stream=None) -> int:
    out = _u64(0)
    _check(load().ipm_read_merge_bytes(_ptr(ws), _stream(stream), ctypes.byref(out)),
           "ipm_read_merge_bytes")
    return int(out.value)


SPLIT_MODEL_HIDDEN = 32


class IpmSplitModel(ctypes.Structure):
    """Mirror of ipm_split_model (the struct itself lives in device memory)."""
    _fields_ = [("w1", ctypes.c_float * SPLIT_MODEL_HIDDEN),
                ("b1", ctypes.c_float * SPLIT_MODEL_HIDDEN),
                ("w2", ctypes.c_float * SPLIT_MODEL_HIDDEN), ("b2", ctypes.c_float),
                ("loss", ctypes.c_float), ("steps", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class IpmSplitTrainOptions(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


class IpmSplitStats(ctypes.Structure):
    _fields_ = [("diagonals", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("probes", ctypes.c_uint64), ("abs_err_sum", ctypes.c_uint64),
                ("abs_err_max", ctypes.c_uint64)]


def ipm_split_model_train_workspace_bytes(nsamples: int) -> int:
    out = _sz(0)
    _check(load().ipm_split_model_train_workspace_bytes(nsamples, ctypes.byref(out)),
           "ipm_split_model_train_workspace_bytes")
    return int(out.value)


def ipm_split_model_train(buf, len_a: int, len_b: int, key_dtype, diags, nsamples: int,
                          model, ws, steps: int = 300, lr: float = 1e-2, beta1: float = 0.9,
                          beta2: float = 0.999, eps: float = 1e-8,
                          ws_bytes: int | None = None, stream=None) -> None:
    """model: device buffer of sizeof(IpmSplitModel) bytes holding the initial
    parameters; trained in place.  diags: device uint64 (int64) array of diagonals."""
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    opt = IpmSplitTrainOptions(int(steps), float(lr), float(beta1), float(beta2), float(eps))
    _check(load().ipm_split_model_train(_ptr(buf), len_a, len_b, _dt(key_dtype), _ptr(diags),
                                        nsamples, ctypes.byref(opt), _ptr(model), _ptr(ws),
                                        wsb, _stream(stream)), "ipm_split_model_train")


def ipm_split_model_forward(model, x, n: int, y, stream=None) -> None:
    _check(load().ipm_split_model_forward(_ptr(model), _ptr(x), n, _ptr(y), _stream(stream)),
           "ipm_split_model_forward")


def ipm_split_model_loss_grad(model, x, t, n: int, grad, stream=None) -> None:
    _check(load().ipm_split_model_loss_grad(_ptr(model), _ptr(x), _ptr(t), n, _ptr(grad),
                                            _stream(stream)), "ipm_split_model_loss_grad")


def ipm_merge_splits_learned(buf, len_a: int, len_b: int, key_dtype, num_pairs: int, model,
                             split_a, stats=None, stream=None) -> None:
    _check(load().ipm_merge_splits_learned(_ptr(buf), len_a, len_b, _dt(key_dtype), num_pairs,
                                           _ptr(model), _ptr(split_a), _ptr(stats),
                                           _stream(stream)), "ipm_merge_splits_learned")


def ipm_merge_inplace_learned(buf, len_a: int, len_b: int, key_dtype, model, ws,
                              log2_pairs: int = 0, ws_bytes: int | None = None,
                              stream=None) -> None:
    wsb = _nbytes(ws) if ws_bytes is None else ws_bytes
    _check(load().ipm_merge_inplace_learned(_ptr(buf), len_a, len_b, _dt(key_dtype),
                                            log2_pairs, _ptr(model), _ptr(ws), wsb,
                                            _stream(stream)), "ipm_merge_inplace_learned")


def ipm_set_fused_levels(levels: int) -> None:
    _check(load().ipm_set_fused_levels(levels), "ipm_set_fused_levels")


def ipm_set_exchange_engine(engine: int) -> None:
    _check(load().ipm_set_exchange_engine(engine), "ipm_set_exchange_engine")


def ipm_set_fused_engine(engine: int) -> None:
    _check(load().ipm_set_fused_engine(engine), "ipm_set_fused_engine")


def ipm_merge_fused_plan(len_a: int, len_b: int, key_dtype, with_values=False):
    """(engine, fused levels) a merge of these sizes would use (engine None: none)."""
    e, f = _u32(0), _u32(0)
    _check(load().ipm_merge_fused_plan(len_a, len_b, _dt(key_dtype), _payload(with_values),
                                       ctypes.byref(e), ctypes.byref(f)),
           "ipm_merge_fused_plan")
    return (None if e.value == 0xFFFFFFFF else int(e.value)), int(f.value)


def ipm_get_fused_levels() -> int:
    out = _u32(0)
    _check(load().ipm_get_fused_levels(ctypes.byref(out)), "ipm_get_fused_levels")
    return int(out.value)


# ------------------------------------------------------------------ conveniences

def workspace(nbytes: int, device=None):
    """A workspace from torch's caching allocator (256-byte aligned)."""
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def merge_inplace(buf, len_a: int, len_b: int, key_dtype, log2_pairs: int = 0, stream=None):
    """Allocate the workspace and run ipm_merge_inplace on a CUDA tensor A|B."""
    ws = workspace(ipm_merge_workspace_bytes(len_a, len_b, key_dtype, False, log2_pairs),
                   buf.device)
    ipm_merge_inplace(buf, len_a, len_b, key_dtype, ws, log2_pairs, stream=stream)
    return ws


def merge_inplace_kv(keys, vals, len_a: int, len_b: int, key_dtype, log2_pairs: int = 0,
                     stream=None, val_dtype=None):
    """Allocate the workspace and merge keys with their payloads (4- or 8-byte: the
    payload tensor's element size when val_dtype is not given)."""
    if val_dtype is None:
        val_dtype = "uint64" if vals.element_size() == 8 else "uint32"
    vb = _ELEM[_dt(val_dtype)]
    ws = workspace(ipm_merge_workspace_bytes(len_a, len_b, key_dtype, vb, log2_pairs),
                   keys.device)
    ipm_merge_inplace_kv(keys, vals, len_a, len_b, key_dtype, ws, val_dtype=val_dtype,
                         log2_pairs=log2_pairs, stream=stream)
    return ws


def ipm_merge_batched_tune_workspace_bytes(buf_len: int, nseg: int, key_dtype,
                                           with_values: bool = False) -> int:
    out = _sz(0)
    _check(load().ipm_merge_batched_tune_workspace_bytes(buf_len, nseg, _dt(key_dtype),
                                                         int(bool(with_values)),
                                                         ctypes.byref(out)),
           "ipm_merge_batched_tune_workspace_bytes")
    return int(out.value)


def _host_segments(h_segs):
    """A C-contiguous host uint64 [nseg, 3] copy of a segment table (or None)."""
    if h_segs is None:
        return None
    import numpy as np
    return np.ascontiguousarray(np.asarray(h_segs, dtype=np.int64).reshape(-1, 3)
                                .view(np.uint64))


def ipm_batched_tune_signature(h_segs, key_dtype, with_values: bool = False) -> str:
    """The autotuner's cache key of a host segment table ([nseg, 3] offset, len_a, len_b)."""
    hs = _host_segments(h_segs)
    out = _u64(0)
    _check(load().ipm_batched_tune_signature(hs.ctypes.data if hs.size else None, hs.shape[0],
                                             _dt(key_dtype), int(bool(with_values)),
                                             ctypes.byref(out)), "ipm_batched_tune_signature")
    return f"{out.value:016x}"


def ipm_merge_batched_tune(buf, vals, buf_len: int, segs, nseg: int, key_dtype, scratch,
                           ws, scratch_vals=None, reps: int = 5, cache_path=None,
                           h_segs=None, val_dtype="uint32", ws_bytes: int | None = None,
                           stream=None) -> dict:
    """Time the candidate option sets of ipm_merge_batched on `scratch` (restored from
    buf before every run) and return the fastest (see ipm_merge_batched_tune in the
    header); the dict holds the chosen options, both times and every candidate's."""
    res = IpmBatchedTuneResult()
    hs = _host_segments(h_segs)
    wsb = (_nbytes(ws) if ws is not None else 0) if ws_bytes is None else ws_bytes
    path = cache_path.encode() if isinstance(cache_path, str) else cache_path
    _check(load().ipm_merge_batched_tune(
        _ptr(buf), _ptr(vals), buf_len, _ptr(segs),
        hs.ctypes.data if hs is not None and hs.size else None, nseg, _dt(key_dtype),
        _dt(val_dtype), _ptr(scratch), _ptr(scratch_vals), _ptr(ws), wsb, reps, path,
        ctypes.addressof(res), _stream(stream) if buf is not None else None),
        "ipm_merge_batched_tune")
    return res.as_dict()


def segment_table(offsets, len_a, len_b, device=None):
    """A device segment table (int64 [nseg, 3]: offset, len_a, len_b) from host lists."""
    import torch
    t = torch.stack([torch.as_tensor(offsets, dtype=torch.int64),
                     torch.as_tensor(len_a, dtype=torch.int64),
                     torch.as_tensor(len_b, dtype=torch.int64)], dim=1).contiguous()
    return t.to(device if device is not None else "cuda")


def merge_batched(buf, segs, key_dtype, vals=None, options=None, stream=None):
    """Allocate the workspace and run ipm_merge_batched over a device segment table."""
    nseg = int(segs.shape[0])
    ws = workspace(ipm_merge_batched_workspace_bytes(buf.numel(), nseg, key_dtype,
                                                     vals is not None, options), buf.device)
    ipm_merge_batched(buf, vals, buf.numel(), segs, nseg, key_dtype, ws, options=options,
                      stream=stream)
    return ws


def split_model_initial_params():
    """Deterministic starting point for training (float32, 97 values w1|b1|w2|b2): the
    hidden units are steps at evenly spaced centres c_h = (h + 1/2)/32 of the input
    range, w1 = 16, b1 = -16 c_h, w2 = 1/64, b2 = 1/2, so y(x) starts as a smooth
    staircase close to y = x (the split of two runs drawn from one distribution)."""
    import numpy as np

    H = SPLIT_MODEL_HIDDEN
    c = (np.arange(H, dtype=np.float64) + 0.5) / H
    p = np.concatenate([np.full(H, 16.0), -16.0 * c, np.full(H, 1.0 / 64), [0.5]])
    return p.astype(np.float32)


def split_model_to_device(params, device=None):
    """A device ipm_split_model (uint8 tensor of its size) holding the 97 parameters."""
    import numpy as np
    import torch

    m = IpmSplitModel()
    p = np.asarray(params, dtype=np.float32)
    H = SPLIT_MODEL_HIDDEN
    m.w1[:] = p[:H].tolist()
    m.b1[:] = p[H:2 * H].tolist()
    m.w2[:] = p[2 * H:3 * H].tolist()
    m.b2 = float(p[3 * H])
    raw = np.frombuffer(bytes(m), dtype=np.uint8).copy()
    return torch.from_numpy(raw).to(device if device is not None else "cuda")


def split_model_from_device(t):
    """(params float32[97], loss, steps) of a device ipm_split_model."""
    import numpy as np

    raw = t.cpu().numpy().tobytes()
    m = IpmSplitModel.from_buffer_copy(raw)
    H = SPLIT_MODEL_HIDDEN
    p = np.concatenate([np.array(m.w1[:], np.float32), np.array(m.b1[:], np.float32),
                        np.array(m.w2[:], np.float32), np.array([m.b2], np.float32)])
    return p, float(m.loss), int(m.steps)


def train_split_model(buf, len_a: int, len_b: int, key_dtype, diags, steps: int = 300,
                      lr: float = 1e-2, params=None, stream=None):
    """Train a device model from the given (or the default initial) parameters on the
    device diagonals `diags`; returns the device model tensor."""
    model = split_model_to_device(split_model_initial_params() if params is None else params,
                                  buf.device)
    n = int(diags.numel())
    ws = workspace(ipm_split_model_train_workspace_bytes(n), buf.device)
    ipm_split_model_train(buf, len_a, len_b, key_dtype, diags, n, model, ws, steps=steps,
                          lr=lr, stream=stream)
    return model
