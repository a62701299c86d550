"""Host <-> device helpers for the GPU parity tests (marshalling only)."""
import numpy as np

STORAGE = {np.dtype(np.int32): np.int32, np.dtype(np.uint32): np.int32,
           np.dtype(np.uint64): np.int64, np.dtype(np.float32): np.float32,
           np.dtype(np.int64): np.int64}
NAME = {np.dtype(np.int32): "int32", np.dtype(np.uint32): "uint32",
        np.dtype(np.uint64): "uint64", np.dtype(np.float32): "float32",
        np.dtype(np.int64): "int64"}


def to_dev(x: np.ndarray, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x).view(STORAGE[x.dtype]).copy()).to(dev)


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(np.dtype(dtype))


def bits(x: np.ndarray) -> np.ndarray:
    return x.view({4: np.uint32, 8: np.uint64}[x.dtype.itemsize])


def first_diff(got: np.ndarray, want: np.ndarray):
    d = np.flatnonzero(bits(got) != bits(want))
    return int(d[0]) if d.size else None
