"""The C-ABI library builds, loads without a GPU and exports every declared symbol.

Only host-side paths are exercised here (queries and argument checks that return
before any CUDA call); compute calls need a GPU and live in the gpu-marked tests.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ipm_[a-z0-9_]+)\s*\(",
                  re.M)


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        names |= set(DECL.findall(open(h).read()))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2005_12648_gb300 import build_ext

    path = build_ext.build_library()
    import paper_2005_12648_gb300 as m

    return m.load(path), m


def test_header_declares_the_hot_path():
    names = declared_symbols()
    for required in ("ipm_merge_inplace", "ipm_merge_inplace_kv", "ipm_merge_splits",
                     "ipm_merge_rearrange", "ipm_merge_pairs", "ipm_rotate",
                     "ipm_merge_workspace_bytes", "ipm_read_device_status",
                     "ipm_merge_batched", "ipm_merge_inplace_learned", "ipm_rotate_cs",
                     "ipm_division_splits", "ipm_rearrange_permute"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    L, m = lib
    names = declared_symbols()
    assert names, "no declarations parsed"
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    # the binding mirrors exactly the declared entry points
    assert set(m.exported_symbols()) == names


def test_host_queries(lib):
    L, m = lib
    # the permutation's workspace: status and counters, an n-bit map, and per round the
    # saved keys (and payloads) of every 31st block of 32 positions plus their 8-byte
    # positions
    n = 3_000_017 + 2_900_011
    cap = 32 * -(-(-(-n // 32)) // 31)
    up = lambda x: -(-x // 256) * 256  # noqa: E731
    for vb in (0, 4, 8):
        want = 512 + up(-(-n // 32) * 4) + up(cap * 4) + up(cap * vb) + up(cap * 8)
        assert m.ipm_rearrange_permute_workspace_bytes(3_000_017, 2_900_011, "int32",
                                                       vb) == want
    assert m.ipm_version() >= 100
    assert m.ipm_status_string(0) == "IPM_OK"
    assert m.ipm_status_string(6) == "IPM_ERR_TIMEOUT"
    G, tile = m.ipm_merge_plan(1 << 28, 1 << 28, "int32")
    assert (1 << G) * tile >= (1 << 29) and (1 << (G - 1)) * tile < (1 << 29)
    G0, tile0 = m.ipm_merge_plan(100, 100, "int32")
    assert G0 == 0 and tile0 >= 200
    Gk, tilek = m.ipm_merge_plan(1 << 26, 1 << 26, "uint32", with_values=True)
    assert tilek < tile and (1 << Gk) * tilek >= (1 << 27)
    ws = m.ipm_merge_workspace_bytes(1 << 28, 1 << 28, "int32")
    # O(P): split table + plans, a few hundred bytes per pair at most
    assert 256 < ws < 400 * (1 << G) + 4096
    assert m.ipm_rotate_workspace_bytes(1000, 10, 4) >= 256
    # CS: status block only when every cycle fits one worker (gcd 1000, cycles of 2)...
    assert m.ipm_rotate_cs_workspace_bytes(1000, 1000, 4) == 256
    # ...else one saved element per segment, at most 2^19 of them
    assert 256 < m.ipm_rotate_cs_workspace_bytes(1000, 9, 8) <= 256 + 8 * 64
    for lx, ly in [(1 << 28, (1 << 28) + 1), ((1 << 30) + 3, 1 << 30), (1 << 40, 1)]:
        assert m.ipm_rotate_cs_workspace_bytes(lx, ly, 8) <= 256 + 8 * (1 << 19)


def test_noalloc_limit_fits_its_fixed_scratch(lib):
    """The no-alloc merge serves up to 2^15 pairs from an 8 MiB array: at the largest
    size it accepts (2^15 full tiles) the plan has exactly 2^15 pairs and the workspace
    the merge needs fits the array, for 4- and 8-byte keys; one key more needs 2^16."""
    L, m = lib
    for dt in ("int32", "uint64"):
        _, tile = m.ipm_merge_plan(1, 1, dt)
        n = (1 << 15) * tile
        G, _ = m.ipm_merge_plan(n // 2, n - n // 2, dt)
        assert G == 15
        assert m.ipm_merge_workspace_bytes(n // 2, n - n // 2, dt) <= 8 << 20
        G1, _ = m.ipm_merge_plan(n // 2, n - n // 2 + 1, dt)
        assert G1 == 16
        # refused on the host, before any device call: a fake address is never touched
        assert L.ipm_merge_inplace_noalloc(0x1000, n // 2, n - n // 2 + 1,
                                           m.DTYPES[dt], None) == 1


def test_wait_limit_setting(lib):
    L, m = lib
    assert m.ipm_get_wait_limit_ns() == 2_000_000_000
    m.ipm_set_wait_limit_ns(5_000)
    assert m.ipm_get_wait_limit_ns() == 5_000
    m.ipm_set_wait_limit_ns(0)  # back to the default
    assert m.ipm_get_wait_limit_ns() == 2_000_000_000
    assert L.ipm_set_wait_limit_ns(2_000_000_001) == 1
    assert m.ipm_get_wait_limit_ns() == 2_000_000_000


def test_argument_errors_return_before_any_cuda_call(lib):
    L, m = lib
    null = None
    # bad dtype
    assert L.ipm_merge_inplace(null, 10, 10, 9, 0, null, 0, null) == 2
    # NULL buffer with data
    assert L.ipm_merge_inplace(null, 10, 10, 0, 0, 4096, 1 << 20, null) == 1
    # misaligned buffer
    assert L.ipm_merge_inplace(0x1001, 10, 10, 0, 0, 4096, 1 << 20, null) == 3
    # workspace too small
    assert L.ipm_merge_inplace(0x1000, 10, 10, 0, 0, 4096, 16, null) == 4
    # pairs that cannot fit one tile
    assert L.ipm_merge_inplace(0x1000, 1 << 28, 1 << 28, 0, 1, 4096, 1 << 30, null) == 1
    # key-value: the payload type is only a width (4 or 8 bytes); an unknown type code
    # is rejected, and so is a payload pointer not aligned to its width
    assert L.ipm_merge_inplace_kv(0x1000, 0x2000, 4, 4, 0, 9, 0, 4096, 1 << 20, null) == 2
    assert L.ipm_merge_inplace_kv(0x1000, 0x2004, 4, 4, 0, 2, 0, 4096, 1 << 20, null) == 3
    # with_values: 0, 1, 4 or 8
    assert L.ipm_merge_workspace_bytes(100, 100, 0, 3, 0, ctypes.byref(ctypes.c_size_t())) == 2
    # splits: zero pairs
    assert L.ipm_merge_splits(0x1000, 4, 4, 0, 0, 0x2000, null) == 1
    # rotate: bad element size
    assert L.ipm_rotate(0x1000, 4, 4, 2, 0x2000, 4096, null) == 2
    assert L.ipm_rotate_cs(0x1000, 4, 4, 2, 0x2000, 4096, null) == 2
    # CS: misaligned buffer, small workspace, NULL buffer
    assert L.ipm_rotate_cs(0x1002, 4, 4, 4, 0x2000, 4096, null) == 3
    assert L.ipm_rotate_cs(0x1000, 1000, 9, 4, 0x2000, 16, null) == 4
    assert L.ipm_rotate_cs(null, 4, 4, 4, 0x2000, 4096, null) == 1
    assert L.ipm_rotate_cs(null, 0, 4, 4, null, 0, null) == 0
    # division: depth, split kind, dtype, NULL outputs, alignment
    assert L.ipm_division_splits(0x1000, 4, 4, 0, 25, 0, 0x2000, 0x3000, null) == 1
    assert L.ipm_division_splits(0x1000, 4, 4, 0, 3, 2, 0x2000, 0x3000, null) == 1
    assert L.ipm_division_splits(0x1000, 4, 4, 7, 3, 0, 0x2000, 0x3000, null) == 2
    assert L.ipm_division_splits(0x1000, 4, 4, 0, 3, 0, null, 0x3000, null) == 1
    assert L.ipm_division_splits(null, 4, 4, 0, 3, 0, 0x2000, 0x3000, null) == 1
    assert L.ipm_division_splits(0x1004, 4, 4, 2, 3, 0, 0x2000, 0x3000, null) == 3
    assert L.ipm_division_splits(0x1000, 4, 4, 0, 3, 0, 0x2004, 0x3000, null) == 3
    # permutation: payload width, NULL table, payload pointer without a width, pairs
    # beyond 2^22, a run beyond 2^40, small workspace, alignment
    sz = ctypes.c_size_t()
    assert L.ipm_rearrange_permute_workspace_bytes(100, 100, 0, 3, ctypes.byref(sz)) == 2
    assert L.ipm_rearrange_permute_workspace_bytes(100, 100, 9, 0, ctypes.byref(sz)) == 2
    assert L.ipm_rearrange_permute(0x1000, null, 4, 4, 0, 0, null, 2, 0x2000, 1 << 20,
                                   null) == 1
    assert L.ipm_rearrange_permute(0x1000, 0x3000, 4, 4, 0, 0, 0x4000, 2, 0x2000, 1 << 20,
                                   null) == 1
    assert L.ipm_rearrange_permute(0x1000, null, 4, 4, 0, 0, 0x4000, 23, 0x2000, 1 << 20,
                                   null) == 1
    assert L.ipm_rearrange_permute(0x1000, null, (1 << 40) + 1, 4, 0, 0, 0x4000, 2,
                                   0x2000, 1 << 62, null) == 1
    assert L.ipm_rearrange_permute(0x1000, null, 1000, 1000, 0, 0, 0x4000, 2, 0x2000, 16,
                                   null) == 4
    assert L.ipm_rearrange_permute(0x1002, null, 4, 4, 0, 0, 0x4000, 2, 0x2000, 1 << 20,
                                   null) == 3
    assert L.ipm_rearrange_permute(0x1000, null, 4, 4, 0, 0, 0x4004, 2, 0x2000, 1 << 20,
                                   null) == 3
    assert L.ipm_rearrange_permute(0x1000, null, 0, 0, 0, 0, 0x4000, 2, 0x2000, 1 << 20,
                                   null) == 0
    # empty inputs are a no-op that succeeds without touching the device
    assert L.ipm_merge_inplace(null, 0, 0, 0, 0, null, 0, null) == 0
    with pytest.raises(m.IpmError):
        m.ipm_merge_workspace_bytes(1, 1, "int32", log2_pairs=40)
