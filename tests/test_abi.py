"""The C ABI builds for sm_103a, loads without a GPU and exports every symbol
that include/*.h declares; host-side validation rejects bad graphs before any
CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1702_07409_gb300 import _build, gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef\s+struct\s*\{.*?\}\s*\w+\s*;", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsg?_[a-z0-9_]+)\s*\(", text)))


def _exported(path):
    L = ctypes.CDLL(path)
    return L


@pytest.fixture(scope="module")
def gpu_lib():
    return ctypes.CDLL(_build.build_gpu())


def test_headers_declare_the_abi():
    names = _declared(os.path.join(ROOT, "include", "founsure_gpu.h"))
    for fn in ("fs_encode", "fs_decode", "fs_update", "fs_repair", "fs_code_create"):
        assert fn in names


def test_every_declared_symbol_is_exported(gpu_lib):
    from paper_1702_07409_gb300 import founsure
    gen_lib = ctypes.CDLL(_build.build_gen())
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        lib = gen_lib if os.path.basename(h) == "fs_gen.h" else gpu_lib
        for name in _declared(h):
            assert hasattr(lib, name), "%s declared in %s is not exported" % (name, h)
    assert set(founsure.EXPORTS) == set(_declared(os.path.join(ROOT, "include", "founsure_gpu.h")))


def test_status_strings(gpu_lib):
    gpu_lib.fs_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert gpu_lib.fs_status_string(s).startswith(b"FS_")


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


def _create(lib, ptr, idx, n_cols, t=64, pre=None):
    ptr = np.ascontiguousarray(ptr, np.int32)
    idx = np.ascontiguousarray(idx, np.int32)
    lt = _Csr(ptr.size - 1, n_cols, ptr.ctypes.data, idx.ctypes.data if idx.size else None)
    h = ctypes.c_void_p()
    lib.fs_code_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    rc = lib.fs_code_create(ctypes.byref(pre) if pre is not None else None, ctypes.byref(lt),
                            t, 0, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("ptr,idx,n_cols,t", [
    ([0, 2, 3], [1, 1, 0], 4, 64),      # repeated neighbour
    ([0, 2, 3], [2, 1, 0], 4, 64),      # row not ascending
    ([0, 2, 3], [0, 4, 1], 4, 64),      # index out of range
    ([0, 2, 1], [0, 1, 2], 4, 64),      # row_ptr decreasing
    ([1, 2, 3], [0, 1, 2], 4, 64),      # row_ptr[0] != 0
    ([0, 1, 2], [0, 1], 4, 40),         # t not a multiple of 16
    ([0, 1, 2], [0, 1], 0, 64),         # no data blocks
])
def test_create_rejects_bad_graphs_on_host(gpu_lib, ptr, idx, n_cols, t):
    rc, h = _create(gpu_lib, ptr, idx, n_cols, t)
    assert rc == 2 and not h.value  # FS_ERR_INVALID, nothing created


def test_generator_library_loads():
    L = gen.lib()
    assert L.fsg_round_count(0.5, 3) == 2
