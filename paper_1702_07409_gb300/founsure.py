"""Python binding of ``libfounsure_gpu.so`` (the C ABI in include/founsure_gpu.h).

Argument marshalling only: every step of encode, decode, update and repair
runs in the library's CUDA kernels. PyTorch supplies device memory and
streams; buffers are passed as ``torch.Tensor`` (CUDA, contiguous) or as raw
device addresses (``int``). There is no CPU fallback: if the library cannot
be built or loaded, or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _build

FS_OK, FS_STALL, FS_ERR_INVALID, FS_ERR_CUDA, FS_ERR_NOMEM, FS_ERR_TIMEOUT, FS_ERR_SCRATCH = range(7)
ENCODE_STATIC_SCRATCH_BYTES = 65536
DECODE_JOINT, DECODE_TWO_PASS = 0, 1
OP_ENCODE, OP_DECODE, OP_UPDATE, OP_REPAIR = 0, 1, 2, 3
OP_SCHEDULE = 4  # batches only: the decoding schedule without its payload
TUNE_PEEL_CTAS, TUNE_GATHER_CTAS, TUNE_DPG_COMPACT, TUNE_L2_HINTS = 1, 2, 3, 4
TUNE_ENCODE_SLICES = 5
TUNE_ROWS_PER_TICKET = 6
TUNE_PEEL_COLUMNS = 7
TUNE_PEEL_FLOW = 8
WS_STATUS_OFFSET = 0

#: every symbol declared in include/founsure_gpu.h
EXPORTS = ("fs_code_create", "fs_code_destroy", "fs_code_info", "fs_code_set_tuning",
           "fs_workspace_bytes",
           "fs_encode", "fs_encode_static", "fs_encode_rows", "fs_decode", "fs_decode_schedule",
           "fs_decode_payload", "fs_decode_path", "fs_update", "fs_repair",
           "fs_batch_create", "fs_batch_run", "fs_batch_status", "fs_batch_destroy",
           "fs_selftest_timeout", "fs_status_string",
           "fs_local_create", "fs_local_destroy", "fs_local_info", "fs_local_groups",
           "fs_local_check2", "fs_local_workspace_bytes", "fs_repair_local", "fs_local_path")
LOCAL_HOST_ONLY = 1


class _Stripe(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("d_data", ctypes.c_void_p),
                ("d_parity", ctypes.c_void_p), ("d_coded", ctypes.c_void_p),
                ("d_erased", ctypes.c_void_p), ("d_data_out", ctypes.c_void_p),
                ("d_unrecovered", ctypes.c_void_p), ("d_n_unrecovered", ctypes.c_void_p),
                ("d_ws", ctypes.c_void_p)]


class FounsureError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s: %s" % (what, status_string(status)))
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class _PathView(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_void_p), ("n_pairs", ctypes.c_void_p),
                ("level_off", ctypes.c_void_p), ("pair_f", ctypes.c_void_p),
                ("pair_g", ctypes.c_void_p), ("parity", ctypes.c_void_p),
                ("plan", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads (building if stale) the CUDA library. Raises if it cannot."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build_gpu())
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        L.fs_code_create.argtypes = [vp, vp, sz, ctypes.c_int, ctypes.POINTER(vp)]
        L.fs_code_create.restype = ctypes.c_int
        L.fs_code_destroy.argtypes = [vp]
        L.fs_code_destroy.restype = None
        L.fs_code_info.argtypes = [vp, vp, vp, vp, vp]
        L.fs_code_info.restype = ctypes.c_int
        L.fs_code_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.fs_code_set_tuning.restype = ctypes.c_int
        L.fs_workspace_bytes.argtypes = [vp, ctypes.c_int, i32]
        L.fs_workspace_bytes.restype = sz
        L.fs_encode.argtypes = [vp, vp, vp, vp, vp, vp]
        L.fs_encode.restype = ctypes.c_int
        L.fs_encode_static.argtypes = [vp, vp, vp, vp, vp, vp]
        L.fs_encode_static.restype = ctypes.c_int
        L.fs_encode_rows.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp]
        L.fs_encode_rows.restype = ctypes.c_int
        L.fs_decode.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.fs_decode.restype = ctypes.c_int
        L.fs_decode_schedule.argtypes = [vp, vp, vp, vp, vp, vp]
        L.fs_decode_schedule.restype = ctypes.c_int
        L.fs_decode_payload.argtypes = [vp, vp, vp, vp, vp]
        L.fs_decode_payload.restype = ctypes.c_int
        L.fs_decode_path.argtypes = [vp, vp, ctypes.POINTER(_PathView)]
        L.fs_decode_path.restype = ctypes.c_int
        L.fs_update.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp]
        L.fs_update.restype = ctypes.c_int
        L.fs_repair.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        L.fs_repair.restype = ctypes.c_int
        L.fs_batch_create.argtypes = [ctypes.POINTER(_Stripe), i32, ctypes.c_int,
                                      ctypes.POINTER(vp)]
        L.fs_batch_create.restype = ctypes.c_int
        L.fs_batch_run.argtypes = [vp, vp]
        L.fs_batch_run.restype = ctypes.c_int
        L.fs_batch_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
        L.fs_batch_status.restype = ctypes.c_int
        L.fs_batch_destroy.argtypes = [vp]
        L.fs_batch_destroy.restype = None
        L.fs_selftest_timeout.argtypes = [vp, vp]
        L.fs_selftest_timeout.restype = ctypes.c_int
        L.fs_local_create.argtypes = [vp, vp, i32, ctypes.c_int, ctypes.POINTER(vp)]
        L.fs_local_create.restype = ctypes.c_int
        L.fs_local_destroy.argtypes = [vp]
        L.fs_local_destroy.restype = None
        L.fs_local_info.argtypes = [vp] + [vp] * 7
        L.fs_local_info.restype = ctypes.c_int
        L.fs_local_groups.argtypes = [vp, vp, vp]
        L.fs_local_groups.restype = ctypes.c_int
        L.fs_local_check2.argtypes = [vp, vp, vp, vp]
        L.fs_local_check2.restype = ctypes.c_int
        L.fs_local_workspace_bytes.argtypes = [vp]
        L.fs_local_workspace_bytes.restype = sz
        L.fs_repair_local.argtypes = [vp, vp, vp, sz, vp, vp, vp, vp]
        L.fs_repair_local.restype = ctypes.c_int
        L.fs_local_path.argtypes = [vp, vp, ctypes.POINTER(_PathView)]
        L.fs_local_path.restype = ctypes.c_int
        L.fs_status_string.argtypes = [ctypes.c_int]
        L.fs_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().fs_status_string(int(s)).decode()


def _check(rc: int, what: str) -> None:
    if rc != FS_OK:
        raise FounsureError(rc, what)


def _call(name: str, *args) -> int:
    """Calls a library function with arguments already marshalled (so a bad
    argument is refused before the library is loaded)."""
    return getattr(lib(), name)(*args)


def _addr(x) -> Optional[int]:
    """Device address of a CUDA tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _nbytes(x) -> int:
    return x.numel() * x.element_size()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Code:
    """A Founsure code on the current CUDA device (fs_code_create).

    ``graph`` is any object with b, m, n, pre_ptr, pre_idx, lt_ptr, lt_idx
    (e.g. ``gen.Graph``; ``chained=True`` marks a precode over the
    intermediates, such as the array LDPC checks); ``block_bytes`` is t (a
    multiple of 16)."""

    def __init__(self, graph, block_bytes: int, mode: int = DECODE_JOINT):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the Founsure GPU library has no CPU path")
        self.b, self.m, self.n = int(graph.b), int(graph.m), int(graph.n)
        self.k_int = self.b + self.m
        self.t = int(block_bytes)
        self.mode = mode
        self._keep = []
        pre = None
        if self.m > 0:
            pp = np.ascontiguousarray(graph.pre_ptr, np.int32)
            pi = np.ascontiguousarray(graph.pre_idx, np.int32)
            self._keep += [pp, pi]
            pre = _Csr(self.m, self.k_int if getattr(graph, "chained", False) else self.b,
                       pp.ctypes.data, pi.ctypes.data if pi.size else None)
        lp = np.ascontiguousarray(graph.lt_ptr, np.int32)
        li = np.ascontiguousarray(graph.lt_idx, np.int32)
        self._keep += [lp, li]
        lt = _Csr(self.n, self.k_int, lp.ctypes.data, li.ctypes.data if li.size else None)
        h = ctypes.c_void_p()
        rc = lib().fs_code_create(ctypes.byref(pre) if pre is not None else None,
                                  ctypes.byref(lt), self.t, mode, ctypes.byref(h))
        _check(rc, "fs_code_create")
        self._h = h
        self._lib = lib()

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.fs_code_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, knob: int, value: int) -> None:
        """Performance knob (fs_code_set_tuning); results never change."""
        _check(lib().fs_code_set_tuning(self._h, knob, value), "fs_code_set_tuning")

    # -- workspaces -----------------------------------------------------------
    def workspace_bytes(self, op: int, n_items: int = 0) -> int:
        return int(lib().fs_workspace_bytes(self._h, op, n_items))

    def workspace(self, op: int, n_items: int = 0, device=None):
        import torch
        return torch.empty(max(self.workspace_bytes(op, n_items), 256), dtype=torch.uint8,
                           device=device or "cuda")

    @staticmethod
    def ws_status(ws) -> int:
        """Device status word of a workspace (synchronises the device)."""
        import torch
        torch.cuda.synchronize()
        return int(ws[WS_STATUS_OFFSET:WS_STATUS_OFFSET + 4].view(torch.int32).item())

    # -- operations -----------------------------------------------------------
    def _need(self, x, nbytes, name):
        if x is not None and not isinstance(x, int) and _nbytes(x) < nbytes:
            raise ValueError("%s holds %d bytes, needs %d" % (name, _nbytes(x), nbytes))

    def encode(self, data, parity, coded, ws, stream=None) -> None:
        self._need(data, self.b * self.t, "data")
        self._need(parity, self.m * self.t, "parity")
        self._need(coded, self.n * self.t, "coded")
        self._need(ws, self.workspace_bytes(OP_ENCODE), "ws")
        _check(_call("fs_encode", self._h, _addr(data), _addr(parity), _addr(coded), _addr(ws),
                     _stream(stream)), "fs_encode")

    def encode_static(self, data, parity, coded, status=None, stream=None) -> None:
        """fs_encode_static: the encode with the library's static scratch area
        instead of a caller workspace (for callers that cannot allocate)."""
        self._need(data, self.b * self.t, "data")
        self._need(parity, self.m * self.t, "parity")
        self._need(coded, self.n * self.t, "coded")
        _check(_call("fs_encode_static", self._h, _addr(data), _addr(parity), _addr(coded),
                     _addr(status), _stream(stream)), "fs_encode_static")

    def encode_rows(self, row_begin, row_end, data, parity, coded, ws, stream=None) -> None:
        self._need(data, self.b * self.t, "data")
        self._need(parity, self.m * self.t, "parity")
        self._need(coded, self.n * self.t, "coded")
        self._need(ws, self.workspace_bytes(OP_ENCODE), "ws")
        _check(_call("fs_encode_rows", self._h, row_begin, row_end, _addr(data), _addr(parity),
                     _addr(coded), _addr(ws), _stream(stream)), "fs_encode_rows")

    def decode(self, coded, erased, data_out, unrecovered, n_unrecovered, ws, stream=None) -> None:
        self._need(coded, self.n * self.t, "coded")
        self._need(erased, self.n, "erased")
        self._need(data_out, self.b * self.t, "data_out")
        self._need(unrecovered, self.k_int, "unrecovered")
        self._need(n_unrecovered, 4, "n_unrecovered")
        self._need(ws, self.workspace_bytes(OP_DECODE), "ws")
        _check(_call("fs_decode", self._h, _addr(coded), _addr(erased), _addr(data_out),
                     _addr(unrecovered), _addr(n_unrecovered), _addr(ws),
                     _stream(stream)), "fs_decode")

    def decode_schedule(self, erased, unrecovered, n_unrecovered, ws, stream=None) -> None:
        self._need(erased, self.n, "erased")
        self._need(unrecovered, self.k_int, "unrecovered")
        self._need(n_unrecovered, 4, "n_unrecovered")
        self._need(ws, self.workspace_bytes(OP_DECODE), "ws")
        _check(_call("fs_decode_schedule", self._h, _addr(erased), _addr(unrecovered),
                     _addr(n_unrecovered), _addr(ws), _stream(stream)),
               "fs_decode_schedule")

    def decode_payload(self, coded, data_out, ws, stream=None) -> None:
        self._need(coded, self.n * self.t, "coded")
        self._need(data_out, self.b * self.t, "data_out")
        self._need(ws, self.workspace_bytes(OP_DECODE), "ws")
        _check(_call("fs_decode_payload", self._h, _addr(coded), _addr(data_out), _addr(ws),
                     _stream(stream)), "fs_decode_payload")

    def decode_path(self, ws):
        """Views into a decode workspace after fs_decode (synchronises):
        returns dict(n_levels, n_pairs, level_off, pair_f, pair_g, parity,
        plan: the payload plan's 8-word header)."""
        import torch
        v = _PathView()
        _check(lib().fs_decode_path(self._h, _addr(ws), ctypes.byref(v)), "fs_decode_path")
        base = ws.data_ptr()

        def at(ptr, count, dtype):
            off = ptr - base
            esz = torch.tensor([], dtype=dtype).element_size()
            return ws[off:off + count * esz].view(dtype)

        torch.cuda.synchronize()
        nl = int(at(v.n_levels, 1, torch.int32).item())
        npairs = int(at(v.n_pairs, 1, torch.int32).item())
        return dict(n_levels=nl, n_pairs=npairs,
                    level_off=at(v.level_off, nl + 1, torch.int32),
                    pair_f=at(v.pair_f, npairs, torch.int32),
                    pair_g=at(v.pair_g, npairs, torch.int32),
                    parity=at(v.parity, self.m * self.t, torch.uint8),
                    plan=at(v.plan, 8, torch.int32))

    def update(self, idx, n_idx: int, new, data, parity, coded, ws, stream=None) -> None:
        self._need(idx, 4 * n_idx, "idx")
        self._need(new, n_idx * self.t, "new")
        self._need(data, self.b * self.t, "data")
        self._need(parity, self.m * self.t, "parity")
        self._need(coded, self.n * self.t, "coded")
        self._need(ws, self.workspace_bytes(OP_UPDATE, n_idx), "ws")
        _check(_call("fs_update", self._h, _addr(idx), n_idx, _addr(new), _addr(data),
                     _addr(parity), _addr(coded), _addr(ws), _stream(stream)), "fs_update")

    def repair(self, lost, n_lost: int, data, parity, coded, ws, stream=None) -> None:
        self._need(lost, 4 * n_lost, "lost")
        self._need(data, self.b * self.t, "data")
        self._need(parity, self.m * self.t, "parity")
        self._need(coded, self.n * self.t, "coded")
        self._need(ws, self.workspace_bytes(OP_REPAIR, n_lost), "ws")
        _check(_call("fs_repair", self._h, _addr(lost), n_lost, _addr(data), _addr(parity),
                     _addr(coded), _addr(ws), _stream(stream)), "fs_repair")


class Batch:
    """fs_batch: many stripes (each with its own Code) encoded or decoded in a
    fixed number of launches. `stripes` is a list of dicts with the fs_stripe
    fields as tensors (or device addresses): encode {code, data, parity,
    coded}; decode {code, coded, erased, data_out, unrecovered, n_unrecovered,
    ws}; schedule (OP_SCHEDULE) {code, erased, unrecovered, n_unrecovered,
    ws}. The tensors are kept alive by the batch; run() only enqueues
    (capturable in a CUDA graph)."""

    def __init__(self, stripes, op: int):
        self._keep = stripes
        arr = (_Stripe * max(len(stripes), 1))()
        for i, s in enumerate(stripes):
            code = s["code"]
            if op == OP_ENCODE:
                code._need(s["data"], code.b * code.t, "data")
                code._need(s.get("parity"), code.m * code.t, "parity")
                code._need(s.get("coded"), code.n * code.t, "coded")
            elif op in (OP_DECODE, OP_SCHEDULE):  # other ops: the library rejects them
                if op == OP_DECODE:
                    code._need(s.get("coded"), code.n * code.t, "coded")
                    code._need(s.get("data_out"), code.b * code.t, "data_out")
                code._need(s.get("erased"), code.n, "erased")
                code._need(s.get("unrecovered"), code.k_int, "unrecovered")
                code._need(s.get("n_unrecovered"), 4, "n_unrecovered")
                code._need(s.get("ws"), code.workspace_bytes(OP_DECODE), "ws")
            arr[i] = _Stripe(code._h, _addr(s.get("data")), _addr(s.get("parity")),
                             _addr(s.get("coded")), _addr(s.get("erased")),
                             _addr(s.get("data_out")), _addr(s.get("unrecovered")),
                             _addr(s.get("n_unrecovered")), _addr(s.get("ws")))
        h = ctypes.c_void_p()
        _check(lib().fs_batch_create(arr, len(stripes), op, ctypes.byref(h)), "fs_batch_create")
        self._h = h

    def run(self, stream=None) -> None:
        _check(lib().fs_batch_run(self._h, _stream(stream)), "fs_batch_run")

    def status(self) -> int:
        """Device status of the last run (blocking)."""
        st = ctypes.c_int32(0)
        _check(lib().fs_batch_status(self._h, ctypes.byref(st)), "fs_batch_status")
        return int(st.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().fs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_timeout(stream=None) -> int:
    """fs_selftest_timeout: runs a kernel whose bounded wait always runs out
    and returns the status it wrote (FS_ERR_TIMEOUT)."""
    import torch
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    _check(lib().fs_selftest_timeout(_addr(st), _stream(stream)), "fs_selftest_timeout")
    return int(st.item())


class Local:
    """Local recovery groups of a graph and repair from them
    (fs_local_create / fs_repair_local): check #2 equations and check #3
    groups by Algorithm 4 and the set-XOR derivations, built on the host; the
    repair peels over the check #3 groups on the device. ``host_only`` skips
    the device copy (groups only, no repair)."""

    def __init__(self, graph, max_sweeps: int = 0, host_only: bool = False):
        if not host_only:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the Founsure GPU library has no CPU path")
        self.b, self.m, self.n = int(graph.b), int(graph.m), int(graph.n)
        self.k_int = self.b + self.m
        self._keep = []
        pre = None
        if self.m > 0:
            pp = np.ascontiguousarray(graph.pre_ptr, np.int32)
            pi = np.ascontiguousarray(graph.pre_idx, np.int32)
            self._keep += [pp, pi]
            pre = _Csr(self.m, self.k_int if getattr(graph, "chained", False) else self.b,
                       pp.ctypes.data, pi.ctypes.data if pi.size else None)
        lp = np.ascontiguousarray(graph.lt_ptr, np.int32)
        li = np.ascontiguousarray(graph.lt_idx, np.int32)
        self._keep += [lp, li]
        lt = _Csr(self.n, self.k_int, lp.ctypes.data, li.ctypes.data if li.size else None)
        h = ctypes.c_void_p()
        self._lib = lib()
        rc = self._lib.fs_local_create(ctypes.byref(pre) if pre is not None else None,
                                       ctypes.byref(lt), int(max_sweeps),
                                       LOCAL_HOST_ONLY if host_only else 0, ctypes.byref(h))
        _check(rc, "fs_local_create")
        self._h = h

    def info(self) -> dict:
        n, k, g, c2 = (ctypes.c_int32() for _ in range(4))
        ge, c2e = ctypes.c_int64(), ctypes.c_int64()
        sw = ctypes.c_int32()
        _check(self._lib.fs_local_info(self._h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(g),
                                       ctypes.byref(ge), ctypes.byref(c2), ctypes.byref(c2e),
                                       ctypes.byref(sw)), "fs_local_info")
        return dict(n=n.value, k_int=k.value, n_groups=g.value, group_entries=ge.value,
                    n_check2=c2.value, check2_entries=c2e.value, sweeps=sw.value)

    def groups(self):
        """Check #3 groups in repair order: (ptr, idx) int32 arrays."""
        i = self.info()
        ptr = np.zeros(i["n_groups"] + 1, np.int32)
        idx = np.zeros(max(i["group_entries"], 1), np.int32)
        _check(self._lib.fs_local_groups(self._h, ptr.ctypes.data, idx.ctypes.data),
               "fs_local_groups")
        return ptr, idx[:i["group_entries"]]

    def check2(self) -> dict:
        """Check #2 equations: {intermediate: tuple of coded blocks}."""
        i = self.info()
        inter = np.zeros(max(i["n_check2"], 1), np.int32)
        ptr = np.zeros(i["n_check2"] + 1, np.int32)
        idx = np.zeros(max(i["check2_entries"], 1), np.int32)
        _check(self._lib.fs_local_check2(self._h, inter.ctypes.data, ptr.ctypes.data,
                                         idx.ctypes.data), "fs_local_check2")
        return {int(inter[q]): tuple(int(x) for x in idx[ptr[q]:ptr[q + 1]])
                for q in range(i["n_check2"])}

    def workspace(self, device=None):
        import torch
        return torch.empty(max(int(self._lib.fs_local_workspace_bytes(self._h)), 256),
                           dtype=torch.uint8, device=device or "cuda")

    def repair(self, lost, coded, block_bytes: int, unrepaired, n_unrepaired, ws,
               stream=None) -> None:
        """Repairs the lost coded blocks of ``coded`` in place (fs_repair_local)."""
        need = ((lost, self.n, "lost"), (coded, self.n * int(block_bytes), "coded"),
                (unrepaired, self.n, "unrepaired"), (n_unrepaired, 4, "n_unrepaired"),
                (ws, int(self._lib.fs_local_workspace_bytes(self._h)), "ws"))
        for x, nbytes, name in need:
            if x is not None and not isinstance(x, int) and _nbytes(x) < nbytes:
                raise ValueError("%s holds %d bytes, needs %d" % (name, _nbytes(x), nbytes))
        _check(self._lib.fs_repair_local(self._h, _addr(lost), _addr(coded), int(block_bytes),
                                         _addr(unrepaired), _addr(n_unrepaired), _addr(ws),
                                         _stream(stream)), "fs_repair_local")

    def path(self, ws):
        """Levels of the last repair on ws (synchronises): list of sets {(f, g)}."""
        import torch
        v = _PathView()
        _check(self._lib.fs_local_path(self._h, _addr(ws), ctypes.byref(v)), "fs_local_path")
        base = ws.data_ptr()

        def at(ptr, count):
            off = ptr - base
            return ws[off:off + 4 * count].view(torch.int32).cpu().numpy()

        torch.cuda.synchronize()
        nl = int(at(v.n_levels, 1)[0])
        npairs = int(at(v.n_pairs, 1)[0])
        lo, f, g = at(v.level_off, nl + 1), at(v.pair_f, npairs), at(v.pair_g, npairs)
        return [set(zip(f[lo[l]:lo[l + 1]].tolist(), g[lo[l]:lo[l + 1]].tolist()))
                for l in range(nl)]

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.fs_local_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
