"""CPU oracle for the Founsure GF(2) gather-XOR path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain byte loops, built with gcc); this
module only marshals numpy arrays. Each function names the passage it
follows:

* :func:`encode`   - Section 2.2 encoding steps (1) precode, (2) LDGM.
* :func:`dpg`      - Algorithm 5 (Decoding Path Generation), Section 3.2.
* :func:`peel`     - the payload of the decoding path (Section 3.1).
* :func:`decode`   - :func:`dpg` then :func:`peel`.
* :func:`peel_immediate` - Algorithm 1 with immediate updates, any order.
* :func:`update`   - a data rewrite followed by a full re-encode (the
  definition the delta update must reproduce).
* :func:`repair`   - lost coded rows recomputed by the encoding definition.
* :func:`cga`      - Algorithm 4 (Check Generation Algorithm).
* :func:`set_xor`  - the set XOR of the check #1 derivation (Section
  "Generating Information for Efficient Repair").
* :func:`local_groups` - check #2 equations and ordered check #3 groups:
  CGA, the two setXOR derivations of that section, smallest group first.
* :func:`local_path` / :func:`repair_local` - repair of lost coded blocks by
  peeling over the check #3 groups, level by level like Algorithm 5.

Readings of the paper: see the header of ``oracle.c``. The decoding
*schedule* (which g decodes which f, level by level) follows from the stated
tie-break (lowest original degree, then lowest constraint index); the tests
check every level of it against the rules with a checker of their own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "oracle.c")
_LIB = os.path.join(_DIR, "liboracle.so")

MODE_JOINT = 0
MODE_TWO_PASS = 1

_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c with gcc (plain -O2, no OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        tmp = _LIB + ".tmp%d" % os.getpid()
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.or_encode.argtypes = [i32, i32, i32, vp, vp, vp, vp, i64, vp, vp, vp]
        L.or_encode.restype = ctypes.c_int
        L.or_dpg.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]
        L.or_dpg.restype = i32
        L.or_peel.argtypes = [i32, i32, i32, vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp]
        L.or_peel.restype = ctypes.c_int
        L.or_peel_immediate.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_peel_immediate.restype = i32
        L.or_cga.argtypes = [i32, i32, vp, vp, i32, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)),
                             ctypes.POINTER(ctypes.c_int64)]
        L.or_cga.restype = i32
        L.or_free.argtypes = [vp]
        L.or_free.restype = None
        L.or_local_dpg.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_local_dpg.restype = i32
        L.or_local_peel.argtypes = [i32, vp, vp, i64, vp, i32, vp, vp]
        L.or_local_peel.restype = ctypes.c_int
        _lib = L
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _p(a: np.ndarray):
    return a.ctypes.data if a.size else None


class _G:
    """Contiguous int32 copies of a graph's CSR arrays (b, m, n + 4 arrays)."""

    def __init__(self, g):
        self.b, self.m, self.n = int(g.b), int(g.m), int(g.n)
        self.pp = _i32(g.pre_ptr) if g.m > 0 else np.zeros(1, np.int32)
        self.pi = _i32(g.pre_idx) if g.pre_idx.size else np.zeros(1, np.int32)
        self.lp = _i32(g.lt_ptr)
        self.li = _i32(g.lt_idx) if g.lt_idx.size else np.zeros(1, np.int32)

    def args(self):
        return (self.b, self.m, self.n, _p(self.pp), _p(self.pi), _p(self.lp), _p(self.li))


def encode(g, data: np.ndarray, t: int):
    """Section 2.2 encoding. ``data`` holds b*t bytes. Returns (parity, coded)
    as (m, t) and (n, t) uint8 arrays."""
    G = _G(g)
    data = _u8(data).reshape(-1)
    assert data.size == G.b * t
    parity = np.zeros((max(G.m, 0), t), dtype=np.uint8)
    coded = np.zeros((G.n, t), dtype=np.uint8)
    rc = lib().or_encode(*G.args(), t, _p(data), _p(parity) if G.m else None, _p(coded))
    if rc != 0:
        raise ValueError("or_encode: bad graph index")
    return parity, coded


@dataclass
class Path:
    """A decoding path: pairs (f, g) in level order, ascending f in a level."""
    pair_f: np.ndarray
    pair_g: np.ndarray
    level_of: np.ndarray
    n_levels: int
    unrecovered: np.ndarray  # uint8 flags over the k_int intermediates

    @property
    def n_pairs(self) -> int:
        return int(self.pair_f.size)

    def levels(self):
        """List of per-level sets {(f, g)}: the part of the path that does not
        depend on how pairs are ordered inside a level."""
        out = [set() for _ in range(self.n_levels)]
        for f, g, l in zip(self.pair_f.tolist(), self.pair_g.tolist(), self.level_of.tolist()):
            out[l].add((f, g))
        return out


def dpg(g, erased: np.ndarray, mode: int = MODE_JOINT) -> Path:
    """Algorithm 5 over the surviving coded rows (erased[j] != 0 drops row j)
    and, in joint mode, the precode checks."""
    G = _G(g)
    k_int = G.b + G.m
    erased = _u8(erased)
    assert erased.size == G.n
    pf = np.zeros(max(k_int, 1), np.int32)
    pg = np.zeros(max(k_int, 1), np.int32)
    lv = np.zeros(max(k_int, 1), np.int32)
    unrec = np.zeros(max(k_int, 1), np.uint8)
    nl = ctypes.c_int32(0)
    npairs = lib().or_dpg(*G.args(), _p(erased) if G.n else None, mode, _p(pf), _p(pg), _p(lv),
                          _p(unrec), ctypes.byref(nl))
    if npairs < 0:
        raise MemoryError("or_dpg failed (%d)" % npairs)
    return Path(pf[:npairs].copy(), pg[:npairs].copy(), lv[:npairs].copy(), int(nl.value),
                unrec[:k_int].copy())


def peel(g, coded: np.ndarray, path: Path, t: int, with_parity: bool = False):
    """Payload of a decoding path. Returns data (b, t) [and parity (m, t)]."""
    G = _G(g)
    coded = _u8(coded).reshape(-1)
    assert coded.size == G.n * t
    data = np.zeros((G.b, t), np.uint8)
    parity = np.zeros((G.m, t), np.uint8) if with_parity else None
    rc = lib().or_peel(*G.args(), t, _p(coded), path.n_pairs, _p(_i32(path.pair_f)),
                       _p(_i32(path.pair_g)), _p(data),
                       _p(parity) if (with_parity and G.m) else None)
    if rc != 0:
        raise MemoryError("or_peel failed")
    return (data, parity) if with_parity else data


def decode(g, coded: np.ndarray, erased: np.ndarray, t: int, mode: int = MODE_JOINT):
    """Algorithm 5 then its payload. Returns (data (b, t), Path)."""
    path = dpg(g, erased, mode)
    return peel(g, coded, path, t), path


def peel_immediate(g, erased: np.ndarray, order: np.ndarray, with_sweeps: bool = False):
    """Algorithm 1 with immediate updates over constraints visited in
    ``order`` (a permutation of 0..n+m-1). Returns the unrecovered flags, and
    with ``with_sweeps`` also the number of sweeps that decoded something
    (the iteration count t_m of Section 3.1)."""
    G = _G(g)
    k_int = G.b + G.m
    unrec = np.zeros(max(k_int, 1), np.uint8)
    order = _i32(order)
    assert order.size == G.n + G.m
    sw = ctypes.c_int32(0)
    lib().or_peel_immediate(*G.args(), _p(_u8(erased)) if G.n else None, _p(order), _p(unrec),
                            ctypes.byref(sw))
    if with_sweeps:
        return unrec[:k_int].copy(), int(sw.value)
    return unrec[:k_int].copy()


def update(g, data: np.ndarray, idx: np.ndarray, new_blocks: np.ndarray, t: int):
    """Rewrites data blocks idx[q] with new_blocks[q], then re-encodes.
    Returns (data', parity', coded')."""
    d = _u8(data).reshape(g.b, t).copy()
    d[_i32(idx)] = _u8(new_blocks).reshape(-1, t)
    parity, coded = encode(g, d, t)
    return d, parity, coded


def repair(g, data: np.ndarray, lost: np.ndarray, t: int) -> np.ndarray:
    """The lost coded rows recomputed from the intermediates by the encoding
    definition. Returns (len(lost), t)."""
    _, coded = encode(g, data, t)
    return coded[_i32(lost)].copy()


# ---------------------------------------------------------------------------
# local recovery groups and repair from them

@dataclass
class CgaColumn:
    """Column j of B and L after Algorithm 4: w = w(b_j), e = the single
    intermediate of b_j when w == 1 (else -1), l = the coded blocks of l_j."""
    w: int
    e: int
    l: tuple


def cga(g, max_sweeps: int = 0):
    """Algorithm 4 on the LT generator matrix of g (k = k_int rows, n
    columns). Returns (sweeps, [CgaColumn per coded block])."""
    G = _G(g)
    out = ctypes.POINTER(ctypes.c_int32)()
    ln = ctypes.c_int64(0)
    sweeps = lib().or_cga(G.b + G.m, G.n, _p(G.lp), _p(G.li), max_sweeps, ctypes.byref(out),
                          ctypes.byref(ln))
    if sweeps < 0:
        raise MemoryError("or_cga failed")
    arr = np.ctypeslib.as_array(out, shape=(ln.value,)).copy() if ln.value else np.zeros(0, np.int32)
    lib().or_free(out)
    cols, o = [], 0
    for _ in range(G.n):
        w, e, k = int(arr[o]), int(arr[o + 1]), int(arr[o + 2])
        cols.append(CgaColumn(w, e, tuple(int(x) for x in arr[o + 3:o + 3 + k])))
        o += 3 + k
    return int(sweeps), cols


def set_xor(*sets) -> tuple:
    """XOR (symmetric difference) of index sets, as a sorted tuple: the set of
    coded blocks whose XOR equals the XOR of the given equations' sides."""
    acc = set()
    for s in sets:
        for x in s:
            acc ^= {int(x)}
    return tuple(sorted(acc))


@dataclass
class LocalGroups:
    """check2[i]: coded blocks whose XOR is intermediate i (the first CGA
    column that reduced to {i}); check3: coded-only zero-sum groups, smallest
    first; sweeps: Algorithm 4 sweeps run."""
    check2: dict
    check3: list
    sweeps: int

    def csr(self):
        """check3 as CSR (ptr, idx) int32 arrays."""
        ptr = np.zeros(len(self.check3) + 1, np.int32)
        for q, grp in enumerate(self.check3):
            ptr[q + 1] = ptr[q] + len(grp)
        idx = np.array([x for grp in self.check3 for x in grp], dtype=np.int32)
        return ptr, idx


def local_groups(g, max_sweeps: int = 0) -> LocalGroups:
    """Check #2 and check #3 equations of g (Section "Generating Information
    for Efficient Repair" and Algorithm 4):
      1. Algorithm 4: zero columns give check #3 groups (column order), unit
         columns check #2 equations (the first column per intermediate);
      2. every coded block s of degree one (N(s) = {i}) with a check #2 set S
         for i adds the group S XOR {s} (the first method);
      3. every precode check j whose members and parity b+j all have check #2
         sets adds the XOR of those sets (the second method, Equation
         setXOR);
      4. empty groups are dropped and repeated groups kept once (first
         occurrence); the groups are ordered by cardinality, ties in the order
         of steps 1-3 (the paper's qsort by cardinality)."""
    sweeps, cols = cga(g, max_sweeps)
    check2, check3 = {}, []
    for c in cols:
        if c.w == 0:
            check3.append(c.l)
        elif c.w == 1 and c.e not in check2:
            check2[c.e] = c.l
    lp, li = np.asarray(g.lt_ptr), np.asarray(g.lt_idx)
    for s in range(int(g.n)):
        row = set_xor(li[lp[s]:lp[s + 1]])
        if len(row) == 1 and row[0] in check2:
            check3.append(set_xor(check2[row[0]], (s,)))
    pp, pi = np.asarray(g.pre_ptr), np.asarray(g.pre_idx)
    for j in range(int(g.m)):
        members = [int(x) for x in pi[pp[j]:pp[j + 1]]] + [int(g.b) + j]
        if all(v in check2 for v in members):
            check3.append(set_xor(*[check2[v] for v in members]))
    seen, uniq = set(), []
    for grp in check3:
        if grp and grp not in seen:
            seen.add(grp)
            uniq.append(grp)
    order = sorted(range(len(uniq)), key=lambda q: (len(uniq[q]), q))
    return LocalGroups(check2, [uniq[q] for q in order], sweeps)


@dataclass
class RepairPath:
    """Pairs (f, g): coded block f repaired from group g, in level order."""
    pair_f: np.ndarray
    pair_g: np.ndarray
    level_of: np.ndarray
    n_levels: int
    unrepaired: np.ndarray  # uint8 flags over the n coded blocks

    @property
    def n_pairs(self) -> int:
        return int(self.pair_f.size)

    def levels(self):
        out = [set() for _ in range(self.n_levels)]
        for f, g, l in zip(self.pair_f.tolist(), self.pair_g.tolist(), self.level_of.tolist()):
            out[l].add((f, g))
        return out


def local_path(g_ptr, g_idx, n: int, lost: np.ndarray) -> RepairPath:
    """Repair schedule over check #3 groups (CSR over coded blocks)."""
    g_ptr, g_idx, lost = _i32(g_ptr), _i32(g_idx), _u8(lost)
    assert lost.size == n
    G = g_ptr.size - 1
    pf = np.zeros(max(n, 1), np.int32)
    pg = np.zeros(max(n, 1), np.int32)
    lv = np.zeros(max(n, 1), np.int32)
    un = np.zeros(max(n, 1), np.uint8)
    nl = ctypes.c_int32(0)
    np_ = lib().or_local_dpg(n, G, _p(g_ptr), _p(g_idx) if g_idx.size else None, _p(lost),
                             _p(pf), _p(pg), _p(lv), _p(un), ctypes.byref(nl))
    if np_ < 0:
        raise MemoryError("or_local_dpg failed")
    return RepairPath(pf[:np_].copy(), pg[:np_].copy(), lv[:np_].copy(), int(nl.value),
                      un[:n].copy())


def repair_local(g_ptr, g_idx, coded: np.ndarray, lost: np.ndarray, t: int):
    """Lost coded blocks repaired from the check #3 groups. coded (n, t) holds
    the stored blocks (the lost ones are ignored). Returns (coded' (n, t) with
    repaired blocks filled in and unrepaired lost blocks zero, RepairPath)."""
    coded = _u8(coded).reshape(-1, t)
    n = coded.shape[0]
    path = local_path(g_ptr, g_idx, n, lost)
    out = coded.copy()
    out[_u8(lost).astype(bool)] = 0
    g_ptr, g_idx = _i32(g_ptr), _i32(g_idx)
    lib().or_local_peel(n, _p(g_ptr), _p(g_idx) if g_idx.size else None, t, _p(out), path.n_pairs,
                        _p(_i32(path.pair_f)), _p(_i32(path.pair_g)))
    return out, path
