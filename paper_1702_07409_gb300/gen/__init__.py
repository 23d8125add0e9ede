"""Seeded synthetic inputs for the Founsure GF(2) gather-XOR path.

A thin ctypes layer over ``libfsgen.so`` (``include/fs_gen.h`` states every
definition: splitmix64, the Robust Soliton and FiniteDist degree
distributions of Section 2.2, Floyd neighbour sampling, the random
left-regular precode, partial Fisher-Yates index draws and the counter-based
byte stream). It produces inputs only; no block arithmetic happens here.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .. import _build

SEED_GRAPH = 1389488782
SEED_PRECODE = SEED_GRAPH + 1
SEED_DATA = 1
SEED_ERASE = 2
SEED_UPDATE = 3
SEED_REPAIR = 4
SEED_NEWDATA = 5
STRIPE_SHIFT = 32
ROUND_SHIFT = 20

DIST_RSD = 0
DIST_FINITE65 = 1
DIST_FINITE40 = 2
DIST_FINITE40_FOLD = 3

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build_gen()
        L = ctypes.CDLL(path)
        u64, i32, i64, dbl, vp = (ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_double, ctypes.c_void_p)
        L.fsg_next.argtypes = [ctypes.POINTER(u64)]
        L.fsg_next.restype = u64
        L.fsg_at.argtypes = [u64, u64]
        L.fsg_at.restype = u64
        L.fsg_uniform_int.argtypes = [ctypes.POINTER(u64), u64]
        L.fsg_uniform_int.restype = u64
        L.fsg_uniform_double.argtypes = [ctypes.POINTER(u64)]
        L.fsg_uniform_double.restype = dbl
        L.fsg_fill_bytes.argtypes = [u64, u64, u64, vp]
        L.fsg_fill_bytes.restype = ctypes.c_int
        L.fsg_pmf.argtypes = [i32, i32, dbl, dbl, vp, i32, vp]
        L.fsg_pmf.restype = ctypes.c_int
        L.fsg_lt_graph_nnz.argtypes = [i32, i32, vp, i32, u64]
        L.fsg_lt_graph_nnz.restype = i64
        L.fsg_lt_graph.argtypes = [i32, i32, vp, i32, u64, vp, vp, i64]
        L.fsg_lt_graph.restype = i64
        L.fsg_precode_graph.argtypes = [i32, i32, i32, u64, vp, vp, i64]
        L.fsg_precode_graph.restype = i64
        L.fsg_sample_indices.argtypes = [i32, i32, u64, vp]
        L.fsg_sample_indices.restype = ctypes.c_int
        L.fsg_round_count.argtypes = [dbl, i32]
        L.fsg_round_count.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def stream(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of splitmix64 seeded with ``seed``."""
    st = ctypes.c_uint64(seed & (2**64 - 1))
    return np.array([lib().fsg_next(ctypes.byref(st)) for _ in range(count)], dtype=np.uint64)


def uniform_ints(seed: int, r: int, count: int) -> np.ndarray:
    st = ctypes.c_uint64(seed & (2**64 - 1))
    return np.array([lib().fsg_uniform_int(ctypes.byref(st), r) for _ in range(count)],
                    dtype=np.uint64)


def uniform_doubles(seed: int, count: int) -> np.ndarray:
    st = ctypes.c_uint64(seed & (2**64 - 1))
    return np.array([lib().fsg_uniform_double(ctypes.byref(st)) for _ in range(count)])


def fill_bytes(seed: int, nbytes: int, offset: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty(nbytes, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= nbytes
    rc = lib().fsg_fill_bytes(seed & (2**64 - 1), offset, nbytes, _ptr(out))
    if rc != 0:
        raise ValueError("fsg_fill_bytes failed")
    return out


def pmf(kind: int, k: int = 0, c: float = 0.0, delta: float = 0.0):
    """Returns (mu, dmax, info) with mu indexed by degree."""
    length = k + 1 if kind == DIST_RSD else 66
    mu = np.zeros(length, dtype=np.float64)
    info = np.zeros(4, dtype=np.float64)
    dmax = lib().fsg_pmf(kind, k, c, delta, _ptr(mu), length, _ptr(info))
    if dmax < 1:
        raise ValueError("fsg_pmf failed (%d)" % dmax)
    return mu, dmax, info


def round_count(fraction: float, n: int) -> int:
    return int(lib().fsg_round_count(fraction, n))


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    out = np.empty(max(count, 1), dtype=np.int32)
    if lib().fsg_sample_indices(n, count, seed & (2**64 - 1), _ptr(out)) != 0:
        raise ValueError("fsg_sample_indices failed")
    return out[:count].copy()


def lt_graph(k_int: int, n: int, mu: np.ndarray, dmax: int, seed: int):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    nnz = lib().fsg_lt_graph_nnz(k_int, n, _ptr(mu), dmax, seed & (2**64 - 1))
    if nnz < 0:
        raise ValueError("fsg_lt_graph_nnz failed")
    ptr = np.empty(n + 1, dtype=np.int32)
    idx = np.empty(max(nnz, 1), dtype=np.int32)
    got = lib().fsg_lt_graph(k_int, n, _ptr(mu), dmax, seed & (2**64 - 1), _ptr(ptr), _ptr(idx), nnz)
    if got != nnz:
        raise ValueError("fsg_lt_graph failed (%d)" % got)
    return ptr, idx[:nnz].copy()


def precode_graph(b: int, m: int, q: int, seed: int):
    qq = min(q, m)
    cap = b * qq
    ptr = np.empty(m + 1, dtype=np.int32)
    idx = np.empty(max(cap, 1), dtype=np.int32)
    got = lib().fsg_precode_graph(b, m, q, seed & (2**64 - 1), _ptr(ptr), _ptr(idx), cap)
    if got != cap:
        raise ValueError("fsg_precode_graph failed (%d)" % got)
    return ptr, idx[:cap].copy()


@dataclass
class Graph:
    """A Founsure code graph: m precode checks over b data blocks (CSR, rows =
    checks) and n LT rows over k_int = b + m intermediates (CSR, rows = coded
    blocks). Intermediates are data 0..b-1 followed by parities b..b+m-1.
    chained: the precode's members are intermediates, check j's below b + j
    (its own parity b + j is not listed), as in the array LDPC precode."""
    b: int
    m: int
    n: int
    pre_ptr: np.ndarray
    pre_idx: np.ndarray
    lt_ptr: np.ndarray
    lt_idx: np.ndarray
    chained: bool = False

    @property
    def k_int(self) -> int:
        return self.b + self.m

    @property
    def e_lt(self) -> int:
        return int(self.lt_ptr[-1])

    @property
    def e_pre(self) -> int:
        return int(self.pre_ptr[-1])


def make_graph(b: int, m: int, n: int, dist: int, c: float = 0.0, delta: float = 0.0,
               q: int = 3, stripe: int = 0, seed_graph: int = SEED_GRAPH) -> Graph:
    """Draws a graph: the precode first (stream seed_graph+1), then the LT rows
    (stream seed_graph). The degree distribution is over k_int inputs."""
    k_int = b + m
    off = stripe << STRIPE_SHIFT
    mu, dmax, _ = pmf(dist, k_int, c, delta)
    if m > 0:
        pp, pi = precode_graph(b, m, q, seed_graph + 1 + off)
    else:
        pp, pi = np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32)
    lp, li = lt_graph(k_int, n, mu, dmax, seed_graph + off)
    return Graph(b, m, n, pp, pi, lp, li)


def largest_prime_factor(x: int) -> int:
    f, best = 2, 1
    while f * f <= x:
        while x % f == 0:
            best, x = f, x // f
        f += 1
    return x if x > 1 else best


def array_precode(b: int, k: int):
    """The array LDPC checks (check #1) of Algorithm 2 for b data blocks and k
    intermediates: p = the largest prime factor of k, k' = k / p,
    j' = k' - b / p. Check r = i + j p (j < j', i < p) has the k' - j'
    members
        k' p - (j' - j + m - 1) p - ((m (j' - j - 1) - i - 1 + p) mod p) - 1,
    m = 1 .. k' - j', and its parity is intermediate b + r. The members of the
    checks of block j are data blocks and parities of blocks j-1, j-2, ...,
    so the parities are computed block by block. Returns the CSR (ptr, idx)
    of the m = k - b checks, members ascending. Needs p | b and 1 <= j' < k'."""
    p = largest_prime_factor(k)
    kp = k // p
    if k < 2 or b <= 0 or b % p or not (1 <= kp - b // p < kp):
        raise ValueError("no array LDPC code for b=%d, k=%d (p=%d)" % (b, k, p))
    jp = kp - b // p
    rows = []
    for j in range(jp):
        for i in range(p):
            rows.append(sorted(kp * p - (jp - j + mm - 1) * p - ((mm * (jp - j - 1) - i - 1 + p) % p) - 1
                               for mm in range(1, kp - jp + 1)))
    ptr = np.zeros(len(rows) + 1, np.int32)
    for r, row in enumerate(rows):
        ptr[r + 1] = ptr[r] + len(row)
    return ptr, np.array([v for row in rows for v in row], dtype=np.int32)


def make_graph_array(b: int, k: int, n: int, dist: int, c: float = 0.0, delta: float = 0.0,
                     stripe: int = 0, seed_graph: int = SEED_GRAPH) -> Graph:
    """A graph with the array LDPC precode of Algorithm 2 (k - b chained
    checks) and LT rows over the k intermediates drawn as in make_graph."""
    off = stripe << STRIPE_SHIFT
    mu, dmax, _ = pmf(dist, k, c, delta)
    pp, pi = array_precode(b, k)
    lp, li = lt_graph(k, n, mu, dmax, seed_graph + off)
    return Graph(b, k - b, n, pp, pi, lp, li, chained=True)


def n_for_rate(k: int) -> int:
    """n = floor((13k+5)/10), the stated reading of "n = 1.3k"."""
    return (13 * k + 5) // 10
