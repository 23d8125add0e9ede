"""The array LDPC precode (Algorithm 2, check #1): its checks against values
worked by hand, its structure (each block of checks reads data and parities of
earlier blocks only), and the oracle's encode / decode of a chained precode
pinned by identities the checks must satisfy on encoded bytes."""
import os

import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_checks_match_the_hand_worked_values():
    want = {}
    for line in open(os.path.join(GOLDEN, "array_ldpc_checks.txt")):
        if line.startswith("#") or not line.strip():
            continue
        b, k, r, *members = (int(x) for x in line.split())
        want[(b, k, r)] = members
    for (b, k, r), members in want.items():
        ptr, idx = gen.array_precode(b, k)
        assert idx[ptr[r]:ptr[r + 1]].tolist() == members
    ptr, idx = gen.array_precode(14, 21)
    assert ptr.size - 1 == 7 and idx.size == 14  # the whole k = 21 table is listed


@pytest.mark.parametrize("b,k", [(14, 21), (21, 35), (117, 143), (4154, 4288), (120, 150)])
def test_structure(b, k):
    """k - b checks of k' - j' distinct members each; check r reads only
    intermediates below b + r; a check of block j >= 1 reads a parity of block
    j - 1; every data block is read by some check."""
    ptr, idx = gen.array_precode(b, k)
    p = gen.largest_prime_factor(k)
    kp, jp = k // p, k // p - b // p
    assert ptr.size - 1 == k - b == jp * p
    seen = np.zeros(b, bool)
    for r in range(k - b):
        row = idx[ptr[r]:ptr[r + 1]]
        assert row.size == kp - jp and np.unique(row).size == row.size
        assert row.max() < b + r
        j = r // p
        if j >= 1:
            assert any(b + (j - 1) * p <= v < b + j * p for v in row)
        seen[row[row < b]] = True
    assert seen.all()


def test_bad_parameters_are_rejected():
    with pytest.raises(ValueError):
        gen.array_precode(10, 21)  # p = 7 does not divide b
    with pytest.raises(ValueError):
        gen.array_precode(21, 21)  # j' = 0: no checks


@pytest.mark.parametrize("b,k,n", [(21, 35, 50), (117, 143, 190)])
def test_oracle_encode_satisfies_every_check_and_decodes(b, k, n):
    """Every check (members + its parity b + r) XORs to zero on the encoded
    bytes, every coded block is the XOR of its row, and the joint decode of an
    erasure pattern returns the data."""
    g = gen.make_graph_array(b, k, n, gen.DIST_RSD, 0.1, 0.05, stripe=2)  # a ripple at this size
    t = 32
    data = gen.fill_bytes(gen.SEED_DATA + 2, b * t).reshape(b, t)
    par, cod = oracle.encode(g, data, t)
    inter = np.concatenate([data, par])
    for r in range(g.m):
        acc = inter[b + r].copy()
        for v in g.pre_idx[g.pre_ptr[r]:g.pre_ptr[r + 1]]:
            acc ^= inter[v]
        assert not acc.any()
    for s in range(n):
        acc = np.zeros(t, np.uint8)
        for v in g.lt_idx[g.lt_ptr[s]:g.lt_ptr[s + 1]]:
            acc ^= inter[v]
        assert np.array_equal(acc, cod[s])
    er = np.zeros(n, np.uint8)
    er[gen.sample_indices(n, gen.round_count(0.1, n), gen.SEED_ERASE + 2)] = 1
    out, path = oracle.decode(g, cod, er, t)
    ok = path.unrecovered[:b] == 0
    assert ok.sum() > 0 and np.array_equal(out[ok], data[ok])


def test_library_local_groups_on_a_chained_code():
    """The library's check #2 / check #3 equations of an array-precoded code
    (host only) equal the oracle's."""
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph_array(117, 143, 190, gen.DIST_FINITE40, stripe=2)
    want = oracle.local_groups(g)
    loc = fs.Local(g, host_only=True)
    ptr, idx = loc.groups()
    wptr, widx = want.csr()
    assert np.array_equal(ptr, wptr) and np.array_equal(idx, widx)
    assert loc.check2() == want.check2
