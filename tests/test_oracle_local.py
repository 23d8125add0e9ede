"""The oracle's local recovery groups (Algorithm 4 and the two set-XOR
derivations) and its repair from check #3 groups, pinned against the paper's
printed example, a closed form of Algorithm 4, identities the groups must
satisfy on encoded bytes, and hand-worked repair schedules."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _graph_from_rows(b, rows, checks=()):
    def csr(rs):
        ptr = np.zeros(len(rs) + 1, np.int32)
        for j, r in enumerate(rs):
            ptr[j + 1] = ptr[j] + len(r)
        return ptr, np.array([v for r in rs for v in sorted(r)], dtype=np.int32)
    lp, li = csr(rows)
    pp, pi = csr(list(checks))
    return gen.Graph(b, len(checks), len(rows), pp, pi, lp, li)


def test_setxor_matches_the_printed_example():
    check2, want = {}, None
    for line in open(os.path.join(GOLDEN, "setxor_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "check2":
            check2[int(f[1])] = tuple(int(x) for x in f[2:])
        else:
            want = tuple(int(x) for x in f[1:])
    assert oracle.set_xor(*check2.values()) == want


def test_setxor_derivation_on_precode_checks():
    """The second derivation: each check #1 group (a precode check's members
    and its parity) whose members all have check #2 sets contributes the set
    XOR of those sets as a check #3 group."""
    g = gen.make_graph(60, 6, 90, gen.DIST_FINITE40, stripe=0)
    lg = oracle.local_groups(g)
    pp, pi = np.asarray(g.pre_ptr), np.asarray(g.pre_idx)
    derived = 0
    for j in range(g.m):
        members = [int(x) for x in pi[pp[j]:pp[j + 1]]] + [g.b + j]
        if all(v in lg.check2 for v in members):
            grp = oracle.set_xor(*[lg.check2[v] for v in members])
            assert not grp or grp in lg.check3
            derived += 1
    assert derived == g.m


def test_setxor_derivation_on_degree_one_blocks():
    """The first derivation: a coded block s of degree one (s = intermediate
    i) and the check #2 set S of i give the check #3 group S XOR {s} (which is
    empty when S is {s} itself)."""
    g = gen.make_graph(200, 0, 260, gen.DIST_RSD, 0.1, 0.05, stripe=4)
    lg = oracle.local_groups(g)
    lp, li = np.asarray(g.lt_ptr), np.asarray(g.lt_idx)
    ones = [s for s in range(g.n) if lp[s + 1] - lp[s] == 1 and int(li[lp[s]]) in lg.check2]
    new = 0
    for s in ones:
        grp = oracle.set_xor(lg.check2[int(li[lp[s]])], (s,))
        assert not grp or grp in lg.check3
        new += bool(grp)
    assert len(ones) > 0 and new > 0


def _cga_brute(g, cols):
    """Recomputes b_j as the XOR of the original columns named by l_j."""
    lp, li = np.asarray(g.lt_ptr), np.asarray(g.lt_idx)
    for c in cols:
        b = oracle.set_xor(*[li[lp[s]:lp[s + 1]] for s in c.l]) if c.l else ()
        assert len(b) == c.w
        assert c.e == (b[0] if len(b) == 1 else -1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cga_columns_stay_xors_of_their_sets(seed):
    g = gen.make_graph(80, 0, 110, gen.DIST_RSD, 0.1, 0.05, stripe=seed)
    sweeps, cols = oracle.cga(g)
    assert sweeps >= 1 and len(cols) == g.n
    _cga_brute(g, cols)


def test_cga_stops_at_a_fixed_point_or_at_n_minus_k_zero_columns():
    """After Algorithm 4 returns, either n - k columns are zero or no pair
    (j, i) meets the replacement rule any more (the last sweep changed
    nothing)."""
    for seed in range(4):
        g = gen.make_graph(40, 0, 52, gen.DIST_FINITE40, stripe=seed)
        _, cols = oracle.cga(g)
        zero = sum(c.w == 0 for c in cols)
        if zero >= g.n - g.k_int:
            continue
        lp, li = np.asarray(g.lt_ptr), np.asarray(g.lt_idx)
        B = [set(oracle.set_xor(*[li[lp[s]:lp[s + 1]] for s in c.l])) for c in cols]
        for j, i in itertools.permutations(range(g.n), 2):
            assert not (2 * len(B[j]) > len(B[i]) and len(B[j] ^ B[i]) < len(B[j]))


def test_cga_closed_form_on_identity_plus_random_columns():
    """B = [I_k | R]: the unit columns stay (check #2: intermediate i is coded
    block i) and each column j >= k reduces to zero against the unit columns
    of its members, leaving the check #3 group {j} + R_j."""
    k, extra = 12, 7
    rng = np.random.default_rng(5)
    rows = [[i] for i in range(k)]
    for _ in range(extra):
        rows.append(sorted(rng.choice(k, size=int(rng.integers(2, 6)), replace=False).tolist()))
    g = _graph_from_rows(k, rows)
    sweeps, cols = oracle.cga(g)
    for i in range(k):
        assert cols[i].w == 1 and cols[i].e == i and cols[i].l == (i,)
    for j in range(k, k + extra):
        assert cols[j].w == 0 and cols[j].l == tuple(sorted([j] + rows[j]))
    lg = oracle.local_groups(g)
    assert lg.check2 == {i: (i,) for i in range(k)}
    assert sorted(lg.check3) == sorted(tuple(sorted([j] + rows[j])) for j in range(k, k + extra))
    assert [len(x) for x in lg.check3] == sorted(len(x) for x in lg.check3)


@pytest.mark.parametrize("shape", [(100, 0, 150, gen.DIST_RSD), (300, 12, 400, gen.DIST_FINITE40)])
def test_groups_hold_on_encoded_bytes(shape):
    """Every check #3 group XORs to zero and every check #2 set XORs to its
    intermediate, on real encoded bytes (Section 2.2 encoding)."""
    b, m, n, dist = shape
    g = gen.make_graph(b, m, n, dist, 0.1, 0.05) if dist == gen.DIST_RSD else gen.make_graph(b, m, n, dist)
    t = 32
    data = gen.fill_bytes(gen.SEED_DATA, b * t).reshape(b, t)
    parity, coded = oracle.encode(g, data, t)
    inter = np.concatenate([data, parity]) if m else data
    lg = oracle.local_groups(g)
    assert lg.check3 and lg.check2
    for grp in lg.check3:
        acc = np.zeros(t, np.uint8)
        for s in grp:
            acc ^= coded[s]
        assert not acc.any()
    for i, grp in lg.check2.items():
        acc = np.zeros(t, np.uint8)
        for s in grp:
            acc ^= coded[s]
        assert np.array_equal(acc, inter[i])


def _csr(groups):
    ptr = np.zeros(len(groups) + 1, np.int32)
    for q, grp in enumerate(groups):
        ptr[q + 1] = ptr[q] + len(grp)
    return ptr, np.array([x for grp in groups for x in grp], dtype=np.int32)


def test_repair_schedule_by_hand():
    """Groups over coded blocks 0..5: g0 = {0, 1}, g1 = {1, 2, 3}, g2 = {1, 4},
    g3 = {3, 5}. Lost {0, 1, 3}: level 0 offers 1 (g2: only unknown 1) and 3
    (g3); g1 has two unknowns. Level 1: g0 offers 0. Block 1 comes from g2 (its
    only offer), not g1."""
    ptr, idx = _csr([(0, 1), (1, 2, 3), (1, 4), (3, 5)])
    lost = np.array([1, 1, 0, 1, 0, 0], np.uint8)
    path = oracle.local_path(ptr, idx, 6, lost)
    assert path.levels() == [{(1, 2), (3, 3)}, {(0, 0)}]
    assert not path.unrepaired.any()


def test_repair_takes_the_smallest_group():
    """Block 0 lost, offered by g0 = {0, 1, 2} and g1 = {0, 3}: the smaller g1
    wins; with equal sizes the lower index wins."""
    ptr, idx = _csr([(0, 1, 2), (0, 3)])
    assert oracle.local_path(ptr, idx, 4, np.array([1, 0, 0, 0], np.uint8)).levels() == [{(0, 1)}]
    ptr, idx = _csr([(0, 1), (0, 3)])
    assert oracle.local_path(ptr, idx, 4, np.array([1, 0, 0, 0], np.uint8)).levels() == [{(0, 0)}]
    ptr, idx = _csr([(0, 1, 2)])  # two unknowns: nothing to repair
    path = oracle.local_path(ptr, idx, 3, np.array([1, 1, 0], np.uint8))
    assert path.n_pairs == 0 and path.unrepaired.tolist() == [1, 1, 0]


def _closure(groups, lost):
    """The repaired set by immediate peeling, in any order (BP's result does
    not depend on the order)."""
    unknown = set(np.nonzero(lost)[0].tolist())
    changed = True
    while changed:
        changed = False
        for grp in groups:
            u = [s for s in grp if s in unknown]
            if len(u) == 1:
                unknown.discard(u[0])
                changed = True
    return unknown


@pytest.mark.parametrize("frac", [0.02, 0.1, 0.3])
def test_repair_recovers_the_stored_blocks(frac):
    g = gen.make_graph(300, 12, 400, gen.DIST_FINITE40, stripe=1)
    t = 48
    data = gen.fill_bytes(gen.SEED_DATA + 7, g.b * t).reshape(g.b, t)
    _, coded = oracle.encode(g, data, t)
    lg = oracle.local_groups(g)
    ptr, idx = lg.csr()
    lost = np.zeros(g.n, np.uint8)
    lost[gen.sample_indices(g.n, gen.round_count(frac, g.n), gen.SEED_ERASE + 3)] = 1
    out, path = oracle.repair_local(ptr, idx, coded, lost, t)
    left = _closure(lg.check3, lost)
    assert set(np.nonzero(path.unrepaired)[0].tolist()) == left
    ok = ~path.unrepaired.astype(bool)
    assert np.array_equal(out[ok], coded[ok])
    assert not out[path.unrepaired.astype(bool)].any()
    assert path.n_pairs == int(lost.sum()) - len(left) > 0


@pytest.mark.parametrize("seed", range(6))
def test_repair_schedule_obeys_the_rules(seed):
    """Random groups and lost sets: every level is exactly the set of lost
    blocks that some group with one unknown names (against the state at the
    level start), each from its smallest (cardinality, index) such group, and
    the unrepaired blocks are the lost blocks no level reached."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 120))
    groups = [tuple(sorted(rng.choice(n, size=int(rng.integers(2, 9)), replace=False).tolist()))
              for _ in range(int(rng.integers(5, 60)))]
    lost = (rng.random(n) < rng.uniform(0.05, 0.5)).astype(np.uint8)
    ptr, idx = _csr(groups)
    path = oracle.local_path(ptr, idx, n, lost)
    unknown = set(np.nonzero(lost)[0].tolist())
    for pairs in path.levels():
        cand = {}
        for q, grp in enumerate(groups):
            u = [s for s in grp if s in unknown]
            if len(u) == 1:
                cand.setdefault(u[0], []).append((len(grp), q))
        assert {f for f, _ in pairs} == set(cand)
        for f, q in pairs:
            assert (len(groups[q]), q) == min(cand[f])
        unknown -= {f for f, _ in pairs}
    assert set(np.nonzero(path.unrepaired)[0].tolist()) == unknown
