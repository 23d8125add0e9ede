"""Pins for the CPU oracle against facts the paper and the mathematics fix:
a GF(2) matrix product computed another way, linearity, decode(encode(x)) = x,
brute-force Gaussian elimination over every erasure subset of tiny graphs
(the simDisk idea of Section 2.1), independence of the peeling fixpoint from
the visiting order (Section 3.1), |DP| = 2k on success (Section 3.2), and
update = re-encode / repair = pre-loss bytes."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen


def _rand_graph(rng, b, m, n, max_deg, q=2):
    """A small graph drawn with numpy (independent of the generator)."""
    k_int = b + m
    pre_rows = [[] for _ in range(m)]
    if m:
        for i in range(b):
            for j in rng.choice(m, size=min(q, m), replace=False):
                pre_rows[j].append(i)
    pp = np.zeros(m + 1, np.int32)
    for j in range(m):
        pp[j + 1] = pp[j] + len(pre_rows[j])
    pi = np.array([v for r in pre_rows for v in sorted(r)], dtype=np.int32)
    lp = np.zeros(n + 1, np.int32)
    li = []
    for j in range(n):
        # low degrees are common, as in a soliton-like law
        d = min(int(rng.choice([1, 1, 2, 2, 2, 3, max_deg])), k_int)
        li.extend(sorted(rng.choice(k_int, size=d, replace=False).tolist()))
        lp[j + 1] = len(li)
    return gen.Graph(b, m, n, pp, pi, lp, np.array(li, dtype=np.int32))


def _dense_generator(g):
    """The code as a dense GF(2) matrix over the b data blocks: rows = n coded
    blocks, built by composing the precode and LT incidence matrices."""
    P = np.zeros((g.m, g.b), np.int64)
    for j in range(g.m):
        P[j, g.pre_idx[g.pre_ptr[j]:g.pre_ptr[j + 1]]] = 1
    I = np.concatenate([np.eye(g.b, dtype=np.int64), P], axis=0)  # k_int x b
    L = np.zeros((g.n, g.k_int), np.int64)
    for j in range(g.n):
        L[j, g.lt_idx[g.lt_ptr[j]:g.lt_ptr[j + 1]]] = 1
    return (L @ I) % 2, P


def _gf2_matmul_bytes(M, X):
    """Y = M X over GF(2) on byte rows, via unpacked bits and an integer
    matrix product (no XOR loop)."""
    bits = np.unpackbits(X, axis=1).astype(np.int64)
    return np.packbits(((M @ bits) % 2).astype(np.uint8), axis=1)


@pytest.mark.parametrize("b,m,n,t,seed", [(12, 4, 20, 16, 1), (40, 0, 60, 48, 2),
                                          (33, 7, 50, 80, 3), (5, 5, 9, 16, 4)])
def test_encode_equals_gf2_matrix_product(b, m, n, t, seed):
    rng = np.random.default_rng(seed)
    g = _rand_graph(rng, b, m, n, max_deg=7)
    data = rng.integers(0, 256, size=(b, t), dtype=np.uint8)
    parity, coded = oracle.encode(g, data, t)
    G, P = _dense_generator(g)
    assert np.array_equal(coded, _gf2_matmul_bytes(G, data))
    if m:
        assert np.array_equal(parity, _gf2_matmul_bytes(P, data))


def test_encode_linearity_and_degree_one():
    g = gen.make_graph(60, 6, 90, gen.DIST_RSD, 0.1, 0.05)
    t = 32
    x = gen.fill_bytes(11, 60 * t).reshape(60, t)
    y = gen.fill_bytes(12, 60 * t).reshape(60, t)
    px, cx = oracle.encode(g, x, t)
    py, cy = oracle.encode(g, y, t)
    pz, cz = oracle.encode(g, x ^ y, t)
    assert np.array_equal(cz, cx ^ cy) and np.array_equal(pz, px ^ py)
    inter = np.concatenate([x, px])
    deg = np.diff(g.lt_ptr)
    assert (deg == 1).any()
    for j in np.nonzero(deg == 1)[0]:
        assert np.array_equal(cx[j], inter[g.lt_idx[g.lt_ptr[j]]])
    # a precode check is a zero-sum set of data and its parity (check #1)
    for j in range(g.m):
        s = px[j].copy()
        for i in g.pre_idx[g.pre_ptr[j]:g.pre_ptr[j + 1]]:
            s ^= x[i]
        assert not s.any()


def _constraint_masks(g, erased, mode_stage=None):
    """Bitmask rows of the received constraints over the k_int intermediates."""
    rows = []
    for j in range(g.n):
        if not erased[j]:
            r = 0
            for v in g.lt_idx[g.lt_ptr[j]:g.lt_ptr[j + 1]]:
                r |= 1 << int(v)
            rows.append(r)
    for j in range(g.m):
        r = 1 << (g.b + j)
        for v in g.pre_idx[g.pre_ptr[j]:g.pre_ptr[j + 1]]:
            r |= 1 << int(v)
        rows.append(r)
    return rows


def _gf2_determined(rows, k_int):
    """Gaussian elimination over GF(2): the set of unknowns whose unit vector
    lies in the row space (the symbols any decoder could recover), and the
    rank."""
    basis = {}  # pivot bit -> row
    for r in rows:
        for p in sorted(basis, reverse=True):
            if r >> p & 1:
                r ^= basis[p]
        if r:
            p = r.bit_length() - 1
            # keep the basis reduced on the new pivot
            for q in list(basis):
                if basis[q] >> p & 1:
                    basis[q] ^= r
            basis[p] = r
    det = set()
    for v in range(k_int):
        e = 1 << v
        for p in sorted(basis, reverse=True):
            if e >> p & 1:
                e ^= basis[p]
        if e == 0:
            det.add(v)
    return det, len(basis)


@pytest.mark.parametrize("seed,b,m,n", [(3, 5, 3, 10), (4, 7, 2, 12), (6, 8, 0, 12), (7, 5, 3, 11)])
def test_exhaustive_erasures_against_elimination(seed, b, m, n):
    """Every erasure subset of a tiny code (simDisk, Section 2.1)."""
    rng = np.random.default_rng(seed)
    g = _rand_graph(rng, b, m, n, max_deg=4)
    k_int = b + m
    t = 16
    data = rng.integers(0, 256, size=(b, t), dtype=np.uint8)
    parity, coded = oracle.encode(g, data, t)
    inter = np.concatenate([data, parity]) if m else data
    complete = 0
    for mask in range(1 << n):
        erased = np.array([(mask >> j) & 1 for j in range(n)], np.uint8)
        out, path = oracle.decode(g, coded, erased, t)
        recovered = {v for v in range(k_int) if not path.unrecovered[v]}
        det, rank = _gf2_determined(_constraint_masks(g, erased), k_int)
        # peeling never claims more than elimination can determine
        assert recovered <= det
        assert path.n_pairs == len(recovered)
        if len(recovered) == k_int:
            complete += 1
            assert rank == k_int
            assert np.array_equal(out, data)
        # every recovered byte is the source; the rest is zero
        for v in range(b):
            if v in recovered:
                assert np.array_equal(out[v], data[v])
            else:
                assert not out[v].any()
        # the peeling fixpoint does not depend on the visiting order
        order = rng.permutation(n + m).astype(np.int32)
        unrec_imm, sweeps = oracle.peel_immediate(g, erased, order, with_sweeps=True)
        assert np.array_equal(unrec_imm, path.unrecovered)
        # immediate updates reach the fixpoint in no more sweeps than the
        # delayed schedule has levels (Section 3.1: t_m <= t-bar_m)
        assert sweeps <= path.n_levels
        _check_path_rules(g, erased, path)
        # the two-pass decoder: its own rules, never more than the joint one,
        # never more than elimination, and its bytes are the source
        out2, path2 = oracle.decode(g, coded, erased, t, oracle.MODE_TWO_PASS)
        _check_path_rules(g, erased, path2, oracle.MODE_TWO_PASS)
        rec2 = {v for v in range(k_int) if not path2.unrecovered[v]}
        assert rec2 <= recovered
        for v in range(b):
            if v in rec2:
                assert np.array_equal(out2[v], data[v])
            else:
                assert not out2[v].any()
    assert complete > 0


def _check_path_rules(g, erased, path, mode=oracle.MODE_JOINT):
    """Algorithm 5 rules checked level by level: each g had exactly one
    unknown f at the start of its level, f was unknown, each f appears once,
    g is the lowest (degree, index) among that level's candidates for f, and
    a level holds every f some candidate offers. After the last level no
    candidate is left (the fixpoint).

    Joint mode: the candidates are the surviving coded rows and the precode
    checks. Two-pass mode (founsureDec in Section 2.2: BP on the LT code, then
    BP on the precode): stage 0 admits only surviving coded rows and runs
    until a level finds none; from then on only precode checks, until a level
    finds none; a stage never returns to coded rows. Returns the number of
    stage-0 levels (the whole path in joint mode)."""
    known = np.zeros(g.k_int, bool)

    def vars_of(c):
        if c < g.n:
            return list(g.lt_idx[g.lt_ptr[c]:g.lt_ptr[c + 1]])
        j = c - g.n
        return list(g.pre_idx[g.pre_ptr[j]:g.pre_ptr[j + 1]]) + [g.b + j]

    def candidates(cons):
        cand = {}
        for c in cons:
            if c < g.n and erased[c]:
                continue
            unk = [v for v in vars_of(c) if not known[v]]
            if len(unk) == 1:
                cand.setdefault(unk[0], []).append((len(vars_of(c)), c))
        return cand

    lt_rows, checks = range(g.n), range(g.n, g.n + g.m)
    two_pass = mode == oracle.MODE_TWO_PASS
    stage = 0
    stage0_levels = None
    seen = set()
    for lvl, pairs in enumerate(path.levels()):
        if two_pass:
            cand = candidates(lt_rows if stage == 0 else checks)
            if stage == 0 and not cand:
                # stage 0 reached its fixpoint: this level opens stage 1
                stage, stage0_levels = 1, lvl
                cand = candidates(checks)
        else:
            cand = candidates(range(g.n + g.m))
        assert {f for f, _ in pairs} == set(cand)
        for f, c in pairs:
            assert f not in seen
            seen.add(f)
            assert (len(vars_of(c)), c) == min(cand[f])
            if two_pass:
                assert (c < g.n) == (stage == 0)
        for f, _ in pairs:
            known[f] = True
    if two_pass:
        if stage == 0:
            stage0_levels = path.n_levels
            assert not candidates(lt_rows)
        assert not candidates(checks)
    else:
        assert not candidates(range(g.n + g.m))
        stage0_levels = path.n_levels
    assert np.array_equal(~known, path.unrecovered.astype(bool))
    return stage0_levels


def _lt_only_graph(g):
    """The LT layer alone, as a code with k_int data blocks and no precode:
    its peeling fixpoint is what stage 0 of the two-pass decoder reaches."""
    return gen.Graph(g.k_int, 0, g.n, np.zeros(1, np.int32), np.zeros(0, np.int32),
                     np.asarray(g.lt_ptr, np.int32), np.asarray(g.lt_idx, np.int32))


def _checks_closure(g, known):
    """Precode-only peeling from the state ``known`` with immediate updates
    (plain sets): the fixpoint stage 1 of the two-pass decoder must reach."""
    known = set(np.nonzero(known)[0].tolist())
    rows = [set(g.pre_idx[g.pre_ptr[j]:g.pre_ptr[j + 1]].tolist()) | {g.b + j} for j in range(g.m)]
    changed = True
    while changed:
        changed = False
        for r in rows:
            unk = r - known
            if len(unk) == 1:
                known |= unk
                changed = True
    return known


def test_dpg_rules_config1_and_success_size():
    b, n, t = 100, 150, 1024
    g = gen.make_graph(b, 0, n, gen.DIST_RSD, 0.1, 0.05)
    data = gen.fill_bytes(1, b * t).reshape(b, t)
    _, coded = oracle.encode(g, data, t)
    erased = np.zeros(n, np.uint8)
    erased[gen.sample_indices(n, 30, gen.SEED_ERASE)] = 1
    out, path = oracle.decode(g, coded, erased, t)
    _check_path_rules(g, erased, path)
    rec = path.unrecovered == 0
    assert np.array_equal(out[rec], data[rec])
    # with nothing erased and enough rows, peeling finishes: |DP| = k pairs
    g2 = gen.make_graph(b, 0, 400, gen.DIST_RSD, 0.1, 0.05)
    _, coded2 = oracle.encode(g2, data, t)
    out2, path2 = oracle.decode(g2, coded2, np.zeros(400, np.uint8), t)
    if path2.unrecovered.sum() == 0:
        assert path2.n_pairs == b
        assert np.array_equal(out2, data)


def test_precoded_decode_both_modes():
    b, m, n, t = 400, 20, 560, 64
    g = gen.make_graph(b, m, n, gen.DIST_FINITE40)
    data = gen.fill_bytes(7, b * t).reshape(b, t)
    parity, coded = oracle.encode(g, data, t)
    erased = np.zeros(n, np.uint8)
    erased[gen.sample_indices(n, gen.round_count(0.1, n), 21)] = 1
    out_j, path_j = oracle.decode(g, coded, erased, t, oracle.MODE_JOINT)
    out_2, path_2 = oracle.decode(g, coded, erased, t, oracle.MODE_TWO_PASS)
    _check_path_rules(g, erased, path_j)
    n0 = _check_path_rules(g, erased, path_2, oracle.MODE_TWO_PASS)
    # stage 0 recovers exactly the LT layer's own peeling fixpoint (visited
    # in several random orders with immediate updates), and stage 1 exactly
    # the precode's closure from there
    lt = _lt_only_graph(g)
    rng = np.random.default_rng(5)
    stage0 = np.zeros(g.k_int, bool)
    for lvl_pairs in path_2.levels()[:n0]:
        for f, _ in lvl_pairs:
            stage0[f] = True
    for _ in range(3):
        order = rng.permutation(n).astype(np.int32)
        assert np.array_equal(oracle.peel_immediate(lt, erased, order) == 0, stage0)
    assert _checks_closure(g, stage0) == set(np.nonzero(path_2.unrecovered == 0)[0].tolist())
    # the joint fixpoint contains whatever the two-pass schedule recovers
    assert np.all(path_j.unrecovered <= path_2.unrecovered)
    for out, path in ((out_j, path_j), (out_2, path_2)):
        rec = path.unrecovered[:b] == 0
        assert np.array_equal(out[rec], data[rec])
        assert not out[~rec].any()
    # parities recovered by the payload are the encoder's parities
    d, p = oracle.peel(g, coded, path_j, t, with_parity=True)
    prec = path_j.unrecovered[b:] == 0
    assert np.array_equal(p[prec], parity[prec])


def test_update_is_reencode_by_linearity_and_repair_restores():
    b, m, n, t = 200, 10, 280, 48
    g = gen.make_graph(b, m, n, gen.DIST_FINITE40)
    data = gen.fill_bytes(3, b * t).reshape(b, t)
    par0, cod0 = oracle.encode(g, data, t)
    idx = gen.sample_indices(b, 5, gen.SEED_UPDATE)
    new = gen.fill_bytes(gen.SEED_NEWDATA, 5 * t).reshape(5, t)
    d1, par1, cod1 = oracle.update(g, data, idx, new, t)
    delta = np.zeros_like(data)
    delta[idx] = data[idx] ^ new
    pd, cd = oracle.encode(g, delta, t)
    assert np.array_equal(par1, par0 ^ pd) and np.array_equal(cod1, cod0 ^ cd)
    assert np.array_equal(d1[idx], new)
    lost = gen.sample_indices(n, 14, gen.SEED_REPAIR)
    rep = oracle.repair(g, d1, lost, t)
    assert np.array_equal(rep, cod1[lost])


def test_empty_and_degenerate_graphs():
    t = 16
    # a precode check with no members has a zero parity; decoding it costs no input
    g = gen.Graph(3, 1, 3, np.array([0, 0], np.int32), np.zeros(0, np.int32),
                  np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32))
    data = np.arange(3 * t, dtype=np.uint8).reshape(3, t)
    parity, coded = oracle.encode(g, data, t)
    assert not parity.any() and np.array_equal(coded, data)
    out, path = oracle.decode(g, coded, np.zeros(3, np.uint8), t)
    assert path.n_pairs == 4 and path.unrecovered.sum() == 0
    assert np.array_equal(out, data)
    # everything erased: nothing recovered, all zeros
    out, path = oracle.decode(g, coded, np.ones(3, np.uint8), t)
    assert path.unrecovered[:3].all() and not out.any()
    # no coded rows at all
    g0 = gen.Graph(2, 0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32),
                   np.zeros(1, np.int32), np.zeros(0, np.int32))
    out, path = oracle.decode(g0, np.zeros((0, t), np.uint8), np.zeros(0, np.uint8), t)
    assert path.n_pairs == 0 and path.n_levels == 0 and not out.any()


def _hand_graph():
    """b = 3 data blocks (0, 1, 2), m = 2 parities (3, 4), n = 4 coded rows:
    check 0 = {0, 1} + parity 3 (constraint 4), check 1 = {} + parity 4
    (constraint 5: an empty check, its parity is the zero block);
    c0 = {0}, c1 = {0, 1}, c2 = {3, 2}, c3 = {4, 2}; nothing erased."""
    return gen.Graph(3, 2, 4, np.array([0, 2, 2], np.int32), np.array([0, 1], np.int32),
                     np.array([0, 1, 3, 5, 7], np.int32),
                     np.array([0, 0, 1, 3, 2, 4, 2], np.int32))


def test_two_pass_and_joint_differ_on_a_hand_worked_graph():
    """Both schedules worked by hand from Algorithm 5 and the founsureDec
    description (Section 2.2).

    Joint: level 0 has c0 -> 0 and check 1 -> 4 (degree 1 from the start);
    level 1 c1 -> 1 and c3 -> 2 (4 is known); level 2 offers 3 through c2
    (degree 2) and check 0 (degree 3): c2 wins. Everything is recovered.

    Two-pass: stage 0 (coded rows only) takes c0 -> 0, then c1 -> 1, then
    stops (c2, c3 hold two unknowns each); stage 1 (checks only) takes check
    0 -> 3 and check 1 -> 4 in one level, then stops. Block 2 stays
    unrecovered: c2 and c3 now have one unknown each, but the decoder runs BP
    at most twice and does not return to the coded rows."""
    g = _hand_graph()
    t = 16
    data = np.arange(3 * t, dtype=np.uint8).reshape(3, t) * 7
    parity, coded = oracle.encode(g, data, t)
    assert np.array_equal(parity[0], data[0] ^ data[1]) and not parity[1].any()
    erased = np.zeros(4, np.uint8)

    out_j, pj = oracle.decode(g, coded, erased, t, oracle.MODE_JOINT)
    assert pj.levels() == [{(0, 0), (4, 5)}, {(1, 1), (2, 3)}, {(3, 2)}]
    assert pj.n_levels == 3 and not pj.unrecovered.any()
    assert np.array_equal(out_j, data)

    out_2, p2 = oracle.decode(g, coded, erased, t, oracle.MODE_TWO_PASS)
    assert p2.levels() == [{(0, 0)}, {(1, 1)}, {(3, 4), (4, 5)}]
    assert p2.n_levels == 3
    assert p2.unrecovered.tolist() == [0, 0, 1, 0, 0]
    assert np.array_equal(out_2[:2], data[:2]) and not out_2[2].any()
    _, par2 = oracle.peel(g, coded, p2, t, with_parity=True)
    assert np.array_equal(par2, parity)

    assert _check_path_rules(g, erased, p2, oracle.MODE_TWO_PASS) == 2
    # Algorithm 1 in index order with immediate updates: the first sweep
    # decodes 0 (c0), 1 (c1), 3 (check 0, its members now known) and 4
    # (check 1); c2 and c3 still held two unknowns when visited. The second
    # sweep decodes 2 (c2); the third changes nothing. Two productive sweeps
    # against three delayed levels.
    unrec, sweeps = oracle.peel_immediate(g, erased, np.arange(6, dtype=np.int32),
                                          with_sweeps=True)
    assert not unrec.any() and sweeps == 2


def test_immediate_sweeps_never_exceed_delayed_levels():
    """Section 3.1: the delayed schedule (Algorithm 5) converges no sooner
    than Algorithm 1 with immediate updates, to the same set (t_m <= t-bar_m);
    on a code of a few hundred blocks, in several visiting orders."""
    b, m, n = 300, 16, 420
    g = gen.make_graph(b, m, n, gen.DIST_FINITE40)
    erased = np.zeros(n, np.uint8)
    erased[gen.sample_indices(n, gen.round_count(0.1, n), 33)] = 1
    path = oracle.dpg(g, erased)
    rng = np.random.default_rng(8)
    orders = [np.arange(n + m, dtype=np.int32)] + [rng.permutation(n + m).astype(np.int32)
                                                   for _ in range(3)]
    for order in orders:
        unrec, sweeps = oracle.peel_immediate(g, erased, order, with_sweeps=True)
        assert np.array_equal(unrec, path.unrecovered)
        assert 1 <= sweeps <= path.n_levels
