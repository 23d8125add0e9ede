"""Pins for the seeded input generator (splitmix64, degree distributions,
graph sampling, index draws). The generator holds no coding arithmetic; it is
pinned here against published values, closed forms and invariants."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1702_07409_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_splitmix64_known_answer():
    rows = _golden_rows("splitmix64_kat.txt")
    seed = int(rows[0][1])
    want = [int(r[0]) for r in rows[1:]]
    got = [int(x) for x in gen.stream(seed, len(want))]
    assert got == want


def test_counter_form_matches_stream():
    seed = 0xDEADBEEF12345
    s = gen.stream(seed, 50)
    for w in (0, 1, 7, 49):
        assert int(gen.lib().fsg_at(seed, w)) == int(s[w])


def test_fill_bytes_little_endian_and_offsets():
    seed = 99
    words = gen.stream(seed, 8)
    want = np.frombuffer(words.astype("<u8").tobytes(), dtype=np.uint8)
    got = gen.fill_bytes(seed, 64)
    assert np.array_equal(got, want)
    # any window equals the same slice of the whole stream
    for off, ln in ((3, 17), (8, 8), (13, 40), (0, 1)):
        assert np.array_equal(gen.fill_bytes(seed, ln, offset=off), want[off:off + ln])


def test_uniform_maps():
    seed = 5
    raw = gen.stream(seed, 1000)
    ints = gen.uniform_ints(seed, 37, 1000)
    # high 64 bits of x * r
    want = [(int(x) * 37) >> 64 for x in raw]
    assert [int(v) for v in ints] == want
    assert ints.max() < 37
    dbl = gen.uniform_doubles(seed, 1000)
    assert np.array_equal(dbl, (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)
    assert dbl.min() >= 0.0 and dbl.max() < 1.0


def _rsd_closed_form(k, c, delta):
    """Luby's Robust Soliton written with harmonic numbers instead of a sum
    over degrees: beta = 1 + (R/k) H_{s-1} + R ln(R/delta)/k."""
    R = c * math.log(k / delta) * math.sqrt(k)
    s = min(max(int(math.floor(k / R)), 1), k)
    H = sum(Fraction(1, d) for d in range(1, s))
    beta = 1.0 + (R / k) * float(H) + max(0.0, R * math.log(R / delta) / k)
    return R, s, beta


@pytest.mark.parametrize("k,c,delta", [(100, 0.1, 0.05), (4096, 0.05, 0.01), (64, 0.05, 0.01),
                                       (1000, 0.2, 0.5), (4224, 0.1, 0.05)])
def test_rsd_closed_form(k, c, delta):
    mu, dmax, info = gen.pmf(gen.DIST_RSD, k, c, delta)
    R, s, beta = _rsd_closed_form(k, c, delta)
    assert dmax == k
    assert info[0] == pytest.approx(R, rel=1e-14)
    assert int(info[1]) == s
    assert info[2] == pytest.approx(beta, rel=1e-12)
    assert mu[0] == 0.0
    assert abs(mu.sum() - 1.0) < 1e-12
    # rho alone telescopes to exactly 1: 1/k + sum_{d=2..k} 1/(d(d-1)) = 1
    rho = Fraction(1, k) + sum(Fraction(1, d * (d - 1)) for d in range(2, k + 1))
    assert rho == 1
    # shape: mu(d) * beta = rho(d) + tau(d)
    for d in (1, 2, 3, s - 1, s, s + 1, k):
        if d < 1 or d > k:
            continue
        r = 1.0 / k if d == 1 else 1.0 / (d * (d - 1))
        if d < s:
            tau = R / (d * k)
        elif d == s:
            tau = max(0.0, R * math.log(R / delta) / k)
        else:
            tau = 0.0
        assert mu[d] * info[2] == pytest.approx(r + tau, rel=1e-12)


def test_rsd_config1_values():
    # k=100, c=0.1, delta=0.05: R = 0.1 ln(2000) 10
    _, _, info = gen.pmf(gen.DIST_RSD, 100, 0.1, 0.05)
    assert info[0] == pytest.approx(math.log(2000.0), rel=1e-14)
    assert int(info[1]) == 13  # floor(100 / 7.6009)


def test_omega_golden_and_renormalisation():
    rows = _golden_rows("omega_raptor.txt")
    deg = [int(r[0]) for r in rows]
    val = [float(r[1]) for r in rows]
    raw = sum(val)
    assert raw == pytest.approx(0.999998, abs=1e-12)
    mu, dmax, info = gen.pmf(gen.DIST_FINITE65)
    assert dmax == 65
    assert info[2] == pytest.approx(raw, abs=1e-15)
    for d, v in zip(deg, val):
        assert mu[d] == pytest.approx(v / raw, rel=1e-13)
    assert abs(mu.sum() - 1.0) < 1e-14
    # max-degree-40, DROP: degrees 64 and 65 removed, rest renormalised
    mu40, dmax40, info40 = gen.pmf(gen.DIST_FINITE40)
    kept = sum(v for d, v in zip(deg, val) if d <= 40)
    assert dmax40 == 19
    for d, v in zip(deg, val):
        assert mu40[d] == pytest.approx(v / kept if d <= 40 else 0.0, rel=1e-13, abs=0)
    assert info40[3] == pytest.approx(sum(d * v for d, v in zip(deg, val) if d <= 40) / kept,
                                      rel=1e-13)
    # FOLD: their mass moves to degree 40
    muf, dmaxf, _ = gen.pmf(gen.DIST_FINITE40_FOLD)
    assert dmaxf == 40
    assert muf[40] == pytest.approx((val[-1] + val[-2]) / raw, rel=1e-13)


def _check_csr(ptr, idx, n_rows, n_cols):
    assert ptr[0] == 0 and ptr.size == n_rows + 1
    assert np.all(np.diff(ptr) >= 0) and ptr[-1] == idx.size
    for r in range(n_rows):
        row = idx[ptr[r]:ptr[r + 1]]
        assert np.all(row >= 0) and np.all(row < n_cols)
        assert np.all(np.diff(row) > 0), "row %d not strictly ascending" % r


def test_lt_graph_structure_and_degree_law():
    k, n = 300, 4000
    mu, dmax, info = gen.pmf(gen.DIST_RSD, k, 0.1, 0.05)
    ptr, idx = gen.lt_graph(k, n, mu, dmax, 777)
    _check_csr(ptr, idx, n, k)
    deg = np.diff(ptr)
    assert deg.min() >= 1
    # mean degree within 5 standard errors of the distribution's mean
    mean = info[3]
    var = float(np.sum(mu * (np.arange(mu.size) - mean) ** 2))
    assert abs(deg.mean() - mean) < 5 * math.sqrt(var / n)
    # frequency of degree 2 (about 1/2 / beta) within 5 sigma
    p2 = mu[2]
    assert abs(np.mean(deg == 2) - p2) < 5 * math.sqrt(p2 * (1 - p2) / n)
    # neighbours are uniform: every column hit close to E/k times
    counts = np.bincount(idx, minlength=k)
    e = idx.size / k
    chi2 = float(np.sum((counts - e) ** 2 / e))
    assert chi2 < k + 6 * math.sqrt(2 * k)
    # nnz helper agrees with the graph it predicts
    assert gen.lib().fsg_lt_graph_nnz(k, n, mu.ctypes.data, dmax, 777) == idx.size


def test_precode_graph_left_regular():
    b, m, q = 500, 40, 3
    ptr, idx = gen.precode_graph(b, m, q, 4242)
    _check_csr(ptr, idx, m, b)
    assert np.array_equal(np.bincount(idx, minlength=b), np.full(b, q))
    # q > m: every data block joins every check
    ptr2, idx2 = gen.precode_graph(10, 2, 3, 1)
    assert np.array_equal(np.diff(ptr2), [10, 10])


def test_make_graph_config2_shape():
    g = gen.make_graph(4096, 128, 5400, gen.DIST_FINITE40)
    assert g.k_int == 4224 and g.e_pre == 4096 * 3
    assert np.diff(g.lt_ptr).max() <= 19
    assert 4.0 < g.e_lt / 5400 < 4.3


def test_sample_indices_and_round_count():
    s = gen.sample_indices(5400, 1080, 2)
    assert s.size == 1080 and np.unique(s).size == 1080
    assert s.min() >= 0 and s.max() < 5400
    full = gen.sample_indices(50, 50, 9)
    assert sorted(full.tolist()) == list(range(50))
    # a prefix of a longer draw is the shorter draw
    assert np.array_equal(gen.sample_indices(100, 10, 3), gen.sample_indices(100, 30, 3)[:10])
    assert gen.round_count(0.2, 5400) == 1080
    assert gen.round_count(0.01, 4096) == 41   # 40.96 rounds up
    assert gen.round_count(0.05, 5400) == 270
    assert gen.round_count(0.5, 3) == 2        # half rounds up
    assert gen.n_for_rate(100) == 130 and gen.n_for_rate(4096) == 5325
