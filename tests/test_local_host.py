"""The library's local recovery groups (fs_local_create, host part: Algorithm
4, the set-XOR derivations, cardinality order) equal the oracle's, group by
group and in the same order. Runs on the CPU: the groups are built on the
host and FS_LOCAL_HOST_ONLY skips the device copy."""
import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen


def _graph_from_rows(b, rows):
    ptr = np.zeros(len(rows) + 1, np.int32)
    for j, r in enumerate(rows):
        ptr[j + 1] = ptr[j] + len(r)
    idx = np.array([v for r in rows for v in sorted(r)], dtype=np.int32)
    return gen.Graph(b, 0, len(rows), np.zeros(1, np.int32), np.zeros(0, np.int32), ptr, idx)


def _graphs():
    rng = np.random.default_rng(5)
    rows = [[i] for i in range(12)] + [sorted(rng.choice(12, size=int(rng.integers(2, 6)),
                                                         replace=False).tolist()) for _ in range(7)]
    return [gen.make_graph(100, 0, 150, gen.DIST_RSD, 0.1, 0.05),
            gen.make_graph(300, 12, 400, gen.DIST_FINITE40, stripe=1),
            gen.make_graph(60, 6, 90, gen.DIST_FINITE40, stripe=3),  # Algorithm 4 finds nothing
            gen.make_graph(1000, 0, 1300, gen.DIST_RSD, 0.05, 0.01, stripe=2),
            _graph_from_rows(12, rows)]


@pytest.mark.parametrize("gi", range(5))
def test_library_groups_equal_the_oracle(gi):
    from paper_1702_07409_gb300 import founsure as fs
    g = _graphs()[gi]
    want = oracle.local_groups(g)
    loc = fs.Local(g, host_only=True)
    info = loc.info()
    assert info["sweeps"] == want.sweeps
    ptr, idx = loc.groups()
    wptr, widx = want.csr()
    assert np.array_equal(ptr, wptr) and np.array_equal(idx, widx)
    assert loc.check2() == want.check2
    loc.close()


def test_max_sweeps_and_bad_graphs():
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph(100, 0, 150, gen.DIST_RSD, 0.1, 0.05)
    one = fs.Local(g, max_sweeps=1, host_only=True)
    assert one.info()["sweeps"] == 1 == oracle.local_groups(g, max_sweeps=1).sweeps
    assert np.array_equal(one.groups()[1], oracle.local_groups(g, max_sweeps=1).csr()[1])
    bad = gen.Graph(4, 0, 2, np.zeros(1, np.int32), np.zeros(0, np.int32),
                    np.array([0, 2, 3], np.int32), np.array([1, 1, 0], np.int32))  # repeated index
    with pytest.raises(fs.FounsureError):
        fs.Local(bad, host_only=True)
