"""simDisk sweeps: every combination of failed disks is one erasure pattern
whose decoding schedule (Algorithm 5) the GPU runs in a batch; the counts and
flags must equal the oracle's, pattern by pattern."""
import math

import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen
from paper_1702_07409_gb300 import simdisk


def test_patterns_cover_every_combination():
    n, disks = 103, 7
    d = simdisk.disk_of_blocks(n, disks)
    assert d.min() == 0 and d.max() == disks - 1
    assert all(np.diff(d) >= 0) and np.bincount(d).max() == math.ceil(n / disks)
    for f in (0, 1, 2, 3, 7):
        combos, flags = simdisk.failure_patterns(n, disks, f)
        assert len(combos) == math.comb(disks, f) == flags.shape[0]
        assert len(set(combos)) == len(combos)
        for c, fl in zip(combos, flags):
            assert fl.astype(bool).tolist() == [int(x) in c for x in d]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(300, 12, 400, gen.DIST_FINITE40), (200, 0, 260, gen.DIST_RSD)])
def test_sweeps_match_the_oracle(shape):
    b, m, n, dist = shape
    g = gen.make_graph(b, m, n, dist, 0.1, 0.05) if dist == gen.DIST_RSD else gen.make_graph(b, m, n, dist)
    sd = simdisk.SimDisk(g, 10, max_batch=16)  # several batches per sweep
    tolerated = []
    for f in (1, 2, 3):
        combos, flags = simdisk.failure_patterns(n, 10, f)
        nun, unrec = sd.schedule(flags)
        for i in range(len(combos)):
            path = oracle.dpg(g, flags[i])
            assert np.array_equal(unrec[i], path.unrecovered)
            assert int(nun[i]) == int(path.unrecovered.sum())
        tolerated.append(sd.run(f)["tolerated"])
    assert tolerated[0] >= tolerated[1] >= tolerated[2]


@pytest.mark.gpu
def test_schedule_batches_need_no_payload_buffers():
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph(100, 0, 150, gen.DIST_RSD, 0.1, 0.05)
    code = fs.Code(g, 16)
    er = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
    st = {"code": code, "erased": er, "unrecovered": torch.empty(g.b, dtype=torch.uint8, device="cuda"),
          "n_unrecovered": torch.empty(1, dtype=torch.int32, device="cuda"),
          "ws": code.workspace(fs.OP_DECODE)}
    b = fs.Batch([st], fs.OP_SCHEDULE)
    b.run()
    torch.cuda.synchronize()
    assert int(st["n_unrecovered"].item()) == int(oracle.dpg(g, np.zeros(g.n, np.uint8)).unrecovered.sum())
    with pytest.raises(fs.FounsureError):
        fs.Batch([dict(st, ws=None)], fs.OP_SCHEDULE)
