"""Repair from local recovery groups on the GPU (fs_repair_local) against the
oracle, byte for byte: the repaired blocks, the unrepaired flags and count,
the repair path level by level, and untouched surviving blocks."""
import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

pytestmark = pytest.mark.gpu


def _case(g, t, frac, seed):
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    data = gen.fill_bytes(gen.SEED_DATA + seed, g.b * t).reshape(g.b, t)
    _, coded = oracle.encode(g, data, t)
    lost = np.zeros(g.n, np.uint8)
    lost[gen.sample_indices(g.n, gen.round_count(frac, g.n), gen.SEED_ERASE + seed)] = 1
    want = oracle.local_groups(g)
    ptr, idx = want.csr()
    want_out, want_path = oracle.repair_local(ptr, idx, coded, lost, t)
    loc = fs.Local(g)
    d_coded = torch.from_numpy(coded.copy()).cuda()
    d_coded[torch.from_numpy(lost.astype(bool)).cuda()] = 0x77  # the lost blocks are gone
    d_lost = torch.from_numpy(lost).cuda()
    unrep = torch.full((g.n,), 9, dtype=torch.uint8, device="cuda")
    nun = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ws = loc.workspace()
    loc.repair(d_lost, d_coded, t, unrep, nun, ws)
    torch.cuda.synchronize()
    assert np.array_equal(d_coded.cpu().numpy(), want_out)
    assert np.array_equal(unrep.cpu().numpy(), want_path.unrepaired)
    assert int(nun.item()) == int(want_path.unrepaired.sum())
    assert loc.path(ws) == want_path.levels()
    assert int(ws[:4].view(torch.int32).item()) == fs.FS_OK
    return want_path


@pytest.mark.parametrize("t", [16, 48, 4096 + 16])
def test_repair_small_codes(t):
    path = _case(gen.make_graph(300, 12, 400, gen.DIST_FINITE40, stripe=1), t, 0.1, 1)
    assert path.n_pairs > 0


@pytest.mark.parametrize("frac", [0.02, 0.3])
def test_repair_rsd_code(frac):
    _case(gen.make_graph(1000, 0, 1300, gen.DIST_RSD, 0.05, 0.01, stripe=2), 1024, frac, 2)


def test_repair_full_size_precoded_stripe():
    """b = 4096 x 64 KiB, m = 128, n = 5400, 5% (270) of the coded blocks
    lost."""
    path = _case(gen.make_graph(4096, 128, 5400, gen.DIST_FINITE40), 65536, 0.05, 4)
    assert path.n_pairs > 200


def test_repair_edge_cases():
    """Nothing lost: nothing changes; a host-only object cannot repair."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph(300, 12, 400, gen.DIST_FINITE40, stripe=1)
    loc = fs.Local(g)
    coded = torch.randint(0, 256, (g.n, 32), dtype=torch.uint8, device="cuda")
    before = coded.clone()
    unrep = torch.empty(g.n, dtype=torch.uint8, device="cuda")
    nun = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = loc.workspace()
    loc.repair(torch.zeros(g.n, dtype=torch.uint8, device="cuda"), coded, 32, unrep, nun, ws)
    torch.cuda.synchronize()
    assert torch.equal(coded, before) and int(nun.item()) == 0 and loc.path(ws) == []
    host = fs.Local(g, host_only=True)
    with pytest.raises(fs.FounsureError):
        host.repair(torch.zeros(g.n, dtype=torch.uint8, device="cuda"), coded, 32, unrep, nun, ws)
    with pytest.raises(fs.FounsureError):
        loc.repair(torch.zeros(g.n, dtype=torch.uint8, device="cuda"), coded, 24, unrep, nun, ws)
