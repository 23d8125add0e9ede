"""A randomized differential sweep of the CUDA path against the oracle: many
small codes drawn at random (plain LT, precoded, array-precoded; RSD and
FiniteDist degrees; block sizes with ragged 16-byte tails; erasure rates from
none to most; tuning knobs), each encoded, decoded, updated and repaired on
the GPU and compared byte for byte with the oracle; every fourth code is
also repaired from its local recovery groups."""
import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

pytestmark = pytest.mark.gpu

KNOBS = [None, (1, 2), (3, 0), (5, 0), (5, 2), (7, 1), (6, 3)]


def _draw(seed):
    rng = np.random.default_rng(1000 + seed)
    kind = ("plain", "pre", "array")[seed % 3]
    t = int(rng.choice([16, 32, 48, 80, 1024, 4096 + 16]))
    dist = int(rng.choice([gen.DIST_RSD, gen.DIST_FINITE40]))
    if kind == "array":
        b, k = [(14, 21), (21, 35), (117, 143), (120, 150), (4154, 4288)][seed % 5]
        n = int(k * rng.uniform(1.25, 1.6))
        g = gen.make_graph_array(b, k, n, dist, 0.1, 0.05, stripe=seed)
    else:
        b = int(rng.integers(1, 700))
        m = int(rng.integers(1, max(2, b // 8 + 1))) if kind == "pre" else 0
        n = int((b + m) * rng.uniform(1.1, 1.7)) + 1
        g = gen.make_graph(b, m, n, dist, 0.1, 0.05, stripe=seed)
    frac = float(rng.choice([0.0, 0.05, 0.2, 0.35, 0.7]))
    return g, t, frac, KNOBS[seed % len(KNOBS)], rng


@pytest.mark.parametrize("seed", range(60))
def test_random_code(seed):
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    g, t, frac, knob, rng = _draw(seed)
    b, m, n = g.b, g.m, g.n
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    host = lambda x: x.cpu().numpy()
    data = gen.fill_bytes(gen.SEED_DATA + seed, b * t).reshape(b, t)
    code = fs.Code(g, t)
    if knob:
        code.set_tuning(*knob)
    d = dev(data)
    p = torch.empty((m, t), dtype=torch.uint8, device="cuda") if m else None
    cd = torch.empty((n, t), dtype=torch.uint8, device="cuda")
    code.encode(d, p, cd, code.workspace(fs.OP_ENCODE))
    par, cod = oracle.encode(g, data, t)
    torch.cuda.synchronize()
    assert np.array_equal(host(cd), cod)
    if m:
        assert np.array_equal(host(p), par)
    # decode
    er = np.zeros(n, np.uint8)
    er[gen.sample_indices(n, gen.round_count(frac, n), gen.SEED_ERASE + seed)] = 1
    out = torch.full((b, t), 0xA5, dtype=torch.uint8, device="cuda")
    unrec = torch.empty(b + m, dtype=torch.uint8, device="cuda")
    nun = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = code.workspace(fs.OP_DECODE)
    code.decode(cd, dev(er), out, unrec, nun, ws)
    want, path = oracle.decode(g, cod, er, t)
    torch.cuda.synchronize()
    assert np.array_equal(host(unrec), path.unrecovered)
    assert int(host(nun)[0]) == int(path.unrecovered.sum())
    assert np.array_equal(host(out), want)
    assert fs.Code.ws_status(ws) == fs.FS_OK
    # repair (conventional, from the resident intermediates)
    nl = int(rng.integers(0, n + 1))
    lost = gen.sample_indices(n, nl, gen.SEED_REPAIR + seed)
    if nl:
        cd[dev(lost.astype(np.int64))] = 0
    code.repair(dev(lost.astype(np.int32)), nl, d, p, cd, code.workspace(fs.OP_REPAIR))
    torch.cuda.synchronize()
    assert np.array_equal(host(cd), cod)
    # repair from the local recovery groups (coded blocks only)
    if seed % 4 == 0 and n <= 1200:
        loc = fs.Local(g)
        gl = oracle.local_groups(g)
        gptr, gidx = gl.csr()
        lost_f = np.zeros(n, np.uint8)
        lost_f[gen.sample_indices(n, gen.round_count(0.05, n), gen.SEED_REPAIR + seed + 1)] = 1
        want_l, lpath = oracle.repair_local(gptr, gidx, cod, lost_f, t)
        cl = dev(cod.copy())
        unr = torch.empty(n, dtype=torch.uint8, device="cuda")
        nunr = torch.empty(1, dtype=torch.int32, device="cuda")
        lws = loc.workspace()
        loc.repair(dev(lost_f), cl, t, unr, nunr, lws)
        torch.cuda.synchronize()
        assert np.array_equal(host(cl), want_l)
        assert np.array_equal(host(unr), lpath.unrepaired)
        assert loc.path(lws) == lpath.levels()
    # update (every precode kind)
    u = int(rng.integers(0, b + 1))
    idx = gen.sample_indices(b, u, gen.SEED_UPDATE + seed)
    new = gen.fill_bytes(gen.SEED_NEWDATA + seed, u * t).reshape(u, t)
    code.update(dev(idx.astype(np.int32)), u, dev(new), d, p, cd, code.workspace(fs.OP_UPDATE, u))
    d2, par2, cod2 = oracle.update(g, data, idx, new, t)
    torch.cuda.synchronize()
    assert np.array_equal(host(d), d2) and np.array_equal(host(cd), cod2)
    if m:
        assert np.array_equal(host(p), par2)
