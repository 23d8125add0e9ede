"""Parity of the CUDA path (through the C ABI) with the CPU oracle, bit for
bit: coded and parity bytes, recovered data, unrecovered flags and counts,
the per-level decoding path (Algorithm 5) and device status words."""
import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

pytestmark = pytest.mark.gpu


def _fs():
    from paper_1702_07409_gb300 import founsure
    return founsure


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(x):
    return x.cpu().numpy()


def _erased(n, frac, seed):
    e = np.zeros(n, np.uint8)
    e[gen.sample_indices(n, gen.round_count(frac, n), seed)] = 1
    return e


class Case:
    def __init__(self, b, m, n, t, dist, c=0.0, delta=0.0, seed_data=gen.SEED_DATA, stripe=0,
                 mode=0):
        self.g = gen.make_graph(b, m, n, dist, c, delta, stripe=stripe)
        self.b, self.m, self.n, self.t = b, m, n, t
        self.data = gen.fill_bytes(seed_data + (stripe << gen.STRIPE_SHIFT), b * t).reshape(b, t)
        self.code = _fs().Code(self.g, t, mode)
        self.mode = mode

    def encode_gpu(self):
        import torch
        d = _dev(self.data)
        p = torch.empty((self.m, self.t), dtype=torch.uint8, device="cuda") if self.m else None
        cd = torch.empty((self.n, self.t), dtype=torch.uint8, device="cuda")
        ws = self.code.workspace(_fs().OP_ENCODE)
        self.code.encode(d, p, cd, ws)
        torch.cuda.synchronize()
        return d, p, cd

    def decode_gpu(self, coded_dev, erased):
        import torch
        out = torch.full((self.b, self.t), 0xA5, dtype=torch.uint8, device="cuda")
        unrec = torch.empty(self.b + self.m, dtype=torch.uint8, device="cuda")
        nun = torch.empty(1, dtype=torch.int32, device="cuda")
        ws = self.code.workspace(_fs().OP_DECODE)
        self.code.decode(coded_dev, _dev(erased), out, unrec, nun, ws)
        torch.cuda.synchronize()
        return out, unrec, nun, ws


def _path_levels(view):
    lo = _host(view["level_off"])
    f = _host(view["pair_f"])
    g = _host(view["pair_g"])
    return [set(zip(f[lo[l]:lo[l + 1]].tolist(), g[lo[l]:lo[l + 1]].tolist()))
            for l in range(view["n_levels"])]


def _check_decode(case, coded_np, coded_dev, erased):
    out, unrec, nun, ws = case.decode_gpu(coded_dev, erased)
    want, path = oracle.decode(case.g, coded_np, erased, case.t, case.mode)
    assert np.array_equal(_host(unrec), path.unrecovered)
    assert int(_host(nun)[0]) == int(path.unrecovered.sum())
    assert np.array_equal(_host(out), want)
    view = case.code.decode_path(ws)
    assert view["n_levels"] == path.n_levels and view["n_pairs"] == path.n_pairs
    assert _path_levels(view) == path.levels()
    if case.m:
        _, par = oracle.peel(case.g, coded_np, path, case.t, with_parity=True)
        got = _host(view["parity"]).reshape(case.m, case.t)
        ok = path.unrecovered[case.b:] == 0
        assert np.array_equal(got[ok], par[ok])
    path.plan = _host(view["plan"])
    path.big = (case.b + case.m) * case.t >= 64 << 20  # the default key walk's size
    return path


@pytest.mark.parametrize("t", [1024, 16, 48, 4096 + 16])
def test_config1_plain_lt(t):
    """k=100 x t, RSD(0.1, 0.05), n=150, 30 erasures (usually a stall)."""
    case = Case(100, 0, 150, t, gen.DIST_RSD, 0.1, 0.05)
    _, _, cd = case.encode_gpu()
    _, want = oracle.encode(case.g, case.data, t)
    assert np.array_equal(_host(cd), want)
    for s in range(3):
        erased = np.zeros(150, np.uint8)
        erased[gen.sample_indices(150, 30, gen.SEED_ERASE + (s << gen.ROUND_SHIFT))] = 1
        _check_decode(case, want, cd, erased)
    # nothing erased, then everything erased
    _check_decode(case, want, cd, np.zeros(150, np.uint8))
    _check_decode(case, want, cd, np.ones(150, np.uint8))


@pytest.mark.parametrize("mode", [0, 1])
def test_precoded_midsize_both_modes(mode):
    case = Case(700, 40, 950, 272, gen.DIST_FINITE40, mode=mode)
    _, p, cd = case.encode_gpu()
    par, cod = oracle.encode(case.g, case.data, case.t)
    assert np.array_equal(_host(p), par) and np.array_equal(_host(cd), cod)
    for s, frac in enumerate((0.1, 0.2, 0.3)):
        _check_decode(case, cod, cd, _erased(case.n, frac, gen.SEED_ERASE + (s << 20)))


def test_config2_full_size_encode_decode():
    """k=4096 x 64 KiB, 128 checks (3 per data block), n=5400, FiniteDist
    max-degree-40, 20% erasures: full comparison with the oracle."""
    case = Case(4096, 128, 5400, 65536, gen.DIST_FINITE40)
    _, p, cd = case.encode_gpu()
    par, cod = oracle.encode(case.g, case.data, case.t)
    assert np.array_equal(_host(p), par)
    assert np.array_equal(_host(cd), cod)
    path = _check_decode(case, cod, cd, _erased(case.n, 0.2, gen.SEED_ERASE))
    assert path.unrecovered.sum() == 0
    # a stalled draw is reproduced exactly too
    _check_decode(case, cod, cd, _erased(case.n, 0.2, gen.SEED_ERASE + (2 << 20)))


def test_config2_full_size_two_pass_key_walk():
    """The full-size precoded stripe decoded in the paper's two passes (the
    LT rows to their fixpoint, then the checks) by the default payload, the
    key walk, whose plan must have been made (this draw leaves 87
    intermediates that the joint decoder recovers); a second draw too."""
    case = Case(4096, 128, 5400, 65536, gen.DIST_FINITE40, mode=1)
    _, p, cd = case.encode_gpu()
    _, cod = oracle.encode(case.g, case.data, case.t)
    path = _check_decode(case, cod, cd, _erased(case.n, 0.2, gen.SEED_ERASE))
    assert path.n_pairs > 4000
    assert path.plan[2] == 1 and path.plan[7] == 1, path.plan
    _check_decode(case, cod, cd, _erased(case.n, 0.2, gen.SEED_ERASE + (2 << 20)))


def test_update_and_repair_rounds():
    """Config-4 shape at reduced t: rewrite 1% of data, then repair 5% of coded."""
    import torch
    b, m, n, t = 4096, 128, 5400, 4096
    case = Case(b, m, n, t, gen.DIST_FINITE40)
    d, p, cd = case.encode_gpu()
    data = case.data.copy()
    u = gen.round_count(0.01, b)
    ws_u = case.code.workspace(_fs().OP_UPDATE, u)
    ws_r = case.code.workspace(_fs().OP_REPAIR)
    for rnd in range(2):
        idx = gen.sample_indices(b, u, gen.SEED_UPDATE + (rnd << gen.ROUND_SHIFT))
        new = gen.fill_bytes(gen.SEED_NEWDATA + (rnd << gen.ROUND_SHIFT), u * t).reshape(u, t)
        case.code.update(_dev(idx), u, _dev(new), d, p, cd, ws_u)
        data, par, cod = oracle.update(case.g, data, idx, new, t)
        assert case.code.ws_status(ws_u) == 0
        assert np.array_equal(_host(d), data)
        assert np.array_equal(_host(p), par)
        assert np.array_equal(_host(cd), cod)
        nl = gen.round_count(0.05, n)
        lost = gen.sample_indices(n, nl, gen.SEED_REPAIR + (rnd << gen.ROUND_SHIFT))
        cd[torch.from_numpy(lost).long().cuda()] = 0
        case.code.repair(_dev(lost), nl, d, p, cd, ws_r)
        assert case.code.ws_status(ws_r) == 0
        assert np.array_equal(_host(cd), cod)


def test_config4_full_size_rounds():
    """Config 4 at its own size: the precoded stripe (b=4096 x 64 KiB, m=128,
    n=5400) through 10 rounds of 1% of the data rewritten (41 blocks) and 5%
    of the coded blocks lost and repaired (270). Every round, every block is
    compared with the oracle on two sampled byte slices (byte slices are
    independent copies of the same problem, so the oracle encodes only those
    columns); at full width the delta-updated parities and coded blocks must
    equal a fresh encode of the updated data, and the repaired blocks the
    bytes they had before the loss."""
    import torch
    b, m, n, t = 4096, 128, 5400, 65536
    case = Case(b, m, n, t, gen.DIST_FINITE40)
    d, p, cd = case.encode_gpu()
    cols = np.r_[0:4096, t // 2 + 1024:t // 2 + 3072]  # two slices, 6 KiB of every block
    ts = cols.size
    data_s = case.data[:, cols].copy()
    u, nl = gen.round_count(0.01, b), gen.round_count(0.05, n)
    ws_u = case.code.workspace(_fs().OP_UPDATE, u)
    ws_r = case.code.workspace(_fs().OP_REPAIR)
    ws_e = case.code.workspace(_fs().OP_ENCODE)
    dcols = torch.from_numpy(cols).cuda()
    p2 = torch.empty_like(p)
    cd2 = torch.empty_like(cd)
    for rnd in range(10):
        idx = gen.sample_indices(b, u, gen.SEED_UPDATE + (rnd << gen.ROUND_SHIFT))
        new = gen.fill_bytes(gen.SEED_NEWDATA + (rnd << gen.ROUND_SHIFT), u * t).reshape(u, t)
        case.code.update(_dev(idx), u, _dev(new), d, p, cd, ws_u)
        data_s, par_s, cod_s = oracle.update(case.g, data_s, idx, new[:, cols], ts)
        assert case.code.ws_status(ws_u) == 0
        assert np.array_equal(_host(d.index_select(1, dcols)), data_s)
        assert np.array_equal(_host(p.index_select(1, dcols)), par_s)
        assert np.array_equal(_host(cd.index_select(1, dcols)), cod_s)
        case.code.encode(d, p2, cd2, ws_e)
        assert torch.equal(p2, p) and torch.equal(cd2, cd)
        lost = gen.sample_indices(n, nl, gen.SEED_REPAIR + (rnd << gen.ROUND_SHIFT))
        dl = torch.from_numpy(lost).long().cuda()
        before = cd.index_select(0, dl)
        cd.index_fill_(0, dl, 0)
        case.code.repair(_dev(lost), nl, d, p, cd, ws_r)
        assert case.code.ws_status(ws_r) == 0
        assert torch.equal(cd.index_select(0, dl), before)
        assert np.array_equal(_host(cd.index_select(0, dl).index_select(1, dcols)),
                              oracle.repair(case.g, data_s, lost, ts))


def test_encode_rows_and_empty_calls():
    import torch
    case = Case(300, 12, 420, 64, gen.DIST_FINITE40)
    d, p, cd = case.encode_gpu()
    _, cod = oracle.encode(case.g, case.data, case.t)
    cd2 = torch.zeros_like(cd)
    ws = case.code.workspace(_fs().OP_ENCODE)
    ws[:4].view(torch.int32).fill_(_fs().FS_ERR_INVALID)  # a stale status from an earlier call
    case.code.encode_rows(100, 250, d, p, cd2, ws)
    torch.cuda.synchronize()
    got = _host(cd2)
    assert np.array_equal(got[100:250], cod[100:250]) and not got[:100].any() and not got[250:].any()
    assert _fs().Code.ws_status(ws) == _fs().FS_OK
    # n_idx = 0 and n_lost = 0 leave everything untouched
    before = (_host(d).copy(), _host(p).copy(), _host(cd).copy())
    case.code.update(None, 0, None, d, p, cd, case.code.workspace(_fs().OP_UPDATE, 0))
    case.code.repair(None, 0, d, p, cd, case.code.workspace(_fs().OP_REPAIR))
    torch.cuda.synchronize()
    assert all(np.array_equal(x, y) for x, y in zip(before, (_host(d), _host(p), _host(cd))))


def test_device_detected_bad_indices():
    import torch
    fs = _fs()
    case = Case(200, 8, 260, 32, gen.DIST_FINITE40)
    d, p, cd = case.encode_gpu()
    snapshot = (_host(d).copy(), _host(p).copy(), _host(cd).copy())
    new = _dev(np.zeros((2, 32), np.uint8))
    ws = case.code.workspace(fs.OP_UPDATE, 2)
    case.code.update(_dev(np.array([5, 5], np.int32)), 2, new, d, p, cd, ws)   # repeated
    assert case.code.ws_status(ws) == fs.FS_ERR_INVALID
    case.code.update(_dev(np.array([5, 200], np.int32)), 2, new, d, p, cd, ws)  # out of range
    assert case.code.ws_status(ws) == fs.FS_ERR_INVALID
    # a rejected update changes nothing
    assert all(np.array_equal(x, y) for x, y in zip(snapshot, (_host(d), _host(p), _host(cd))))
    wr = case.code.workspace(fs.OP_REPAIR)
    case.code.repair(_dev(np.array([3, 260, -1], np.int32)), 3, d, p, cd, wr)
    assert case.code.ws_status(wr) == fs.FS_ERR_INVALID
    _, cod = oracle.encode(case.g, case.data, 32)
    assert np.array_equal(_host(cd), cod)  # row 3 recomputed to the same bytes
    # a clean call on the same workspace reads FS_OK again
    case.code.repair(_dev(np.array([3], np.int32)), 1, d, p, cd, wr)
    assert case.code.ws_status(wr) == fs.FS_OK


def test_host_side_rejections():
    import torch
    fs = _fs()
    case = Case(64, 0, 90, 32, gen.DIST_RSD, 0.1, 0.05)
    d = torch.zeros(64 * 32 + 16, dtype=torch.uint8, device="cuda")
    cd = torch.zeros(90 * 32 + 16, dtype=torch.uint8, device="cuda")
    ws = case.code.workspace(fs.OP_ENCODE)
    with pytest.raises(fs.FounsureError) as ei:
        case.code.encode(d[1:], None, cd, ws)      # misaligned input
    assert ei.value.status == fs.FS_ERR_INVALID
    with pytest.raises(fs.FounsureError):
        case.code.encode(d, d, cd, ws)              # parity given for m == 0
    g = case.g
    bad = gen.Graph(g.b, 0, g.n, g.pre_ptr, g.pre_idx, g.lt_ptr, g.lt_idx.copy())
    bad.lt_idx[0] = 10 ** 6
    with pytest.raises(fs.FounsureError):
        fs.Code(bad, 32)
    with pytest.raises(fs.FounsureError):
        fs.Code(g, 24)                               # t not a multiple of 16


def test_zero_coded_rows():
    import torch
    fs = _fs()
    g = gen.Graph(4, 0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32),
                  np.zeros(1, np.int32), np.zeros(0, np.int32))
    code = fs.Code(g, 16)
    out = torch.full((4, 16), 7, dtype=torch.uint8, device="cuda")
    unrec = torch.empty(4, dtype=torch.uint8, device="cuda")
    nun = torch.empty(1, dtype=torch.int32, device="cuda")
    code.decode(None, None, out, unrec, nun, code.workspace(fs.OP_DECODE))
    torch.cuda.synchronize()
    assert not _host(out).any() and _host(unrec).all() and int(_host(nun)[0]) == 4


def _csr(rows):
    ptr = np.zeros(len(rows) + 1, np.int32)
    for j, r in enumerate(rows):
        ptr[j + 1] = ptr[j] + len(r)
    return ptr, np.array([v for r in rows for v in sorted(r)], dtype=np.int32)


def _graph_from_rows(b, rows, checks=()):
    """LT rows over the intermediates and precode checks over the data."""
    ptr, idx = _csr(rows)
    pptr, pidx = _csr(list(checks))
    return gen.Graph(b, len(checks), len(rows), pptr, pidx, ptr, idx)


def _check_plain(g, t, erased, tuning=None):
    import torch
    fs = _fs()
    data = gen.fill_bytes(11, g.b * t).reshape(g.b, t)
    code = fs.Code(g, t)
    for knob, value in (tuning or {}).items():
        code.set_tuning(knob, value)
    _, cod = oracle.encode(g, data, t)
    cd = _dev(cod)
    out = torch.empty((g.b, t), dtype=torch.uint8, device="cuda")
    unrec = torch.empty(g.b + g.m, dtype=torch.uint8, device="cuda")
    nun = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = code.workspace(fs.OP_DECODE)
    code.decode(cd, _dev(erased), out, unrec, nun, ws)
    want, path = oracle.decode(g, cod, erased, t)
    torch.cuda.synchronize()
    assert np.array_equal(_host(unrec), path.unrecovered)
    assert np.array_equal(_host(out), want)
    view = code.decode_path(ws)
    assert view["n_levels"] == path.n_levels
    assert _path_levels(view) == path.levels()
    if g.m:
        _, par = oracle.peel(g, cod, path, t, with_parity=True)
        got = _host(view["parity"]).reshape(g.m, t)
        ok = path.unrecovered[g.b:] == 0
        assert np.array_equal(got[ok], par[ok])
    assert fs.Code.ws_status(ws) == fs.FS_OK
    path.plan = _host(view["plan"])
    path.big = (g.b + g.m) * t >= 64 << 20  # the default key walk's size
    return path


@pytest.mark.parametrize("cols", [0, 1])
def test_wide_level_takes_the_direct_path(cols):
    """600 degree-1 rows: one level of 600 pairs, more than a shared-memory
    stage of the slice payload holds, so it reads the path straight from
    global memory; the column payload has no segment for them."""
    b = 600
    rows = [[j] for j in range(b)] + [[j, (j + 1) % b] for j in range(40)]
    g = _graph_from_rows(b, rows)
    erased = np.zeros(len(rows), np.uint8)
    erased[gen.sample_indices(b, 30, 5)] = 1
    path = _check_plain(g, 48, erased, {_fs().TUNE_PEEL_COLUMNS: cols})
    assert max(len(s) for s in path.levels()) > 256


@pytest.mark.parametrize("cols", [0, 1])
def test_long_chain_takes_the_direct_path(cols):
    """Row 0 = {0}, row j = {j-1, j}: one symbol per level, 1100 levels (the
    column payload: 1099 steps of one segment)."""
    b = 1100
    rows = [[0]] + [[j - 1, j] for j in range(1, b)]
    g = _graph_from_rows(b, rows)
    path = _check_plain(g, 32, np.zeros(b, np.uint8), {_fs().TUNE_PEEL_COLUMNS: cols})
    assert path.n_levels == b


@pytest.mark.parametrize("cols", [0, 1])
@pytest.mark.parametrize("t", [16, 4096 + 48])
def test_wide_check_level_splits_into_steps(cols, t):
    """64 precode checks of 32 data blocks each (check j: j, j + 64, ...);
    every data block and parity has its own degree-1 row. Erasing rows 0..63
    leaves each check one unknown, so one level recovers 64 data blocks from
    zero-payload constraints of 33 members: 320 column segments, more than
    one step of 256 holds."""
    b, m = 2048, 64
    checks = [[j + 64 * i for i in range(32)] for j in range(m)]
    rows = [[v] for v in range(b + m)]
    g = _graph_from_rows(b, rows, checks)
    erased = np.zeros(len(rows), np.uint8)
    erased[:64] = 1
    path = _check_plain(g, t, erased, {_fs().TUNE_PEEL_COLUMNS: cols})
    assert path.n_levels == 2 and not path.unrecovered.any()
    assert all(gg >= len(rows) for f, gg in path.levels()[1])


@pytest.mark.parametrize("knob,value", [(1, 2), (1, 4), (2, 1), (3, 0), (4, 1), (5, 0), (5, 2),
                                        (5, 3), (7, 1), (8, 0), (8, 1), (8, 3)])
def test_tuning_knobs_leave_results_unchanged(knob, value):
    """Payload CTAs per SM, one gather CTA per SM, general (not compact)
    decoding schedule, L2 eviction hints, row-gather encode, 16- and 32-byte
    slice encode, column payload, the level walk, the barrier-free
    (dataflow) walk and the key walk at this size (the default keeps it for
    larger stripes)."""
    import torch
    fs = _fs()
    case = Case(1500, 60, 2000, 4096 + 32, gen.DIST_FINITE40)
    case.code.set_tuning(knob, value)
    _, p, cd = case.encode_gpu()
    par, cod = oracle.encode(case.g, case.data, case.t)
    assert np.array_equal(_host(p), par) and np.array_equal(_host(cd), cod)
    for s in range(2):
        _check_decode(case, cod, cd, _erased(case.n, 0.15, gen.SEED_ERASE + (s << 20)))
    with pytest.raises(fs.FounsureError):
        case.code.set_tuning(knob, 99)


@pytest.mark.parametrize("rows", [1, 3, 16])
def test_row_gather_encode_rows_per_ticket(rows):
    """The row-gather encode (slices off) with 1, 3 or 16 coded rows per work
    ticket, precoded and plain codes, ragged block size."""
    fs = _fs()
    for b, m, n, t in ((1500, 60, 2000, 4096 + 32), (300, 0, 400, 48)):
        case = Case(b, m, n, t, gen.DIST_FINITE40)
        case.code.set_tuning(fs.TUNE_ENCODE_SLICES, 0)
        case.code.set_tuning(fs.TUNE_ROWS_PER_TICKET, rows)
        _, p, cd = case.encode_gpu()
        par, cod = oracle.encode(case.g, case.data, case.t)
        assert np.array_equal(_host(cd), cod)
        if m:
            assert np.array_equal(_host(p), par)
    with pytest.raises(fs.FounsureError):
        case.code.set_tuning(fs.TUNE_ROWS_PER_TICKET, 17)


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait that nothing will satisfy gives up after its limit, reports
    FS_ERR_TIMEOUT, and the context still runs kernels afterwards."""
    fs = _fs()
    assert fs.selftest_timeout() == fs.FS_ERR_TIMEOUT
    case = Case(100, 0, 150, 1024, gen.DIST_RSD, 0.1, 0.05)
    _, _, cd = case.encode_gpu()
    _, want = oracle.encode(case.g, case.data, case.t)
    assert np.array_equal(_host(cd), want)


@pytest.mark.parametrize("t", [1024, 4096 + 16])
def test_large_code_encodes_in_parts(t):
    """A code whose slice tables do not fit beside two slot buffers (RSD
    k=4096, n=5325: ~190 KB of tables) is encoded in several parts, each
    reading the data again; the result is the oracle's."""
    case = Case(4096, 0, 5325, t, gen.DIST_RSD, 0.05, 0.01)
    _, _, cd = case.encode_gpu()
    _, want = oracle.encode(case.g, case.data, t)
    assert np.array_equal(_host(cd), want)
    pre = Case(3000, 96, 4000, 2048, gen.DIST_RSD, 0.05, 0.01)  # parts with parities
    _, p, cd = pre.encode_gpu()
    par, cod = oracle.encode(pre.g, pre.data, pre.t)
    assert np.array_equal(_host(cd), cod) and np.array_equal(_host(p), par)


def test_column_payload_without_its_plan_reports_invalid():
    """The column payload's plan is built by the decoding schedule only when
    that payload is selected; a payload run after a schedule without it
    reports FS_ERR_INVALID in the workspace status and writes nothing."""
    import torch
    fs = _fs()
    case = Case(300, 12, 400, 64, gen.DIST_FINITE40)
    _, _, cd = case.encode_gpu()
    er = _dev(_erased(case.n, 0.1, gen.SEED_ERASE))
    out = torch.full((case.b, case.t), 0x5A, dtype=torch.uint8, device="cuda")
    unrec = torch.empty(case.b + case.m, dtype=torch.uint8, device="cuda")
    nun = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = case.code.workspace(fs.OP_DECODE)
    case.code.decode_schedule(er, unrec, nun, ws)  # slice payload selected: no plan
    case.code.set_tuning(fs.TUNE_PEEL_COLUMNS, 1)
    case.code.decode_payload(cd, out, ws)
    assert fs.Code.ws_status(ws) == fs.FS_ERR_INVALID
    assert bool((out == 0x5A).all())
    # with the plan (schedule run with the column payload selected) it decodes
    ws2 = case.code.workspace(fs.OP_DECODE)
    case.code.decode(cd, er, out, unrec, nun, ws2)
    assert fs.Code.ws_status(ws2) == fs.FS_OK
    want, _ = oracle.decode(case.g, _host(cd), _host(er), case.t)
    assert np.array_equal(_host(out), want)


def test_code_extension_encodes_only_the_new_rows():
    """The paper's update (making a code stronger): e more coded blocks from
    the same degree distribution. The generator keeps the first n rows when
    n grows, so the extended code is the old one plus rows n..n+e-1, and
    fs_encode_rows computes just those from the resident data; the old coded
    blocks stay as they are, and the extended code decodes erasures the old
    one could not."""
    import torch
    fs = _fs()
    b, m, n, e, t = 600, 24, 700, 200, 64
    g = gen.make_graph(b, m, n, gen.DIST_FINITE40, stripe=9)
    gx = gen.make_graph(b, m, n + e, gen.DIST_FINITE40, stripe=9)
    assert np.array_equal(gx.lt_ptr[:n + 1], g.lt_ptr) and np.array_equal(gx.pre_idx, g.pre_idx)
    data = gen.fill_bytes(gen.SEED_DATA + 9, b * t).reshape(b, t)
    par, cod = oracle.encode(g, data, t)
    parx, codx = oracle.encode(gx, data, t)
    assert np.array_equal(codx[:n], cod) and np.array_equal(parx, par)
    code_x = fs.Code(gx, t)
    d = _dev(data)
    p = _dev(par)
    cd = torch.zeros((n + e, t), dtype=torch.uint8, device="cuda")
    cd[:n] = _dev(cod)
    code_x.encode_rows(n, n + e, d, p, cd, code_x.workspace(fs.OP_ENCODE))
    torch.cuda.synchronize()
    assert np.array_equal(_host(cd), codx)
    erased = np.zeros(n + e, np.uint8)
    erased[gen.sample_indices(n, gen.round_count(0.35, n), gen.SEED_ERASE + 9)] = 1
    old = oracle.dpg(g, erased[:n])
    new = oracle.dpg(gx, erased)
    assert int(new.unrecovered.sum()) < int(old.unrecovered.sum())
    case = Case.__new__(Case)
    case.g, case.b, case.m, case.n, case.t, case.code, case.mode = gx, b, m, n + e, t, code_x, 0
    _check_decode(case, codx, cd, erased)


@pytest.mark.parametrize("t", [48, 4096 + 16])
def test_array_precode_encode_decode(t):
    """The array LDPC precode of Algorithm 2 (b = 4154, k = 4288: p = 67, two
    levels of 67 checks, the second reading parities of the first) under an
    LT code of n = 5574: the level-by-level encode and the joint decode are
    bit-exact against the oracle, and so are a delta update and a batched
    encode (parity levels in order)."""
    import torch
    fs = _fs()
    b, k, n = 4154, 4288, 5574
    g = gen.make_graph_array(b, k, n, gen.DIST_FINITE40)
    m = k - b
    data = gen.fill_bytes(gen.SEED_DATA + 5, b * t).reshape(b, t)
    code = fs.Code(g, t)
    d = _dev(data)
    p = torch.empty((m, t), dtype=torch.uint8, device="cuda")
    cd = torch.empty((n, t), dtype=torch.uint8, device="cuda")
    code.encode(d, p, cd, code.workspace(fs.OP_ENCODE))
    torch.cuda.synchronize()
    par, cod = oracle.encode(g, data, t)
    assert np.array_equal(_host(p), par) and np.array_equal(_host(cd), cod)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cd.zero_()
    code.encode_static(d, p, cd, st)
    torch.cuda.synchronize()
    assert np.array_equal(_host(cd), cod)
    case = Case.__new__(Case)
    case.g, case.b, case.m, case.n, case.t, case.code, case.mode = g, b, m, n, t, code, 0
    path = _check_decode(case, cod, cd, _erased(n, 0.15, gen.SEED_ERASE + 5))
    assert path.n_pairs > 0
    # the delta update runs the parity levels in order: rewrite 2% of the data
    u = gen.round_count(0.02, b)
    idx = gen.sample_indices(b, u, gen.SEED_UPDATE + 5)
    new = gen.fill_bytes(gen.SEED_NEWDATA + 5, u * t).reshape(u, t)
    cd.copy_(_dev(cod))
    code.update(_dev(idx.astype(np.int32)), u, _dev(new), d, p, cd, code.workspace(fs.OP_UPDATE, u))
    d2, par2, cod2 = oracle.update(g, data, idx, new, t)
    torch.cuda.synchronize()
    assert np.array_equal(_host(d), d2) and np.array_equal(_host(p), par2)
    assert np.array_equal(_host(cd), cod2)
    d.copy_(_dev(data))
    p.copy_(_dev(par))
    cd.copy_(_dev(cod))
    # a batch encode of the chained code beside a data-only precoded one (one
    # precode launch per level), eager and from a captured CUDA graph
    g2 = gen.make_graph(300, 12, 400, gen.DIST_FINITE40, stripe=5)
    data2 = gen.fill_bytes(gen.SEED_DATA + 6, 300 * t).reshape(300, t)
    code2 = fs.Code(g2, t)
    d2b, p2b = _dev(data2), torch.empty((12, t), dtype=torch.uint8, device="cuda")
    cd2 = torch.empty((400, t), dtype=torch.uint8, device="cuda")
    pb = torch.empty_like(p)
    cdb = torch.empty_like(cd)
    enc = fs.Batch([{"code": code, "data": d, "parity": pb, "coded": cdb},
                    {"code": code2, "data": d2b, "parity": p2b, "coded": cd2}], fs.OP_ENCODE)
    enc.run()
    torch.cuda.synchronize()
    par2, cod2b = oracle.encode(g2, data2, t)
    assert np.array_equal(_host(pb), par) and np.array_equal(_host(cdb), cod)
    assert np.array_equal(_host(p2b), par2) and np.array_equal(_host(cd2), cod2b)
    pb.zero_()
    cdb.zero_()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            enc.run(torch.cuda.current_stream())
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(_host(pb), par) and np.array_equal(_host(cdb), cod)
    assert enc.status() == fs.FS_OK
    out = torch.empty((b, t), dtype=torch.uint8, device="cuda")
    dec = fs.Batch([{"code": code, "coded": cd, "erased": _dev(_erased(n, 0.15, gen.SEED_ERASE + 5)),
                     "data_out": out, "unrecovered": torch.empty(k, dtype=torch.uint8, device="cuda"),
                     "n_unrecovered": torch.empty(1, dtype=torch.int32, device="cuda"),
                     "ws": code.workspace(fs.OP_DECODE)}], fs.OP_DECODE)
    dec.run()
    torch.cuda.synchronize()
    want, _ = oracle.decode(g, cod, _erased(n, 0.15, gen.SEED_ERASE + 5), t)
    assert np.array_equal(_host(out), want)


def test_chained_precode_validation():
    """A chained check may read only earlier parities, and the checks must
    come in level order."""
    fs = _fs()
    lt = [[0], [1], [2], [3], [4], [5], [0, 4]]

    def graph(checks):
        ptr = np.zeros(len(checks) + 1, np.int32)
        for j, r in enumerate(checks):
            ptr[j + 1] = ptr[j] + len(r)
        idx = np.array([v for r in checks for v in r], np.int32)
        lp = np.zeros(len(lt) + 1, np.int32)
        for j, r in enumerate(lt):
            lp[j + 1] = lp[j] + len(r)
        return gen.Graph(3, len(checks), len(lt), ptr, idx, lp,
                         np.array([v for r in lt for v in r], np.int32), chained=True)

    fs.Code(graph([[0, 1], [2, 3], [1, 3, 4]]), 16).close()  # levels 0, 1, 2
    with pytest.raises(fs.FounsureError):
        fs.Code(graph([[0, 1], [2, 4], [1, 2]]), 16)  # check 1 reads its own parity
    with pytest.raises(fs.FounsureError):
        fs.Code(graph([[0, 1], [2, 3], [1, 2]]), 16)  # level 1 before level 0


@pytest.mark.parametrize("walk", [0, 1, 2, 3])
@pytest.mark.parametrize("case", ["precoded_joint", "precoded_two_pass", "long_chain", "wide_checks",
                                  "rsd_plain", "array_precode", "config2", "plan_overflow",
                                  "general_schedule"])
def test_flow_payload_matches_oracle(case, walk):
    """The payload walks, byte for byte against the oracle: walk 0 (level
    by level), walk 1 (FS_TUNE_PEEL_FLOW = 1, no level barriers; precode
    checks summed in shared-memory slots), walk 3 (the key walk: one barrier
    per level, every heavy pair chained through its output block, its pieces
    in the member order the schedule recorded) and walk 2 (the default: the
    key walk from 64 MiB of intermediates, here only the full-size stripe,
    the level walk below). Cases:
    precoded, both decoding modes, several erasure rates; one symbol per
    level (1100 keys: more than the key walk's table, so walk 3 falls back to
    the level walk); checks of 32 members in one level (after a level of 2112
    pairs, more than the key walk's stage: walk 3 falls back); long RSD rows (units
    of more than one round of loads); a chained (array) precode whose checks
    read parities; the full-size precoded stripe; a path whose key plan
    exceeds the plan kernel's tables (8000 pairs, 47 K loads) and the general
    (not compact) schedule, which records no member order: walks 2 and 3 fall
    back to the level walk there. Walk 3 must have run on its plan wherever it
    fits, and walks 0 (and 2 below its size) made none (the plan header says
    so)."""
    fs = _fs()
    flow = {fs.TUNE_PEEL_FLOW: walk}
    paths = []
    if case.startswith("precoded"):
        c = Case(700, 40, 950, 272, gen.DIST_FINITE40, mode=1 if case.endswith("two_pass") else 0)
        c.code.set_tuning(fs.TUNE_PEEL_FLOW, walk)
        _, p, cd = c.encode_gpu()
        _, cod = oracle.encode(c.g, c.data, c.t)
        for s, frac in enumerate((0.1, 0.2, 0.3)):
            paths.append(_check_decode(c, cod, cd, _erased(c.n, frac, gen.SEED_ERASE + (s << 20))))
    elif case == "long_chain":
        b = 1100
        g = _graph_from_rows(b, [[0]] + [[j - 1, j] for j in range(1, b)])
        path = _check_plain(g, 32, np.zeros(b, np.uint8), flow)
        assert path.n_levels == b
        if walk >= 2:
            assert path.plan[7] == 0  # no key walk: the level walk ran
    elif case == "wide_checks":
        b, m = 2048, 64
        g = _graph_from_rows(b, [[v] for v in range(b + m)],
                             [[j + 64 * i for i in range(32)] for j in range(m)])
        erased = np.zeros(b + m, np.uint8)
        erased[:64] = 1
        path = _check_plain(g, 4096 + 48, erased, flow)
        assert not path.unrecovered.any()
        if walk >= 2:
            # level 0 holds 2112 whole pairs, more than the key walk's stage
            # of 1024 units: the level walk ran
            assert path.plan[7] == 0
        else:
            paths.append(path)
    elif case == "rsd_plain":
        g = gen.make_graph(2000, 0, 2600, gen.DIST_RSD, 0.05, 0.01)
        for s in range(2):
            paths.append(_check_plain(g, 1024 + 16, _erased(2600, 0.1, gen.SEED_ERASE + (s << 20)), flow))
    elif case == "plan_overflow":
        g = gen.make_graph(8000, 0, 10400, gen.DIST_RSD, 0.05, 0.01)
        path = _check_plain(g, 64, _erased(10400, 0.1, gen.SEED_ERASE), flow)
        assert path.n_pairs == 8000
        if walk >= 2:
            assert path.plan[7] == 0  # no key walk: the level walk ran
    elif case == "general_schedule":
        c = Case(700, 40, 950, 272, gen.DIST_FINITE40)
        c.code.set_tuning(fs.TUNE_PEEL_FLOW, walk)
        c.code.set_tuning(fs.TUNE_DPG_COMPACT, 0)
        _, p, cd = c.encode_gpu()
        _, cod = oracle.encode(c.g, c.data, c.t)
        path = _check_decode(c, cod, cd, _erased(c.n, 0.2, gen.SEED_ERASE))
        if walk >= 2:
            assert path.plan[7] == 0  # no member order: the level walk ran
    elif case == "array_precode":
        # p = 67, two levels of 67 checks (the second reads parities of the first)
        g = gen.make_graph_array(1005, 1139, 1481, gen.DIST_FINITE40)
        paths.append(_check_plain(g, 512, _erased(g.n, 0.15, gen.SEED_ERASE), flow))
    else:
        c = Case(4096, 128, 5400, 65536, gen.DIST_FINITE40)
        c.code.set_tuning(fs.TUNE_PEEL_FLOW, walk)
        _, p, cd = c.encode_gpu()
        _, cod = oracle.encode(c.g, c.data, c.t)
        paths.append(_check_decode(c, cod, cd, _erased(c.n, 0.2, gen.SEED_ERASE)))
    for path in paths:
        keys = walk == 3 or (walk == 2 and path.big)
        if keys and path.n_pairs:
            assert path.plan[2] == 1 and path.plan[7] == 1, path.plan
        if walk == 0 or (walk == 2 and not path.big):
            assert not path.plan.any(), path.plan  # no plan
