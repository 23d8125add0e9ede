"""Serving loop: each request's result is the same whether it runs alone
(one request per launch, in arrival order) or mixed into continuously formed
batches with other requests; admission never exceeds the memory budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests(seed=7, n_req=48):
    from paper_1702_07409_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs, sid = [], 100
    t_now = 0.0
    live = list(range(6))  # the pre-populated stripes 0..5
    for i in range(n_req):
        t_now += float(rng.exponential(1e-4))
        u = rng.random()
        if u < 0.4:
            k = int(rng.choice([32, 64, 128, 300]))
            t = int(rng.choice([64, 1024, 4096]))
            reqs.append(Request(i, "encode", t_now, k=k, t=t, target=sid, seed=1000 + i))
            live.append(sid)
            sid += 1
        elif u < 0.75:
            reqs.append(Request(i, "decode", t_now, target=int(rng.choice(live)), seed=2000 + i,
                                erase_frac=float(rng.uniform(0.05, 0.25))))
        elif u < 0.9:
            reqs.append(Request(i, "update", t_now, target=int(rng.choice(live)), seed=3000 + i,
                                n_update=2))
        else:
            reqs.append(Request(i, "repair", t_now, target=int(rng.choice(live)), seed=4000 + i,
                                n_lost=3))
    return reqs


def _serve(batching, budget=1 << 30):
    import torch
    from paper_1702_07409_gb300.serve import Server
    srv = Server(budget, streams=3 if batching else 1, batching=batching)
    for i in range(6):
        srv.add_resident(i, k=int([32, 64, 128, 300, 64, 32][i]), t=int([64, 1024, 4096, 64, 4096, 1024][i]),
                         seed=10 + i)
    reqs = srv.run(_requests(), realtime=False)
    torch.cuda.synchronize()
    dec = {r.rid: (r.out["data_out"].cpu().numpy(), int(r.out["n_unrecovered"].item()))
           for r in reqs if r.kind == "decode" and not r.out.get("dropped")}
    state = {sid: (st.data.cpu().numpy(), st.coded.cpu().numpy()) for sid, st in srv.stripes.items()}
    peak, budget_ = srv.peak, srv.budget
    waves = srv.n_waves
    srv.close()
    return dec, state, peak, budget_, reqs, waves


def test_mixed_equals_alone_and_budget_holds():
    dec_m, st_m, peak_m, budget, reqs_m, waves_m = _serve(True)
    dec_a, st_a, peak_a, _, reqs_a, waves_a = _serve(False)
    assert waves_m < waves_a  # requests were grouped
    assert peak_m <= budget and peak_a <= budget
    assert dec_m.keys() == dec_a.keys() and len(dec_m) > 5
    for rid in dec_m:
        assert np.array_equal(dec_m[rid][0], dec_a[rid][0])
        assert dec_m[rid][1] == dec_a[rid][1]
    assert st_m.keys() == st_a.keys()
    for sid in st_m:
        assert np.array_equal(st_m[sid][0], st_a[sid][0])
        assert np.array_equal(st_m[sid][1], st_a[sid][1])
    assert all(r.done is not None for r in reqs_m)


def test_decode_recovers_the_stripe_data():
    """A decode of a stripe with 10% erased returns its data (recovered
    blocks) and zeros (unrecovered ones). The warm-up before it leaves no
    stripe and no bytes behind."""
    import torch
    from paper_1702_07409_gb300.serve import Request, Server
    srv = Server(1 << 30, streams=2)
    srv.warm_up(((32, 1024), (300, 64)))
    assert not srv.stripes and srv.resident == 0 and srv.transient == 0 and not srv.waiting
    srv.add_resident(0, k=128, t=4096, seed=5)
    data = srv.stripes[0].data.clone()
    reqs = srv.run([Request(0, "decode", 0.0, target=0, seed=9, erase_frac=0.1)], realtime=False)
    torch.cuda.synchronize()
    out = reqs[0].out["data_out"]
    un = reqs[0].out["unrecovered"].bool()
    assert torch.equal(out[~un], data[~un]) and bool((out[un] == 0).all())
    srv.close()


def test_budget_eviction_rejection_and_cancel():
    """Admission under a small budget: resident stripes are evicted least
    recently used first, a later request on an evicted stripe is dropped, a
    request larger than the whole budget is rejected (not left waiting), a
    waiting request can be withdrawn, and the budget is never exceeded."""
    import torch
    from paper_1702_07409_gb300.serve import Request, Server
    k, t = 64, 4096
    stripe_bytes = (k + round(k * 1.3)) * t
    srv = Server(int(3.5 * stripe_bytes), streams=2)
    for i in range(3):
        srv.add_resident(i, k=k, t=t, seed=20 + i)
    assert list(srv.stripes) == [0, 1, 2]
    # a new stripe needs room: the least recently used (0) goes
    srv.run([Request(0, "encode", 0.0, k=k, t=t, target=10, seed=99)], realtime=False)
    assert 0 not in srv.stripes and 10 in srv.stripes and srv.evictions == 1
    # a decode of the evicted stripe is dropped, one of a resident stripe is served
    reqs = srv.run([Request(1, "decode", 0.0, target=0, seed=5, erase_frac=0.1),
                    Request(2, "decode", 0.0, target=1, seed=6, erase_frac=0.1)], realtime=False)
    assert reqs[0].out.get("dropped") and not reqs[1].out.get("dropped")
    # larger than the whole budget: rejected
    before = set(srv.stripes)
    big = srv.run([Request(3, "encode", 0.0, k=4096, t=65536, target=11, seed=7)], realtime=False)
    assert big[0].out.get("rejected") and 11 not in srv.stripes
    assert set(srv.stripes) == before  # nothing evicted for it
    # withdrawn before admission
    srv.submit(Request(4, "decode", 0.0, target=2, seed=8, erase_frac=0.1))
    assert srv.cancel(4) and not srv.cancel(4) and not srv.waiting
    torch.cuda.synchronize()
    assert srv.peak <= srv.budget
    srv.close()


def test_served_results_match_the_oracle():
    """Every result of a mixed, continuously batched run against the oracle:
    the run is replayed on the host stripe by stripe in arrival order (the
    order the server keeps for each stripe), each decode's bytes and
    unrecovered count are compared, and each stripe's final data and coded
    bytes are compared after its updates and repairs. The inputs are the
    server's own seeded draws: graphs from its code rule, erasures, indices
    and lost rows from the generator, bytes from the same seeded torch
    generator."""
    import torch
    import oracle
    from paper_1702_07409_gb300 import gen
    from paper_1702_07409_gb300.serve import Server
    srv = Server(1 << 30, streams=3, batching=True)
    shapes = list(zip([32, 64, 128, 300, 64, 32], [64, 1024, 4096, 64, 4096, 1024]))
    for i, (k, t) in enumerate(shapes):
        srv.add_resident(i, k=k, t=t, seed=10 + i)
    reqs = srv.run(_requests(), realtime=False)
    torch.cuda.synchronize()

    def seeded_bytes(seed, rows, cols):
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        return torch.randint(0, 256, (rows, cols), dtype=torch.uint8, device="cuda",
                             generator=g).cpu().numpy()

    def graph(k, t):
        n = int(round(k / srv.rate))
        return gen.make_graph(k, 0, n, gen.DIST_RSD, 0.05, 0.01, stripe=(k * 131 + t) & 0xFFF)

    state = {}
    for i, (k, t) in enumerate(shapes):
        g = graph(k, t)
        d = seeded_bytes(10 + i, k, t)
        state[i] = [g, t, d, oracle.encode(g, d, t)[1]]
    checked = {"decode": 0, "update": 0, "repair": 0, "encode": 0}
    for r in sorted(reqs, key=lambda q: (q.arrival, q.rid)):
        if r.out.get("dropped") or r.out.get("rejected"):
            continue
        checked[r.kind] += 1
        if r.kind == "encode":
            g = graph(r.k, r.t)
            d = seeded_bytes(r.seed, r.k, r.t)
            state[r.target] = [g, r.t, d, oracle.encode(g, d, r.t)[1]]
            continue
        g, t, d, c = state[r.target]
        if r.kind == "decode":
            er = np.zeros(g.n, np.uint8)
            er[gen.sample_indices(g.n, gen.round_count(r.erase_frac, g.n), r.seed)] = 1
            want, path = oracle.decode(g, c, er, t)
            assert np.array_equal(r.out["data_out"].cpu().numpy(), want)
            assert int(r.out["n_unrecovered"].item()) == int(path.unrecovered.sum())
        elif r.kind == "update":
            idx = gen.sample_indices(g.b, r.n_update, r.seed)
            d, _, c = oracle.update(g, d, idx, seeded_bytes(r.seed, r.n_update, t), t)
            state[r.target] = [g, t, d, c]
        else:  # a repair puts back exactly the stored bytes of the lost rows
            lost = gen.sample_indices(g.n, r.n_lost, r.seed)
            assert np.array_equal(oracle.repair(g, d, lost, t), c[lost])
    assert all(v > 0 for v in checked.values()), checked
    for sid, st in srv.stripes.items():
        g, t, d, c = state[sid]
        assert np.array_equal(st.data.cpu().numpy(), d)
        assert np.array_equal(st.coded.cpu().numpy(), c)
    srv.close()
