"""The bench's N>1 path on CPU: two gloo ranks, each running its own stripe.

Under torchrun every rank encodes and decodes an independent stripe (stripes
partition the data, Section 2.2), so the only cross-rank traffic is a barrier
and the max-reduction of the timed duration; the reference arm runs on rank 0
alone. These tests drive those pieces with world_size 2 on the gloo backend
and check each rank's stripe against the oracle.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_1702_07409_gb300 import gen
        res = {}
        assert bench.dist_env() == (rank, world, rank)
        # max over ranks of each rank's timed duration
        res["max"] = bench.reduce_max(10.0 + 5.0 * rank, "cpu")
        bench.barrier()
        # this rank's own stripe: a small precoded graph, encoded and decoded
        # by the oracle with 20% of the coded blocks erased
        b, m, n, t = 60, 6, 90, 32
        g = gen.make_graph(b, m, n, gen.DIST_FINITE40, stripe=rank)
        data = gen.fill_bytes(gen.SEED_DATA + (rank << gen.STRIPE_SHIFT), b * t).reshape(b, t)
        parity, coded = oracle.encode(g, data, t)
        er = np.zeros(n, np.uint8)
        er[gen.sample_indices(n, gen.round_count(0.2, n), gen.SEED_ERASE + (rank << gen.STRIPE_SHIFT))] = 1
        path = oracle.dpg(g, er)
        dec = oracle.peel(g, coded, path, t)
        ok = path.unrecovered[:b] == 0
        res["decoded"] = bool(np.array_equal(dec[ok], data[ok]))
        res["graph"] = (np.asarray(g.lt_idx).tobytes(), np.asarray(g.pre_idx).tobytes())
        # the reference arm prints on rank 0 only; other ranks return at once
        if rank != 0:
            class A:
                pass
            res["ref_returned"] = bench.run_reference(A()) is None
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_stripes():
    import oracle
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(out.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0]["max"] == results[1]["max"] == 15.0
    assert results[0]["decoded"] and results[1]["decoded"]
    assert results[0]["graph"] != results[1]["graph"]  # each rank has its own stripe
    assert results[1]["ref_returned"]
