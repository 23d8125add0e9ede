"""Batches of stripes (fs_batch): every stripe of a batch of uneven stripes
(codes, sizes and block lengths all differ) is encoded and decoded exactly as
the oracle does it (Section 2.2 encoding, Algorithm 5 decoding), also when
the batch runs from a captured CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1702_07409_gb300 import gen

pytestmark = pytest.mark.gpu

# (b, m, n, t, dist, c, delta): plain LT with RSD degrees (the batched
# workload's distribution), precoded FiniteDist stripes, ragged block sizes
SHAPES = [
    (64, 0, 84, 4096, gen.DIST_RSD, 0.05, 0.01),
    (300, 12, 400, 48, gen.DIST_FINITE40, 0.0, 0.0),
    (1000, 0, 1300, 1024, gen.DIST_RSD, 0.05, 0.01),
    (150, 8, 200, 16, gen.DIST_FINITE40, 0.0, 0.0),
    (700, 0, 910, 4096 + 16, gen.DIST_RSD, 0.05, 0.01),
    (2000, 64, 2600, 1024, gen.DIST_FINITE40, 0.0, 0.0),
    (90, 0, 117, 16384, gen.DIST_RSD, 0.05, 0.01),
    (512, 16, 700, 256, gen.DIST_FINITE40, 0.0, 0.0),
    (4096, 0, 5325, 1024, gen.DIST_RSD, 0.05, 0.01),  # slice tables in several parts
    (512, 0, 666, 65536, gen.DIST_RSD, 0.05, 0.01),    # a 64 KiB stripe (config 3 draws t up to it)
    (300, 12, 400, 65536, gen.DIST_FINITE40, 0.0, 0.0),
]


def _fs():
    from paper_1702_07409_gb300 import founsure
    return founsure


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(x):
    return x.cpu().numpy()


class Stripe:
    def __init__(self, i, b, m, n, t, dist, c, delta):
        import torch
        fs = _fs()
        self.b, self.m, self.n, self.t = b, m, n, t
        self.g = gen.make_graph(b, m, n, dist, c, delta, stripe=i)
        self.code = fs.Code(self.g, t)
        self.data = gen.fill_bytes(gen.SEED_DATA + (i << gen.STRIPE_SHIFT), b * t).reshape(b, t)
        self.d = _dev(self.data)
        self.p = torch.empty((m, t), dtype=torch.uint8, device="cuda") if m else None
        self.cd = torch.empty((n, t), dtype=torch.uint8, device="cuda")
        frac = 0.10 + 0.15 * ((i * 37) % 16) / 15.0  # 10% .. 25% erased
        er = np.zeros(n, np.uint8)
        er[gen.sample_indices(n, gen.round_count(frac, n), gen.SEED_ERASE + (i << gen.STRIPE_SHIFT))] = 1
        self.erased = er
        self.d_er = _dev(er)
        self.out = torch.full((b, t), 0xA5, dtype=torch.uint8, device="cuda")
        self.unrec = torch.empty(b + m, dtype=torch.uint8, device="cuda")
        self.nun = torch.empty(1, dtype=torch.int32, device="cuda")
        self.ws = self.code.workspace(fs.OP_DECODE)

    def enc(self):
        return {"code": self.code, "data": self.d, "parity": self.p, "coded": self.cd}

    def dec(self):
        return {"code": self.code, "coded": self.cd, "erased": self.d_er, "data_out": self.out,
                "unrecovered": self.unrec, "n_unrecovered": self.nun, "ws": self.ws}

    def check_encode(self):
        par, cod = oracle.encode(self.g, self.data, self.t)
        assert np.array_equal(_host(self.cd), cod)
        if self.m:
            assert np.array_equal(_host(self.p), par)
        return cod

    def check_decode(self, cod):
        want, path = oracle.decode(self.g, cod, self.erased, self.t)
        assert np.array_equal(_host(self.unrec), path.unrecovered)
        assert int(_host(self.nun)[0]) == int(path.unrecovered.sum())
        assert np.array_equal(_host(self.out), want)
        return path


def _stripes():
    return [Stripe(i, *s) for i, s in enumerate(SHAPES)]


def test_batch_encode_decode_match_the_oracle():
    import torch
    fs = _fs()
    st = _stripes()
    enc = fs.Batch([s.enc() for s in st], fs.OP_ENCODE)
    dec = fs.Batch([s.dec() for s in st], fs.OP_DECODE)
    enc.run()
    dec.run()
    torch.cuda.synchronize()
    assert enc.status() == fs.FS_OK and dec.status() == fs.FS_OK
    stalls = 0
    for s in st:
        path = s.check_decode(s.check_encode())
        stalls += int(path.unrecovered[:s.b].any())
        assert fs.Code.ws_status(s.ws) == fs.FS_OK
    enc.close()
    dec.close()
    assert stalls < len(st)  # most stripes decode completely


def test_batch_replays_from_a_cuda_graph():
    import torch
    fs = _fs()
    st = _stripes()
    enc = fs.Batch([s.enc() for s in st], fs.OP_ENCODE)
    dec = fs.Batch([s.dec() for s in st], fs.OP_DECODE)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # a first run outside the capture
        enc.run(side)
        dec.run(side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for s in st:  # poison the outputs, then replay the captured batch twice
        s.cd.fill_(0)
        s.out.fill_(0x5A)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        enc.run(torch.cuda.current_stream())
        dec.run(torch.cuda.current_stream())
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for s in st:
        s.check_decode(s.check_encode())


def test_batch_equals_single_calls_and_rejects_bad_stripes():
    import torch
    fs = _fs()
    st = _stripes()[:4]
    enc = fs.Batch([s.enc() for s in st], fs.OP_ENCODE)
    enc.run()
    torch.cuda.synchronize()
    got = [_host(s.cd).copy() for s in st]
    for s, g in zip(st, got):
        s.cd.fill_(0)
        s.code.encode(s.d, s.p, s.cd, s.code.workspace(fs.OP_ENCODE))
    torch.cuda.synchronize()
    for s, g in zip(st, got):
        assert np.array_equal(_host(s.cd), g)
    bad = st[1].enc()
    bad["parity"] = None  # m > 0 needs parities
    with pytest.raises(fs.FounsureError):
        fs.Batch([st[0].enc(), bad], fs.OP_ENCODE)
    with pytest.raises(fs.FounsureError):
        fs.Batch([st[0].enc()], 7)
    empty = fs.Batch([], fs.OP_DECODE)
    empty.run()
