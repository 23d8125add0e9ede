"""Serving loop: encode / decode / update / repair requests on device-resident
stripes, admitted under an HBM budget and run in continuously formed batches.

Requests arrive over time (the caller supplies arrival times). The scheduler
keeps a FIFO of arrived requests and, whenever it runs, admits every request
that (a) fits the memory budget after its resident stripes and in-flight
requests, evicting idle least-recently-used stripes when needed, and (b)
does not target a stripe that already has a request in flight (so every
stripe sees its requests in arrival order). The admitted requests form one
wave: all encodes as one batch (fs_batch, Section 2.2 encoding of each new
stripe), all decodes as one batch (Algorithm 5 + payload per stripe), updates
and repairs as single calls; the wave is enqueued on the next of a few
streams and a CUDA event marks its end. Requests that arrive while waves run
join later waves as memory and stripes free up, so work of different waves
overlaps on the device. A request's latency is its wave's end event minus its
arrival, both on the device timeline.

Every request's result is independent of how requests were grouped: the
batch kernels compute each stripe exactly as the single calls do, and the
per-stripe ordering rule keeps the order of operations of each stripe.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import founsure as fs
from . import gen


@dataclass
class Request:
    """One request. kind: 'encode' (a new stripe of k blocks of t bytes whose
    data is drawn from seed), 'decode' (the target stripe with a fraction of
    its coded blocks erased), 'update' (n_update data blocks of the target
    rewritten with bytes drawn from seed), 'repair' (n_lost coded blocks of
    the target recomputed)."""
    rid: int
    kind: str
    arrival: float  # seconds from the start of the run
    k: int = 0
    t: int = 0
    target: int = -1  # stripe id (decode / update / repair); encode: the new stripe's id
    seed: int = 0
    erase_frac: float = 0.0
    n_update: int = 0
    n_lost: int = 0
    done: Optional[float] = None  # seconds from the start (device timeline)
    out: dict = field(default_factory=dict)


class _Stripe:
    def __init__(self, sid, code, k, n, t, data, coded):
        self.sid, self.code, self.k, self.n, self.t = sid, code, k, n, t
        self.data, self.coded = data, coded
        self.busy = False
        self.last = 0.0

    @property
    def nbytes(self):
        return (self.k + self.n) * self.t


class Server:
    """budget: device bytes the resident stripes and in-flight requests may
    hold. rate: code rate (n = round(k / rate)). streams: waves in flight."""

    def __init__(self, budget: int, device=None, streams: int = 2, rate: float = 1 / 1.3,
                 max_wave: int = 64, batching: bool = True):
        import torch
        self.torch = torch
        self.budget = int(budget)
        self.device = device or torch.device("cuda")
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max(1, streams))]
        self.rate = rate
        self.max_wave = max_wave if batching else 1
        self.codes = {}
        self.stripes = collections.OrderedDict()  # LRU order
        self.resident = 0  # bytes of resident stripes
        self.transient = 0  # bytes held by in-flight requests
        self.peak = 0
        self.waiting = collections.deque()
        self.waves = []  # (event, requests, transient bytes, batches)
        self.retired = []  # batches of finished waves (freed at close)
        self.next_stream = 0
        self.t0_event = None
        self.evictions = 0
        self.encoding = set()  # stripes whose encode is in flight
        self.n_waves = 0
        self.wave_log = []
        self.t_host0 = time.perf_counter()
        self._pinned = []

    # -- codes and memory --------------------------------------------------
    def code_for(self, k: int, t: int):
        key = (k, t)
        if key not in self.codes:
            n = int(round(k / self.rate))
            g = gen.make_graph(k, 0, n, gen.DIST_RSD, 0.05, 0.01, stripe=(k * 131 + t) & 0xFFF)
            self.codes[key] = (fs.Code(g, t), n)
        return self.codes[key]

    def _need(self, r: Request) -> int:
        """Device bytes request r adds while in flight (encode: the new
        stripe itself, which then stays resident)."""
        if r.kind == "encode":
            _, n = self.code_for(r.k, r.t)
            return (r.k + n) * r.t
        s = self.stripes[r.target]
        if r.kind == "decode":
            return s.k * s.t + s.code.workspace_bytes(fs.OP_DECODE) + s.n + s.k
        if r.kind == "update":
            return r.n_update * s.t + s.code.workspace_bytes(fs.OP_UPDATE, r.n_update)
        return s.code.workspace_bytes(fs.OP_REPAIR) + 4 * r.n_lost

    def _evict_for(self, need: int) -> bool:
        """Frees idle LRU stripes until need fits; False if it cannot."""
        while self.resident + self.transient + need > self.budget:
            victim = next((s for s in self.stripes.values() if not s.busy), None)
            if victim is None:
                return False
            del self.stripes[victim.sid]
            self.resident -= victim.nbytes
            self.evictions += 1
        return True

    # -- scheduling ----------------------------------------------------------
    def add_resident(self, sid: int, k: int, t: int, seed: int):
        """Pre-populates the pool with an encoded stripe (blocking)."""
        r = Request(-1, "encode", 0.0, k=k, t=t, target=sid, seed=seed)
        self.waiting.append(r)
        self.pump(0.0)
        self.drain()

    def warm_up(self, shapes=((64, 16384),)) -> None:
        """Runs one request of each kind on a scratch stripe of each (k, t) in
        shapes, then removes the stripes. A kernel's
        module is loaded on its first launch, and a load that meets a busy
        device holds the host until that work ends (seconds, behind a full
        wave), so every kernel a wave can launch, the library's and torch's,
        is launched once here before serving starts."""
        for j, (k, t) in enumerate(shapes):
            sid = -(1 << 30) - j
            for r in (Request(-1, "encode", 0.0, k=k, t=t, target=sid, seed=1 + j),
                      Request(-2, "decode", 0.0, target=sid, seed=2 + j, erase_frac=0.1),
                      Request(-3, "update", 0.0, target=sid, seed=3 + j, n_update=1),
                      Request(-4, "repair", 0.0, target=sid, seed=4 + j, n_lost=1)):
                self.waiting.append(r)
                self.pump(0.0)
                self.drain()
            st = self.stripes.pop(sid, None)
            if st is not None:
                self.resident -= st.nbytes
        self.peak = self.resident + self.transient

    def submit(self, r: Request):
        self.waiting.append(r)

    def cancel(self, rid: int) -> bool:
        """Withdraws a request that has not been admitted yet (an admitted
        one runs to its end). Returns whether it was withdrawn."""
        for r in self.waiting:
            if r.rid == rid:
                self.waiting.remove(r)
                r.out["cancelled"] = True
                return True
        return False

    def pump(self, now: float) -> None:
        """Retires finished waves, then admits arrived requests (FIFO) into
        one wave and enqueues it."""
        self._retire()
        wave, busy, skipped = [], set(), collections.deque()
        while self.waiting and len(wave) < self.max_wave:
            r = self.waiting.popleft()
            if r.kind == "encode":
                pass
            elif r.target in self.encoding or r.target in busy or (
                    r.target in self.stripes and self.stripes[r.target].busy):
                skipped.append(r)  # its stripe has a request in flight: keep the order
                continue
            elif r.target not in self.stripes:
                r.done = now  # the stripe was evicted (or never existed): nothing to do
                r.out["dropped"] = True
                continue
            need = self._need(r)
            if need > self.budget:  # can never fit: reject it without evicting anything
                r.done = now
                r.out["rejected"] = True
                continue
            target = self.stripes.get(r.target) if r.kind != "encode" else None
            if target is not None:
                target.busy = True  # never evict the stripe this request works on
            if not self._evict_for(need):
                if target is not None:
                    target.busy = False
                skipped.append(r)
                break  # memory is short: later requests wait behind this one
            self.transient += need
            r.out["need"] = need
            busy.add(r.target)
            if r.kind == "encode":
                self.encoding.add(r.target)
            wave.append(r)
        while skipped:
            self.waiting.appendleft(skipped.pop())
        self.peak = max(self.peak, self.resident + self.transient)
        if wave:
            self._launch(wave)

    def _upload(self, a: np.ndarray):
        """Host array to the device without blocking the host: through pinned
        memory, so the copy is queued on the current stream (a copy from
        pageable memory would first wait for that stream's earlier work). The
        pinned buffer is kept until the wave ends."""
        torch = self.torch
        h = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        d = h.to(self.device, non_blocking=True)
        self._pinned.append(h)
        return d

    def _launch(self, wave):
        torch = self.torch
        h0 = time.perf_counter()
        self._pinned = []
        s = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        batches = []
        with torch.cuda.stream(s):
            encs = [r for r in wave if r.kind == "encode"]
            decs = [r for r in wave if r.kind == "decode"]
            tp = {}
            t_a = time.perf_counter()
            if encs:
                items = []
                for r in encs:
                    code, n = self.code_for(r.k, r.t)
                    g = torch.Generator(device=self.device)
                    g.manual_seed(r.seed)
                    data = torch.randint(0, 256, (r.k, r.t), dtype=torch.uint8, device=self.device,
                                         generator=g)
                    coded = torch.empty((n, r.t), dtype=torch.uint8, device=self.device)
                    r.out["stripe"] = _Stripe(r.target, code, r.k, n, r.t, data, coded)
                    items.append({"code": code, "data": data, "coded": coded})
                t_b = time.perf_counter()
                b = fs.Batch(items, fs.OP_ENCODE)
                t_c = time.perf_counter()
                b.run(s)
                batches.append(b)
                tp.update(enc_inputs=t_b - t_a, enc_plan=t_c - t_b, enc_run=time.perf_counter() - t_c)
            t_a = time.perf_counter()
            if decs:
                items = []
                for r in decs:
                    st = self.stripes[r.target]
                    er = np.zeros(st.n, np.uint8)
                    er[gen.sample_indices(st.n, gen.round_count(r.erase_frac, st.n), r.seed)] = 1
                    r.out.update(erased=self._upload(er),
                                 data_out=torch.empty((st.k, st.t), dtype=torch.uint8, device=self.device),
                                 unrecovered=torch.empty(st.k, dtype=torch.uint8, device=self.device),
                                 n_unrecovered=torch.empty(1, dtype=torch.int32, device=self.device),
                                 ws=st.code.workspace(fs.OP_DECODE, device=self.device))
                    items.append({"code": st.code, "coded": st.coded, "erased": r.out["erased"],
                                  "data_out": r.out["data_out"], "unrecovered": r.out["unrecovered"],
                                  "n_unrecovered": r.out["n_unrecovered"], "ws": r.out["ws"]})
                t_b = time.perf_counter()
                b = fs.Batch(items, fs.OP_DECODE)
                t_c = time.perf_counter()
                b.run(s)
                batches.append(b)
                tp.update(dec_inputs=t_b - t_a, dec_plan=t_c - t_b, dec_run=time.perf_counter() - t_c)
            t_a = time.perf_counter()
            for r in wave:
                if r.kind == "update":
                    st = self.stripes[r.target]
                    idx = gen.sample_indices(st.k, r.n_update, r.seed)
                    g = torch.Generator(device=self.device)
                    g.manual_seed(r.seed)
                    new = torch.randint(0, 256, (r.n_update, st.t), dtype=torch.uint8,
                                        device=self.device, generator=g)
                    d_idx = self._upload(idx)
                    ws = st.code.workspace(fs.OP_UPDATE, r.n_update, device=self.device)
                    st.code.update(d_idx, r.n_update, new, st.data, None, st.coded, ws, stream=s)
                    r.out.update(idx=d_idx, new=new, ws=ws)
                elif r.kind == "repair":
                    st = self.stripes[r.target]
                    lost = gen.sample_indices(st.n, r.n_lost, r.seed)
                    d_lost = self._upload(lost)
                    ws = st.code.workspace(fs.OP_REPAIR, device=self.device)
                    # the lost blocks are gone; index_fill_ takes the value as a kernel
                    # argument (an indexed assignment of a Python scalar copies it from
                    # pageable memory, which waits for the stream's queued work)
                    st.coded.index_fill_(0, d_lost.long(), 0)
                    st.code.repair(d_lost, r.n_lost, st.data, None, st.coded, ws, stream=s)
                    r.out.update(lost=d_lost, ws=ws)
            tp["upd_rep"] = time.perf_counter() - t_a
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        self.waves.append((ev, wave, sum(r.out["need"] for r in wave), batches + self._pinned))
        self.n_waves += 1
        # server counters: what the wave held and how long the host took to launch it
        kinds = collections.Counter(r.kind for r in wave)
        self.wave_log.append({"n": len(wave), "kinds": dict(kinds), "host_ms": (time.perf_counter() - h0) * 1e3,
                              "phases_ms": {k: v * 1e3 for k, v in tp.items()},
                              "event": ev, "launched": time.perf_counter() - self.t_host0})

    def _retire(self, block: bool = False):
        keep = []
        for ev, wave, need, batches in self.waves:
            if block:
                ev.synchronize()
            if not ev.query():
                keep.append((ev, wave, need, batches))
                continue
            done = self.t0_event.elapsed_time(ev) * 1e-3 if self.t0_event is not None else 0.0
            self.transient -= need
            for r in wave:
                r.done = done
                if r.kind == "encode":
                    st = r.out.pop("stripe")
                    self.stripes[st.sid] = st
                    self.resident += st.nbytes  # its bytes left the wave's transient share above
                    self.encoding.discard(st.sid)
                    r.out["coded"] = st.coded
                else:
                    st = self.stripes.get(r.target)
                    if st is not None:
                        st.busy = False
                        self.stripes.move_to_end(r.target)
            self.retired.extend(b for b in batches if isinstance(b, fs.Batch))
        self.waves = keep

    def drain(self):
        while self.waves:
            self._retire(block=True)

    def run(self, requests, realtime: bool = True):
        """Serves requests (sorted by arrival). realtime: admit each request no
        earlier than its arrival on the wall clock; otherwise admit in order
        as fast as possible. Returns the requests with done times."""
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        torch.cuda.synchronize()
        self.wave_log = []
        self.n_waves = 0
        self.t0_event = torch.cuda.Event(enable_timing=True)
        self.t0_event.record()
        t0 = time.perf_counter()
        self.t_host0 = t0
        i = 0
        while i < len(reqs) or self.waiting or self.waves:
            now = time.perf_counter() - t0 if realtime else float("inf")
            while i < len(reqs) and (reqs[i].arrival <= now):
                self.waiting.append(reqs[i])
                i += 1
            before = len(self.waves)
            self.pump(now)
            if len(self.waves) == before and self.waves:
                self._retire()
                time.sleep(20e-6)
            elif not self.waves and not self.waiting and i < len(reqs):
                time.sleep(min(1e-3, max(0.0, reqs[i].arrival - now)))
            elif not self.waves and self.waiting:
                # nothing in flight and nothing admissible: the head cannot fit
                r = self.waiting.popleft()
                r.done = now
                r.out["rejected"] = True
        self.drain()
        return reqs

    def wave_stats(self) -> dict:
        """Summary of the waves of the last run: sizes, host launch time, and
        the device time from one wave's end to the next's (work per wave)."""
        if not self.wave_log:
            return {}
        ends = sorted(self.t0_event.elapsed_time(w["event"]) for w in self.wave_log if w["event"].query())
        gaps = np.diff([0.0] + ends)
        n = np.array([w["n"] for w in self.wave_log])
        host = np.array([w["host_ms"] for w in self.wave_log])
        phases = collections.Counter()
        for w in self.wave_log:
            phases.update(w.get("phases_ms", {}))
        return {"waves": len(self.wave_log), "mean_requests": round(float(n.mean()), 2),
                "host_ms_by_phase": {k: round(v, 1) for k, v in phases.items()},
                "max_requests": int(n.max()), "host_ms_per_wave": round(float(host.mean()), 3),
                "host_ms_total": round(float(host.sum()), 1),
                "device_ms_between_wave_ends": round(float(np.median(gaps)), 3)}

    def close(self):
        self.drain()
        for b in self.retired:
            b.close()
        self.retired = []


def latency_stats(reqs):
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs
                    if r.done is not None and not r.out.get("dropped") and not r.out.get("rejected")])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "served": 0}
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "served": int(lat.size)}
