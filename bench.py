"""Throughput of the Founsure GF(2) gather-XOR path on one GB300 (or N replicas).

One step is one pass of the whole hot path over one precoded stripe:
  encode   - precode parities + LT/LDGM coded blocks (fs_encode)
  decode   - Algorithm 5 schedule + its payload (fs_decode_schedule,
             fs_decode_payload) of the coded blocks with 20% erased
  update   - 1% of data blocks rewritten, deltas pushed into parities and
             coded blocks (fs_update)
  repair   - 5% of coded blocks recomputed from the intermediates (fs_repair)
Workload: b=4096 data blocks x 64 KiB (256 MiB), 128 precode checks (each data
block in 3), n=5400 coded blocks, max-degree-40 FiniteDist degrees, seeded
synthetic bytes. Every input is larger than the 129 MB L2, so no flush is
needed between steps.

value = (data bytes encoded + data bytes recovered by decode) / step time,
steps timed with CUDA events on the launching stream. Per-op times come from
events around each call on the same stream.

--impl reference times the CPU oracle (plain C loops, one core) on a byte
slice of every block of the same stripe and prints the same JSON line.
Under torchrun each rank runs its own stripe (replicas; no data exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1702_07409_gb300 import gen  # noqa: E402

B, M, N_CODED, T = 4096, 128, 5400, 65536
ERASE_FRAC, UPDATE_FRAC, REPAIR_FRAC = 0.20, 0.01, 0.05
METRIC = "encode & BP-decode source GB/s"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the payload (k_peel_keys, the default key walk) and of the slice encode
# (k_slices) at this workload, taken with
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none -k regex:"k_peel|k_slices|k_key_plan" -s 12 -c 4
#       python bench.py --steps 2 --warmup 3 --no-cpu-baseline --no-extras
# on one GB300. Valid only while those two kernels are unchanged.
PEEL_TRAFFIC_BYTES = 649121024 + 310724096
SLICES_TRAFFIC_BYTES = 268601600 + 313820160
# the payload's walk (FS_TUNE_PEEL_FLOW; the library's default is 2): its
# kernel, and the plan kernels the decoding schedule adds for it
PEEL_KERNEL = {0: "k_peel", 1: "k_peel_flow", 2: "k_peel_keys", 3: "k_peel_keys"}
PLAN_KERNELS = {0: [], 1: ["k_flow_units", "k_flow_place"], 2: ["k_key_plan"], 3: ["k_key_plan"]}
# the key walk's payload is followed by a level-walk launch that returns at
# once where the key walk had its plan
FALLBACK_KERNELS = {0: [], 1: [], 2: ["k_peel"], 3: ["k_peel"]}
DEFAULT_WALK = 2


def walk_of(args):
    return DEFAULT_WALK if getattr(args, "peel_flow", None) is None else args.peel_flow


WORKLOAD = ("precoded LDGM stripe: b=4096 x 64 KiB data, m=128 checks (3 per data block), "
            "n=5400, FiniteDist max-degree-40, 20% erasures; step = encode + decode + "
            "1% update + 5% repair")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(x: float, device) -> float:
    """Max of x over ranks (x itself on a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


class NoGC:
    """Python's garbage collector off inside a timed region (as timeit does):
    a collection pause between two launches would leave the GPU idle and
    count as step time. Collects once on entry, outside the timed work."""

    def __enter__(self):
        import gc
        gc.collect()
        self.was = gc.isenabled()
        gc.disable()
        return self

    def __exit__(self, *exc):
        import gc
        if self.was:
            gc.enable()
        return False


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))
        return out


class Stripe:
    """Device-resident state of one stripe and the seeded inputs of its steps."""

    def __init__(self, stripe: int, n_rounds: int, device, tuning=None, overlap=True,
                 two_pass=False):
        import torch
        self.overlap = overlap
        self.side = torch.cuda.Stream(device=device)
        from paper_1702_07409_gb300 import founsure as fs
        self.fs = fs
        off = stripe << gen.STRIPE_SHIFT
        self.g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40, stripe=stripe)
        self.code = fs.Code(self.g, T, fs.DECODE_TWO_PASS if two_pass else fs.DECODE_JOINT)
        if tuning:
            for knob, value in tuning.items():
                self.code.set_tuning(knob, value)
        host = gen.fill_bytes(gen.SEED_DATA + off, B * T).reshape(B, T)
        self.host_data = torch.from_numpy(host).pin_memory()
        self.p = torch.empty((M, T), dtype=torch.uint8, device=device)
        self.cd = torch.empty((N_CODED, T), dtype=torch.uint8, device=device)
        er = np.zeros(N_CODED, np.uint8)
        er[gen.sample_indices(N_CODED, gen.round_count(ERASE_FRAC, N_CODED),
                              gen.SEED_ERASE + off)] = 1
        self.host_erased = torch.from_numpy(er).pin_memory()
        # two sets of per-step inputs and outputs: the end-to-end loop uploads
        # step i+1 and reads back step i-1 while step i computes
        self.bufs = []
        for _ in range(2):
            self.bufs.append({
                "d": self.host_data.to(device),
                "erased": self.host_erased.to(device),
                "out": torch.empty((B, T), dtype=torch.uint8, device=device),
                "unrec": torch.empty(B + M, dtype=torch.uint8, device=device),
                "nun": torch.empty(1, dtype=torch.int32, device=device),
            })
        self.s_in = torch.cuda.Stream(device=device)
        self.s_out = torch.cuda.Stream(device=device)
        self.u = gen.round_count(UPDATE_FRAC, B)
        self.nl = gen.round_count(REPAIR_FRAC, N_CODED)
        self.n_rounds = n_rounds
        idx, new, lost = [], [], []
        for r in range(n_rounds):
            idx.append(gen.sample_indices(B, self.u, gen.SEED_UPDATE + off + (r << gen.ROUND_SHIFT)))
            new.append(gen.fill_bytes(gen.SEED_NEWDATA + off + (r << gen.ROUND_SHIFT),
                                      self.u * T).reshape(self.u, T))
            lost.append(gen.sample_indices(N_CODED, self.nl,
                                           gen.SEED_REPAIR + off + (r << gen.ROUND_SHIFT)))
        self.host_idx = torch.from_numpy(np.stack(idx)).pin_memory()
        self.host_new = torch.from_numpy(np.stack(new)).pin_memory()
        self.host_lost = torch.from_numpy(np.stack(lost)).pin_memory()
        self.idx = self.host_idx.to(device)
        self.new = self.host_new.to(device)
        self.lost = self.host_lost.to(device)
        self.ws_e = self.code.workspace(fs.OP_ENCODE, device=device)
        self.ws_d = self.code.workspace(fs.OP_DECODE, device=device)
        self.ws_u = self.code.workspace(fs.OP_UPDATE, self.u, device=device)
        self.ws_r = self.code.workspace(fs.OP_REPAIR, device=device)
        self.host_out = torch.empty((B, T), dtype=torch.uint8).pin_memory()
        self.host_nun = torch.empty(1, dtype=torch.int32).pin_memory()
        self.nun_reads = []

    # launches of this library's kernels per step, besides the decoding
    # plan's (encode 1: the slice kernel; decode 2: schedule + payload;
    # update 4; repair 1)
    LAUNCHES_PER_STEP = 8

    @property
    def nun(self):
        return self.bufs[0]["nun"]

    @property
    def unrec(self):
        return self.bufs[0]["unrec"]

    def step(self, r: int, ev=None, k: int = 0):
        """encode, decode (schedule + payload), update, repair on input set k.
        The decoding schedule needs only the erasure flags, so with overlap on
        it runs on a side stream beside the encode (the payload waits for
        both)."""
        import torch
        c = self.code
        bk = self.bufs[k]
        r %= self.n_rounds
        main = torch.cuda.current_stream()
        if self.overlap:
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                if ev: ev[6].record()
                c.decode_schedule(bk["erased"], bk["unrec"], bk["nun"], self.ws_d)
                if ev: ev[7].record()
        if ev: ev[0].record()
        c.encode(bk["d"], self.p, self.cd, self.ws_e)
        if ev: ev[1].record()
        if self.overlap:
            main.wait_stream(self.side)
        else:
            if ev: ev[6].record()
            c.decode_schedule(bk["erased"], bk["unrec"], bk["nun"], self.ws_d)
            if ev: ev[7].record()
        if ev: ev[2].record()
        c.decode_payload(self.cd, bk["out"], self.ws_d)
        if ev: ev[3].record()
        c.update(self.idx[r], self.u, self.new[r], bk["d"], self.p, self.cd, self.ws_u)
        if ev: ev[4].record()
        c.repair(self.lost[r], self.nl, bk["d"], self.p, self.cd, self.ws_r)
        if ev: ev[5].record()

    def run_e2e(self, rounds):
        """The steps of `rounds` from pinned host buffers: each step's inputs
        are copied in and its decoded data and unrecovered count copied back.
        Uploads run on one copy stream, read-backs on another, so step i+1's
        upload and step i-1's read-back overlap step i's kernels (input sets
        alternate)."""
        import torch
        main = torch.cuda.current_stream()
        n = len(rounds)
        in_done = [torch.cuda.Event() for _ in range(n)]
        comp_done = [torch.cuda.Event() for _ in range(n)]
        out_done = [torch.cuda.Event() for _ in range(n)]
        for i, r in enumerate(rounds):
            k = i & 1
            bk = self.bufs[k]
            r %= self.n_rounds
            with torch.cuda.stream(self.s_in):
                if i >= 2:  # input set k is free once step i-2's kernels are done
                    self.s_in.wait_event(comp_done[i - 2])
                bk["d"].copy_(self.host_data, non_blocking=True)
                bk["erased"].copy_(self.host_erased, non_blocking=True)
                self.idx[r].copy_(self.host_idx[r], non_blocking=True)
                self.new[r].copy_(self.host_new[r], non_blocking=True)
                self.lost[r].copy_(self.host_lost[r], non_blocking=True)
                in_done[i].record(self.s_in)
            main.wait_event(in_done[i])
            if i >= 2:  # output set k has been read back
                main.wait_event(out_done[i - 2])
            self.step(r, k=k)
            comp_done[i].record(main)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(comp_done[i])
                self.host_out.copy_(bk["out"], non_blocking=True)
                self.host_nun.copy_(bk["nun"], non_blocking=True)
                out_done[i].record(self.s_out)
        main.wait_stream(self.s_out)

    def h2d_bytes(self):
        return B * T + N_CODED + self.u * 4 + self.u * T + self.nl * 4

    def d2h_bytes(self):
        return B * T + 4


def run_gpu(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    peak, peak_kind = peaks()
    from paper_1702_07409_gb300 import founsure as fs
    tuning = {}
    if args.peel_ctas:
        tuning[fs.TUNE_PEEL_CTAS] = args.peel_ctas
    if args.gather_ctas:
        tuning[fs.TUNE_GATHER_CTAS] = args.gather_ctas
    if args.l2_hints:
        tuning[fs.TUNE_L2_HINTS] = 1
    if args.peel_flow is not None:
        tuning[fs.TUNE_PEEL_FLOW] = args.peel_flow

    st = Stripe(rank, max(args.steps, 1) + args.warmup, device, tuning,
                overlap=not args.serial_schedule, two_pass=args.two_pass)
    torch.cuda.synchronize()

    # warm-up; also checks the decode outcome of this erasure draw
    for r in range(args.warmup):
        st.step(r)
    torch.cuda.synchronize()
    n_unrec = int(st.nun.item())
    unrec_data = int(st.unrec[:B].sum().item())
    recovered = (B - unrec_data) * T

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with NoGC(), ClockSampler(local) as clk:
        t0.record()
        for i in range(K):
            st.step(args.warmup + i, evs[i])
        t1.record()
        torch.cuda.synchronize()
    barrier()
    ms_total = reduce_max(t0.elapsed_time(t1), device)
    ms_step = ms_total / K
    spans = {"encode": (0, 1), "decode_schedule": (6, 7), "decode_payload": (2, 3),
             "update": (3, 4), "repair": (4, 5)}
    op_ms = {o: statistics.mean(evs[i][a].elapsed_time(evs[i][b]) for i in range(K))
             for o, (a, b) in spans.items()}

    # e2e: the same steps from pinned host memory, copies inside the timed region
    st.run_e2e(list(range(min(args.warmup, 3))))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with NoGC():
        e0.record()
        st.run_e2e([args.warmup + i for i in range(K)])
        e1.record()
        torch.cuda.synchronize()
    barrier()
    ms_e2e = reduce_max(e0.elapsed_time(e1), device) / K
    # the last step's read-back: the decoded data equal the uploaded data
    e2e_ok = bool(torch.equal(st.host_out, st.host_data)) if n_unrec == 0 else None
    if e2e_ok is False:
        raise RuntimeError("end-to-end read-back differs from the uploaded data")

    src_bytes = B * T + recovered
    gbs = world * src_bytes / (ms_step * 1e-3) / 1e9
    gbs_e2e = world * src_bytes / (ms_e2e * 1e-3) / 1e9

    # roofline of the kernel with the largest share of the step: the payload
    # (k_peel_keys by default). Algorithmic bytes = the coded payloads of the pairs whose
    # constraint is a coded row (read) + the recovered data blocks (written).
    g = st.g
    dec_pairs_lt = None
    try:
        view = st.code.decode_path(st.ws_d)
        pg = view["pair_g"].cpu().numpy()
        dec_pairs_lt = int((pg < N_CODED).sum())
    except Exception:
        pass
    dec_bytes = ((dec_pairs_lt or 0) + (B - unrec_data)) * T
    dec_gbs = dec_bytes / (op_ms["decode_payload"] * 1e-3) / 1e9
    # encode (k_slices): data read once, parities and coded blocks written once
    enc_bytes = (B + M + N_CODED) * T
    enc_gbs = enc_bytes / (op_ms["encode"] * 1e-3) / 1e9
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": round(gbs, 2), "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded splitmix64 bytes and graphs)",
        "config": {"workload": WORKLOAD, "b": B, "m": M, "n": N_CODED, "block_bytes": T,
                   "e_lt": g.e_lt, "e_pre": g.e_pre, "erased": int(st.host_erased.sum().item()),
                   "unrecovered": n_unrec, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "schedule_beside_encode": not args.serial_schedule,
                   "decoding": "two-pass (LT, then precode)" if args.two_pass else "joint",
                   "tuning": {"peel_ctas": args.peel_ctas or 1,
                              "gather_ctas": args.gather_ctas or 8,
                              "peel_flow": walk_of(args)}},
        "ops_ms": {k: round(v, 4) for k, v in op_ms.items()},
        "encode_source_gbs": round(B * T / (op_ms["encode"] * 1e-3) / 1e9, 1),
        "decode_source_gbs": round(recovered / ((op_ms["decode_schedule"] +
                                                  op_ms["decode_payload"]) * 1e-3) / 1e9, 1),
        "roofline": {"bound": "hbm", "kernel": f"{PEEL_KERNEL[walk_of(args)]} (fs_decode_payload)",
                     "achieved": round(dec_gbs, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(dec_gbs / peak, 4),
                     "traffic": PEEL_TRAFFIC_BYTES if T == 65536 and walk_of(args) == DEFAULT_WALK else None,
                     "algorithmic_bytes": dec_bytes},
        "encode_roofline": {"bound": "hbm", "kernel": "k_slices<2> (fs_encode)",
                            "achieved": round(enc_gbs, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(enc_gbs / peak, 4),
                            "traffic": SLICES_TRAFFIC_BYTES if T == 65536 else None,
                            "algorithmic_bytes": enc_bytes},
        "e2e": {"value": round(gbs_e2e, 2), "unit": "GB/s", "ms_per_step": round(ms_e2e, 4),
                "h2d_bytes_per_step": st.h2d_bytes(), "d2h_bytes_per_step": st.d2h_bytes(),
                "copies": "uploads and read-backs on two copy streams, overlapping the "
                          "neighbouring steps' kernels (two input sets)",
                "readback_verified": e2e_ok},
        "gpu_launches": (Stripe.LAUNCHES_PER_STEP + len(PLAN_KERNELS[walk_of(args)]) +
                         len(FALLBACK_KERNELS[walk_of(args)])) * K,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(extras(args, st, device, dec_bytes, peak, peak_kind))
        del st
        torch.cuda.empty_cache()
        line["batched"] = compact_batched(batched_measure(args, device, args.extras_stripes, 5))
        torch.cuda.empty_cache()
        line["serving"] = compact_serving(serving_measure(args, device, args.extras_requests))
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_slice, args.cpu_steps)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.cpu_slice, args.cpu_steps)
        line["levels"] = level_counts(line.get("decode_roofline", {}).get("levels_gpu"))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extras(args, st, device, dec_bytes, peak, peak_kind):
    """Numbers beside the step, on one GPU: the decode as a decode-only call
    pays it (schedule, then payload, serially) against its own roofline, and
    the latency of the small plain-LT code (k = 100 x 1 KiB, RSD(0.1, 0.05),
    n = 150, 30 erased), where a launch's latency, not bandwidth, is what a
    caller sees."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    bk = st.bufs[0]
    K = max(args.steps, 10)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for i in range(3):
        st.code.decode_schedule(bk["erased"], bk["unrec"], bk["nun"], st.ws_d)
        st.code.decode_payload(st.cd, bk["out"], st.ws_d)
    torch.cuda.synchronize()
    for i in range(K):
        ev[i][0].record()
        st.code.decode_schedule(bk["erased"], bk["unrec"], bk["nun"], st.ws_d)
        ev[i][1].record()
        st.code.decode_payload(st.cd, bk["out"], st.ws_d)
        ev[i][2].record()
    torch.cuda.synchronize()
    sch = statistics.median(e[0].elapsed_time(e[1]) for e in ev)
    pay = statistics.median(e[1].elapsed_time(e[2]) for e in ev)
    tot = statistics.median(e[0].elapsed_time(e[2]) for e in ev)
    view = st.code.decode_path(st.ws_d)
    ach = dec_bytes / (tot * 1e-3) / 1e9
    out = {"decode_roofline": {
        "bound": "hbm",
        "kernel": " + ".join(["k_dpg_compact"] + PLAN_KERNELS[walk_of(args)] + [PEEL_KERNEL[walk_of(args)]]) +
                  " (fs_decode: schedule, then payload)",
        "ms": round(tot, 4), "schedule_ms": round(sch, 4), "payload_ms": round(pay, 4),
        "achieved": round(ach, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
        "frac": round(ach / peak, 4), "algorithmic_bytes": dec_bytes,
        "levels_gpu": int(view["n_levels"])}}

    # config 1: k = 100 x 1 KiB, plain LT, RSD(0.1, 0.05), n = 150, 30 erased
    b1, n1, t1 = 100, 150, 1024
    g1 = gen.make_graph(b1, 0, n1, gen.DIST_RSD, 0.1, 0.05)
    c1 = fs.Code(g1, t1)
    d1 = torch.from_numpy(gen.fill_bytes(gen.SEED_DATA, b1 * t1).reshape(b1, t1)).to(device)
    cd1 = torch.empty((n1, t1), dtype=torch.uint8, device=device)
    er1 = np.zeros(n1, np.uint8)
    er1[gen.sample_indices(n1, 30, gen.SEED_ERASE)] = 1
    der1 = torch.from_numpy(er1).to(device)
    o1 = torch.empty((b1, t1), dtype=torch.uint8, device=device)
    u1 = torch.empty(b1, dtype=torch.uint8, device=device)
    nu1 = torch.empty(1, dtype=torch.int32, device=device)
    we1, wd1 = c1.workspace(fs.OP_ENCODE, device=device), c1.workspace(fs.OP_DECODE, device=device)
    R = 200
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(R)]
    for i in range(R + 5):
        e = evs[i - 5] if i >= 5 else None
        if e: e[0].record()
        c1.encode(d1, None, cd1, we1)
        if e: e[1].record()
        c1.decode(cd1, der1, o1, u1, nu1, wd1)
        if e: e[2].record()
    torch.cuda.synchronize()
    enc_us = statistics.median(e[0].elapsed_time(e[1]) for e in evs) * 1e3
    dec_us = statistics.median(e[1].elapsed_time(e[2]) for e in evs) * 1e3
    out["config1_latency"] = {
        "workload": "k=100 x 1 KiB, plain LT, RSD(0.1, 0.05), n=150, 30 coded blocks erased",
        "encode_us": round(enc_us, 2), "decode_us": round(dec_us, 2), "unit": "us",
        "unrecovered": int(nu1.item()), "calls": R,
        "note": "one call each, median of %d back-to-back calls on one stream (CUDA events)" % R}
    c1.close()
    return out


def compact_batched(line):
    """The batched-stripes line cut to what the step line carries."""
    return {"stripes": int(line["config"]["workload"].split()[0]),
            "graph_replay_ms": line["ms_per_step"], "per_stripe_ms": line["per_stripe_ms"],
            "eager_ms": line["batched_eager_ms"],
            "speedup_vs_per_stripe": line["speedup_vs_per_stripe"],
            "source_gbs": line["value"], "achieved": line["roofline"]["achieved"],
            "frac": line["roofline"]["frac"], "unit": "GB/s",
            "outputs_equal_per_stripe": line["outputs_equal_per_stripe"],
            "workload": line["config"]["workload"]}


def compact_serving(line):
    """The serving line cut to what the step line carries."""
    b, o = line["batched"], line["one_request_per_launch"]
    keep = ("p50_ms", "p99_ms", "served", "gbs", "waves", "dropped", "rejected")
    return {"requests": line["steps"], "workload": line["config"]["workload"],
            "continuous_batching": {k: b.get(k) for k in keep},
            "one_request_per_launch": {k: o.get(k) for k in keep}}


def _oracle_step(g, data, erased, idx, new, lost, t):
    import oracle
    par, cod = oracle.encode(g, data, t)
    out, path = oracle.decode(g, cod, erased, t)
    data, par, cod = oracle.update(g, data, idx, new, t)
    oracle.repair(g, data, lost, t)
    return out, path, data


def cpu_baseline(slice_bytes: int, steps: int = 2):
    """The oracle timed on a byte slice of every block of the same stripe."""
    import oracle
    oracle.build()
    g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40)
    t = slice_bytes
    data = gen.fill_bytes(gen.SEED_DATA, B * t).reshape(B, t)
    er = np.zeros(N_CODED, np.uint8)
    er[gen.sample_indices(N_CODED, gen.round_count(ERASE_FRAC, N_CODED), gen.SEED_ERASE)] = 1
    u, nl = gen.round_count(UPDATE_FRAC, B), gen.round_count(REPAIR_FRAC, N_CODED)
    src = 0
    t0 = time.perf_counter()
    for r in range(steps):
        idx = gen.sample_indices(B, u, gen.SEED_UPDATE + (r << gen.ROUND_SHIFT))
        new = gen.fill_bytes(gen.SEED_NEWDATA + (r << gen.ROUND_SHIFT), u * t).reshape(u, t)
        lost = gen.sample_indices(N_CODED, nl, gen.SEED_REPAIR + (r << gen.ROUND_SHIFT))
        out, path, data = _oracle_step(g, data, er, idx, new, lost, t)
        src += B * t + int((path.unrecovered[:B] == 0).sum()) * t
    dt = time.perf_counter() - t0
    return {"value": round(src / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d steps of the same stripe, graph and erasures on a %d-byte slice of "
                      "every block (full block 65536 B)" % (steps, t),
            "seconds": round(dt, 2)}


def _oracle_proc(slice_bytes, steps, seed_off, q, go, warmup=0):
    """One process of the all-cores baseline: the unchanged oracle on its own
    byte slice of every block (its data drawn from seed + seed_off); after
    `warmup` untimed steps it reports ready and starts its timed steps when
    every process is ready (go)."""
    import oracle
    g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40)
    t = slice_bytes
    data = gen.fill_bytes(gen.SEED_DATA + seed_off, B * t).reshape(B, t)
    er = np.zeros(N_CODED, np.uint8)
    er[gen.sample_indices(N_CODED, gen.round_count(ERASE_FRAC, N_CODED), gen.SEED_ERASE)] = 1
    u, nl = gen.round_count(UPDATE_FRAC, B), gen.round_count(REPAIR_FRAC, N_CODED)
    for r in range(warmup):
        idx = gen.sample_indices(B, u, gen.SEED_UPDATE + (r << gen.ROUND_SHIFT))
        new = gen.fill_bytes(gen.SEED_NEWDATA + (r << gen.ROUND_SHIFT), u * t).reshape(u, t)
        lost = gen.sample_indices(N_CODED, nl, gen.SEED_REPAIR + (r << gen.ROUND_SHIFT))
        _, _, data = _oracle_step(g, data, er, idx, new, lost, t)
    q.put(("ready", 0, 0.0))
    go.wait(600)
    src = 0
    t0 = time.perf_counter()
    for r in range(warmup, warmup + steps):
        idx = gen.sample_indices(B, u, gen.SEED_UPDATE + (r << gen.ROUND_SHIFT))
        new = gen.fill_bytes(gen.SEED_NEWDATA + (r << gen.ROUND_SHIFT), u * t).reshape(u, t)
        lost = gen.sample_indices(N_CODED, nl, gen.SEED_REPAIR + (r << gen.ROUND_SHIFT))
        out, path, data = _oracle_step(g, data, er, idx, new, lost, t)
        src += B * t + int((path.unrecovered[:B] == 0).sum()) * t
    q.put(("done", src, time.perf_counter() - t0))


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_all_cores(slice_bytes: int, steps: int, warmup: int = 0):
    """The oracle, unchanged, in one process per host core, each on its own
    byte slice of every block of the same stripe (Section 3.1's parallel
    scheme: every byte slice is an independent copy of the same problem),
    all timed steps started together. Processes are spawned (not forked: the
    caller may hold a CUDA context). Returns (source bytes, wall seconds,
    cores)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = host_cores()
    ctx = mp.get_context("spawn")
    q, go = ctx.Queue(), ctx.Event()
    procs = [ctx.Process(target=_oracle_proc, args=(slice_bytes, steps, p, q, go, warmup))
             for p in range(n)]
    for pr in procs:
        pr.start()
    for _ in range(n):
        assert q.get(timeout=600)[0] == "ready"
    t0 = time.perf_counter()
    go.set()
    done = [q.get(timeout=900) for _ in range(n)]
    wall = time.perf_counter() - t0
    for pr in procs:
        pr.join(timeout=600)
    return sum(x[1] for x in done), wall, n


def cpu_baseline_all_cores(slice_bytes: int, steps: int):
    """cpu_baseline on every host core (see oracle_all_cores)."""
    per = max(1, steps // 2)
    src, wall, n = oracle_all_cores(slice_bytes, per)
    return {"value": round(src / wall / 1e9, 4), "unit": "GB/s", "cores": n, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": "%d processes, each %d steps of the same stripe, graph and erasures on its "
                      "own %d-byte slice of every block (distinct seeded bytes per process)"
                      % (n, per, slice_bytes),
            "seconds": round(wall, 2)}


def level_counts(levels_gpu):
    """Algorithm 5's level count (the delayed schedule, which the GPU runs)
    beside Algorithm 1's count of sweeps with immediate updates (t_m of
    Section 3.1), both from the oracle on the stripe's erasure draw."""
    import oracle
    g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40)
    er = np.zeros(N_CODED, np.uint8)
    er[gen.sample_indices(N_CODED, gen.round_count(ERASE_FRAC, N_CODED), gen.SEED_ERASE)] = 1
    path = oracle.dpg(g, er)
    order = np.arange(N_CODED + M, dtype=np.int32)
    unrec, sweeps = oracle.peel_immediate(g, er, order, with_sweeps=True)
    return {"algorithm5_delayed_levels": int(path.n_levels), "gpu_levels": levels_gpu,
            "algorithm1_immediate_sweeps": int(sweeps),
            "same_recovered_set": bool(np.array_equal(unrec, path.unrecovered)),
            "note": "Algorithm 1 visits the constraints in index order (coded rows, then checks)"}


def run_reference(args):
    """The reference arm: the oracle (the paper has no runnable reference),
    unchanged, on the machine's host cores: one process per core, each running
    the step (encode, decode, 1% update, 5% repair) of the same stripe on its
    own byte slice of every block; W untimed steps, then K timed steps started
    together. A step is one oracle step on every core's slice."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    t = args.cpu_slice
    src, wall, n = oracle_all_cores(t, args.steps, args.warmup)
    v = src / wall / 1e9
    ms = wall * 1e3 / max(args.steps, 1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded splitmix64 bytes and graphs)",
        "config": {"workload": WORKLOAD, "b": B, "m": M, "n": N_CODED, "block_bytes": T,
                   "sample_block_bytes": t},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": n, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": "each step: the same stripe on a %d-byte slice of every block "
                                   "in each of %d processes (one per host core, distinct seeded "
                                   "bytes)" % (t, n)},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batched(args):
    """The batched-stripes workload as its own JSON line (see batched_measure)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    line = batched_measure(args, device, args.stripes, args.steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batched_measure(args, device, S, K):
    """Many uneven stripes (plain LT, RSD(0.05, 0.01) degrees): k uniform in
    [64, 4096], t from {4, 16, 64} KiB, n = round(1.3 k), 10-25% of each
    stripe's coded blocks erased. One step = encode + decode of every stripe.
    Compares one CUDA-graph replay of the batch (fs_batch: a fixed number of
    launches), the same batch run eagerly, and per-stripe fs_encode +
    fs_decode calls; the batched outputs are checked against the per-stripe
    ones byte for byte. Returns the JSON line (a dict)."""
    import torch
    from paper_1702_07409_gb300 import autotune
    from paper_1702_07409_gb300 import founsure as fs
    rank, world, local = dist_env()
    peak, peak_kind = peaks()
    rng = np.random.default_rng(gen.SEED_GRAPH + rank)
    ks = rng.integers(64, 4097, S)
    ts = rng.choice([4096, 16384, 65536], S)
    fr = rng.uniform(0.10, 0.25, S)
    gen_t = torch.Generator(device=device)
    gen_t.manual_seed(gen.SEED_DATA + rank)
    st = []
    for i in range(S):
        k, t = int(ks[i]), int(ts[i])
        n = int(round(1.3 * k))
        g = gen.make_graph(k, 0, n, gen.DIST_RSD, 0.05, 0.01, stripe=(rank << 12) + i)
        code = fs.Code(g, t)
        er = np.zeros(n, np.uint8)
        er[gen.sample_indices(n, gen.round_count(float(fr[i]), n),
                              gen.SEED_ERASE + ((rank << 12) + i << gen.STRIPE_SHIFT))] = 1
        s = {"code": code, "k": k, "n": n, "t": t,
             "data": torch.randint(0, 256, (k, t), dtype=torch.uint8, device=device, generator=gen_t),
             "coded": torch.empty((n, t), dtype=torch.uint8, device=device),
             "erased": torch.from_numpy(er).to(device),
             "data_out": torch.empty((k, t), dtype=torch.uint8, device=device),
             "unrecovered": torch.empty(k, dtype=torch.uint8, device=device),
             "n_unrecovered": torch.empty(1, dtype=torch.int32, device=device),
             "ws": code.workspace(fs.OP_DECODE, device=device),
             "ws_e": code.workspace(fs.OP_ENCODE, device=device)}
        st.append(s)
    enc_keys = ("code", "data", "coded")
    dec_keys = ("code", "coded", "erased", "data_out", "unrecovered", "n_unrecovered", "ws")

    # the project's autotuner: CTAs per SM of the batched row kernel
    tuned = autotune.tune_batch_encode([s["code"] for s in st],
                                       lambda: fs.Batch([{k: s[k] for k in enc_keys} for s in st],
                                                        fs.OP_ENCODE))
    enc = fs.Batch([{k: s[k] for k in enc_keys} for s in st], fs.OP_ENCODE)
    dec = fs.Batch([{k: s[k] for k in dec_keys} for s in st], fs.OP_DECODE)

    def per_stripe():
        for s in st:
            s["code"].encode(s["data"], None, s["coded"], s["ws_e"])
            s["code"].decode(s["coded"], s["erased"], s["data_out"], s["unrecovered"],
                             s["n_unrecovered"], s["ws"])

    # per-stripe reference outputs, then the batched ones must equal them
    per_stripe()
    torch.cuda.synchronize()
    ref = [(s["coded"].clone(), s["data_out"].clone(), s["unrecovered"].clone()) for s in st]
    for s in st:
        s["coded"].zero_()
        s["data_out"].zero_()
    side = torch.cuda.Stream(device=device)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        enc.run(side)
        dec.run(side)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        enc.run(torch.cuda.current_stream())
        dec.run(torch.cuda.current_stream())
    graph.replay()
    torch.cuda.synchronize()
    same = all(torch.equal(s["coded"], r[0]) and torch.equal(s["data_out"], r[1]) and
               torch.equal(s["unrecovered"], r[2]) for s, r in zip(st, ref))
    if not same:
        raise RuntimeError("batched outputs differ from the per-stripe outputs")
    recovered = sum(int(s["k"] - s["unrecovered"].sum().item()) * s["t"] for s in st)
    src = sum(s["k"] * s["t"] for s in st) + recovered
    enc_bytes = sum((s["k"] + s["n"]) * s["t"] for s in st)
    dec_bytes = 2 * recovered  # plain LT: one coded payload read and one block written per pair

    def timed(fn, K):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        barrier()
        return reduce_max(e0.elapsed_time(e1), device) / K

    with ClockSampler(local) as clk:
        ms_graph = timed(graph.replay, K)
    ms_eager = timed(lambda: (enc.run(), dec.run()), K)
    ms_per = timed(per_stripe, max(1, K // 4))
    clocks = clk.summary()
    gbs = world * src / (ms_graph * 1e-3) / 1e9
    alg = (enc_bytes + dec_bytes) / (ms_graph * 1e-3) / 1e9
    line = {
        "metric": METRIC + " (batched stripes)", "value": round(gbs, 2), "unit": "GB/s",
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_graph, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded device random bytes, splitmix64 graphs)",
        "config": {"workload": "%d stripes, plain LT, RSD(0.05, 0.01), k uniform [64, 4096], "
                               "t from {4, 16, 64} KiB, n = 1.3 k, 10-25%% erased; step = encode + "
                               "decode of every stripe" % S,
                   "source_bytes": int(sum(s["k"] * s["t"] for s in st)),
                   "l2": "inputs larger than L2 (no flush)"},
        "per_stripe_ms": round(ms_per, 3), "batched_eager_ms": round(ms_eager, 3),
        "speedup_vs_per_stripe": round(ms_per / ms_graph, 2),
        "autotune": tuned,
        "roofline": {"bound": "hbm", "kernel": "fs_batch encode + decode launches",
                     "achieved": round(alg, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(alg / peak, 4), "traffic": None,
                     "algorithmic_bytes": enc_bytes + dec_bytes},
        "outputs_equal_per_stripe": same,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    enc.close()
    dec.close()
    for s_ in st:
        s_["code"].close()
    del st, enc, dec, graph, ref
    return line


def run_repair_local(args):
    """Repair from local recovery groups at the precoded stripe (b = 4096 x
    64 KiB, m = 128, n = 5400): the check #2 / check #3 equations are built
    once on the host (Algorithm 4 and the set-XOR derivations), then 5% of
    the coded blocks (270, the repair seed) are lost and repaired in place
    from the check #3 groups by fs_repair_local. One step = one repair. Also
    times the conventional repair from resident intermediates (fs_repair) on
    the same lost blocks and counts the blocks each reads: the groups read
    only coded blocks, the conventional repair needs the intermediates (and
    with coded blocks alone, a full decode first)."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    peak, peak_kind = peaks()
    g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40)
    h0 = time.perf_counter()
    loc = fs.Local(g)
    build_s = time.perf_counter() - h0
    info = loc.info()
    code = fs.Code(g, T)
    gen_t = torch.Generator(device=device)
    gen_t.manual_seed(gen.SEED_DATA + rank)
    data = torch.randint(0, 256, (B, T), dtype=torch.uint8, device=device, generator=gen_t)
    par = torch.empty((M, T), dtype=torch.uint8, device=device)
    coded = torch.empty((N_CODED, T), dtype=torch.uint8, device=device)
    code.encode(data, par, coded, code.workspace(fs.OP_ENCODE))
    stored = coded.clone()
    lost_idx = gen.sample_indices(N_CODED, gen.round_count(REPAIR_FRAC, N_CODED), gen.SEED_REPAIR)
    lost = np.zeros(N_CODED, np.uint8)
    lost[lost_idx] = 1
    d_lost = torch.from_numpy(lost).to(device)
    coded[d_lost.bool()] = 0  # the lost blocks are gone
    unrep = torch.empty(N_CODED, dtype=torch.uint8, device=device)
    nun = torch.empty(1, dtype=torch.int32, device=device)
    ws = loc.workspace(device)
    loc.repair(d_lost, coded, T, unrep, nun, ws)
    torch.cuda.synchronize()
    n_unrep = int(nun.item())
    ok = ~unrep.bool()
    if not torch.equal(coded[ok], stored[ok]):
        raise RuntimeError("local repair differs from the stored blocks")
    levels = loc.path(ws)
    pairs = [pg for lv in levels for pg in lv]
    gptr, gidx = loc.groups()
    gather = sum(int(gptr[q + 1] - gptr[q]) - 1 for _, q in pairs)
    distinct = set()
    for f, q in pairs:
        distinct.update(int(x) for x in gidx[gptr[q]:gptr[q + 1]] if x != f)
    alg_bytes = (len(distinct) + len(pairs)) * T  # distinct coded blocks read + repaired written
    lp = np.asarray(g.lt_ptr)
    lt_i = np.asarray(g.lt_idx)
    conv_inter = set()
    for sidx in lost_idx:
        conv_inter.update(int(x) for x in lt_i[lp[sidx]:lp[sidx + 1]])
    d_lost_idx = torch.from_numpy(np.asarray(lost_idx, np.int32)).to(device)
    rws = code.workspace(fs.OP_REPAIR)

    def timed(fn, K):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    K = args.steps
    with ClockSampler(local) as clk:
        ms = timed(lambda: loc.repair(d_lost, coded, T, unrep, nun, ws), K)
    ms_conv = timed(lambda: code.repair(d_lost_idx, len(lost_idx), data, par, coded, rws), K)
    clocks = clk.summary()
    torch.cuda.synchronize()
    if not torch.equal(coded, stored):
        raise RuntimeError("repairs left the coded blocks different from the stored ones")
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    line = {
        "metric": "local-group repair time", "value": round(ms, 4), "unit": "ms",
        "n_gpus": 1, "steps": K, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded device random bytes, splitmix64 graph)",
        "config": {"workload": "precoded LDGM stripe b=4096 x 64 KiB, m=128, n=5400, "
                               "FiniteDist max-degree-40; 5%% of the coded blocks (%d) lost and "
                               "repaired from check #3 groups" % len(lost_idx),
                   "groups": info["n_groups"], "group_entries": info["group_entries"],
                   "check2": info["n_check2"], "algorithm4_sweeps": info["sweeps"],
                   "groups_build_s": round(build_s, 2)},
        "repaired": len(pairs), "unrepaired": n_unrep, "levels": len(levels),
        "blocks_read": {"local_gather": gather, "local_distinct": len(distinct),
                        "conventional_intermediates": len(conv_inter),
                        "decode_then_encode": "every coded payload a full decode uses "
                                              "(about k_int = %d blocks)" % (B + M)},
        "conventional_repair_ms": round(ms_conv, 4),
        "roofline": {"bound": "hbm", "kernel": "k_local_dpg + k_local_peel (fs_repair_local)",
                     "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "algorithmic_bytes": alg_bytes,
                     "note": "algorithmic = distinct coded blocks read + repaired blocks "
                             "written; the gathers read %d blocks in all" % gather},
        "gpu_launches": 2 * K,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_simdisk(args):
    """The paper's simDisk sweep at the precoded stripe (b = 4096, m = 128,
    n = 5400): the coded blocks striped over 10 disks (540 each), every
    combination of 1-4 failed disks (10 + 45 + 120 + 210 = 385 erasure
    patterns), each a symbolic decode (Algorithm 5, no payload). One step =
    one batch of all patterns (fs_batch, FS_OP_SCHEDULE; one CTA per pattern),
    device-timed; the patterns' outcomes are checked against the oracle on a
    sample. cpu_baseline: the oracle's schedule on a sample of the patterns."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    from paper_1702_07409_gb300 import simdisk
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    disks, fmax = 10, 4
    g = gen.make_graph(B, M, N_CODED, gen.DIST_FINITE40)
    sd = simdisk.SimDisk(g, disks, device=device)
    code, n, k = sd.code, N_CODED, B + M
    combos, flags = [], []
    for f in range(1, fmax + 1):
        c, fl = simdisk.failure_patterns(n, disks, f)
        combos += c
        flags.append(fl)
    flags = np.concatenate(flags)
    P = flags.shape[0]
    d_er = torch.from_numpy(flags).to(device)
    unrec = torch.empty((P, k), dtype=torch.uint8, device=device)
    nun = torch.empty(P, dtype=torch.int32, device=device)
    ws = torch.empty((P, sd.ws_bytes), dtype=torch.uint8, device=device)
    stripes = [{"code": code, "erased": d_er.data_ptr() + i * n,
                "unrecovered": unrec.data_ptr() + i * k, "n_unrecovered": nun.data_ptr() + 4 * i,
                "ws": ws.data_ptr() + i * sd.ws_bytes} for i in range(P)]
    batch = fs.Batch(stripes, fs.OP_SCHEDULE)
    for _ in range(args.warmup):
        batch.run()
    torch.cuda.synchronize()
    K = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record()
        for _ in range(K):
            batch.run()
        e1.record()
        torch.cuda.synchronize()
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / K
    got = nun.cpu().numpy()
    # cpu_baseline leg: the oracle's schedule on a sample of the patterns (its
    # outcomes must also equal the batch's)
    import oracle
    oracle.build()
    sample = list(range(0, P, max(1, P // 12)))[:12]
    t0 = time.perf_counter()
    for i in sample:
        if int(oracle.dpg(g, flags[i]).unrecovered.sum()) != int(got[i]):
            raise RuntimeError("simDisk pattern %d differs from the oracle" % i)
    cpu_s = (time.perf_counter() - t0) / len(sample)
    per_f, o = {}, 0
    for f in range(1, fmax + 1):
        c = math.comb(disks, f)
        per_f[str(f)] = {"patterns": c, "tolerated": round(float(np.mean(got[o:o + c] == 0)), 4)}
        o += c
    line = {
        "metric": "simDisk erasure patterns per second", "value": round(P / (ms * 1e-3), 1),
        "unit": "patterns/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (splitmix64 graph)",
        "config": {"workload": "precoded stripe b=4096, m=128, n=5400 striped over %d disks "
                               "(%d blocks each); every combination of 1-%d failed disks, one "
                               "symbolic decode each" % (disks, -(-n // disks), fmax),
                   "patterns": P},
        "by_failures": per_f,
        "cpu_baseline": {"value": round(1.0 / cpu_s, 2), "unit": "patterns/s", "cores": 1,
                         "kind": "oracle", "sample": "%d of the %d patterns" % (len(sample), P)},
        "gpu_launches": 1 * K,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    batch.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_array(args):
    """The array LDPC precode of Algorithm 2 at a size like the precoded
    stripe: b = 4154 data blocks of 64 KiB, k = 4288 intermediates (p = 67,
    k' = 64, j' = 2: 134 checks in two levels, the second reading parities of
    the first), n = 5574 = 1.3 k coded blocks, FiniteDist max-degree-40, 20%
    erased. One step = encode (one row-gather launch per precode level, then
    the LT rows) + decode (schedule beside nothing: serial, then payload).
    The delta update does not apply to chained precodes. cpu_baseline: the
    oracle's encode + decode on a 16 KiB slice of every block."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    peak, peak_kind = peaks()
    b, k = 4154, 4288
    n, m = (13 * k + 5) // 10, k - b
    g = gen.make_graph_array(b, k, n, gen.DIST_FINITE40)
    code = fs.Code(g, T)
    if args.peel_flow is not None:
        code.set_tuning(fs.TUNE_PEEL_FLOW, args.peel_flow)
    gen_t = torch.Generator(device=device)
    gen_t.manual_seed(gen.SEED_DATA + rank)
    data = torch.randint(0, 256, (b, T), dtype=torch.uint8, device=device, generator=gen_t)
    par = torch.empty((m, T), dtype=torch.uint8, device=device)
    coded = torch.empty((n, T), dtype=torch.uint8, device=device)
    er = np.zeros(n, np.uint8)
    er[gen.sample_indices(n, gen.round_count(ERASE_FRAC, n), gen.SEED_ERASE)] = 1
    d_er = torch.from_numpy(er).to(device)
    out = torch.empty((b, T), dtype=torch.uint8, device=device)
    unrec = torch.empty(k, dtype=torch.uint8, device=device)
    nun = torch.empty(1, dtype=torch.int32, device=device)
    ews, dws = code.workspace(fs.OP_ENCODE), code.workspace(fs.OP_DECODE)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def step(record=False):
        if record:
            evs[0].record()
        code.encode(data, par, coded, ews)
        if record:
            evs[1].record()
        code.decode_schedule(d_er, unrec, nun, dws)
        if record:
            evs[2].record()
        code.decode_payload(coded, out, dws)
        if record:
            evs[3].record()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    un = unrec[:b].bool()
    if not torch.equal(out[~un], data[~un]):
        raise RuntimeError("array-precoded decode differs from the data")
    recovered = int((~un).sum().item())
    view = code.decode_path(dws)
    g_arr = view["pair_g"].cpu().numpy()
    coded_pairs = int((g_arr < n).sum())
    K = args.steps
    t_enc, t_sch, t_pay = [], [], []
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record()
        for _ in range(K):
            step(record=True)
            torch.cuda.synchronize()
            t_enc.append(evs[0].elapsed_time(evs[1]))
            t_sch.append(evs[1].elapsed_time(evs[2]))
            t_pay.append(evs[2].elapsed_time(evs[3]))
        t1.record()
        torch.cuda.synchronize()
    clocks = clk.summary()
    enc_ms, sch_ms, pay_ms = (statistics.mean(x) for x in (t_enc, t_sch, t_pay))
    ms = enc_ms + sch_ms + pay_ms
    src = (b + recovered) * T
    enc_bytes = (b + m + n) * T
    pay_bytes = (coded_pairs + recovered) * T

    import oracle  # cpu_baseline leg
    oracle.build()
    ts = args.cpu_slice
    hdata = gen.fill_bytes(gen.SEED_DATA, b * ts).reshape(b, ts)
    c0 = time.perf_counter()
    _, hcod = oracle.encode(g, hdata, ts)
    hout, hpath = oracle.decode(g, hcod, er, ts)
    cpu_s = time.perf_counter() - c0
    cpu_src = (b + int((hpath.unrecovered[:b] == 0).sum())) * ts
    line = {
        "metric": METRIC + " (array LDPC precode)", "value": round(src / (ms * 1e-3) / 1e9, 2),
        "unit": "GB/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded device random bytes, splitmix64 LT graph, Algorithm 2 precode)",
        "config": {"workload": "array LDPC precode b=4154 x 64 KiB, k=4288 (p=67, two levels of 67 "
                               "checks), n=5574, FiniteDist max-degree-40, 20% erased; step = "
                               "encode + decode (schedule, payload), serial",
                   "unrecovered": int(unrec.sum().item()),
                   "l2": "inputs larger than L2 (no flush)"},
        "ops_ms": {"encode": round(enc_ms, 4), "decode_schedule": round(sch_ms, 4),
                   "decode_payload": round(pay_ms, 4)},
        "roofline": {"bound": "hbm", "kernel": f"{PEEL_KERNEL[walk_of(args)]} (fs_decode_payload)",
                     "achieved": round(pay_bytes / (pay_ms * 1e-3) / 1e9, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(pay_bytes / (pay_ms * 1e-3) / 1e9 / peak, 4), "traffic": None,
                     "algorithmic_bytes": pay_bytes},
        "encode_roofline": {"bound": "hbm", "kernel": "k_rows (fs_encode, one launch per precode "
                                                      "level + the LT rows)",
                            "achieved": round(enc_bytes / (enc_ms * 1e-3) / 1e9, 1), "peak": peak,
                            "unit": "GB/s",
                            "frac": round(enc_bytes / (enc_ms * 1e-3) / 1e9 / peak, 4),
                            "traffic": None, "algorithmic_bytes": enc_bytes},
        "cpu_baseline": {"value": round(cpu_src / cpu_s / 1e9, 4), "unit": "GB/s", "cores": 1,
                         "kind": "oracle", "sample": "encode + decode of the same code and "
                                                     "erasures on a %d-byte slice of every block" % ts},
        # per step: the precode's two levels and the LT rows, the schedule, the payload
        "gpu_launches": 5 * K,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serving(args):
    """The serving workload as its own JSON line (see serving_measure)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    line = serving_measure(args, device, args.requests)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_measure(args, device, n_requests):
    """Requests served from device-resident stripes (paper_1702_07409_gb300.serve):
    Poisson arrivals (mean 2000 requests/s, seeded exponential gaps) of encode
    60% / decode 25% / update 10% / repair 5%; stripe sizes log-uniform in
    [1, 256] MiB over the powers of two (each of the 9 sizes equally likely,
    so codes are reused), t = 16 or 64 KiB, n = 1.3 k, RSD(0.05, 0.01);
    decodes erase 10-25% of the target's coded blocks, updates rewrite 1% of
    its data blocks, repairs recompute 5% of its coded blocks; decode /
    update / repair pick a resident stripe at random from a pre-populated
    pool; admission under a 120 GB budget. Continuous batching is compared
    with one request per launch on the same stream of requests. Returns the
    JSON line (a dict)."""
    import torch
    from paper_1702_07409_gb300.serve import Request, Server, latency_stats
    rank, world, local = dist_env()
    budget = int(args.budget_gb * 1e9)
    sizes = [1 << (20 + j) for j in range(9)]  # 1 MiB .. 256 MiB

    def draw(n_req, meta):
        """meta: stripe id -> (k, n) of the resident pool; grows with encodes.
        The same seed every time: both serving modes see the same stream."""
        rng = np.random.default_rng(gen.SEED_GRAPH + 5 + rank)
        reqs, sid, t_now = [], 1 << 20, 0.0
        live = list(meta)
        for i in range(n_req):
            t_now += float(rng.exponential(1.0 / args.rate))
            u = rng.random()
            if u < 0.60:
                size = sizes[int(rng.integers(0, 9))]  # log-uniform over the 9 sizes
                t = int(rng.choice([16384, 65536]))
                reqs.append(Request(i, "encode", t_now, k=size // t, t=t, target=sid, seed=10**6 + i))
                meta[sid] = (size // t, int(round(1.3 * (size // t))))
                live.append(sid)
                sid += 1
            elif u < 0.85:
                reqs.append(Request(i, "decode", t_now, target=int(rng.choice(live)), seed=2 * 10**6 + i,
                                    erase_frac=float(rng.uniform(0.10, 0.25))))
            elif u < 0.95:  # 1% of the target's data blocks rewritten
                tg = int(rng.choice(live))
                reqs.append(Request(i, "update", t_now, target=tg, seed=3 * 10**6 + i,
                                    n_update=max(1, meta[tg][0] // 100)))
            else:  # 5% of the target's coded blocks lost
                tg = int(rng.choice(live))
                reqs.append(Request(i, "repair", t_now, target=tg, seed=4 * 10**6 + i,
                                    n_lost=max(1, meta[tg][1] // 20)))
        return reqs

    def serve(batching):
        srv = Server(budget, device=device, streams=3 if batching else 1, batching=batching)
        for size in sizes:  # every code the stream can ask for, built before the clock starts
            for t in (16384, 65536):
                srv.code_for(size // t, t)
        # every kernel loaded before the clock starts: the smallest and the
        # largest code of the stream (their decodes take different kernels)
        srv.warm_up(((sizes[0] // 65536, 65536), (sizes[-1] // 16384, 16384)))
        meta = {}
        prng = np.random.default_rng(77 + rank)
        for p in range(args.pool):
            size = sizes[int(prng.integers(0, 9))]
            t = int(prng.choice([16384, 65536]))
            srv.add_resident(p, size // t, t, seed=500 + p)
            meta[p] = (size // t, srv.stripes[p].n)
        reqs = draw(n_requests, meta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reqs = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        served = [r for r in reqs if r.done is not None and not r.out.get("dropped")
                  and not r.out.get("rejected")]
        bytes_ = 0
        for r in served:
            if r.kind == "encode":
                bytes_ += r.k * r.t
            elif r.kind == "decode":
                bytes_ += int(r.out["data_out"].numel())
        span = max(r.done for r in served) if served else wall
        res = dict(latency_stats(reqs), gbs=round(bytes_ / span / 1e9, 2), span_s=round(span, 3),
                   wave_stats=srv.wave_stats(),
                   waves=srv.n_waves, peak_gb=round(srv.peak / 1e9, 2), evictions=srv.evictions,
                   dropped=sum(1 for r in reqs if r.out.get("dropped")),
                   rejected=sum(1 for r in reqs if r.out.get("rejected")))
        srv.close()
        return res

    with ClockSampler(local) as clk:
        batched = serve(True)
    single = serve(False)
    clocks = clk.summary()
    line = {
        "metric": "served source GB/s, p50/p99 latency", "value": batched["gbs"], "unit": "GB/s",
        "n_gpus": world, "steps": n_requests, "warmup": 0, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded device random bytes, splitmix64 graphs, Poisson arrivals)",
        "config": {"workload": "serving: Poisson %g requests/s, encode 60 / decode 25 / update 10 / "
                               "repair 5 %%, stripes 1-256 MiB (the 9 powers of two equally likely), "
                               "t 16 or 64 KiB, n = 1.3 k, budget %g GB, pool %d"
                               % (args.rate, args.budget_gb, args.pool),
                   "requests": n_requests},
        "batched": batched, "one_request_per_launch": single,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"]},
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-slice", type=int, default=16384,
                    help="bytes of each block the CPU oracle processes per step")
    ap.add_argument("--cpu-steps", type=int, default=12,
                    help="steps of the oracle in cpu_baseline (about 0.85 s each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the decode-only, config-1, batched and serving numbers of the "
                         "default line")
    ap.add_argument("--extras-stripes", type=int, default=512,
                    help="stripes of the batched object in the default line")
    ap.add_argument("--extras-requests", type=int, default=600,
                    help="requests of the serving object in the default line")
    ap.add_argument("--l2-hints", action="store_true",
                    help="tuning knob: L2 evict-last / evict-first hints")
    ap.add_argument("--peel-flow", type=int, choices=[0, 1, 2, 3], default=None,
                    help="tuning knob FS_TUNE_PEEL_FLOW: 0 the level walk, 1 the dataflow walk "
                         "without level barriers, 2 the key walk from 64 MiB of intermediates, "
                         "3 the key walk at any size (default: the library's, 2)")
    ap.add_argument("--two-pass", action="store_true",
                    help="decode in the paper's two passes (LT code, then the precode) "
                         "instead of jointly")
    ap.add_argument("--serial-schedule", action="store_true",
                    help="run the decoding schedule after the encode instead of beside it")
    ap.add_argument("--peel-ctas", type=int, default=0, help="tuning knob (1..8)")
    ap.add_argument("--gather-ctas", type=int, default=0, help="tuning knob (1..16)")

    ap.add_argument("--workload", default="stripe",
                    choices=["stripe", "batched", "serving", "repair_local", "simdisk", "array"],
                    help="stripe: the precoded stripe step (default); batched: many uneven "
                         "stripes through fs_batch vs per-stripe calls; serving: a Poisson "
                         "stream of requests on resident stripes; repair_local: repair of 5%% "
                         "lost coded blocks from local recovery groups; simdisk: every "
                         "combination of 1-4 failed disks out of 10, symbolic decodes; array: "
                         "the array LDPC precode of Algorithm 2")
    ap.add_argument("--requests", type=int, default=2000, help="requests of --workload serving")
    ap.add_argument("--rate", type=float, default=2000.0, help="mean arrivals per second (serving)")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="HBM budget (serving)")
    ap.add_argument("--pool", type=int, default=64, help="pre-populated stripes (serving)")
    ap.add_argument("--stripes", type=int, default=512, help="stripes of --workload batched")
    ap.add_argument("--block-bytes", type=int, default=65536,
                    help="block size t (default 65536; smaller only for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    globals()["T"] = args.block_bytes
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "repair_local":
        run_repair_local(args)
    elif args.workload == "simdisk":
        run_simdisk(args)
    elif args.workload == "array":
        run_array(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
