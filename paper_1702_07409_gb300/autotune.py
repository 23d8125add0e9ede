"""Autotuner for batches of stripes.

The batched encode runs a persistent row-gather kernel whose resident CTAs
per SM (FS_TUNE_GATHER_CTAS, 1..4 for that kernel) and rows per work ticket
(FS_TUNE_ROWS_PER_TICKET) trade latency hiding against the L2 working set;
which is best depends on the stripes' block sizes and degrees.
tune_batch_encode times a batch once per candidate on the GPU it will run on
and keeps the fastest (it sets the knobs on every code, so batches created
afterwards use them).
"""
from __future__ import annotations


def _cuda_timer(fn, runs: int) -> float:
    """Milliseconds per call of fn, CUDA events on the current stream."""
    import torch
    fn()  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(runs):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / runs


def tune_batch_encode(codes, make_batch, candidates=((2, 16), (3, 16), (4, 16), (3, 8), (4, 8),
                                                     (4, 4), (4, 2)),
                      runs: int = 3, timer=_cuda_timer) -> dict:
    """Times make_batch() (an encode Batch over `codes`) for each candidate
    (CTAs per SM, rows per ticket) of the row-gather kernel and keeps the
    fastest (fewer rows per ticket narrow the byte range the tickets in
    flight cover, which decides how much of the gathered inputs L2 keeps).

    codes       the stripes' Code objects
    make_batch  builds the batch (after the knobs are set on every code)
    Returns {"knobs", "best", "ms": {"ctas x rows": ms per run}}."""
    from . import founsure as fs
    times = {}
    for cand in candidates:
        ctas, rows = cand
        for code in codes:
            code.set_tuning(fs.TUNE_GATHER_CTAS, ctas)
            code.set_tuning(fs.TUNE_ROWS_PER_TICKET, rows)
        batch = make_batch()
        try:
            times[cand] = float(timer(batch.run, runs))
        finally:
            batch.close()
    best = min(times, key=times.get)
    for code in codes:
        code.set_tuning(fs.TUNE_GATHER_CTAS, best[0])
        code.set_tuning(fs.TUNE_ROWS_PER_TICKET, best[1])
    return {"knobs": ["gather_ctas", "rows_per_ticket"], "best": list(best),
            "ms": {"%dx%d" % k: round(v, 4) for k, v in times.items()}}
