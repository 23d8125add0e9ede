"""Autotuner for batches of stripes.

The batched encode runs a persistent row-gather kernel whose resident CTAs
per SM (FS_TUNE_GATHER_CTAS, 1..5 for that kernel) trade latency hiding
against L2 working set; which is best depends on the stripes' block sizes and
degrees. tune_batch_encode times a batch once per candidate on the GPU it
will run on and keeps the fastest (it sets that knob on every code, so
batches created afterwards use it).
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


def tune_batch_encode(codes, make_batch, candidates=(2, 3, 4, 5), runs: int = 3,
                      timer=_cuda_timer) -> dict:
    """Times make_batch() (an encode Batch over `codes`) for each candidate
    value of the CTAs-per-SM knob and keeps the fastest.

    codes       the stripes' Code objects
    make_batch  builds the batch (after the knob is set on every code)
    Returns {"knob", "best", "ms": {candidate: ms per run}}."""
    from . import founsure as fs
    times = {}
    for c in candidates:
        for code in codes:
            code.set_tuning(fs.TUNE_GATHER_CTAS, c)
        batch = make_batch()
        try:
            times[c] = float(timer(batch.run, runs))
        finally:
            batch.close()
    best = min(times, key=times.get)
    for code in codes:
        code.set_tuning(fs.TUNE_GATHER_CTAS, best)
    return {"knob": "gather_ctas", "best": best,
            "ms": {str(k): round(v, 4) for k, v in times.items()}}
