"""The batch autotuner's selection logic (host only: fake codes, batches and
timer)."""
from paper_1702_07409_gb300 import autotune


class FakeCode:
    def __init__(self):
        self.knobs = {}

    def set_tuning(self, knob, value):
        self.knobs[knob] = value


class FakeBatch:
    made = []

    def __init__(self, ctas):
        self.ctas = ctas
        self.closed = False
        FakeBatch.made.append(self)

    def run(self):
        pass

    def close(self):
        self.closed = True


def test_tuner_keeps_the_fastest_candidate_and_sets_it_on_every_code(monkeypatch):
    from paper_1702_07409_gb300 import founsure as fs
    codes = [FakeCode() for _ in range(3)]
    cost = {(3, 16): 5.0, (4, 8): 2.5, (5, 4): 3.0, (5, 16): 4.0}

    def make():
        return FakeBatch((codes[0].knobs[fs.TUNE_GATHER_CTAS], codes[0].knobs[fs.TUNE_ROWS_PER_TICKET]))

    def timer(fn, runs):
        fn()
        return cost[FakeBatch.made[-1].ctas]

    res = autotune.tune_batch_encode(codes, make, candidates=tuple(cost), timer=timer)
    assert res["best"] == [4, 8]
    assert all(c.knobs[fs.TUNE_GATHER_CTAS] == 4 and c.knobs[fs.TUNE_ROWS_PER_TICKET] == 8
               for c in codes)
    assert all(b.closed for b in FakeBatch.made)
    assert res["ms"] == {"3x16": 5.0, "4x8": 2.5, "5x4": 3.0, "5x16": 4.0}
