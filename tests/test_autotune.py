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
    cost = {2: 5.0, 3: 2.5, 4: 3.0, 5: 4.0}

    def make():
        return FakeBatch(codes[0].knobs[fs.TUNE_GATHER_CTAS])

    def timer(fn, runs):
        fn()
        return cost[FakeBatch.made[-1].ctas]

    res = autotune.tune_batch_encode(codes, make, timer=timer)
    assert res["best"] == 3
    assert all(c.knobs[fs.TUNE_GATHER_CTAS] == 3 for c in codes)
    assert all(b.closed for b in FakeBatch.made)
    assert res["ms"] == {"2": 5.0, "3": 2.5, "4": 3.0, "5": 4.0}
