"""Host-side admission of the serving loop (no GPU needed): the wave a pump
admits, per-stripe ordering, dropped and rejected requests, LRU eviction
that never touches a stripe in use, and cancellation. The device side
(launching a wave, retiring it) is replaced by a recorder."""
import collections

import pytest

pytest.importorskip("torch")

from paper_1702_07409_gb300 import serve  # noqa: E402

T = 1024


class _FakeCode:
    def workspace_bytes(self, op, n_items=0):
        return 256 + 16 * n_items


def _server(budget, max_wave=64):
    """A Server without device state: pump() admits, _launch records."""
    s = serve.Server.__new__(serve.Server)
    s.budget = budget
    s.max_wave = max_wave
    s.stripes = collections.OrderedDict()
    s.resident = s.transient = s.peak = s.evictions = 0
    s.waiting = collections.deque()
    s.encoding = set()
    s.launched = []
    s._launch = lambda wave: s.launched.append([r.rid for r in wave])
    s._retire = lambda block=False: None
    s.code_for = lambda k, t: (_FakeCode(), 2 * k)
    return s


def _resident(s, sid, k=4):
    st = serve._Stripe(sid, _FakeCode(), k, 2 * k, T, None, None)
    s.stripes[sid] = st
    s.resident += st.nbytes
    return st


def _req(rid, kind, target, **kw):
    return serve.Request(rid, kind, 0.0, target=target, **kw)


def test_one_request_per_stripe_per_wave_in_order():
    s = _server(1 << 30)
    _resident(s, 1)
    _resident(s, 2)
    for r in (_req(0, "decode", 1, erase_frac=0.1), _req(1, "update", 1, n_update=2),
              _req(2, "repair", 2, n_lost=1), _req(3, "decode", 9)):
        s.submit(r)
    s.pump(0.0)
    assert s.launched == [[0, 2]]  # rid 1 waits for stripe 1, rid 3's stripe does not exist
    assert [r.rid for r in s.waiting] == [1]
    assert s.stripes[1].busy and s.stripes[2].busy


def test_missing_stripe_is_dropped_and_oversized_request_rejected():
    s = _server(64 * T)
    _resident(s, 1)
    drop, big = _req(0, "decode", 7), serve.Request(1, "encode", 0.0, k=1000, t=T, target=5)
    s.submit(drop)
    s.submit(big)
    s.pump(0.5)
    assert drop.out.get("dropped") and drop.done == 0.5
    assert big.out.get("rejected") and big.done == 0.5
    assert s.launched == [] and s.evictions == 0 and 1 in s.stripes


def test_eviction_takes_idle_stripes_in_lru_order_and_spares_the_target():
    st = [None] * 3
    s = _server(3 * 12 * T + 1024)  # three stripes of (4 + 8) blocks, little room besides
    for i in range(3):
        st[i] = _resident(s, i)
    # a repair on the least recently used stripe needs more room: stripe 1 goes, not 0
    s.submit(_req(0, "repair", 0, n_lost=200))
    s.pump(0.0)
    assert s.launched == [[0]]
    assert list(s.stripes) == [0, 2] and s.evictions == 1
    assert s.resident + s.transient <= s.budget


def test_short_memory_holds_the_queue_behind_the_first_waiting_request():
    s = _server(12 * T + 512)
    a = _resident(s, 1)
    a.busy = True  # in flight: cannot be evicted
    s.submit(serve.Request(0, "encode", 0.0, k=4, t=T, target=2))
    s.submit(_req(1, "repair", 1, n_lost=1))
    s.pump(0.0)
    assert s.launched == [] and [r.rid for r in s.waiting] == [0, 1]
    a.busy = False
    s.pump(0.0)  # now stripe 1 can be evicted for the encode
    assert s.launched == [[0]] and 1 not in s.stripes


def test_cancel_withdraws_only_waiting_requests():
    s = _server(1 << 30)
    _resident(s, 1)
    r0, r1 = _req(0, "decode", 1), _req(1, "update", 1, n_update=1)
    s.submit(r0)
    s.submit(r1)
    s.pump(0.0)  # r0 admitted, r1 waits behind it
    assert not s.cancel(0)
    assert s.cancel(1) and r1.out.get("cancelled") and not s.waiting
