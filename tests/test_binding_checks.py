"""Argument checks of the Python binding (no GPU needed): every hot call
refuses a buffer smaller than its operation needs before it reaches the
library, naming the buffer, and refuses host tensors of the right size (the
library has no CPU path)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1702_07409_gb300 import founsure as fs  # noqa: E402

B, M, N, T = 8, 2, 12, 32
WS = {fs.OP_ENCODE: 512, fs.OP_DECODE: 4096, fs.OP_REPAIR: 256}


def _code():
    """A Code without a device handle: only the host-side checks run."""
    c = fs.Code.__new__(fs.Code)
    c.b, c.m, c.n, c.t, c.k_int = B, M, N, T, B + M
    c._h = None
    c.workspace_bytes = lambda op, n_items=0: WS.get(op, 256 + 64 * n_items)
    return c


def _buf(nbytes):
    return torch.zeros(nbytes, dtype=torch.uint8)


# operation -> (method, positional arguments in order: a byte size per buffer,
# or ("int", value) for a count)
CALLS = {
    "encode": ("encode", [("data", B * T), ("parity", M * T), ("coded", N * T),
                          ("ws", WS[fs.OP_ENCODE])]),
    "encode_rows": ("encode_rows", [("int", 0), ("int", N), ("data", B * T), ("parity", M * T),
                                    ("coded", N * T), ("ws", WS[fs.OP_ENCODE])]),
    "decode": ("decode", [("coded", N * T), ("erased", N), ("data_out", B * T),
                          ("unrecovered", B + M), ("n_unrecovered", 4),
                          ("ws", WS[fs.OP_DECODE])]),
    "decode_schedule": ("decode_schedule", [("erased", N), ("unrecovered", B + M),
                                            ("n_unrecovered", 4), ("ws", WS[fs.OP_DECODE])]),
    "decode_payload": ("decode_payload", [("coded", N * T), ("data_out", B * T),
                                          ("ws", WS[fs.OP_DECODE])]),
    "update": ("update", [("idx", 4 * 3), ("int", 3), ("new", 3 * T), ("data", B * T),
                          ("parity", M * T), ("coded", N * T), ("ws", 256 + 64 * 3)]),
    "repair": ("repair", [("lost", 4 * 2), ("int", 2), ("data", B * T), ("parity", M * T),
                          ("coded", N * T), ("ws", WS[fs.OP_REPAIR])]),
}


def _args(spec, short=None):
    out = []
    for name, size in spec:
        if name == "int":
            out.append(size)
        else:
            out.append(_buf(size - 1 if name == short else size))
    return out


@pytest.mark.parametrize("op", sorted(CALLS))
def test_each_short_buffer_is_refused_by_name(op):
    method, spec = CALLS[op]
    c = _code()
    for name, _ in spec:
        if name == "int":
            continue
        with pytest.raises(ValueError, match=r"^%s holds" % name):
            getattr(c, method)(*_args(spec, short=name))


@pytest.mark.parametrize("op", sorted(CALLS))
def test_host_tensors_are_refused(op):
    """Sizes pass; the buffers are host memory, which no call accepts."""
    method, spec = CALLS[op]
    with pytest.raises(ValueError, match="expected a CUDA tensor"):
        getattr(_code(), method)(*_args(spec))


BATCH = {
    fs.OP_DECODE: [("coded", N * T), ("erased", N), ("data_out", B * T), ("unrecovered", B + M),
                   ("n_unrecovered", 4), ("ws", WS[fs.OP_DECODE])],
    fs.OP_SCHEDULE: [("erased", N), ("unrecovered", B + M), ("n_unrecovered", 4),
                     ("ws", WS[fs.OP_DECODE])],
}


@pytest.mark.parametrize("op", sorted(BATCH))
def test_batch_stripes_are_checked(op):
    """A batch refuses a stripe with a short buffer before it is created."""
    spec = BATCH[op]
    for short, _ in spec:
        stripe = {"code": _code()}
        stripe.update({name: _buf(size - 1 if name == short else size) for name, size in spec})
        with pytest.raises(ValueError, match=r"^%s holds" % short):
            fs.Batch([stripe], op)
