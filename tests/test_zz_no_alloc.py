"""fs_encode_static: the encode entry point for callers that cannot allocate
device memory (a storage service that reserves all of its device memory at
start-up, or a binding without a device allocator). It must produce exactly
what fs_encode produces, call after call, from its static scratch area.

This file is collected last on purpose, so a run that stops at the first
failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_1702_07409_gb300 import gen

pytestmark = pytest.mark.gpu


def _encode_both(fs, g, t, seed):
    """Encodes seeded data with fs_encode and with fs_encode_static (called
    directly through the C ABI) and returns both outputs and the status."""
    import torch
    code = fs.Code(g, t)
    data = torch.from_numpy(gen.fill_bytes(seed, g.b * t).reshape(g.b, t)).cuda()
    p0 = torch.empty((g.m, t), dtype=torch.uint8, device="cuda") if g.m else None
    c0 = torch.empty((g.n, t), dtype=torch.uint8, device="cuda")
    code.encode(data, p0, c0, code.workspace(fs.OP_ENCODE))
    p1 = torch.full((g.m, t), 0x5A, dtype=torch.uint8, device="cuda") if g.m else None
    c1 = torch.full((g.n, t), 0x5A, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = fs.lib().fs_encode_static(code._h, ctypes.c_void_p(data.data_ptr()),
                                   ctypes.c_void_p(p1.data_ptr()) if p1 is not None else None,
                                   ctypes.c_void_p(c1.data_ptr()),
                                   ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream))
    assert rc == fs.FS_OK
    torch.cuda.synchronize()
    return (p0, c0), (p1, c1), int(status.item()), code


def test_static_encode_matches_encode_twice_in_a_row():
    from paper_1702_07409_gb300 import founsure as fs
    cases = [
        (gen.make_graph(600, 24, 800, gen.DIST_FINITE40), 4096 + 48, 7),
        (gen.make_graph(100, 0, 150, gen.DIST_RSD, 0.1, 0.05), 1024, 1),
    ]
    for g, t, seed in cases:
        for call in range(2):  # the second call reuses the area the first left behind
            (p0, c0), (p1, c1), status, _ = _encode_both(fs, g, t, seed + call)
            assert status == fs.FS_OK
            assert np.array_equal(c1.cpu().numpy(), c0.cpu().numpy())
            if g.m:
                assert np.array_equal(p1.cpu().numpy(), p0.cpu().numpy())


def test_static_encode_area_covers_large_blocks():
    """The static area holds the encode workspace of large-block codes too:
    the host check that would refuse a code beyond it lets them through, and
    a precoded code of 16 MiB blocks encodes through the static area exactly
    as through fs_encode."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph(8, 0, 12, gen.DIST_RSD, 0.1, 0.05)
    code = fs.Code(g, 256 * 1024 * 1024)  # 256 MiB blocks; nothing is allocated for them
    assert code.workspace_bytes(fs.OP_ENCODE) <= fs.ENCODE_STATIC_SCRATCH_BYTES
    code.close()
    g = gen.make_graph(12, 3, 18, gen.DIST_FINITE40)
    (p0, c0), (p1, c1), status, code = _encode_both(fs, g, 16 * 1024 * 1024, 9)
    assert status == fs.FS_OK
    assert torch.equal(c1, c0) and torch.equal(p1, p0)
    code.close()


def test_static_encode_rejects_bad_pointers():
    """Host-side checks, before anything is enqueued: a null data or coded
    pointer, a missing parity buffer for a precoded code, and a buffer not on
    a 16-byte boundary each return FS_ERR_INVALID."""
    import torch
    from paper_1702_07409_gb300 import founsure as fs
    g = gen.make_graph(60, 4, 90, gen.DIST_FINITE40)
    t = 1024
    code = fs.Code(g, t)
    data = torch.zeros((g.b * t + 16,), dtype=torch.uint8, device="cuda")
    par = torch.empty((g.m * t + 16,), dtype=torch.uint8, device="cuda")
    cod = torch.empty((g.n * t + 16,), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = ctypes.c_void_p

    def call(d, p, c):
        return fs.lib().fs_encode_static(code._h, d, p, c, None, stream)

    d, p, c = vp(data.data_ptr()), vp(par.data_ptr()), vp(cod.data_ptr())
    assert call(None, p, c) == fs.FS_ERR_INVALID
    assert call(d, p, None) == fs.FS_ERR_INVALID
    assert call(d, None, c) == fs.FS_ERR_INVALID            # the code has parities
    assert call(vp(data.data_ptr() + 1), p, c) == fs.FS_ERR_INVALID
    assert call(d, p, vp(cod.data_ptr() + 8)) == fs.FS_ERR_INVALID
    torch.cuda.synchronize()
    assert call(d, p, c) == fs.FS_OK                         # the same buffers, aligned
    torch.cuda.synchronize()
    code.close()
