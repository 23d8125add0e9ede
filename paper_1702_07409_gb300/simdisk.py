"""The paper's simDisk utility on the GPU: the n coded blocks of a code are
spread over `disks` disks, and every combination of `failures` failed disks
is one erasure pattern whose decoding schedule (Algorithm 5 alone, no
payload) says whether the code tolerates it. All patterns of a sweep run as
batches of symbolic decodes (fs_batch with FS_OP_SCHEDULE), one CTA each."""
from __future__ import annotations

import itertools

import numpy as np

from . import founsure as fs


def disk_of_blocks(n: int, disks: int) -> np.ndarray:
    """Disk of each coded block: the blocks striped over the disks in
    contiguous runs of ceil(n / disks) (the last disk may hold fewer)."""
    q = -(-n // disks)
    return np.arange(n) // q


def failure_patterns(n: int, disks: int, failures: int, disk_of=None):
    """(combos, flags): every combination of `failures` failed disks, in
    lexicographic order, and the erasure flags (len(combos) x n, uint8) of
    the coded blocks each one loses."""
    disk_of = disk_of_blocks(n, disks) if disk_of is None else np.asarray(disk_of)
    combos = list(itertools.combinations(range(disks), failures))
    flags = np.zeros((len(combos), n), np.uint8)
    for i, c in enumerate(combos):
        flags[i] = np.isin(disk_of, c)
    return combos, flags


class SimDisk:
    """Failure sweeps of one code (its graph) over `disks` disks. The code is
    created with 16-byte blocks: the schedule does not depend on the block
    size, and its workspace stays small."""

    def __init__(self, graph, disks: int, disk_of=None, max_batch: int = 1024, device=None):
        import torch
        self.torch = torch
        self.graph = graph
        self.disks = disks
        self.disk_of = disk_of
        self.max_batch = max_batch
        self.device = device or torch.device("cuda")
        self.code = fs.Code(graph, 16)
        self.ws_bytes = self.code.workspace_bytes(fs.OP_DECODE)

    def schedule(self, flags: np.ndarray, stream=None):
        """Symbolic decodes of the erasure patterns flags (P x n). Returns
        (n_unrecovered (P,), unrecovered flags (P, k_int))."""
        torch = self.torch
        code, n, k = self.code, self.code.n, self.code.k_int
        P = flags.shape[0]
        nun_all = np.zeros(P, np.int32)
        unrec_all = np.zeros((P, k), np.uint8)
        for c0 in range(0, P, self.max_batch):
            c1 = min(P, c0 + self.max_batch)
            m = c1 - c0
            d_er = torch.from_numpy(np.ascontiguousarray(flags[c0:c1])).to(self.device)
            unrec = torch.empty((m, k), dtype=torch.uint8, device=self.device)
            nun = torch.empty(m, dtype=torch.int32, device=self.device)
            ws = torch.empty((m, self.ws_bytes), dtype=torch.uint8, device=self.device)
            stripes = [{"code": code, "erased": d_er.data_ptr() + i * n,
                        "unrecovered": unrec.data_ptr() + i * k,
                        "n_unrecovered": nun.data_ptr() + 4 * i,
                        "ws": ws.data_ptr() + i * self.ws_bytes} for i in range(m)]
            b = fs.Batch(stripes, fs.OP_SCHEDULE)
            b.run(stream)
            torch.cuda.synchronize()
            nun_all[c0:c1] = nun.cpu().numpy()
            unrec_all[c0:c1] = unrec.cpu().numpy()
            b.close()
        return nun_all, unrec_all

    def run(self, failures: int) -> dict:
        """Every combination of `failures` failed disks: the combinations,
        each one's unrecovered-intermediate count, and the fraction the code
        tolerates (nothing unrecovered)."""
        combos, flags = failure_patterns(self.code.n, self.disks, failures, self.disk_of)
        nun, _ = self.schedule(flags)
        return {"combos": combos, "n_unrecovered": nun,
                "tolerated": float(np.mean(nun == 0)) if len(combos) else 1.0}
