"""Helpers for the GPU tests: device buffers (torch supplies memory and the
stream), host<->device copies of uint32 data, and workspaces."""
from __future__ import annotations

import numpy as np
import torch

SENTINEL = 0xDEADBEEF


def dev():
    return torch.device("cuda", 0)


def to_dev(x: np.ndarray, pad: int = 0) -> torch.Tensor:
    """uint32 numpy -> device int32 tensor (bit copy), with `pad` extra slots."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    t = torch.empty(x.size + pad, dtype=torch.int32, device=dev())
    if x.size:
        t[: x.size].copy_(torch.from_numpy(x.view(np.int32)))
    if pad:
        t[x.size:].fill_(np.int32(np.uint32(SENTINEL).view(np.int32)))
    return t


def empty(n: int, fill=SENTINEL) -> torch.Tensor:
    t = torch.empty(max(n, 1), dtype=torch.int32, device=dev())
    t.fill_(int(np.uint32(fill).view(np.int32)))
    return t


def to_host(t: torch.Tensor, n: int | None = None) -> np.ndarray:
    a = t.detach().cpu().numpy().view(np.uint32)
    return a if n is None else a[:n]


def word(t: torch.Tensor, i: int = 0) -> int:
    return int(np.int32(t[i].item()).view(np.uint32))


def stream():
    return torch.cuda.current_stream().cuda_stream


class Workspace:
    """Device workspace for the single-pass kernels (256-byte aligned)."""

    def __init__(self, ka, capacity: int, tile=None, batch_items: int | None = None):
        if batch_items is None:
            s, nbytes = ka.ka_workspace_size(capacity, tile)
        else:
            s, nbytes = ka.ka_batch_workspace_size(batch_items, capacity, tile)
        assert s == 0, s
        self.nbytes = nbytes
        self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev())
        base = self.buf.data_ptr()
        self.ptr = (base + 255) // 256 * 256
        assert ka.ka_workspace_init(self.ptr, nbytes, stream()) == 0

    def status(self, ka):
        s, dev_status = ka.ka_workspace_status(self.ptr, stream())
        assert s == 0
        return dev_status

    def header_words(self):
        off = self.ptr - self.buf.data_ptr()
        return self.buf[off: off + 256].view(torch.int64)
