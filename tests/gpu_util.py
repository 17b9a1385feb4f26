"""Helpers for the GPU parity tests: device buffers with canaries, error bounds."""

import numpy as np

CANARY = 64  # elements of sentinel before and after each output buffer


def torch_dtype(np_dtype):
    import torch
    return torch.float64 if np.dtype(np_dtype) == np.float64 else torch.float32


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class CanaryOut:
    """An output buffer with sentinel elements on both sides (catches tail overruns)."""

    def __init__(self, shape, dtype):
        import torch
        n = int(np.prod(shape))
        self.n = n
        self.buf = torch.full((n + 2 * CANARY,), 12345.0, dtype=torch_dtype(dtype), device="cuda")
        self.out = self.buf[CANARY:CANARY + n].view(*shape)

    def intact(self) -> bool:
        b = self.buf.cpu().numpy()
        return bool(np.all(b[:CANARY] == 12345.0) and np.all(b[CANARY + self.n:] == 12345.0))


def fma_bound(D, u, layout, unit):
    """Per-output bound (N + 2) * unit * sum_j |D[f,i,j]| |u[e,j]| for an N-term FMA chain."""
    import oracle
    N = D.shape[-1]
    mag = oracle.contract(np.abs(np.asarray(D, np.float64)), np.abs(np.asarray(u, np.float64)), layout)
    return (N + 2) * unit * mag + 1e-300
