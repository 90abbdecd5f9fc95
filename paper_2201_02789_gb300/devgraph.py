"""Device copies of a generated CSR graph and its np_csr descriptor (input marshalling)."""
from __future__ import annotations

import numpy as np

from . import nestpar as npb


class DevGraph:
    """A CSR graph (gen.Csr) copied to the GPU, with its np_csr descriptor."""

    def __init__(self, g, device="cuda:0"):
        import torch
        self.g = g
        self.n, self.m = g.n, g.m
        self.row_ptr = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).to(device)
        self.col = torch.from_numpy(np.ascontiguousarray(g.col) if g.m else np.zeros(1, np.int32)).to(device)
        w = g.w if g.w is not None else np.ones(g.m, np.uint32)
        self.w = torch.from_numpy(np.ascontiguousarray(w).view(np.int32) if g.m else np.zeros(1, np.int32)).to(device)
        self.csr = npb.make_csr(self.row_ptr, self.col, self.w, n=g.n, m=g.m)
