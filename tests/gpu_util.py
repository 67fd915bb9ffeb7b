"""Helpers for the GPU tests: device buffers with guard canaries, workspace
allocation and normwise errors.  Inputs come from the seeded generators in
`synth`; expected values come only from the oracle."""
import numpy as np
import torch

import paper_1205_1098_gb300 as bto

GUARD = 64                 # canary elements on each side of an output
CANARY = -1234.5678125     # exactly representable
TOL64 = 1e-12              # FP64 normwise relative tolerance


def dev(a, dtype=torch.float64):
    """Host numpy array (any layout) -> flat device tensor in memory order."""
    a = np.asarray(a)
    flat = a.ravel(order="F") if a.ndim == 2 else a.ravel()
    return torch.from_numpy(np.ascontiguousarray(flat)).to(device="cuda", dtype=dtype)


class Out:
    """A device output buffer of `n` elements between two canary guard bands."""

    def __init__(self, n, dtype=torch.float64, fill=np.nan):
        self.n = n
        self.buf = torch.full((n + 2 * GUARD,), CANARY, dtype=dtype, device="cuda")
        self.t = self.buf[GUARD:GUARD + n]
        if n:
            self.t.fill_(fill)

    def ptr(self):
        return self.t.data_ptr() if self.n else 0

    def host(self):
        g = self.buf.cpu().numpy()
        assert np.all(g[:GUARD] == CANARY) and np.all(g[GUARD + self.n:] == CANARY), "guard band overwritten"
        return g[GUARD:GUARD + self.n].copy()


def ws(op, form, m, n, a_type=0):
    nbytes = bto.bto_workspace_bytes(op, form, m, n, a_type)
    t = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device="cuda")
    t.fill_(0xA5)   # arbitrary content: kernels must not depend on it
    return t, nbytes


def p(t):
    return 0 if t is None or t.numel() == 0 else t.data_ptr()


def relerr(got, ref):
    got, ref = np.asarray(got, np.float64).ravel(), np.asarray(ref, np.float64).ravel()
    if ref.size == 0:
        return 0.0
    nr = np.linalg.norm(ref)
    d = np.linalg.norm(got - ref)
    return d / nr if nr > 0 else d


def sync():
    torch.cuda.synchronize()
