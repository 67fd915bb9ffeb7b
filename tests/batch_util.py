"""Builds seeded batches of BICGK/GEMVER instances for the batched form."""
import ctypes

import numpy as np
import torch

import paper_1205_1098_gb300 as bto
import synth

OP = {"bicgk": 0, "gemver": 2}


class Batch:
    """Host copies of every instance's inputs, device buffers and descriptors."""

    def __init__(self, specs, seed=7, kind=synth.KIND_UNIFORM):
        # specs: list of (op, m, n, lda) ; ldb = lda
        self.specs = specs
        self.descs = (bto.BatchDesc * len(specs))()
        self.keep, self.host, self.outs = [], [], []
        for i, (op, m, n, lda) in enumerate(specs):
            base = 1000 * i
            A = synth.to_f32(np.nan_to_num(synth.matrix(seed, base, m, n, lda=lda, kind=kind), nan=0.0))
            d = self.descs[i]
            d.op, d.m, d.n, d.lda, d.ldb = OP[op], m, n, lda, lda
            d.alpha, d.beta = 1.5, 1.25
            dA = torch.from_numpy(np.ascontiguousarray(A.ravel(order="F"))).cuda()
            d.A = dA.data_ptr() if dA.numel() else 0
            self.keep.append(dA)
            lens = [n, m] if op == "bicgk" else [m, n, m, n, m, n]
            ins = []
            for k, ln in enumerate(lens):
                v = synth.to_f32(synth.vector(seed, base + 1 + k, ln, kind))
                t = torch.from_numpy(v).cuda()
                self.keep.append(t)
                d.in_[k] = t.data_ptr() if ln else 0
                ins.append(v)
            olen = [m, n] if op == "bicgk" else [n, m]
            outs = []
            for k, ln in enumerate(olen):
                t = torch.full((max(ln, 1),), np.nan, dtype=torch.float32, device="cuda")
                self.keep.append(t)
                d.out[k] = t.data_ptr() if ln else 0
                outs.append((t, ln))
            B = None
            if op == "gemver":
                B = torch.full((max(lda * n, 1),), np.nan, dtype=torch.float32, device="cuda")
                self.keep.append(B)
                d.B = B.data_ptr() if lda * n else 0
            self.host.append((A, ins))
            self.outs.append((outs, B))

    def run(self, tile_cols=0, graph=False, reps=1):
        nb = bto.bto_batch_workspace_bytes(self.descs, tile_cols)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        self.ws = ws
        bto.bto_batch_prepare(len(self.specs), self.descs, tile_cols, ws, nb, None)
        if graph:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                bto.bto_batch_run(ws, nb, s)   # warm-up outside the capture
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                bto.bto_batch_run(ws, nb, torch.cuda.current_stream())
            for _ in range(reps):
                g.replay()
        else:
            for _ in range(reps):
                bto.bto_batch_run(ws, nb, None)
        torch.cuda.synchronize()
        return bto.bto_device_status(ws)

    def result(self, i):
        (outs, B) = self.outs[i]
        op, m, n, lda = self.specs[i]
        res = [t.cpu().numpy()[:ln].astype(np.float64) for (t, ln) in outs]
        if op == "gemver":
            Bh = B.cpu().numpy()[:lda * n].reshape(n, lda).T[:m].astype(np.float64) if n else np.zeros((m, 0))
            res.append(Bh)
        return res


def logu_sizes(seed, count, lo=32, hi=2048):
    u = synth.vector(seed, 500, 2 * count) * 0.5 + 0.5
    sizes = np.round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    ops = np.where(synth.vector(seed, 501, count) < 0, "bicgk", "gemver")
    return [(ops[i], int(sizes[2 * i]), int(sizes[2 * i + 1])) for i in range(count)]
