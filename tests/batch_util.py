"""Builds seeded batches of BICGK/GEMVER/ATAX/GESUMMV instances for the
batched form, and recomputes each instance with the oracle."""
import numpy as np
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth

OP = {"bicgk": 0, "atax": 1, "gemver": 2, "gesummv": 3}
ALPHA, BETA = 1.5, 1.25


def _stored(a64, t):
    """FP64 array -> (numpy storage array, FP64 value of the stored numbers)."""
    if t == "f32":
        q = synth.to_f32(a64)
        return q, q.astype(np.float64)
    bits = synth.to_bf16_bits(a64)
    return bits, synth.bf16_bits_to_f64(bits)


def _dev_stored(q, t):
    flat = np.ascontiguousarray(q.ravel(order="F") if q.ndim == 2 else q)
    return torch.from_numpy(flat if t == "f32" else flat.view(np.int16)).cuda()


def _host_stored(tensor, t):
    a = tensor.cpu().numpy()
    return a.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(a.view(np.uint16))


class Batch:
    """Host copies of every instance's inputs, device buffers and descriptors.

    specs: list of (op, m, n, lda) or (op, m, n, lda, dtype) with dtype 'f32' or 'bf16'."""

    def __init__(self, specs, seed=7, kind=synth.KIND_UNIFORM):
        self.specs = [tuple(s) + ("f32",) if len(s) == 4 else tuple(s) for s in specs]
        self.descs = (bto.BatchDesc * len(self.specs))()
        self.keep, self.host, self.outs = [], [], []
        for i, (op, m, n, lda, t) in enumerate(self.specs):
            base = 1000 * i
            d = self.descs[i]
            d.op, d.a_type, d.m, d.n, d.lda, d.ldb = OP[op], (1 if t == "f32" else 2), m, n, lda, lda
            d.alpha, d.beta = ALPHA, BETA
            A64 = np.nan_to_num(synth.matrix(seed, base, m, n, lda=lda, kind=kind), nan=0.0)
            Aq, Ad = _stored(A64, t)
            dA = _dev_stored(Aq, t)
            d.A = dA.data_ptr() if dA.numel() else 0
            self.keep.append(dA)
            B2d = None
            if op == "gesummv":
                B64 = np.nan_to_num(synth.matrix(seed, base + 50, m, n, lda=lda, kind=kind), nan=0.0)
                Bq, B2d = _stored(B64, t)
                dB = _dev_stored(Bq, t)
                d.B = dB.data_ptr() if dB.numel() else 0
                self.keep.append(dB)
            lens = {"bicgk": [n, m], "gemver": [m, n, m, n, m, n], "atax": [n], "gesummv": [n]}[op]
            ins = []
            for k, ln in enumerate(lens):
                v = synth.to_f32(synth.vector(seed, base + 1 + k, ln, kind))
                tv = torch.from_numpy(v).cuda()
                self.keep.append(tv)
                d.in_[k] = tv.data_ptr() if ln else 0
                ins.append(v.astype(np.float64))
            olen = {"bicgk": [m, n], "gemver": [n, m], "atax": [n], "gesummv": [m]}[op]
            outs = []
            for k, ln in enumerate(olen):
                to = torch.full((max(ln, 1),), np.nan, dtype=torch.float32, device="cuda")
                self.keep.append(to)
                d.out[k] = to.data_ptr() if ln else 0
                outs.append((to, ln))
            Bout = None
            if op == "gemver":
                Bout = torch.zeros(max(lda * n, 1), dtype=torch.float32 if t == "f32" else torch.int16, device="cuda")
                self.keep.append(Bout)
                d.B = Bout.data_ptr() if lda * n else 0
            self.host.append((Ad[:m] if m else np.zeros((1, n)), B2d[:m] if B2d is not None and m else None, ins, A64[:m]))
            self.outs.append((outs, Bout))

    def submit(self, tile_cols=0, staging=None):
        """One bto_batch_submit call (plan, copy and launch), through `staging`
        (pinned host memory) when given."""
        nb = bto.bto_batch_workspace_bytes(self.descs, tile_cols)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        ws.fill_(0xA5)
        self.ws = ws
        sb = 0 if staging is None else staging.numel()
        bto.bto_batch_submit(len(self.specs), self.descs, tile_cols, ws, nb, staging, sb, None)
        torch.cuda.synchronize()
        return bto.bto_device_status(ws)

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
        (outs, Bout) = self.outs[i]
        op, m, n, lda, t = self.specs[i]
        res = [to.cpu().numpy()[:ln].astype(np.float64) for (to, ln) in outs]
        if op == "gemver":
            res.append(_host_stored(Bout, t)[:lda * n].reshape(n, lda).T[:m] if n else np.zeros((m, 0)))
        return res

    def reference(self, i):
        """Oracle results for instance i on its stored values.  GEMVER's x and w
        are recomputed from the returned B (formed in FP32 on the device)."""
        op, m, n, lda, t = self.specs[i]
        Ad, B2d, v, _ = self.host[i]
        if op == "bicgk":
            return list(O.bicgk(m, n, Ad, v[0], v[1]))
        if op == "atax":
            return [O.atax(m, n, BETA, Ad, v[0])]
        if op == "gesummv":
            return [O.gesummv(m, n, ALPHA, Ad, BETA, B2d if B2d is not None else np.zeros((1, n)), v[0])]
        Bex, _, _ = O.gemver(m, n, ALPHA, BETA, Ad, *v)
        Bret = self.result(i)[2]
        zm, zn = np.zeros(m), np.zeros(n)
        _, xo, wo = O.gemver(m, n, ALPHA, BETA, Bret if m else np.zeros((1, n)), zm, zn, zm, zn, v[4], v[5])
        return [xo, wo, Bex]

    def b_bound_ok(self, i):
        """GEMVER's B: within one storage ulp plus the FP32 evaluation error."""
        op, m, n, lda, t = self.specs[i]
        Ad, _, v, _ = self.host[i]
        Bret, Bex = self.result(i)[2], self.reference(i)[2]
        ulp = np.spacing(np.abs(Bex).astype(np.float32)).astype(np.float64) * (2.0 ** 16 if t == "bf16" else 1.0)
        mag = np.abs(Ad[:m]) + np.abs(np.outer(v[0], v[1])) + np.abs(np.outer(v[2], v[3]))
        return bool(np.all(np.abs(Bret - Bex) <= ulp + 2.0 ** -23 * mag))


def logu_sizes(seed, count, lo=32, hi=2048, ops=("bicgk", "gemver")):
    u = synth.vector(seed, 500, 2 * count) * 0.5 + 0.5
    sizes = np.round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    pick = ((synth.vector(seed, 501, count) * 0.5 + 0.5) * len(ops)).astype(np.int64)
    return [(ops[min(p, len(ops) - 1)], int(sizes[2 * i]), int(sizes[2 * i + 1])) for i, p in enumerate(pick)]
