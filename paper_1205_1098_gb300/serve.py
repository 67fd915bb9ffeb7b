"""Serving loop: continuous batching of GEMVER/BiCGK/ATAX/GESUMMV requests.

Requests arrive as a seeded Poisson process.  Each names a kernel, a size n
and a storage type (FP32 or BF16) for its matrix; operands are resident on
the device (the leading n x n block of an 8192 x 8192 matrix of that type, and
prefixes of resident vectors), so no request moves its inputs over the host
link.  The loop:

  * moves arrived requests into a FIFO;
  * admits requests from the head of the FIFO while their outputs (including
    GEMVER's B) plus the batch workspace fit the HBM budget, up to `max_batch`
    per batch, whenever one of `streams` launch slots is free: requests that
    arrive while earlier batches are on the GPU join the next batch
    (continuous batching), and batches on different streams overlap;
  * launches each batch with bto_batch_prepare / bto_batch_run on its stream
    and records an event;
  * polls the events, stamps each finished request's completion time, and
    releases its memory from the budget.

Latency is completion minus arrival (host clock).  Throughput counts each
finished request's compulsory bytes.  All device work runs in libbto's
kernels; this module only schedules.
"""
import collections
import time

import numpy as np
import torch

from . import _lib as L

OPS = ("gemver", "bicgk", "atax", "gesummv")
OPCODE = {"bicgk": 0, "atax": 1, "gemver": 2, "gesummv": 3}
NMAX = 8192
ALPHA, BETA = 1.5, 1.25


def make_trace(seed, rate, duration, nmin=64, nmax=NMAX, count=None):
    """Seeded request trace: arrival times (s), kernel, n, storage type."""
    import synth
    n_req = count if count is not None else int(rate * duration * 1.2) + 16
    k = np.arange(n_req, dtype=np.uint64)
    u = lambda aid: (synth.u64(seed, aid, k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    gaps = -np.log1p(-u(600)) / rate
    t = np.cumsum(gaps)
    ops = (u(601) * len(OPS)).astype(np.int64)
    n = np.round(np.exp(np.log(nmin) + u(602) * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    bf16 = u(603) < 0.5
    if count is None:
        keep = t < duration
        t, ops, n, bf16 = t[keep], ops[keep], n[keep], bf16[keep]
    return [dict(id=i, t=float(t[i]), op=OPS[ops[i]], n=int(n[i]), dtype="bf16" if bf16[i] else "f32")
            for i in range(len(t))]


def compulsory_bytes(op, n, dtype):
    e = 2 if dtype == "bf16" else 4
    mn = n * n
    return {"gemver": 3 * e * mn + 4 * 8 * n, "bicgk": e * mn + 4 * 4 * n,
            "atax": e * mn + 4 * 2 * n, "gesummv": 2 * e * mn + 4 * 2 * n}[op]


class Server:
    def __init__(self, budget_bytes=40e9, streams=4, max_batch=64, tile_cols=256, seed=4, device=None):
        import synth
        self.budget = float(budget_bytes)
        self.used = 0.0
        self.max_batch = max_batch
        self.tile_cols = tile_cols
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        f32 = dict(dtype=torch.float32, device="cuda")
        # Resident operands: two matrices per storage type and the vector pool.
        self.mats = {}
        for t, code in (("f32", 1), ("bf16", 2)):
            dt = torch.float32 if t == "f32" else torch.int16
            mats = []
            for aid in (0, 1):
                a = torch.empty(NMAX * NMAX, dtype=dt, device="cuda")
                (L.bto_fill_f32 if t == "f32" else L.bto_fill_bf16)(seed, 10 * code + aid, 0, NMAX, NMAX, 0, a, NMAX, None)
                mats.append(a)
            self.mats[t] = mats
        self.vecs = []
        for aid in range(6):
            v = torch.empty(NMAX, **f32)
            L.bto_fill_f32(seed, 100 + aid, 0, NMAX, 1, 0, v, NMAX, None)
            self.vecs.append(v)
        torch.cuda.synchronize()

    # ------------------------------------------------------------ requests
    def _outputs(self, r):
        n, op = r["n"], r["op"]
        f32 = dict(dtype=torch.float32, device="cuda")
        outs = {"bicgk": [n, n], "gemver": [n, n], "atax": [n], "gesummv": [n]}[op]
        r["out"] = [torch.empty(ln, **f32) for ln in outs]
        mem = 4.0 * sum(outs)
        if op == "gemver":
            dt = torch.float32 if r["dtype"] == "f32" else torch.int16
            r["B"] = torch.empty(n * n, dtype=dt, device="cuda")
            mem += r["B"].numel() * r["B"].element_size()
        return mem

    def _fill_desc(self, d, r):
        n, op, t = r["n"], r["op"], r["dtype"]
        d.op, d.a_type = OPCODE[op], 1 if t == "f32" else 2
        d.m = d.n = n
        d.lda = d.ldb = NMAX
        d.alpha, d.beta = ALPHA, BETA
        d.A = self.mats[t][0].data_ptr()
        if op == "gesummv":
            d.B = self.mats[t][1].data_ptr()
        elif op == "gemver":
            d.ldb = n
            d.B = r["B"].data_ptr()
        nin = {"bicgk": 2, "gemver": 6, "atax": 1, "gesummv": 1}[op]
        for k in range(nin):
            d.in_[k] = self.vecs[k].data_ptr()
        for k, o in enumerate(r["out"]):
            d.out[k] = o.data_ptr()

    def _launch(self, batch, stream):
        descs = (L.BatchDesc * len(batch))()
        for d, r in zip(descs, batch):
            self._fill_desc(d, r)
        nb = L.bto_batch_workspace_bytes(descs, self.tile_cols)
        ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            L.bto_batch_prepare(len(batch), descs, self.tile_cols, ws, nb, stream)
            L.bto_batch_run(ws, nb, stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return ws, nb, ev

    # ------------------------------------------------------------ the loop
    def run(self, trace, keep_results=False, max_wall=None):
        """Serves `trace`; returns stats and, if asked, every request's outputs."""
        torch.cuda.synchronize()
        pending = collections.deque()
        waiting = collections.deque(trace)
        inflight = []            # (requests, ws, ws_bytes, event, stream index)
        free = list(range(len(self.streams)))
        done, nbytes, batches, peak = [], 0, 0, 0.0
        t0 = time.perf_counter()
        deadline = None if max_wall is None else t0 + max_wall
        while waiting or pending or inflight:
            now = time.perf_counter() - t0
            while waiting and waiting[0]["t"] <= now:
                pending.append(waiting.popleft())
            # Completions.
            still = []
            for (reqs, ws, wsb, ev, si) in inflight:
                if ev.query():
                    tc = time.perf_counter() - t0
                    for r in reqs:
                        r["done"] = tc
                        nbytes += compulsory_bytes(r["op"], r["n"], r["dtype"])
                        self.used -= r["mem"]
                        if not keep_results:
                            r.pop("out", None)
                            r.pop("B", None)
                        done.append(r)
                    self.used -= wsb
                    r0 = reqs[0]
                    r0.setdefault("_status", L.bto_device_status(ws, self.streams[si]))
                    free.append(si)
                else:
                    still.append((reqs, ws, wsb, ev, si))
            inflight = still
            # Admission into a new batch on a free stream.
            if free and pending:
                batch = []
                while pending and len(batch) < self.max_batch:
                    r = pending[0]
                    need = 4.0 * 6 * r["n"] + (r["n"] * r["n"] * (2 if r["dtype"] == "bf16" else 4)
                                              if r["op"] == "gemver" else 0) + 64e6
                    if self.used + need > self.budget and (batch or inflight):
                        break            # wait for memory to free up
                    # (a request larger than the whole budget runs alone when nothing else is admitted)
                    pending.popleft()
                    r["mem"] = self._outputs(r)
                    self.used += r["mem"]
                    peak = max(peak, self.used)
                    r["admit"] = time.perf_counter() - t0
                    batch.append(r)
                if batch:
                    si = free.pop()
                    ws, wsb, ev = self._launch(batch, self.streams[si])
                    self.used += wsb
                    peak = max(peak, self.used)
                    inflight.append((batch, ws, wsb, ev, si))
                    batches += 1
            elif not inflight and not pending and waiting:
                # Idle until the next arrival.
                wait = waiting[0]["t"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-4))
            if deadline is not None and time.perf_counter() > deadline:
                break
        wall = time.perf_counter() - t0
        lat = np.array([r["done"] - r["t"] for r in done]) if done else np.zeros(1)
        status = [r["_status"] for r in done if "_status" in r]
        return {
            "requests": len(done), "batches": batches, "wall_s": wall,
            "offered_rate": len(trace) / max(trace[-1]["t"], 1e-9) if trace else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "gbs": nbytes / wall / 1e9,
            "status_ok": all(s == 0 for s in status), "peak_bytes": peak, "budget_bytes": self.budget,
        }, done
