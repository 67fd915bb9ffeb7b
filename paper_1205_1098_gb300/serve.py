"""Serving: continuous batching of GEMVER/BiCGK/ATAX/GESUMMV requests.

Requests arrive as a seeded Poisson process.  Each names a kernel, a size n
and a storage type (FP32 or BF16) for its matrix; operands are resident on
the device (the leading n x n block of an 8192 x 8192 matrix of that type, and
prefixes of resident vectors), so no request moves its inputs over the host
link.  The scheduling loop is libbto's native bto_serve_run: arrivals join a
FIFO; whenever one of `streams` launch slots is free, the head of the FIFO
is launched, either alone through its single-instance reduced-precision
entry point (n >= `direct_n`: one large matrix spread over every SM) or as a
batch of up to `max_batch` requests through the batched form (continuous
batching: requests that arrive while earlier launches run join the next
one, and launches on different slots overlap); outputs, GEMVER's B and the
workspaces come from a device arena of `budget_bytes` (the HBM budget),
and admission waits while they do not fit.  Python's part is the resident
operands, the arena, the trace and the statistics.

Latency is completion minus arrival (the loop's clock).  Throughput counts
each finished request's compulsory bytes.
"""
import ctypes
import gc

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
    def __init__(self, budget_bytes=40e9, streams=4, max_batch=64, tile_cols=256, seed=4, device=None,
                 direct_n=1024, staging_bytes=4 << 20):
        self.budget = float(budget_bytes)
        self.max_batch = max_batch
        self.tile_cols = tile_cols
        self.direct_n = direct_n
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
        # The budget is one device arena; plans and status words go through pinned staging.
        self.arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device="cuda")
        self.staging = torch.empty(int(staging_bytes), dtype=torch.uint8, pin_memory=True)
        self._handles = (ctypes.c_void_p * streams)(*[s.cuda_stream for s in self.streams])
        torch.cuda.synchronize()

    def _cfg(self, keep_results, max_wall):
        c = L.ServeCfg()
        for ti, t in enumerate(("f32", "bf16")):
            for k in range(2):
                c.A[ti][k] = self.mats[t][k].data_ptr()
        for k in range(6):
            c.vec[k] = self.vecs[k].data_ptr()
        c.arena, c.arena_bytes = self.arena.data_ptr(), self.arena.numel()
        c.staging, c.staging_bytes = self.staging.data_ptr(), self.staging.numel()
        c.streams, c.nstreams = ctypes.addressof(self._handles), len(self.streams)
        c.nmax, c.direct_n = NMAX, int(self.direct_n or 0)
        c.max_wall = float(max_wall or 0.0)
        c.alpha, c.beta = ALPHA, BETA
        c.max_batch, c.tile_cols, c.keep_results = self.max_batch, self.tile_cols, int(bool(keep_results))
        return c

    def _view(self, off, count, dtype):
        nb = count * torch.empty((), dtype=dtype).element_size()
        return self.arena[off:off + nb].view(dtype).clone()

    def run(self, trace, keep_results=False, max_wall=None):
        """Serves `trace` (requests sorted by arrival time); returns stats and the
        finished requests (with copies of their outputs if `keep_results`).

        Python's cyclic garbage collector is paused for the call: a collection
        over many request records would otherwise delay the next one.
        """
        n_req = len(trace)
        reqs = (L.ServeReq * max(n_req, 1))()
        for i, r in enumerate(trace):
            reqs[i].t, reqs[i].op, reqs[i].n = r["t"], OPCODE[r["op"]], r["n"]
            reqs[i].a_type = L.BTO_F32 if r["dtype"] == "f32" else L.BTO_BF16
        res = (L.ServeRes * max(n_req, 1))()
        stats = L.ServeStats()
        cfg = self._cfg(keep_results, max_wall)
        torch.cuda.synchronize()
        gc_was_on = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            status = L.bto_serve_run(cfg, n_req, reqs, res, stats)
        finally:
            if gc_was_on:
                gc.enable()
        done, nbytes, statuses = [], 0, []
        for i, r in enumerate(trace):
            x = res[i]
            if x.done < 0 or x.status == L.BTO_ERR_BUDGET:
                continue
            d = dict(r, admit=x.admit, done=x.done, direct=bool(x.direct), _status=x.status)
            statuses.append(x.status)
            nbytes += compulsory_bytes(r["op"], r["n"], r["dtype"])
            if keep_results:
                n = r["n"]
                d["out"] = [self._view(x.out[k], n, torch.float32) for k in range(2) if x.out[k] >= 0]
                if r["op"] == "gemver":
                    # n columns of leading dimension n rounded up to 8, returned as n x n
                    ldb = (n + 7) // 8 * 8
                    Bs = self._view(x.out[2], n * ldb, torch.float32 if r["dtype"] == "f32" else torch.int16)
                    d["B"] = Bs.view(n, ldb)[:, :n].contiguous().view(-1)
            done.append(d)
        wall = stats.wall_s
        lat = np.array([d["done"] - d["t"] for d in done]) if done else np.zeros(1)
        return {
            "requests": len(done), "batches": int(stats.batches), "direct": int(stats.direct),
            "rejected": int(stats.rejected), "wall_s": wall,
            "offered_rate": n_req / max(trace[-1]["t"], 1e-9) if trace else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "gbs": nbytes / max(wall, 1e-9) / 1e9,
            "status_ok": status == L.BTO_OK and all(s == 0 for s in statuses),
            "peak_bytes": float(stats.peak_bytes), "budget_bytes": self.budget,
            "loop": {"max_gap_ms": stats.max_gap_s * 1e3, "max_gap_at_s": stats.max_gap_at_s,
                     "max_admit_ms": stats.max_admit_s * 1e3, "max_complete_ms": stats.max_complete_s * 1e3,
                     "max_oversleep_ms": stats.max_oversleep_s * 1e3, "max_fifo": int(stats.max_fifo),
                     "fifo_at_max_gap": int(stats.fifo_at_max_gap), "sleeps": int(stats.sleeps),
                     "blocking_copies": int(stats.blocking_copies), "max_query_ms": stats.max_query_s * 1e3},
            "p99_ms_by_second": _p99_by_second(done),
        }, done


def _p99_by_second(done):
    """99th-percentile latency (ms) of the requests arriving in each whole second."""
    if not done:
        return []
    t = np.array([d["t"] for d in done])
    lat = np.array([d["done"] - d["t"] for d in done])
    out = []
    for s in range(int(t.max()) + 1):
        sel = (t >= s) & (t < s + 1)
        if sel.any():
            out.append(round(float(np.percentile(lat[sel], 99) * 1e3), 3))
    return out
