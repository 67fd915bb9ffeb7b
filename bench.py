"""Benchmark: the FP64 kernel suite at n = 16384 (fused), beside its unfused
form, the end-to-end path from pinned host memory, and the oracle on the
host's cores.

One step runs every fused Table I kernel once on resident synthetic inputs:
BICGK, ATAX, GESUMMV, GEMVER, DGEMV and DGEMVT on 16384 x 16384 FP64
column-major matrices (2 GiB each), and AXPYDOT, WAXPBY and VADD on 2^26
element vectors.  `value` is the suite's effective bandwidth: the sum of
each kernel's compulsory bytes (every input read once, every output written
once, GEMVER's B written once and read back once) divided by the step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own replica of the workload (the kernels
do not shard); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MAT = 16384
N_VEC = 1 << 26
SEED = 1
ALPHA, BETA = 1.5, 1.2
FP64_FLOP_PER_CLK_PER_SM = 4.0   # 2 FP64 FMA per clock per SM (the unit's issue rate)
# DFMA throughput measured on this GB300 with a register-only probe (8
# independent chains per thread, 4-8 blocks per SM): 1.91 FMA per clock per SM.
FP64_FMA_PER_CLK_MEASURED = 1.91

KERNELS = ["bicgk", "atax", "gesummv", "gemver", "dgemv", "dgemvt", "axpydot", "waxpby", "vadd"]
MATRIX_KERNELS = KERNELS[:6]
# Launches of our kernels per call (panel pass(es) + combine(s); ATAX: its cooperative kernel + combine).
LAUNCHES = {"bicgk": 2, "atax": 2, "gesummv": 2, "gemver": 4, "dgemv": 2, "dgemvt": 4,
            "axpydot": 2, "waxpby": 1, "vadd": 1}
UNFUSED_LAUNCHES = {"bicgk": 4, "atax": 5, "gesummv": 4, "gemver": 8, "dgemv": 3, "dgemvt": 5,
                    "axpydot": 4, "waxpby": 3, "vadd": 3}


def compulsory_bytes(k, m, n, N):
    e = 8
    return {
        "bicgk": e * m * n + e * (2 * m + 2 * n),
        "atax": e * m * n + e * 2 * n,
        "gesummv": 2 * e * m * n + e * (n + m),
        "gemver": 3 * e * m * n + e * (4 * m + 4 * n),
        "dgemv": e * m * n + e * (n + 2 * m),
        "dgemvt": 2 * e * m * n + e * (2 * m + 2 * n),
        "axpydot": 4 * e * N + e,
        "waxpby": 3 * e * N,
        "vadd": 4 * e * N,
    }[k]


def unfused_bytes(k, m, n, N):
    # Bytes the one-kernel-per-BLAS-call form moves (its own traffic).
    e = 8
    return {
        "bicgk": 2 * e * m * n + e * (2 * m + 2 * n),
        "atax": 2 * e * m * n + e * (2 * m + 4 * n),
        "gesummv": 2 * e * m * n + e * (3 * m + 2 * n),
        "gemver": 8 * e * m * n + e * (6 * m + 6 * n),
        "dgemv": e * m * n + e * (n + 4 * m),
        "dgemvt": 2 * e * m * n + e * (4 * n + 3 * m),
        "axpydot": 7 * e * N + e,
        "waxpby": 7 * e * N,
        "vadd": 8 * e * N,
    }[k]


def flops(k, m, n, N):
    return {"bicgk": 4 * m * n, "atax": 4 * m * n, "gesummv": 4 * m * n, "gemver": 8 * m * n,
            "dgemv": 2 * m * n, "dgemvt": 4 * m * n, "axpydot": 4 * N, "waxpby": 3 * N,
            "vadd": 2 * N}[k]


# DRAM bytes (read + write) per call, from one ncu capture (--set full) of the
# same kernels at n = 8192 on a GB300; traffic grows with m n, so the bench
# scales it to its own size.  Set to None for a kernel changed since then.
# The headline metric and workload, shared by this arm and the reference arm.
METRIC = ("fused FP64 kernel-suite effective HBM bandwidth (GEMVER/BiCGK/ATAX/GESUMMV/DGEMV/DGEMVT at "
          "n=16384, AXPYDOT/WAXPBY/VADD at 2^26) vs unfused")
WORKLOAD = "FP64 kernel suite: 16384x16384 column-major matrices, 2^26-element vectors"
NCU_TRAFFIC_N = 8192
NCU_TRAFFIC = {
    "gemver": (537.580544 + 492.955392) * 1e6 + (537.008128 + 8.569088) * 1e6,
    "atax": (545.888768 + 3.536128) * 1e6,
}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


class Suite:
    """Device buffers and one call per fused (or unfused) kernel."""

    def __init__(self, torch, bto, m=N_MAT, n=N_MAT, N=N_VEC):
        import synth
        self.torch, self.bto = torch, bto
        self.m, self.n, self.N = m, n, N
        f64 = dict(dtype=torch.float64, device="cuda")
        self.A = torch.empty(m * n, **f64)
        self.B2 = torch.empty(m * n, **f64)       # GESUMMV's second matrix
        self.Bout = torch.empty(m * n, **f64)     # GEMVER's B
        bto.bto_fill_f64(SEED, 0, 0, m, n, 0, self.A, m, None)
        bto.bto_fill_f64(SEED, 1, 0, m, n, 0, self.B2, m, None)
        self.vec = {}
        for k, ln, aid in [("p", n, 1), ("r", m, 2), ("x", n, 3), ("ym", m, 4), ("zn", n, 5),
                           ("u1", m, 11), ("v1", n, 12), ("u2", m, 13), ("v2", n, 14),
                           ("gy", m, 15), ("gz", n, 16)]:
            self.vec[k] = torch.empty(ln, **f64)
            bto.bto_fill_f64(SEED, aid, 0, ln, 1, 0, self.vec[k], ln, None)
        for k, ln in [("q", m), ("s", n), ("y_atax", n), ("y_ges", m), ("gx", n), ("gw", m),
                      ("z_dgemv", m), ("tx", n), ("tw", m)]:
            self.vec[k] = torch.empty(ln, **f64)
        self.big = {}
        for k, aid in [("w", 20), ("v", 21), ("u", 22), ("xx", 23), ("yy", 24), ("zz", 25)]:
            self.big[k] = torch.empty(N, **f64)
            bto.bto_fill_f64(SEED, aid, 0, N, 1, 0, self.big[k], N, None)
        for k in ("z_ax", "w_wx", "x_va"):
            self.big[k] = torch.empty(N, **f64)
        self.r = torch.empty(1, **f64)
        self.ws = {}
        for form in (0, 1, 2, 3):
            ks = KERNELS if form < 2 else [k for k in KERNELS if k in MATRIX_KERNELS]
            if not ks:
                continue
            size = max(bto.bto_workspace_bytes(k, form, m if k in MATRIX_KERNELS else 0,
                                               n if k in MATRIX_KERNELS else N) for k in ks)
            self.ws[form] = (torch.empty(size, dtype=torch.uint8, device="cuda"), size)
        torch.cuda.synchronize()

    def call(self, k, form=0):
        """form 0 fused, 1 unfused, 2 double-float fused, 3 double-float unfused
        (the vector kernels have no double-float form and run as forms 0 / 1)."""
        b, v, g, m, n, N = self.bto, self.vec, self.big, self.m, self.n, self.N
        if form >= 2 and k in MATRIX_KERNELS:
            df = {"bicgk": "bicgk", "atax": "atax", "gesummv": "gesummv", "gemver": "gemver", "dgemv": "dgemv",
                  "dgemvt": "dgemvt"}[k]
            f = getattr(b, ("bto_unfused_%s_df" if form == 3 else "bto_%s_df") % df)
            ws, wb = self.ws[form]
            return self._matrix_call(k, f, ws, wb)
        form = form - 2 if form >= 2 else form
        ws, wb = self.ws[form]
        u = form == 1
        if k == "bicgk":
            (b.bto_unfused_bicgk if u else b.bto_bicgk)(m, n, self.A, m, v["p"], v["r"], v["q"], v["s"], ws, wb, None)
        elif k == "atax":
            (b.bto_unfused_atax if u else b.bto_atax)(m, n, BETA, self.A, m, v["x"], v["y_atax"], ws, wb, None)
        elif k == "gesummv":
            (b.bto_unfused_gesummv if u else b.bto_gesummv)(m, n, ALPHA, self.A, m, -0.75, self.B2, m, v["x"],
                                                            v["y_ges"], ws, wb, None)
        elif k == "gemver":
            (b.bto_unfused_gemver if u else b.bto_gemver)(m, n, ALPHA, BETA, self.A, m, v["u1"], v["v1"], v["u2"],
                                                          v["v2"], v["gy"], v["gz"], self.Bout, m, v["gx"],
                                                          v["gw"], ws, wb, None)
        elif k == "dgemv":
            (b.bto_unfused_dgemv if u else b.bto_dgemv)(m, n, ALPHA, self.A, m, v["x"], -0.5, v["ym"],
                                                        v["z_dgemv"], ws, wb, None)
        elif k == "dgemvt":
            (b.bto_unfused_dgemvt if u else b.bto_dgemvt)(m, n, ALPHA, BETA, self.A, m, v["ym"], v["zn"],
                                                          v["tx"], v["tw"], ws, wb, None)
        elif k == "axpydot":
            (b.bto_unfused_axpydot if u else b.bto_axpydot)(N, 0.75, g["w"], g["v"], g["u"], g["z_ax"], self.r,
                                                            ws, wb, None)
        elif k == "waxpby":
            (b.bto_unfused_waxpby if u else b.bto_waxpby)(N, ALPHA, g["xx"], -0.25, g["yy"], g["w_wx"], None)
        elif k == "vadd":
            (b.bto_unfused_vadd if u else b.bto_vadd)(N, g["w"], g["yy"], g["zz"], g["x_va"], None)


def _matrix_call(self, k, f, ws, wb):
    m, n, v = self.m, self.n, self.vec
    if k == "bicgk":
        f(m, n, self.A, m, v["p"], v["r"], v["q"], v["s"], ws, wb, None)
    elif k == "atax":
        f(m, n, BETA, self.A, m, v["x"], v["y_atax"], ws, wb, None)
    elif k == "gesummv":
        f(m, n, ALPHA, self.A, m, -0.75, self.B2, m, v["x"], v["y_ges"], ws, wb, None)
    elif k == "gemver":
        f(m, n, ALPHA, BETA, self.A, m, v["u1"], v["v1"], v["u2"], v["v2"], v["gy"], v["gz"], self.Bout, m,
          v["gx"], v["gw"], ws, wb, None)
    elif k == "dgemv":
        f(m, n, ALPHA, self.A, m, v["x"], -0.5, v["ym"], v["z_dgemv"], ws, wb, None)
    elif k == "dgemvt":
        f(m, n, ALPHA, BETA, self.A, m, v["ym"], v["zn"], v["tx"], v["tw"], ws, wb, None)


Suite._matrix_call = _matrix_call

# Array ids of the suite's device fills (bto_fill_f64 with seed SEED).
SUITE_AIDS = {"A": 0, "B2": 1, "p": 1, "r": 2, "x": 3, "ym": 4, "zn": 5, "u1": 11, "v1": 12, "u2": 13, "v2": 14,
              "gy": 15, "gz": 16}


def sampled_errors(suite, nsamp=16):
    """Normwise relative error of sampled outputs of the matrix kernels the
    suite last ran, against FP64 products computed with numpy from the
    generator's rows and columns (rows of A for A v, columns for A^T v;
    GEMVER's x_j from column j of B = A + u1 v1^T + u2 v2^T)."""
    import synth
    m, n = suite.m, suite.n
    vec = {k: synth.vector(SEED, SUITE_AIDS[k], m if k in ("r", "ym", "u1", "u2", "gy") else n)
           for k in ("p", "r", "x", "ym", "zn", "u1", "v1", "u2", "v2", "gy", "gz")}
    host = {k: suite.vec[k].cpu().numpy() for k in ("q", "s", "y_ges", "z_dgemv", "tx", "gx")}
    I = np.unique(np.linspace(0, m - 1, nsamp).astype(np.int64))
    J = np.unique(np.linspace(0, n - 1, nsamp).astype(np.int64))
    RA, RB = synth.matrix_rows(SEED, 0, m, n, I), synth.matrix_rows(SEED, 1, m, n, I)
    CA = synth.matrix_cols(SEED, 0, m, n, J)

    def rel(g, o):
        g, o = np.asarray(g), np.asarray(o)
        return float(np.linalg.norm(g - o) / np.linalg.norm(o))

    CB = CA + np.outer(vec["u1"], vec["v1"][J]) + np.outer(vec["u2"], vec["v2"][J])
    return {"bicgk_q": rel(host["q"][I], RA @ vec["p"]), "bicgk_s": rel(host["s"][J], CA.T @ vec["r"]),
            "gesummv_y": rel(host["y_ges"][I], ALPHA * (RA @ vec["x"]) - 0.75 * (RB @ vec["x"])),
            "dgemv_z": rel(host["z_dgemv"][I], ALPHA * (RA @ vec["x"]) - 0.5 * vec["ym"][I]),
            "dgemvt_x": rel(host["tx"][J], BETA * (CA.T @ vec["ym"]) + vec["zn"][J]),
            "gemver_x": rel(host["gx"][J], BETA * (CB.T @ vec["gy"]) + vec["gz"][J]),
            "reference": "FP64 products (numpy) from the generator's rows and columns",
            "samples": "%d rows and %d columns, evenly spaced" % (len(I), len(J))}


def df_form(torch, suite, steps, warmup, dist, hbm, kern64):
    """The double-float form of the matrix kernels (bto_*_df) beside its
    unfused form (bto_unfused_*_df), inside the same suite step (the vector
    kernels run their FP64 forms)."""
    m, n, N = suite.m, suite.n, suite.N
    ms, kern = timed_steps(torch, suite, steps, warmup, 2, dist)
    spread = dict(timed_steps.spread)
    errs = sampled_errors(suite)
    ums, ukern = timed_steps(torch, suite, steps, max(3, warmup // 2), 3, dist)
    per = {}
    for k in MATRIX_KERNELS:
        t = kern[k] * 1e-3
        gbs = compulsory_bytes(k, m, n, N) / t / 1e9
        med, p10, p90 = spread[k]
        per[k] = {"ms": round(kern[k], 4), "ms_p10": round(p10, 4), "ms_p90": round(p90, 4),
                  "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3),
                  "unfused_ms": round(ukern[k], 4),
                  "unfused_own_gbs": round(unfused_bytes(k, m, n, N) / (ukern[k] * 1e-3) / 1e9, 1),
                  "fused_speedup": round(ukern[k] / kern[k], 3),
                  "byte_ratio": round(unfused_bytes(k, m, n, N) / compulsory_bytes(k, m, n, N), 3),
                  "speedup_vs_fp64_form": round(kern64[k] / kern[k], 3)}
    dom = max(MATRIX_KERNELS, key=lambda k: kern[k])
    step_bytes = suite_bytes(m, n, N)
    return {"ms_per_step": round(ms, 4), "value": round(step_bytes / (ms * 1e-3) / 1e9, 1),
            "unit": "GB/s of fused compulsory bytes (same suite, matrix kernels in the double-float form)",
            "unfused_ms_per_step": round(ums, 4), "kernels": per, "err_vs_fp64": errs,
            "tolerance": 1e-12,
            "roofline": {"kernel": "bto_%s_df (all launches of one call)" % dom, "bound": "hbm",
                         "achieved": per[dom]["gbs"], "peak": hbm, "unit": "GB/s", "frac": per[dom]["hbm_frac"]}}


def timed_steps(torch, suite, steps, warmup, form, dist, per_kernel=True):
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        for k in KERNELS:
            suite.call(k, form)
    ev = {k: [] for k in KERNELS}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(steps):
        for k in KERNELS:
            if per_kernel:
                a = torch.cuda.Event(enable_timing=True)
                a.record(st)
            suite.call(k, form)
            if per_kernel:
                e = torch.cuda.Event(enable_timing=True)
                e.record(st)
                ev[k].append((a, e))
    t1.record(st)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total = t0.elapsed_time(t1)
    kern = {k: (sum(a.elapsed_time(e) for a, e in ev[k]) / len(ev[k]) if ev[k] else None) for k in KERNELS}
    # Per-kernel spread over the steps (median, p10, p90 in ms).
    spread = {k: tuple(float(v) for v in np.percentile([a.elapsed_time(e) for a, e in ev[k]], [50, 10, 90]))
              for k in KERNELS if ev[k]}
    timed_steps.spread = spread
    return total / steps, kern


def e2e_steps(torch, bto, steps, warmup, m, n, N):
    """Same suite through the public API from pinned host buffers: every step
    copies its inputs host->device, runs the fused kernels and reads every
    output back; copies in both directions overlap the kernels."""
    import synth
    pin = dict(dtype=torch.float64, pin_memory=True)
    hA = torch.empty(m * n, **pin)
    hB = torch.empty(m * n, **pin)
    # host inputs (generated once on the device, then copied into pinned memory)
    tmp = torch.empty(m * n, dtype=torch.float64, device="cuda")
    bto.bto_fill_f64(SEED, 0, 0, m, n, 0, tmp, m, None); hA.copy_(tmp)
    bto.bto_fill_f64(SEED, 1, 0, m, n, 0, tmp, m, None); hB.copy_(tmp)
    del tmp
    hv = {k: torch.from_numpy(synth.vector(SEED, 30 + i, ln)).pin_memory()
          for i, (k, ln) in enumerate([("p", n), ("r", m), ("x", n), ("ym", m), ("zn", n), ("u1", m),
                                       ("v1", n), ("u2", m), ("v2", n), ("gy", m), ("gz", n)])}
    hbig = {}
    for i, k in enumerate(("w", "v", "u", "xx", "yy", "zz")):
        t = torch.empty(N, dtype=torch.float64, device="cuda")
        bto.bto_fill_f64(SEED, 40 + i, 0, N, 1, 0, t, N, None)
        hbig[k] = torch.empty(N, **pin)
        hbig[k].copy_(t)
        del t
    outs_h = {k: torch.empty(ln, **pin) for k, ln in [("q", m), ("s", n), ("y_atax", n), ("y_ges", m),
                                                       ("gx", n), ("gw", m), ("z_dgemv", m), ("tx", n),
                                                       ("tw", m), ("r", 1)]}
    outs_big_h = {k: torch.empty(N, **pin) for k in ("z_ax", "w_wx", "x_va")}
    hBout = torch.empty(m * n, **pin)
    suite = Suite.__new__(Suite)
    suite.torch, suite.bto, suite.m, suite.n, suite.N = torch, bto, m, n, N
    f64 = dict(dtype=torch.float64, device="cuda")
    suite.A, suite.B2, suite.Bout = (torch.empty(m * n, **f64) for _ in range(3))
    suite.vec = {k: torch.empty(t.numel(), **f64) for k, t in hv.items()}
    suite.vec.update({k: torch.empty(t.numel(), **f64) for k, t in outs_h.items() if k != "r"})
    suite.big = {k: torch.empty(N, **f64) for k in list(hbig) + list(outs_big_h)}
    suite.r = torch.empty(1, **f64)
    suite.ws = {}
    size = max(bto.bto_workspace_bytes(k, 0, m if k in MATRIX_KERNELS else 0, n if k in MATRIX_KERNELS else N)
               for k in KERNELS)
    suite.ws[0] = (torch.empty(size, dtype=torch.uint8, device="cuda"), size)
    h2d = hA.numel() * 8 + hB.numel() * 8 + sum(t.numel() * 8 for t in hv.values()) + \
        sum(t.numel() * 8 for t in hbig.values())
    d2h = sum(t.numel() * 8 for t in outs_h.values()) + sum(t.numel() * 8 for t in outs_big_h.values()) + \
        hBout.numel() * 8

    # Copies overlap the kernels: inputs go host->device on their own stream in
    # the order the kernels need them, each kernel waits for its own inputs
    # only, and results go back on a third stream as soon as they exist
    # (GEMVER's 2 GiB B while the other matrix kernels run).  A step's inputs
    # are copied once the previous step's kernels are done with the input
    # buffers, so they overlap the previous step's read-back (the link carries
    # both directions at once); a kernel group overwrites its outputs only
    # after the previous step has read them back.
    sC = torch.cuda.current_stream()
    sH = torch.cuda.Stream()
    sD = torch.cuda.Stream()
    prev = {}

    def rec(stream):
        e = torch.cuda.Event()
        e.record(stream)
        return e

    def after_readback(group):
        if group in prev:
            sC.wait_event(prev[group])

    def step():
        sH.wait_stream(sC)
        with torch.cuda.stream(sH):
            for k, t in hbig.items():
                suite.big[k].copy_(t, non_blocking=True)
            e_big = rec(sH)
            for k, t in hv.items():
                suite.vec[k].copy_(t, non_blocking=True)
            suite.A.copy_(hA, non_blocking=True)
            e_a = rec(sH)
            suite.B2.copy_(hB, non_blocking=True)
            e_b = rec(sH)
        sC.wait_event(e_big)
        after_readback("vector")
        for k in ("axpydot", "waxpby", "vadd"):
            suite.call(k, 0)
        sD.wait_event(rec(sC))
        with torch.cuda.stream(sD):
            for k, t in outs_big_h.items():
                t.copy_(suite.big[k], non_blocking=True)
            outs_h["r"].copy_(suite.r, non_blocking=True)
        prev["vector"] = rec(sD)
        sC.wait_event(e_a)
        after_readback("gemver")
        suite.call("gemver", 0)
        sD.wait_event(rec(sC))
        with torch.cuda.stream(sD):
            hBout.copy_(suite.Bout, non_blocking=True)
            for k in ("gx", "gw"):
                outs_h[k].copy_(suite.vec[k], non_blocking=True)
        prev["gemver"] = rec(sD)
        after_readback("matrix")
        for k in ("bicgk", "atax", "dgemv", "dgemvt"):
            suite.call(k, 0)
        sC.wait_event(e_b)
        suite.call("gesummv", 0)
        sD.wait_event(rec(sC))
        with torch.cuda.stream(sD):
            for k, t in outs_h.items():
                if k not in ("r", "gx", "gw"):
                    t.copy_(suite.vec[k], non_blocking=True)
        prev["matrix"] = rec(sD)

    st = sC
    for _ in range(warmup):
        step()
    sC.wait_stream(sD)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for _ in range(steps):
        step()
    sC.wait_stream(sD)
    t1.record(st)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps, h2d, d2h


def suite_bytes(m, n, N, fn=compulsory_bytes):
    return sum(fn(k, m, n, N) for k in KERNELS)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_SAMPLE_CACHE = {}


def oracle_sample(n_mat, n_vec, reps=1, parallel=False):
    """The oracle suite on the host: returns (seconds, compulsory bytes).
    parallel: the all-core build (OpenMP over independent outputs, bit-equal
    to the serial oracle); else the serial oracle on one thread."""
    import oracle as O
    import synth
    m = n = n_mat
    key = (n_mat, n_vec)
    if key not in _SAMPLE_CACHE:
        _SAMPLE_CACHE.clear()
        _SAMPLE_CACHE[key] = (synth.matrix(SEED, 0, m, n), synth.matrix(SEED, 1, m, n),
                              {k: synth.vector(SEED, i, n)
                               for i, k in enumerate(["p", "r", "x", "y", "z", "u1", "v1", "u2", "v2"])},
                              {k: synth.vector(SEED, 20 + i, n_vec) for i, k in enumerate(["w", "v", "u"])})
    A, B, v, big = _SAMPLE_CACHE[key]
    L = O.lib_par() if parallel else O.lib()
    t = time.perf_counter()
    for _ in range(reps):
        O.bicgk(m, n, A, v["p"], v["r"], L=L)
        O.atax(m, n, BETA, A, v["x"], L=L)
        O.gesummv(m, n, ALPHA, A, -0.75, B, v["x"], L=L)
        O.gemver(m, n, ALPHA, BETA, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"], L=L)
        O.dgemv(m, n, ALPHA, A, v["x"], -0.5, v["y"], L=L)
        O.dgemvt(m, n, ALPHA, BETA, A, v["y"], v["z"], L=L)
        O.axpydot(n_vec, 0.75, big["w"], big["v"], big["u"], L=L)
        O.waxpby(n_vec, ALPHA, big["w"], -0.25, big["v"], L=L)
        O.vadd(n_vec, big["w"], big["v"], big["u"], L=L)
    return time.perf_counter() - t, reps * suite_bytes(m, n, n_vec)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ns, nv = 4096, 1 << 23
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(ns, nv, parallel=True)
    secs, nbytes = 0.0, 0
    for _ in range(args.steps):
        s, b = oracle_sample(ns, nv, parallel=True)
        secs += s
        nbytes += b
    value = nbytes / secs / 1e9
    sample = ("per step: the oracle (plain C, FP64) on all %d host cores (OpenMP over independent outputs, "
              "bit-identical to the serial oracle) on the suite at n=%d matrices and %d-element vectors, "
              "a bounded sample of the n=16384 / 2^26 workload" % (cores, ns, nv))
    print(json.dumps({
        "impl": "reference", "metric": METRIC,
        "value": round(value, 4), "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (SplitMix64 uniform[-1,1), seed 1)",
        "config": {"workload": "FP64 kernel suite sample: %dx%d column-major matrices, %d-element vectors "
                               "(a bounded sample of the 16384x16384 / 2^26 workload)" % (ns, ns, nv),
                   "parallelism": "single"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def precision_form(torch, bto, hbm, steps, n=32768):
    """The reduced-precision storage form at n = 32768 (A in BF16 or FP32):
    time per call (CUDA events), effective bandwidth over its compulsory bytes,
    and sampled normwise errors computed with numpy in FP64, against the
    stored values and against the original FP64 data."""
    import synth
    out = {}
    m = n
    rows = np.linspace(0, m - 1, 16).astype(np.int64)
    f32 = dict(dtype=torch.float32, device="cuda")
    pv = synth.vector(6, 1, n); rv = synth.vector(6, 2, m)
    p32, r32 = synth.to_f32(pv), synth.to_f32(rv)
    dp, dr = torch.from_numpy(p32).cuda(), torch.from_numpy(r32).cuda()
    ids = synth.GEMVER_IDS
    gv = {k: synth.vector(6, ids[k], n) for k in ("u1", "v1", "u2", "v2", "y", "z")}
    g32 = {k: synth.to_f32(v) for k, v in gv.items()}
    dg = {k: torch.from_numpy(v).cuda() for k, v in g32.items()}
    st = torch.cuda.current_stream()

    def deq(a64, t):
        return synth.to_f32(a64).astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(synth.to_bf16_bits(a64))

    def rel(a, b):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    for t, at, es in (("bf16", 2, 2), ("f32", 1, 4)):
        for variant in ("plain", "colscaled"):
            cs = synth.colscale(6, n) if variant == "colscaled" else None
            dcs = torch.from_numpy(cs).cuda() if cs is not None else None
            tdt = torch.float32 if t == "f32" else torch.int16
            A = torch.empty(m * n, dtype=tdt, device="cuda")
            (bto.bto_fill_f32 if t == "f32" else bto.bto_fill_bf16)(6, 0, 0, m, n, dcs, A, m, None)
            q, s_ = torch.empty(m, **f32), torch.empty(n, **f32)
            wb = bto.bto_workspace_bytes("bicgk", 0, m, n, at)
            wsb = torch.empty(wb, dtype=torch.uint8, device="cuda")
            res = {}
            for _ in range(3):
                bto.bto_bicgk_ex(m, n, at, A, m, dp, dr, q, s_, wsb, wb, None)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(); e0.record(st)
            for _ in range(steps):
                bto.bto_bicgk_ex(m, n, at, A, m, dp, dr, q, s_, wsb, wb, None)
            e1.record(st); torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            byts = es * m * n + 4 * (2 * m + 2 * n)
            R64 = synth.matrix_rows(6, 0, m, n, rows, scale=cs)
            C64 = synth.matrix_cols(6, 0, m, n, rows, scale=cs)
            qh, sh = q.cpu().numpy()[rows], s_.cpu().numpy()[rows]
            res["bicgk"] = {"ms": round(ms, 4), "gbs": round(byts / ms / 1e6, 1),
                            "hbm_frac": round(byts / ms / 1e6 / hbm, 3),
                            "err_vs_stored": {"q": rel(qh, deq(R64, t) @ p32.astype(np.float64)),
                                              "s": rel(sh, deq(C64, t).T @ r32.astype(np.float64))},
                            "err_vs_fp64_data": {"q": rel(qh, R64 @ pv), "s": rel(sh, C64.T @ rv)}}
            del wsb
            if variant == "plain":
                B = torch.empty(m * n, dtype=tdt, device="cuda")
                x, w = torch.empty(n, **f32), torch.empty(m, **f32)
                wb = bto.bto_workspace_bytes("gemver", 0, m, n, at)
                wsb = torch.empty(wb, dtype=torch.uint8, device="cuda")
                args = [dg[k] for k in ("u1", "v1", "u2", "v2", "y", "z")]
                for _ in range(3):
                    bto.bto_gemver_ex(m, n, 1.5, 1.2, at, A, m, *args, B, m, x, w, wsb, wb, None)
                torch.cuda.synchronize(); e0.record(st)
                for _ in range(steps):
                    bto.bto_gemver_ex(m, n, 1.5, 1.2, at, A, m, *args, B, m, x, w, wsb, wb, None)
                e1.record(st); torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                byts = 3 * es * m * n + 4 * (4 * m + 4 * n)
                Bcols = B.view(n, m)[torch.from_numpy(rows).cuda()].cpu().numpy()
                Bc = Bcols.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(Bcols.view(np.uint16))
                xall = x.cpu().numpy().astype(np.float64)
                xh = xall[rows]
                xref = 1.2 * (Bc @ g32["y"].astype(np.float64)) + g32["z"][rows].astype(np.float64)
                # w on sampled rows, from the returned B (those rows, every column) and x
                Brows = B.view(n, m)[:, torch.from_numpy(rows).cuda()].cpu().numpy().T
                Br = Brows.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(Brows.view(np.uint16))
                wref = 1.5 * (Br @ xall)
                wh = w.cpu().numpy()[rows]
                Bx64 = (C64 + np.outer(gv["u1"], gv["v1"][rows]) + np.outer(gv["u2"], gv["v2"][rows]))
                x64 = 1.2 * (Bx64.T @ gv["y"]) + gv["z"][rows]
                res["gemver"] = {"ms": round(ms, 4), "gbs": round(byts / ms / 1e6, 1),
                                 "hbm_frac": round(byts / ms / 1e6 / hbm, 3),
                                 "err_vs_stored": {"x": rel(xh, xref), "w": rel(wh, wref)},
                                 "err_vs_fp64_data": {"B": rel(Bc, Bx64.T), "x": rel(xh, x64)}}
                del B, wsb
            del A
            torch.cuda.empty_cache()
            out["%s_%s" % (t, variant)] = res
    return out


def gemver_small(torch, bto, hbm, reps=30, n=2048):
    """GEMVER at n = 2048, FP64 (seed 0, alpha 1.5, beta 1.2): its 32 MiB matrix
    fits in L2, so it is timed warm (back-to-back calls) and cold (a 512 MiB
    write between calls evicts L2).  Median of `reps` calls each."""
    f64 = dict(dtype=torch.float64, device="cuda")
    A, B = torch.empty(n * n, **f64), torch.empty(n * n, **f64)
    bto.bto_fill_f64(0, 0, 0, n, n, 0, A, n, None)
    vec = []
    for aid in range(1, 7):
        v = torch.empty(n, **f64)
        bto.bto_fill_f64(0, aid, 0, n, 1, 0, v, n, None)
        vec.append(v)
    x, w = torch.empty(n, **f64), torch.empty(n, **f64)
    nb = bto.bto_workspace_bytes("gemver", 0, n, n)
    wsb = torch.empty(nb, dtype=torch.uint8, device="cuda")
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()

    def call():
        bto.bto_gemver(n, n, 1.5, 1.2, A, n, *vec, B, n, x, w, wsb, nb, None)

    out = {}
    for mode in ("warm", "cold"):
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        evs = []
        for _ in range(reps):   # all queued, one wait: host launch gaps stay out of the events
            if mode == "cold":
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            call()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
        byts = compulsory_bytes("gemver", n, n, 0)
        out[mode] = {"ms": round(ms, 4), "gbs": round(byts / ms / 1e6, 1), "hbm_frac": round(byts / ms / 1e6 / hbm, 3)}
    out["note"] = ("A, B 32 MiB each: warm runs from L2; cold evicts L2 with a 512 MiB write before every call; "
                   "one cooperative launch (both passes, a bounded grid barrier between them)")
    return out


def schedule_search_form(torch, n=N_MAT, pop=8, gens=5, seed=0):
    """The measured-cost schedule search (f2) on each FP64 matrix kernel at
    n x n: genetic search (seeded with the fused automatic schedule) and
    exhaustive search over the same space, each with its number of distinct
    schedules measured; fitness = median of 5 calls (CUDA events)."""
    from paper_1205_1098_gb300 import schedule_search as S
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for op in S.OPS:
        prob = S.Problem(op, n, n)
        auto = prob.fitness((True, 0, 0))
        ga = S.mfga(op, prob.fitness, sms, pop=pop, gens=gens, seed=seed)
        ex = S.exhaustive(op, prob.fitness, sms)
        name = lambda o: "%s, panels %s, row blocks %s" % ("fused" if o[0] else "unfused", o[1] or "auto", o[2] or "auto")
        out[op] = {"fused_auto_ms": round(auto, 4),
                   "ga": {"best": name(ga["best"]), "ms": round(ga["best_ms"], 4), "evaluations": ga["evaluations"]},
                   "exhaustive": {"best": name(ex["best"]), "ms": round(ex["best_ms"], 4),
                                  "evaluations": ex["evaluations"]}}
        del prob
        torch.cuda.empty_cache()
    return out


def layout_form(torch, bto, fp64_peak, n=N_MAT, reps=7, seed=1):
    """Storage order and transposition (f1) at n x n: each FP64 matrix kernel on
    column-major storage (the ordinary entry point) and on row-major storage
    (bto_*_layout), and DGEMV with and without transposition in both orders.
    Median of `reps` calls after 2 warm-ups (CUDA events); both matrices are
    2 GiB, larger than L2."""
    f64 = dict(dtype=torch.float64, device="cuda")
    A, B, Bo = (torch.empty(n * n, **f64) for _ in range(3))
    bto.bto_fill_f64(seed, 0, 0, n, n, 0, A, n, None)
    bto.bto_fill_f64(seed, 1, 0, n, n, 0, B, n, None)
    v = []
    for aid in range(10, 18):
        t = torch.empty(n, **f64)
        bto.bto_fill_f64(seed, aid, 0, n, 1, 0, t, n, None)
        v.append(t)
    o1, o2 = torch.empty(n, **f64), torch.empty(n, **f64)
    st = torch.cuda.current_stream()
    COL, ROW = bto.BTO_COL_MAJOR, bto.BTO_ROW_MAJOR

    def time(call):
        for _ in range(2):
            call()
        evs = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            call()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    def calls(op, lay, trans, ws, nb):
        if op == "bicgk":
            return lambda: bto.bto_bicgk_layout(lay, n, n, A, n, v[0], v[1], o1, o2, ws, nb)
        if op == "atax":
            return lambda: bto.bto_atax_layout(lay, n, n, 1.25, A, n, v[0], o1, ws, nb)
        if op == "gemver":
            return lambda: bto.bto_gemver_layout(lay, n, n, 1.5, 1.2, A, n, *v[2:8], Bo, n, o1, o2, ws, nb)
        if op == "gesummv":
            return lambda: bto.bto_gesummv_layout(lay, n, n, 1.5, A, n, -0.75, B, n, v[0], o1, ws, nb)
        if op == "dgemv":
            return lambda: bto.bto_dgemv_layout(lay, trans, n, n, 1.5, A, n, v[0], -0.5, v[1], o1, ws, nb)
        return lambda: bto.bto_dgemvt_layout(lay, n, n, 1.5, 1.2, A, n, v[1], v[0], o1, o2, ws, nb)

    out = {}
    cases = [(op, 0) for op in ("bicgk", "atax", "gemver", "gesummv", "dgemvt")] + [("dgemv", 0), ("dgemv", 1)]
    for op, trans in cases:
        row = {}
        for lay, name in ((COL, "col_major"), (ROW, "row_major")):
            nb = bto.bto_layout_workspace_bytes(op, lay, trans, n, n)
            ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
            ms = time(calls(op, lay, trans, ws, nb))
            tf = flops(op, n, n, 0) / ms / 1e9
            row[name] = {"ms": round(ms, 4), "fp64_tflops": round(tf, 4), "fp64_frac": round(tf / fp64_peak, 3)}
            del ws
        out[op + ("_trans" if trans else "")] = row
    out["note"] = ("row-major A is the column-major A^T: BICGK one pass, GEMVER/DGEMVT two, GESUMMV one pass "
                   "per matrix, BATAX two passes (A read twice)")
    del A, B, Bo
    torch.cuda.empty_cache()
    return out


GEN_SPECS = {
    "bicgk": ("in: A : matrix, p r : vector\nout: q s : vector\nq = A * p\ns = A' * r", 4),
    "gemver": ("in: A : matrix, u1 v1 u2 v2 y z : vector, alpha beta : scalar\nout: B : matrix, x w : vector\n"
               "B = A + u1 * v1' + u2 * v2'\nx = beta * B' * y + z\nw = alpha * B * x", 8),
    "batax_row": ("in: x : vector, beta : scalar, A : matrix(row)\nout: y : vector\n"
                  "y = beta * A' * (A * x)", 4),
    "chain": ("in: A C : matrix, p r : vector\nout: q s v : vector\nq = A * p\ns = A' * r\nv = C * q + 2 * s", 6),
}


def generator_form(torch, bto, fp64_peak, n=N_MAT, reps=7, seed=1):
    """Sequences planned by the generator (f3) from their statement form, timed
    as one native program call each at n x n (median of `reps` after 2
    warm-ups), beside the hand-written entry point where there is one.  FLOPs:
    2 per matrix element per product, 4 for GEMVER's update."""
    from paper_1205_1098_gb300 import generator as G
    f64 = dict(dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    def time(call):
        for _ in range(2):
            call()
        evs = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            call()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    out = {}
    for name, (text, fl) in GEN_SPECS.items():
        P = G.compile(text)
        shapes = {k: (n, n) for k, d in P.decls.items() if d[0] == "matrix" and d[2] == "in"}
        bind, aid = {}, 0
        for k, d in sorted(P.decls.items()):
            aid += 1
            if d[0] == "scalar":
                bind[k] = 1.25
            elif d[0] == "matrix":
                bind[k] = torch.empty(n * n, **f64)
                if d[2] == "in":
                    bto.bto_fill_f64(seed, aid, 0, n, n, 0, bind[k], n, None)
            else:
                bind[k] = torch.empty(n, **f64)
                bto.bto_fill_f64(seed, aid, 0, n, 1, 0, bind[k], n, None)
        prog, keep = P.program(bind, shapes)
        nb = bto.bto_program_workspace_bytes(prog)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        ms = time(lambda: bto.bto_program_run(prog, ws, nb, None))
        tf = fl * n * n / ms / 1e9
        row = {"passes": [s["mode"] for s in P.passes], "ms": round(ms, 4), "fp64_tflops": round(tf, 4),
               "fp64_frac": round(tf / fp64_peak, 3)}
        if name in ("bicgk", "gemver"):
            hnb = bto.bto_workspace_bytes(name, 0, n, n)
            hws = torch.empty(hnb, dtype=torch.uint8, device="cuda")
            b = bind
            if name == "bicgk":
                call = lambda: bto.bto_bicgk(n, n, b["A"], n, b["p"], b["r"], b["q"], b["s"], hws, hnb)
            else:
                call = lambda: bto.bto_gemver(n, n, 1.25, 1.25, b["A"], n, b["u1"], b["v1"], b["u2"], b["v2"],
                                              b["y"], b["z"], b["B"], n, b["x"], b["w"], hws, hnb)
            row["hand_written_ms"] = round(time(call), 4)
            del hws
        # The measured-cost choice among every distinct legal fusion plan of
        # the program (the generator's search enumerates them all; Max-Fuse is
        # the first), on the same bindings.
        res = G.search(text, bind, shapes, reps=reps)
        row["fusion_search"] = {
            "choices": [{"policy": pol, "passes": passes, "ms": round(ms, 4)} for pol, passes, ms in res["table"]],
            "best": res["best"], "best_ms": round(res["best_ms"], 4),
            "max_fuse_ms": round(res["table"][0][2], 4),
            "max_fuse_is_best": res["table"][0][0] == res["best"]}
        out[name] = row
        del bind, keep, ws, prog
        torch.cuda.empty_cache()
    return out


def sparse_form(torch, bto, hbm, m=1 << 20, avg=32, reps=7, seed=11):
    """CSR BICGK and BATAX (f4) on a seeded m x m matrix with `avg` entries per
    row on average (synth.csr: uniform row lengths 0..2 avg, uniform random
    columns), median of `reps` calls after 2 warm-ups.  Algorithmic bytes:
    12 per stored entry (value + int32 column), the row pointers, and each
    vector read or written once (BATAX reads the entries twice; its fraction
    is over one read)."""
    import synth
    rp, col, val = synth.csr(seed, 70, m, m, avg)
    nnz = len(col)
    d_rp, d_col, d_val = (torch.from_numpy(a).cuda() for a in (rp, col, val))
    f64 = dict(dtype=torch.float64, device="cuda")
    p, r, q, s = (torch.empty(m, **f64) for _ in range(4))
    bto.bto_fill_f64(seed, 1, 0, m, 1, 0, p, m, None)
    bto.bto_fill_f64(seed, 2, 0, m, 1, 0, r, m, None)
    nb = bto.bto_csr_workspace_bytes("atax", m, m, nnz)
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()

    def time(call):
        for _ in range(2):
            call()
        evs = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            call()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    out = {"m": m, "nnz": nnz, "avg_row": avg}
    base = 12 * nnz + 8 * (m + 1)
    for name, call, vec in (
            ("bicgk", lambda: bto.bto_csr_bicgk(m, m, nnz, d_rp, d_col, d_val, p, r, q, s, ws, nb), 8 * 4 * m),
            ("batax", lambda: bto.bto_csr_atax(m, m, nnz, d_rp, d_col, d_val, 0.75, p, q, ws, nb), 8 * 2 * m)):
        ms = time(call)
        gbs = (base + vec) / ms / 1e6
        out[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3)}
    torch.cuda.synchronize()
    out["status"] = int(ws[:4].view(torch.int32).cpu().numpy()[0])
    del d_rp, d_col, d_val
    torch.cuda.empty_cache()
    return out


def structured_form(torch, bto, hbm, fp64_peak, reps=7):
    """Banded and triangular BICGK and BATAX (f4): an upper triangle of order
    16384 in full storage (the synthetic 16384 x 16384 matrix, seed 1, array
    id 0; entries below the diagonal are never read) and in packed storage
    (entry k of the packed array is value k of array id 0), and a band of
    kl = ku = 32 diagonals at m = n = 2^20 in band storage (ld = 65, filled
    as a 65 x 2^20 matrix, seed 11).  Median of `reps` calls after 2
    warm-ups.  Compulsory bytes: the stored entries once (8 each) and each
    vector once; BATAX reads A twice (two passes), so its fraction of HBM is
    over one read.  Every stored entry costs two FP64 FMAs: the FP64 fraction
    is 4 flops per entry over the derived FP64 peak."""
    st = torch.cuda.current_stream()
    f64 = dict(dtype=torch.float64, device="cuda")

    def time(call):
        for _ in range(2):
            call()
        evs = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            call()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    out = {}
    n = 16384
    cases = [("tri_upper_full_n16384", "tri", 0, n, n, 0, n - 1),
             ("tri_upper_packed_n16384", "tri", 1, n, n, 0, n - 1),
             ("band_kl32_ku32_2e20", "band", bto.BTO_STORE_BAND, 1 << 20, 1 << 20, 32, 32)]
    for name, kind, sto, m, nn, kl, ku in cases:
        if kind == "tri" and sto == 0:
            A = torch.empty(m * nn, **f64)
            bto.bto_fill_f64(1, 0, 0, m, nn, 0, A, m, None)
            ld, entries = m, nn * (nn + 1) // 2
        elif kind == "tri":
            entries = nn * (nn + 1) // 2
            A = torch.empty(entries, **f64)
            bto.bto_fill_f64(1, 0, 0, entries, 1, 0, A, entries, None)
            ld = 1
        else:
            ld = kl + ku + 1
            A = torch.empty(ld * nn, **f64)
            bto.bto_fill_f64(11, 0, 0, ld, nn, 0, A, ld, None)
            entries = sum(min(m, j + kl + 1) - max(0, j - ku) for j in (0, 1, nn - 2, nn - 1)) + (nn - 4) * ld
        p, r, q, s = (torch.empty(max(m, nn), **f64) for _ in range(4))
        bto.bto_fill_f64(1, 1, 0, nn, 1, 0, p, nn, None)
        bto.bto_fill_f64(1, 2, 0, m, 1, 0, r, m, None)
        nb = bto.bto_band_workspace_bytes("atax", m, nn, kl, ku)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        if kind == "tri":
            calls = (("bicgk", lambda: bto.bto_tri_bicgk(0, 0, sto, nn, A, ld, p, r, q, s, ws, nb), 8 * 2 * (m + nn)),
                     ("batax", lambda: bto.bto_tri_atax(0, 0, sto, nn, 0.75, A, ld, p, s, ws, nb), 8 * 2 * nn))
        else:
            calls = (("bicgk", lambda: bto.bto_band_bicgk(sto, m, nn, kl, ku, 0, A, ld, p, r, q, s, ws, nb),
                      8 * 2 * (m + nn)),
                     ("batax", lambda: bto.bto_band_atax(sto, m, nn, kl, ku, 0, 0.75, A, ld, p, s, ws, nb),
                      8 * 2 * nn))
        row = {"m": m, "n": nn, "kl": kl, "ku": ku, "entries": entries}
        for op, call, vec in calls:
            ms = time(call)
            gbs = (8 * entries + vec) / ms / 1e6
            tfl = 4 * entries / ms / 1e9
            row[op] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3),
                       "fp64_tflops": round(tfl, 3), "fp64_frac": round(tfl / fp64_peak, 3)}
        out[name] = row
        del A, ws, p, r, q, s
        torch.cuda.empty_cache()
    out["bound"] = "fp64 (two FMAs per stored entry)"
    return out


def mrhs_form(torch, bto, hbm, steps, n=8192, k=64, seed=6):
    """Multi-right-hand-side BICGK: Q = A P, S = A^T R with A n x n BF16 and
    k BF16 right-hand sides, FP32 Q and S, on the tensor cores.  Each timed
    call is bracketed by CUDA events after an L2 flush (a 512 MiB read), so
    A comes from HBM every time.  Effective bandwidth is over the compulsory
    bytes (A once, P and R once, Q and S written once); the tensor rate is
    4 n^2 k flops over the same time.  Sampled normwise errors are computed
    with numpy in FP64 on the stored BF16 values."""
    import synth
    st = torch.cuda.current_stream()
    A = torch.empty(n * n, dtype=torch.int16, device="cuda")
    bto.bto_fill_bf16(seed, 0, 0, n, n, 0, A, n, None)
    Pb = synth.to_bf16_bits(synth.matrix(seed, 1, n, k)).ravel(order="F")
    Rb = synth.to_bf16_bits(synth.matrix(seed, 2, n, k)).ravel(order="F")
    dP = torch.from_numpy(Pb.view(np.int16).copy()).cuda()
    dR = torch.from_numpy(Rb.view(np.int16).copy()).cuda()
    Q = torch.empty(n * k, dtype=torch.float32, device="cuda")
    S = torch.empty(n * k, dtype=torch.float32, device="cuda")
    wb = bto.bto_bicgk_mrhs_workspace_bytes(n, n, k)
    wsb = torch.empty(wb, dtype=torch.uint8, device="cuda")
    flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")

    def call():
        bto.bto_bicgk_mrhs(n, n, k, A, n, dP, n, dR, n, Q, n, S, n, wsb, wb, None)

    for _ in range(3):
        call()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        flush.sum()            # reads 512 MiB: evicts A without leaving dirty lines in L2
        e0.record(st)
        call()
        e1.record(st)
    torch.cuda.synchronize()
    per_call = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms = float(np.median(per_call))
    ms_mean = float(np.mean(per_call))
    status = bto.bto_device_status(wsb)
    byts = 2 * n * n + 2 * 2 * k * n + 2 * 4 * k * n
    fl = 4.0 * n * n * k
    rows = np.linspace(0, n - 1, 8).astype(np.int64)
    Pq = synth.bf16_bits_to_f64(Pb.reshape(k, n).T)
    Rq = synth.bf16_bits_to_f64(Rb.reshape(k, n).T)
    Ar = synth.bf16_bits_to_f64(synth.to_bf16_bits(synth.matrix_rows(seed, 0, n, n, rows)))
    Ac = synth.bf16_bits_to_f64(synth.to_bf16_bits(synth.matrix_cols(seed, 0, n, n, rows)))
    Qh = Q.view(k, n).T.cpu().numpy()[rows].astype(np.float64)
    Sh = S.view(k, n).T.cpu().numpy()[rows].astype(np.float64)
    qref, sref = Ar @ Pq, Ac.T @ Rq
    del A, flush, wsb
    torch.cuda.empty_cache()
    return {"workload": "A %dx%d BF16, k=%d BF16 right-hand sides, Q/S FP32" % (n, n, k),
            "ms": round(ms, 4), "ms_mean": round(ms_mean, 4), "calls": len(per_call),
            "gbs": round(byts / ms / 1e6, 1), "hbm_frac": round(byts / ms / 1e6 / hbm, 3),
            "tflops": round(fl / ms / 1e9, 1), "compulsory_bytes": byts, "flops": fl, "status": status,
            "l2": "flushed (512 MiB read) before every timed call",
            "sampled_err": {"q": float(np.linalg.norm(Qh - qref) / np.linalg.norm(qref)),
                            "s": float(np.linalg.norm(Sh - sref) / np.linalg.norm(sref))}}


def batched_form(torch, bto, hbm, steps, count=4096, seed=3, tile=0):
    """Config 4: `count` BICGK/GEMVER instances (50/50 by a draw), m, n
    log-uniform in [32, 2048], FP32, one persistent launch, replayed from a
    CUDA graph; the panel width is chosen by the measured-cost tuner."""
    import synth
    from paper_1205_1098_gb300 import autotune
    u = synth.vector(seed, 500, 2 * count) * 0.5 + 0.5
    sizes = np.round(np.exp(np.log(32) + u * (np.log(2048) - np.log(32)))).astype(np.int64)
    ops = np.where(synth.vector(seed, 501, count) < 0, 0, 2)
    descs = (bto.BatchDesc * count)()
    keep = []
    outs = []
    f32 = dict(dtype=torch.float32, device="cuda")
    nbytes = 0
    for i in range(count):
        m, n = int(sizes[2 * i]), int(sizes[2 * i + 1])
        op = int(ops[i])
        d = descs[i]
        lda = (m + 3) // 4 * 4      # columns start on 16 bytes (padded leading dimension)
        d.op, d.a_type, d.m, d.n, d.lda, d.ldb, d.alpha, d.beta = op, 1, m, n, lda, lda, 1.5, 1.25
        A = torch.empty(lda * n, **f32)
        bto.bto_fill_f32(seed, 1000 * i, 0, m, n, 0, A, lda, None)
        keep.append(A)
        d.A = A.data_ptr()
        lens = [n, m] if op == 0 else [m, n, m, n, m, n]
        for k, ln in enumerate(lens):
            t = torch.empty(ln, **f32)
            bto.bto_fill_f32(seed, 1000 * i + 1 + k, 0, ln, 1, 0, t, ln, None)
            keep.append(t)
            d.in_[k] = t.data_ptr()
        o = []
        for k, ln in enumerate([m, n] if op == 0 else [n, m]):
            t = torch.empty(ln, **f32)
            keep.append(t)
            d.out[k] = t.data_ptr()
            o.append(t)
        if op == 2:
            B = torch.empty(lda * n, **f32)
            keep.append(B)
            d.B = B.data_ptr()
            o.append(B)
            nbytes += 3 * 4 * m * n + 4 * (4 * m + 4 * n)
        else:
            nbytes += 4 * m * n + 4 * (2 * m + 2 * n)
        outs.append(o)
    torch.cuda.synchronize()
    if tile:
        best, cand_ms = tile, {}           # profiling runs: a fixed panel width, no tuner
    else:
        best, cand_ms = autotune.tune(descs, use_cache=False)
    nb = bto.bto_batch_workspace_bytes(descs, best)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    bto.bto_batch_prepare(count, descs, best, ws, nb, None)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bto.bto_batch_run(ws, nb, s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bto.bto_batch_run(ws, nb, torch.cuda.current_stream())
    for _ in range(3):
        g.replay()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        g.replay()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    status = bto.bto_device_status(ws)
    one = bto.bto_batch_one_launch(ws)
    # Sampled accuracy: FP64 products (numpy) on the stored FP32 values; GEMVER's x and w from the
    # returned B (x with the returned B, w with the returned B and x).
    f32h = lambda a64: synth.to_f32(a64).astype(np.float64)
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    errs = {"bicgk": [], "gemver": []}
    for i in np.unique(np.linspace(0, count - 1, 32).astype(np.int64)):
        m, n, op = int(sizes[2 * i]), int(sizes[2 * i + 1]), int(ops[i])
        lda = (m + 3) // 4 * 4
        vin = [f32h(synth.vector(seed, 1000 * int(i) + 1 + k, ln))
               for k, ln in enumerate([n, m] if op == 0 else [m, n, m, n, m, n])]
        got = [t.cpu().numpy().astype(np.float64) for t in outs[i]]
        if op == 0:
            A64 = f32h(synth.matrix(seed, 1000 * int(i), m, n))
            errs["bicgk"].append(max(rel(got[0], A64 @ vin[0]), rel(got[1], A64.T @ vin[1])))
        else:
            Bret = got[2][:lda * n].reshape(n, lda).T[:m]
            errs["gemver"].append(max(rel(got[0], 1.25 * (Bret.T @ vin[4]) + vin[5]),
                                      rel(got[1], 1.5 * (Bret @ got[0]))))
    sampled = {"instances": sum(len(v) for v in errs.values()),
               "max_err": {k: (float(max(v)) if v else None) for k, v in errs.items()},
               "reference": "FP64 products (numpy) on the stored FP32 values; GEMVER's x and w from the returned B"}
    return {"instances": count, "ms": round(ms, 4), "gbs": round(nbytes / ms / 1e6, 1),
            "sampled_err": sampled,
            "hbm_frac": round(nbytes / ms / 1e6 / hbm, 3), "compulsory_bytes": nbytes,
            "tile_cols": best, "tuner_ms": {str(k): round(v, 4) for k, v in cand_ms.items()},
            "status": status,
            "launch": ("CUDA graph of bto_batch_run: one cooperative launch (both stages' TMA sweeps and combines, "
                       "bounded grid barriers)" if one else
                       "CUDA graph of bto_batch_run (TMA-path sweeps and combines; fallback kernels)"),
            "layout": "column-major, leading dimension rounded up to a multiple of 4 floats"}


def serving_form(torch, duration=10.0, rate=20000.0, seed=4, runs_n=3):
    """Config 5: Poisson arrivals at `rate` of mixed GEMVER/BiCGK/ATAX/GESUMMV
    requests, n log-uniform in [64, 8192], FP32 or BF16 matrices by a seeded
    flag, resident operands, admission under a 40 GB budget."""
    from paper_1205_1098_gb300.serve import Server, make_trace
    srv = Server(budget_bytes=40e9, streams=4, max_batch=64, tile_cols=256, seed=seed)
    srv.run(make_trace(seed + 1, rate, 0.0, count=200))          # warm-up trace
    trace = make_trace(seed, rate, duration)
    runs = []
    for _ in range(runs_n):
        stats, _ = srv.run(trace, max_wall=duration * 6)
        stats.update({"duration_s": duration, "rate_per_s": rate, "trace_requests": len(trace)})
        runs.append(_rounded(stats))
    out = dict(runs[-1])
    out["runs"] = [{k: r[k] for k in ("p50_ms", "p99_ms", "mean_ms", "gbs", "loop", "p99_ms_by_second")}
                   for r in runs]
    out["sampled_err"] = serving_errors(srv, make_trace(seed + 2, rate, 0.0, nmax=4096, count=200), seed)
    return out


def serving_errors(srv, trace, seed, nsamp=24):
    """Accuracy of served requests: a short trace (n up to 4096) served with
    its outputs kept; every k-th request's outputs against FP64 products
    (numpy) on the stored operands (the leading n x n blocks of the resident
    matrices, dequantized; GEMVER's x and w from the returned B)."""
    import synth
    from paper_1205_1098_gb300.serve import ALPHA, BETA
    stats, done = srv.run(trace, keep_results=True)
    rel = lambda a, b: float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    errs = {}
    for r in done[::max(1, len(done) // nsamp)]:
        n, op, t = r["n"], r["op"], r["dtype"]
        code = 1 if t == "f32" else 2

        def block(aid):
            A = synth.matrix_cols(seed, aid, 8192, 8192, np.arange(n))[:n]
            return synth.to_f32(A).astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(synth.to_bf16_bits(A))
        v = [synth.to_f32(synth.vector(seed, 100 + k, 8192))[:n].astype(np.float64) for k in range(6)]
        got = [o.cpu().numpy().astype(np.float64) for o in r["out"]]
        if op == "gemver":
            Bb = r["B"].cpu().numpy()
            Bret = (Bb.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(Bb.view(np.uint16))).reshape(n, n).T
            xr = BETA * (Bret.T @ v[4]) + v[5]
            e = max(rel(got[0], xr), rel(got[1], ALPHA * (Bret @ xr)))
        else:
            A = block(10 * code)
            if op == "bicgk":
                e = max(rel(got[0], A @ v[0]), rel(got[1], A.T @ v[1]))
            elif op == "atax":
                e = rel(got[0], BETA * (A.T @ (A @ v[0])))
            else:
                e = rel(got[0], ALPHA * (A @ v[0]) + BETA * (block(10 * code + 1) @ v[0]))
        errs.setdefault("%s_%s" % (op, t), []).append(e)
    return {"requests": sum(len(x) for x in errs.values()), "status_ok": bool(stats["status_ok"]),
            "max_err": {k: max(x) for k, x in sorted(errs.items())},
            "reference": "FP64 products (numpy) on the stored operands; GEMVER's x and w from the returned B"}


def _rounded(d):
    if isinstance(d, float):
        return round(d, 4)
    if isinstance(d, dict):
        return {k: _rounded(v) for k, v in d.items()}
    if isinstance(d, list):
        return [_rounded(v) for v in d]
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-df", action="store_true", help="skip the double-float form")
    ap.add_argument("--df-only", action="store_true", help="profiling runs: only the double-float form at --n")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--only", default=None, help="comma-separated kernels (profiling runs)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-only", type=float, default=0.0, help="profiling runs: only serving, for this many s")
    ap.add_argument("--batched-only", action="store_true", help="profiling runs: only the batched form")
    ap.add_argument("--batched-count", type=int, default=4096, help="instances in the batched form")
    ap.add_argument("--batched-tile", type=int, default=0, help="profiling runs: fixed panel width (no tuner)")
    ap.add_argument("--no-search", action="store_true", help="skip the schedule search")
    ap.add_argument("--search-only", type=int, default=0, help="only the schedule search, at this n")
    ap.add_argument("--mrhs-only", type=int, default=0, help="profiling runs: only multi-RHS BICGK with this k")
    ap.add_argument("--no-mrhs", action="store_true")
    ap.add_argument("--no-layout", action="store_true", help="skip the row-major / transposed forms")
    ap.add_argument("--layout-only", action="store_true", help="only the row-major / transposed forms")
    ap.add_argument("--no-generator", action="store_true", help="skip the generated sequences")
    ap.add_argument("--no-sparse", action="store_true", help="skip the CSR forms")
    ap.add_argument("--sparse-only", action="store_true", help="only the CSR forms")
    ap.add_argument("--no-structured", action="store_true", help="skip the banded and triangular forms")
    ap.add_argument("--structured-only", action="store_true", help="only the banded and triangular forms")
    ap.add_argument("--gemver2048-only", action="store_true", help="only GEMVER at n = 2048")
    ap.add_argument("--generator-only", action="store_true", help="only the generated sequences")
    ap.add_argument("--precision-only", type=int, default=0,
                    help="profiling runs: only the reduced-precision form at this n")
    ap.add_argument("--n", type=int, default=N_MAT, help="matrix size (profiling runs)")
    ap.add_argument("--nvec", type=int, default=N_VEC, help="vector length (profiling runs)")
    args = ap.parse_args()
    if args.only:
        global KERNELS
        KERNELS = [k for k in KERNELS if k in args.only.split(",")]
    if args.impl == "reference":
        run_reference(args)
        return
    if args.serving_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        print(json.dumps({"serving": serving_form(torch, duration=args.serving_only)}))
        return
    if args.batched_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        print(json.dumps({"batched_form": batched_form(torch, bto, hbm, args.steps, count=args.batched_count,
                                                       tile=args.batched_tile)}))
        return
    if args.mrhs_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        print(json.dumps({"mrhs": mrhs_form(torch, bto, hbm, args.steps, n=args.n if args.n != N_MAT else 8192,
                                            k=args.mrhs_only)}))
        return
    if args.sparse_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        print(json.dumps({"sparse": sparse_form(torch, bto, hbm)}))
        return
    if args.gemver2048_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        print(json.dumps({"gemver_n2048": gemver_small(torch, bto, hbm)}))
        return
    if args.structured_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, sm_max, _ = load_peaks()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = FP64_FLOP_PER_CLK_PER_SM * sms * sm_max * 1e6 / 1e12
        print(json.dumps({"structured": structured_form(torch, bto, hbm, peak)}))
        return
    if args.generator_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        _, sm_max, _ = load_peaks()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = FP64_FLOP_PER_CLK_PER_SM * sms * sm_max * 1e6 / 1e12
        print(json.dumps({"generator": generator_form(torch, bto, peak, n=args.n)}))
        return
    if args.layout_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        _, sm_max, _ = load_peaks()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        peak = FP64_FLOP_PER_CLK_PER_SM * sms * sm_max * 1e6 / 1e12
        print(json.dumps({"layout": layout_form(torch, bto, peak, n=args.n)}))
        return
    if args.df_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        suite = Suite(torch, bto, args.n, args.n, args.nvec)
        _, kern64 = timed_steps(torch, suite, 1, 0, 0, None)
        print(json.dumps({"df_form": df_form(torch, suite, args.steps, args.warmup, None, hbm, kern64)}))
        return
    if args.search_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        print(json.dumps({"schedule_search": schedule_search_form(torch, n=args.search_only)}))
        return
    if args.precision_only:
        import torch
        from paper_1205_1098_gb300 import build
        build.build()
        import paper_1205_1098_gb300 as bto
        hbm, _, _ = load_peaks()
        print(json.dumps({"precision_form": precision_form(torch, bto, hbm, args.steps, n=args.precision_only)}))
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    from paper_1205_1098_gb300 import build
    build.build()
    import paper_1205_1098_gb300 as bto
    from paper_1205_1098_gb300 import replicas

    m = n = args.n
    N = args.nvec
    hbm, sm_max, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    fp64_peak = FP64_FLOP_PER_CLK_PER_SM * sms * sm_max * 1e6 / 1e12   # TFLOP/s

    suite = Suite(torch, bto, m, n, N)
    with Clocks(local) as clk:
        ms, kern = timed_steps(torch, suite, args.steps, args.warmup, 0, dist)
    clocks = clk.summary()
    # max over ranks
    step_bytes = suite_bytes(m, n, N)
    value, ms = replicas.job_rate(torch, dist, step_bytes, ms, device="cuda")

    per = {}
    for k in KERNELS:
        t = kern[k] * 1e-3
        gbs = compulsory_bytes(k, m, n, N) / t / 1e9
        tf = flops(k, m, n, N) / t / 1e12
        med, p10, p90 = timed_steps.spread[k]
        per[k] = {"ms": round(kern[k], 4), "ms_median": round(med, 4), "ms_p10": round(p10, 4),
                  "ms_p90": round(p90, 4), "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3),
                  "fp64_tflops": round(tf, 4), "fp64_frac": round(tf / fp64_peak, 3),
                  "bound": "alu" if tf / fp64_peak > gbs / hbm else "hbm"}

    unfused = None
    if not args.no_unfused:
        ums, ukern = timed_steps(torch, suite, args.steps, max(3, args.warmup // 2), 1, dist)
        unfused = {"ms_per_step": round(ums, 3), "value": round(step_bytes / (ums * 1e-3) / 1e9, 1),
                   "unit": "GB/s of fused compulsory bytes", "speedup_fused": round(ums / ms, 3)}
        for k in KERNELS:
            per[k]["unfused_ms"] = round(ukern[k], 4)
            per[k]["unfused_own_gbs"] = round(unfused_bytes(k, m, n, N) / (ukern[k] * 1e-3) / 1e9, 1)
            per[k]["fused_speedup"] = round(ukern[k] / kern[k], 3)
            per[k]["byte_ratio"] = round(unfused_bytes(k, m, n, N) / compulsory_bytes(k, m, n, N), 3)

    dff = None
    if not args.no_df:
        dff = df_form(torch, suite, args.steps, args.warmup, dist, hbm, kern)

    # Roofline of the dominant kernel (largest share of the step).
    dom = max(KERNELS, key=lambda k: kern[k])
    d = per[dom]
    traffic = NCU_TRAFFIC.get(dom)
    if traffic is not None:
        traffic = round(traffic * (m * n) / NCU_TRAFFIC_N ** 2)
    if d["bound"] == "alu":
        roof = {"kernel": "bto_%s (all launches of one call)" % dom, "bound": "alu",
                "achieved": d["fp64_tflops"], "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                "frac": d["fp64_frac"], "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read+write of the same launches at n=%d, scaled by m n"
                                  % NCU_TRAFFIC_N,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x %d SMs x %.0f MHz" % (sms, sm_max),
                "peak_measured": round(2 * FP64_FMA_PER_CLK_MEASURED * sms * sm_max * 1e6 / 1e12, 4),
                "frac_of_measured": round(d["fp64_tflops"] / (2 * FP64_FMA_PER_CLK_MEASURED * sms * sm_max * 1e6
                                                             / 1e12), 3),
                "peak_measured_source": "DFMA throughput probe on this GPU: %.2f FMA/clk/SM" % FP64_FMA_PER_CLK_MEASURED,
                "hbm_frac_of_%s" % peak_src: d["hbm_frac"]}
    else:
        roof = {"kernel": "bto_%s (all launches of one call)" % dom, "bound": "hbm",
                "achieved": d["gbs"], "peak": hbm, "unit": "GB/s", "frac": d["hbm_frac"],
                "traffic": traffic, "peak_source": peak_src}

    e2e = None
    if not args.no_e2e:
        del suite
        torch.cuda.empty_cache()
        ems, h2d, d2h = e2e_steps(torch, bto, max(2, args.steps // 3), 1, m, n, N)
        evalue, ems = replicas.job_rate(torch, dist, step_bytes, ems, device="cuda")
        e2e = {"value": round(evalue, 2), "unit": "GB/s",
               "ms_per_step": round(ems, 3), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    prec = None
    if not args.no_precision and not args.only:
        try:
            del suite
        except NameError:
            pass
        torch.cuda.empty_cache()
        prec = precision_form(torch, bto, hbm, max(3, args.steps // 3))
    batched = None
    if not args.no_batched and not args.only:
        torch.cuda.empty_cache()
        batched = batched_form(torch, bto, hbm, max(3, args.steps // 3))
    mrhs = None
    if not args.no_mrhs and not args.only:
        torch.cuda.empty_cache()
        mrhs = mrhs_form(torch, bto, hbm, max(10, args.steps))
    serving = None
    if not args.no_serving and not args.only:
        torch.cuda.empty_cache()
        serving = serving_form(torch)
    small = None
    if not args.only:
        torch.cuda.empty_cache()
        small = gemver_small(torch, bto, hbm)
    layout = None
    if not args.no_layout and not args.only:
        torch.cuda.empty_cache()
        layout = layout_form(torch, bto, fp64_peak, n=m)
    gen = None
    if not args.no_generator and not args.only:
        torch.cuda.empty_cache()
        gen = generator_form(torch, bto, fp64_peak, n=m)
    sparse = None
    if not args.no_sparse and not args.only:
        torch.cuda.empty_cache()
        sparse = sparse_form(torch, bto, hbm)
    structured = None
    if not args.no_structured and not args.only:
        torch.cuda.empty_cache()
        structured = structured_form(torch, bto, hbm, fp64_peak)
    search = None
    if not args.no_search and not args.only:
        torch.cuda.empty_cache()
        search = schedule_search_form(torch, n=m)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ns, nv = 8192, 1 << 25
        cores = host_cores()
        psecs, pbytes = oracle_sample(ns, nv, parallel=True)
        secs, nbytes = oracle_sample(ns, nv)
        cpu = {"value": round(pbytes / psecs / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": "the oracle (plain C, FP64) on all %d host cores (OpenMP over independent outputs, "
                         "bit-identical to the serial oracle) on the same suite at n=%d matrices and "
                         "%d-element vectors (%.1f s), bytes scaled the same way" % (cores, ns, nv, psecs),
               "serial": {"value": round(nbytes / secs / 1e9, 4), "unit": "GB/s", "cores": 1,
                          "seconds": round(secs, 2)}}

    launches = args.steps * sum(LAUNCHES[k] for k in KERNELS)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC,
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (SplitMix64 uniform[-1,1), seed 1), generated on the device",
            "config": {"workload": WORKLOAD, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "every input is larger than L2 (2 GiB matrices, 512 MiB vectors); no flush"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "kernels": per, "unfused": unfused,
            "df_form_n16384": dff,
            "precision_form_n32768": prec,
            "batched_4096": batched,
            "mrhs_8192_k64": mrhs,
            "serving": serving,
            "gemver_n2048": small,
            "schedule_search": search,
            "layout_n16384": layout,
            "generator_n16384": gen,
            "csr_2e20_avg32": sparse,
            "structured": structured,
            "peaks": {"hbm_gbs": hbm, "hbm_source": peak_src, "fp64_tflops": round(fp64_peak, 4)},
        }))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
