"""Measured-cost search over the schedules of the FP64 matrix kernels.

The paper's compiler chooses, per kernel and machine, which loops to fuse and
how to partition them, with an empirical search: a genetic algorithm (MFGA,
Section IV) whose organisms are fusion and partition choices, whose fitness
is the measured run time of the generated code, and which keeps a cache of
every measured fitness; its search is checked against exhaustive
enumeration on the small kernels.  This module is that search over the GPU
schedules of this library:

  fused       -- the fused entry point (bto_<op>) or the one-kernel-per-BLAS-
                 call sequence (bto_unfused_<op>): which loops share a pass;
  panels      -- the number of column panels (the column partition p(j));
  row_blocks  -- the number of row blocks (the row partition p(i)).

Panels and row blocks are set with bto_schedule_set; 0 is the automatic
choice.  The population is seeded with the maximally fused automatic
schedule (the paper seeds with Max-Fuse) plus random organisms; each
generation keeps its best organism and fills the rest with children of two
parents chosen by tournament (k = 2), with uniform crossover of the genes and
mutation of each gene with probability p_mut.  Fitness is the median time of
a few calls on the GPU (CUDA events), cached by (device, library version,
op, m, n, schedule).  ATAX's fused kernel has its own plan, so for it the
partition genes of a fused organism are ignored (one organism stands for
all of them).
"""
import random

from . import _lib as L

OPS = ("bicgk", "atax", "gemver", "gesummv", "dgemv", "dgemvt")
ROW_BLOCKS = (0, 1, 2, 4, 8)


def panel_choices(sms):
    """Candidate panel counts: automatic, and fractions and multiples of the SM count."""
    return (0, sms // 4, sms // 2, sms, 2 * sms, 4 * sms)


def space(op, sms):
    """Every schedule of `op` (canonical organisms, no duplicates)."""
    out = []
    for fused in (True, False):
        for p in panel_choices(sms):
            for r in ROW_BLOCKS:
                o = canonical(op, (fused, p, r))
                if o not in out:
                    out.append(o)
    return out


def canonical(op, org):
    fused, p, r = org
    if op == "atax" and fused:
        return (True, 0, 0)
    return (bool(fused), int(p), int(r))


def mfga(op, fitness, sms, pop=8, gens=6, p_mut=0.3, seed=0):
    """Genetic search; `fitness(organism) -> ms` (lower is better, cached by
    the caller).  Returns {best, best_ms, evaluations, history}."""
    rng = random.Random(seed)
    panels = panel_choices(sms)
    genes = [(True, False), panels, ROW_BLOCKS]
    seen = {}

    def fit(o):
        o = canonical(op, o)
        if o not in seen:
            seen[o] = fitness(o)
        return seen[o]

    def rand_org():
        return canonical(op, tuple(rng.choice(g) for g in genes))

    def mutate(o):
        # The partition genes are ordered: mostly a step to a neighbouring
        # value, sometimes a fresh draw; the fusion gene flips.
        out = list(o)
        for i in range(3):
            if rng.random() >= p_mut:
                continue
            if i == 0:
                out[0] = not out[0]
            elif rng.random() < 0.7:
                k = genes[i].index(out[i]) + rng.choice((-1, 1))
                out[i] = genes[i][min(max(k, 0), len(genes[i]) - 1)]
            else:
                out[i] = rng.choice(genes[i])
        return canonical(op, tuple(out))

    population = [canonical(op, (True, 0, 0))]
    while len(population) < pop:
        population.append(rand_org())
    history = []
    for _ in range(gens):
        scored = sorted(population, key=fit)
        history.append((scored[0], fit(scored[0])))
        children = [scored[0]]                     # elitism
        while len(children) < pop:
            a = min(rng.sample(population, 2), key=fit)
            b = min(rng.sample(population, 2), key=fit)
            child = mutate(tuple(a[i] if rng.random() < 0.5 else b[i] for i in range(3)))
            for _ in range(4):                     # keep the population diverse
                if child not in children:
                    break
                child = mutate(child)
            children.append(child)
        population = children
    best = min(population + list(seen), key=fit)
    return {"best": best, "best_ms": fit(best), "evaluations": len(seen), "history": history}


def exhaustive(op, fitness, sms):
    """Every schedule measured; returns {best, best_ms, evaluations, table}."""
    table = {o: fitness(o) for o in space(op, sms)}
    best = min(table, key=table.get)
    return {"best": best, "best_ms": table[best], "evaluations": len(table), "table": table}


class Problem:
    """Device operands of one FP64 operation at m x n (seeded fills), and the
    measured time of one schedule."""

    def __init__(self, op, m, n, seed=1, reps=5):
        import torch
        self.torch, self.op, self.m, self.n, self.reps = torch, op, m, n, reps
        f64 = dict(dtype=torch.float64, device="cuda")
        self.A = torch.empty(m * n, **f64)
        L.bto_fill_f64(seed, 0, 0, m, n, 0, self.A, m, None)
        self.B = None
        if op == "gesummv":
            self.B = torch.empty(m * n, **f64)
            L.bto_fill_f64(seed, 1, 0, m, n, 0, self.B, m, None)
        if op == "gemver":
            self.B = torch.empty(m * n, **f64)
        self.v = []
        for aid, ln in enumerate((n, m, m, n, m, n, m, n)):
            t = torch.empty(max(ln, 1), **f64)
            L.bto_fill_f64(seed, 10 + aid, 0, ln, 1, 0, t, max(ln, 1), None)
            self.v.append(t)
        self.o = [torch.empty(max(m, n), **f64) for _ in range(2)]
        self.ws = None
        self.cache = {}
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        self.key = "%s|sm%d|v%d|%s|%dx%d" % (props.name, props.multi_processor_count, L.bto_version(), op, m, n)

    def _call(self, fused, ws, nb):
        m, n, A, v, o = self.m, self.n, self.A, self.v, self.o
        f = getattr(L, ("bto_" if fused else "bto_unfused_") + self.op)
        if self.op == "bicgk":
            f(m, n, A, m, v[0], v[1], o[0], o[1], ws, nb, None)
        elif self.op == "atax":
            f(m, n, 1.25, A, m, v[0], o[0], ws, nb, None)
        elif self.op == "gemver":
            f(m, n, 1.5, 1.2, A, m, v[2], v[3], v[4], v[5], v[6], v[7], self.B, m, o[0], o[1], ws, nb, None)
        elif self.op == "gesummv":
            f(m, n, 1.5, A, m, -0.75, self.B, m, v[0], o[0], ws, nb, None)
        elif self.op == "dgemv":
            f(m, n, 1.5, A, m, v[0], -0.5, v[1], o[0], ws, nb, None)
        else:
            f(m, n, 1.5, 1.2, A, m, v[1], v[0], o[0], o[1], ws, nb, None)

    def fitness(self, org):
        """Median ms of `reps` calls under schedule `org` (cached)."""
        org = canonical(self.op, org)
        key = self.key + "|%d,%d,%d" % (int(org[0]), org[1], org[2])
        if key in self.cache:
            return self.cache[key]
        torch = self.torch
        fused, panels, rows = org
        op_id, form = L.OPS[self.op], (0 if fused else 1)
        L.bto_schedule_set(op_id, form, panels, rows)
        try:
            nb = L.bto_workspace_bytes(op_id, form, self.m, self.n)
            ws = torch.empty(max(nb, 1) + 256, dtype=torch.uint8, device="cuda")
            for _ in range(2):
                self._call(fused, ws, nb)
            st = torch.cuda.current_stream()
            evs = []
            for _ in range(self.reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                self._call(fused, ws, nb)
                e1.record(st)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in evs)[len(evs) // 2]
        finally:
            L.bto_schedule_set(op_id, form, 0, 0)
        self.cache[key] = ms
        return ms
