"""Measured-cost tuner for the batched form's panel width.

Like the empirical search of the paper (every candidate is run and timed, and
a fitness cache keeps what was measured), but over the GPU schedule's one
free parameter: the column-panel width of the work items (the split factor).
Each candidate is prepared, run once to warm up, then timed over `reps`
launches with CUDA events; the fastest wins.  Results are cached in a JSON
file keyed by the batch's shape signature, the device and the library
version, and reused on later calls.
"""
import hashlib
import json
import os

import torch

from . import _lib as L

CANDIDATES = (32, 64, 128, 256, 512)
CACHE = os.environ.get("BTO_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json"))


def signature(descs):
    """Shape signature of a batch: ops and sizes (not the data)."""
    h = hashlib.sha256()
    for d in descs:
        h.update(("%d,%d,%d,%d;" % (d.op, d.m, d.n, d.lda)).encode())
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%s|sm%d|v%d|%d" % (h.hexdigest()[:24], p.name, p.multi_processor_count, L.bto_version(), len(descs))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def time_candidate(descs, tile_cols, reps=5, stream=None):
    """Mean milliseconds of bto_batch_run for one panel width."""
    nb = L.bto_batch_workspace_bytes(descs, tile_cols)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    st = stream or torch.cuda.current_stream()
    L.bto_batch_prepare(len(descs), descs, tile_cols, ws, nb, st)
    L.bto_batch_run(ws, nb, st)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        L.bto_batch_run(ws, nb, st)
    e1.record(st)
    torch.cuda.synchronize()
    if L.bto_device_status(ws) != 0:
        raise RuntimeError("batched run reported a device timeout")
    return e0.elapsed_time(e1) / reps


def tune(descs, candidates=CANDIDATES, reps=5, use_cache=True):
    """Returns (best panel width, {width: ms}); measures unless cached."""
    key = signature(descs)
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        return e["best"], {int(k): v for k, v in e["ms"].items()}
    ms = {c: time_candidate(descs, c, reps) for c in candidates}
    best = min(ms, key=ms.get)
    if use_cache:
        cache[key] = {"best": best, "ms": {str(k): v for k, v in ms.items()}}
        _save(cache)
    return best, ms
