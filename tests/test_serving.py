"""The serving loop (continuous batching under an HBM budget): every request
finishes, results are the same bits alone and in the mix, sampled results
match the oracle on the stored values, and the budget is respected."""
import copy

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_util import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server():
    from paper_1205_1098_gb300 import build
    build.build()
    from paper_1205_1098_gb300.serve import Server
    return Server(budget_bytes=6e9, streams=4, max_batch=32, tile_cols=256, seed=4)


def _host_block(seed, t, n, aid):
    # Leading n x n block of the resident 8192 x 8192 matrix (array id aid).
    A = synth.matrix_cols(seed, aid, 8192, 8192, np.arange(n))[:n]
    if t == "f32":
        return synth.to_f32(A).astype(np.float64)
    return synth.bf16_bits_to_f64(synth.to_bf16_bits(A))


def _host_vec(seed, k, n):
    return synth.to_f32(synth.vector(seed, 100 + k, 8192))[:n].astype(np.float64)


def _oracle(r, seed=4):
    n, op, t = r["n"], r["op"], r["dtype"]
    code = 1 if t == "f32" else 2
    A = np.asfortranarray(_host_block(seed, t, n, 10 * code))
    v = [_host_vec(seed, k, n) for k in range(6)]
    if op == "bicgk":
        return list(O.bicgk(n, n, A, v[0], v[1]))
    if op == "atax":
        return [O.atax(n, n, 1.25, A, v[0])]
    if op == "gesummv":
        B = np.asfortranarray(_host_block(seed, t, n, 10 * code + 1))
        return [O.gesummv(n, n, 1.5, A, 1.25, B, v[0])]
    Bret = r["B"].cpu().numpy()
    Bret = (Bret.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(Bret.view(np.uint16))).reshape(n, n).T
    z = np.zeros(n)
    _, x, w = O.gemver(n, n, 1.5, 1.25, np.asfortranarray(Bret), z, z, z, z, v[4], v[5])
    return [x, w]


def test_serving_trace_alone_vs_mix_and_oracle(server):
    from paper_1205_1098_gb300.serve import make_trace
    trace = make_trace(seed=4, rate=20000.0, duration=0.0, nmax=1024, count=300)
    stats, done = server.run(copy.deepcopy(trace), keep_results=True)
    assert stats["requests"] == len(trace) and stats["status_ok"]
    assert stats["batches"] > 1 and stats["p99_ms"] >= stats["p50_ms"] > 0
    byid = {r["id"]: r for r in done}
    small = [r for r in trace if r["n"] <= 400][:12]
    assert small
    for r in small:
        got = byid[r["id"]]
        ref = _oracle(got)
        for k, ro in enumerate(ref):
            g = got["out"][k].cpu().numpy().astype(np.float64)
            assert relerr(g, ro) <= 1e-6, (r, k, relerr(g, ro))
    # Each request alone gives the same bits as in the mix.
    for r in trace[::37]:
        _, alone = server.run([dict(r, t=0.0)], keep_results=True)
        a, b = alone[0], byid[r["id"]]
        for k in range(len(b["out"])):
            assert torch.equal(a["out"][k], b["out"][k]), (r, k)
        if r["op"] == "gemver":
            assert torch.equal(a["B"], b["B"]), r


def test_serving_budget_is_respected(server):
    from paper_1205_1098_gb300.serve import Server, make_trace
    trace = make_trace(seed=5, rate=20000.0, duration=0.0, nmin=512, nmax=2048, count=120)
    small = Server.__new__(Server)
    small.__dict__.update(server.__dict__)
    small.budget = 0.25e9
    small.arena = server.arena[:int(small.budget)]
    stats, done = small.run(trace)
    assert stats["requests"] == len(trace) and stats["status_ok"] and stats["rejected"] == 0
    assert 0 < stats["peak_bytes"] <= small.budget


def test_serving_rejects_what_cannot_fit(server):
    """A request whose outputs exceed the whole budget ends with BTO_ERR_BUDGET;
    the others are served."""
    from paper_1205_1098_gb300.serve import Server
    small = Server.__new__(Server)
    small.__dict__.update(server.__dict__)
    small.budget = 2 << 20
    small.arena = server.arena[:small.budget]
    trace = [dict(id=0, t=0.0, op="bicgk", n=256, dtype="f32"),
             dict(id=1, t=0.0, op="gemver", n=1024, dtype="f32"),     # B alone is 4 MiB
             dict(id=2, t=0.0, op="atax", n=300, dtype="bf16")]
    stats, done = small.run(trace)
    assert stats["rejected"] == 1 and stats["requests"] == 2 and stats["status_ok"]
    assert sorted(d["id"] for d in done) == [0, 2]


def test_serving_direct_path_alone_vs_mix_and_oracle(server):
    """Requests with n >= direct_n run alone through the single-instance
    entry points while smaller ones are batched around them."""
    from paper_1205_1098_gb300.serve import make_trace
    trace = make_trace(seed=9, rate=20000.0, duration=0.0, nmin=512, nmax=4096, count=48)
    server.direct_n, saved = 2048, server.direct_n
    try:
        stats, done = server.run(copy.deepcopy(trace), keep_results=True)
    finally:
        server.direct_n = saved
    assert stats["requests"] == len(trace) and stats["status_ok"]
    assert stats["direct"] > 0 and stats["batches"] > 0
    byid = {r["id"]: r for r in done}
    picked = {}
    for r in trace:
        if r["n"] >= 2048 and r["op"] not in picked:
            picked[r["op"]] = r
    assert len(picked) >= 3, picked.keys()
    for r in picked.values():
        got = byid[r["id"]]
        for k, ro in enumerate(_oracle(got)):
            g = got["out"][k].cpu().numpy().astype(np.float64)
            assert relerr(g, ro) <= 1e-6, (r, k, relerr(g, ro))
        server.direct_n = 2048
        try:
            _, alone = server.run([dict(r, t=0.0)], keep_results=True)
        finally:
            server.direct_n = saved
        assert alone[0]["direct"]
        for k in range(len(got["out"])):
            assert torch.equal(alone[0]["out"][k], got["out"][k]), (r, k)
        if r["op"] == "gemver":
            assert torch.equal(alone[0]["B"], got["B"]), r
