"""The C ABI: the library builds, loads and exports every symbol include/bto.h
declares, the binding's argument kinds match the header, and argument
validation rejects bad calls before anything touches a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bto.h")


def _decls():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.findall(r"(?:bto_status|int|const char\s*\*)\s*(bto_\w+)\s*\(([^;]*)\);", src)


def _kind(a):
    if "*" in a:
        return "p"
    if "size_t" in a:
        return "z"
    if "uint64_t" in a:
        return "u"
    if "int64_t" in a:
        return "i"
    if "double" in a:
        return "d"
    if "float" in a:
        return "f"
    if "bto_stream_t" in a:
        return "s"
    if "void" == a.strip():
        return ""
    if "int" in a:
        return "k"
    return "?"


@pytest.fixture(scope="module")
def L():
    build.build()
    return bto.lib()


def test_every_declared_symbol_is_exported(L):
    names = [n for n, _ in _decls()]
    assert len(names) >= 27
    for n in names:
        assert hasattr(L, n), "libbto.so does not export " + n


def test_binding_kinds_match_header():
    for name, args in _decls():
        if name in _lib.SIGNATURES:
            got = "".join(_kind(a) for a in args.split(","))
            assert got == _lib.SIGNATURES[name], name


def test_status_strings(L):
    assert bto.bto_version() >= 100
    for s in range(7):
        assert bto.bto_status_string(s).startswith("BTO_")


def test_validation_without_gpu(L):
    # Negative sizes, short leading dimensions and NULL operands are rejected
    # before any CUDA call.
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk(-1, 4, 0, 1, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.status == _lib.BTO_ERR_INVALID_VALUE and e.value.arg == 1
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk(8, 4, 4096, 7, 4096, 8192, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 4   # lda < m
    with pytest.raises(bto.BtoError) as e:
        bto.bto_gemver(8, 4, 1.0, 1.0, 0, 8, 64, 128, 192, 256, 320, 384, 448, 8, 512, 576, 0, 0, 0)
    assert e.value.arg == 5   # A NULL with m*n > 0
    with pytest.raises(bto.BtoError) as e:   # output overlaps an input
        bto.bto_vadd(16, 4096, 8192, 12288, 4096 + 64, 0)
    assert e.value.arg == 5
    with pytest.raises(bto.BtoError) as e:   # misaligned double pointer
        bto.bto_waxpby(4, 1.0, 4097, 1.0, 8192, 12288, 0)
    assert e.value.arg == 3
    with pytest.raises(bto.BtoError) as e:
        bto.bto_workspace_bytes(99, 0, 1, 1)
    assert e.value.arg == 1
    with pytest.raises(bto.BtoError) as e:
        bto.bto_fill_f64(0, 0, 7, 4, 4, 0, 4096, 4, 0)
    assert e.value.arg == 3
    # The ring-wait fault injection takes a block index and a limit of 1..10000 ms.
    with pytest.raises(bto.BtoError) as e:
        bto.bto_debug_df_stall(8, 4, 4096, 8, 4096, 8192, 12288, 16384, 0, 0, -1, 50, 0)
    assert e.value.status == _lib.BTO_ERR_INVALID_VALUE and e.value.arg == 11
    with pytest.raises(bto.BtoError) as e:
        bto.bto_debug_df_stall(8, 4, 4096, 8, 4096, 8192, 12288, 16384, 0, 0, 0, 0, 0)
    assert e.value.arg == 12


def test_mrhs_validation_without_gpu(L):
    # Multi-RHS BICGK: k outside 16..96 or not a multiple of 16, negative
    # sizes, short leading dimensions, odd BF16 pointers and overlapping
    # outputs are rejected before any CUDA call.
    for k in (0, 8, 24, 112):
        with pytest.raises(bto.BtoError) as e:
            bto.bto_bicgk_mrhs(64, 64, k, 4096, 64, 8192, 64, 12288, 64, 16384, 64, 32768, 64, 0, 0, 0)
        assert e.value.arg == 3
        with pytest.raises(bto.BtoError) as e:
            bto.bto_bicgk_mrhs_workspace_bytes(64, 64, k)
        assert e.value.arg == 3
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_mrhs(-1, 64, 16, 4096, 64, 8192, 64, 12288, 64, 16384, 64, 32768, 64, 0, 0, 0)
    assert e.value.arg == 1
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_mrhs(64, 64, 16, 4096, 63, 8192, 64, 12288, 64, 16384, 64, 32768, 64, 0, 0, 0)
    assert e.value.arg == 5   # lda < m
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_mrhs(64, 64, 16, 4097, 64, 8192, 64, 12288, 64, 16384, 64, 32768, 64, 0, 0, 0)
    assert e.value.arg == 4   # A not 2-byte aligned
    with pytest.raises(bto.BtoError) as e:   # Q overlaps S
        bto.bto_bicgk_mrhs(64, 64, 16, 4096, 64, 8192, 64, 12288, 64, 16384, 64, 16384 + 64, 64, 0, 0, 0)
    assert e.value.arg == 10


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the C layout (gcc on the header)."""
    structs = {
        "bto_batch_desc": (_lib.BatchDesc, {"in": "in_"}),
        "bto_serve_req": (_lib.ServeReq, {}),
        "bto_serve_res": (_lib.ServeRes, {}),
        "bto_serve_cfg": (_lib.ServeCfg, {}),
        "bto_serve_stats": (_lib.ServeStats, {}),
        "bto_instr": (_lib.Instr, {}),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bto.h"', "int main(void) {"]
    for cname, (cls, rename) in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        back = {v: k for k, v in rename.items()}
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, back.get(fname, fname)))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, (cls, _) in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_serve_validation_without_gpu(L):
    cfg = _lib.ServeCfg()
    stats = _lib.ServeStats()
    reqs = (_lib.ServeReq * 2)()
    res = (_lib.ServeRes * 2)()
    streams = (ctypes.c_void_p * 1)(0)

    def run():
        try:
            _lib.bto_serve_run(cfg, 2, reqs, res, stats)
        except bto.BtoError as e:
            return e.status, e.arg
        return None

    assert run() == (bto.BTO_ERR_INVALID_VALUE, 1)           # no streams, no arena
    cfg.nstreams, cfg.streams = 1, ctypes.addressof(streams)
    cfg.arena, cfg.arena_bytes = 1 << 20, 1 << 30
    cfg.max_batch, cfg.tile_cols, cfg.nmax = 8, 256, 1024
    cfg.A[0][0] = cfg.A[0][1] = 1 << 21
    for k in range(6):
        cfg.vec[k] = 1 << 22
    cfg.tile_cols = 100
    assert run() == (bto.BTO_ERR_INVALID_VALUE, 1)           # tile width not a multiple of 16
    cfg.tile_cols = 256
    reqs[0].t, reqs[0].op, reqs[0].a_type, reqs[0].n = 0.0, 0, bto.BTO_F32, 64
    reqs[1].t, reqs[1].op, reqs[1].a_type, reqs[1].n = 0.0, 9, bto.BTO_F32, 64
    assert run() == (bto.BTO_ERR_INVALID_VALUE, 3)           # unknown op
    reqs[1].op, reqs[1].n = 2, 4096
    assert run() == (bto.BTO_ERR_INVALID_VALUE, 3)           # n > nmax
    reqs[1].n, reqs[1].a_type = 64, bto.BTO_BF16
    assert run() == (bto.BTO_ERR_INVALID_VALUE, 3)           # no resident BF16 matrix
    reqs[1].a_type, reqs[0].t = bto.BTO_F32, 1.0
    assert run() == (bto.BTO_ERR_INVALID_VALUE, 3)           # arrivals out of order


def test_schedule_overrides_without_gpu(L):
    """bto_schedule_set/get: per (op, form), validated, 0 = automatic, no GPU."""
    try:
        for form in (0, 1):
            assert bto.bto_schedule_get("gemver", form) == (0, 0)
        bto.bto_schedule_set(bto.OPS["gemver"], 1, 96, 3)
        assert bto.bto_schedule_get("gemver", 1) == (96, 3)
        assert bto.bto_schedule_get("gemver", 0) == (0, 0)
        for bad, arg in (((9, 0, 1, 1), 1), ((8, 0, 1, 1), 1), ((0, 2, 1, 1), 2), ((0, 0, -1, 1), 3),
                         ((0, 0, 1, (1 << 20) + 1), 4)):
            with pytest.raises(bto.BtoError) as e:
                bto.bto_schedule_set(*bad)
            assert e.value.status == bto.BTO_ERR_INVALID_VALUE and e.value.arg == arg, bad
    finally:
        bto.bto_schedule_set(bto.OPS["gemver"], 1, 0, 0)
    assert bto.bto_schedule_get("gemver", 1) == (0, 0)


def test_batch_one_launch_query_without_gpu(L):
    # No device work: a NULL workspace is argument 1; a workspace nothing was
    # prepared in runs the multi-launch form.
    with pytest.raises(bto.BtoError) as e:
        bto.bto_batch_one_launch(None)
    assert e.value.status == bto.BTO_ERR_INVALID_VALUE and e.value.arg == 1
    assert bto.bto_batch_one_launch(0x10000) is False
