"""ctypes binding of libbto.so: the C entry points under the same names.

Argument marshalling only.  Pointer arguments accept a torch tensor (its
data_ptr() is passed), an int address, or None (NULL).  Stream arguments
accept a torch.cuda.Stream, an int handle, or None (the current torch
stream of the current device).  A non-zero status raises BtoError.  There
is no fallback: if the library is not built, loading it raises.
"""
import ctypes
import os

from . import build as _build

_c_i64, _c_u64, _c_f64, _c_int = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
_c_ptr, _c_size = ctypes.c_void_p, ctypes.c_size_t

# Argument kinds: i = int64, u = uint64, d = double, p = pointer, z = size_t,
# s = stream, k = int, f = float
SIGNATURES = {
    "bto_bicgk": "iipipppppzs",
    "bto_atax": "iidpipppzs",
    "bto_gemver": "iiddpipppppppipppzs",
    "bto_gesummv": "iidpidpipppzs",
    "bto_dgemv": "iidpipdpppzs",
    "bto_dgemvt": "iiddpipppppzs",
    "bto_axpydot": "idppppppzs",
    "bto_waxpby": "idpdpps",
    "bto_vadd": "ipppps",
    "bto_unfused_bicgk": "iipipppppzs",
    "bto_unfused_atax": "iidpipppzs",
    "bto_unfused_gemver": "iiddpipppppppipppzs",
    "bto_unfused_gesummv": "iidpidpipppzs",
    "bto_unfused_dgemv": "iidpipdpppzs",
    "bto_unfused_dgemvt": "iiddpipppppzs",
    "bto_unfused_axpydot": "idppppppzs",
    "bto_unfused_waxpby": "idpdpps",
    "bto_unfused_vadd": "ipppps",
    "bto_fill_f64": "uukiippis",
    "bto_fill_f32": "uukiippis",
    "bto_fill_bf16": "uukiippis",
    "bto_debug_atax_stall": "iidpipppziks",
    "bto_debug_batch_stall": "pzkks",
    "bto_debug_gemver_stall": "iiddpipppppppipppzkks",
    "bto_debug_df_stall": "iipipppppzkks",
    "bto_debug_lpt": "ipkp",
    "bto_bicgk_noalloc": "iipipppps",
    "bto_bicgk_ex": "iikpipppppzs",
    "bto_gemver_ex": "iiffkpipppppppipppzs",
    "bto_atax_ex": "iifkpipppzs",
    "bto_gesummv_ex": "iiffkpipipppzs",
    "bto_batch_prepare": "kpkpzs",
    "bto_batch_run": "pzs",
    "bto_batch_submit": "kpkpzpzs",
    "bto_schedule_set": "kkkk",
    "bto_bicgk_mrhs": "iiipipipipipipzs",
    "bto_bicgk_layout": "kiipipppppzs",
    "bto_atax_layout": "kiidpipppzs",
    "bto_gemver_layout": "kiiddpipppppppipppzs",
    "bto_gesummv_layout": "kiidpidpipppzs",
    "bto_dgemv_layout": "kkiidpipdpppzs",
    "bto_dgemvt_layout": "kiiddpipppppzs",
    "bto_csr_bicgk": "iiippppppppzs",
    "bto_csr_atax": "iiipppdpppzs",
    "bto_band_bicgk": "kiiiikpipppppzs",
    "bto_band_atax": "kiiiikdpipppzs",
    "bto_tri_bicgk": "kkkipipppppzs",
    "bto_tri_atax": "kkkidpipppzs",
}
# The double-float forms take the FP64 forms' arguments.
for _k in ("bicgk", "atax", "gemver", "gesummv", "dgemv", "dgemvt"):
    SIGNATURES["bto_%s_df" % _k] = SIGNATURES["bto_" + _k]
    SIGNATURES["bto_unfused_%s_df" % _k] = SIGNATURES["bto_unfused_" + _k]
_KIND = {"i": _c_i64, "u": _c_u64, "d": _c_f64, "f": ctypes.c_float, "p": _c_ptr, "z": _c_size,
         "s": _c_ptr, "k": _c_int}

BTO_OK, BTO_ERR_INVALID_VALUE, BTO_ERR_UNSUPPORTED, BTO_ERR_WORKSPACE = 0, 1, 2, 3
BTO_ERR_CUDA, BTO_ERR_TIMEOUT, BTO_ERR_BUDGET = 4, 5, 6
BTO_F64, BTO_F32, BTO_BF16 = 0, 1, 2
BTO_FORM_FUSED, BTO_FORM_UNFUSED, BTO_FORM_DF, BTO_FORM_DF_UNFUSED = 0, 1, 2, 3
BTO_COL_MAJOR, BTO_ROW_MAJOR = 0, 1
BTO_NO_TRANS, BTO_TRANS = 0, 1
BTO_STORE_FULL, BTO_STORE_BAND, BTO_STORE_PACKED = 0, 1, 2
BTO_UPPER, BTO_LOWER = 0, 1
OPS = {"bicgk": 0, "atax": 1, "gemver": 2, "gesummv": 3, "dgemv": 4, "dgemvt": 5,
       "axpydot": 6, "waxpby": 7, "vadd": 8}


class BtoError(RuntimeError):
    def __init__(self, func, status, arg):
        self.status, self.arg = status, arg
        msg = "%s failed: %s" % (func, _status_string(status))
        if arg:
            msg += " (argument %d)" % arg
        super().__init__(msg)


_LIB = None


def lib():
    """The loaded libbto.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libbto.so is not built (%s); run paper_1205_1098_gb300.build.build() "
                               "or __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, sig in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = [_KIND[c] for c in sig]
            f.restype = _c_int
        L.bto_version.restype = _c_int
        L.bto_status_string.argtypes = [_c_int]
        L.bto_status_string.restype = ctypes.c_char_p
        L.bto_last_invalid_arg.restype = _c_int
        L.bto_workspace_bytes.argtypes = [_c_int, _c_int, _c_i64, _c_i64, _c_int, ctypes.POINTER(_c_size)]
        L.bto_workspace_bytes.restype = _c_int
        L.bto_device_status.argtypes = [_c_ptr, _c_ptr, ctypes.POINTER(_c_int)]
        L.bto_device_status.restype = _c_int
        L.bto_batch_one_launch.argtypes = [_c_ptr, ctypes.POINTER(_c_int)]
        L.bto_batch_one_launch.restype = _c_int
        L.bto_bicgk_mrhs_workspace_bytes.argtypes = [_c_i64, _c_i64, _c_i64, ctypes.POINTER(_c_size)]
        L.bto_bicgk_mrhs_workspace_bytes.restype = _c_int
        _LIB = L
    return _LIB


def _status_string(s):
    return lib().bto_status_string(int(s)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, (ctypes.Array, ctypes.Structure)):
        return ctypes.addressof(x)
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _conv(kind, v):
    if kind == "p":
        return _ptr(v)
    if kind == "s":
        return _stream(v)
    if kind in ("d", "f"):
        return float(v)
    return int(v)


def _make(name):
    sig = SIGNATURES[name]

    def call(*args):
        if len(args) == len(sig) - 1 and sig[-1] == "s":
            args = args + (None,)
        if len(args) != len(sig):
            raise TypeError("%s takes %d arguments (%d given)" % (name, len(sig), len(args)))
        L = lib()
        st = getattr(L, name)(*[_conv(k, a) for k, a in zip(sig, args)])
        if st != BTO_OK:
            raise BtoError(name, st, L.bto_last_invalid_arg())
        return st

    call.__name__ = name
    call.__doc__ = "C entry point %s (see include/bto.h); argument kinds %s." % (name, sig)
    return call


for _name in SIGNATURES:
    globals()[_name] = _make(_name)


def bto_version():
    return lib().bto_version()


def bto_status_string(status):
    return _status_string(status)


def bto_last_invalid_arg():
    return lib().bto_last_invalid_arg()


def bto_workspace_bytes(op, form, m, n, a_type=BTO_F64):
    """Workspace size in bytes; `op` may be a bto_op value or a name such as 'bicgk'."""
    if isinstance(op, str):
        op = OPS[op]
    out = _c_size(0)
    L = lib()
    st = L.bto_workspace_bytes(int(op), int(form), int(m), int(n), int(a_type), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


def bto_csr_workspace_bytes(op, m, n, nnz):
    """Workspace bytes of bto_csr_bicgk / bto_csr_atax (op: 'bicgk', 'atax' or a bto_op value)."""
    if isinstance(op, str):
        op = OPS[op]
    out = _c_size(0)
    L = lib()
    st = L.bto_csr_workspace_bytes(_c_int(int(op)), _c_i64(int(m)), _c_i64(int(n)), _c_i64(int(nnz)),
                                   ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_csr_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


def bto_band_workspace_bytes(op, m, n, kl, ku):
    """Workspace bytes of bto_band_bicgk / bto_band_atax (op: 'bicgk', 'atax' or a bto_op value)."""
    if isinstance(op, str):
        op = OPS[op]
    out = _c_size(0)
    L = lib()
    st = L.bto_band_workspace_bytes(_c_int(int(op)), _c_i64(int(m)), _c_i64(int(n)), _c_i64(int(kl)),
                                    _c_i64(int(ku)), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_band_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


def bto_tri_workspace_bytes(op, uplo, n):
    """Workspace bytes of bto_tri_bicgk / bto_tri_atax."""
    if isinstance(op, str):
        op = OPS[op]
    out = _c_size(0)
    L = lib()
    st = L.bto_tri_workspace_bytes(_c_int(int(op)), _c_int(int(uplo)), _c_i64(int(n)), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_tri_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


def bto_layout_workspace_bytes(op, layout, trans, m, n):
    """Workspace bytes of the bto_*_layout entry points (op: a bto_op value or a name)."""
    if isinstance(op, str):
        op = OPS[op]
    out = _c_size(0)
    L = lib()
    L.bto_layout_workspace_bytes.argtypes = [_c_int, _c_int, _c_int, _c_i64, _c_i64, ctypes.POINTER(_c_size)]
    L.bto_layout_workspace_bytes.restype = _c_int
    st = L.bto_layout_workspace_bytes(int(op), int(layout), int(trans), int(m), int(n), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_layout_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


class Instr(ctypes.Structure):
    """bto_instr of include/bto.h (one instruction of a pass program)."""
    _fields_ = [("op", ctypes.c_int32), ("mode", ctypes.c_int32), ("reverse", ctypes.c_int32),
                ("slot_q", ctypes.c_int32), ("slot_q2", ctypes.c_int32), ("slot_s", ctypes.c_int32),
                ("src1", ctypes.c_int32), ("src2", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("Bout", ctypes.c_void_p), ("ldbo", ctypes.c_int64),
                ("p", ctypes.c_void_p), ("r", ctypes.c_void_p),
                ("u1", ctypes.c_void_p), ("v1", ctypes.c_void_p), ("u2", ctypes.c_void_p), ("v2", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("a1", ctypes.c_double), ("a2", ctypes.c_double), ("b", ctypes.c_double)]


BTO_INSTR_PASS, BTO_INSTR_COMBINE, BTO_INSTR_WAXPBY = 0, 1, 2
BTO_PASS_QS, BTO_PASS_Q, BTO_PASS_S, BTO_PASS_G1, BTO_PASS_Q2, BTO_PASS_G1Q = 0, 1, 2, 3, 4, 5
BTO_PROGRAM_MAX_SLOTS, BTO_PROGRAM_MAX_INSTRS = 64, 4096


def _program_fn(name, argtypes):
    f = getattr(lib(), name)
    f.argtypes = argtypes
    f.restype = _c_int
    return f


def bto_program_check(prog):
    """(status, bad_index) of the structural check of a ctypes Instr array."""
    bad = _c_int(-1)
    f = _program_fn("bto_program_check", [_c_ptr, _c_int, ctypes.POINTER(_c_int)])
    st = f(ctypes.addressof(prog) if len(prog) else None, len(prog), ctypes.byref(bad))
    return st, bad.value


def bto_program_workspace_bytes(prog):
    out = _c_size(0)
    f = _program_fn("bto_program_workspace_bytes", [_c_ptr, _c_int, ctypes.POINTER(_c_size)])
    st = f(ctypes.addressof(prog) if len(prog) else None, len(prog), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_program_workspace_bytes", st, lib().bto_last_invalid_arg())
    return out.value


def bto_program_run(prog, ws, ws_bytes, stream=None):
    f = _program_fn("bto_program_run", [_c_ptr, _c_int, _c_ptr, _c_size, _c_ptr])
    st = f(ctypes.addressof(prog) if len(prog) else None, len(prog), _ptr(ws), int(ws_bytes), _stream(stream))
    if st != BTO_OK:
        raise BtoError("bto_program_run", st, lib().bto_last_invalid_arg())
    return st


def bto_bicgk_mrhs_workspace_bytes(m, n, k):
    """Workspace bytes of bto_bicgk_mrhs for an m x n A and k right-hand sides."""
    out = _c_size(0)
    L = lib()
    st = L.bto_bicgk_mrhs_workspace_bytes(int(m), int(n), int(k), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_bicgk_mrhs_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


def bto_panel_plan(op, form, m, n, sms):
    """(row_blocks, panels) of the tile plan of the FP64 or double-float forms (host only)."""
    if isinstance(op, str):
        op = OPS[op]
    a, b = _c_int(0), _c_int(0)
    L = lib()
    L.bto_panel_plan.argtypes = [_c_int, _c_int, _c_i64, _c_i64, _c_int, ctypes.POINTER(_c_int),
                                 ctypes.POINTER(_c_int)]
    L.bto_panel_plan.restype = _c_int
    st = L.bto_panel_plan(int(op), int(form), int(m), int(n), int(sms), ctypes.byref(a), ctypes.byref(b))
    if st != BTO_OK:
        raise BtoError("bto_panel_plan", st, L.bto_last_invalid_arg())
    return a.value, b.value


def bto_schedule_get(op, form):
    """(panels, row_blocks) set for (op, form); 0 means automatic."""
    if isinstance(op, str):
        op = OPS[op]
    a, b = _c_int(0), _c_int(0)
    L = lib()
    L.bto_schedule_get.argtypes = [_c_int, _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]
    L.bto_schedule_get.restype = _c_int
    st = L.bto_schedule_get(int(op), int(form), ctypes.byref(a), ctypes.byref(b))
    if st != BTO_OK:
        raise BtoError("bto_schedule_get", st, L.bto_last_invalid_arg())
    return a.value, b.value


def bto_device_status(ws, stream=None):
    out = _c_int(0)
    L = lib()
    st = L.bto_device_status(_ptr(ws), _stream(stream), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_device_status", st, L.bto_last_invalid_arg())
    return out.value


def bto_batch_one_launch(ws):
    """True when bto_batch_run takes the one-launch form for workspace ws."""
    out = _c_int(0)
    L = lib()
    st = L.bto_batch_one_launch(_ptr(ws), ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_batch_one_launch", st, L.bto_last_invalid_arg())
    return out.value == 1


class BatchDesc(ctypes.Structure):
    """bto_batch_desc of include/bto.h."""
    _fields_ = [("op", ctypes.c_int32), ("a_type", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("A", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("in_", ctypes.c_void_p * 6), ("out", ctypes.c_void_p * 2)]


def bto_batch_workspace_bytes(descs, tile_cols=0):
    """Workspace bytes for a ctypes array of BatchDesc."""
    out = _c_size(0)
    L = lib()
    L.bto_batch_workspace_bytes.argtypes = [_c_int, ctypes.c_void_p, _c_int, ctypes.POINTER(_c_size)]
    L.bto_batch_workspace_bytes.restype = _c_int
    st = L.bto_batch_workspace_bytes(len(descs), ctypes.cast(descs, ctypes.c_void_p), int(tile_cols),
                                     ctypes.byref(out))
    if st != BTO_OK:
        raise BtoError("bto_batch_workspace_bytes", st, L.bto_last_invalid_arg())
    return out.value


class ServeReq(ctypes.Structure):
    """bto_serve_req of include/bto.h."""
    _fields_ = [("t", ctypes.c_double), ("op", ctypes.c_int32), ("a_type", ctypes.c_int32), ("n", ctypes.c_int64)]


class ServeRes(ctypes.Structure):
    """bto_serve_res of include/bto.h."""
    _fields_ = [("admit", ctypes.c_double), ("done", ctypes.c_double), ("out", ctypes.c_int64 * 3),
                ("status", ctypes.c_int32), ("direct", ctypes.c_int32)]


class ServeCfg(ctypes.Structure):
    """bto_serve_cfg of include/bto.h."""
    _fields_ = [("A", (ctypes.c_void_p * 2) * 2), ("vec", ctypes.c_void_p * 6), ("arena", ctypes.c_void_p),
                ("staging", ctypes.c_void_p), ("streams", ctypes.c_void_p), ("arena_bytes", ctypes.c_size_t),
                ("staging_bytes", ctypes.c_size_t), ("nmax", ctypes.c_int64), ("direct_n", ctypes.c_int64),
                ("max_wall", ctypes.c_double), ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("nstreams", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("tile_cols", ctypes.c_int32),
                ("keep_results", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    """bto_serve_stats of include/bto.h."""
    _fields_ = [("served", ctypes.c_int64), ("batches", ctypes.c_int64), ("direct", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("wall_s", ctypes.c_double), ("peak_bytes", ctypes.c_double),
                ("max_gap_s", ctypes.c_double), ("max_gap_at_s", ctypes.c_double), ("max_admit_s", ctypes.c_double),
                ("max_complete_s", ctypes.c_double), ("max_oversleep_s", ctypes.c_double),
                ("max_fifo", ctypes.c_int64), ("fifo_at_max_gap", ctypes.c_int64), ("sleeps", ctypes.c_int64),
                ("blocking_copies", ctypes.c_int64), ("max_query_s", ctypes.c_double)]


def bto_serve_run(cfg, count, reqs, res, stats):
    """Runs the serving loop over reqs[:count]; returns its status (BTO_OK or the
    first launch or device status that was not), raising only for invalid
    arguments."""
    L = lib()
    L.bto_serve_run.argtypes = [ctypes.c_void_p, _c_i64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.bto_serve_run.restype = _c_int
    st = L.bto_serve_run(ctypes.addressof(cfg), int(count), ctypes.cast(reqs, ctypes.c_void_p),
                         ctypes.cast(res, ctypes.c_void_p), ctypes.addressof(stats))
    if st in (BTO_ERR_INVALID_VALUE, BTO_ERR_WORKSPACE):
        raise BtoError("bto_serve_run", st, L.bto_last_invalid_arg())
    return st


def exported_symbols():
    """Names the binding expects libbto.so to export."""
    return sorted(list(SIGNATURES) + ["bto_version", "bto_status_string", "bto_last_invalid_arg",
                                      "bto_workspace_bytes", "bto_device_status",
                                      "bto_bicgk_mrhs_workspace_bytes", "bto_batch_workspace_bytes",
                                      "bto_serve_run", "bto_schedule_get", "bto_layout_workspace_bytes",
                                      "bto_program_check", "bto_program_workspace_bytes", "bto_program_run",
                                      "bto_panel_plan", "bto_band_workspace_bytes", "bto_tri_workspace_bytes",
                                      "bto_csr_workspace_bytes"])
