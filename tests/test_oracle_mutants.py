"""Planted mistakes in the oracle must fail at least one pin (no GPU).

Each mutant is a copy of the oracle's C source with one plausible mistake (a
dropped term, a wrong sign, a wrong operand or index), compiled into a
temporary library on the CPU.  The pin suite is run against it and must
reject it; the real oracle passes the same suite (test_oracle_pins.py).
"""
import os

import pytest

import oracle
from oracle import build as obuild
from oracle_pins import PINS

MUTANTS = [
    ("bicgk_q_sign", "q[i] += AT(A, lda, i, j) * p[j];", "q[i] -= AT(A, lda, i, j) * p[j];"),
    ("bicgk_s_index", "s[j] += AT(A, lda, i, j) * r[i];", "s[j] += AT(A, lda, i, j) * r[0];"),
    ("atax_dropped_scale", "y[j] = t1[j] * beta;", "y[j] = t1[j];"),
    ("atax_t1_uses_x", "t1[j] += AT(A, lda, i, j) * t0[i];", "t1[j] += AT(A, lda, i, j) * x[j];"),
    ("gemver_wrong_v", "AT(B, ldb, i, j) + u2[i] * v2[j];", "AT(B, ldb, i, j) + u2[i] * v1[j];"),
    ("gemver_dropped_z",
     "x[j] = beta * t[j] + z[j];\n    for (int64_t i = 0; i < m; i++) t2[i] = 0.0;\n"
     "    for (int64_t i = 0; i < m; i++)\n        for (int64_t j = 0; j < n; j++)\n"
     "            t2[i] += AT(B, ldb",
     "x[j] = beta * t[j];\n    for (int64_t i = 0; i < m; i++) t2[i] = 0.0;\n"
     "    for (int64_t i = 0; i < m; i++)\n        for (int64_t j = 0; j < n; j++)\n"
     "            t2[i] += AT(B, ldb"),
    ("gemver_w_uses_A", "t2[i] += AT(B, ldb, i, j) * x[j];", "t2[i] += AT(A, lda, i, j) * x[j];"),
    ("gesummv_wrong_sum", "y[i] = alpha * ta[i] + beta * tb[i];", "y[i] = alpha * ta[i] + beta * ta[i];"),
    ("dgemv_dropped_beta", "z[i] = alpha * t[i] + beta * y[i];", "z[i] = alpha * t[i] + y[i];"),
    ("dgemvt_w_uses_z", "t2[i] += AT(A, lda, i, j) * x[j];\n    for (int64_t i = 0; i < m; i++)\n        w[i] = alpha * t2[i];\n    free(t); free(t2);\n    return 0;\n}\n\n/* AXPYDOT",
     "t2[i] += AT(A, lda, i, j) * z[j];\n    for (int64_t i = 0; i < m; i++)\n        w[i] = alpha * t2[i];\n    free(t); free(t2);\n    return 0;\n}\n\n/* AXPYDOT"),
    ("axpydot_sign", "z[i] = w[i] - alpha * v[i];\n    double acc", "z[i] = w[i] + alpha * v[i];\n    double acc"),
    ("waxpby_wrong_operand", "w[i] = alpha * x[i] + beta * y[i];", "w[i] = alpha * x[i] + beta * x[i];"),
    ("vadd_order", "x[i] = (w[i] + y[i]) + z[i];", "x[i] = w[i] + (y[i] + z[i]);"),
    ("vadd_wrong_operand", "x[i] = (w[i] + y[i]) + z[i];", "x[i] = (w[i] + y[i]) + y[i];"),
    ("dot2_dropped_error", "s = s + (q + r);", "s = s + q;"),
    ("dot2_no_twoproduct", "*y = fma(a, b, -p);", "*y = 0.0;"),
    ("mrhs_wrong_column", "oracle_bicgk(m, n, A, lda, P + (size_t)c * (size_t)ldp, R + (size_t)c * (size_t)ldr,",
     "oracle_bicgk(m, n, A, lda, P, R + (size_t)c * (size_t)ldr,"),
    ("row_dot_sign", "acc += row[j] * p[j];", "acc -= row[j] * p[j];"),
    ("csr_q_sign", "acc += val[k] * p[col[k]];", "acc -= val[k] * p[col[k]];"),
    ("csr_s_wrong_row", "s[col[k]] += val[k] * r[i];", "s[col[k]] += val[k] * r[0];"),
    ("csr_atax_dropped_beta", "for (int64_t j = 0; j < n; j++) y[j] *= beta;", ""),
    ("csr_atax_drops_last_entry",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) acc += val[k] * x[col[k]];",
     "for (int64_t k = row_ptr[i]; k + 1 < row_ptr[i + 1]; k++) acc += val[k] * x[col[k]];"),
    ("csr_atax_t_transposed",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) y[col[k]] += val[k] * t[i];",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) y[col[k]] += val[k] * x[col[k]];"),
    ("band_row_offset_sign", "A[(size_t)(b->ku + i - j) + (size_t)j * (size_t)b->ld]",
     "A[(size_t)(b->ku - i + j) + (size_t)j * (size_t)b->ld]"),
    ("band_uses_kl_offset", "A[(size_t)(b->ku + i - j) + (size_t)j * (size_t)b->ld]",
     "A[(size_t)(b->kl + i - j) + (size_t)j * (size_t)b->ld]"),
    ("packed_lower_offset", "(b->kl == 0 ? i : i - j)", "(b->kl == 0 ? i : i - j + 1)"),
    ("packed_column_length", "off += (kl == 0) ? c + 1 : n - c;", "off += (kl == 0) ? c : n - c;"),
    ("band_unit_ignored", "if (b->unit && i == j) return 1.0;", ""),
    ("band_q_drops_last_super",
     "for (int64_t j = (i - kl > 0 ? i - kl : 0); j <= i + ku && j < n; j++)\n            acc += band_get(&b, i, j) * p[j];",
     "for (int64_t j = (i - kl > 0 ? i - kl : 0); j < i + ku && j < n; j++)\n            acc += band_get(&b, i, j) * p[j];"),
    ("band_s_drops_first_sub",
     "for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < m; i++)\n            acc += band_get(&b, i, j) * r[i];",
     "for (int64_t i = (j - ku > 0 ? j - ku + 1 : 0); i <= j + kl && i < m; i++)\n            acc += band_get(&b, i, j) * r[i];"),
    ("band_s_wrong_vector_index", "acc += band_get(&b, i, j) * r[i];", "acc += band_get(&b, i, j) * r[j % (m > 0 ? m : 1)];"),
    ("band_atax_dropped_beta", "for (int64_t j = 0; j < n; j++) y[j] = y[j] * beta;",
     "for (int64_t j = 0; j < n; j++) y[j] = y[j];"),
    ("band_atax_second_uses_x", "acc += band_get(&b, i, j) * t[i];", "acc += band_get(&b, i, j) * x[i % (n > 0 ? n : 1)];"),
]


def _fails(L):
    for pin in PINS:
        try:
            pin(L)
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, "mutation site must be unique: " + name
    mpath = tmp_path / ("mut_%s.c" % name)
    mpath.write_text(src.replace(old, new))
    lib = obuild.build(src=str(mpath), out=str(tmp_path / ("libmut_%s.so" % name)), force=True)
    assert _fails(oracle.lib(lib)), "planted mistake %s passed every pin" % name
