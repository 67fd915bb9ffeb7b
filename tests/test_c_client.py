"""The C ABI from a plain C program: include/bto.h compiles under gcc as C99,
a client links libbto.so and calls entry points that need no device
(version, status strings, argument validation with its position, the tile
plan query, the program check) and gets the documented answers."""
import os
import subprocess

from paper_1205_1098_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "bto.h"

int main(void) {
    if (bto_version() < 100) return 10;
    if (strncmp(bto_status_string(BTO_ERR_WORKSPACE), "BTO_ERR_WORKSPACE", 17) != 0) return 11;
    /* lda < m: rejected before any device call, argument 4 named. */
    double dummy[4];
    bto_status st = bto_bicgk(8, 4, dummy, 7, dummy, dummy, dummy, dummy, NULL, 0, NULL);
    if (st != BTO_ERR_INVALID_VALUE || bto_last_invalid_arg() != 4) return 12;
    int rb = 0, pn = 0;
    if (bto_panel_plan(BTO_OP_GEMVER, BTO_FORM_FUSED, 16384, 16384, 152, &rb, &pn) != BTO_OK) return 13;
    if (rb != 8 || pn != 152) return 14;
    /* A program whose combine reads a slot no pass wrote. */
    bto_instr prog[1];
    memset(prog, 0, sizeof(prog));
    prog[0].op = BTO_INSTR_COMBINE;
    prog[0].n = 4;
    prog[0].out = dummy;
    prog[0].src1 = 3;
    prog[0].src2 = -1;
    int bad = -2;
    if (bto_program_check(prog, 1, &bad) != BTO_ERR_INVALID_VALUE || bad != 0) return 15;
    prog[0].src1 = -1;
    if (bto_program_check(prog, 1, &bad) != BTO_OK || bad != -1) return 16;
    printf("ok\n");
    return 0;
}
"""


def test_c_client(tmp_path):
    lib = build.build()
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", os.path.dirname(lib), "-lbto",
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
