"""The arithmetic behind the tensor-core epilogue's sign counts, checked on the
host CPU with the C library's fmaf under round-toward-minus-infinity (IEEE 754
fused multiply-add, the same operation as the GPU's fma.rm).

A counter c in [1, 2) holds ulp 2^-23.  For |D| <= 4.25 (every D the MMA can
produce) the exact value c + D 2^-30 lies within 2^-28 of c, so rounding it
toward minus infinity gives c - 2^-23 when D < 0 and c itself when D >= 0,
minus zero included.  Starting from 1.5, the number of negative D among k <=
2^22 values is bits(1.5) - bits(c).  The cases below cover zeros of both
signs, subnormals, the largest |D| and long runs."""
import os
import shutil
import subprocess
import tempfile

import pytest

PROGRAM = r"""
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
static uint32_t bits(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
int main(void) {
    const float edge[] = {0.f, -0.f, 1e-45f, -1e-45f, 1.17549435e-38f, -1.17549435e-38f, 4.25f, -4.25f,
                          1e-7f, -1e-7f, 3e-5f, -3e-5f, 2.f, -2.f};
    const int nedge = (int)(sizeof edge / sizeof edge[0]);
    const float tiny = ldexpf(1.f, -30);
    int bad = 0;
    srand(11);
    for (int trial = 0; trial < 20000; ++trial) {
        const int len = trial == 0 ? 4096 : 64;
        float c = 1.5f;
        int want = 0;
        fesetround(FE_DOWNWARD);
        for (int i = 0; i < len; ++i) {
            float d;
            if (trial == 0) d = -1.f;  /* one long run of negatives */
            else if (rand() % 4 == 0) d = edge[rand() % nedge];
            else d = ((float)rand() / (float)RAND_MAX * 8.5f - 4.25f) * (rand() % 3 == 0 ? 1e-6f : 1.f);
            volatile float vd = d, vt = tiny, vc = c;
            c = fmaf(vd, vt, vc);
            want += d < 0.f;
        }
        fesetround(FE_TONEAREST);
        if ((int)(bits(1.5f) - bits(c)) != want) ++bad;
    }
    printf("%d\n", bad);
    return 0;
}
"""


def test_round_down_fma_counts_negative_values():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "c.c"), os.path.join(d, "c")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run([cc, "-O2", "-frounding-math", "-o", exe, src, "-lm"], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.strip()
    assert out == "0", f"{out} runs miscounted"
