"""The integer-only FP32 -> 2^-32 fixed-point conversion used for the
per-cluster sums of log q (csrc/fixedpoint.h), compiled for the host and
checked against rounding the exact product x * 2^32 to nearest even in FP64:
exhaustively over every FP32 value whose scaled magnitude needs rounding
(|x| in [2^-33, 2^-9)), on samples elsewhere, on ties, and on saturation."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>
#include "fixedpoint.h"

static float f_of(uint32_t b) { float x; memcpy(&x, &b, 4); return x; }
static uint64_t rng = 0x9E3779B97F4A7C15ull;
static uint32_t next(void) {            /* splitmix64 */
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)(z ^ (z >> 31));
}
static long bad = 0;
static void check(float x, int64_t want) {
    int64_t got = fixed32_from_float(x);
    if (got != want && bad++ < 10) printf("x=%a got %lld want %lld\n", x, (long long)got, (long long)want);
}
static int64_t ref(float x) { return (int64_t)nearbyint((double)x * 4294967296.0); }

int main(void) {
    /* every value that needs rounding: exponent field 94 .. 117, both signs */
    for (uint32_t e = 94; e <= 117; ++e)
        for (uint32_t m = 0; m < (1u << 23); ++m)
            for (uint32_t s = 0; s < 2; ++s) {
                float x = f_of((s << 31) | (e << 23) | m);
                check(x, ref(x));
            }
    /* exact shifts (118 .. 157) and values that round to zero (0 .. 93): samples */
    for (long i = 0; i < 20000000; ++i) {
        uint32_t b = next();
        uint32_t e = (b >> 23) & 0xFF;
        if (e > 157) b = (b & 0x807FFFFFu) | ((118u + e % 40u) << 23);
        float x = f_of(b);
        check(x, ref(x));
    }
    /* ties: (k + 1/2) 2^-32 goes to the even neighbour */
    for (int k = 0; k < 64; ++k) {
        float x = (float)ldexp(k + 0.5, -32);
        int64_t even = (k % 2 == 0) ? k : k + 1;
        check(x, even);
        check(-x, -even);
    }
    /* saturation (|x| >= 2^31), infinities and NaN */
    const int64_t mx = 9223372036854775807LL, mn = -9223372036854775807LL - 1;
    check(2147483648.0f, mx);
    check(-2147483648.0f, mn);
    check(f_of(0x7F7FFFFFu), mx);
    check(f_of(0x7F800000u), mx);
    check(f_of(0xFF800000u), mn);
    check(f_of(0x7FC00000u), 0);
    check(f_of(0x4EFFFFFFu), ref(f_of(0x4EFFFFFFu)));   /* largest below 2^31 */
    check(0.0f, 0);
    check(-0.0f, 0);
    printf("bad %ld\n", bad);
    return bad != 0;
}
"""


def test_fixed_point_conversion_matches_exact_rounding(tmp_path):
    cc = shutil.which("g++") or shutil.which("c++")
    if cc is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "fx.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "fx"
    subprocess.run([cc, "-O2", "-I", os.path.join(ROOT, "paper_1812_10048_gb300", "csrc"),
                    str(src), "-o", str(exe), "-lm"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
