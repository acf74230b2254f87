"""Host check of the integer-pipe binary64 <-> binary32 conversions
(paper_2006_07964_gb300/csrc/fpconv.h) against the C casts, which round to
nearest with ties to even (IEEE-754).  The mixed form's RK stage uses them
for its FP32 increment and its FP32 state copy.

Documented differences, checked as such: no binary32 subnormal is produced
or read (magnitudes below 2^-126 become a signed zero), and any NaN may come
out as any NaN.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2006_07964_gb300", "csrc")

PROGRAM = r"""
#include "fpconv.h"
#include <float.h>
#include <math.h>
#include <stdio.h>

static uint64_t st = 0x2006079640000001ull;
static uint64_t next64(void) {   /* splitmix64 */
    uint64_t z = (st += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static long bad = 0, n_tie = 0, n_flush = 0, n_exact = 0;

static void check_d2f(double x) {
    const float got = hx_f64_to_f32(x), want = (float)x;
    if (isnan(x)) { if (!isnan(got)) ++bad; return; }
    if (fabs(x) < FLT_MIN) {
        ++n_flush;
        if (hx_bits_f32(got) != (signbit(x) ? 0x80000000u : 0u)) ++bad;
        return;
    }
    ++n_exact;
    if (hx_bits_f32(got) != hx_bits_f32(want)) {
        if (bad < 5) printf("d2f %a: got %a want %a\n", x, (double)got, (double)want);
        ++bad;
    }
}

static void check_f2d(float f) {
    const double got = hx_f32_to_f64(f);
    if (isnan(f)) { if (!isnan(got)) ++bad; return; }
    if (f != 0.0f && fabsf(f) < FLT_MIN) {
        if (hx_bits_f64(got) != (signbit(f) ? 0x8000000000000000ull : 0ull)) ++bad;
        return;
    }
    if (hx_bits_f64(got) != hx_bits_f64((double)f)) {
        if (bad < 5) printf("f2d %a: got %a\n", (double)f, got);
        ++bad;
    }
}

int main(void) {
    /* special and boundary values */
    const double sp[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, -NAN, DBL_MAX, -DBL_MAX, DBL_MIN,
                         FLT_MAX, -FLT_MAX, FLT_MIN, -FLT_MIN, 0x1.fffffefffffffp127, 0x1.ffffffp127,
                         0x1.fffffep127, 0x1.ffffff000001p127, 0x1p128, 0x1.fffffffffffffp-127,
                         0x1p-127, 0x1p-149, 0x1.0000010000000p0, 0x1.0000030000000p0, 3.0e38, 1.0e-300};
    for (unsigned i = 0; i < sizeof sp / sizeof sp[0]; ++i) check_d2f(sp[i]);
    /* random bit patterns (all classes), values of the solver's scale, exact ties */
    for (long i = 0; i < 4000000; ++i) {
        const uint64_t r = next64();
        check_d2f(hx_f64_from_bits(r));
        check_f2d(hx_f32_from_bits((uint32_t)r));
        check_f2d(hx_f32_from_bits((uint32_t)(r >> 32)));
        const double v = ((double)(r >> 11) / 9007199254740992.0 - 0.5) * ldexp(1.0, (int)(r & 63) - 32);
        check_d2f(v);
        /* halfway between a float and its successor, both signs */
        const float a = hx_f32_from_bits((uint32_t)(r >> 32) & 0x7f7fffffu);
        if (a >= FLT_MIN && a < FLT_MAX) {
            const double mid = 0.5 * ((double)a + (double)nextafterf(a, INFINITY));
            ++n_tie;
            check_d2f(mid);
            check_d2f(-mid);
        }
    }
    printf("bad %ld exact %ld flushed %ld ties %ld\n", bad, n_exact, n_flush, n_tie);
    return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_fpconv_matches_c_casts(tmp_path):
    src = tmp_path / "fpconv_check.c"
    exe = tmp_path / "fpconv_check"
    src.write_text(PROGRAM)
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", CSRC, str(src), "-o", str(exe), "-lm"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    fields = dict(zip(out.stdout.split()[0::2], map(int, out.stdout.split()[1::2])))
    assert fields["bad"] == 0
    assert fields["exact"] > 4_000_000 and fields["ties"] > 1_000_000 and fields["flushed"] > 100_000
