"""The integer-to-FP64 step of the tensor-core epilogues (tc_ptx.cuh), on the
host, against exact 128-bit integer arithmetic:

* ozaki_window8 / sgemm_window10 are floor(V / 2^8) and floor(V / 2^10) of
  the fixed-point recombination V of the slice levels, for levels up to the
  bounds the kernels guarantee;
* window_to_double(x, sc) is x 2^sc rounded to nearest with ties away from
  zero, a signed zero below 2^-1022 and an infinity from 2^1024 on;
* levels4_to_i64 is D_0 2^24 + D_1 2^16 + D_2 2^8 + D_3 for FP32 levels up
  to 2^22 in magnitude, and exact_to_double(V, sc) is V 2^sc (no rounding for
  |V| < 2^53) with the same flush and saturation;
* grid32(x, e) is trunc(|x| 2^(32 - e)) for |x| < 2^e, and bf16_digit_pair
  the exact BF16 of one byte of each of two such values; grid33 and
  f16_digit_pair the same for 33 bits and 11-bit FP16 digits;
* mul_pairs and h3_signed_digits give the signed 11-bit digits of a product
  of two FP32 pairs within 2^-23 + 2^-25 of the exact product (in units of
  the leading digit), and f16_int_pair encodes them exactly.

The routines are __host__ __device__; the test compiles them with g++ from
the header itself."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2112_10526_gb300", "csrc", "tc_ptx.cuh")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <random>
#define __host__
#define __device__
#define __forceinline__ inline
%s
typedef __int128 i128;
static i128 floor_shift(i128 v, int s) {  // floor(v / 2^s), written without >>
    const i128 p = (i128)1 << s;
    i128 q = v / p;
    if (v %% p != 0 && v < 0) q -= 1;
    return q;
}
// x 2^sc, ties away from zero, flushed / saturated like the kernels
static double ref_round(long long x, int sc) {
    const bool neg = x < 0;
    unsigned long long m = neg ? 0ULL - (unsigned long long)x : (unsigned long long)x;
    if (m == 0) return neg ? -0.0 : 0.0;
    int bl = 0; for (unsigned long long t = m; t; t >>= 1) ++bl;
    unsigned long long q = m; int sh = 0;
    if (bl > 53) {
        sh = bl - 53;
        const unsigned long long rem = m & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
        q = m >> sh;
        if (rem >= half) ++q;
    }
    int qbl = 0; for (unsigned long long t = q; t; t >>= 1) ++qbl;
    const int e = qbl - 1 + sh + sc;  // exponent of the leading one after rounding
    double r;
    if (e < -1022) r = 0.0;
    else if (e > 1023) r = INFINITY;
    else r = ldexp((double)q, sh + sc);
    return neg ? -r : r;
}
static bool same(double a, double b) { return memcmp(&a, &b, 8) == 0; }
int main() {
    std::mt19937_64 g(11);
    long bad = 0, n = 0;
    auto rnd_bound = [&](long long bound) {  // uniform-ish in [-bound, bound], often near the ends
        long long v;
        switch (g() %% 4) {
            case 0: v = bound; break;
            case 1: v = bound - (long long)(g() %% 1000); break;
            case 2: v = (long long)(g() %% (unsigned long long)(bound + 1)); break;
            default: v = (long long)(g() >> (64 - 1 - (int)(g() %% 24)));
        }
        if (v > bound) v = bound;
        return (g() & 1) ? -v : v;
    };
    // 1. the Ozaki window: |D_g| <= (g - 1) 64 255^2
    for (long it = 0; it < 1000000; ++it) {
        int d[7];
        for (int i = 0; i < 7; ++i) d[i] = (int)rnd_bound((long long)(i + 1) * 64 * 255 * 255);
        i128 V = 0;
        for (int i = 0; i < 7; ++i) V += (i128)d[i] << (8 * (6 - i));
        ++n;
        if ((i128)ozaki_window8(d) != floor_shift(V, 8)) { if (bad < 5) printf("ozaki window %%ld\n", it); ++bad; }
    }
    // 2. the S-GEMM window: |D_t| <= 255 x 65792 < 2^24
    for (long it = 0; it < 1000000; ++it) {
        int d[7];
        const int SB = 1 + (int)(g() %% 7);
        for (int i = 0; i < 7; ++i) d[i] = i < SB ? (int)rnd_bound(255LL * 65792) : 0;
        i128 V = 0;
        for (int i = 0; i < 7; ++i) V += (i128)d[i] << (8 * (6 - i));
        ++n;
        if ((i128)sgemm_window10(d) != floor_shift(V, 10)) { if (bad < 5) printf("sgemm window %%ld\n", it); ++bad; }
    }
    // 3. the rounding: random bit lengths, exact ties, carries into the next
    //    binade, and scales across both ends of the exponent range
    for (long it = 0; it < 3000000; ++it) {
        long long x;
        const int kind = (int)(it %% 5);
        const int bl = 1 + (int)(g() %% 63);
        unsigned long long m = (g() >> (64 - bl)) | (1ULL << (bl - 1));
        if (kind == 1 && bl > 54) {  // an exact tie at the 53-bit rounding
            const int sh = bl - 53;
            m = (m >> sh << sh) | (1ULL << (sh - 1));
            m &= ~((1ULL << (sh - 1)) - 1);
            m |= 1ULL << (sh - 1);
        } else if (kind == 2 && bl > 53) {  // all ones: rounds up to the next power of two
            m = (bl == 64) ? ~0ULL >> 1 : ((1ULL << bl) - 1);
        } else if (kind == 3) {
            m = (unsigned long long)(g() %% 3);
        }
        m &= ~(1ULL << 63);
        x = (g() & 1) ? -(long long)m : (long long)m;
        int sc;
        switch (g() %% 3) {
            case 0: sc = (int)(g() %% 200) - 100; break;
            case 1: sc = -1085 + (int)(g() %% 80); break;   // near the flush to zero
            default: sc = 960 + (int)(g() %% 80);           // near the saturation
        }
        ++n;
        const double got = window_to_double(x, sc), ref = ref_round(x, sc);
        if (!same(got, ref) && !(m == 0 && got == 0.0 && ref == 0.0)) {
            if (bad < 5) printf("round x=%%lld sc=%%d got %%a ref %%a\n", x, sc, got, ref);
            ++bad;
        }
    }
    // 4. the 4-level combination: |D_t| < 2^22, exact FP32 integers
    for (long it = 0; it < 1000000; ++it) {
        long long d[4];
        for (int i = 0; i < 4; ++i) d[i] = rnd_bound((1LL << 22) - 1);
        const long long want = (d[0] << 24) + (d[1] << 16) + (d[2] << 8) + d[3];
        ++n;
        if (levels4_to_i64((float)d[0], (float)d[1], (float)d[2], (float)d[3]) != want) {
            if (bad < 5) printf("levels4 %%ld\n", it);
            ++bad;
        }
    }
    // 5. the exact conversion: |V| < 2^53 at every scale
    for (long it = 0; it < 1000000; ++it) {
        const int bl = (int)(g() %% 54);
        unsigned long long m = bl == 0 ? 0ULL : ((g() >> (64 - bl)) | (1ULL << (bl - 1)));
        const long long x = (g() & 1) ? -(long long)m : (long long)m;
        int sc;
        switch (g() %% 3) {
            case 0: sc = (int)(g() %% 200) - 100; break;
            case 1: sc = -1075 + (int)(g() %% 80); break;
            default: sc = 960 + (int)(g() %% 80);
        }
        ++n;
        const double got = exact_to_double(x, sc), ref = ref_round(x, sc);
        if (!same(got, ref) && !(m == 0 && got == 0.0 && ref == 0.0)) {
            if (bad < 5) printf("exact x=%%lld sc=%%d got %%a ref %%a\n", x, sc, got, ref);
            ++bad;
        }
    }
    // 6. the 4-slice digits: grid32 is trunc(|x| 2^(32 - e)) (ldexp is exact
    //    here), bf16_digit_pair the BF16 of a byte of each of two such values
    for (long it = 0; it < 1000000; ++it) {
        const int e = (int)(g() %% 200) - 100;
        const int bl = (int)(g() %% 70);  // |x| / 2^e from 2^-70 up to just below 1
        double x = ldexp((double)(g() >> 11) / 9007199254740992.0, e - bl);
        if (g() & 1) x = -x;
        if (!(fabs(x) < ldexp(1.0, e))) continue;
        uint32_t sg;
        const uint32_t y = grid32(x, e, sg);
        const uint32_t want = (uint32_t)floor(ldexp(fabs(x), 32 - e));
        ++n;
        if (y != want || sg != (std::signbit(x) ? 1u : 0u)) {
            if (bad < 5) printf("grid32 x=%%a e=%%d got %%u want %%u\n", x, e, y, want);
            ++bad;
        }
        const uint32_t y1 = (uint32_t)(g() >> 32);
        for (uint32_t byte = 0; byte < 4; ++byte) {
            const uint32_t pr = bf16_digit_pair(y, y1, byte, 0x80000000u);
            const uint32_t lo = pr & 0xFFFFu, hi2 = pr >> 16;
            float flo, fhi;
            const uint32_t blo = lo << 16, bhi = hi2 << 16;
            memcpy(&flo, &blo, 4);
            memcpy(&fhi, &bhi, 4);
            if (flo != (float)((y >> (8 * byte)) & 255u) || fhi != -(float)((y1 >> (8 * byte)) & 255u)) {
                if (bad < 5) printf("digit pair byte %%u of %%u %%u\n", byte, y, y1);
                ++bad;
            }
        }
    }
    // 7. the 3-slice FP16 digits: grid33 is trunc(|x| 2^(33 - e)); the FP16
    //    digit pairs hold the 11-bit fields of two such values exactly
    for (long it = 0; it < 1000000; ++it) {
        const int e = (int)(g() %% 200) - 100;
        const int bl = (int)(g() %% 70);
        double x = ldexp((double)(g() >> 11) / 9007199254740992.0, e - bl);
        if (g() & 1) x = -x;
        if (!(fabs(x) < ldexp(1.0, e))) continue;
        uint32_t sg;
        const unsigned long long y = grid33(x, e, sg);
        const unsigned long long want = (unsigned long long)floor(ldexp(fabs(x), 33 - e));
        ++n;
        if (y != want || sg != (std::signbit(x) ? 1u : 0u)) {
            if (bad < 5) printf("grid33 x=%%a e=%%d got %%llu want %%llu\n", x, e, y, want);
            ++bad;
        }
        const unsigned long long y1 = g() >> 31;
        for (int sh = 0; sh <= 22; sh += 11) {
            const uint32_t pr = f16_digit_pair(y, y1, sh, 0x80000000u);
            const uint32_t d0 = (uint32_t)(y >> sh) & 0x7FFu, d1 = (uint32_t)(y1 >> sh) & 0x7FFu;
            // decode the two FP16 halves
            auto dec = [](uint32_t hb) {
                const int ex = (int)((hb >> 10) & 0x1F), mt = (int)(hb & 0x3FF);
                const double v = ex == 0 ? ldexp((double)mt, -24) : ldexp(1.0 + mt / 1024.0, ex - 15);
                return (hb & 0x8000u) ? -v : v;
            };
            if (dec(pr & 0xFFFFu) != (double)d0 || dec(pr >> 16) != -(double)d1) {
                if (bad < 5) printf("f16 digit pair shift %%d of %%llu %%llu\n", sh, y, y1);
                ++bad;
            }
        }
    }
    // 8. the 3-slice digits of the CG's J^T g operand, from FP32 pairs: t and
    //    g'' as pairs (hi = fl32(x), lo = fl32(x - hi)), x = t g'' 2^(11 - cT)
    //    with |t| < 2^cT and |g''| < 1.  d0 + 2^-11 d1 + 2^-22 d2 must lie
    //    within 2^-23 + 2^-25 of x (plus 2^-40 for the dropped lo x lo term
    //    and the pair product's roundings), the digits must be integers with
    //    |d0| <= 2048, |d1| <= 1025, |d2| <= 1024, and the FP16 pairs must
    //    hold them exactly.
    auto dec16 = [](uint32_t hb) {
        const int ex = (int)((hb >> 10) & 0x1F), mt = (int)(hb & 0x3FF);
        const double v = ex == 0 ? ldexp((double)mt, -24) : ldexp(1.0 + mt / 1024.0, ex - 15);
        return (hb & 0x8000u) ? -v : v;
    };
    long near_edge = 0;
    for (long it = 0; it < 1000000; ++it) {
        const int cT = -(int)(g() %% 60);
        const int drop = (g() %% 4 == 0) ? (int)(g() %% 40) : 0;  // entries far below the column bound
        double t = ldexp((double)(g() >> 11) / 9007199254740992.0, cT - drop);
        if (it %% 7 == 3) t = ldexp(1.0 - ldexp(1.0, -53), cT);  // just below the bound
        if (g() %% 50 == 0) t = 0.0;
        if (g() & 1) t = -t;
        double gg = (double)(g() >> 11) / 9007199254740992.0;
        if (g() %% 4 == 0) gg = ldexp(gg, -(int)(g() %% 30));
        if (it %% 7 == 3) gg = 1.0 - ldexp(1.0, -53);
        if (g() & 1) gg = -gg;
        const float th = (float)t, tl = (float)(t - (double)th);
        const float gh = (float)gg, gl = (float)(gg - (double)gh);
        float ph, pl, d0, d1, d2;
        mul_pairs(th, tl, gh, gl, ph, pl);
        const float sc = ldexpf(1.0f, 11 - cT);
        h3_signed_digits(ph * sc, pl * sc, d0, d1, d2);
        const long double x = (long double)t * (long double)gg * ldexpl(1.0L, 11 - cT);
        const long double approx = (long double)d0 + ldexpl((long double)d1, -11) + ldexpl((long double)d2, -22);
        const long double err = fabsl(approx - x);
        const bool ints = d0 == rintf(d0) && d1 == rintf(d1) && d2 == rintf(d2);
        const bool range = fabsf(d0) <= 2048.f && fabsf(d1) <= 1025.f && fabsf(d2) <= 1024.f;
        if (fabsl(x) > 2047.0L) ++near_edge;
        ++n;
        if (!ints || !range || !(err <= ldexpl(1.0L, -23) + ldexpl(1.0L, -25) + ldexpl(1.0L, -40))) {
            if (bad < 5) printf("h3 digits t=%%a g=%%a cT=%%d: %%g %%g %%g err %%Lg\n", t, gg, cT, d0, d1, d2, err);
            ++bad;
        }
        const uint32_t p01 = f16_int_pair(d0, d1), p2 = f16_int_pair(d2, -d0);
        if (dec16(p01 & 0xFFFFu) != (double)d0 || dec16(p01 >> 16) != (double)d1 ||
            dec16(p2 & 0xFFFFu) != (double)d2 || dec16(p2 >> 16) != -(double)d0) {
            if (bad < 5) printf("f16 int pair %%g %%g %%g\n", d0, d1, d2);
            ++bad;
        }
    }
    if (near_edge < 1000) { printf("too few cases near |x| = 2^11: %%ld\n", near_edge); ++bad; }
    printf("checked %%ld bad %%ld\n", n, bad);
    return bad != 0 || n < 8800000;
}
"""


def _extract():
    src = open(HEADER).read()
    a = src.index("__host__ __device__ __forceinline__ int clz64_any")
    b = src.index("\n}\n", src.index("uint32_t f16_int_pair(")) + 3
    return src[a:b]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_epilogue_windows_rounding_and_exact_conversion_match_int128():
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "f2b.cpp")
        exe = os.path.join(d, "f2b")
        with open(cpp, "w") as f:
            f.write(HARNESS % _extract())
        subprocess.run(["g++", "-O2", "-std=c++17", cpp, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert re.search(r"bad 0$", r.stdout.strip())
