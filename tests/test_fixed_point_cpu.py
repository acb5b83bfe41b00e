"""The integer-to-FP64 rounding of the tensor-core epilogues (fixed_to_bits in
tc_ptx.cuh: V = hi 2^32 + lo, |V| < 2^75, times 2^sc) against exact round-to-
nearest-even of the 128-bit integer, on the host.  The routine is
__host__ __device__; the test compiles it with g++ from the header itself."""
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
static double ref_round(__int128 V, int sc) {
    __int128 av = V < 0 ? -V : V;
    if (av == 0) return 0.0;
    int p = 0; __int128 t = av; while (t >>= 1) p++;
    double r;
    if (p <= 52) r = (double)(long long)av;
    else {
        int sh = p - 52; __int128 q = av >> sh, rem = av - (q << sh), half = ((__int128)1) << (sh - 1);
        unsigned long long m = (unsigned long long)q; if (rem > half || (rem == half && (m & 1))) m++;
        r = ldexp((double)m, sh);
    }
    r = ldexp(r, sc);
    return V < 0 ? -r : r;
}
int main() {
    std::mt19937_64 g(11);
    long bad = 0, n = 0;
    auto rnd = [&](int bits) { long long v = (long long)(g() >> (64 - bits)); return (g() & 1) ? -v : v; };
    for (long it = 0; it < 3000000; ++it) {
        long long hi, lo;
        switch (it %% 7) {
            case 0: hi = rnd(43); lo = rnd(51); break;
            case 1: hi = 0; lo = rnd(1 + g() %% 50); break;
            case 2: hi = rnd(1 + g() %% 42); lo = rnd(1 + g() %% 50); break;
            case 3: hi = (long long)(g() %% 5) - 2; lo = rnd(33); break;
            case 4: hi = rnd(31); lo = ((long long)(g() %% 3) - 1) << 32; break;
            case 5: hi = rnd(43); lo = ((long long)(g() & 0xFFF)) << (g() %% 40); if (g() & 1) lo = -lo; break;
            default: {  // exact ties of the 53-bit rounding
                const int b = 54 + (int)(g() %% 20);
                __int128 V = ((__int128)((g() | 1ULL) >> 11) << (b - 53)) | ((__int128)1 << (b - 54));
                if (g() & 1) V = -V;
                hi = (long long)(V >> 32); lo = (long long)(V - ((__int128)hi << 32));
            }
        }
        const int sc = (int)(g() %% 200) - 100;
        const __int128 V = ((__int128)hi << 32) + lo;
        bool ok; int E;
        const unsigned long long bits = fixed_to_bits(hi, lo, sc, ok, E);
        if (!ok) continue;
        ++n;
        double got; memcpy(&got, &bits, 8);
        const double ref = ref_round(V, sc);
        if (got != ref) { if (bad < 5) printf("mismatch hi=%%lld lo=%%lld sc=%%d\n", hi, lo, sc); ++bad; }
    }
    printf("checked %%ld bad %%ld\n", n, bad);
    return bad != 0 || n < 2000000;
}
"""


def _extract():
    src = open(HEADER).read()
    a = src.index("__host__ __device__ __forceinline__ int clz64_any")
    b = src.index("\n}\n", src.index("fixed_to_bits(")) + 3
    return src[a:b]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_fixed_to_bits_rounds_like_exact_int128():
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "f2b.cpp")
        exe = os.path.join(d, "f2b")
        with open(cpp, "w") as f:
            f.write(HARNESS % _extract())
        subprocess.run(["g++", "-O2", "-std=c++17", cpp, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert re.search(r"bad 0$", r.stdout.strip())
