"""The residual kernel's integer form of (x - y)^2 against IEEE binary64 (CPU).

The GPU's binary64 pipe is narrow, so the residual kernel computes d = RN64(x - y) and
q = RN64(d * d) for binary32 inputs with integer operations (csrc/exact_sqdiff.h), falling back to
binary64 instructions outside its range.  Close pairs first try a shorter path: a binary32
difference shown exact by TwoSum, squared exactly in 48 bits.  The header also compiles for the host; this test builds
a small driver with the host compiler and compares the integer path with the host's IEEE binary64
arithmetic on random pairs (any bits, close values, every exponent gap), on pairs whose D^2 needs a
round-half-to-even decision, and on special values.
"""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_05657_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <random>
#include "exact_sqdiff.h"
static uint64_t ieee(uint32_t ux, uint32_t uy) {
    float x, y;
    memcpy(&x, &ux, 4);
    memcpy(&y, &uy, 4);
    volatile double d = (double)x - (double)y;
    volatile double q = d * d;
    double qq = q;
    uint64_t b;
    memcpy(&b, &qq, 8);
    return b;
}
static uint32_t f32(uint32_t sign, uint32_t e, uint32_t m) { return (sign << 31) | (e << 23) | (m & 0x7fffffu); }
int main(int argc, char **argv) {
    const uint64_t n = strtoull(argv[1], 0, 10);
    std::mt19937_64 rng(1809);
    uint64_t total = 0, fast = 0, bad = 0, ties = 0, exact = 0;
    auto check = [&](uint32_t ux, uint32_t uy) {
        uint64_t q;
        total++;
        float x, y;
        memcpy(&x, &ux, 4);
        memcpy(&y, &uy, 4);
        if (hda::sqdiff_f32_exact(x, y, q)) {
            exact++;
            if (q != ieee(ux, uy)) {
                if (bad < 5) printf("exact-path mismatch %08x %08x\n", ux, uy);
                bad++;
            }
        }
        if (!hda::sqdiff_f32_bits(ux, uy, q)) return;
        fast++;
        if (q != ieee(ux, uy)) {
            if (bad < 5) printf("mismatch %08x %08x\n", ux, uy);
            bad++;
        }
    };
    for (uint64_t i = 0; i < n; i++) {
        const uint64_t r = rng();
        const uint32_t ux = (uint32_t)r;
        uint32_t uy;
        switch ((r >> 32) & 3) {
        case 0: uy = (uint32_t)(r >> 32); break;                                            // any bits
        case 1: uy = ux + (uint32_t)((int64_t)((r >> 40) % 2000001) - 1000000); break;      // close
        case 2: {                                                                            // gap 0..59
            const uint32_t g = (uint32_t)((r >> 40) % 60);
            uy = (ux & 0x807fffffu) | (((((ux >> 23) & 0xffu) + 256u - 30u + g) & 0xffu) << 23);
            uy ^= (uint32_t)(r >> 50) & 0x7fffu;
            break;
        }
        default: uy = ux ^ (1u << ((r >> 40) & 31)); break;                                  // one bit
        }
        check(ux, uy);
    }
    // ties: D odd with D^2 of 54 bits (the last bit shifted out is the only one): exponents 3
    // apart, D = 8 Mx - My
    for (uint64_t D = 94906267ull; D < 134217728ull; D += 2 * 1009) {
        const uint64_t my0 = (1u << 23) + (rng() % (1u << 22));
        const uint64_t my = my0 + (8 - (D + my0) % 8) % 8;
        const uint64_t mx = (D + my) / 8;
        if (mx < (1u << 23) || mx >= (1u << 24) || my >= (1u << 24)) continue;
        const uint32_t e = 100 + (uint32_t)(rng() % 50);
        check(f32(0, e + 3, (uint32_t)mx), f32(0, e, (uint32_t)my));
        ties++;
    }
    const uint32_t sp[] = {0u, 0x80000000u, 0x3f800000u, 0xbf800000u, 0x00800000u, 0x7f7fffffu, 0xff7fffffu,
                           0x3f800001u, 0x3effffffu, 0x4b800000u, 0x33800000u, 0x007fffffu, 0x7f800000u,
                           0xff800000u, 0x7fc00000u, 0x00000001u};
    for (uint32_t a : sp)
        for (uint32_t b : sp) check(a, b);
    // residual-like pairs: a value and its neighbour after one more averaging step, the common
    // case of the exact path
    for (uint64_t i = 0; i < n / 4; i++) {
        const uint64_t r = rng();
        const uint32_t ux = 0x3c000000u + (uint32_t)(r % 0x3000000u);  // about 2^-7 .. 2^-1
        const uint32_t uy = ux + (uint32_t)((int64_t)((r >> 32) % 4097) - 2048);
        check(ux, uy);
    }
    printf("%llu %llu %llu %llu %llu\n", (unsigned long long)total, (unsigned long long)fast,
           (unsigned long long)bad, (unsigned long long)ties, (unsigned long long)exact);
    return 0;
}
"""


def test_integer_square_difference_matches_ieee_binary64():
    cxx = os.environ.get("CXX", "g++")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "drv.cpp")
        exe = os.path.join(d, "drv")
        open(src, "w").write(DRIVER)
        r = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe, src],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no host C++ compiler: %s" % r.stderr[:200])
        out = subprocess.run([exe, "20000000"], capture_output=True, text=True, check=True).stdout.split()
    total, fast, bad, ties, exact = (int(v) for v in out)
    assert bad == 0
    assert fast > total // 2  # the integer path serves most pairs
    assert exact > total // 5  # close pairs take the exact-difference path
    assert ties > 10000
