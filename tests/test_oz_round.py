"""The Ozaki combine's integer arithmetic (csrc/oz_round.cuh), compiled for the
host.  The digit sums S = sum_d q_d 2^(beta (s-1-d)) must equal the exact
integer (Python) as 128-bit two's complement words, both the generic loop and
the fixed-(s, beta) Horner halves; the rounding's bit pattern must equal
ldexp(fma((double)hi, 2^64, (double)lo), e2), the FP64 evaluation it replaces,
computed here exactly with Python integers (int -> float conversion rounds to
nearest, ties to even)."""
import math
import os
import struct
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_1403_5044_b300", "csrc", "oz_round.cuh")

DRIVER = r'''
#include <cstdio>
#include <cstring>
#include "oz_round.cuh"
template <int S, int B> void horner(const int32_t *q, int64_t &h, uint64_t &l) { oz_horner<S, B>(q, h, l); }
int main(int argc, char **argv) {
    if (argc > 1) {   // digit sums: lines "s beta q_0 .. q_(s-1)"
        int s, beta;
        while (scanf("%d %d", &s, &beta) == 2) {
            int32_t q[16];
            for (int d = 0; d < s; ++d) scanf("%d", &q[d]);
            int64_t h1, h2 = 0; uint64_t l1, l2 = 0;
            oz_sum_any(q, s, beta, h1, l1);
            if (s == 10 && beta == 6) horner<10, 6>(q, h2, l2);
            else if (s == 8 && beta == 7) horner<8, 7>(q, h2, l2);
            else if (s == 12 && beta == 5) horner<12, 5>(q, h2, l2);
            else if (s == 7 && beta == 8) horner<7, 8>(q, h2, l2);
            else { h2 = h1; l2 = l1; }
            printf("%lld %llu %lld %llu\n", (long long)h1, (unsigned long long)l1, (long long)h2, (unsigned long long)l2);
        }
        return 0;
    }
    long long hi; unsigned long long lo; int e2;
    while (scanf("%lld %llu %d", &hi, &lo, &e2) == 3) {
        bool fb;
        unsigned long long b = oz_round_bits(hi, lo, e2, &fb);
        printf("%llu %d\n", b, fb ? 1 : 0);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("ozr")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)])
    return str(exe)


def ldexp(x, e):
    try:
        return math.ldexp(x, e)
    except OverflowError:   # IEEE: +-inf
        return math.copysign(math.inf, x)


def reference(hi, lo, e2):
    v = float(hi * 2 ** 64 + int(float(lo)))   # RN(lo), then RN of the exact sum
    return ldexp(v, e2)


def cases():
    rng = np.random.default_rng(20260)
    out = []
    for _ in range(4000):   # the combine's range: |S| < 2^80
        hi = int(rng.integers(-2 ** 16, 2 ** 16))
        lo = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        out.append((hi, lo, int(rng.integers(-200, 200))))
    for _ in range(2000):   # small magnitudes of both signs
        v = int(rng.integers(-2 ** 62, 2 ** 62)) >> int(rng.integers(0, 62))
        out.append((-1 if v < 0 else 0, v % 2 ** 64, int(rng.integers(-80, 80))))
    for k in range(1, 12):   # ties and near-ties of the low word's rounding (bit length 64)
        for q in (2 ** 53 - 1, 2 ** 53 - 2, 2 ** 52 + 1, 2 ** 52):
            base = q << k
            if base >= 2 ** 64:
                continue
            for d in (-1, 0, 1):
                lo = (base | (1 << (k - 1))) + d
                if 0 <= lo < 2 ** 64:
                    for hi in (0, 1, -1, 2 ** 15, -2 ** 15):
                        out.append((hi, lo, 0))
    for hi in (-3, -2, -1, 0, 1, 2):   # the low word rounding up to 2^64
        for lo in (2 ** 64 - 1, 2 ** 64 - 1024, 2 ** 64 - 1025, 2 ** 64 - 2048, 2 ** 63):
            out.append((hi, lo, 3))
    for e2 in (-1100, -1074, -1030, -1022, 960, 1000, 1023):   # the ldexp fallback
        out.append((5, 12345, e2))
        out.append((-7, 99, e2))
    out.append((0, 0, 17))
    return out


def test_integer_rounding_matches_the_fp64_evaluation(prog):
    cs = cases()
    inp = "".join("%d %d %d\n" % c for c in cs)
    res = subprocess.run([prog], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    bad = []
    nfb = 0
    for (hi, lo, e2), line in zip(cs, res):
        b, fb = (int(x) for x in line.split())
        got = struct.unpack("<d", struct.pack("<Q", b))[0]
        if fb:
            nfb += 1
            got = ldexp(got, e2)   # the caller's fallback
        want = reference(hi, lo, e2)
        if struct.pack("<d", got) != struct.pack("<d", want):
            bad.append((hi, lo, e2, got, want))
    assert not bad, bad[:5]
    assert nfb >= 8   # the out-of-range cases took the fallback


def test_digit_sums_are_the_exact_integer(prog):
    rng = np.random.default_rng(7)
    rows = []
    for s, beta in ((10, 6), (8, 7), (12, 5), (7, 8), (14, 4)):
        for k in range(400):
            lim = 2 ** 25 - 1 if k % 4 else 2 ** int(rng.integers(1, 25))
            q = [int(v) for v in rng.integers(-lim, lim + 1, size=s)]
            if k == 0:
                q = [2 ** 25 - 1] * s
            elif k == 1:
                q = [-(2 ** 25 - 1)] * s
            rows.append((s, beta, q))
    inp = "".join("%d %d %s\n" % (s, b, " ".join(map(str, q))) for s, b, q in rows)
    out = subprocess.run([prog, "sums"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (s, beta, q), line in zip(rows, out):
        h1, l1, h2, l2 = (int(x) for x in line.split())
        S = sum(v * 2 ** (beta * (s - 1 - d)) for d, v in enumerate(q))
        want_hi, want_lo = S >> 64, S % 2 ** 64   # floor division: two's complement words
        assert (h1, l1) == (want_hi, want_lo), (s, beta, q)
        assert (h2, l2) == (want_hi, want_lo), (s, beta, q)
