"""The cluster form's exact fixed-point dot products (csrc/cg_exact.cuh), built for the
host and checked against exact rational arithmetic: the rounding of an integer sum to
fp64 (nearest, ties to even, subnormal results, overflow) and the three-level sum
(warp, CTA, cluster) of fp64 terms within its truncation bound."""
import math
import os
import random
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GUARD = 10


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = tmp_path_factory.mktemp("exact") / "exact_sum_driver"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe), os.path.join(HERE, "exact_sum_driver.cpp")],
                   check=True)
    return exe


def run(exe, lines):
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [struct.unpack("<d", int(t, 16).to_bytes(8, "little"))[0] for t in out.stdout.split()]


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def rounded(q):
    """q rounded to the nearest fp64 value, ties to even (Python's float(Fraction))."""
    try:
        return float(q)
    except OverflowError:
        return math.inf if q > 0 else -math.inf


def conv_line(T, E):
    return f"conv {T & ((1 << 128) - 1):032x} {E}"


def test_integer_to_fp64_rounds_to_nearest_even(driver):
    rng = random.Random(5)
    cases = []
    for _ in range(3000):
        nb = rng.randint(1, 80)
        T = rng.getrandbits(nb) * rng.choice((1, -1))
        E = rng.choice((1, 2, 5, 11, 40, 63, 64, 1000, 1075, 2000, 2040, 2046, rng.randint(1, 2046)))
        cases.append((T, E))
    # exact ties at several positions, both parities of the kept bit, normal and subnormal
    for sh in (1, 2, 7, 20, 27):
        for base in ((1 << 52) + 4, (1 << 52) + 5, (1 << 53) - 1):
            cases.append(((base << sh) + (1 << (sh - 1)), 1075))
            cases.append((-((base << sh) + (1 << (sh - 1))), 1075))
    # just above and below a tie, the difference far below bit 63 (the sticky bit decides)
    for base in ((1 << 52) + 4, (1 << 52) + 5):
        for d in (1, -1):
            cases.append(((base << 27) + (1 << 26) + d, 1075))
            cases.append((-((base << 27) + (1 << 26) + d), 1500))
    for m in (1, 2, 3, 5, 1023, (1 << 52) - 1, 1 << 52):
        for E in (1, 2, 3, 6, 11, 12):
            cases.append((m, E))
            cases.append((2 * m + 1, E))
    cases += [(0, 1075), ((1 << 79) - 1, 2046), (-(1 << 79), 2046), (1, 1)]
    for cmd in ("conv", "convi"):   # the rounding as used, and its integer-only path on every case
        got = run(driver, [conv_line(T, E).replace("conv", cmd, 1) for T, E in cases])
        for (T, E), g in zip(cases, got):
            want = rounded(Fraction(T) * Fraction(2) ** (E - 1075 - GUARD))
            assert bits(g) == bits(want) or (g == 0.0 and want == 0.0), (cmd, T, E, g, want)


def random_term(rng):
    kind = rng.random()
    if kind < 0.05:
        return 0.0
    if kind < 0.1:
        return rng.choice((1, -1)) * rng.randint(1, 1 << 20) * 2.0 ** -1074   # subnormal
    return rng.choice((1, -1)) * rng.random() * 2.0 ** rng.randint(-60, 60)


@pytest.mark.parametrize("w,g", [(1, 1), (32, 8), (5, 3)])
def test_three_level_sum_is_within_its_truncation_bound(driver, w, g):
    rng = random.Random(11 + w)
    sets = []
    for _ in range(300):
        n = rng.choice((1, 2, 31, 32, 33, 100, 256, 4096))
        spread = rng.choice((0, 4, 40))
        sets.append([random_term(rng) if spread == 40 else rng.choice((1, -1)) * rng.random()
                     * 2.0 ** rng.randint(-spread, spread) for _ in range(n)])
    lines = [f"sum {w} {g} {len(s)} " + " ".join(f"{bits(x):x}" for x in s) for s in sets]
    got = run(driver, lines)
    for s, res in zip(sets, got):
        exact = sum(Fraction(x) for x in s)
        emax = max(max(1, (bits(x) >> 52) & 0x7FF) for x in s)
        unit = Fraction(2) ** (emax - 1075 - GUARD)
        groups = -(-len(s) // w)
        slack = (len(s) + groups + -(-groups // g)) * unit   # truncation: below one unit per term and per entry
        assert abs(Fraction(res) - exact) <= slack + abs(Fraction(rounded(exact)) - exact) + \
            Fraction(math.ulp(abs(rounded(exact + slack)) + abs(rounded(exact - slack)))) / 2, (len(s), res)


def test_terms_on_the_common_grid_sum_exactly(driver):
    """Integers times one power of two: no truncation, so the result is the exact sum
    rounded once (the same bits as the correctly rounded rational sum)."""
    rng = random.Random(3)
    sets = []
    for _ in range(300):
        k = rng.randint(-40, 40)
        sets.append([rng.randint(-(1 << 53) + 1, (1 << 53) - 1) * 2.0 ** k for _ in range(rng.choice((2, 32, 500)))])
    got = run(driver, [f"sum 32 8 {len(s)} " + " ".join(f"{bits(x):x}" for x in s) for s in sets])
    for s, res in zip(sets, got):
        want = rounded(sum(Fraction(x) for x in s))
        assert bits(res) == bits(want) or (res == 0.0 and want == 0.0), (s[:3], res, want)


def test_non_finite_terms_give_nan(driver):
    lines = [f"sum 32 8 3 {bits(1.0):x} {bits(math.inf):x} {bits(2.0):x}",
             f"sum 32 8 2 {bits(math.nan):x} {bits(1.0):x}",
             f"sum 1 4 40 " + " ".join(f"{bits(float(i)):x}" for i in range(39)) + f" {bits(-math.inf):x}"]
    for g in run(driver, lines):
        assert math.isnan(g)
