"""CPU checks of the double-word arithmetic and the integer-pipe conversions.

csrc/dword.cuh holds the double-word (FP32 pair) operations the hybrid opening pass
computes in (Joldes, Muller and Popescu, ACM TOMS 2017) and the conversions between
binary64 and double words done on the fields of the IEEE 754 encodings.  The header
compiles for the host as well; tests/native/dword_check.cpp drives that host build, and
every result is compared here with exact rational arithmetic (fractions.Fraction):

* widen_f: binary32 -> binary64 exact (normal numbers, zero, inf, NaN; subnormals -> 0);
* dw_of: hi + lo = x to 2^-48 relative, |x - hi| <= 2^-24 |hi|, |lo| <= ulp(hi)/2;
  |x| beyond the FP32 range -> inf, NaN -> NaN;
* dw_to_double: the correctly rounded binary64 of hi + lo;
* dw_add within 3u^2, dw_mul within 7u^2, dw_mulf within 4u^2 of the exact result
  (u = 2^-24), outputs normalised (|lo| at most half the binary32 spacing at hi).
"""
import math
import shutil
import struct
import subprocess
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
U = Fraction(1, 2 ** 24)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("dword") / "dword_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{ROOT}",
                    str(ROOT / "tests" / "native" / "dword_check.cpp"), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[:len(lines)]
    return run


def f32(bits):
    return struct.unpack("<f", struct.pack("<I", bits))[0]


def b32(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def f64(bits):
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def b64(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def normalised(hi, lo):
    """hi is a nearest binary32 of hi + lo: |lo| at most half the binary32 spacing next to hi
    on lo's side (the spacing below a power of two is half the one above)."""
    if lo == 0.0:
        return True
    e = math.frexp(hi)[1] - 1                       # |hi| = m 2^e, 1 <= m < 2
    up = Fraction(2) ** (e - 23)
    toward_zero = (lo < 0) != (hi < 0)
    spacing = up / 2 if (toward_zero and abs(hi) == 2.0 ** e) else up
    return abs(Fraction(lo)) <= spacing / 2


def rand_dw(rng, e_lo=-40, e_hi=40, sub=False):
    """a normalised double word: hi random, |lo| <= ulp(hi)/2"""
    hi = np.float32(rng.choice([-1.0, 1.0]) * rng.uniform(1.0, 2.0) * 2.0 ** int(rng.integers(e_lo, e_hi)))
    e = math.frexp(float(hi))[1] - 1
    lo = np.float32(rng.uniform(-1.0, 1.0) * 2.0 ** (e - 24))
    if sub:
        lo = np.float32(rng.uniform(-1.0, 1.0) * 2.0 ** -140)
    if abs(float(lo)) > 2.0 ** (e - 24):
        lo = np.float32(0.0)
    return float(hi), float(lo)


def exact(hi, lo):
    return Fraction(hi) + Fraction(lo)


def test_widen_is_exact(checker):
    rng = np.random.default_rng(11)
    vals = [0.0, -0.0, 1.0, -1.5, 3.4e38, 1.2e-38, float("inf"), -float("inf"), float("nan"), 1e-40, -2e-45]
    vals += [s * m * 2.0 ** e for s, m, e in
             zip(rng.choice([-1.0, 1.0], 500), rng.uniform(1, 2, 500), rng.integers(-126, 128, 500))]
    vals = [float(np.float32(v)) for v in vals]          # the binary32 inputs
    got = checker([f"W {b32(v):08x}" for v in vals])
    for v, g in zip(vals, got):
        d = f64(int(g, 16))
        if math.isnan(v):
            assert math.isnan(d)
        elif v != 0.0 and abs(v) < 2.0 ** -126:          # binary32 subnormal -> signed zero
            assert d == 0.0 and math.copysign(1.0, d) == math.copysign(1.0, v)
        else:
            assert d == v and math.copysign(1.0, d) == math.copysign(1.0, v), (v, d)


def test_split_of_binary64(checker):
    rng = np.random.default_rng(12)
    xs = [float(s * m * 2.0 ** e) for s, m, e in
          zip(rng.choice([-1.0, 1.0], 3000), rng.uniform(1, 2, 3000), rng.integers(-126, 128, 3000))]
    # values one binary64 ulp either side of binary32 numbers and of rounding ties (carries)
    base = [float(np.float32(x)) for x in xs[:500]]
    xs += [math.nextafter(b, math.inf) for b in base] + [math.nextafter(b, -math.inf) for b in base]
    xs += [b + math.ulp(np.float32(b)) / 2 for b in base[:200]]
    xs += [0.0, -0.0, 1e-200, -1e-100, 2.0 ** -126, 2.0 ** -80, 2.0 ** -103, 3.4e38]
    got = checker([f"S {b64(x):016x}" for x in xs])
    for x, g in zip(xs, got):
        hs, ls = g.split()
        hi, lo = f32(int(hs, 16)), f32(int(ls, 16))
        err = abs(exact(hi, lo) - Fraction(x))
        if abs(x) >= 2.0 ** -80:
            assert err <= Fraction(2) ** -48 * abs(Fraction(x)), (x, hi, lo)
            assert abs(Fraction(x) - Fraction(hi)) <= U * abs(Fraction(hi)), (x, hi)
            assert normalised(hi, lo), (x, hi, lo)
        elif abs(x) >= 2.0 ** -126:
            assert err <= U * abs(Fraction(x)), (x, hi, lo)
        else:
            assert hi == 0.0 and lo == 0.0, (x, hi, lo)
    inf, nan, big = checker([f"S {b64(math.inf):016x}", f"S {b64(math.nan):016x}", f"S {b64(-1e300):016x}"])
    assert f32(int(inf.split()[0], 16)) == math.inf
    assert math.isnan(f32(int(nan.split()[0], 16)))
    assert f32(int(big.split()[0], 16)) == -math.inf


def test_join_is_correctly_rounded(checker):
    rng = np.random.default_rng(13)
    pairs = [rand_dw(rng, -100, 100) for _ in range(3000)] + [rand_dw(rng, -60, -50, sub=True) for _ in range(50)]
    got = checker([f"T {b32(h):08x} {b32(l):08x}" for h, l in pairs])
    for (h, l), g in zip(pairs, got):
        d = f64(int(g, 16))
        if l != 0.0 and abs(l) < 2.0 ** -126:             # subnormal low word: widened as zero
            assert d == h
        else:
            assert d == float(exact(h, l)), (h, l, d)


def _check_op(checker, op, operands, bound):
    lines = []
    for a, b in operands:
        if op == "F":
            lines.append(f"F {b32(a[0]):08x} {b32(a[1]):08x} {b32(b):08x}")
        else:
            lines.append(f"{op} {b32(a[0]):08x} {b32(a[1]):08x} {b32(b[0]):08x} {b32(b[1]):08x}")
    worst = Fraction(0)
    for (a, b), g in zip(operands, checker(lines)):
        hs, ls = g.split()
        rh, rl = f32(int(hs, 16)), f32(int(ls, 16))
        ea = exact(*a)
        eb = Fraction(b) if op == "F" else exact(*b)
        want = ea + eb if op == "A" else ea * eb
        if want == 0:
            assert rh == 0.0 and rl == 0.0
            continue
        rel = abs(exact(rh, rl) - want) / abs(want)
        worst = max(worst, rel)
        assert rel <= bound * U * U, (op, a, b, rh, rl, float(rel / (U * U)))
        assert normalised(rh, rl), (op, a, b, rh, rl)   # normalised output
    return float(worst / (U * U))


def test_double_word_sum(checker):
    rng = np.random.default_rng(14)
    ops = []
    for k in range(4000):
        a = rand_dw(rng)
        if k % 4 == 0:            # near cancellation: b close to -a
            b = rand_dw(rng, -40, 40)
            b = (float(np.float32(-a[0] * (1 + rng.uniform(-1e-6, 1e-6)))), float(np.float32(b[1] * 1e-3)))
            e = math.frexp(b[0])[1] - 1
            if abs(b[1]) > 2.0 ** (e - 24):
                b = (b[0], 0.0)
        elif k % 4 == 1:          # very different magnitudes
            b = rand_dw(rng, -80, -60)
        else:
            b = rand_dw(rng)
        ops.append((a, b))
    worst = _check_op(checker, "A", ops, 3)
    assert worst <= 3


def test_double_word_products(checker):
    rng = np.random.default_rng(15)
    ops = [(rand_dw(rng, -30, 30), rand_dw(rng, -30, 30)) for _ in range(4000)]
    assert _check_op(checker, "M", ops, 7) <= 7
    opsf = [(rand_dw(rng, -30, 30), float(np.float32(rng.choice([-1, 1]) * rng.uniform(1, 2) * 2.0 ** int(rng.integers(-30, 30)))))
            for _ in range(4000)]
    assert _check_op(checker, "F", opsf, 4) <= 4
