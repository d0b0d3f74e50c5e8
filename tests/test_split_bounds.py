"""The split bounds behind the tensor-core rejection test, checked on the
host in exact arithmetic: for a row x and a query y split into 16-bit parts
the way the packing kernel splits them, the products the scorer keeps differ
from x.y by at most the bound the library charges (the constants of the
scorer's c and of the FP16 absolute term).  Vectors mix magnitudes over many
binades, so parts fall below the FP16 normal range and are set to zero."""
import math
from fractions import Fraction

import numpy as np
import pytest

U16 = 2.0 ** -14           # smallest FP16 normal; parts below it are set to zero


def fp16_parts(x):
    """Two FP16 parts of FP32 values (round to nearest, then zeroed below
    the FP16 normal range), remainders exact in FP32."""
    x = np.asarray(x, dtype=np.float32)
    h = x.astype(np.float16).astype(np.float32)
    h[np.abs(h) < U16] = 0.0
    r = (x - h).astype(np.float32)
    assert np.array_equal(r.astype(np.float64), x.astype(np.float64) - h.astype(np.float64))
    l = r.astype(np.float16).astype(np.float32)
    l[np.abs(l) < U16] = 0.0
    return h, l


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even) by their bit pattern."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def bf16_parts(x, nsplit):
    x = np.asarray(x, dtype=np.float32)
    parts, r = [], x
    for _ in range(nsplit):
        p = bf16(r)
        parts.append(p)
        r = (r - p).astype(np.float32)
    return parts


def exact_dot(a, b):
    return sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a, b))


def vectors(rng, d, spread):
    """FP32 vectors whose entries span `spread` binades with random signs."""
    e = rng.integers(-spread, 1, size=d)
    return (rng.standard_normal(d) * np.exp2(e)).astype(np.float32)


@pytest.mark.parametrize("d", [3, 16, 100])
def test_fp16_two_part_bound(d):
    rng = np.random.default_rng(500 + d)
    worst = 0.0
    for trial in range(120):
        spread = [4, 20, 40][trial % 3]
        x = vectors(rng, d, spread)
        y = vectors(rng, d, spread)
        # scale so that the larger norm sits in [2^13, 2^14), as the packing does
        n = max(np.linalg.norm(x.astype(np.float64)), np.linalg.norm(y.astype(np.float64)))
        sigma = 13 - math.frexp(n)[1] + 1
        xs = (x * np.float32(2.0 ** sigma)).astype(np.float32)
        ys = (y * np.float32(2.0 ** sigma)).astype(np.float32)
        x1, x2 = fp16_parts(xs)
        y1, y2 = fp16_parts(ys)
        kept = exact_dot(x1, y1) + exact_dot(x1, y2) + exact_dot(x2, y1)
        err = abs(exact_dot(xs, ys) - kept)
        sabs = float(sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(xs, ys)))
        nx, ny = np.linalg.norm(xs.astype(np.float64)), np.linalg.norm(ys.astype(np.float64))
        bound = 3.01 * 2.0 ** -22 * sabs + 1.001 * U16 * math.sqrt(d) * (nx + ny) + 2 * d * 2.0 ** -28
        assert float(err) <= bound, (trial, float(err), bound)
        worst = max(worst, float(err) / bound)
    assert worst > 0.01          # the vectors do exercise the bound


@pytest.mark.parametrize("nsplit,coef", [(2, 3.1 * 2.0 ** -16), (3, 4.2 * 2.0 ** -24)])
@pytest.mark.parametrize("d", [16, 100])
def test_bf16_split_bounds(nsplit, coef, d):
    """Products with part indices summing to at most nsplit - 1 are kept."""
    rng = np.random.default_rng(600 + d + nsplit)
    worst = 0.0
    for trial in range(80):
        x = vectors(rng, d, [2, 12, 30][trial % 3])
        y = vectors(rng, d, [2, 12, 30][trial % 3])
        xp, yp = bf16_parts(x, nsplit), bf16_parts(y, nsplit)
        kept = sum(exact_dot(xp[a], yp[b]) for a in range(nsplit) for b in range(nsplit)
                   if a + b <= nsplit - 1)
        err = abs(exact_dot(x, y) - kept)
        sabs = float(sum(abs(Fraction(float(u)) * Fraction(float(v))) for u, v in zip(x, y)))
        assert float(err) <= coef * sabs, (trial, float(err), coef * sabs)
        worst = max(worst, float(err) / (coef * sabs))
    assert worst > 0.01


def test_fp16_parts_never_subnormal_and_exact_remainders():
    rng = np.random.default_rng(700)
    x = (rng.standard_normal(4096) * np.exp2(rng.integers(-40, 14, 4096))).astype(np.float32)
    h, l = fp16_parts(x)
    for p in (h, l):
        nz = p[p != 0]
        assert np.all(np.abs(nz) >= U16)
        assert np.array_equal(nz.astype(np.float16).astype(np.float32), nz)   # FP16 values
    e = x.astype(np.float64) - h - l
    assert np.all(np.abs(e) <= 2.0 ** -22 * 1.001 * np.abs(x) + U16)
