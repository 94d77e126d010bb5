"""The pricing scan's fp32 filter never rejects a pair with z < 0 (host check).

The scan (csrc/pricing.cu) decides a pair exactly only if an fp32 filter lets
it through, so the filter must pass every pair whose reduced cost
z = c * 2^fb - lambda_u - lambda_v is negative.  This file evaluates the
filter's arithmetic on the CPU, operation by operation with IEEE binary32
round-to-nearest-even (adds and multiplies in numpy float32, fused
multiply-adds exactly in rationals and rounded once), on pairs placed at the
boundary z = -1, and checks that each passes.  It pins the error analysis in
the kernel's header comment, independently of the GPU.
"""
import math
import sys
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def round_f32(q: Fraction) -> F32:
    """q rounded to binary32, to nearest, ties to even (normal range)."""
    if q == 0:
        return F32(0.0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    m = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    lo = math.floor(m)
    r = m - lo
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return F32(sign * float(lo) * 2.0 ** (e - 23))


def fma32(a, b, c) -> F32:
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def radius(lam: int, fb: int) -> F32:
    # pricing_prep_kernel: r = max(lambda 2^-fb + 1/4, 0); s = (r + 2)(1 + 2^-17)
    r = F32(lam) * F32(2.0 ** -fb) + F32(0.25)  # the product is exact (a power of two)
    r = max(r, F32(0.0))
    return (r + F32(2.0)) * F32(1.0 + 2.0 ** -17)


def filter_value(pu, pv, lu, lv, fb) -> F32:
    """e' of the pair (u, v) as pricing_kernel computes it (j = v, i = u)."""
    su, sv = radius(lu, fb), radius(lv, fb)
    xu, yu = F32(pu[0]), F32(pu[1])
    xv, yv = F32(pv[0]), F32(pv[1])
    au, cu = xu - su, xu + su
    av, cv = xv - sv, xv + sv
    u = av + (-cu)
    w = cv + (-au)
    dy = yv + (-yu)
    return fma32(dy, dy, fma32(u, w, F32(-1.0)))


def exact_cost(pu, pv) -> int:
    d2 = (pu[0] - pv[0]) ** 2 + (pu[1] - pv[1]) ** 2
    c = math.isqrt(d2)
    # nearest integer to sqrt(d2): c or c + 1 (no exact halves for integers)
    return c + 1 if (2 * c + 1) ** 2 < 4 * d2 else c


def boundary_pairs(rng, count, fb, spread):
    """Pairs with lambda_u + lambda_v = c * 2^fb + 1, i.e. z = -1, whose
    distance is just below c + 1/2 (the largest distance that rounds to c):
    there the filter's margin is smallest."""
    pu = rng.integers(0, 1 << 20, size=(200 * count, 2))
    pv = np.clip(pu + rng.integers(-spread, spread + 1, size=pu.shape), 0, (1 << 20) - 1)
    d = np.sqrt(((pu - pv).astype(np.float64) ** 2).sum(axis=1))
    frac = d - np.floor(d + 0.5)  # in [-1/2, 1/2): distance above its rounded value
    pick = np.argsort(-frac)[:count]
    out = []
    for k in pick:
        pu_, pv_ = [int(t) for t in pu[k]], [int(t) for t in pv[k]]
        S = (exact_cost(pu_, pv_) << fb) + 1
        share = rng.uniform(-0.5, 1.5)  # one lambda may be negative
        lu = int(S * share)
        lv = S - lu
        if max(abs(lu), abs(lv)) >= 1 << 29:
            continue
        out.append((pu_, pv_, lu, lv))
    return out


@pytest.mark.parametrize("fb", [1, 4, 8, 9])
@pytest.mark.parametrize("spread", [3, 3000, 300000, (1 << 20) - 1])
def test_filter_passes_every_negative_pair(fb, spread):
    rng = np.random.default_rng(1000 * fb + spread % 997)
    cases = boundary_pairs(rng, 300, fb, spread)
    assert len(cases) > 200
    for pu, pv, lu, lv in cases:
        assert (exact_cost(pu, pv) << fb) - lu - lv == -1
        e = filter_value(pu, pv, lu, lv, fb)
        assert np.signbit(e), (pu, pv, lu, lv, fb, e)


def test_filter_edge_cases():
    # duplicate points (c = 0), axis-aligned pairs, the coordinate range's
    # corners, and one lambda at the bottom of its range
    top = (1 << 20) - 1
    for fb in (1, 8, 9):
        for pu, pv in [([5, 5], [5, 5]), ([0, 0], [top, 0]), ([0, 0], [0, top]), ([0, 0], [top, top]),
                       ([top, 7], [top - 1, 7])]:
            S = (exact_cost(pu, pv) << fb) + 1
            for lu in (S, 1 - (1 << 29) + S if S < (1 << 29) else S, S // 2, 0, -(S // 3)):
                lv = S - lu
                if max(abs(lu), abs(lv)) >= 1 << 29:
                    continue
                assert np.signbit(filter_value(pu, pv, lu, lv, fb)), (pu, pv, lu, lv, fb)


def test_filter_rejects_far_pairs():
    # not a soundness requirement, a sanity check of the arithmetic: a pair
    # far outside both radii is filtered out
    e = filter_value([0, 0], [100000, 0], 256 * 1000, 256 * 1000, 8)
    assert not np.signbit(e) and e > 1e9


def test_round_f32_matches_numpy_on_floats():
    rng = np.random.default_rng(3)
    for v in rng.uniform(-1e12, 1e12, size=2000):
        assert round_f32(Fraction(float(v))) == F32(v)


# Pairs at z = -1 on which the filter without the absolute margin of 2 length
# units (radius r (1 + 2^-19), the form a one-pair-per-instruction filter can
# use) rejects the pair: found by a random search over 10^8 boundary pairs and
# confirmed with the exact evaluation above.  (fb, point u, point v, lambda_u,
# lambda_v)
HARD = [
    (8, [525119, 170879], [526200, 173116], 622970, 12935),
    (8, [1048277, 791946], [1046236, 794201], 608010, 170487),
    (8, [1046534, 514049], [1048461, 512193], 649195, 35606),
    (8, [942413, 25844], [950683, 1408], 1530389, 5073644),
    (8, [820375, 249221], [828083, 257542], 2336571, 566982),
    (8, [853757, 977125], [862163, 960929], 3828429, 842804),
    (9, [1048294, 376970], [1048569, 377243], 49709, 148436),
    (9, [524144, 971550], [524600, 969003], 579756, 744789),
    (9, [524593, 1028042], [525371, 1025788], 823250, 397359),
    (9, [524184, 615278], [525665, 614971], 53548, 720597),
    (9, [679767, 536370], [679324, 554209], 4299390, 4836739),
    (9, [1045257, 350850], [1048575, 342950], 2170331, 2216486),
    (9, [674555, 201176], [668626, 231164], 3199754, 12451063),
    (9, [1039925, 450135], [1048575, 440941], 5574931, 888046),
]


def test_filter_passes_the_hard_pairs(monkeypatch):
    for fb, pu, pv, lu, lv in HARD:
        assert (exact_cost(pu, pv) << fb) - lu - lv == -1
        assert np.signbit(filter_value(pu, pv, lu, lv, fb)), (fb, pu, pv)

    # the same pairs reject a filter whose radius lacks the absolute margin:
    # the margin is needed, and this file would notice it missing
    def radius_without_margin(lam, fb):
        r = max(F32(lam) * F32(2.0 ** -fb) + F32(0.25), F32(0.0))
        return r * F32(1.0 + 2.0 ** -19)
    monkeypatch.setattr(sys.modules[__name__], "radius", radius_without_margin)
    assert all(not np.signbit(filter_value(pu, pv, lu, lv, fb)) for fb, pu, pv, lu, lv in HARD)


@pytest.mark.parametrize("fb", [1, 8, 9])
def test_filter_random_boundary_pairs_vectorised(fb):
    # 10^6 random pairs at z = -1 per fraction; the FMAs in float64 (the
    # first exactly, the second rounded twice, which can only matter at a tie)
    rng = np.random.default_rng(40 + fb)
    N = 1_000_000
    pu = rng.integers(0, 1 << 20, size=(N, 2))
    spread = rng.choice([30, 3000, 30000, 300000], size=(N, 1))
    pv = np.clip(pu + rng.integers(-(1 << 20), 1 << 20, size=pu.shape) % (2 * spread + 1) - spread, 0,
                 (1 << 20) - 1)
    d2 = ((pu - pv) ** 2).sum(axis=1)
    c = np.floor(np.sqrt(d2.astype(np.float64)) + 0.5).astype(np.int64)
    S = (c << fb) + 1
    lu = (S * rng.uniform(-0.5, 1.5, size=N)).astype(np.int64)
    lv = S - lu
    ok = (np.abs(lu) < (1 << 29)) & (np.abs(lv) < (1 << 29))

    def rad(lam):
        r = np.maximum(lam.astype(np.float32) * F32(2.0 ** -fb) + F32(0.25), F32(0))
        return (r + F32(2.0)) * F32(1.0 + 2.0 ** -17)
    su, sv = rad(lu), rad(lv)
    xu, yu = pu[:, 0].astype(np.float32), pu[:, 1].astype(np.float32)
    xv, yv = pv[:, 0].astype(np.float32), pv[:, 1].astype(np.float32)
    u = (xv - sv) + (-(xu + su))
    w = (xv + sv) + (-(xu - su))
    dy = yv + (-yu)
    p = (u.astype(np.float64) * w.astype(np.float64) - 1.0).astype(np.float32)
    e = (dy.astype(np.float64) ** 2 + p.astype(np.float64)).astype(np.float32)
    assert ok.sum() > 0.9 * N
    assert not np.any(ok & ~np.signbit(e))
