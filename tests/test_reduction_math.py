"""The integer identities behind the kernels' 32-bit warp reductions (CPU).

The narrow tail sums a warp's 64-bit values as three 32-bit warp sums of
21-bit chunks and takes a 64-bit minimum as two 32-bit minima (high words,
then the low words of the lanes holding the minimum high word).  These tests
restate both steps with Python integers, the 32-bit sums wrapping as the
hardware's do, and check them against the plain sum and minimum, including
the extremes the kernels allow (each value below 2^64 and the total below
2^64 for the sum; any int64 for the minimum).
"""
import random

M32 = (1 << 32) - 1


def chunked_sum(xs):
    m = (1 << 21) - 1
    s0 = sum(x & m for x in xs) & M32
    s1 = sum((x >> 21) & m for x in xs) & M32
    s2 = sum(x >> 42 for x in xs) & M32
    return (s0 + (s1 << 21) + (s2 << 42)) & ((1 << 64) - 1)


def two_step_min(xs):
    his = [x >> 32 for x in xs]  # arithmetic shift: the signed high word
    mh = min(his)
    ml = min((x & M32) if (x >> 32) == mh else M32 for x in xs)
    return (mh << 32) | ml


def test_chunked_sum_exact_below_2_64():
    rng = random.Random(5)
    for trial in range(3000):
        k = rng.choice([1, 2, 7, 32])
        cap = min(rng.choice([1 << 20, 1 << 40, 1 << 62, 1 << 64]), (1 << 64) // k)
        xs = [rng.randrange(cap) for _ in range(k)] + [0] * (32 - k)
        assert sum(xs) < 1 << 64
        assert chunked_sum(xs) == sum(xs), (trial, xs)
    # chunk sums cannot wrap: 32 lanes of the largest chunk values
    xs = [(1 << 64) // 32 - 1] * 32
    assert chunked_sum(xs) == sum(xs)
    assert 32 * ((1 << 22) - 1) < 1 << 32


def test_two_step_min_matches_int64_min():
    rng = random.Random(6)
    lo, hi = -(1 << 63), (1 << 63) - 1
    for trial in range(3000):
        pool = [rng.randrange(lo, hi + 1) for _ in range(4)] + [0, -1, hi, lo, 1 << 32, (1 << 32) - 1]
        xs = [rng.choice(pool) + rng.randrange(-3, 4) for _ in range(32)]
        xs = [min(max(x, lo), hi) for x in xs]
        assert two_step_min(xs) == min(xs), (trial, xs)
