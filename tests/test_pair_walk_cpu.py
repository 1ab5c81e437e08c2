"""Host-side check of the pair order the adjoint kernel k_adj_cd walks (no GPU): position p of
an atom with n neighbours is the pair (k, k + d mod n), k = p mod n, d = 1 + floor(p / n), with
the quotient taken by a multiply-high with ceil(2^32 / n).  Every unordered pair must appear
once, and within each round of W = min(32, n - 1) consecutive positions the first entries must
be distinct and so must the second ones: that is what lets the kernel add the per-entry
gradients of a round by plain read-modify-write instead of atomics."""
import pytest


def walk(n):
    P = n * (n - 1) // 2
    W = min(32, n - 1)
    magic = ((1 << 32) + n - 1) // n if n > 1 else 0
    rounds = []
    base = 0
    while base < P:
        r = []
        for lane in range(min(W, P - base)):
            p = base + lane
            q = (p * magic) >> 32
            k1 = p - q * n
            k2 = k1 + q + 1
            if k2 >= n:
                k2 -= n
            r.append((k1, k2))
        rounds.append(r)
        base += W
    return rounds


@pytest.mark.parametrize("n", list(range(0, 80)) + [95, 128, 200, 361, 362])
def test_diagonal_walk_covers_pairs_once_with_distinct_entries_per_round(n):
    seen = set()
    for r in walk(n):
        firsts = [a for a, _ in r]
        seconds = [b for _, b in r]
        assert len(set(firsts)) == len(firsts)
        assert len(set(seconds)) == len(seconds)
        for a, b in r:
            assert 0 <= a < n and 0 <= b < n and a != b
            key = (min(a, b), max(a, b))
            assert key not in seen
            seen.add(key)
    assert len(seen) == n * (n - 1) // 2


def test_multiply_high_quotient_is_exact_below_2_16():
    # pairs per atom stay below 2^16 (capacity <= 362): q = floor(p / n) exactly
    for n in (2, 3, 7, 31, 32, 33, 100, 255, 361, 362):
        magic = ((1 << 32) + n - 1) // n
        for p in range(0, n * (n - 1) // 2, max(1, n // 7)):
            assert (p * magic) >> 32 == p // n
