"""The phase count of the compositing warps' in-bucket sort.

After the counting sort on depth buckets, the warp sort in
`csrc/composite.cu` runs odd-even transposition phases over the whole list
(phase 0 compares pairs (2i, 2i + 1), phase 1 pairs (2i + 1, 2i + 2), and so
on), as many as its most crowded bucket holds keys.  That count is enough
because buckets are in order (a compared pair that straddles two buckets is
never swapped) and s phases sort s keys whichever parity their bucket starts
at.  These tests check that property on plain lists: exhaustively for small
buckets at both parities, and on random lists of many buckets up to the
kernel's limit of 64 keys a bucket.
"""
import itertools
import random


def _phases(a, m):
    a = list(a)
    for ph in range(m):
        for i in range(ph % 2, len(a) - 1, 2):
            if a[i] > a[i + 1]:
                a[i], a[i + 1] = a[i + 1], a[i]
    return a


def test_every_small_bucket_at_either_parity():
    for s in range(1, 7):
        for off in (0, 1, 2):
            for p in itertools.permutations(range(s)):
                a = [-10 + i for i in range(off)] + list(p) + [100, 101]
                assert _phases(a, s) == sorted(a), (s, off, p)


def test_fewer_phases_do_not_suffice_for_a_reversed_bucket():
    # the bound is tight: a reversed bucket of s >= 3 keys needs all s phases
    # at either parity (two keys at an even start need only the first)
    cases = [(2, 1)] + [(s, off) for s in range(3, 9) for off in (0, 1)]
    for s, off in cases:
        a = [-10 + i for i in range(off)] + list(range(s))[::-1]
        assert _phases(a, s - 1) != sorted(a), (s, off)


def test_random_lists_of_ordered_buckets():
    rng = random.Random(2407)
    for _ in range(400):
        sizes = [rng.choice([0, 1, 1, 2, 3, rng.randint(0, 64)]) for _ in range(rng.randint(1, 30))]
        a = []
        for b, sz in enumerate(sizes):
            vals = [b + rng.random() for _ in range(sz)]
            rng.shuffle(vals)
            a += vals
        assert _phases(a, max(sizes)) == sorted(a)
