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


def _equi_buckets(depth, NB, coarse=32):
    """The warp sort's equi-depth bucket of each depth word, in FP32 as the
    kernel computes it: coarse bins even over [lo, hi], each given buckets in
    proportion to its keys (at least one when it has any), a key placed by
    its position within its bin."""
    import numpy as np
    f32 = np.float32
    d = np.asarray(depth, dtype=np.uint32)
    lo, hi = d.min(), d.max()
    scale = f32(coarse) / (f32(np.uint32(hi - lo)) + f32(1.0))
    t = (d - lo).astype(f32) * scale
    c = np.minimum(coarse - 1, t.astype(np.int64))
    nc = np.bincount(c, minlength=coarse)
    nb = nc * (NB - coarse) // len(d) + (nc > 0)
    first = np.concatenate([[0], np.cumsum(nb)[:-1]])
    frac = (t - c.astype(f32)) * nb[c].astype(f32)
    b = first[c] + np.minimum(nb[c] - 1, frac.astype(np.int64))
    return b, int(nb.sum()), first[c], nb[c]


def _even_buckets(depth, NB):
    import numpy as np
    f32 = np.float32
    d = np.asarray(depth, dtype=np.uint32)
    lo, hi = d.min(), d.max()
    scale = f32(NB) / (f32(np.uint32(hi - lo)) + f32(1.0))
    return np.minimum(NB - 1, ((d - lo).astype(f32) * scale).astype(np.int64))


def test_equi_depth_buckets_are_ordered():
    """The phases need buckets in key order: a deeper key never takes an
    earlier bucket.  Each key's bucket lies in its own bin's range, so bins
    never share one, and on clustered depths the most crowded bucket (the
    phase count) holds fewer keys than with buckets even over [lo, hi].
    Clustered, uniform, tied and extreme depth words."""
    import numpy as np
    rng = np.random.default_rng(2407)
    cases, crowd_eq, crowd_even = [], 0, 0
    for n in (64, 65, 180, 252, 511, 512, 1000):
        core = rng.normal(0x40800000, 0x00100000, size=n).astype(np.int64)
        back = rng.integers(0x3F800000, 0x40E00000, size=n)
        mix = np.where(rng.random(n) < 0.8, core, back)
        cases += [mix, back, np.full(n, 12345), rng.integers(0, 2, size=n),
                  rng.integers(0, 0x0FFFFFFF, size=n), np.r_[np.zeros(n - 1), [0x0FFFFFFF]]]
        NB = min(1 << int(np.ceil(np.log2(n))), 352)
        crowd_eq += np.bincount(_equi_buckets(mix, NB)[0]).max()
        crowd_even += np.bincount(_even_buckets(mix, NB)).max()
    assert crowd_eq * 3 < crowd_even * 2, (crowd_eq, crowd_even)
    for d in cases:
        d = np.clip(np.asarray(d, dtype=np.int64), 0, 0x0FFFFFFF)
        n = len(d)
        NB = 1
        while NB < n:
            NB <<= 1
        NB = min(NB, 352)
        b, used, first, nb = _equi_buckets(d, NB)
        assert used <= NB and b.min() >= 0 and b.max() < NB
        assert np.all(b >= first) and np.all(b < first + nb)
        o = np.argsort(d, kind="stable")
        assert np.all(np.diff(b[o]) >= 0)
