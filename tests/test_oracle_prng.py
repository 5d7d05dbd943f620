"""Pins of the oracle's keyed PRNG, bounded draw and Fisher-Yates shuffle
against values and properties fixed outside the oracle."""
import ctypes as C
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_kat.txt")
M64 = (1 << 64) - 1


def _kat():
    out = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        st, vals = line.split(":")
        out.append((int(st), [int(v) for v in vals.split()]))
    return out


def test_splitmix64_known_answers():
    L = O.lib()
    for state, expect in _kat():
        s = C.c_uint64(state)
        got = [L.orc_next(C.byref(s)) for _ in expect]
        assert got == expect


def test_bounded_is_multiply_high():
    """Lemire's map: the draw is floor(x * n / 2^64) of the stream output x
    (checked with exact integer division, not the 128-bit split)."""
    L = O.lib()
    for n in [1, 2, 3, 7, 10, 1000, 2**31 - 1, 2**32, 12352]:
        s = C.c_uint64(0)
        s2 = C.c_uint64(0)
        for _ in range(50):
            x = L.orc_next(C.byref(s2))
            if (x * n) & M64 < ((1 << 64) % n):
                break  # a rejection: covered by the next test
            assert L.orc_bounded(C.byref(s), n) == (x * n) >> 64


def test_bounded_rejection():
    """n = 2^63 + 1 rejects about half the outputs: the accepted value is the
    high half for the first x whose low half is at least 2^64 mod n."""
    L = O.lib()
    n = (1 << 63) + 1
    t = (1 << 64) % n
    s = C.c_uint64(99)
    ref = C.c_uint64(99)
    rejected = 0
    for _ in range(200):
        v = L.orc_bounded(C.byref(s), n)
        while True:
            x = L.orc_next(C.byref(ref))
            if (x * n) & M64 >= t:
                break
            rejected += 1
        assert v == (x * n) >> 64 and v < n
    assert rejected > 50  # the loop was exercised


def test_bounded_uniform_chi2():
    L = O.lib()
    n, draws = 7, 70000
    s = C.c_uint64(2024)
    counts = np.bincount([L.orc_bounded(C.byref(s), n) for _ in range(draws)], minlength=n)
    exp = draws / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 22.46  # p = 0.001 at 6 dof


def _fy(seed, n):
    a = np.zeros(n, np.uint32)
    s = C.c_uint64(seed)
    O.lib().orc_fisher_yates(C.byref(s), n, a.ctypes.data_as(C.c_void_p))
    return a


@pytest.mark.parametrize("n,trials,crit", [(3, 24000, 20.52), (4, 48000, 49.73)])
def test_fisher_yates_uniform_over_all_permutations(n, trials, crit):
    """Every one of the n! permutations appears, equally often (chi-square,
    p = 0.001). Sattolo's variant (j < i) or an off-by-one in the bound
    would miss permutations and fail."""
    perms = {p: i for i, p in enumerate(itertools.permutations(range(n)))}
    counts = np.zeros(len(perms))
    for k in range(trials):
        counts[perms[tuple(int(v) for v in _fy(O.lib().orc_mix(k), n))]] += 1
    assert (counts > 0).all()
    exp = trials / len(perms)
    assert float(((counts - exp) ** 2 / exp).sum()) < crit


def test_fisher_yates_position_marginals():
    n, trials = 9, 9000
    m = np.zeros((n, n))
    for k in range(trials):
        a = _fy(k * 7919 + 1, n)
        m[np.arange(n), a] += 1
    exp = trials / n
    chi2 = ((m - exp) ** 2 / exp).sum()
    assert chi2 < 130.0  # 64 dof (row/col sums fixed), p ~ 1e-6 cut


def test_fisher_yates_small_cases():
    assert list(_fy(5, 0)) == []
    assert list(_fy(5, 1)) == [0]
    # n = 2: the single draw j = bounded(2) decides the swap
    for seed in range(20):
        s = C.c_uint64(seed)
        j = O.lib().orc_bounded(C.byref(s), 2)
        assert list(_fy(seed, 2)) == ([1, 0] if j == 0 else [0, 1])


def test_stream_seeds_distinct():
    L = O.lib()
    seeds = {L.orc_stream_seed(0x1234, tag, ep, idx)
             for tag in (1, 2, 3, 4) for ep in range(4) for idx in range(64)}
    assert len(seeds) == 4 * 4 * 64
