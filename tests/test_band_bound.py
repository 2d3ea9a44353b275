"""The diagonal band that the traceback classification gives a job must hold every
optimal path ending at the job's best cell (CPU; exhaustive enumeration).

With S = a*j* - best, a path's insertions cost at least o + (a + e) each beyond
the first opening (the match each displaces plus its extension), its deletions
o + e each, so #I <= (S - o)/(a + e) and #D <= (S - o)/e (none below o + a + e,
resp. o + e).  Going back from (i*, j*), a deletion moves the path one diagonal
(d = i - j) down and an insertion one up, so every cell of such a path lies on
d* - #D max .. d* + #I max.  The library's band passes compute only those
diagonals; this test checks the bound itself on every optimal path of tiny
random cases."""
import random

import pytest

from bruteforce import LOCAL, GLOCAL, best_score, enumerate_paths

SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (3, 1, 0, 1), (2, 5, 1, 3), (1, 3, 4, 2)]


def band_of(scoring, best, i_end, j_end):
    a, b, o, e = scoring
    slack = a * j_end - best
    dmax = (slack - o) // e if slack >= o + e else 0
    imax = (slack - o) // (a + e) if slack >= o + a + e else 0
    d = i_end - j_end
    return d - dmax, d + imax


def diagonals(i0, j0, ops):
    i, j = i0, j0
    ds = [i - j]
    for c in ops:
        if c in "MD":
            i += 1
        if c in "MI":
            j += 1
        ds.append(i - j)
    return ds


@pytest.mark.parametrize("scoring", SCHEMES)
@pytest.mark.parametrize("mode", [LOCAL, GLOCAL])
def test_every_optimal_path_lies_in_the_band(scoring, mode):
    rng = random.Random(hash((scoring, mode)) & 0xffff)
    checked = 0
    for _ in range(120):
        n, m = rng.randint(1, 5), rng.randint(1, 7)
        T = "".join(rng.choice("AC") for _ in range(m))
        R = "".join(rng.choice("AC") for _ in range(n))
        best = best_score(T, R, scoring, mode)
        if best is None or (mode == LOCAL and best <= 0):
            continue
        paths = [p for p in enumerate_paths(T, R, scoring, mode)
                 if p[0] == best and p[3] >= 1 and p[4] >= 1]
        for i_end, j_end in {(p[3], p[4]) for p in paths}:
            lo, hi = band_of(scoring, best, i_end, j_end)
            for sc, i0, j0, i1, j1, ops in paths:
                if (i1, j1) != (i_end, j_end):
                    continue
                ds = diagonals(i0, j0, ops)
                assert lo <= min(ds) and max(ds) <= hi, (T, R, ops, lo, hi)
                checked += 1
    assert checked > 50


def test_the_opening_term_is_needed_and_sufficient():
    """A single deletion of length L costs o + e*L: the bound admits exactly L
    deletions for S = o + e*L and L - 1 for one less."""
    a, b, o, e = (1, 2, 2, 1)
    for L in range(1, 6):
        S = o + e * L
        lo, hi = band_of((a, b, o, e), a * 10 - S, 10 + L, 10)
        assert (10 + L - 10) - lo == L
        lo, _ = band_of((a, b, o, e), a * 10 - (S - 1), 10 + L, 10)
        assert (10 + L - 10) - lo == L - 1
