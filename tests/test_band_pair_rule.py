"""The paired byte-height band pass and the band walk, restated in the pass's
16-bit pair arithmetic and checked against the oracle's traceback (no GPU).

Band (from the best cell (i*, j*) and S = a j* - best): at most (S - o)/e
deletions and (S - o)/(a + e) insertions, so an optimal path stays on the
diagonals [d* - #D, d* + #I] (d* = i* - j*); class width B the smallest of 8, 16,
32, 64 that holds them.  The pass runs two jobs at once, one in each 16-bit half of
a 32-bit word, in the recurrence of Methods section 3 shifted by beta = o + e:
X = H, E~ = E + beta, F~ = F + beta, G~ = max(X(i-1,j-1) + delta + beta, beta),
X = max(G~, E~, F~) - beta, the last subtraction one 32-bit add with a fixed carry
(every maximum is >= beta), delta + beta one multiply-add of the two match bits.
Cells left of column 0 are computed as columns that never match (they come out
H = 0, which makes column 0 the border).  The kernel runs two rows at once, the second
one slot behind, in place; that order must give the same heights as row by row.  The walk from (i*, j*) over the stored
heights (diagonal first; else F(i,j) = H decides a deletion, scanned along the row
and stopped once it reaches H or a bound min(best, a min(i',j)) puts every later
term below it; gap runs while strictly above H(neighbour) + S_GO) must give the
oracle's CIGAR and begins.
"""
import numpy as np
import pytest

import oracle

NEG16 = -16384
NEG = -(1 << 29)
SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (1, 2, 3, 2), (2, 4, 4, 2)]   # mismatch <= o + e


def s16(v):
    v &= 0xFFFF
    return v - 65536 if v >= 32768 else v


def pk(lo, hi):
    return (lo & 0xFFFF) | ((hi & 0xFFFF) << 16)


def lo16(v):
    return s16(v)


def hi16(v):
    return s16(v >> 16)


def addmax(a, b, c):                                  # per half: max(a + b, c), no carry across
    return pk(max(lo16(a) + lo16(b), lo16(c)), max(hi16(a) + hi16(b), hi16(c)))


def max3(a, b, c):
    return pk(max(lo16(a), lo16(b), lo16(c)), max(hi16(a), hi16(b), hi16(c)))


def band_of(a, o, e, istar, jstar, best):
    S = a * jstar - best
    dmax = (S - o) // e if (e > 0 and S >= o + e) else 0
    imax = (S - o) // (a + e) if S >= o + a + e else 0
    width = dmax + imax + 1
    for B in (8, 16, 32, 64):
        if width <= B:
            return B, (istar - jstar) - dmax
    return None, None


def pair_pass(jobs, B, a, b, o, e, two_rows=False):
    """Heights of both jobs: {(i, j): H} for the band cells of real columns (i >= 0).
    two_rows: the kernel's order, rows j and j + 1 together with the second one slot
    behind (row j + 1's slot k - 1 computed right after row j's slot k), in place."""
    beta = o + e
    GE2, BETA2 = pk(-e, -e), pk(beta, beta)
    SB2, AB = pk(-b + beta, -b + beta), a + b
    GO2C = 0 if beta == 0 else ((((-beta) & 0xFFFF) + (((-beta - 1) & 0xFFFF) << 16)) & 0xFFFFFFFF)
    NEG2 = pk(NEG16, NEG16)
    X = [0 if k < B else NEG2 for k in range(B + 1)]
    E = [NEG2] * (B + 1)
    out = [{}, {}]
    rows = max(jb["rows"] for jb in jobs)
    left = {}                                          # row -> [xleft, fleft]

    def cell(j, k):
        xleft, fleft = left[j]
        sel = 0
        for h, jb in enumerate(jobs):
            i = j + jb["dlo"] + k
            rb = jb["read"][j - 1] if j - 1 < len(jb["read"]) else -1
            if 1 <= i <= len(jb["win"]) and jb["win"][i - 1] == rb:
                sel |= 1 << (16 * h)
        d2 = (sel * AB + SB2) & 0xFFFFFFFF
        en = addmax(E[k + 1], GE2, X[k + 1])
        fn = addmax(fleft, GE2, xleft)
        gt = addmax(X[k], d2, BETA2)
        x = (max3(gt, en, fn) + GO2C) & 0xFFFFFFFF
        X[k], E[k] = x, en
        left[j] = [x, fn]
        for h, jb in enumerate(jobs):
            i = j + jb["dlo"] + k
            if j <= jb["rows"] and i >= 0:
                v = lo16(x) if h == 0 else hi16(x)
                assert 0 <= v <= 254
                out[h][(i, j)] = v

    j = 1
    if two_rows:
        while j + 1 <= rows:
            left[j] = [NEG2, NEG2]
            left[j + 1] = [NEG2, NEG2]
            for k in range(B + 1):
                if k < B:
                    cell(j, k)
                if k >= 1:
                    cell(j + 1, k - 1)
            j += 2
    while j <= rows:
        left[j] = [NEG2, NEG2]
        for k in range(B):
            cell(j, k)
        j += 1
    return out


def band_walk(hts, jb, a, b, o, e):
    GO, GE, sa, sb = -(o + e), -e, a, -b
    B, dlo = jb["B"], jb["dlo"]

    def height(ii, jj):
        if jj == 0:
            return 0 if ii >= 0 else NEG
        k = ii - jj - dlo
        if k < 0 or k >= B:
            return NEG
        return hts[(ii, jj)]

    rev = []

    def emit(op):
        if rev and rev[-1][1] == op:
            rev[-1][0] += 1
        else:
            rev.append([1, op])

    i, j, h, best = jb["istar"], jb["jstar"], jb["best"], jb["best"]
    state, cur = 0, 0
    budget = 2 * (i + jb["rows"]) + 4
    if height(i, j) != h:
        return None
    while True:
        budget -= 1
        if budget < 0:
            return None
        if state == 0:
            if i == 0 or j == 0 or h <= 0:
                break
            hd = height(i - 1, j - 1)
            if hd != NEG and hd + (sa if jb["win"][i - 1] == jb["read"][j - 1] else sb) == h:
                emit(0)
                i, j, h = i - 1, j - 1, hd
                continue
            f = NEG
            for kk in range(1, i + 1):
                if min(best, sa * min(j, i - kk)) + GO + (kk - 1) * GE < h:
                    break
                hx = height(i - kk, j)
                if hx == NEG:
                    break
                f = max(f, hx + GO + (kk - 1) * GE)
                if f >= h:
                    break
            state, cur = (2 if f == h else 1), h
        elif state == 2:
            if i < 1:
                return None
            emit(2)
            hn = height(i - 1, j)
            i -= 1
            if hn != NEG and cur <= hn + GO:
                state, h = 0, hn
            else:
                cur -= GE
        else:
            if j < 1:
                return None
            emit(1)
            hn = height(i, j - 1)
            j -= 1
            if hn != NEG and cur <= hn + GO:
                state, h = 0, hn
            else:
                cur -= GE
    return [(ln, op) for ln, op in reversed(rev)], i, j


def cigar_core(cig):
    runs, num = [], ""
    for ch in cig:
        if ch.isdigit():
            num += ch
        else:
            if ch != "S":
                runs.append((int(num), oracle.OPS.index(ch)))
            num = ""
    return runs


def mutated_pair(rng, alphabet):
    letters = "ACGT"[:alphabet]
    m = int(rng.integers(20, 70))
    n = int(rng.integers(8, min(40, m)))
    win = "".join(rng.choice(list(letters), m))
    s0 = int(rng.integers(0, m - n + 1))
    read = list(win[s0:s0 + n])
    for _ in range(int(rng.integers(0, 6))):
        p = int(rng.integers(0, len(read)))
        r = rng.random()
        if r < 0.4:
            read[p] = str(rng.choice(list(letters)))
        elif r < 0.7 and len(read) > 2:
            del read[p]
        else:
            read.insert(p, str(rng.choice(list(letters))))
    return win, "".join(read)


@pytest.mark.parametrize("scoring", SCHEMES)
@pytest.mark.parametrize("alphabet", [4, 2])
def test_paired_band_pass_and_walk_match_the_oracle(scoring, alphabet):
    rng = np.random.default_rng(7 + 11 * alphabet + 3 * sum(scoring))
    a, b, o, e = scoring
    assert b <= o + e                                  # the pair form's condition
    pending, checked, left_of_column_0 = [], 0, 0
    for _ in range(300):
        win, read = mutated_pair(rng, alphabet)
        res, cig = oracle.align_pair(win, read, scoring=scoring, mode=oracle.LOCAL)
        if int(res["flags"]) & oracle.EMPTY:
            continue
        istar, jstar, best = int(res["ref_end"]), int(res["read_end"]), int(res["score"])
        B, dlo = band_of(a, o, e, istar, jstar, best)
        if B is None:
            continue
        job = dict(win=oracle.codes(win).tolist(), read=oracle.codes(read).tolist(), rows=jstar, dlo=dlo,
                   B=B, istar=istar, jstar=jstar, best=best, cig=cig, res=res)
        pending.append(job)
        if len(pending) < 2:
            continue
        pair, pending = pending, []
        Bp = max(p["B"] for p in pair)                 # the pair runs at the wider class
        for p in pair:
            p["B"] = Bp
        hts = pair_pass(pair, Bp, a, b, o, e)
        assert pair_pass(pair, Bp, a, b, o, e, two_rows=True) == hts   # the two-row order
        for h, p in enumerate(pair):
            out = band_walk(hts[h], p, a, b, o, e)
            assert out is not None, (p["cig"], scoring)
            ops, ib, jb = out
            assert ops == cigar_core(p["cig"]), (ops, p["cig"], scoring)
            assert jb == int(p["res"]["read_begin"]) and ib == int(p["res"]["ref_begin"])
            checked += 1
            left_of_column_0 += p["dlo"] < 0
    assert checked > 100 and left_of_column_0 > 0, (checked, left_of_column_0)
