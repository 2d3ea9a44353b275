"""The height-walk rule of the LOCAL traceback, checked against the oracle's own
traceback (no GPU).

The byte-height passes store H only, and the walk re-derives every decision from
the heights (Methods section 3 backtracks through the recurrence's sources, the
diagonal first on ties): at (i, j) in state H the diagonal when H(i-1,j-1) + delta
= H; else a deletion when F(i,j) = H, an insertion otherwise, with E(i,j) looked
at first (E below H leaves the deletion as the only source); a gap run extends
while its value is strictly above H(neighbour) + S_GO.  E and F are rebuilt as
maxima of H + S_GO + (k-1) S_GE up the column / along the row, and a scan stops
once a bound on every later term falls below H: H(i',j') <= best and, in LOCAL,
H(i',j') <= a min(i',j').  The walk reads one height an iteration (the scans are
states of the loop, not inner loops).  This restates that loop over the oracle's
full H matrix and requires the oracle's CIGAR and begins, over schemes with and
without a gap-extend cost, two- and four-letter alphabets and reads with planted
substitutions and indels.
"""
import numpy as np
import pytest

import oracle

NEG = -(1 << 29)
SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (1, 3, 1, 0), (3, 1, 0, 1), (1, 10, 0, 1)]


def flat_walk(H, T, R, i, j, h, a, b, o, e):
    """(forward ops [(len, op)], 0-based window begin, 0-based read begin) or None."""
    GO, GE, sa, sb = -(o + e), -e, a, -b
    m, n = H.shape[0] - 1, H.shape[1] - 1
    hmax = h

    def height(ii, jj):
        return NEG if (ii < 0 or jj < 0 or ii > m or jj > n) else int(H[ii, jj])

    rev = []

    def emit(op):
        if rev and rev[-1][1] == op:
            rev[-1][0] += 1
        else:
            rev.append([1, op])

    state, kk, acc, cur = "H", 0, NEG, 0
    budget = 2 * (m + n) + 4
    while True:
        ii = -1
        jj = 0
        if state in ("scanE", "scanF"):
            up = state == "scanE"
            lim = j if up else i
            hb = min(hmax, sa * ((j - kk) if up else min(j, i - kk)))
            if kk <= lim and hb + GO + (kk - 1) * GE >= h:
                ii, jj = (i, j - kk) if up else (i - kk, j)
        else:
            budget -= 1
            if budget < 0:
                return None
            if state == "H":
                if i == 0 or j == 0 or h <= 0:
                    break
                ii, jj = i - 1, j - 1
            elif state == "D":
                if i < 1:
                    return None
                ii, jj = i - 1, j
            else:
                if j < 1:
                    return None
                ii, jj = i, j - 1
        hx = height(ii, jj) if ii >= 0 else NEG
        if state == "H":
            if hx != NEG and hx + (sa if T[i - 1] == R[j - 1] else sb) == h:
                emit(0)
                i, j, h = i - 1, j - 1, hx
            else:
                state, kk, acc, cur = "scanE", 1, NEG, h
        elif state in ("scanE", "scanF"):
            stop = hx == NEG
            if not stop:
                acc = max(acc, hx + GO + (kk - 1) * GE)
                stop = acc >= h
            if not stop:
                kk += 1
            elif state == "scanE":
                if acc < h:
                    state = "D"
                else:
                    state, kk, acc = "scanF", 1, NEG
            else:
                state = "D" if acc == h else "I"
        elif state == "D":
            emit(2)
            i -= 1
            if hx != NEG and cur <= hx + GO:
                state, h = "H", hx
            else:
                cur -= GE
        else:
            emit(1)
            j -= 1
            if hx != NEG and cur <= hx + GO:
                state, h = "H", hx
            else:
                cur -= GE
    return [(ln, op) for ln, op in reversed(rev)], i, j


def random_pair(rng, alphabet):
    letters = "ACGT"[:alphabet]
    n = int(rng.integers(1, 40))
    m = int(rng.integers(1, 60))
    win = "".join(rng.choice(list(letters), m))
    if m > n and rng.random() < 0.6:                 # a read taken from the window, then mutated
        s0 = int(rng.integers(0, m - n + 1))
        read = list(win[s0:s0 + n])
        for _ in range(int(rng.integers(0, 5))):
            p = int(rng.integers(0, len(read)))
            r = rng.random()
            if r < 0.4:
                read[p] = str(rng.choice(list(letters)))
            elif r < 0.7 and len(read) > 1:
                del read[p]
            else:
                read.insert(p, str(rng.choice(list(letters))))
        read = "".join(read)
    else:
        read = "".join(rng.choice(list(letters), n))
    return win, read


@pytest.mark.parametrize("scoring", SCHEMES)
@pytest.mark.parametrize("alphabet", [4, 2])
def test_height_walk_matches_the_oracle_traceback(scoring, alphabet):
    rng = np.random.default_rng(101 + 7 * alphabet + sum(scoring))
    a, b, o, e = scoring
    walked = gapped = 0
    for _ in range(500):
        win, read = random_pair(rng, alphabet)
        res, cig = oracle.align_pair(win, read, scoring=scoring, mode=oracle.LOCAL)
        if int(res["flags"]) & oracle.EMPTY:
            continue
        H, _, _ = oracle.matrices(win, read, scoring=scoring, mode=oracle.LOCAL)
        istar = int(res["ref_end"])                  # 1-based window column of the best cell
        jstar = int(res["read_end"])
        best = int(res["score"])
        assert int(H[istar, jstar]) == best
        out = flat_walk(H, oracle.codes(win), oracle.codes(read), istar, jstar, best, a, b, o, e)
        assert out is not None, (win, read, scoring)
        ops, ib, jb = out
        core = []
        for part in _cigar_runs(cig):
            if part[1] != 4:
                core.append(part)
        assert ops == core, (win, read, scoring, ops, cig)
        assert jb == int(res["read_begin"]) and ib == int(res["ref_begin"]), (win, read, ib, jb, res)
        walked += 1
        gapped += any(op != 0 for _, op in ops)
    assert walked > 200 and gapped >= 5, (walked, gapped)


def _cigar_runs(cig: str):
    runs, num = [], ""
    for ch in cig:
        if ch.isdigit():
            num += ch
        else:
            runs.append((int(num), oracle.OPS.index(ch)))
            num = ""
    return runs
