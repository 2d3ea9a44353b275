"""ORACLE -- test infrastructure only (see oracle/__init__.py for who may import it).

Plain Python restatement of the read-level steps that follow the alignment of
a read's candidate windows (Methods, "Effort limit for dynamic programming"
and "Paired-end alignment"; Experiments, mapping quality):

* ``effort_limit``: of the candidate windows of each read keep the ``ceiling``
  with the most supporting seeds.  The paper ranks candidates by their number
  of supporting seeds and aligns only the best ``ceiling`` of them; ties are
  not covered there and go to the earlier candidate here.  Kept candidates
  stay in their input order.
* ``select``: per read, the best aligned candidate (score, then smallest
  reference end, then earliest job), the second-best hit at a distinct
  location over all the read's hits, and a mapping quality from the two.
  With ``paired`` the reads 2p and 2p+1 are the two ends of fragment p: the
  best properly paired combination (orientation and fragment length within
  [frag_min, frag_max]) is chosen when one exists; otherwise each end is
  reported on its own (the paper aligns the ends individually then).

The paper fixes neither the mapping-quality formula (it adopts BWA's scoring
so that its qualities are compatible) nor the tie rules; the readings used
are stated on each function.  Everything here is integer arithmetic over the
per-job results of the alignment (``oracle.RESULT_DTYPE`` or the library's
result records: fields score, second, ref_begin, ref_end, second_ref_end,
flags).
"""
from __future__ import annotations

import numpy as np

NO_SCORE = -(2 ** 31)
NO_JOB = 0xFFFFFFFF
MAPQ_MAX = 60
EMPTY, BELOW_MIN = 1, 2          # per-job result flags
FLAG_RC = 1                      # job flag: the read was reverse-complemented

# read result flags
ALIGNED, PAIRED, PROPER, MATE_ALIGNED, REVERSE = 1, 2, 4, 8, 16
PAIR_FR, PAIR_FF = 0, 1

READ_DTYPE = np.dtype([("job", np.uint32), ("score", np.int32), ("second", np.int32),
                       ("mapq", np.int32), ("flags", np.uint32), ("n_cand", np.uint32),
                       ("frag_len", np.int64)])


def effort_limit(support, read_first, ceiling):
    """Indices of the kept candidates (ascending) and the per-read offsets into them.

    Read r owns candidates read_first[r] .. read_first[r+1]-1.  A candidate is
    kept when fewer than ``ceiling`` candidates of its read rank above it, a
    candidate ranking above another when it has more supporting seeds, or as
    many and comes earlier."""
    kept, first = [], [0]
    for r in range(len(read_first) - 1):
        lo, hi = int(read_first[r]), int(read_first[r + 1])
        for c in range(lo, hi):
            above = 0
            for k in range(lo, hi):
                if support[k] > support[c] or (support[k] == support[c] and k < c):
                    above += 1
            if above < ceiling:
                kept.append(c)
        first.append(len(kept))
    return np.array(kept, np.int64), np.array(first, np.int64)


def mapq_of(best, second, match, mismatch):
    """Mapping quality from the best score and the second-best score at another
    location (reading): 60 without a second hit, 0 when the second is as good,
    else 20 per mismatch-equivalent (match + mismatch score units) of the gap
    between them, at most 60."""
    if second == NO_SCORE:
        return MAPQ_MAX
    d = int(best) - int(second)
    if d <= 0:
        return 0
    if match + mismatch <= 0:
        return MAPQ_MAX
    return min(MAPQ_MAX, (20 * d) // (match + mismatch))


def _aligned(res, j):
    return (int(res["flags"][j]) & (EMPTY | BELOW_MIN)) == 0


def _begin(res, read_len, j):
    """Leftmost reference base of job j's alignment; without a traceback
    (ref_begin -1) the read is taken as ungapped: ref_end - n."""
    b = int(res["ref_begin"][j])
    return b if b >= 0 else int(res["ref_end"][j]) - int(read_len[j])


def _second_around(res, cands, end, n):
    """Best hit of the read (each aligned job's best and its own second) whose
    reference end is at least n from ``end``."""
    s = NO_SCORE
    for j in cands:
        if not _aligned(res, j):
            continue
        for sc, e in ((int(res["score"][j]), int(res["ref_end"][j])),
                      (int(res["second"][j]), int(res["second_ref_end"][j]))):
            if sc == NO_SCORE:
                continue
            if abs(e - end) >= n and sc > s:
                s = sc
    return s


def _single(res, read_len, flags, cands, match, mismatch):
    best = None
    for j in cands:
        if not _aligned(res, j):
            continue
        key = (-int(res["score"][j]), int(res["ref_end"][j]), j)
        if best is None or key < best[0]:
            best = (key, j)
    if best is None:
        return None
    j = best[1]
    second = _second_around(res, cands, int(res["ref_end"][j]), int(read_len[j]))
    return j, second, mapq_of(int(res["score"][j]), second, match, mismatch)


def _frag(res, read_len, flags, j1, j2, orientation, fmin, fmax):
    """Fragment length if jobs j1 (end 1) and j2 (end 2) are properly paired, else None.

    FR: one end forward and the other reverse-complemented; the fragment runs
    from the forward end's first base to the reverse end's last base.  FF: both
    ends on the same strand; on the forward strand end 1 comes first, on the
    reverse strand end 2 does."""
    s1, s2 = int(flags[j1]) & FLAG_RC, int(flags[j2]) & FLAG_RC
    if orientation == PAIR_FR:
        if s1 == s2:
            return None
        f, r = (j1, j2) if s1 == 0 else (j2, j1)
        frag = int(res["ref_end"][r]) - _begin(res, read_len, f)
    else:
        if s1 != s2:
            return None
        first, last = (j1, j2) if s1 == 0 else (j2, j1)
        frag = int(res["ref_end"][last]) - _begin(res, read_len, first)
    return frag if fmin <= frag <= fmax else None


def select(jobs_flags, read_len, res, read_first, *, match=1, mismatch=2, paired=False,
           orientation=PAIR_FR, frag_min=0, frag_max=0):
    """Per-read results (READ_DTYPE) from the per-job results ``res``.

    jobs_flags / read_len: the jobs' flags and read lengths; read_first: per-read
    candidate offsets (length n_reads + 1)."""
    n_reads = len(read_first) - 1
    out = np.zeros(n_reads, READ_DTYPE)
    out["job"] = NO_JOB
    out["second"] = NO_SCORE
    cands = [range(int(read_first[r]), int(read_first[r + 1])) for r in range(n_reads)]
    singles = [_single(res, read_len, jobs_flags, cands[r], match, mismatch) for r in range(n_reads)]

    def put(r, j, second, mapq, extra):
        out["job"][r] = j
        out["score"][r] = int(res["score"][j])
        out["second"][r] = second
        out["mapq"][r] = mapq
        out["flags"][r] = ALIGNED | extra | (REVERSE if int(jobs_flags[j]) & FLAG_RC else 0)

    for r in range(n_reads):
        out["n_cand"][r] = len(cands[r])
    if not paired:
        for r in range(n_reads):
            if singles[r] is not None:
                put(r, *singles[r], 0)
        return out

    for p in range(n_reads // 2):
        r1, r2 = 2 * p, 2 * p + 1
        best = None
        proper = []
        for j1 in cands[r1]:
            if not _aligned(res, j1):
                continue
            for j2 in cands[r2]:
                if not _aligned(res, j2):
                    continue
                fr = _frag(res, read_len, jobs_flags, j1, j2, orientation, frag_min, frag_max)
                if fr is None:
                    continue
                total = int(res["score"][j1]) + int(res["score"][j2])
                proper.append((j1, j2, total))
                key = (-total, j1, j2)
                if best is None or key < best[0]:
                    best = (key, j1, j2, total, fr)
        mate1 = MATE_ALIGNED if singles[r2] is not None else 0
        mate2 = MATE_ALIGNED if singles[r1] is not None else 0
        out["flags"][r1] = PAIRED
        out["flags"][r2] = PAIRED
        if best is None:
            # no proper pair: each end on its own
            if singles[r1] is not None:
                put(r1, *singles[r1], PAIRED | mate1)
            else:
                out["flags"][r1] |= mate1
            if singles[r2] is not None:
                put(r2, *singles[r2], PAIRED | mate2)
            else:
                out["flags"][r2] |= mate2
            continue
        _, c1, c2, total, fr = best
        e1, e2 = int(res["ref_end"][c1]), int(res["ref_end"][c2])
        n1, n2 = int(read_len[c1]), int(read_len[c2])
        pair_second = NO_SCORE
        for j1, j2, t in proper:
            if abs(int(res["ref_end"][j1]) - e1) >= n1 or abs(int(res["ref_end"][j2]) - e2) >= n2:
                pair_second = max(pair_second, t)
        pair_mapq = mapq_of(total, pair_second, match, mismatch)
        for r, c, e, n in ((r1, c1, e1, n1), (r2, c2, e2, n2)):
            second = _second_around(res, cands[r], e, n)
            q = max(pair_mapq, mapq_of(int(res["score"][c]), second, match, mismatch))
            put(r, c, second, q, PAIRED | PROPER | MATE_ALIGNED)
            out["frag_len"][r] = fr
    return out
