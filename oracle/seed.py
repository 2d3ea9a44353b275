"""ORACLE -- test infrastructure only (see oracle/__init__.py for who may import it).

Plain restatement of the seeding front end that produces the candidate windows
of a read (Methods, "Implementation details of SOAP3-dp", step 3, and "Effort
limit for dynamic programming"): seeds are taken at regular intervals along the
read and along its reverse complement, aligned back to the reference, and the
regions their hits point to become candidate windows, each scored by its
number of supporting seeds.

The paper leaves the seed length, the interval, the treatment of repetitive
seeds, the merging of hits into regions and the window margins to its
supplementary material, which is not available; the readings used here are:

* seeds: for a read of length n and each strand (the read as given, then its
  reverse complement), the substrings of length ``lam`` at offsets
  0, step, 2*step, ... while offset + lam <= n;
* occurrences: every reference position p with ref[p : p + lam] equal to the
  seed (exact matches); a seed with more than ``max_occ`` occurrences is too
  repetitive and contributes none;
* a hit of the seed at offset o on position p implies the strand's sequence
  starts at d = p - o (its diagonal);
* regions: per read and strand, the hits sorted by (d, seed index) are cut
  where two consecutive diagonals differ by more than ``join``; a region's
  window is [max(0, d_min - pad), min(L, d_max + n + pad)), at most
  SA_MAX_WINDOW bases from its start;
* support: the number of distinct seeds with a hit in the region;
* order: the forward regions by d_min, then the reverse-complement regions by
  d_min; reverse-complement candidates carry the job flag FLAG_RC.

Finding the positions of a lambda-mer uses a sort of all lambda-mers of the
reference as the grouping step (equal codes become adjacent); it computes
exactly the set {p : ref[p:p+lam] == seed}, with no index structure of the
library's kind (no BWT, no occurrence counts, no lookup table).
"""
from __future__ import annotations

import numpy as np

FLAG_RC = 1
MAX_WINDOW = 65536

_CODE = np.full(256, 255, np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _CODE[_c] = _i
    _CODE[ord(chr(_c).lower())] = _i


def codes(seq_u8: np.ndarray) -> np.ndarray:
    """2-bit codes A=0 C=1 G=2 T=3 of an ASCII sequence (anything else raises)."""
    c = _CODE[np.asarray(seq_u8, np.uint8)]
    if (c == 255).any():
        raise ValueError("sequence has a base other than A, C, G, T")
    return c


def revcomp_codes(c: np.ndarray) -> np.ndarray:
    return (3 - c[::-1]).astype(np.uint8)


def kmer_code(c: np.ndarray) -> int:
    v = 0
    for x in c:
        v = (v << 2) | int(x)
    return v


class KmerTable:
    """All lam-mers of a reference, grouped: the code of ref[p:p+lam] for every
    p in 0..L-lam, and the positions ordered by (code, p)."""

    def __init__(self, ref_u8: np.ndarray, lam: int):
        if not 1 <= lam <= 32:
            raise ValueError("lam must be 1..32")
        c = codes(ref_u8).astype(np.uint64)
        self.L = len(c)
        self.lam = lam
        npos = self.L - lam + 1
        if npos <= 0:
            self.sorted_codes = np.zeros(0, np.uint64)
            self.order = np.zeros(0, np.int64)
            return
        acc = np.zeros(npos, np.uint64)
        for i in range(lam):
            acc = (acc << np.uint64(2)) | c[i:i + npos]
        self.order = np.argsort(acc, kind="stable")
        self.sorted_codes = acc[self.order]

    def occurrences(self, seed_code: int) -> np.ndarray:
        """Ascending positions p with ref[p:p+lam] == the seed."""
        key = np.uint64(seed_code)
        lo = int(np.searchsorted(self.sorted_codes, key, "left"))
        hi = int(np.searchsorted(self.sorted_codes, key, "right"))
        return self.order[lo:hi]


def read_regions(table: KmerTable, read_codes: np.ndarray, step: int, max_occ: int, pad: int,
                 join: int):
    """Regions of one strand's sequence: list of (ref_pos, win_len, support, d_min)."""
    lam, L = table.lam, table.L
    n = len(read_codes)
    hits = []                                        # (d, seed index)
    k = 0
    for o in range(0, n - lam + 1, step):
        occ = table.occurrences(kmer_code(read_codes[o:o + lam]))
        if 0 < len(occ) <= max_occ:
            for p in occ:
                hits.append((int(p) - o, k))
        k += 1
    hits.sort()
    regions = []
    i = 0
    while i < len(hits):
        j = i
        while j + 1 < len(hits) and hits[j + 1][0] - hits[j][0] <= join:
            j += 1
        d_min, d_max = hits[i][0], hits[j][0]
        start = max(0, d_min - pad)
        end = min(L, d_max + n + pad)
        end = min(end, start + MAX_WINDOW)
        support = len({s for _, s in hits[i:j + 1]})
        regions.append((start, end - start, support, d_min))
        i = j + 1
    return regions


def seed_candidates(ref_u8, reads_u8, read_off, read_len, *, lam=20, step=10, max_occ=256, pad=24,
                    join=16, table: KmerTable | None = None):
    """Candidate windows of every read.

    Returns a dict of per-candidate arrays (read_off uint64, read_len uint32,
    flags uint32, ref_pos uint64, win_len uint32, support uint32) and read_first
    (uint64, n_reads + 1): read r owns candidates read_first[r] .. read_first[r+1]-1."""
    table = table or KmerTable(ref_u8, lam)
    if table.lam != lam:
        raise ValueError("table built for another seed length")
    reads_u8 = np.asarray(reads_u8, np.uint8)
    cols = {k: [] for k in ("read_off", "read_len", "flags", "ref_pos", "win_len", "support")}
    first = [0]
    for r in range(len(read_len)):
        o, n = int(read_off[r]), int(read_len[r])
        fwd = codes(reads_u8[o:o + n])
        for flag, seq in ((0, fwd), (FLAG_RC, revcomp_codes(fwd))):
            for start, wl, sup, _ in read_regions(table, seq, step, max_occ, pad, join):
                cols["read_off"].append(o)
                cols["read_len"].append(n)
                cols["flags"].append(flag)
                cols["ref_pos"].append(start)
                cols["win_len"].append(wl)
                cols["support"].append(sup)
        first.append(len(cols["ref_pos"]))
    dt = {"read_off": np.uint64, "read_len": np.uint32, "flags": np.uint32, "ref_pos": np.uint64,
          "win_len": np.uint32, "support": np.uint32}
    out = {k: np.asarray(v, dt[k]) for k, v in cols.items()}
    return out, np.asarray(first, np.uint64)
