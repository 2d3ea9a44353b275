"""The seeded input generators (CPU): the same seed gives the same bytes, and the
paired multi-candidate recipe has the structure it states (every read has its
source window among its candidates, end 2 is reverse-complemented, supports and
candidate counts in their ranges)."""
import numpy as np

import workloads

RC = bytes.maketrans(b"ACGT", b"TGCA")


def test_generators_are_deterministic():
    a = workloads.uneven(seed=3, n_jobs=500, genome_len=2_000_000)
    b = workloads.uneven(seed=3, n_jobs=500, genome_len=2_000_000)
    for f in ("reads", "read_off", "read_len", "ref_pos", "win_len", "flags"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    p = workloads.pairs(seed=3, n_pairs=300, genome_len=2_000_000)
    q = workloads.pairs(seed=3, n_pairs=300, genome_len=2_000_000)
    for f in ("ref", "reads", "read_first", "support", "ref_pos", "win_len", "flags", "read_truth"):
        assert np.array_equal(getattr(p, f), getattr(q, f))


def test_pairs_structure():
    n_pairs, n = 400, 150
    w = workloads.pairs(seed=5, n_pairs=n_pairs, genome_len=2_000_000, decoy_max=20, dup=0.3)
    first = w.read_first.astype(np.int64)
    assert first[0] == 0 and (np.diff(first) >= 1).all() and first[-1] == w.n_jobs
    counts = np.diff(first)
    assert counts.max() <= 1 + 1 + 1 + 20
    assert ((w.support >= 1) & (w.support <= 24)).all()
    assert (w.read_len == n).all()
    for r in range(w.n_reads):
        lo, hi = first[r], first[r + 1]
        end2 = r % 2 == 1
        assert (w.flags[lo:hi] == (1 if end2 else 0)).all()
        assert (w.read_off[lo:hi] == r * n).all()
        src = int(w.read_truth[r])
        # the source window: it contains the read's source span
        covers = [(int(w.ref_pos[j]) <= src and src + n <= int(w.ref_pos[j]) + int(w.win_len[j]))
                  for j in range(lo, hi)]
        assert any(covers), r
    # fragment geometry: end 2's source lies downstream of end 1's within the insert range
    ins = w.read_truth[1::2].astype(np.int64) + n - w.read_truth[0::2].astype(np.int64)
    assert (ins >= n).all() and 300 < np.median(ins) < 700
    # end 2 is the reverse complement of the fragment's last bases (up to mutations:
    # compare the first 30 bases, before most indels shift the rest)
    ident = []
    for p in range(50):
        back = bytes(w.reads[(2 * p + 1) * n:(2 * p + 2) * n]).translate(RC)[::-1]
        src = int(w.read_truth[2 * p + 1])
        ident.append(np.mean([x == y for x, y in zip(back[:30], bytes(w.ref[src:src + 30]))]))
    assert np.median(ident) >= 0.9
