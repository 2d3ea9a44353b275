"""ORACLE -- test infrastructure only: field-by-field comparison of library
results (sa_result rows + compacted CIGAR ops) with oracle results."""
from __future__ import annotations

import numpy as np

FIELDS = ("score", "second", "read_begin", "read_end", "ref_begin", "ref_end", "second_ref_end",
          "flags")


def compare(gpu_res, gpu_cigar, orc_res, orc_ops, max_report: int = 10):
    """Return a list of human-readable mismatches (empty when bit-exact)."""
    bad = []
    n = len(orc_res)
    if len(gpu_res) != n:
        return [f"result count {len(gpu_res)} != {n}"]
    for f in FIELDS:
        g = gpu_res[f].astype(np.int64)
        o = orc_res[f].astype(np.int64)
        idx = np.nonzero(g != o)[0]
        for k in idx[:max_report]:
            bad.append(f"job {k}: {f} gpu={g[k]} oracle={o[k]}")
    if orc_ops is not None:
        glen = gpu_res["cigar_len"].astype(np.int64)
        olen = orc_res["n_ops"].astype(np.int64)
        idx = np.nonzero(glen != olen)[0]
        for k in idx[:max_report]:
            bad.append(f"job {k}: cigar_len gpu={glen[k]} oracle={olen[k]}")
        if not len(idx):
            off = gpu_res["cigar_off"].astype(np.int64)
            for k in range(n):
                L = int(olen[k])
                if L and not np.array_equal(gpu_cigar[off[k]:off[k] + L], orc_ops[k, :L]):
                    bad.append(f"job {k}: cigar differs")
                    if len(bad) >= max_report:
                        break
    return bad
