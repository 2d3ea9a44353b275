"""The C-ABI library loads on the CPU and exports every function include/sa.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libsa():
    from paper_1302_5507_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sa_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sa_create_reference", "sa_destroy_reference", "sa_align_batch",
                     "sa_align_batch_dev", "sa_server_create", "sa_submit", "sa_poll",
                     "sa_server_destroy", "sa_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libsa):
    for name in declared_functions():
        assert hasattr(libsa, name), f"{name} declared in sa.h but not exported"


def test_struct_layouts_match_header():
    import paper_1302_5507_gb300 as sa
    assert sa.JOB_DTYPE.itemsize == 32
    assert sa.RESULT_DTYPE.itemsize == 56
    assert ctypes.sizeof(sa.sa_params) == 4 * 4 + 8 * 4
    p = sa.sa_default_params()
    assert (p.sc.match, p.sc.mismatch, p.sc.gap_open, p.sc.gap_extend) == (1, 2, 2, 1)
    assert p.min_score == sa.SA_NO_SCORE and p.want_cigar == 1


def test_invalid_arguments_fail_without_gpu(libsa):
    import paper_1302_5507_gb300 as sa
    # NULL handles are rejected before any CUDA call
    assert sa.lib().sa_destroy_reference(None) == sa.SA_EINVAL
    assert "NULL" in sa.sa_last_error()
    p = sa.make_params()
    p.mode = 7
    rc, _ = sa.sa_align_batch(None, p, None, 0, None, 0, None, None, 0)
    assert rc == sa.SA_EINVAL


def test_read_level_layouts_and_null_handles(libsa):
    import paper_1302_5507_gb300 as sa
    assert sa.READ_RESULT_DTYPE.itemsize == 32
    assert ctypes.sizeof(sa.sa_select_params) == 4 * 4 + 4 + 4 + 8 + 8
    assert ctypes.sizeof(sa.sa_server_stats) == 8 * 8
    L = sa.lib()
    sp = sa.make_select_params(paired=True, frag_min=300, frag_max=700)
    assert L.sa_select(None, ctypes.byref(sp), None, None, None, 0, None) == sa.SA_EINVAL
    assert L.sa_select_dev(None, ctypes.byref(sp), None, None, None, 0, None, None) == sa.SA_EINVAL
    n = ctypes.c_uint32(0)
    assert L.sa_effort_limit(None, None, None, None, 0, 30, None, None, None, ctypes.byref(n)) == sa.SA_EINVAL
    assert L.sa_server_get_stats(None, None) == sa.SA_EINVAL
    assert "NULL" in sa.sa_last_error()


def test_seeding_layouts_and_null_handles(libsa):
    import paper_1302_5507_gb300 as sa
    assert ctypes.sizeof(sa.sa_seed_params) == 6 * 4
    p = sa.make_seed_params()
    assert (p.seed_len, p.seed_step, p.max_occ, p.pad, p.join) == (20, 10, 256, 24, 16)
    L = sa.lib()
    n = ctypes.c_uint64(7)
    assert L.sa_seed_index_create(None, None) == sa.SA_EINVAL
    assert L.sa_seed_index_destroy(None) == sa.SA_EINVAL
    assert L.sa_seed_index_info(None, None, None) == sa.SA_EINVAL
    assert L.sa_seed_candidates_dev(None, ctypes.byref(p), None, 0, None, None, 0, None, None, None, 0,
                                    ctypes.byref(n), None) == sa.SA_EINVAL
    assert L.sa_seed_candidates(None, ctypes.byref(p), None, 0, None, None, 0, None, None, None, 0,
                                ctypes.byref(n)) == sa.SA_EINVAL
    assert "NULL" in sa.sa_last_error()
