"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point the header declares.  No compute call is made.  CPU only."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(mh_[a-z_0-9]+)\s*\(", src))
    typedef_fns = set(re.findall(r"\(\*\s*(mh_[a-z_0-9]+)\)", src))
    return sorted(names - typedef_fns)


@pytest.fixture(scope="module")
def lib():
    from paper_1409_7208_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("mh_pack_reads", "mh_count_kmers", "mh_mercy_kmers", "mh_build_sdbg"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    import paper_1409_7208_gb300 as mh
    assert sorted(mh.SYMBOLS) == _declared()


def test_error_strings_without_gpu(lib):
    import paper_1409_7208_gb300 as mh
    L = mh.load_library()
    assert L.mh_strerror(mh.MH_EINVAL) == b"invalid argument"
    assert L.mh_strerror(mh.MH_ETIMEOUT).startswith(b"bounded")
    # NULL arguments are rejected before any CUDA call
    assert L.mh_create(None, None) == mh.MH_EINVAL
    assert L.mh_count_kmers(None, None, 21, 2, None) == mh.MH_EINVAL
    assert L.mh_run_batch(None, None, 0, 31, 2, 1, 0, None) == mh.MH_EINVAL
    assert L.mh_sort_shape(None) == -1


def test_objects_are_sm103a():
    """Every object was compiled for sm_103a only (cuobjdump is not used: the
    build command line is the evidence)."""
    from paper_1409_7208_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
