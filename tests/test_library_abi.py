"""The C-ABI library builds for sm_103a, loads, and exports every symbol
that include/ms.h declares (no compute calls: no GPU needed)."""
import re
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_builds_and_exports_header_symbols():
    from paper_2209_04487_gb300 import build
    build.build()
    import ctypes
    lib = ctypes.CDLL(build.LIB)
    hdr = open(os.path.join(ROOT, "include", "ms.h")).read()
    names = set(re.findall(r"\b(ms_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in sorted(names):
        assert hasattr(lib, n), n
    from paper_2209_04487_gb300 import binding
    assert set(binding.EXPORTED) == names


def test_status_strings():
    from paper_2209_04487_gb300 import binding as B
    codes = (B.MS_OK, B.MS_EINVAL, B.MS_ENOMEM, B.MS_ECUDA, B.MS_ENUMERIC, B.MS_ETIMEOUT,
             B.MS_EUNSUPPORTED, B.MS_EIO)
    texts = [B.LIB.ms_status_string(code) for code in codes]
    assert all(texts) and b"unknown status" not in texts and len(set(texts)) == len(codes)
