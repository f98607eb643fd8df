"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point that include/dmrg_rotate.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "dmrg_rotate.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^DMRG_API\s+[\w\s\*]+?\b(dmrg_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0909_5662_gb300 import build
    return build.build()


def test_header_declares_boundary():
    syms = declared_symbols()
    for name in ("dmrg_rotate_ops", "dmrg_rotate_ops_blocked", "dmrg_rotate_ops_backward",
                 "dmrg_orthonormality_error", "dmrg_correlations", "dmrg_create", "dmrg_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(dmrg_\w+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    # and nothing but the C ABI leaks out
    assert exported == set(declared_symbols())


def test_library_loads_and_binding_matches(libpath):
    from paper_0909_5662_gb300 import _capi
    lib = _capi.load()
    for name in declared_symbols():
        assert hasattr(lib, name)
    assert set(_capi.exported_names()) == set(declared_symbols())
    assert lib.dmrg_status_string(0) == b"DMRG_OK"
    assert lib.dmrg_status_string(6) == b"DMRG_ERR_TIMEOUT"


def test_null_handle_is_rejected(libpath):
    from paper_0909_5662_gb300 import _capi
    lib = _capi.load()
    n = ctypes.c_size_t()
    assert lib.dmrg_rotate_ops_workspace(None, 1, 4, 4, 4, 3, ctypes.byref(n)) == 1
    assert lib.dmrg_destroy(None) == 1
    assert lib.dmrg_create(None) == 1


def test_library_is_sm103a_only(libpath):
    from paper_0909_5662_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_umd_partition():
    from paper_0909_5662_gb300 import umd_partition
    for L in (0, 1, 7, 150, 152):
        for p in (1, 2, 3, 8):
            parts = [umd_partition(L, p, r) for r in range(p)]
            assert parts[0][0] == 0 and parts[-1][1] == L
            for (a, b), (c, _) in zip(parts, parts[1:]):
                assert b == c
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
            # the first L mod p ranks hold the extra operator
            assert sizes == sorted(sizes, reverse=True)


def _header_enum(name):
    text = open(HEADER).read()
    body = re.search(r"typedef enum \{([^}]*)\}\s*" + name + r";", text).group(1)
    return {k: int(v) for k, v in re.findall(r"(DMRG_\w+)\s*=\s*(\d+)", body)}


def test_binding_enums_match_header():
    # the Python names of options and precisions carry the header's values
    from paper_0909_5662_gb300 import _capi
    opts = _header_enum("dmrg_option")
    assert {("DMRG_OPT_" + k.upper()): v for k, v in _capi.OPTION.items()} == opts
    precs = _header_enum("dmrg_precision")
    assert {("DMRG_PREC_" + k.upper()): v for k, v in _capi.PRECISION.items()} == precs
