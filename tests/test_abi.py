"""The C ABI library loads and exports every entry point that include/spin.h
declares; host-only entry points agree with the oracle (no GPU needed)."""
import os
import re

import pytest

from oracle import dls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "spin.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(si_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1811_00901_gb300 import _build
    _build.build()
    import paper_1811_00901_gb300 as spin
    return spin.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("si_mesh_create", "si_generate", "si_generate_batched", "si_serve_create",
                     "si_serve_submit", "si_serve_wait", "si_get_stats", "si_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_1811_00901_gb300 as spin
    assert set(_declared()) <= set(spin.exported_names())


@pytest.mark.parametrize("kind", ["STATIC", "SS", "GSS", "FAC"])
@pytest.mark.parametrize("units,workers,mc", [(100, 4, 1), (1000, 7, 1), (3125, 304, 1), (1, 152, 1),
                                              (5000, 13, 8), (0, 5, 1), (12, 40, 3)])
def test_library_chunk_tables_match_oracle(lib, kind, units, workers, mc):
    import paper_1811_00901_gb300 as spin
    k = {"STATIC": dls.STATIC, "SS": dls.SS, "GSS": dls.GSS, "FAC": dls.FAC}[kind]
    expect = dls.chunk_starts(k, units, workers, mc if k != dls.STATIC else 1)
    got = spin.si_chunk_table(kind, units, workers, mc)
    assert got == expect


def test_candidate_threshold_matches_oracle(lib):
    import oracle
    import paper_1811_00901_gb300 as spin
    for W, B in [(16, 0.05), (32, 0.01), (64, 0.005), (4, 1.0), (2, 0.3), (128, 0.001)]:
        assert spin.si_candidate_rc2(W, B) == oracle.candidate_rc2(W, B)


def test_invalid_chunk_table_args(lib):
    import ctypes
    n = ctypes.c_int64()
    assert lib.si_chunk_table(9, 10, 2, 1, None, 0, ctypes.byref(n)) != 0
    assert lib.si_chunk_table(0, 10, 0, 1, None, 0, ctypes.byref(n)) != 0
    assert lib.si_last_error()
