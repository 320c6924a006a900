"""The C ABI library loads and exports every entry point that include/spin.h
declares; host-only entry points agree with the oracle (no GPU needed)."""
import os
import re

import numpy as np
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


@pytest.mark.parametrize("cov", [0.0, 0.25, 0.7, 1.0, 3.5, 100.0])
@pytest.mark.parametrize("units,workers,mc", [(1000, 4, 1), (12_500, 456, 1), (100_000, 304, 2), (7, 64, 1),
                                              (0, 8, 1), (250_000, 1, 1)])
def test_library_fac_prob_tables_match_oracle(lib, cov, units, workers, mc):
    """Probabilistic factoring: both sides evaluate the rule in IEEE double,
    from the same FP32 value of cov."""
    import paper_1811_00901_gb300 as spin
    c32 = float(np.float32(cov))
    expect = dls.chunk_starts(dls.FAC_PROB, units, workers, mc, cov=c32)
    got = spin.si_schedule_chunks(spin.make_schedule("FAC_PROB", min_chunk=mc, fac_cov=cov), units, workers)
    assert got == expect


def test_candidate_threshold_matches_oracle(lib):
    import oracle
    import paper_1811_00901_gb300 as spin
    for W, B in [(16, 0.05), (32, 0.01), (64, 0.005), (4, 1.0), (2, 0.3), (128, 0.001)]:
        assert spin.si_candidate_rc2(W, B) == oracle.candidate_rc2(W, B)


def test_nearest_bin_threshold_covers_every_counted_pair(lib):
    """The library culls the nearest-bin count at si_candidate_rc2_binned; the
    oracle's counted pairs (all-pairs, no culling) must all lie within it."""
    import oracle
    import paper_1811_00901_gb300 as spin
    from paper_1811_00901_gb300 import workloads as wl
    pts, nrm = wl.heightfield(2500, 8)
    for W, B in [(16, 0.05), (32, 0.01), (5, 0.1)]:
        _, _, dmax = oracle.spin_images_nearest(pts, nrm, W, B, -1.0, query_idx=np.arange(0, 2500, 5).astype(np.int32))
        assert float(dmax.max()) <= spin.si_candidate_rc2_binned(W, B, "NEAREST")
        assert spin.si_candidate_rc2_binned(W, B, "BILINEAR") == spin.si_candidate_rc2(W, B)


def test_invalid_chunk_table_args(lib):
    import ctypes
    n = ctypes.c_int64()
    assert lib.si_chunk_table(9, 10, 2, 1, None, 0, ctypes.byref(n)) != 0
    assert lib.si_chunk_table(0, 10, 0, 1, None, 0, ctypes.byref(n)) != 0
    assert lib.si_last_error()
    import paper_1811_00901_gb300 as spin
    bad = spin.make_schedule("FAC_PROB", fac_cov=-1.0)
    assert lib.si_schedule_chunks(ctypes.byref(bad), 10, 2, None, 0, ctypes.byref(n)) != 0
    bad = spin.make_schedule("FAC_PROB", fac_cov=float("nan"))
    assert lib.si_schedule_chunks(ctypes.byref(bad), 10, 2, None, 0, ctypes.byref(n)) != 0
    # the adaptive rules decide their chunks on the device: no table
    for kind in ("AWF", "AF"):
        sc = spin.make_schedule(kind)
        assert lib.si_schedule_chunks(ctypes.byref(sc), 10, 2, None, 0, ctypes.byref(n)) != 0


def test_tuning_table_json_round_trip(lib, tmp_path):
    """The tuning table is host state: load, nearest-class lookup, save, clear."""
    import json

    import paper_1811_00901_gb300 as spin
    spin.si_tune_clear()
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"entries": [
        {"W": 32, "log2n": 16, "log2m": 16, "kind": 3, "min_chunk": 2, "num_workers": 0, "group": 16,
         "grid_div": 8, "order": 1, "ms": 8.5},
        {"W": 16, "log2n": 12, "log2m": 12, "kind": 1, "min_chunk": 1, "num_workers": 304, "group": 32,
         "grid_div": 4, "ms": 0.3}]}))
    spin.si_tune_load(str(path))
    s = spin.si_tune_lookup(32, 100_000, 100_000)  # log2 = 16: exact class
    assert (s.kind, s.min_chunk, s.group, s.grid_div, s.order) == (3, 2, 16, 8, 1)
    s = spin.si_tune_lookup(32, 150_000, 40_000)  # nearest class with the same W
    assert s.kind == 3
    s = spin.si_tune_lookup(16, 4096, 4096)
    assert (s.kind, s.num_workers, s.group, s.order) == (1, 304, 32, 0)  # no "order": grid order
    assert spin.si_tune_lookup(64, 4096, 4096) is None  # no entry for W = 64
    out = tmp_path / "u.json"
    spin.si_tune_save(str(out))
    d = json.loads(out.read_text())
    assert len(d["entries"]) == 2
    spin.si_tune_clear()
    assert spin.si_tune_lookup(32, 100_000, 100_000) is None
    spin.si_tune_load(str(out))
    assert spin.si_tune_lookup(32, 100_000, 100_000).grid_div == 8
    assert spin.si_tune_lookup(32, 100_000, 100_000).order == 1
    spin.si_tune_clear()
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"W": 8, "log2n": 1, "log2m": 1, "kind": 9, "min_chunk": 1, '
                   '"num_workers": 0, "group": 1, "grid_div": 1}]}')
    with pytest.raises(spin.SpinError):
        spin.si_tune_load(str(bad))


@pytest.mark.parametrize("W,group,binning", [(1, 0, 0), (129, 0, 0), (32, 3, 0), (32, 0, 7)])
def test_default_workers_rejects_bad_arguments(W, group, binning):
    """Argument checks come before any device query, so they hold without a GPU."""
    import paper_1811_00901_gb300 as spin
    with pytest.raises(spin.SpinError) as e:
        spin.si_default_workers(W, spin.make_schedule("FAC", group=group, binning=binning))
    assert e.value.status == spin.SI_ERR_INVALID
