"""Pins of the oracle's loop-scheduling chunk sequences (Sec. 2.2, Algorithm 3)."""
import json
import os

import pytest

from oracle import dls

KINDS = {"STATIC": dls.STATIC, "SS": dls.SS, "GSS": dls.GSS, "FAC": dls.FAC}


def test_hand_evaluated_sequences(golden_dir):
    with open(os.path.join(golden_dir, "dls_sequences.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        seq = dls.chunk_sequence(KINDS[c["kind"]], c["n"], c["P"])
        if "sizes" in c:
            assert seq == c["sizes"], c
        else:
            assert seq[: len(c["prefix"])] == c["prefix"], c
            assert len(seq) == c["count"], c


@pytest.mark.parametrize("kind", [dls.SS, dls.GSS, dls.FAC])
@pytest.mark.parametrize("n,P,mc", [(0, 3, 1), (1, 1, 1), (1, 64, 1), (97, 5, 1),
                                    (1000, 7, 1), (100_000, 304, 1), (5000, 13, 8),
                                    (12345, 1, 3)])
def test_dynamic_rules_partition(kind, n, P, mc):
    seq = dls.chunk_sequence(kind, n, P, mc)
    assert sum(seq) == n
    assert all(c >= 1 for c in seq)
    # every chunk except the last respects min_chunk
    assert all(c >= mc for c in seq[:-1])
    starts = dls.chunk_starts(kind, n, P, mc)
    assert starts[0] == 0 and starts[-1] == n
    assert all(b > a for a, b in zip(starts, starts[1:]))


@pytest.mark.parametrize("n,P", [(100, 4), (1000, 7), (100_000, 304), (31, 64)])
def test_gss_non_increasing(n, P):
    seq = dls.chunk_sequence(dls.GSS, n, P)
    assert all(b <= a for a, b in zip(seq, seq[1:]))
    assert seq[0] == -(-n // P)


@pytest.mark.parametrize("n,P", [(100, 4), (1000, 7), (100_000, 304)])
def test_fac_batches(n, P):
    seq = dls.chunk_sequence(dls.FAC, n, P)
    # batches of P equal chunks (the final batch may be cut short / clamped)
    for b in range(0, len(seq) - P, P):
        batch = seq[b: b + P]
        assert len(set(batch)) == 1
    # each batch hands out about half of what remains
    rem = n
    for b in range(0, len(seq), P):
        c = seq[b]
        assert c == max(1, -(-rem // (2 * P))) or c == rem
        rem -= sum(seq[b: b + P])


def test_ss_is_unit():
    assert dls.chunk_sequence(dls.SS, 17, 4) == [1] * 17
    assert dls.chunk_sequence(dls.SS, 17, 4, min_chunk=5) == [5, 5, 5, 2]


@pytest.mark.parametrize("n,P", [(0, 4), (3, 8), (100, 4), (101, 4), (100_000, 304)])
def test_static_blocks(n, P):
    seq = dls.chunk_sequence(dls.STATIC, n, P)
    assert len(seq) == P
    assert sum(seq) == n
    assert max(seq) - min(seq) <= 1
