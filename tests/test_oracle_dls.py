"""Pins of the oracle's loop-scheduling chunk sequences (Sec. 2.2, Algorithm 3)."""
import json
import os

import pytest

from oracle import dls

KINDS = {"STATIC": dls.STATIC, "SS": dls.SS, "GSS": dls.GSS, "FAC": dls.FAC, "FAC_PROB": dls.FAC_PROB}


def test_hand_evaluated_sequences(golden_dir):
    with open(os.path.join(golden_dir, "dls_sequences.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        seq = dls.chunk_sequence(KINDS[c["kind"]], c["n"], c["P"], cov=c.get("cov", 0.0))
        if "sizes" in c:
            assert seq == c["sizes"], c
        else:
            assert seq[: len(c["prefix"])] == c["prefix"], c
            assert len(seq) == c["count"], c


@pytest.mark.parametrize("kind", [dls.SS, dls.GSS, dls.FAC, dls.FAC_PROB])
@pytest.mark.parametrize("n,P,mc", [(0, 3, 1), (1, 1, 1), (1, 64, 1), (97, 5, 1),
                                    (1000, 7, 1), (100_000, 304, 1), (5000, 13, 8),
                                    (12345, 1, 3)])
def test_dynamic_rules_partition(kind, n, P, mc):
    seq = dls.chunk_sequence(kind, n, P, mc, cov=0.7)
    assert sum(seq) == n
    assert all(c >= 1 for c in seq)
    # every chunk except the last respects min_chunk
    assert all(c >= mc for c in seq[:-1])
    starts = dls.chunk_starts(kind, n, P, mc, cov=0.7)
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


@pytest.mark.parametrize("n,P", [(100, 4), (1000, 7), (100_000, 304), (3, 8)])
def test_fac_prob_without_variance_is_one_static_batch(n, P):
    """cov = 0 gives b_0 = 0, x_0 = 1: the first batch hands out ceil(N / P)
    per worker, i.e. the whole loop (the rule's deterministic limit)."""
    seq = dls.chunk_sequence(dls.FAC_PROB, n, P, cov=0.0)
    c = -(-n // P)
    assert all(x == c for x in seq[:-1]) and 0 < seq[-1] <= c
    assert len(seq) <= P


@pytest.mark.parametrize("n,P", [(1000, 4), (100_000, 304), (12_500, 456)])
def test_fac_prob_batches(n, P):
    """Batches of P equal chunks, non-increasing; more variance, smaller first
    batch; for j >= 1, x_j >= 2, so a batch never hands out more than half of
    what remains (plus rounding)."""
    for cov in (0.25, 1.0, 4.0):
        seq = dls.chunk_sequence(dls.FAC_PROB, n, P, cov=cov)
        firsts = seq[::P]
        for b in range(0, len(seq) - P, P):
            assert len(set(seq[b: b + P])) == 1
        assert all(y <= x for x, y in zip(firsts, firsts[1:]))
        rem = n - P * seq[0]
        for b in range(P, len(seq), P):
            assert seq[b] <= max(1, -(-rem // (2 * P))), (cov, b)
            rem -= sum(seq[b: b + P])
    f = [dls.chunk_sequence(dls.FAC_PROB, n, P, cov=cov)[0] for cov in (0.0, 0.5, 1.0, 2.0, 8.0)]
    assert all(y <= x for x, y in zip(f, f[1:]))
