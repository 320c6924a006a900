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


def test_af_without_variance_is_the_speed_weighted_share():
    """D = 0: the chunk is R (1 / mu_i) / sum_j (1 / mu_j), so one request per
    worker hands out exactly R, each worker in proportion to its speed (for
    equal speeds GSS's R / P)."""
    mus = [1.0, 2.0, 4.0, 0.5]
    R = 1000
    xs = [dls.af_chunk(m, mus, [0.0] * 4, R) for m in mus]
    assert abs(sum(xs) - R) < 1e-9
    inv = [1.0 / m for m in mus]
    for x, w in zip(xs, inv):
        assert abs(x - R * w / sum(inv)) < 1e-9
    assert abs(dls.af_chunk(3.0, [3.0] * 8, [0.0] * 8, 800) - 100.0) < 1e-12


def test_af_hand_evaluated():
    """Two workers, mu = (1, 2), sigma^2 = (1, 4), R = 10, by hand: D = 1/1 +
    4/2 = 3, E = 1 / (1 + 1/2) = 2/3, ER = 20/3; worker 1 gets
    (3 + 40/3 - sqrt(9 + 80)) / 2 = 3.44968..., worker 2 half that."""
    x1 = dls.af_chunk(1.0, [1.0, 2.0], [1.0, 4.0], 10)
    x2 = dls.af_chunk(2.0, [1.0, 2.0], [1.0, 4.0], 10)
    assert abs(x1 - (3.0 + 40.0 / 3.0 - 89.0 ** 0.5) / 2.0) < 1e-12
    assert abs(x1 - 3.4496761) < 1e-6
    assert abs(x2 - x1 / 2.0) < 1e-12


@pytest.mark.parametrize("seed", range(5))
def test_af_chunk_time_plus_deviation_is_the_share_of_the_rest(seed):
    """T = mu_i x_i satisfies T + sqrt(D T) = E R with 0 <= T <= E R; larger
    variances give smaller chunks; the chunk grows with R."""
    import random
    rng = random.Random(seed)
    P = rng.randint(1, 64)
    mus = [rng.uniform(0.1, 10.0) for _ in range(P)]
    var = [rng.uniform(0.0, 4.0) * m * m for m in mus]
    R = rng.randint(1, 100_000)
    i = rng.randrange(P)
    x = dls.af_chunk(mus[i], mus, var, R)
    D = sum(v / m for m, v in zip(mus, var))
    E = 1.0 / sum(1.0 / m for m in mus)
    T = mus[i] * x
    assert 0.0 <= T <= E * R * (1 + 1e-12)
    assert abs(T + (D * T) ** 0.5 - E * R) <= 1e-9 * E * R
    assert dls.af_chunk(mus[i], mus, [2.0 * v + 0.1 for v in var], R) < x
    assert dls.af_chunk(mus[i], mus, var, 2 * R) > x
