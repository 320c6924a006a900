"""Chunk sequences of the loop-scheduling rules (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and bench.py's CPU legs may import
this module.  It shares no code with the CUDA library.

The scheduled loop is the outer loop over images (Algorithm 1, "Parallel for
i = 0 -> N").  The master of Algorithm 3 repeatedly calls
getChunk(DM, schedulingStep, N, workersCount) and hands out the range
[scheduledTasks, scheduledTasks + chunk).  The rules (Sec. 2.2):

* STATIC -- N / P contiguous iterations per worker, decided before the loop
  runs (PSIA, Sec. 2.1).  Reading for P not dividing N: worker k receives
  [floor(k N / P), floor((k + 1) N / P)).
* SS     -- one iteration per request.
* GSS    -- the remaining iterations divided by the number of workers,
  rounded up (guided self-scheduling); reading: never below ``min_chunk``.
* FAC    -- batches of P equal chunks.  The paper gives no batch-size rule;
  reading: each batch hands out chunks of ceil(R / (2 P)) (the usual FAC2
  rule, R = iterations remaining when the batch starts), never below
  ``min_chunk``.

* FAC_PROB -- factoring with the batch size of its original probabilistic
  rule (Hummel, Schonberg and Flynn 1992, the paper's reference for FAC),
  for iterations whose times have coefficient of variation cov = sigma / mu:
  at the start of batch j, with R_j iterations remaining,
  b_j = P / (2 sqrt(R_j)) * cov, x_0 = 1 + b_0^2 + b_0 sqrt(b_0^2 + 2),
  x_j = 2 + b_j^2 + b_j sqrt(b_j^2 + 4) for j >= 1, and the batch hands out
  P chunks of ceil(R_j / (x_j P)), never below ``min_chunk``.  The rule's
  quantities are real numbers; they are evaluated in IEEE double in this
  order, and the ceiling taken of the double quotient.

* AF -- adaptive factoring (Banicescu and Liu 2000), one of the "more
  complex" rules the paper leaves to future work.  Worker i, whose time per
  iteration has mean mu_i and variance sigma_i^2, asks for a chunk while R
  iterations remain and receives
  x_i = (D + 2 E R - sqrt(D^2 + 4 D E R)) / (2 mu_i),
  D = sum_j sigma_j^2 / mu_j, E = 1 / sum_j 1 / mu_j (see ``af_chunk``).
  With T = mu_i x_i, the chunk's expected time, T is the smaller root of
  T^2 - (D + 2 E R) T + (E R)^2 = 0, i.e. T + sqrt(D T) = E R: the time of
  the chunk plus a deviation allowance equals one worker's share of the
  remaining work.  Without variance (D = 0) the chunk is the worker's
  speed-weighted share of R, R (1 / mu_i) / sum_j (1 / mu_j).  The rule's
  inputs are measured while the loop runs, so it has no chunk table.

Readings common to all rules (Algorithm 3 leaves both implicit): the
scheduling step advances by one per assignment, and every chunk is clamped to
the iterations that remain.  ``min_chunk`` (>= 1) is a lower bound on the
chunk of SS, GSS and FAC; SS with ``min_chunk = k`` hands out k iterations per
request.
"""

import math

STATIC, SS, GSS, FAC, FAC_PROB = 0, 1, 2, 3, 4
NAMES = {STATIC: "STATIC", SS: "SS", GSS: "GSS", FAC: "FAC", FAC_PROB: "FAC_PROB"}


def _ceil_div(a, b):
    return -(-a // b)


def fac_prob_batch_chunk(batch, remaining, workers, cov):
    """The probabilistic factoring chunk of batch ``batch`` (see FAC_PROB)."""
    b = workers / (2.0 * math.sqrt(remaining)) * cov
    if batch == 0:
        x = 1.0 + b * b + b * math.sqrt(b * b + 2.0)
    else:
        x = 2.0 + b * b + b * math.sqrt(b * b + 4.0)
    return int(math.ceil(remaining / (x * workers)))


def af_chunk(mu_i, mus, variances, remaining):
    """Adaptive factoring's chunk (real-valued, before rounding) for a worker
    with mean iteration time ``mu_i``, given every worker's mean time ``mus``
    and variance ``variances`` and ``remaining`` iterations (see AF)."""
    d = sum(v / m for m, v in zip(mus, variances))
    e = 1.0 / sum(1.0 / m for m in mus)
    r = float(remaining)
    return (d + 2.0 * e * r - math.sqrt(d * d + 4.0 * d * e * r)) / (2.0 * mu_i)


def get_chunk(kind, step, remaining, n, workers, min_chunk=1, fac_batch=None, cov=0.0):
    """Chunk size for one scheduling step (Algorithm 3's getChunk).

    ``fac_batch`` carries the FAC batch chunk between calls: a dict that the
    caller keeps for the whole loop.  ``cov`` is FAC_PROB's sigma / mu.
    """
    min_chunk = max(1, int(min_chunk))
    if kind == STATIC:
        k = step
        chunk = (k + 1) * n // workers - k * n // workers
    elif kind == SS:
        chunk = min_chunk
    elif kind == GSS:
        chunk = max(min_chunk, _ceil_div(remaining, workers))
    elif kind == FAC:
        if step % workers == 0:
            fac_batch["c"] = max(min_chunk, _ceil_div(remaining, 2 * workers))
        chunk = fac_batch["c"]
    elif kind == FAC_PROB:
        if step % workers == 0:
            fac_batch["c"] = max(min_chunk, fac_prob_batch_chunk(step // workers, remaining, workers, cov))
        chunk = fac_batch["c"]
    else:
        raise ValueError("unknown schedule kind %r" % (kind,))
    return min(chunk, remaining)


def chunk_sequence(kind, n, workers, min_chunk=1, cov=0.0):
    """The master loop of Algorithm 3 run to completion, without workers.

    Returns the list of chunk sizes in the order they are handed out.  For
    STATIC the list has exactly ``workers`` entries (some may be 0 when
    N < P); for the dynamic rules every entry is >= 1 and they sum to N.
    """
    if n < 0 or workers < 1:
        raise ValueError("need n >= 0 and workers >= 1")
    scheduled = 0
    step = 0
    sizes = []
    state = {}
    if kind == STATIC:
        for k in range(workers):
            sizes.append(get_chunk(STATIC, k, n - scheduled, n, workers))
            scheduled += sizes[-1]
        return sizes
    while scheduled < n:
        c = get_chunk(kind, step, n - scheduled, n, workers, min_chunk, state, cov)
        sizes.append(c)
        scheduled += c
        step += 1
    return sizes


def chunk_starts(kind, n, workers, min_chunk=1, cov=0.0):
    """Prefix form: starts[s] .. starts[s + 1] is the range of step s."""
    starts = [0]
    for c in chunk_sequence(kind, n, workers, min_chunk, cov):
        starts.append(starts[-1] + c)
    return starts
