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

Readings common to all rules (Algorithm 3 leaves both implicit): the
scheduling step advances by one per assignment, and every chunk is clamped to
the iterations that remain.  ``min_chunk`` (>= 1) is a lower bound on the
chunk of SS, GSS and FAC; SS with ``min_chunk = k`` hands out k iterations per
request.
"""

STATIC, SS, GSS, FAC = 0, 1, 2, 3
NAMES = {STATIC: "STATIC", SS: "SS", GSS: "GSS", FAC: "FAC"}


def _ceil_div(a, b):
    return -(-a // b)


def get_chunk(kind, step, remaining, n, workers, min_chunk=1, fac_batch=None):
    """Chunk size for one scheduling step (Algorithm 3's getChunk).

    ``fac_batch`` carries the FAC batch chunk between calls: a dict that the
    caller keeps for the whole loop.
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
    else:
        raise ValueError("unknown schedule kind %r" % (kind,))
    return min(chunk, remaining)


def chunk_sequence(kind, n, workers, min_chunk=1):
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
        c = get_chunk(kind, step, n - scheduled, n, workers, min_chunk, state)
        sizes.append(c)
        scheduled += c
        step += 1
    return sizes


def chunk_starts(kind, n, workers, min_chunk=1):
    """Prefix form: starts[s] .. starts[s + 1] is the range of step s."""
    starts = [0]
    for c in chunk_sequence(kind, n, workers, min_chunk):
        starts.append(starts[-1] + c)
    return starts
