"""Splitting a batch of independent systems across ranks (host logic of the multi-GPU path).

The systems of a batched solve share nothing (each has its own graph, noise maps and
parameters), so a batch shards across GPUs with no communication on the data path: every
rank solves its own subset with one ``sylv_solve_batched`` call.  The per-iteration cost of a
system is proportional to its pixels times sources times right-hand sides (every kernel of the
iteration streams n k values per right-hand side), so the subsets are balanced on that work.
"""


def partition_batch(work, world):
    """Disjoint subsets of ``range(len(work))``, one per rank, with nearly equal total work:
    the largest system first, each to the rank with the least work so far (longest-processing-
    time-first; the heaviest rank exceeds the mean by less than the largest single system).
    Ties go to the lower rank, so every rank computes the same split.  Each subset is
    returned in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    loads = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += work[i]
    return [sorted(p) for p in parts]
