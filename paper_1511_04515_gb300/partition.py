"""Instance partitioning for batched runs on several GPUs (one process per GPU).

A batch of independent circuits shards with no exchange on the data path: each rank builds a
batched context from its own instances, runs it, and the per-instance results are gathered on
the host at the end.  Instances go to ranks by longest-processing-time-first on an estimated
cost (node count times the stage count or 1), which bounds the slowest rank at 4/3 of the
optimum.  A single circuit does not shard (every G^-1 couples all its nodes): replicas only.
"""
from __future__ import annotations

from typing import Callable, List, Sequence


def instance_cost(circ) -> float:
    """Relative cost of one instance: its node count (the solves and the Krylov vectors scale
    with it; the step count of one family varies much less between instances)."""
    return float(circ.n)


def lpt_partition(costs: Sequence[float], nparts: int) -> List[List[int]]:
    """Indices of `costs` split into nparts lists by the library's longest-processing-time-
    first rule (ers_partition_lpt: largest first onto the least-loaded part, ties to the
    lowest part number); each list is returned in increasing index order."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    from paper_1511_04515_gb300 import build, ers
    build.build()                     # host-only entry point of the library
    part = ers.partition_lpt(list(costs), nparts) if len(costs) else []
    parts: List[List[int]] = [[] for _ in range(nparts)]
    for i, p in enumerate(part):
        parts[int(p)].append(i)
    return parts


def run_sharded(circuits: Sequence, run: Callable[[Sequence], list], rank: int, world: int,
                gather: Callable[[object], list] = None) -> list:
    """Run this rank's share of `circuits` with run(instances) -> per-instance results, then
    gather every rank's (indices, results) and return all results in input order (on every
    rank; `gather` is an all-gather of Python objects, e.g. torch.distributed.all_gather_object
    wrapped to return the list).  With world == 1 nothing is exchanged."""
    parts = lpt_partition([instance_cost(c) for c in circuits], world)
    mine = parts[rank]
    res = run([circuits[i] for i in mine]) if mine else []
    if len(res) != len(mine):
        raise RuntimeError("run() must return one result per instance")
    if world == 1:
        return list(res)
    everything = gather((mine, list(res)))
    out = [None] * len(circuits)
    for idx, rs in everything:
        for i, r in zip(idx, rs):
            out[i] = r
    if any(r is None for r in out):
        raise RuntimeError("an instance was not run by any rank")
    return out
