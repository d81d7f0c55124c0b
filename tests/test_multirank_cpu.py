"""The multi-GPU path of batched runs, on CPU: instances partitioned over two gloo ranks with
no exchange on the data path, results gathered on the host at the end.  Each rank runs its
share with the oracle (the CUDA path needs a GPU; the partition and gather logic is the same),
and the gathered results must equal a single-process run instance by instance."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1511_04515_gb300.partition import lpt_partition, run_sharded, instance_cost


def test_lpt_partition_covers_every_instance_once():
    rng = np.random.default_rng(0)
    costs = rng.integers(1, 1000, size=37).astype(float)
    for k in (1, 2, 3, 8):
        parts = lpt_partition(costs, k)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(37))
        loads = [costs[p].sum() for p in parts]
        # LPT bound: the largest load is at most 4/3 of the best possible makespan, which is at
        # least max(mean load, largest item)
        assert max(loads) <= 4 / 3 * max(costs.sum() / k, costs.max()) + 1e-9


def test_lpt_partition_edge_cases():
    assert lpt_partition([], 3) == [[], [], []]
    assert lpt_partition([5.0], 2) == [[0], []]
    with pytest.raises(ValueError):
        lpt_partition([1.0], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _circuits():
    from synth import circuits as S
    return [S.random_rc(n=8 + 3 * k, seed=k, t_end=20e-12) for k in range(5)]


def _run_oracle(insts):
    from oracle import ers_oracle as O
    out = []
    for c in insts:
        x, t, st = O.er_run(c, t_end=c.t_end, tol=1e-6, x0=np.zeros(c.n))
        out.append((x, st.steps))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def gather(obj):
        lst = [None] * world
        dist.all_gather_object(lst, obj)
        return lst

    circs = _circuits()
    calls = []

    def run(insts):
        calls.append(len(insts))
        return _run_oracle(insts)

    res = run_sharded(circs, run, rank, world, gather)
    dist.destroy_process_group()
    q.put((rank, calls, [(np.asarray(x), s) for x, s in res]))


def test_two_rank_sharded_run_matches_single_process():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circs = _circuits()
    parts = lpt_partition([instance_cost(c) for c in circs], world)
    ref = _run_oracle(circs)
    for rank, calls, res in got:
        assert calls == [len(parts[rank])]          # each rank ran only its own share
        assert len(res) == len(circs)
        for (x, s), (xr, sr) in zip(res, ref):
            assert s == sr and np.array_equal(x, xr)


def test_missing_share_is_reported():
    """The host gather notices an instance that no rank returned (a rank whose results were
    lost) and a run() that returns the wrong number of results."""
    circs = _circuits()
    parts = lpt_partition([instance_cost(c) for c in circs], 2)

    def run(insts):
        return [("ok", c.n) for c in insts]

    def gather_dropping_rank1(obj):
        return [obj]                     # rank 1's (indices, results) never arrive

    with pytest.raises(RuntimeError, match="not run by any rank"):
        run_sharded(circs, run, 0, 2, gather_dropping_rank1)
    with pytest.raises(RuntimeError, match="one result per instance"):
        run_sharded(circs, lambda insts: [], 0, 2, lambda o: [o, o])
    assert parts[0] and parts[1]


def _dying_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)                      # dies between steps, before the gather

    def gather(obj):
        lst = [None] * world
        dist.all_gather_object(lst, obj)
        return lst

    try:
        run_sharded(_circuits(), lambda insts: [c.n for c in insts], rank, world, gather)
        q.put((rank, "returned"))
    except Exception as ex:             # the peer's absence must surface as an error
        q.put((rank, "error: " + type(ex).__name__))


def test_rank_that_dies_is_detected_by_the_survivor():
    """A rank that exits before the result gather: the surviving rank's collective ends with
    an error (peer closed, or the 10 s process-group timeout) instead of waiting forever."""
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dying_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        rank, outcome = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert rank == 0 and outcome.startswith("error"), outcome
