"""Multi-process sharding logic on CPU (gloo, world size 2): event assignment and
the combination of per-rank timings; no GPU and no data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1811_04141_gb300.shard import balance_events, combine, event_costs, events_for_rank, split_events


def test_event_assignment():
    assert events_for_rank(0, 2, 20) == list(range(0, 20))
    assert events_for_rank(1, 2, 20) == list(range(20, 40))
    shards = [list(split_events(41, r, 4)) for r in range(4)]
    assert sum(shards, []) == list(range(41))
    assert max(map(len, shards)) - min(map(len, shards)) <= 1
    with pytest.raises(ValueError):
        events_for_rank(2, 2, 5)


def test_balance_events_greedy():
    import numpy as np
    costs = [10, 1, 7, 3, 3, 8, 2, 9]
    shards = balance_events(costs, 3)
    assert sorted(sum(shards, [])) == list(range(8))            # every event once
    loads = [sum(costs[e] for e in s) for s in shards]
    assert max(loads) - min(loads) <= max(costs)                 # greedy bound
    assert shards == [[0, 1, 4], [3, 6, 7], [2, 5]] and loads == [14, 14, 15]
    # log-uniform event sizes (as in the uneven workload): within 2 % of the mean
    rng = np.random.default_rng(3)
    c = np.floor(np.exp(rng.uniform(np.log(100), np.log(20000), 512)))
    loads = [c[s].sum() for s in balance_events(c, 8)]
    assert max(loads) / np.mean(loads) < 1.02
    # contiguous shards of the same events are far less even
    cont = [c[list(split_events(512, r, 8))].sum() for r in range(8)]
    assert max(cont) / np.mean(cont) > max(loads) / np.mean(loads)
    # the cost estimate: seeds x (1 + hits per bin)
    evo = np.array([0, 100, 100, 400])
    se = np.array([0, 0, 2, 2, 2])
    assert np.allclose(event_costs(evo, se, 100), [2 * 2.0, 0.0, 3 * 4.0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = combine(dist, 100.0 * (rank + 1), 2.0 + rank)
    q.put((rank, units, ms, events_for_rank(rank, world, 3)))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, ms, evs in res:
        assert units == 300.0 and ms == 3.0          # sum of units, slowest step
        assert evs == list(range(3 * rank, 3 * rank + 3))
    assert res[0][3] != res[1][3]                    # disjoint shards
    assert combine(None, 5, 1.5) == (5.0, 1.5)


def test_reference_arm_runs_on_cpu():
    """bench.py --impl reference times the oracle on host cores and prints its line."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
