"""The N > 1 path of bench.py on the CPU: world_size-2 gloo ranks.  Every rank runs its own
replica (no collective on the data path); the job's time is the slowest rank's, taken with
one all-reduce MAX, and the throughput is all ranks' units over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, world, device="cpu")
    value = bench.replica_throughput(1e6, ms_max, world)
    r, w, lr = bench._dist_env()
    dist.barrier()
    q.put((rank, ms_max, value, r, w))
    dist.destroy_process_group()


def test_two_gloo_ranks_time_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, r, w in out:
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1e6 / 0.150)
        assert (r, w) == (rank, 2)


def _replica_worker(rank, world, port, q):
    """One rank of the replicas path with a real solve on it: the rank's own seeded workload
    (bench.py seeds the quadrant + vortex state with the rank), three steps of the oracle as
    the rank's solver, its own wall time, then the one all-reduce of the timing."""
    import sys
    import time
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle as O
    from paper_2402_03074_gb300 import inputs as I
    w = I.quadrant_vortex_2d(rank, 64, window=(16, 16, 24, 20))
    P = O.Problem(dim=2, eq=O.EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1, y0=w.y0, y1=w.y1,
                  bc=w.bc)
    dist.barrier()
    t0 = time.perf_counter()
    U, t, ns, st = O.run(P, w.U0, 0.0, 1e9, max_steps=3)
    ms = 1e3 * (time.perf_counter() - t0)
    ms_max = bench.max_over_ranks(ms, world, device="cpu")
    units = w.nx * w.ny * 3 * ns
    value = bench.replica_throughput(units, ms_max, world)
    dist.barrier()
    q.put((rank, ms, ms_max, value, units, st, U.sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    """Each rank solves its own seeded replica with no data exchange: its result equals the
    same solve run alone in this process, the two ranks' states differ (their seeds), and the
    job's throughput is both ranks' cell-stages over the slower rank's time."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    from paper_2402_03074_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms_max = max(o[1] for o in out)
    for rank, ms, mx, value, units, st, usum in out:
        assert st == 0 and mx == pytest.approx(ms_max)
        assert value == pytest.approx(2 * units / (ms_max / 1e3))
        w = I.quadrant_vortex_2d(rank, 64, window=(16, 16, 24, 20))
        P = O.Problem(dim=2, eq=O.EULER, nx=w.nx, ny=w.ny, x0=w.x0, x1=w.x1, y0=w.y0,
                      y1=w.y1, bc=w.bc)
        assert usum == O.run(P, w.U0, 0.0, 1e9, max_steps=3)[0].sum()
    assert out[0][6] != out[1][6]


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(10.0, 1000.0, 1) == 10.0
