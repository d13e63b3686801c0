"""Multi-rank plumbing of bench.py on the CPU: two gloo ranks (127.0.0.1).

The data path has no collective (streams are sharded across ranks); the
bench only needs a barrier and the max of the ranks' step times. These tests
run bench.Dist in two processes and check both, and check that a rank that
fails between steps makes the other rank's next barrier raise, not hang.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.barrier()
    m = d.max(10.0 * (rank + 1))
    d.barrier()
    q.put((rank, d.world, m))
    d.close()


def test_two_gloo_ranks_barrier_and_max():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert res == [(0, 2, 20.0), (1, 2, 20.0)]


def _rank_fails(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(timeout_s=20.0)
    d.barrier()  # step 1 done on both ranks
    if rank == 1:
        raise SystemExit(3)  # rank 1 fails between steps, with nothing in flight
    try:
        d.barrier()
        q.put((rank, "no error"))
    except Exception as e:  # the peer is gone: the barrier must raise
        q.put((rank, "raised: " + type(e).__name__))


def test_a_failed_rank_makes_the_next_barrier_raise():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_fails, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes[1] == 3, codes
    rank, what = q.get(timeout=5)
    assert rank == 0 and what.startswith("raised"), what
