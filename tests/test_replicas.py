"""The multi-GPU path is replicas only (each rank an independent chain, no
collective on the data path); what crosses ranks is the measurement: a
barrier, the maximum step time and the summed work.  Checked here with two
gloo ranks on the CPU, and the single-process fallback."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1805_03560_gb300.replicas import Replicas
    r = Replicas("gloo")
    r.barrier()
    out = dict(rank=r.rank, world=r.world, max=r.allmax(1.5 + rank),
               sum=r.allsum(10.0 * (rank + 1)), seed=r.seed(7))
    r.barrier()
    r.close()
    q.put(out)


def test_two_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in res] == [2, 2]
    # every rank sees the slowest step time and the total work
    assert [d["max"] for d in res] == [2.5, 2.5]
    assert [d["sum"] for d in res] == [30.0, 30.0]
    # independent chains: different input seeds per replica
    assert res[0]["seed"] != res[1]["seed"]


def test_single_process(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1805_03560_gb300.replicas import Replicas
    r = Replicas()
    assert (r.world, r.rank) == (1, 0)
    r.barrier()
    assert r.allmax(3.25) == 3.25 and r.allsum(4.0) == 4.0
    assert r.seed(7) == 7
    r.close()
