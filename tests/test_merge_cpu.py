"""Host merge of partial sums across processes (gloo, CPU ranks): the merge
equals one run over all paths, it is order-independent, and a rank that
drops out makes the others fail with an error instead of hanging."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2108_03076_gb300 import merge  # noqa: E402


def test_merge_is_fixed_order_and_matches_single_run():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(10_000) * 3 + 1
    parts = [np.array([c.sum(), (c * c).sum(), len(c)]) for c in np.array_split(x, 7)]
    m = merge.merge_sums(parts)
    price, se = merge.estimate(m)
    assert price == pytest.approx(x.mean(), rel=1e-13)
    assert se == pytest.approx(x.std(ddof=1) / np.sqrt(len(x)), rel=1e-10)
    assert m[2] == len(x)
    with pytest.raises(ValueError):
        merge.estimate([1.0, 1.0, 1.0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _send(q, msg):
    q.put(msg)
    q.close()
    q.join_thread()   # flush before the process may leave abruptly


def _worker(rank, ws, port, drop, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local = np.array([[10.0 * (rank + 1), 100.0 * (rank + 1), 5.0], [rank, rank, 1.0]])
    if drop and rank == ws - 1:
        _send(q, (rank, "dropped"))
        os._exit(0)   # leaves between steps, before the exchange
    try:
        out = merge.allgather_sums(local, timeout_s=3.0)
        _send(q, (rank, out.tolist()))
    except RuntimeError as e:
        _send(q, (rank, f"error: {e}"))
        os._exit(0)   # the peer is gone: skip process-group teardown
    dist.destroy_process_group()


def _run(ws, drop):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, drop, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=60) for _ in range(ws))
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return res


def test_two_rank_merge():
    res = _run(2, drop=False)
    want = [[10.0 + 20.0, 100.0 + 200.0, 10.0], [1.0, 1.0, 2.0]]
    assert res[0] == want and res[1] == want


def test_dropped_rank_is_detected():
    res = _run(2, drop=True)
    assert res[1] == "dropped"
    assert isinstance(res[0], str) and res[0].startswith("error") and "check in" in res[0]
