"""The multi-process product path: each "rank" prices its own path range of
one contract with pc_price_async (Philox counters use the global path
index), two gloo CPU processes merge the ranks' (sum, sum of squares, n)
with merge.allgather_sums, and the merged result equals one launch over the
union of the ranges: n exactly, the sums to FP64 rounding (they add the
same per-path values in another order), the price and standard error to
1e-12.  The ranks' triples are recorded from real launches on this GPU;
the merging processes are spawned and touch no GPU."""
import os
import socket

import numpy as np
import pytest

from gpu_common import Engine, torch
import workloads as W
from paper_2108_03076_gb300 import merge

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, local, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    out = merge.allgather_sums(np.asarray(local), timeout_s=30.0)
    q.put((rank, out.tolist()))
    dist.destroy_process_group()


def test_ranks_merge_to_one_launch_over_the_union():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    eng = Engine()
    try:
        w = W.worst_of_autocall()
        m, k = eng.model(w.market), eng.contract(w.il_text, w.tparams)
        n, ranks = (1 << 18) + 64 * 5 + 3, 2
        full = eng.sums(m, k, ranks * n, w.seed)
        parts = [eng.sums(m, k, n, w.seed, offset=r * n) for r in range(ranks)]
    finally:
        eng.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ranks, port, [list(parts[r][:3])], q)) for r in range(ranks)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(ranks))
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    got = np.asarray(res[0])[0]
    assert res[0] == res[1]
    assert got[2] == ranks * n == full[2]
    np.testing.assert_allclose(got[:2], full[:2], rtol=1e-13, atol=0)
    pm, sm = merge.estimate(got)
    pf, sf = merge.estimate(full[:3])
    assert pm == pytest.approx(pf, rel=1e-12) and sm == pytest.approx(sf, rel=1e-9)
