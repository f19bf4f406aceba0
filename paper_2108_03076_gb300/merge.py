"""Host-side merge of Monte Carlo partial sums across path ranges and processes.

Paths are independent and their Philox counters use the global path index,
so pricing the ranges [r*N, (r+1)*N) on R processes and adding the
per-range triples (sum x, sum x^2, n) gives the same estimator as one run
over R*N paths.  The merge is a fixed-order sum (rank 0, 1, ...), so the
result does not depend on arrival order.  Only these three doubles per
contract cross process boundaries; nothing on the data path is a
collective.
"""
from __future__ import annotations

import math
from datetime import timedelta
from typing import Iterable, Sequence, Tuple

import numpy as np


def merge_sums(parts: Iterable[Sequence[float]]) -> np.ndarray:
    """Fixed-order sum of (sum, sumsq, n) triples (rows); returns [3]."""
    out = np.zeros(3, dtype=np.float64)
    for p in parts:
        p = np.asarray(p, dtype=np.float64)
        out += p[:3]
    return out


def estimate(sums: Sequence[float]) -> Tuple[float, float]:
    """(price, standard error) from a merged (sum, sumsq, n) triple."""
    s, s2, n = float(sums[0]), float(sums[1]), float(sums[2])
    if n < 2:
        raise ValueError("need at least two paths for a standard error")
    mean = s / n
    var = max(0.0, (s2 - n * mean * mean) / (n - 1.0))
    return mean, math.sqrt(var / n)


def allgather_sums(local: np.ndarray, timeout_s: float = 30.0, group=None) -> np.ndarray:
    """Merge per-rank triples over a torch.distributed process group with a
    CPU backend (the default group, or `group`, e.g. a gloo group beside an
    NCCL default): every rank contributes `local` ([k, 3] for k contracts)
    and gets the fixed-order merge [k, 3].  Before the exchange each rank
    checks in through the default store; a rank that has not checked in
    within `timeout_s` makes every waiting rank raise RuntimeError instead
    of blocking in the collective."""
    import torch
    import torch.distributed as dist

    local = np.atleast_2d(np.asarray(local, dtype=np.float64))
    ws, rank = dist.get_world_size(group), dist.get_rank(group)
    store = _store()
    key = f"pc_merge_{_next_round()}"
    store.set(f"{key}/{rank}", "1")
    try:
        store.wait([f"{key}/{r}" for r in range(ws)], timedelta(seconds=timeout_s))
    except Exception as e:  # noqa: BLE001 - the store raises a backend-specific error
        raise RuntimeError(f"merge: a rank did not check in within {timeout_s} s") from e
    t = torch.from_numpy(local.copy())
    parts = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(parts, t, group=group)
    return np.stack([merge_sums([p.numpy()[i] for p in parts]) for i in range(local.shape[0])])


_round = [0]


def _next_round() -> int:
    _round[0] += 1
    return _round[0]


def _store():
    import torch.distributed as dist
    from torch.distributed import distributed_c10d as c10d
    pg = dist.group.WORLD
    st = c10d._get_default_store() if hasattr(c10d, "_get_default_store") else None
    if st is None:
        raise RuntimeError("no torch.distributed store available")
    return st
