"""Multi-rank host logic on CPU with world size 2 over gloo (no GPU).

1. The benchmark's replicas: which batches each rank answers and how the
   ranks' timings combine.
2. The sharded query of the design (id range split over ranks): every rank
   counts the SC-scores of its own ids, one all-reduce of the (Ns+1)-bin
   score histogram gives the cut theta, an exclusive scan over ranks of the
   ties at theta applies the lowest-id rule, every rank re-ranks its own
   candidates, and an all-gather + merge of the local top-k gives the answer.
   The result must equal the single-process oracle.  The per-rank scores come
   from the oracle restricted to the rank's ids (the local S4 of a shard).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _replicas_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2411_14754_gb300 import replicas as R
    _init(rank, world, port)
    try:
        nb = 6
        order = R.batch_order(rank, world, nb)
        mine = order[: nb // world]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        elapsed = 10.0 + 5.0 * rank           # ms
        queries = 100.0 * (rank + 1)
        ms, q = R.reduce_throughput(dist, torch.device("cpu"), elapsed, queries, world)
        out.put((rank, gathered, ms, q))
    finally:
        dist.destroy_process_group()


def test_replicas_answer_every_batch_once_and_reduce_to_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_replicas_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = [out.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, ms, q in res:
        flat = sorted(b for part in gathered for b in part)
        assert flat == list(range(6))
        assert ms == 15.0 and q == 300.0


def _sharded_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2411_14754_gb300 import workloads as W
    _init(rank, world, port)
    try:
        n, d, Ns, sk, k = 3000, 24, 4, 6, 7
        X = W.random_data(31, n, d, "int")
        Q = W.random_data(32, 5, d, "int")
        idx = oracle.build_index(X, Ns, sk, 3, W.random_init_ids(33, n, Ns, sk))
        lo, hi = rank * n // world, (rank + 1) * n // world     # this rank's ids
        results = []
        for q in Q:
            T, C = oracle.collision_threshold(0.08, n), oracle.candidate_count(0.03, n, k)
            full = oracle.query(X, idx, q, k, T, C)            # the single-process answer
            sc = full["scores"][lo:hi]                          # local S4 of the shard
            hist = torch.tensor(np.bincount(sc, minlength=Ns + 1), dtype=torch.int64)
            dist.all_reduce(hist)                               # one small all-reduce
            ge = torch.flip(torch.cumsum(torch.flip(hist, [0]), 0), [0]).numpy()   # ge[s] = #scores >= s
            theta = max([s for s in range(1, Ns + 1) if ge[s] >= C] or [0])
            n_gt = int(ge[theta + 1]) if theta + 1 <= Ns else 0
            need_eq = C - n_gt
            eq_local = np.flatnonzero(sc == theta) + lo          # ties in id order
            cnt = torch.tensor([len(eq_local)], dtype=torch.int64)
            allc = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
            dist.all_gather(allc, cnt)
            eq_before = int(sum(int(c) for c in allc[:rank]))   # exclusive scan over ranks
            take = max(0, min(len(eq_local), need_eq - eq_before))
            cands = np.concatenate([np.flatnonzero(sc > theta) + lo, eq_local[:take]]).astype(np.int64)
            ids, dd = oracle.rerank(X, q, cands, k) if len(cands) else (np.full(k, -1), np.full(k, np.inf))
            gathered = [None] * world
            dist.all_gather_object(gathered, (ids.tolist(), dd.tolist(), cands.tolist()))
            allids = np.array([i for g in gathered for i in g[0]], dtype=np.int64)
            alld = np.array([x for g in gathered for x in g[1]])
            ok = allids >= 0
            order = np.lexsort((allids[ok], alld[ok]))[:k]
            merged = allids[ok][order]
            all_cands = sorted(c for g in gathered for c in g[2])
            results.append((merged.tolist(), full["ids"].tolist(), all_cands, sorted(full["cands"].tolist())))
        out.put((rank, results))
    finally:
        dist.destroy_process_group()


def test_sharded_query_equals_the_single_process_oracle():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_sharded_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    res = [out.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, results in res:
        for merged, single, cands, single_cands in results:
            assert cands == single_cands
            assert merged == single
