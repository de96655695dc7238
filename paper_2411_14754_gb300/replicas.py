"""Host logic of running the query path on several GPUs as independent
replicas (one process per GPU, each with its own index copy): which query
batches a rank answers, and how the ranks' timings combine into one
throughput figure.  No collective runs on the data path; the only collectives
combine timings after the timed region.
"""


def batch_order(rank: int, world: int, nb: int):
    """The batches rank `rank` of `world` answers in step order: step s takes
    batch (rank + s * world) mod nb, so that over nb/world steps the ranks
    together answer every batch once (when world divides nb)."""
    return [(rank + i * world) % nb for i in range(nb)]


def reduce_throughput(tdist, device, elapsed_ms: float, queries: float, world: int):
    """(slowest rank's elapsed ms, total queries over the ranks): the job's
    throughput is queries / elapsed.  With world == 1 nothing is reduced."""
    if world <= 1:
        return float(elapsed_ms), float(queries)
    import torch
    t = torch.tensor([float(elapsed_ms), float(queries)], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    tdist.all_reduce(mx, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(sm, op=tdist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])
