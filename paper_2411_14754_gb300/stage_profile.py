"""Per-stage cycle split of the query kernel.

Runs one batch of a workload through suco_query_debug with only the stage
clocks requested (the kernel's normal path plus a clock64 stamp by thread 0
of every CTA at each stage boundary) and prints, per stage, the mean cycles
per (query, CTA) and the share of the query's time.  Stage boundaries follow
the kernel's barriers, so a stage's time includes the wait at its closing
barrier.

  python -m paper_2411_14754_gb300.stage_profile --workload 5 --alpha 0.04 --beta 0.0036
"""
import argparse
import json

import numpy as np
import torch

from . import suco as S
from . import workloads as W

STAGES = [  # (name, first slot, last slot)
    ("S0 thresholds, query row", 1, 2),
    ("S1-S3 centroid distances, ranks, cell cut", 2, 3),
    ("cluster barrier 1 (wait)", 3, 4),
    ("copy of the other CTAs' tables", 4, 5),
    ("S4 SC-score scan", 5, 6),
    ("S4 counters to bit planes", 6, 7),
    ("S5 score counts", 7, 8),
    ("cluster barrier 2 (wait)", 8, 9),
    ("S5 cut", 9, 10),
    ("S5 candidate hand-off", 10, 11),
    ("cluster barrier 3 (wait)", 11, 12),
    ("S6 distances of the candidates", 12, 13),
    ("S6 local top-k and hand-off", 13, 14),
    ("cluster barrier 4 (wait)", 14, 15),
]


def profile(index, Qd, k, alpha, beta, **kw):
    """Stage clocks [nq][16][20] of one launch (after one untimed warm-up launch)."""
    S.suco_query_batch(index, Qd, k, alpha, beta, **kw)
    out = S.suco_query_debug(index, Qd, k, alpha, beta, want=("stage_clock",), **kw)
    torch.cuda.synchronize()
    return out["stage_clock"].cpu().numpy()


def summarise(clk):
    rows = clk[:, :, 1] != -1
    CL = int(rows.sum(axis=1).max())
    c = clk[:, :CL, :].astype(np.float64)
    total = c[:, :, 15] - c[:, :, 1]
    res = []
    for name, a, b in STAGES:
        d = c[:, :, b] - c[:, :, a]
        res.append(dict(stage=name, cycles=float(d.mean()), share=float(d.sum() / total.sum())))
    merge = c[:, 0, 16] - c[:, 0, 15]
    res.append(dict(stage="merge of the local top-k lists (CTA 0)", cycles=float(merge.mean()),
                    share=float(merge.sum() / (c[:, 0, 16] - c[:, 0, 1]).sum())))
    seg = dict(list_segments=float(c[:, :, 18].mean()), scan=float(c[:, :, 19].mean()))
    return dict(cluster_size=CL, queries=int(clk.shape[0]), mean_query_cycles=float(total.mean()),
                stages=res, s4_split=seg)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", type=int, default=5)
    p.add_argument("--alpha", type=float, default=None)
    p.add_argument("--beta", type=float, default=None)
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--precision", default="fp32")
    p.add_argument("--json", action="store_true")
    a = p.parse_args(argv)
    w = W.WORKLOADS[a.workload]
    X = torch.from_numpy(W.dataset(w.number)).cuda()
    index = S.suco_build_index(X, w.Ns, w.sqrtK, w.kmeans_iters,
                               init_ids=W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK))
    del X
    if a.precision != "fp32":
        S.suco_add_reduced_copies(index)
    Q = torch.from_numpy(W.queries(w.number, nq=a.batch or w.batch)).cuda()
    alpha = w.alpha if a.alpha is None else a.alpha
    beta = w.beta if a.beta is None else a.beta
    res = summarise(profile(index, Q, w.k, alpha, beta, precision=a.precision))
    res.update(workload=w.name, alpha=alpha, beta=beta, precision=a.precision)
    if a.json:
        print(json.dumps(res))
    else:
        print(f"{w.name}, alpha={alpha}, beta={beta}, {a.precision} re-rank, {res['queries']} queries, "
              f"clusters of {res['cluster_size']}: {res['mean_query_cycles']:.0f} cycles per query and CTA")
        print("| stage | cycles per query and CTA | share |\n|---|---|---|")
        for r in res["stages"]:
            print(f"| {r['stage']} | {r['cycles']:.0f} | {100 * r['share']:.1f} % |")
        sp = res["s4_split"]
        print(f"\nS4 scan: {sp['list_segments']:.0f} cycles listing segments, {sp['scan']:.0f} scanning")
    S.suco_free(index)


if __name__ == "__main__":
    main()
