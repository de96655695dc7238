"""Benchmark of the SuCo query path on one GB300 (or N, one process per GPU).

A step is one batch of queries through the whole query path (centroid
distances, cell activation, SC-score counting, candidate selection, exact
re-rank, top-k).  Default workload: 1,000,000 points, d=256, drawn from a hard
Gaussian mixture (2000 components, sigma log-uniform in [0.5, 8], 10% uniform
noise), Ns=16, sqrtK=50, k=10, 10,000 evaluation queries in batches of 1024.
There the ratio network (trained first on this GPU from plain-SuCo labels on
200,000 training queries) predicts each query's alpha and beta: a step is one
predict launch and one query launch.  Both the learned arm and the plain
fixed-ratio arm are timed at their fastest operating point whose mean
recall@10 reaches 0.95 on the evaluation queries.  Other workloads
(--workload 1..4) time the plain path at the workload's own alpha and beta.
The index is built on the GPU beforehand; queries are resident in device
memory for the timed value and copied from pinned host memory for the
end-to-end figure.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 5] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (launched by torchrun) every rank
holds its own index replica and answers its own query batches (no data-path
collective); the value is the total over ranks divided by the slowest rank.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2411_14754_gb300 import replicas  # noqa: E402 (which batches a rank answers, timing reduction)

METRIC = "QPS at recall@10>=0.95 on 1 GB300, learned-alpha/BF16 vs plain FP32; % HBM peak"
# the side lines (fixed operating points, SC-Linear) do not target a recall
METRIC_FIXED = "QPS at a fixed alpha/beta on 1 GB300 (recall reported, not targeted); % HBM peak"
METRIC_SCL = "QPS of SC-Linear (Algorithm 1, no index) at a fixed alpha/beta on 1 GB300"
UNIT = "queries/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--workload", type=int, default=5)
    p.add_argument("--n-train", type=int, default=0, help="training queries of the ratio network "
                   "(0: the workload's own count)")
    p.add_argument("--target-recall", type=float, default=0.95)
    p.add_argument("--impl", default="suco", choices=["suco", "reference"])
    p.add_argument("--cluster-size", type=int, default=0)
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--recall-sample", type=int, default=256)
    p.add_argument("--plain", action="store_true", help="time the fixed-ratio path at the workload's own alpha and "
                   "beta even where the workload trains the ratio network")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline sample")
    p.add_argument("--exact-rerank", type=int, default=512, help="survivors of the BF16/FP8 coarse re-rank")
    p.add_argument("--guard", type=float, default=0.002,
                   help="operating points are chosen on the validation split at target + guard")
    p.add_argument("--margin-candidates", type=int, default=6,
                   help="cheapest margin pairs (by modelled bytes) timed for the learned arm")
    p.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp8"],
                   help="re-rank precision of the fixed-ratio path")
    p.add_argument("--label-mode", default="full", choices=["full", "lagrange"],
                   help="per-query training labels of the ratio network (learn.labels_from_recalls)")
    p.add_argument("--sc-linear", action="store_true", help="time SC-Linear (Algorithm 1, no index) instead")
    p.add_argument("--build", action="store_true", help="time the index build (Algorithm 2) instead")
    p.add_argument("--rank-precision", default="fp32", choices=["fp32", "bf16", "fp8"],
                   help="centroid-distance arithmetic of the fixed-ratio path (bf16: tensor cores)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def workload_config(w, batch=None):
    """The workload as both arms name it (the method each arm runs is reported
    outside this dict)."""
    return {"workload": f"{w.name}: n={w.n}, d={w.d}, Ns={w.Ns}, sqrtK={w.sqrtK}, k={w.k}",
            "stands_in_for": w.stands_in_for, "queries": w.nq, "batch": w.batch if batch is None else batch,
            "l2": "inputs larger than L2 (dataset copy in HBM >> 129 MB)", "parallelism": "query-sharded replicas"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("suco_query.cu", "suco_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2411_14754_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(workload, operating_point=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (and, where given, at the same operating-point
    setup); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
    except Exception:
        return None
    e = t.get(str(workload))
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None
    if operating_point is not None and e.get("operating_point") != operating_point:
        return None
    return e.get("dram_bytes_per_launch")


def learned_setup(L, label_mode, margin):
    """What decides the learned arm's operating points: the label grid and
    mode and the chosen margins (a traffic record holds for these only)."""
    return {"labels": label_mode, "alpha_grid": list(L.ALPHA_GRID), "beta_grid": list(L.BETA_GRID),
            "margin": [float(m) for m in margin]}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), reasons=parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r["reasons"]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes_per_query(w, T, C, teff_mean_total):
    """Bytes the method must move per query: the uint32 ids of the retrieved
    cells (sum over subspaces of T_eff) and the C candidate rows (d FP32).
    The SC-score array never leaves shared memory, so it adds nothing."""
    return 4.0 * teff_mean_total + 4.0 * C * w.d


def run_cpu_baseline(w, X, Q, threads, alpha=None, beta=None, target_s=15.0):
    """The FP64 oracle on the host cores over a bounded sample of the same
    workload: a probe of 2*threads queries sizes the sample to about
    target_s seconds of CPU work."""
    import oracle
    alpha = w.alpha if alpha is None else alpha
    beta = w.beta if beta is None else beta
    T = oracle.collision_threshold(alpha, w.n)
    C = oracle.candidate_count(beta, w.n, w.k)
    from paper_2411_14754_gb300 import workloads as W
    t0 = time.time()
    idx = oracle.build_index(X, w.Ns, w.sqrtK, 2, W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK),
                             nthreads=threads)
    build_s = time.time() - t0
    probe = min(len(Q), 2 * threads)
    t0 = time.time()
    oracle.query_batch(X, idx, Q[:probe], w.k, T, C, rank_precision=0, nthreads=threads)
    per_q = (time.time() - t0) / probe
    sample_q = int(min(len(Q), max(probe, round(target_s / max(per_q, 1e-9)))))
    t0 = time.time()
    oracle.query_batch(X, idx, Q[:sample_q], w.k, T, C, rank_precision=0, nthreads=threads)
    dt = time.time() - t0
    return {"value": sample_q / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {sample_q} of the {len(Q)} queries of the same workload at alpha={alpha}, "
                      f"beta={beta}, FP64 oracle (Algorithms 3-4), OpenMP over queries on {threads} host threads; "
                      f"oracle index built with 2 Lloyd iterations in {build_s:.1f}s (index build not timed)",
            "seconds": dt}


def run_cpu_baseline_on_index(pkg, index, w, X, Q, gt, T, C, target_s=10.0):
    """The FP64 oracle (Algorithms 3-4) answering from the GPU's own index
    (exported with suco_export_index) at the same per-query thresholds T_b and
    C_b, single-threaded and with OpenMP over queries on every host core.  Each
    run is a bounded sample (about target_s seconds of CPU work, sized by a
    probe); its recall@k is measured against the same exact k-NN."""
    import oracle
    from paper_2411_14754_gb300 import learn as L
    ex = pkg.suco_export_index(index)
    idx = dict(Ns=w.Ns, sqrtK=w.sqrtK, centroids=ex["centroids"], cell_off=ex["cell_off"].astype(np.int64),
               perm=ex["perm"].astype(np.int64))
    T = np.asarray(T, dtype=np.int64)
    C = np.asarray(C, dtype=np.int64)
    runs = {}
    for threads in sorted({1, oracle.max_threads()}):
        probe = min(len(Q), 2 * threads)
        t0 = time.time()
        oracle.query_batch(X, idx, Q[:probe], w.k, T[:probe], C[:probe], rank_precision=0, nthreads=threads)
        per_q = (time.time() - t0) / probe
        m = int(min(len(Q), max(probe, round(target_s / max(per_q, 1e-9)))))
        t0 = time.time()
        ids, _ = oracle.query_batch(X, idx, Q[:m], w.k, T[:m], C[:m], rank_precision=0, nthreads=threads)
        dt = time.time() - t0
        runs[threads] = {"value": m / dt, "queries": m, "seconds": dt,
                         "recall_at_k": float(L.recall_rows(ids, gt[:m]).mean())}
    allc = max(runs)
    return {"value": runs[allc]["value"], "unit": UNIT, "cores": allc, "kind": "oracle",
            "sample": (f"the first {runs[allc]['queries']} evaluation queries, FP64 oracle (Algorithms 3-4) on the "
                       f"GPU-built index (suco_export_index) at the same per-query T_b, C_b, OpenMP over queries on "
                       f"{allc} host threads"),
            "seconds": runs[allc]["seconds"], "recall_at_k": runs[allc]["recall_at_k"],
            "single_thread": runs[1], "index": "the GPU-built index, exported", "mean_T": float(T[:runs[allc]['queries']].mean()),
            "mean_C": float(C[:runs[allc]["queries"]].mean())}


def exact_knn_host(X, Qs, k, shortlist=64, chunk=64):
    """Exact k nearest ids (ties by id) on the host: an FP32 matrix product
    shortlists candidates, FP64 differences decide among them."""
    xn = (X.astype(np.float64) ** 2).sum(1)
    out = np.empty((len(Qs), k), np.int64)
    for s0 in range(0, len(Qs), chunk):
        q = Qs[s0:s0 + chunk]
        d = xn[None, :] - 2.0 * (q @ X.T).astype(np.float64)
        cand = np.argpartition(d, shortlist, axis=1)[:, :shortlist]
        for j in range(len(q)):
            c = cand[j]
            ex = ((X[c].astype(np.float64) - q[j].astype(np.float64)) ** 2).sum(1)
            out[s0 + j] = c[np.lexsort((c, ex))[:k]]
    return out


def run_reference(args):
    """The oracle (FP64, Algorithms 3-4, OpenMP over queries) on the host cores:
    the workload's own index build (same initial ids, same Lloyd iterations,
    untimed) and its fixed ratios alpha, beta; each step answers a bounded
    sample of the evaluation queries."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2411_14754_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    X = W.dataset(w.number)
    Q = W.queries(w.number)
    threads = oracle.max_threads()
    T = oracle.collision_threshold(w.alpha, w.n)
    C = oracle.candidate_count(w.beta, w.n, w.k)
    idx = oracle.build_index(X, w.Ns, w.sqrtK, w.kmeans_iters, W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK),
                             nthreads=threads)
    per_step = max(threads, 16)
    times = []
    answered = []
    for s in range(args.warmup + args.steps):
        q0 = (s * per_step) % (w.nq - per_step)
        qs = Q[q0:q0 + per_step]
        t0 = time.time()
        ids, _ = oracle.query_batch(X, idx, qs, w.k, T, C, rank_precision=0, nthreads=threads)
        if s >= args.warmup:
            times.append(time.time() - t0)
            answered.append((q0, ids))
    tot = sum(times)
    value = per_step * len(times) / tot
    qsel = np.concatenate([np.arange(q0, q0 + per_step) for q0, _ in answered])
    gt = exact_knn_host(X, Q[qsel], w.k)
    got = np.concatenate([ids for _, ids in answered])
    rec = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / w.k for a, b in zip(got, gt)]))
    sample = (f"{per_step} queries per step of the same workload through the FP64 CPU oracle "
              f"(Algorithms 3-4) at alpha={w.alpha}, beta={w.beta}, OpenMP over queries on {threads} host threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w), "impl": "reference",
            "method": {"arm": "CPU oracle", "alpha": w.alpha, "beta": w.beta, "index_lloyd_iterations": w.kmeans_iters},
            "recall_at_k": rec,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precision_report(pkg, index, w, X, q0, ids_s, dist_s, rec, args, gt):
    """Relative error |d - d64| / d64 of every returned squared distance (max,
    p99), recall against FP32 and, for a tensor-core ranking, the relative
    error of its half-subspace tables against the FP64 squared distances of the
    unrounded query and centroids."""
    ids = ids_s.cpu().numpy()
    dist = dist_s.cpu().numpy().astype(np.float64)
    Q = q0.cpu().numpy()
    rel = []
    for j in range(len(Q)):
        ok = ids[j] >= 0
        d64 = ((X[ids[j][ok]].astype(np.float64) - Q[j].astype(np.float64)[None, :]) ** 2).sum(1)
        rel.append(np.abs(dist[j][ok] - d64) / np.maximum(d64, 1e-300))
    rel = np.concatenate(rel)
    out = {"result_rel_error_max": float(rel.max()), "result_rel_error_p99": float(np.percentile(rel, 99)),
           "queries": int(len(Q))}
    if args.precision != "fp32" or args.rank_precision != "fp32":
        from oracle import recall as _recall
        ids32, _ = pkg.suco_query_batch(index, q0, w.k, w.alpha, w.beta)
        out["recall_fp32"] = _recall(ids32.cpu().numpy(), np.stack(gt))
        out["recall_delta_vs_fp32"] = rec - out["recall_fp32"]
    if args.rank_precision != "fp32":
        dbg = pkg.suco_query_debug(index, q0, w.k, w.alpha, w.beta, want=("dtab",), precision=args.precision,
                                   rank_precision=args.rank_precision, exact_rerank=args.exact_rerank)
        tab = dbg["dtab"].cpu().numpy().astype(np.float64)
        cent = pkg.suco_export_index(index)["centroids"].astype(np.float64)
        s = w.d // w.Ns
        terr = []
        for i in range(w.Ns):
            ln = w.d - (w.Ns - 1) * s if i == w.Ns - 1 else s
            for h, (ho, hl) in enumerate(((i * s, ln // 2), (i * s + ln // 2, ln - ln // 2))):
                qh = Q[:, ho:ho + hl].astype(np.float64)
                ref = ((qh[:, None, :] - cent[i, h, None, :, :hl]) ** 2).sum(-1)
                terr.append((np.abs(tab[:, i, h, :] - ref) / np.maximum(ref, 1e-300)).ravel())
        terr = np.concatenate(terr)
        out["rank_table_rel_error_median"] = float(np.median(terr))
        out["rank_table_rel_error_p99"] = float(np.percentile(terr, 99))
    return out


# fixed (alpha, beta) points the plain arm may take; its operating point is the
# fastest one whose mean recall reaches the target on the evaluation queries
PLAIN_ALPHAS = (0.02, 0.05, 0.08, 0.12, 0.16, 0.2, 0.25, 0.3, 0.4)
PLAIN_BETAS = (0.002, 0.005, 0.008, 0.012, 0.016, 0.024, 0.032)


def time_loop(torch, stream, steps, warmup, fn, marks=1, label=None):
    """Runs fn(s, ev) for warmup + steps steps; a timed step may record its
    internal marks ev[0 .. marks-2]; the step's start and end are recorded
    here.  Returns (total ms, per-step ms of each of the ``marks`` parts),
    measured with CUDA events on ``stream``."""
    for s in range(warmup):
        fn(s, None)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(marks + 1)] for _ in range(steps)]
    if label:
        torch.cuda.nvtx.range_push(label)  # lets a profiler select these launches (ncu --nvtx-include)
    for s in range(steps):
        ev[s][0].record(stream)
        fn(warmup + s, ev[s][1:marks])
        ev[s][marks].record(stream)
    if label:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    total = ev[0][0].elapsed_time(ev[-1][-1])
    parts = [[ev[s][j].elapsed_time(ev[s][j + 1]) for j in range(marks)] for s in range(steps)]
    return total, parts


def note(msg, t0=[time.time()]):  # noqa: B006 (start time of the process)
    print(f"[bench {time.time() - t0[0]:7.1f}s] {msg}", file=sys.stderr, flush=True)


def run_learned(args, torch, tdist, pkg, W, rank, local_rank, world, dev):
    """Learned per-query ratios vs plain fixed ratios, each at its fastest
    operating point with mean recall@k >= target on the evaluation queries."""
    from paper_2411_14754_gb300 import learn as L
    w = W.WORKLOADS[args.workload]
    t_setup = time.time()
    X = W.dataset(w.number)
    Xd = torch.from_numpy(X).to(dev)
    t0 = time.time()
    index = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, w.kmeans_iters,
                                 init_ids=W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    note(f"index built in {build_s:.1f}s")
    # the network is trained on this GPU (setup, not timed)
    n_train = args.n_train or w.n_train
    t0 = time.time()
    Qt = torch.from_numpy(W.queries(w.number, nq=n_train, train=True)).to(dev)
    model, rep = L.fit(index, Xd, Qt, w.k, target=args.target_recall, log=note, label_mode=args.label_mode)
    del Qt
    train_s = time.time() - t0
    note(f"trained: {json.dumps(rep)}")
    Qall = W.queries(w.number)
    Qe = torch.from_numpy(Qall).to(dev)
    gt = L.exact_knn(Xd, Qe, w.k)
    del Xd
    target = args.target_recall
    stream = torch.cuda.current_stream(dev)

    pkg.suco_add_reduced_copies(index)  # BF16 copy of the dataset for the coarse re-rank
    B = w.batch
    nb = (w.nq + B - 1) // B
    batches = [Qe[i * B:(i + 1) * B] for i in range(nb)]
    order = replicas.batch_order(rank, world, nb)
    outs = [(torch.empty((b.shape[0], w.k), dtype=torch.int32, device=dev),
             torch.empty((b.shape[0], w.k), dtype=torch.float32, device=dev)) for b in batches]
    ab = [(torch.empty(b.shape[0], device=dev), torch.empty(b.shape[0], device=dev)) for b in batches]
    cur = {}

    def learned_step(s, ev, q=None):
        bi = order[s % nb]
        qb = batches[bi] if q is None else q
        pkg.suco_mlp_predict(index, cur["st"], qb, alpha=ab[bi][0], beta=ab[bi][1], stream=stream)
        if ev:
            ev[0].record(stream)
        pkg.suco_query_batch(index, qb, w.k, L.FALLBACK[0], L.BETA_RANGE[1], out_ids=outs[bi][0],
                             out_dist=outs[bi][1], alpha_per_query=ab[bi][0], beta_per_query=ab[bi][1], stream=stream,
                             precision=cur["precision"], exact_rerank=args.exact_rerank)
        return qb.shape[0]

    # Operating points are chosen on the validation split of the training
    # queries only (held out from the network's training, never the evaluation
    # queries), at the target plus a guard band of about two standard errors
    # of that split's mean recall; the evaluation recall is then measured and
    # reported as it comes out.
    Qv, gv = model.validation["Q"], model.validation["gt"]
    sel_target = target + args.guard
    vb = [Qv[i:i + B] for i in range(0, Qv.shape[0], B)]

    def val_recall_learned(prec):
        al, be = L.predict(index, model, Qv)
        ids, _ = pkg.suco_query_batch(index, Qv, w.k, L.FALLBACK[0], L.BETA_RANGE[1], alpha_per_query=al,
                                      beta_per_query=be, precision=prec, exact_rerank=args.exact_rerank)
        return float(L.recall_rows(ids.cpu().numpy(), gv).mean())

    # learned arm: margins added to the network's log alpha and log beta; every
    # pair of a grid is tried on the validation split, the pairs reaching the
    # selection target are ranked by modelled bytes, and the cheapest few are
    # timed in both re-rank precisions; the fastest is the learned arm
    by_prec = {}
    for prec in ("fp32", "bf16"):
        cands = L.margin_grid(index, model, Qv, gv, w.k, target=sel_target, precision=prec,
                              exact_rerank=args.exact_rerank)[:args.margin_candidates]
        if not cands:  # nothing reaches the target: the common margin search's answer
            m, r = L.tune_offsets(index, model, Qv, gv, w.k, target=sel_target, precision=prec,
                                  exact_rerank=args.exact_rerank)
            cands = [(0.0, m, m, r)]
        best = None
        for cost, ma, mb, r in cands:
            model.offsets = (ma, mb)
            cur.update(st=model.struct(), precision=prec)
            ms, _ = time_loop(torch, stream, 2 * nb, 2, learned_step)
            qps = 2 * w.nq / (ms / 1000.0)
            if best is None or qps > best["qps_probe"]:
                best = {"margin": [ma, mb], "val_recall": r, "qps_probe": qps, "modelled_bytes": cost}
        by_prec[prec] = best
        note(f"learned {prec}: margins {best['margin']}, validation recall {best['val_recall']:.4f}, "
             f"probe {best['qps_probe']:.0f} q/s")
    learned_prec = max(by_prec, key=lambda p: by_prec[p]["qps_probe"])
    margin = by_prec[learned_prec]["margin"]
    model.offsets = tuple(margin)
    cur.update(st=model.struct(), precision=learned_prec)
    ids_e, _ = L.query_learned(index, model, Qe, w.k, precision=learned_prec, exact_rerank=args.exact_rerank)
    rec_learned = float(L.recall_rows(ids_e.cpu().numpy(), gt).mean())
    st = cur["st"]

    def plain_step_fn(alpha, beta):
        def f(s, ev):
            bi = order[s % nb]
            pkg.suco_query_batch(index, batches[bi], w.k, alpha, beta, out_ids=outs[bi][0], out_dist=outs[bi][1],
                                 stream=stream)
        return f

    # plain arm: the fastest grid point whose validation recall reaches the selection target
    plain = None
    rec_grid = {}
    for a in PLAIN_ALPHAS:
        for bt in PLAIN_BETAS:
            ids, _ = pkg.suco_query_batch(index, Qv, w.k, a, bt)
            r = float(L.recall_rows(ids.cpu().numpy(), gv).mean())
            rec_grid[f"{a},{bt}"] = r
            if r >= sel_target:
                ms, _ = time_loop(torch, stream, 2 * nb, 2, plain_step_fn(a, bt))
                qps = 2 * w.nq / (ms / 1000.0)
                if plain is None or qps > plain["qps_probe"]:
                    plain = {"alpha": a, "beta": bt, "val_recall": r, "qps_probe": qps}
    if plain is not None:
        ids, _ = pkg.suco_query_batch(index, Qe, w.k, plain["alpha"], plain["beta"])
        plain["recall_at_k"] = float(L.recall_rows(ids.cpu().numpy(), gt).mean())
    note(f"plain operating point: {plain}")
    setup_s = time.time() - t_setup

    # timed region: the learned path, one predict + one query launch per batch
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    nq_step = [batches[order[s % nb]].shape[0] for s in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        total_ms, parts = time_loop(torch, stream, args.steps, args.warmup, learned_step, marks=2, label="timed")
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    nqueries = float(sum(nq_step))
    total_ms, all_q = replicas.reduce_throughput(tdist, dev, total_ms, nqueries, world)
    value = all_q / (total_ms / 1000.0)
    predict_ms = statistics.mean(p[0] for p in parts)
    query_ms = statistics.mean(p[1] for p in parts)

    # the plain arm timed the same way (for the comparison)
    plain_line = None
    if plain is not None:
        pms, _ = time_loop(torch, stream, args.steps, args.warmup, plain_step_fn(plain["alpha"], plain["beta"]))
        plain_line = dict(plain, value=sum(nq_step) / (pms / 1000.0), unit=UNIT, ms_per_step=pms / args.steps)
        plain_line.pop("qps_probe")

    # end to end through the public API: pinned host queries in, host results out
    hq = [b.cpu().pin_memory() for b in batches]
    hout = [(torch.empty(o[0].shape, dtype=torch.int32).pin_memory(),
             torch.empty(o[1].shape, dtype=torch.float32).pin_memory()) for o in outs]
    dq = [torch.empty_like(b) for b in batches]
    h2d = d2h = 0

    def e2e_step(s, ev):
        bi = order[s % nb]
        dq[bi].copy_(hq[bi], non_blocking=True)
        learned_step(s, None, q=dq[bi])
        hout[bi][0].copy_(outs[bi][0], non_blocking=True)
        hout[bi][1].copy_(outs[bi][1], non_blocking=True)

    e2e_ms, _ = time_loop(torch, stream, args.steps, args.warmup, e2e_step)
    for s in range(args.steps):
        bi = order[(args.warmup + s) % nb]
        h2d += hq[bi].numel() * 4
        d2h += hout[bi][0].numel() * 4 + hout[bi][1].numel() * 4
    e_ms, e_q = replicas.reduce_throughput(tdist, dev, e2e_ms, float(sum(nq_step)), world)
    e2e_value = e_q / (e_ms / 1000.0)

    # roofline of the query kernel: per query 4 * sum_i T_eff,i id bytes and
    # 4 * C_b * d row bytes, C_b from the query's own beta (with the BF16
    # re-rank: 2 * C_b * d coarse bytes and 4 * min(R, C_b) * d exact bytes)
    R = args.exact_rerank or 512
    bytes_steps = 0.0
    per_batch = {}
    for bi in set(order[(args.warmup + s) % nb] for s in range(args.steps)):
        al, be = L.predict(index, model, batches[bi])
        dbg = pkg.suco_query_debug(index, batches[bi], w.k, L.FALLBACK[0], L.BETA_RANGE[1], want=("t_eff",),
                                   alpha_per_query=al, beta_per_query=be)
        teff = float(dbg["t_eff"].double().sum().item())
        Cs = [pkg.suco_thresholds(w.n, L.FALLBACK[0], min(float(x), L.BETA_RANGE[1]), w.k)[1]
              for x in be.cpu().numpy()]
        if learned_prec == "bf16":
            rows = sum((2.0 * c + 4.0 * R) * w.d if c > R else 4.0 * c * w.d for c in Cs)
        else:
            rows = sum(4.0 * c * w.d for c in Cs)
        per_batch[bi] = 4.0 * teff + rows
    for s in range(args.steps):
        bytes_steps += per_batch[order[(args.warmup + s) % nb]]
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = bytes_steps / args.steps / (query_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": (committed_traffic(f"{w.number}-learned", learned_setup(L, args.label_mode, margin))
                            if learned_prec == "fp32" else None),
                "peak_source": peak_src,
                "kernel": f"suco_query_kernel (learned per-query alpha/beta, {learned_prec} re-rank, one launch per batch)",
                "algorithmic_bytes_per_query": bytes_steps / sum(nq_step), "mean_launch_ms": query_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as _o
        al, be = L.predict(index, model, Qe)
        a_np, b_np = al.cpu().numpy(), be.cpu().numpy()
        Tq = [_o.collision_threshold(float(a), w.n) for a in a_np]
        Cq = [_o.candidate_count(min(float(b), L.BETA_RANGE[1]), w.n, w.k) for b in b_np]
        cpu = run_cpu_baseline_on_index(pkg, index, w, X, Qall, gt, Tq, Cq, target_s=args.cpu_seconds / 2)
        cpu["operating_point"] = "the learned arm's per-query alpha_b, beta_b (thresholds T_b, C_b)"

    if rank == 0:
        cfg = workload_config(w)
        method = {"arm": "learned per-query alpha/beta", "network": f"MLP {3 * w.Ns}-{model.H}-2, GELU, BF16 weights",
                  "n_train": n_train, "labels": args.label_mode, "rerank": ("FP32" if learned_prec == "fp32" else
                                                 f"{learned_prec.upper()} coarse + exact FP32 top {R}"),
                  "selection": (f"margins and precision chosen on the {Qv.shape[0]} validation queries of the training "
                                f"set at recall >= {sel_target:.3f}; recall_at_k measured on the {w.nq} evaluation "
                                f"queries")}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "method": method, "recall_at_k": rec_learned, "k": w.k, "target_recall": target,
                "margin": margin, "learned_precision": learned_prec, "learned_by_precision": by_prec,
                "plain_fp32": plain_line,
                "speedup_vs_plain": (value / plain_line["value"]) if plain_line else None,
                "predict_ms_per_step": predict_ms, "query_ms_per_step": query_ms,
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                        "d2h_bytes_per_step": d2h // args.steps},
                "clocks": clk.summary(), "gpu_launches": 2 * args.steps,
                "index_build_s": build_s, "train_s": train_s, "setup_s": setup_s,
                "training": rep, "plain_grid_val_recall": rec_grid}
        print(json.dumps(line), flush=True)
    pkg.suco_free(index)


def run_batching(args, torch, tdist, pkg, W, rank, local_rank, world, dev):
    """A stream of queries with per-query k and alpha drawn uniformly from the
    workload's mixes: one launch per batch through the persistent kernel (each
    cluster takes the next unanswered query from a work counter), the launch
    shape picked by the autotuner, each batch's launch captured once in a CUDA
    graph and replayed in the timed region."""
    w = W.WORKLOADS[args.workload]
    X = W.dataset(w.number)
    Qall = W.queries(w.number)
    ks, als = W.per_query_mix(w.number, w.nq)
    kmax = int(max(w.k_mix))
    Xd = torch.from_numpy(X).to(dev)
    t0 = time.time()
    index = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, w.kmeans_iters,
                                 init_ids=W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    note(f"index built in {build_s:.1f}s")
    B = w.batch
    nb = (w.nq + B - 1) // B
    sl = [slice(i * B, min(w.nq, (i + 1) * B)) for i in range(nb)]
    batches = [torch.from_numpy(Qall[c]).to(dev) for c in sl]
    kq = [torch.from_numpy(ks[c].astype(np.int32)).to(dev) for c in sl]
    aq = [torch.from_numpy(als[c].astype(np.float32)).to(dev) for c in sl]
    outs = [(torch.empty((b.shape[0], kmax), dtype=torch.int32, device=dev),
             torch.empty((b.shape[0], kmax), dtype=torch.float32, device=dev)) for b in batches]
    order = replicas.batch_order(rank, world, nb)
    amax = float(max(w.alpha_mix))
    shape = pkg.suco_autotune(index, batches[0], kmax, amax, w.beta, k_per_query=kq[0], alpha_per_query=aq[0])
    note(f"autotuned launch shape (cluster size, threads): {shape}")
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))

    def launch(bi, st):
        pkg.suco_query_batch(index, batches[bi], kmax, amax, w.beta, out_ids=outs[bi][0], out_dist=outs[bi][1],
                             k_per_query=kq[bi], alpha_per_query=aq[bi], stream=st)

    mine = sorted(set(order))
    with torch.cuda.stream(stream):
        for bi in mine:
            launch(bi, stream)  # first call of each shape outside capture
    torch.cuda.synchronize()
    graphs = {}
    for bi in mine:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            launch(bi, stream)
        graphs[bi] = g
    torch.cuda.synchronize()

    def step(s, ev):
        graphs[order[s % nb]].replay()

    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    nq_step = [batches[order[s % nb]].shape[0] for s in range(args.steps)]
    with ClockSampler(local_rank) as clk, torch.cuda.stream(stream):
        total_ms, parts = time_loop(torch, stream, args.steps, args.warmup, step, label="timed")
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    total_ms, all_q = replicas.reduce_throughput(tdist, dev, total_ms, float(sum(nq_step)), world)
    value = all_q / (total_ms / 1000.0)
    mean_launch_ms = total_ms / args.steps

    # end to end: pinned host queries, k and alpha copied into the captured input buffers, graph replay, results back
    hq = [b.cpu().pin_memory() for b in batches]
    hk = [t.cpu().pin_memory() for t in kq]
    ha = [t.cpu().pin_memory() for t in aq]
    hout = [(torch.empty(o[0].shape, dtype=torch.int32).pin_memory(),
             torch.empty(o[1].shape, dtype=torch.float32).pin_memory()) for o in outs]

    def e2e_step(s, ev):
        bi = order[s % nb]
        batches[bi].copy_(hq[bi], non_blocking=True)
        kq[bi].copy_(hk[bi], non_blocking=True)
        aq[bi].copy_(ha[bi], non_blocking=True)
        graphs[bi].replay()
        hout[bi][0].copy_(outs[bi][0], non_blocking=True)
        hout[bi][1].copy_(outs[bi][1], non_blocking=True)

    with torch.cuda.stream(stream):
        e2e_ms, _ = time_loop(torch, stream, args.steps, args.warmup, e2e_step)
    h2d = d2h = 0
    for s in range(args.steps):
        bi = order[(args.warmup + s) % nb]
        h2d += hq[bi].numel() * 4 + hk[bi].numel() * 4 + ha[bi].numel() * 4
        d2h += hout[bi][0].numel() * 4 + hout[bi][1].numel() * 4
    e_ms, e_q = replicas.reduce_throughput(tdist, dev, e2e_ms, float(sum(nq_step)), world)
    e2e_value = e_q / (e_ms / 1000.0)

    # recall@k_b of a sample of queries against exact k-NN, and T_eff for the roofline
    from paper_2411_14754_gb300 import learn as L
    ns = min(args.recall_sample, batches[0].shape[0])
    q0 = batches[0][:ns]
    gt = L.exact_knn(Xd, q0, kmax, chunk=64)
    ids0 = outs[0][0][:ns].cpu().numpy()
    kk = ks[:ns]
    rec = float(np.mean([len(set(ids0[j, :kk[j]].tolist()) & set(gt[j, :kk[j]].tolist())) / kk[j]
                         for j in range(ns)]))
    dbg = pkg.suco_query_debug(index, q0, kmax, amax, w.beta, want=("t_eff",), k_per_query=kq[0][:ns].contiguous(),
                               alpha_per_query=aq[0][:ns].contiguous())
    teff = float(dbg["t_eff"].double().sum(dim=1).mean().item())
    del Xd
    Cc = pkg.suco_thresholds(w.n, amax, w.beta, kmax)[1]
    bpq = 4.0 * teff + 4.0 * Cc * w.d
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    peak_src = "measured" if peaks.get("hbm_gbs") else "fallback"
    achieved = bpq * B / (mean_launch_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": committed_traffic(f"{w.number}-mix"), "peak_source": peak_src,
                "kernel": "suco_query_kernel (mixed per-query k and alpha, multi-pass over the id range, "
                          "CUDA-graph replay, one launch per batch)",
                "algorithmic_bytes_per_query": bpq, "mean_launch_ms": mean_launch_ms}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as _o
        cpu = run_cpu_baseline(w, X, Qall, _o.max_threads(), alpha=float(np.mean(w.alpha_mix)),
                               target_s=args.cpu_seconds)
    if rank == 0:
        cfg = workload_config(w, B)
        method = {"arm": (f"beta={w.beta}, per-query k in {list(w.k_mix)} and alpha in {list(w.alpha_mix)} drawn "
                          f"uniformly, FP32")}
        cfg["launch"] = {"cluster_size": shape[0], "threads": shape[1], "cuda_graphs": True, "persistent": True}
        line = {"metric": METRIC_FIXED, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": mean_launch_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "method": method,
                "recall_at_k": rec, "recall_note": "mean over a sample of recall@k_b with each query's own k_b",
                "t_eff_per_query": teff, "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                        "d2h_bytes_per_step": d2h // args.steps},
                "clocks": clk.summary(), "gpu_launches": args.steps, "index_build_s": build_s}
        print(json.dumps(line), flush=True)
    pkg.suco_free(index)


def run_sc_linear(args, torch, tdist, pkg, W, rank, local_rank, world, dev):
    """SC-Linear (Algorithm 1): every point's distance to the query in every
    subspace, the exact alpha*n nearest per subspace, SC-scores, the beta*n
    best candidates, exact re-rank.  A step is one batch of queries."""
    w = W.WORKLOADS[args.workload]
    X = W.dataset(w.number)
    Xd = torch.from_numpy(X).to(dev)
    index = pkg.suco_build_index(Xd, w.Ns, 2, 0, seed=1)   # SC-Linear reads the dataset copy and the layout only
    del Xd
    B = 64
    Qall = W.queries(w.number, nq=max(B * 4, 256))
    nb = len(Qall) // B
    batches = [torch.from_numpy(Qall[i * B:(i + 1) * B]).to(dev) for i in range(nb)]
    order = replicas.batch_order(rank, world, nb)
    ws = torch.empty(pkg.suco_sc_linear_workspace_size(index, B, w.k, w.beta), dtype=torch.uint8, device=dev)
    outs = [(torch.empty((B, w.k), dtype=torch.int32, device=dev), torch.empty((B, w.k), dtype=torch.float32,
                                                                               device=dev)) for _ in batches]
    stream = torch.cuda.current_stream(dev)

    def step(s, ev):
        bi = order[s % nb]
        pkg.suco_sc_linear(index, batches[bi], w.k, w.alpha, w.beta, workspace=ws, out_ids=outs[bi][0],
                           out_dist=outs[bi][1], stream=stream)

    if world > 1:
        tdist.barrier()
    with ClockSampler(local_rank) as clk:
        total_ms, _ = time_loop(torch, stream, args.steps, args.warmup, step, label="timed")
    total_ms, all_q = replicas.reduce_throughput(tdist, dev, total_ms, float(B * args.steps), world)
    value = all_q / (total_ms / 1000.0)
    from paper_2411_14754_gb300 import learn as L
    Xg = torch.from_numpy(X).to(dev)
    gt = L.exact_knn(Xg, batches[0], w.k)
    del Xg
    rec = float(L.recall_rows(outs[0][0].cpu().numpy(), gt).mean())
    # the distance pass dominates: per point, query and dimension one FP32
    # subtract and one fused multiply-add; peak = 152 SMs x 128 FP32 lanes x clock
    peak = 152 * 128 * 2.07e9 / 1e12
    achieved = 2.0 * w.n * w.d * B / (total_ms / args.steps / 1000.0) / 1e12
    if rank == 0:
        line = {"metric": METRIC_SCL, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(w, B),
                "method": {"arm": f"SC-Linear (Algorithm 1, no index), alpha={w.alpha}, beta={w.beta}"},
                "recall_at_k": rec, "recall_sample": B, "k": w.k,
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 instr/s",
                             "frac": achieved / peak, "traffic": None,
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                             "kernel": "whole SC-Linear path per step (the distance pass dominates)"},
                "clocks": clk.summary(), "gpu_launches": 9 * args.steps, "cpu_baseline": None,
                "e2e": None}
        print(json.dumps(line), flush=True)
    pkg.suco_free(index)


def run_build(args, torch, tdist, pkg, W, rank, local_rank, world, dev):
    """Algorithm 2 on the GPU (K-means per half-subspace, t Lloyd iterations,
    then the IMI), a step being one whole build of the workload's index, with
    the FP64 oracle's build of the same index timed on the host cores beside
    it (one Lloyd iteration, the CPU figure per iteration)."""
    w = W.WORKLOADS[args.workload]
    X = W.dataset(w.number)
    Xd = torch.from_numpy(X).to(dev)
    init = W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK)
    stream = torch.cuda.current_stream(dev)

    def step(s, ev):
        ix = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, w.kmeans_iters, init_ids=init, stream=stream)
        pkg.suco_free(ix)

    with ClockSampler(local_rank) as clk:
        total_ms, _ = time_loop(torch, stream, args.steps, args.warmup, step, label="timed")
    build_s = total_ms / args.steps / 1000.0
    # assignment work: per Lloyd iteration (and the final assignment) every
    # point's distance to sqrtK centroids in every half: one subtract and one
    # fused multiply-add per dimension
    instr = 2.0 * (w.kmeans_iters + 1) * w.n * w.d * w.sqrtK
    peak = 152 * 128 * 2.07e9 / 1e12
    achieved = instr / build_s / 1e12
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        t0 = time.time()
        oracle.build_index(X, w.Ns, w.sqrtK, 1, init, nthreads=oracle.max_threads())
        dt = time.time() - t0
        cpu = {"value": dt, "unit": "s per Lloyd iteration (with the final assignment and the IMI)",
               "cores": oracle.max_threads(), "kind": "oracle",
               "sample": f"the same index with 1 of the {w.kmeans_iters} Lloyd iterations, FP64, OpenMP over halves"}
    if rank == 0:
        line = {"metric": "index build time (Algorithm 2)", "value": build_s, "unit": "s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(w),
                "method": {"arm": f"GPU build: K-means, {w.kmeans_iters} Lloyd iterations per half-subspace, then "
                                  "the IMI (CSR by radix sort)"},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 instr/s",
                             "frac": achieved / peak, "traffic": None,
                             "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                             "kernel": "whole build (the assignment passes dominate the arithmetic)"},
                "cpu_baseline": cpu, "clocks": clk.summary(), "gpu_launches": None, "e2e": None}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as tdist

    import paper_2411_14754_gb300 as pkg
    from paper_2411_14754_gb300 import workloads as W

    rank, local_rank, world = dist_env()
    if world > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pkg.load_library()
    w = W.WORKLOADS[args.workload]
    if args.build:
        run_build(args, torch, tdist, pkg, W, rank, local_rank, world, dev)
        if world > 1:
            tdist.destroy_process_group()
        return
    if args.sc_linear:
        run_sc_linear(args, torch, tdist, pkg, W, rank, local_rank, world, dev)
        if world > 1:
            tdist.destroy_process_group()
        return
    if w.k_mix and not args.plain:
        run_batching(args, torch, tdist, pkg, W, rank, local_rank, world, dev)
        if world > 1:
            tdist.destroy_process_group()
        return
    if w.n_train and not args.plain:
        run_learned(args, torch, tdist, pkg, W, rank, local_rank, world, dev)
        if world > 1:
            tdist.destroy_process_group()
        return
    X = W.dataset(w.number)
    Qall = W.queries(w.number)
    Xd = torch.from_numpy(X).to(dev)
    t0 = time.time()
    index = pkg.suco_build_index(Xd, w.Ns, w.sqrtK, w.kmeans_iters,
                                 init_ids=W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK))
    torch.cuda.synchronize()
    build_s = time.time() - t0
    del Xd
    if args.precision != "fp32" or args.rank_precision != "fp32":
        pkg.suco_add_reduced_copies(index)
    qkw = dict(precision=args.precision, rank_precision=args.rank_precision, exact_rerank=args.exact_rerank)
    B = w.batch
    nb = (w.nq + B - 1) // B
    # every rank answers different batches (query-sharded replicas)
    batches = [torch.from_numpy(Qall[i * B:(i + 1) * B]).to(dev) for i in range(nb)]
    order = replicas.batch_order(rank, world, nb)
    stream = torch.cuda.current_stream(dev)
    outs = [(torch.empty((b.shape[0], w.k), dtype=torch.int32, device=dev),
             torch.empty((b.shape[0], w.k), dtype=torch.float32, device=dev)) for b in batches]

    def step(s):
        bi = order[s % nb]
        pkg.suco_query_batch(index, batches[bi], w.k, w.alpha, w.beta, out_ids=outs[bi][0], out_dist=outs[bi][1],
                             cluster_size=args.cluster_size, threads=args.threads, stream=stream, **qkw)
        return batches[bi].shape[0]

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    nqueries = 0
    with ClockSampler(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
        ev[0].record(stream)
        for s in range(args.steps):
            nqueries += step(args.warmup + s)
            ev[s + 1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    # slowest rank decides; queries are summed over ranks
    total_ms, all_queries = replicas.reduce_throughput(tdist, dev, total_ms, float(nqueries), world)
    value = all_queries / (total_ms / 1000.0)

    # end to end through the public API: pinned host queries in, host results out, every step
    hq = [b.cpu().pin_memory() for b in batches]
    hout = [(torch.empty(o[0].shape, dtype=torch.int32).pin_memory(),
             torch.empty(o[1].shape, dtype=torch.float32).pin_memory()) for o in outs]
    dq = [torch.empty_like(b) for b in batches]
    h2d = d2h = 0

    def e2e_step(s):
        bi = order[s % nb]
        dq[bi].copy_(hq[bi], non_blocking=True)
        pkg.suco_query_batch(index, dq[bi], w.k, w.alpha, w.beta, out_ids=outs[bi][0], out_dist=outs[bi][1],
                             cluster_size=args.cluster_size, threads=args.threads, stream=stream, **qkw)
        hout[bi][0].copy_(outs[bi][0], non_blocking=True)
        hout[bi][1].copy_(outs[bi][1], non_blocking=True)
        return (hq[bi].numel() * 4, hout[bi][0].numel() * 4 + hout[bi][1].numel() * 4, hq[bi].shape[0])

    for s in range(args.warmup):
        e2e_step(s)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eq = 0
    e0.record(stream)
    for s in range(args.steps):
        a, b, c = e2e_step(s)
        h2d += a
        d2h += b
        eq += c
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e_ms, e_q = replicas.reduce_throughput(tdist, dev, e2e_ms, float(eq), world)
    e2e_value = e_q / (e_ms / 1000.0)

    # recall@k against exact k-NN (GPU brute force shortlist, FP64 re-check), and T_eff for the roofline
    from oracle import recall as _recall
    ns = min(args.recall_sample, batches[0].shape[0])
    q0 = batches[0][:ns]
    ids_s, dist_s = pkg.suco_query_batch(index, q0, w.k, w.alpha, w.beta, cluster_size=args.cluster_size,
                                         threads=args.threads, **qkw)
    dbg = pkg.suco_query_debug(index, q0, w.k, w.alpha, w.beta, cluster_size=args.cluster_size,
                               threads=args.threads, want=("t_eff",), **qkw)
    torch.backends.cuda.matmul.allow_tf32 = False
    Xg = torch.from_numpy(X).to(dev)
    gt = []
    for s0 in range(0, ns, 64):
        qq = q0[s0:s0 + 64]
        dd = torch.cdist(qq, Xg)
        cand = torch.topk(dd, w.k + 32, largest=False).indices.cpu().numpy()
        for j in range(qq.shape[0]):
            c = cand[j]
            exact = ((X[c].astype(np.float64) - qq[j].cpu().numpy().astype(np.float64)) ** 2).sum(1)
            gt.append(c[np.lexsort((c, exact))[:w.k]])
    del Xg
    rec = _recall(ids_s.cpu().numpy(), np.stack(gt))
    teff_total = float(dbg["t_eff"].double().sum(dim=1).mean().item())
    # per-result error of the returned squared distances against FP64, and, for
    # a reduced-precision mode, its recall change against FP32 on the same
    # queries and the error of its cell-ranking tables against the FP64
    # distances of the unrounded vectors
    err = precision_report(pkg, index, w, X, q0, ids_s, dist_s, rec, args, gt)
    T, Cc = pkg.suco_thresholds(w.n, w.alpha, w.beta, w.k)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    bpq = algorithmic_bytes_per_query(w, T, Cc, teff_total)
    if args.precision != "fp32" and Cc > args.exact_rerank:
        eb = 2.0 if args.precision == "bf16" else 1.0
        bpq = 4.0 * teff_total + (eb * Cc + 4.0 * args.exact_rerank) * w.d
    mean_launch_ms = statistics.mean(step_ms)
    achieved = bpq * B / (mean_launch_ms / 1000.0) / 1e9
    # the committed capture is of the FP32 path; another precision has none
    traffic = committed_traffic(w.number) if args.precision == "fp32" and args.rank_precision == "fp32" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_source": peak_src,
                "kernel": "suco_query_kernel (whole query path, one launch per batch)",
                "algorithmic_bytes_per_query": bpq, "mean_launch_ms": mean_launch_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as _o
        threads = _o.max_threads()
        cpu = run_cpu_baseline(w, X, Qall, threads, target_s=args.cpu_seconds)

    if rank == 0:
        cfg = workload_config(w, B)
        method = {"arm": f"fixed alpha={w.alpha}, beta={w.beta}", "rerank": args.precision,
                  "exact_rerank": args.exact_rerank, "cell_ranking": args.rank_precision}
        line = {"metric": METRIC_FIXED, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "method": method, "recall_at_k": rec, "k": w.k,
                "T": T, "C": Cc, "t_eff_per_query": teff_total, "precision_report": err,
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                        "d2h_bytes_per_step": d2h // args.steps},
                "clocks": clk.summary(), "gpu_launches": args.steps * (2 if args.rank_precision != "fp32" else 1),
                "index_build_s": build_s}
        print(json.dumps(line), flush=True)
    pkg.suco_free(index)
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
