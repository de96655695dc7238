"""Driver of the learned per-query ratios: labels, training, margin tuning, use.

Every piece of arithmetic on the path runs in libsuco's kernels (features,
network forward and backward, AdamW, the query itself); this module only
orders the calls.  The exact k-NN ground truth used for labels and recall is
measurement, not the path: a TF32 matrix product shortlists candidates and
exact FP32 differences decide among them.

Labels: for each training query, the plain query path runs over a grid of
(alpha, beta); the label is the cheapest grid point (by the bytes the path
must move, 4*Ns*alpha*n + 4*beta*n*d) at which that query's recall@k is 1,
or the largest grid point when none reaches it.  The network regresses
(log alpha, log beta) of the label.  At use, margins added to both outputs are
tuned on a validation split so that the mean recall@k reaches the target.
"""
import math
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np
import torch

from . import suco as S

ALPHA_GRID = (0.005, 0.01, 0.02, 0.03, 0.05, 0.08, 0.12, 0.2)
BETA_GRID = (0.0005, 0.001, 0.002, 0.003, 0.005, 0.008, 0.016)
FALLBACK = (0.05, 0.005)
# clamps of the predicted ratios; the beta bound also sizes the query kernel's
# candidate slots (shared memory), so it stays at the grid's largest beta
ALPHA_RANGE = (ALPHA_GRID[0] / 4, min(1.0, 1.5 * ALPHA_GRID[-1]))
BETA_RANGE = (BETA_GRID[0] / 4, BETA_GRID[-1])


def exact_knn(Xd: torch.Tensor, Qd: torch.Tensor, k: int, shortlist: int = 1000, chunk: int = 1024):
    """Exact k nearest ids (ties by id) of every query: a TF32 matrix product
    shortlists ``shortlist`` points (its error, about 2^-11 of |q||x|, is far
    below the gap to the shortlist's edge on these workloads), then FP32
    differences re-rank them and ties fall to the lower id."""
    out = np.empty((Qd.shape[0], k), np.int64)
    xn = (Xd * Xd).sum(1)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        for s in range(0, Qd.shape[0], chunk):
            q = Qd[s:s + chunk]
            d = xn[None, :] - 2.0 * (q @ Xd.T)
            cand = torch.topk(d, min(shortlist, Xd.shape[0]), dim=1, largest=False).indices
            rows = Xd[cand]                                   # [c][shortlist][d]
            ex = ((rows - q[:, None, :]) ** 2).sum(-1)        # FP32 difference form
            ex64 = ex.double().cpu().numpy()
            cid = cand.cpu().numpy()
            for j in range(q.shape[0]):
                o = np.lexsort((cid[j], ex64[j]))[:k]
                out[s + j] = cid[j][o]
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def recall_rows(ids: np.ndarray, gt: np.ndarray) -> np.ndarray:
    """|ids_b intersect gt_b| / k per row (ids within a row are distinct)."""
    ids = np.asarray(ids)
    gt = np.asarray(gt)
    k = gt.shape[1]
    hit = (ids[:, :, None] == gt[:, None, :]) & (gt[:, None, :] >= 0)
    return hit.any(axis=2).sum(axis=1) / k


def path_bytes(alpha, beta, n, d, Ns):
    return 4.0 * Ns * alpha * n + 4.0 * beta * n * d


def grid_recalls(index: S.SucoIndex, Qd: torch.Tensor, gt: np.ndarray, k: int, alphas=ALPHA_GRID,
                 betas=BETA_GRID, batch: int = 4096):
    """recall[q, ia, ib] of the plain path at every grid point."""
    nq = Qd.shape[0]
    rec = np.zeros((nq, len(alphas), len(betas)))
    for ia, a in enumerate(alphas):
        for ib, b in enumerate(betas):
            for s in range(0, nq, batch):
                ids, _ = S.suco_query_batch(index, Qd[s:s + batch], k, a, b)
                rec[s:s + batch, ia, ib] = recall_rows(ids.cpu().numpy(), gt[s:s + batch])
    return rec


def labels_from_recalls(rec, n, d, Ns, alphas=ALPHA_GRID, betas=BETA_GRID, mode="lagrange", target=0.95):
    """Per-query (log alpha, log beta) labels from grid recalls rec[q, ia, ib].

    mode "full": the cheapest grid point at which the query's recall is 1 (the
    largest point when none is); at k = 10 that is the cheapest point where the
    query alone passes a 0.95 recall target.
    mode "lagrange": the point maximising recall - lam * bytes for one common
    lam >= 0, the largest lam whose mean recall over the queries still reaches
    the target (bisection); a query then gets more bytes only where they buy
    recall at a rate of at least lam, which is the cheapest way to reach a
    target mean recall on this grid."""
    cost = np.array([[path_bytes(a, b, n, d, Ns) for b in betas] for a in alphas]).reshape(-1)
    R = rec.reshape(rec.shape[0], -1)
    la = np.log(np.repeat(np.asarray(alphas, np.float64), len(betas)))
    lb = np.log(np.tile(np.asarray(betas, np.float64), len(alphas)))
    if mode == "full":
        order = np.argsort(cost, kind="stable")
        ok = R[:, order] >= 1.0
        first = np.where(ok.any(axis=1), ok.argmax(axis=1), len(order) - 1)
        pick = order[first]
    elif mode == "lagrange":
        cn = cost / cost.max()

        def choose(lam):
            return np.argmax(R - lam * cn[None, :], axis=1)   # ties: the first (cheaper alpha) point

        lo, hi = 0.0, 1.0
        while R[np.arange(len(R)), choose(hi)].mean() >= target and hi < 1e6:
            hi *= 2.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if R[np.arange(len(R)), choose(mid)].mean() >= target:
                lo = mid
            else:
                hi = mid
        # at lam = lo the mean recall reaches the target (lo = 0 takes the best recall of every query)
        pick = choose(lo)
    else:
        raise ValueError(mode)
    return np.stack([la[pick], lb[pick]], axis=1).astype(np.float32)


@dataclass
class Mlp:
    """Network parameters on the device: FP32 masters, BF16 copies, AdamW moments."""
    F: int
    H: int = 256
    device: str = "cuda"
    seed: int = 0
    offsets: Sequence[float] = (0.0, 0.0)
    tensors: dict = field(default_factory=dict)
    # held-out training queries that choose operating points (set by fit):
    # Q (device tensor), gt (exact k-NN ids)
    validation: dict = field(default_factory=dict)

    def __post_init__(self):
        rng = np.random.default_rng(self.seed)
        t = self.tensors
        dev = self.device
        t["W1"] = torch.tensor(rng.standard_normal((self.F, self.H)) / math.sqrt(self.F), dtype=torch.float32,
                               device=dev)
        t["b1"] = torch.zeros(self.H, dtype=torch.float32, device=dev)
        t["W2"] = torch.tensor(rng.standard_normal((self.H, 2)) / math.sqrt(self.H), dtype=torch.float32, device=dev)
        t["b2"] = torch.tensor([math.log(FALLBACK[0]), math.log(FALLBACK[1])], dtype=torch.float32, device=dev)
        t["w1b"] = t["W1"].to(torch.bfloat16)
        t["w2b"] = t["W2"].to(torch.bfloat16)
        t["mean"] = torch.zeros(self.F, dtype=torch.float32, device=dev)
        t["std"] = torch.ones(self.F, dtype=torch.float32, device=dev)
        for p in ("W1", "b1", "W2", "b2"):
            t["m_" + p] = torch.zeros_like(t[p])
            t["v_" + p] = torch.zeros_like(t[p])
            t["g_" + p] = torch.zeros_like(t[p])
        self.step = 0

    def struct(self, offsets=None, clamp_alpha=ALPHA_RANGE, clamp_beta=BETA_RANGE):
        t = self.tensors
        off = self.offsets if offsets is None else offsets
        m = S.SucoMlp()
        m.in_dim, m.hidden, m.out_dim, m.reserved0 = self.F, self.H, 2, 0
        m.w1, m.b1 = t["w1b"].data_ptr(), t["b1"].data_ptr()
        m.w2, m.b2 = t["w2b"].data_ptr(), t["b2"].data_ptr()
        m.feat_mean, m.feat_std = t["mean"].data_ptr(), t["std"].data_ptr()
        m.out_offset[0], m.out_offset[1] = float(off[0]), float(off[1])
        m.log_alpha_min, m.log_alpha_max = math.log(clamp_alpha[0]), math.log(clamp_alpha[1])
        m.log_beta_min, m.log_beta_max = math.log(clamp_beta[0]), math.log(clamp_beta[1])
        m.fallback_alpha, m.fallback_beta = FALLBACK
        return m

    def set_standardisation(self, feats: torch.Tensor):
        self.tensors["mean"].copy_(feats.mean(0))
        self.tensors["std"].copy_(feats.std(0).clamp_min(1e-6))

    def set_output_bias(self, targets: torch.Tensor):
        """Start the output bias at the mean target (AdamW moves it only about lr per step)."""
        self.tensors["b2"].copy_(targets.float().mean(0))

    def save(self, path):
        np.savez(path, **{k: self.tensors[k].float().cpu().numpy() for k in ("W1", "b1", "W2", "b2", "mean", "std")},
                 offsets=np.asarray(self.offsets, np.float32), F=self.F, H=self.H)

    @classmethod
    def load(cls, path, device="cuda"):
        z = np.load(path)
        m = cls(int(z["F"]), int(z["H"]), device=device, offsets=tuple(z["offsets"].tolist()))
        for k in ("W1", "b1", "W2", "b2", "mean", "std"):
            m.tensors[k].copy_(torch.from_numpy(z[k]))
        m.tensors["w1b"] = m.tensors["W1"].to(torch.bfloat16)
        m.tensors["w2b"] = m.tensors["W2"].to(torch.bfloat16)
        return m


def train(model: Mlp, feats: torch.Tensor, targets: torch.Tensor, epochs: int = 30, batch: int = 1024,
          lr: float = 3e-3, weight_decay: float = 1e-4, seed: int = 0):
    """Mini-batch AdamW on the MSE of (log alpha, log beta); returns the mean loss per epoch."""
    t = model.tensors
    N, F, H = feats.shape[0], model.F, model.H
    dev = feats.device
    rng = np.random.default_rng(seed)
    z1 = torch.empty((batch, H), device=dev)
    h = torch.empty((batch, H), device=dev)
    y = torch.empty((batch, 2), device=dev)
    dz1 = torch.empty((batch, H), device=dev)
    dy = torch.empty((batch, 2), device=dev)
    loss = torch.zeros(1, device=dev)
    hist = []
    st = model.struct()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(N)).to(dev)
        tot, nb = 0.0, 0
        for s in range(0, N - batch + 1, batch):
            sel = perm[s:s + batch]
            xb = feats[sel].contiguous()
            tb = targets[sel].contiguous()
            S.suco_mlp_forward(st, xb, z1, h, y)
            S.suco_mlp_backward(st, xb, z1, h, y, tb, dz1, dy, t["g_W1"], t["g_b1"], t["g_W2"], t["g_b2"], loss)
            model.step += 1
            for p, bcopy in (("W1", t["w1b"]), ("b1", None), ("W2", t["w2b"]), ("b2", None)):
                S.suco_adamw_step(t[p], t["g_" + p], t["m_" + p], t["v_" + p], lr, model.step,
                                  weight_decay=weight_decay if p in ("W1", "W2") else 0.0, bf16_copy=bcopy)
            tot += float(loss.item())
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist


def predict(index: S.SucoIndex, model: Mlp, Qd: torch.Tensor, offsets=None):
    return S.suco_mlp_predict(index, model.struct(offsets), Qd)


def query_learned(index: S.SucoIndex, model: Mlp, Qd: torch.Tensor, k: int, offsets=None, **kw):
    """Predict (alpha, beta) per query, then run the query path with them."""
    alpha, beta = predict(index, model, Qd, offsets)
    return S.suco_query_batch(index, Qd, k, FALLBACK[0], BETA_RANGE[1], alpha_per_query=alpha,
                              beta_per_query=beta, **kw)


def tune_offsets(index, model, Qd, gt, k, target=0.95, grid=np.arange(-1.0, 2.51, 0.125), **kw):
    """Smallest common margin (log space, added to both outputs) whose mean
    recall@k on (Qd, gt) reaches the target; the largest tried if none does.
    Extra keywords go to the query (e.g. precision).  Returns (margin, recall)."""
    r = 0.0
    for m in grid:
        ids, _ = query_learned(index, model, Qd, k, offsets=(m, m), **kw)
        r = float(recall_rows(ids.cpu().numpy(), gt).mean())
        if r >= target:
            return float(m), r
    return float(grid[-1]), r


def margin_grid(index, model, Qd, gt, k, target=0.95, grid=np.arange(-0.5, 2.01, 0.25), **kw):
    """Separate margins for log alpha and log beta: for every pair (ma, mb) of
    the grid, the mean recall@k on (Qd, gt) and the mean modelled path bytes
    of the predicted ratios.  Returns the pairs reaching the target as
    (bytes, ma, mb, recall), cheapest first."""
    out = []
    for ma in grid:
        for mb in grid:
            alpha, beta = predict(index, model, Qd, offsets=(ma, mb))
            ids, _ = S.suco_query_batch(index, Qd, k, FALLBACK[0], BETA_RANGE[1], alpha_per_query=alpha,
                                        beta_per_query=beta, **kw)
            r = float(recall_rows(ids.cpu().numpy(), gt).mean())
            if r >= target:
                a_np = alpha.cpu().numpy().astype(np.float64)
                b_np = np.minimum(beta.cpu().numpy().astype(np.float64), BETA_RANGE[1])
                cost = float(np.mean(path_bytes(a_np, b_np, index.n, index.d, index.Ns)))
                out.append((cost, float(ma), float(mb), r))
    out.sort()
    return out


def cheapest_fixed(rec_mean, n, d, Ns, target=0.95, alphas=ALPHA_GRID, betas=BETA_GRID):
    """The fixed (alpha, beta) grid point of least path bytes whose mean recall
    reaches the target (the largest point if none does)."""
    best = None
    for ia, a in enumerate(alphas):
        for ib, b in enumerate(betas):
            if rec_mean[ia, ib] >= target:
                c = path_bytes(a, b, n, d, Ns)
                if best is None or c < best[0]:
                    best = (c, a, b)
    if best is None:
        return alphas[-1], betas[-1]
    return best[1], best[2]


def fit(index: S.SucoIndex, Xd: torch.Tensor, Qtrain: torch.Tensor, k: int, val_frac: float = 0.1,
        target: float = 0.95, hidden: int = 256, epochs: int = 30, batch: int = 1024, lr: float = 3e-3,
        seed: int = 0, gt=None, log=None, label_mode: str = "full", label_target: float = 0.96):
    """Whole training recipe on one index: exact k-NN of the training queries,
    grid labels from the plain path, network training on the GPU, then the
    margin that brings the validation split to the target mean recall@k.
    Returns (model, report dict)."""
    say = log or (lambda *a: None)
    nq = Qtrain.shape[0]
    nval = max(1, int(round(nq * val_frac)))
    ntr = nq - nval
    if gt is None:
        gt = exact_knn(Xd, Qtrain, k)
    say(f"ground truth for {nq} training queries")
    rec = grid_recalls(index, Qtrain, gt, k)
    say("grid recalls done")
    lab = labels_from_recalls(rec[:ntr], index.n, index.d, index.Ns, mode=label_mode, target=label_target)
    feats = S.suco_query_features(index, Qtrain)
    model = Mlp(3 * index.Ns, hidden, device=str(Qtrain.device), seed=seed)
    model.set_standardisation(feats[:ntr])
    tgt = torch.from_numpy(lab).to(Qtrain.device)
    model.set_output_bias(tgt)
    hist = train(model, feats[:ntr].contiguous(), tgt, epochs=epochs, batch=min(batch, ntr), lr=lr, seed=seed)
    say(f"loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    Qv, gv = Qtrain[ntr:].contiguous(), gt[ntr:]
    margin, r = tune_offsets(index, model, Qv, gv, k, target=target)
    model.offsets = (margin, margin)
    model.validation = dict(Q=Qv.clone(), gt=gv)
    alpha, beta = predict(index, model, Qv)
    a_np, b_np = alpha.cpu().numpy().astype(np.float64), beta.cpu().numpy().astype(np.float64)
    learned_bytes = float(np.mean(path_bytes(a_np, b_np, index.n, index.d, index.Ns)))
    fa, fb = cheapest_fixed(rec[ntr:].mean(axis=0), index.n, index.d, index.Ns, target=target)
    report = dict(n_train=ntr, n_val=nval, loss_first=hist[0], loss_last=hist[-1], margin=margin,
                  val_recall=r, val_mean_alpha=float(a_np.mean()), val_mean_beta=float(b_np.mean()),
                  val_learned_path_bytes=learned_bytes, fixed_alpha=fa, fixed_beta=fb,
                  fixed_val_recall=float(rec[ntr:].mean(axis=0)[ALPHA_GRID.index(fa), BETA_GRID.index(fb)]),
                  fixed_path_bytes=path_bytes(fa, fb, index.n, index.d, index.Ns),
                  label_hist={f"{a},{b}": int(((np.abs(lab[:, 0] - math.log(a)) < 1e-6)
                                                & (np.abs(lab[:, 1] - math.log(b)) < 1e-6)).sum())
                              for a in ALPHA_GRID for b in BETA_GRID})
    return model, report


def main(argv=None):
    """Train the ratio network for one workload and save it (FP32 weights,
    feature standardisation and the tuned margin) to an .npz file."""
    import argparse
    import json
    import time

    from . import workloads as W

    p = argparse.ArgumentParser(description=main.__doc__)
    p.add_argument("--workload", type=int, default=5)
    p.add_argument("--n-train", type=int, default=0, help="training queries (0: the workload's own count)")
    p.add_argument("--epochs", type=int, default=30)
    p.add_argument("--target", type=float, default=0.95)
    p.add_argument("--out", required=True)
    a = p.parse_args(argv)
    w = W.WORKLOADS[a.workload]
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f}s] {m}", flush=True)  # noqa: E731
    dev = torch.device("cuda")
    Xd = torch.from_numpy(W.dataset(w.number)).to(dev)
    index = S.suco_build_index(Xd, w.Ns, w.sqrtK, w.kmeans_iters,
                               init_ids=W.kmeans_init_ids(w.number, w.n, w.Ns, w.sqrtK))
    log("index built")
    ntr = a.n_train or w.n_train
    Qt = torch.from_numpy(W.queries(w.number, nq=ntr, train=True)).to(dev)
    model, rep = fit(index, Xd, Qt, w.k, target=a.target, epochs=a.epochs, log=log)
    model.save(a.out)
    rep["workload"] = w.name
    rep["seconds"] = time.time() - t0
    print(json.dumps(rep))
    S.suco_free(index)


if __name__ == "__main__":
    main()
