"""Training and checkpointing of the learned row-size predictor.

The predictor estimates nnz(C_i) for every row of a product from three
features (nnz(A_i), flops_i, max_p nnz(B_p)), the last two relative to the
output width, so that the SpGEMM can size its
hash tables and its column-batch count without the symbolic phase (paper
Sec. 5, approximate memory estimation; Sec. 7.4, batch count of batched
SpGEMM).  Training data are squares C = A.A of the generated matrix
families (R-MAT, ER, banded); labels are exact row sizes from the library's
own symbolic kernel; features come from its flop-count kernel; training
runs in its BF16 forward/backward kernels.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import cb, gen

HERE = os.path.dirname(os.path.abspath(__file__))
CHECKPOINT = os.path.join(HERE, "sizer_checkpoint.npz")
TAU = 0.9


def init_params(seed: int = 0) -> np.ndarray:
    """He-style seeded initialisation, flat in the library's parameter layout."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2.0 / 3), (64, 3))
    W2 = rng.normal(0, math.sqrt(2.0 / 64), (64, 64))
    w3 = rng.normal(0, math.sqrt(1.0 / 64), 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]]).astype(np.float32)


def product_rows(A_host, device="cuda"):
    """(features [m,4], exact row sizes [m]) of A.A on the device, live rows only."""
    dA = cb.DeviceCSR.from_host(A_host.with_values(np.ones(A_host.nnz, np.uint8)), "or_and_bool",
                                device)
    feat = cb.row_features(dA, dA)
    nnz = cb.row_nnz(dA, dA)
    live = feat[:, 1] > 0
    return feat[live].contiguous(), nnz[live].contiguous()


def dataset(indices, device="cuda", cfg: int = 5):
    feats, labels = [], []
    for i in indices:
        f, y = product_rows(gen.training_family(int(i), cfg=cfg), device)
        feats.append(f)
        labels.append(y)
    return torch.cat(feats), torch.cat(labels)


def inputs(feat: torch.Tensor) -> torch.Tensor:
    """The network's inputs before standardisation (the library's transform)."""
    f = feat.double()
    lw = torch.log2(torch.clamp(f[:, 3], min=1.0))
    return torch.stack([torch.log2(1.0 + f[:, 0]), torch.log2(1.0 + f[:, 1]) - lw,
                        torch.log2(1.0 + f[:, 2]) - lw], 1)


def normalisation(feat: torch.Tensor) -> np.ndarray:
    L = inputs(feat)
    return np.concatenate([L.mean(0).cpu().numpy(), L.std(0).cpu().numpy() + 1e-3]).astype(np.float32)


def shuffle(feat, labels, seed=0):
    g = torch.Generator(device=feat.device).manual_seed(seed)
    perm = torch.randperm(feat.shape[0], device=feat.device, generator=g)
    return feat[perm].contiguous(), labels[perm].contiguous()


def train(feat, labels, epochs=20, batch=4096, lr=2e-3, seed=0, norm=None):
    """Train a fresh model (norm from the data unless given); returns (model, epoch losses)."""
    norm = normalisation(feat) if norm is None else norm
    model = cb.MLP(init_params(seed), norm)
    f, y = shuffle(feat, labels, seed)
    losses = model.train(f, y, epochs=epochs, batch=batch, lr=lr, tau=TAU)
    return model, losses


def save(model, path: str = CHECKPOINT, meta: dict | None = None) -> None:
    params, norm, step = model.get()
    np.savez(path, params=params, norm=norm, step=np.int64(step),
             meta=json.dumps(meta or {}))


def load(path: str = CHECKPOINT):
    z = np.load(path)
    return cb.MLP(z["params"], z["norm"]), json.loads(str(z["meta"]))


def evaluate(model, feat, labels, ncols: int, margin: float = 0.25) -> dict:
    """Prediction quality on rows: over-allocation of capacities and overflow rate."""
    _, pred = model.predict(feat, ncols)
    cap = torch.minimum(torch.ceil(pred.double() * (1 + margin)).long(),
                        torch.clamp(feat[:, 1].long(), max=ncols))
    cap = torch.maximum(cap, pred)
    y = labels
    return {
        "rows": int(y.numel()),
        "sum_pred_over_sum_true": float(pred.sum().item() / max(int(y.sum().item()), 1)),
        "sum_cap_over_sum_true": float(cap.sum().item() / max(int(y.sum().item()), 1)),
        "overflow_rows": float((cap < y).double().mean().item()),
        "median_abs_log2_err": float(torch.median(torch.abs(torch.log2(pred.double().clamp(min=1))
                                                            - torch.log2(y.double()))).item()),
        "sum_bound_over_sum_true": float(torch.clamp(feat[:, 1].long(), max=ncols).sum().item()
                                         / max(int(y.sum().item()), 1)),
    }


def _gen_one(i):
    A = gen.training_family(int(i))
    return int(i), A.nrows, A.ncols, A.row_ptr, A.col


def training_set(count: int = 2000, workers: int = 0, device="cuda", log=print):
    """Features and labels of the first `count` matrices of the training
    family, generated by a spawn-started process pool (numpy only) and
    labelled on the GPU."""
    import multiprocessing as mp
    import time
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    feats, labels = [], []
    t0 = time.time()
    with mp.get_context("spawn").Pool(workers) as pool:
        for n_done, (i, nr, nc, rp, col) in enumerate(pool.imap_unordered(_gen_one, range(count), 4)):
            f, y = product_rows(gen.CSR(nr, nc, rp, col))
            feats.append(f)
            labels.append(y)
            if log and (n_done + 1) % 250 == 0:
                log(f"  {n_done + 1}/{count} matrices, {sum(x.shape[0] for x in feats)} rows, "
                    f"{time.time() - t0:.1f}s")
    return torch.cat(feats), torch.cat(labels)


def main(argv=None):
    import argparse
    import time
    ap = argparse.ArgumentParser(description="train the learned row-size predictor")
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=CHECKPOINT)
    args = ap.parse_args(argv)
    t0 = time.time()
    feat, lab = training_set(args.count)
    t1 = time.time()
    model, losses = train(feat, lab, epochs=args.epochs, batch=args.batch, lr=args.lr)
    torch.cuda.synchronize()
    t2 = time.time()
    meta = {"matrices": args.count, "rows": int(feat.shape[0]), "epochs": args.epochs,
            "batch": args.batch, "lr": args.lr, "tau": TAU,
            "epoch_loss": [float(x) for x in losses], "data_seconds": round(t1 - t0, 1),
            "train_seconds": round(t2 - t1, 2),
            "family": "gen.training_family: R-MAT s12-16 a in [0.45,0.65], ER n 2^12-2^16 deg 4-64, "
                      "banded bw 8-256 deg 4-64; C = A.A"}
    save(model, args.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
