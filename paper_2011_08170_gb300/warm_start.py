"""Training and use of the learned warm start.

The network (16 -> 128 -> 128 -> 1, include/f2m.h) learns lambda_v / s_v from
the sorted distances of node v to its 16 nearest neighbours.  Its training
data come from GDP itself: seeded synthetic instances are solved to certified
optimality with the batched solver, and each node contributes one sample
(features of v, final lambda_v / s_v).  Every step runs in the library: the
candidate graphs (f2m_knn_csr), the solves (f2m_create_batch / f2m_solve_batch),
the features (f2m_features) and the training (f2m_mlp_train, forward and
backward on the tensor cores, Adam).  PyTorch only holds the device arrays.

    python -m paper_2011_08170_gb300.warm_start --instances 2000 --n 20000 \\
        --epochs 8 --out paper_2011_08170_gb300/warm_start_mlp.npy

writes the trained fp32 parameter vector (18,817 floats).
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

import instances as I

from . import (f2m_batch_get_lambda, f2m_create_batch, f2m_destroy_batch, f2m_features, f2m_knn_csr,
               f2m_mlp_create, f2m_mlp_get_params, f2m_mlp_train, f2m_solve_batch)

DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warm_start_mlp.npy")


def instance_points(i: int, n: int, seed0: int) -> np.ndarray:
    """Training instance i: seed seed0 + i, uniform if i is even, clustered (the
    70 % mixture) if odd."""
    seed = seed0 + i
    return I.uniform_points(n, seed) if i % 2 == 0 else I.mixture_points(n, seed)


def training_set(count: int, n: int, seed0: int = 10000, k: int = 10, per_batch: int = 64,
                 device: str = "cuda", log=None):
    """(feat [count*n, 16], target [count*n]) float32 CUDA tensors: features of
    every node of `count` solved instances and lambda_v / s_v at the certified
    optimum."""
    import torch

    feats, targets = [], []
    for b0 in range(0, count, per_batch):
        t0 = time.perf_counter()
        ids = range(b0, min(count, b0 + per_batch))
        pts = [instance_points(i, n, seed0) for i in ids]
        inst = []
        for xy in pts:
            rp, col = f2m_knn_csr(xy, k)
            inst.append((xy, rp, col))
        b = f2m_create_batch(inst)
        infos, tot = f2m_solve_batch(b)
        for j, xy in enumerate(pts):
            lam, fb = f2m_batch_get_lambda(b, j)
            feat, scale = f2m_features(xy, device=device)
            lam_t = torch.from_numpy(lam.astype(np.float64) / float(1 << fb)).to(device)
            feats.append(feat)
            targets.append((lam_t / scale.double()).float())
        f2m_destroy_batch(b)
        if log:
            log(f"instances {b0}..{b0 + len(pts) - 1}: solved in {time.perf_counter() - t0:.2f} s, "
                f"sweeps {int(tot.iterations)}")
    return torch.cat(feats), torch.cat(targets)


def train(feat, target, params0=None, epochs: int = 8, batch: int = 38912, lr: float = 2e-3,
          lr_final_frac: float = 0.05, seed: int = 0, init_seed: int = 0):
    """Trains a network from params0 (default: the seeded initialisation);
    returns (network handle, mean loss per epoch)."""
    p0 = I.mlp_init(init_seed) if params0 is None else np.asarray(params0, np.float32)
    m = f2m_mlp_create(p0)
    losses = f2m_mlp_train(m, feat, target, epochs=epochs, batch=batch, lr=lr,
                           lr_final_frac=lr_final_frac, seed=seed)
    return m, losses


def load_weights(path: str = DEFAULT_WEIGHTS) -> np.ndarray:
    w = np.load(path)
    if w.dtype != np.float32 or w.shape != (I.MLP_NPARAMS,):
        raise ValueError(f"{path}: expected float32 [{I.MLP_NPARAMS}]")
    return w


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--instances", type=int, default=2000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--seed0", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=38912)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    a = ap.parse_args()
    from .build import build
    build()
    t0 = time.perf_counter()
    feat, target = training_set(a.instances, a.n, a.seed0, log=print)
    t1 = time.perf_counter()
    m, losses = train(feat, target, epochs=a.epochs, batch=a.batch, lr=a.lr)
    t2 = time.perf_counter()
    w = f2m_mlp_get_params(m)
    np.save(a.out, w)
    print(f"samples {feat.shape[0]}, data {t1 - t0:.1f} s, training {t2 - t1:.1f} s, "
          f"epoch losses {[round(float(x), 6) for x in losses]}, target variance "
          f"{float(target.var()):.6f}; wrote {a.out}")


if __name__ == "__main__":
    main()
