"""Training and evaluation of the learned self-collision surrogate.

The network (mrs.MLP: sin/cos joint features in, signed clearance out) is
trained on the device by the library's own kernels on data the library
generates: joint vectors uniform within the limits with their exact
self-collision clearance (mrs_self_dataset).  Evaluation reports, on held-out
samples, the false-negative rate at the fallback margin (colliding samples,
exact clearance < 0, whose prediction would skip the exact check), the mean
absolute error and the fraction of samples the surrogate lets skip.
"""
from __future__ import annotations

import time

import numpy as np

from . import mrs


def evaluate(pred, exact, B_self, margin):
    """FN rate and skip fraction of predictions against exact clearances."""
    pred = np.asarray(pred, np.float64).ravel()
    exact = np.asarray(exact, np.float64).ravel()
    skip = pred >= B_self + margin
    colliding = exact < 0
    active = exact < B_self
    fn = int(np.sum(skip & colliding))
    return {
        "samples": int(pred.size),
        "colliding": int(colliding.sum()),
        "false_negatives": fn,
        "fn_rate": fn / max(1, int(colliding.sum())),
        "fn_rate_active": int(np.sum(skip & active)) / max(1, int(active.sum())),
        "skip_fraction": float(skip.mean()),
        "mae": float(np.mean(np.abs(np.clip(exact, -0.1, 0.3) - pred))),
    }


def train_self_surrogate(ctl, arm, n_train=2_000_000, n_val=200_000, epochs=8, batch=4096,
                         lr=1e-3, width=256, layers=3, seed=0, margin=0.03, log=None):
    """Train a surrogate for `arm` of controller `ctl`; returns (net, stats)."""
    t0 = time.perf_counter()
    x, t, _ = ctl.self_dataset(arm, n_train + n_val, seed)
    xt, tt = x[:n_train], t[:n_train]
    xv, tv = x[n_train:], t[n_train:]
    net = mrs.MLP(x.shape[1], width, layers, seed + 1)
    steps = n_train // batch
    losses = []
    for ep in range(epochs):
        rate = lr * (0.5 ** (ep // max(1, epochs // 3)))      # step decay
        for i in range(steps):
            losses.append(net.train_step(xt[i * batch:(i + 1) * batch],
                                         tt[i * batch:(i + 1) * batch], rate))
        if log:
            log(f"epoch {ep}: loss {np.mean(losses[-steps:]):.3e}")
    train_s = time.perf_counter() - t0
    pred = net.forward(xv).cpu().numpy()
    stats = evaluate(pred, tv.cpu().numpy(), float(np.float32(ctl.sc.params["B_self"])), margin)
    stats.update(train_seconds=train_s, final_loss=float(np.mean(losses[-steps:])),
                 n_train=n_train, epochs=epochs)
    return net, stats
