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


def calibrate_margin(pred, exact, B, target_fn):
    """Smallest fallback margin m (>= 0) at which the false-negative rate of
    predictions on these samples is at most target_fn: a colliding sample is
    skipped only when its prediction is at least B + m, so B + m must exceed
    all but a target_fn fraction of the colliding samples' predictions."""
    pred = np.asarray(pred, np.float64).ravel()
    exact = np.asarray(exact, np.float64).ravel()
    pc = np.sort(pred[exact < 0])
    if len(pc) == 0:
        return 0.0
    allowed = int(np.floor(target_fn * len(pc)))      # colliding samples that may be skipped
    edge = pc[len(pc) - allowed - 1]                  # largest prediction that must not skip
    return float(max(0.0, np.nextafter(np.float32(edge), np.float32(np.inf)) - B))


def train_self_surrogate(ctl, arm, n_train=2_000_000, n_val=200_000, epochs=8, batch=4096,
                         lr=1e-3, width=256, layers=3, seed=0, margin=0.03, over_weight=1.0,
                         target_fn=None, log=None):
    """Train a surrogate for `arm` of controller `ctl`; returns (net, stats)
    with the held-out false-negative rate at `margin`, or, with target_fn,
    at the margin calibrated on the first half of the held-out samples to
    that rate and evaluated on the second half (stats["margin"])."""
    t0 = time.perf_counter()
    x, t, _ = ctl.self_dataset(arm, n_train + n_val, seed)
    xt, tt = x[:n_train], t[:n_train]
    xv, tv = x[n_train:], t[n_train:]
    net = mrs.MLP(x.shape[1], width, layers, seed + 1)
    net.set_loss(over_weight)
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
    tvn = tv.cpu().numpy()
    B = float(np.float32(ctl.sc.params["B_self"]))
    if target_fn is not None:
        h = len(pred) // 2
        margin = calibrate_margin(pred[:h], tvn[:h], B, target_fn)
        stats = evaluate(pred[h:], tvn[h:], B, margin)
    else:
        stats = evaluate(pred, tvn, B, margin)
    stats.update(margin=margin, train_seconds=train_s, final_loss=float(np.mean(losses[-steps:])),
                 n_train=n_train, epochs=epochs)
    return net, stats


def train_pair_surrogate(ctl, a, b=None, n_train=5_000_000, n_val=200_000, epochs=4, batch=4096,
                         lr=1e-3, width=256, layers=4, seed=0, margin=0.03, jit_t=0.02,
                         jit_yaw=0.05, over_weight=1.0, target_fn=None, log=None):
    """Train the arm-pair surrogate of arm a against arm b's geometry (b None:
    the first other arm) over the relative poses of every other arm in a's
    frame (jittered); returns (net, stats) with the held-out false-negative
    rate at the coordination buffer B.  With target_fn, the fallback margin is
    calibrated on the first half of the held-out samples to that rate and
    evaluated on the second half (stats["margin"]); otherwise `margin`."""
    A = len(ctl.sc.arms)
    others = [i for i in range(A) if i != a]
    b = others[0] if b is None else b
    poses = np.stack([ctl.relative_pose(a, i) for i in others])
    t0 = time.perf_counter()
    x, t, _, _, _ = ctl.pair_dataset(a, b, n_train + n_val, seed, poses, jit_t, jit_yaw)
    xt, tt = x[:n_train], t[:n_train]
    xv, tv = x[n_train:], t[n_train:]
    net = mrs.MLP(x.shape[1], width, layers, seed + 1)
    net.set_loss(over_weight)
    steps = n_train // batch
    losses = []
    for ep in range(epochs):
        rate = lr * (0.5 ** (ep // max(1, epochs // 3)))
        for i in range(steps):
            losses.append(net.train_step(xt[i * batch:(i + 1) * batch],
                                         tt[i * batch:(i + 1) * batch], rate))
        if log:
            log(f"epoch {ep}: loss {np.mean(losses[-steps:]):.3e}")
    train_s = time.perf_counter() - t0
    pred = net.forward(xv).cpu().numpy()
    tvn = tv.cpu().numpy()
    B = float(np.float32(ctl.sc.params["B"]))
    if target_fn is not None:
        h = len(pred) // 2
        margin = calibrate_margin(pred[:h], tvn[:h], B, target_fn)
        stats = evaluate(pred[h:], tvn[h:], B, margin)
    else:
        stats = evaluate(pred, tvn, B, margin)
    stats.update(margin=margin, train_seconds=train_s,
                 final_loss=float(np.mean(losses[-steps:])), n_train=n_train, epochs=epochs,
                 poses=len(poses), over_weight=over_weight)
    return net, stats
