"""Path-gain surrogate workflow: tracer-generated labels, training on the
GPU with the library's tcgen05 kernels, evaluation against the tracer with
the tracer as fallback for uncertain queries.

Labels: for each (tx, rx) pair, whether the tracer finds a path and the
incoherent path gain 10 log10(sum |a|^2) (isotropic V-polarized antennas),
from rt_compute_paths + rt_cir + rt_pair_gain. Orchestration only: every
numeric step runs in librt_gb300.so.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import rt
from . import scenes as S


def tracer_labels(tracer: rt.Tracer, tx_pos, rx_pos, num_rays: int, max_depth: int, tx_batch: int = 32):
    """x [T*R, 6] (tx xyz, rx xyz) and target [T*R, 2] (has path, gain dB) on the GPU.

    tx_pos [T, 3], rx_pos [T, R, 3]: each transmitter with its own receivers
    (uneven receiver sets of one launch).
    """
    T, R = rx_pos.shape[0], rx_pos.shape[1]
    xs, ts = [], []
    for t0 in range(0, T, tx_batch):
        t1 = min(T, t0 + tx_batch)
        txd = S.Devices(tx_pos[t0:t1], np.zeros((t1 - t0, 3), np.float32), S.V_ISO)
        rxs = rx_pos[t0:t1].reshape(-1, 3)
        off = [i * R for i in range(t1 - t0 + 1)]
        tracer.set_tx(txd.pos, txd.ypr, txd.antenna)
        tracer.set_rx(rxs, np.zeros_like(rxs), S.V_ISO, off)
        tracer.compute_paths(max_depth, num_rays)
        a, _ = tracer.cir_raw()
        ts.append(tracer.pair_gain(a))
        x = np.concatenate([np.repeat(tx_pos[t0:t1], R, axis=0), rxs], 1).astype(np.float32)
        xs.append(torch.as_tensor(x, device=tracer.device))
    return torch.cat(xs), torch.cat(ts)


def set_fourier(sur: rt.Surrogate, sigma_tx: float, sigma_rx: float, rel_frac: float = 0.0,
                sigma_rel: float = 0.0, seed: int = 0):
    """Seeded Fourier matrix B [F x 6] on the normalised (tx, rx) with its own
    scale per coordinate group: the first rel_frac of the rows see only the
    horizontal Tx -> Rx offset (rows (-bx, -by, 0, bx, by, 0), b ~ N(0,
    sigma_rel^2)); the others see the transmitter's coordinates with scale
    sigma_tx and the receiver's with sigma_rx. A small sigma_tx makes the
    network's answer vary slowly with the transmitter position, so that it
    interpolates between the training sites instead of keeping one map per
    site."""
    rng = np.random.default_rng(seed)
    F = sur.F
    n_rel = int(round(rel_frac * F))
    B = np.concatenate([rng.normal(0.0, sigma_tx, (F, 3)), rng.normal(0.0, sigma_rx, (F, 3))], 1)
    if n_rel:
        b = rng.normal(0.0, sigma_rel, (n_rel, 2))
        B[:n_rel] = 0.0
        B[:n_rel, 0:2] = -b
        B[:n_rel, 3:5] = b
    p = sur.params().clone()
    p[-6 * F:] = torch.as_tensor(B.astype(np.float32).ravel(), device=p.device)
    sur.set_params(p)


def head_logit_bias_index(sur: rt.Surrogate) -> int:
    """Index of the path-logit bias in the parameter vector."""
    F, W, L = sur.F, sur.W, sur.L
    return sum((2 * F if l == 0 else W) * W + W for l in range(L)) + 2 * W


def train(sur: rt.Surrogate, x, t, epochs: int, batch: int = 8192, lr: float = 1e-3, lr_end: float = 5e-5,
          seed: int = 0, oversample: int = 1):
    """Adam with a cosine learning-rate schedule; returns per-epoch mean losses.

    oversample > 1 repeats the pairs that have a path that many times (the
    gain term of the loss then sees that many more samples per epoch) and
    afterwards subtracts log(oversample) from the path-logit bias, which
    undoes the shift of the class prior that the repetition causes."""
    if oversample > 1:
        hp = t[:, 0] > 0.5
        x = torch.cat([x] + [x[hp]] * (oversample - 1))
        t = torch.cat([t] + [t[hp]] * (oversample - 1))
    losses = _train(sur, x, t, epochs, batch, lr, lr_end, seed)
    if oversample > 1:
        p = sur.params().clone()
        p[head_logit_bias_index(sur)] -= float(np.log(oversample))
        sur.set_params(p)
    return losses


def _train(sur, x, t, epochs, batch, lr, lr_end, seed):
    n = (x.shape[0] // batch) * batch
    g = torch.Generator(device=x.device).manual_seed(seed)
    steps = epochs * (n // batch)
    losses, k = [], 0
    for _ in range(epochs):
        perm = torch.randperm(x.shape[0], generator=g, device=x.device)[:n]
        xe, te = x[perm].contiguous(), t[perm].contiguous()
        acc = torch.zeros(1, device=x.device)
        for b in range(n // batch):
            f = k / max(steps - 1, 1)
            cur = lr_end + 0.5 * (lr - lr_end) * (1 + np.cos(np.pi * f))
            sur.train_step(xe[b * batch:(b + 1) * batch], te[b * batch:(b + 1) * batch], cur, acc)
            k += 1
        losses.append(float(acc.item()) / (n // batch))
    return losses


def evaluate(sur: rt.Surrogate, x, t, margin: float = 2.0):
    """Surrogate vs tracer on held-out pairs, with tracer fallback.

    The surrogate answers when its path logit is confidently positive (gain)
    or negative (no path): |logit| >= margin; other queries go to the tracer.
    """
    out = sur.infer(x)
    logit, pred = out[:, 0], out[:, 1]
    has = t[:, 0] > 0.5
    sure = logit.abs() >= margin
    ans_gain = sure & (logit > 0)
    ans_none = sure & (logit < 0)
    both = ans_gain & has
    err = (pred[both] - t[both, 1])
    rms = float(torch.sqrt((err ** 2).mean()).item()) if both.any() else float("nan")
    q = (torch.quantile(err.abs(), torch.tensor([0.5, 0.9, 0.99], device=err.device)).tolist()
         if both.any() else [float("nan")] * 3)
    rms_all = float(torch.sqrt(((pred[has] - t[has, 1]) ** 2).mean()).item()) if has.any() else float("nan")
    return {
        "pairs": int(x.shape[0]),
        "pairs_with_path": int(has.sum().item()),
        "rms_db_answered": rms,
        "abs_err_db_p50_p90_p99": q,
        "rms_db_all_path_pairs": rms_all,
        "fallback_fraction": float((~sure).float().mean().item()),
        "false_path": int((ans_gain & ~has).sum().item()),
        "missed_path": int((ans_none & has).sum().item()),
        "class_accuracy": float(((logit > 0) == has).float().mean().item()),
        "margin": margin,
    }


def time_inference(sur: rt.Surrogate, n: int, lo, hi, reps: int = 3, seed: int = 7):
    """Queries per second of rt_mlp_infer on n random queries in the box."""
    g = torch.Generator(device=sur.device).manual_seed(seed)
    lo_t = torch.as_tensor(np.asarray(lo, np.float32), device=sur.device)
    hi_t = torch.as_tensor(np.asarray(hi, np.float32), device=sur.device)
    x = lo_t + (hi_t - lo_t) * torch.rand((n, 6), generator=g, device=sur.device)
    sur.infer(x[:1 << 16])
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sur.infer(x)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return n / (best / 1e3), best


def time_tracer_queries(tracer: rt.Tracer, tx_pos, rx_pos, num_rays: int, max_depth: int, n_rx=None):
    """Tracer (tx, rx) queries per second: compute_paths + cir + pair gain for
    the first transmitter and its first n_rx receivers (all when None) in one
    call, so the ray trace is shared by those receivers."""
    txd = S.Devices(tx_pos[:1], np.zeros((1, 3), np.float32), S.V_ISO)
    rxs = rx_pos[0] if n_rx is None else rx_pos[0][:n_rx]
    tracer.set_tx(txd.pos, txd.ypr, txd.antenna)
    tracer.set_rx(rxs, np.zeros_like(rxs), S.V_ISO)
    for _ in range(2):
        tracer.compute_paths(max_depth, num_rays)
        a, _ = tracer.cir_raw()
        tracer.pair_gain(a)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        tracer.compute_paths(max_depth, num_rays)
        a, _ = tracer.cir_raw()
        tracer.pair_gain(a)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    return len(rxs) / dt, dt
