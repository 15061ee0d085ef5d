"""Gradient-based calibration on top of the adjoint kernels (Sec. III).

Both loops keep the paths frozen: the triangle sequences found by
rt_compute_paths do not depend on the materials or on the transmitter's
orientation, so replaying them is exact for those parameters (Sec. III-A
learns materials, Sec. III-B orients a transmitter). Every forward and
backward evaluation runs in librt_gb300.so (rt_cir, rt_freq_response and
their VJPs); torch only holds the handful of parameters, the loss and the
optimiser state.
"""
from __future__ import annotations

import math

import torch

from . import rt


def _mats_from(u, v):
    """Unconstrained (u, v) -> (eps_r > 1, sigma > 0)."""
    return 1.0 + torch.exp(u), torch.exp(v)


def nmse(H, H_ref):
    """Normalised mean squared error of frequency responses (Sec. III-A)."""
    return (H - H_ref).abs().pow(2).sum() / H_ref.abs().pow(2).sum()


def fit_materials(tracer: rt.Tracer, H_ref, freqs, eps0, sigma0, iters: int = 200, lr: float = 0.05,
                  fixed_tx=None):
    """Learn eps_r [M] and sigma [M] so that H(f) of the stored paths matches H_ref.

    tracer: paths already computed for the scene and devices; H_ref: complex
    [pairs, rx ports, tx ports, K] (e.g. measurements, or a synthetic
    response from the true materials); freqs [K] subcarrier offsets (Hz).
    Parameters are optimised in (log(eps_r - 1), log sigma) with Adam.
    Returns (eps_r, sigma, loss history).
    """
    dev = tracer.device
    freqs = torch.as_tensor(freqs, dtype=torch.float64, device=dev)
    u = torch.log(torch.as_tensor(eps0, dtype=torch.float32, device=dev) - 1.0).clone().requires_grad_(True)
    v = torch.log(torch.as_tensor(sigma0, dtype=torch.float32, device=dev)).clone().requires_grad_(True)
    tx_pos, tx_ypr = fixed_tx if fixed_tx is not None else (tracer._tx_pos, tracer._tx_ypr)
    opt = torch.optim.Adam([u, v], lr=lr)
    hist = []
    for _ in range(iters):
        opt.zero_grad()
        eps, sig = _mats_from(u, v)
        a, tau = rt.CIR.apply(tracer, eps, sig, tx_pos, tx_ypr)
        H = rt.FreqResponse.apply(tracer, a, tau, freqs)
        loss = nmse(H, H_ref)
        loss.backward()
        opt.step()
        hist.append(float(loss.item()))
    eps, sig = _mats_from(u.detach(), v.detach())
    return eps, sig, hist


def orient_transmitter(tracer: rt.Tracer, pair_of_path, yaw0: float, pitch0: float, iters: int = 100,
                       lr: float = 0.05):
    """Gradient ascent of the received power (sum over receivers of the
    incoherent power in dB, Sec. III-B) over the transmitter's yaw and pitch.

    pair_of_path: int64 [P] receiver index of each stored path (from
    tracer.paths()). Returns (yaw, pitch, objective history in dB).
    """
    dev = tracer.device
    M = tracer.n_mat
    mats = tracer._mats.to(dev)
    eps, sig = mats[:, 0].clone(), mats[:, 1].clone()
    pos = tracer._tx_pos.clone()
    ang = torch.tensor([[yaw0, pitch0]], dtype=torch.float32, device=dev, requires_grad=True)
    opt = torch.optim.Adam([ang], lr=lr)
    n_rx = int(pair_of_path.max().item()) + 1 if pair_of_path.numel() else 0
    hist = []
    for _ in range(iters):
        opt.zero_grad()
        ypr = torch.cat([ang, torch.zeros((1, 1), device=dev)], 1)
        a, tau = rt.CIR.apply(tracer, eps, sig, pos, ypr)
        p = a.abs().pow(2).reshape(a.shape[0], -1).sum(1)
        per_rx = torch.zeros(n_rx, device=dev).index_add_(0, pair_of_path, p)
        got = per_rx > 0
        obj = (10.0 * torch.log10(per_rx[got])).sum()
        (-obj).backward()
        opt.step()
        hist.append(float(obj.item()))
    return float(ang[0, 0].item()), float(ang[0, 1].item()), hist


def orient_for_region(tracer: rt.Tracer, grid: dict, max_depth: int, num_rays: int, region, yaw0: float,
                      pitch0: float, iters: int = 60, lr: float = 0.05, tx_port: int = 0):
    """Sec. III-B: gradient ascent of the mean received power (in dB) over the
    cells of `region` ([ny, nx] weights) of the coverage map, over the first
    transmitter's yaw and pitch, through rt_coverage_map_backward. Returns
    (yaw, pitch, objective history in dB)."""
    dev = tracer.device
    reg = torch.as_tensor(region, dtype=torch.float32, device=dev)
    reg = reg / reg.sum()
    ang = torch.tensor([yaw0, pitch0], dtype=torch.float32, device=dev, requires_grad=True)
    base = tracer._tx_ypr.clone()
    opt = torch.optim.Adam([ang], lr=lr)
    hist = []
    for _ in range(iters):
        opt.zero_grad()
        ypr = torch.cat([ang[None], base[:1, 2:3]], 1)
        if base.shape[0] > 1:
            ypr = torch.cat([ypr, base[1:]], 0)
        gain = rt.CoverageMap.apply(tracer, ypr, grid, max_depth, num_rays, tx_port)
        obj = 10.0 * torch.log10((gain[0] * reg).sum())
        (-obj).backward()
        opt.step()
        hist.append(float(obj.item()))
    return float(ang[0].item()), float(ang[1].item()), hist
