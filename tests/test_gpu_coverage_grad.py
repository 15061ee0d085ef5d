"""VJP of the coverage map with respect to the transmitter orientation
(Sec. III-B) against central finite differences of the FP64 oracle's
coverage map on the same rays, and the orientation ascent built on it."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import learning as LG
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, setup

pytestmark = pytest.mark.gpu

GRID = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)


@pytest.fixture(scope="module")
def small_city():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tx, _ = S.city_devices(sc, n_rx=1, half=70.0, tx_antenna=S.TR38901_VH)
    rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    tr = rt.Tracer(0, FC)
    setup(tr, sc, tx, rx)
    yield tr, sc, tx, rx
    tr.close()


def _weights():
    x = GRID["x0"] + GRID["cell"] * (np.arange(GRID["nx"]) + 0.5)
    y = GRID["y0"] + GRID["cell"] * (np.arange(GRID["ny"]) + 0.5)
    X, Y = np.meshgrid(x, y)
    return (1.0 + 0.5 * np.sin(X / 17.0) * np.cos(Y / 23.0)).astype(np.float64)


@pytest.mark.parametrize("port", [0, 1])
def test_coverage_vjp_matches_oracle_fd(small_city, port):
    tr, sc, tx, rx = small_city
    N, D = 20011, 2
    w = _weights()
    g = tr.coverage_map_backward(GRID, D, N, torch.as_tensor(w[None].astype(np.float32)), port)[0].cpu().numpy()
    osc = O.make_scene(sc)
    h = 1e-4
    fd = np.zeros(3)
    for k in range(3):
        L = []
        for sgn in (1.0, -1.0):
            ypr = tx.ypr[0].astype(np.float64).copy()
            ypr[k] += sgn * h
            a, _, _ = O.coverage(osc, FC, tx.pos[0], ypr, tx.antenna, port, rx.antenna, N, D, GRID, 0, N)
            L.append((w * a).sum())
        fd[k] = (L[0] - L[1]) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.all(np.abs(g - fd) <= 2e-3 * np.abs(fd) + 2e-4 * scale), (g, fd)


def test_coverage_autograd_and_region_ascent(small_city):
    tr, sc, tx, rx = small_city
    N, D = 100003, 2
    w = torch.as_tensor(_weights()[None].astype(np.float32), device="cuda")
    ypr = torch.as_tensor(tx.ypr, device="cuda").clone().requires_grad_(True)
    gain = rt.CoverageMap.apply(tr, ypr, GRID, D, N, 0)
    (gain * w).sum().backward()
    direct = tr.coverage_map_backward(GRID, D, N, w, 0)
    assert torch.allclose(ypr.grad, direct, rtol=1e-6, atol=0)
    # Sec. III-B: maximise the mean power in a region, starting turned 70 degrees away from it
    xs = GRID["x0"] + GRID["cell"] * (np.arange(GRID["nx"]) + 0.5)
    ys = GRID["y0"] + GRID["cell"] * (np.arange(GRID["ny"]) + 0.5)
    X, Y = np.meshgrid(xs, ys)
    tx0, ty0 = float(tx.pos[0, 0]), float(tx.pos[0, 1])
    region, yaw0 = None, None
    for k in range(12):                        # the first direction whose disc the rays reach
        phi = 2 * math.pi * k / 12
        cx, cy = tx0 + 35.0 * math.cos(phi), ty0 + 35.0 * math.sin(phi)
        reg = ((X - cx) ** 2 + (Y - cy) ** 2 < 12.0 ** 2).astype(np.float32)
        if reg.sum() < 20:
            continue
        y0 = phi + 1.2
        tr.set_tx(tx.pos, np.array([[y0, 0.1, 0.0]], np.float32), tx.antenna)
        g0, _ = tr.coverage_map(GRID, D, N, 0)
        if float((g0[0].cpu() * torch.as_tensor(reg)).sum()) > 0:
            region, yaw0 = reg, y0
            break
    assert region is not None
    yaw, pitch, hist = LG.orient_for_region(tr, GRID, D, N, region, yaw0, 0.1, iters=60, lr=0.05)
    assert np.isfinite(hist).all()
    assert hist[-1] > hist[0] + 3.0            # mean power in the region up by more than 3 dB
    tr.set_tx(tx.pos, tx.ypr, tx.antenna)
