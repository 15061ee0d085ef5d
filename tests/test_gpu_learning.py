"""Calibration loops of Sec. III on the adjoint kernels: material learning
from frequency responses (Sec. III-A) and transmitter orientation by
gradient ascent of received power (Sec. III-B), paths frozen."""
import math

import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import learning as LG
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tx, rx = S.city_devices(sc, n_rx=64, half=70.0)
    tr = rt.Tracer(0, 3.5e9)
    tr.load_scene(sc)
    tr.set_devices(tx, rx)
    tr.compute_paths(3, 200_000)
    yield tr, sc, tx, rx
    tr.close()


def test_material_recovery_from_frequency_responses(city):
    tr, sc, tx, rx = city
    freqs = (np.arange(128) - 64) * 30e3
    true = torch.as_tensor(sc.materials, dtype=torch.float32, device="cuda").reshape(-1, 2)
    tr.set_materials(true)
    a, tau = tr.cir()
    H_ref = tr.freq_response(a, tau, freqs).detach()
    M = true.shape[0]
    eps, sig, hist = LG.fit_materials(tr, H_ref, freqs, eps0=[3.0] * M, sigma0=[0.03] * M, iters=250, lr=0.05)
    assert hist[-1] < 1e-3 * hist[0]
    # the permittivities of the materials that carry paths are recovered
    seq = tr.paths()["seq"].cpu().numpy()
    used = np.unique(sc.mat_id[seq[seq >= 0]])
    for m in used:
        assert abs(eps[m].item() - true[m, 0].item()) <= 0.05 * true[m, 0].item(), (m, eps[m].item())
    tr.set_materials(true)


def test_transmitter_orientation_ascent(city):
    tr, sc, tx, rx = city
    pair = tr.path_pairs()
    # start turned 90 degrees away (inside the pattern's unsaturated range)
    yaw0, pitch0 = float(tx.ypr[0, 0]) + 0.5 * math.pi, 0.3
    yaw, pitch, hist = LG.orient_transmitter(tr, pair, yaw0, pitch0, iters=150, lr=0.05)
    n_rx = pair.unique().numel()
    assert hist[-1] > hist[0] + 3.0 * n_rx          # at least +3 dB per receiver on average
    assert max(hist[-10:]) - min(hist[-10:]) < 0.05 * n_rx   # converged
    tr.set_tx(tx.pos, tx.ypr, tx.antenna)
