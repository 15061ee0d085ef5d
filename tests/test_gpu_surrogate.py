"""Path-gain surrogate end to end on a small seeded city: tracer labels,
training with the tcgen05 kernels, evaluation at transmitter sites the
network never saw, and what the network gains over the tracer alone (query
throughput at a stated accuracy)."""
import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S
from paper_2303_11103_gb300 import surrogate as SG

pytestmark = pytest.mark.gpu


def test_surrogate_learns_and_outpaces_tracer():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    tr = rt.Tracer(0, 3.5e9)
    tr.load_scene(sc)
    # 80 training sites, and 16 held-out sites drawn independently (never seen)
    tx, rx = S.surrogate_sites(sc, n_tx=80, n_rx_per_tx=256, seed=4, half=70.0, rx_radius=60.0)
    txh, rxh = S.surrogate_sites(sc, n_tx=16, n_rx_per_tx=256, seed=14, half=70.0, rx_radius=60.0)
    tx, rx = np.concatenate([tx, txh]), np.concatenate([rx, rxh])
    x, t = SG.tracer_labels(tr, tx, rx, num_rays=50000, max_depth=2)
    n = x.shape[0]
    assert n == 96 * 256
    has = t[:, 0] > 0.5
    assert 0.05 < has.float().mean().item() < 0.98
    n_train = (80 * 256)
    lo = np.array([-75, -75, 0, -75, -75, 0], np.float32)
    hi = np.array([75, 75, 70, 75, 75, 3], np.float32)
    sur = rt.Surrogate(lo, hi, n_freq=32, width=256, n_hidden=8, sigma=3.0, seed=1)
    losses = SG.train(sur, x[:n_train], t[:n_train], epochs=40, batch=2048, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    assert sur.status() == 0
    ev = SG.evaluate(sur, x[n_train:], t[n_train:])
    # baseline without the network: free-space (Friis) gain for every pair with a path
    d = torch.linalg.norm(x[n_train:, :3] - x[n_train:, 3:], dim=1)
    friis = 20 * torch.log10((3e8 / 3.5e9) / (4 * np.pi * d))
    hv = t[n_train:, 0] > 0.5
    rms_friis = torch.sqrt(((friis[hv] - t[n_train:, 1][hv]) ** 2).mean()).item()
    assert ev["class_accuracy"] > 0.8
    assert ev["rms_db_answered"] < rms_friis
    # throughput: surrogate queries/s vs the tracer's (tx, rx) queries/s on this GPU
    q_sur, _ = SG.time_inference(sur, 1 << 20, lo, hi)
    q_tr, _ = SG.time_tracer_queries(tr, tx, rx, num_rays=50000, max_depth=2)
    assert q_sur > 100 * q_tr
    sur.close()
    tr.close()
