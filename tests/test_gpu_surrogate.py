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
    # 1024 training sites, and 64 held-out sites drawn independently (never seen)
    n_train_tx, n_held_tx, R = 1024, 64, 32
    tx, rx = S.surrogate_sites(sc, n_tx=n_train_tx, n_rx_per_tx=R, seed=4, half=70.0, rx_radius=60.0)
    txh, rxh = S.surrogate_sites(sc, n_tx=n_held_tx, n_rx_per_tx=R, seed=14, half=70.0, rx_radius=60.0)
    tx, rx = np.concatenate([tx, txh]), np.concatenate([rx, rxh])
    x, t = SG.tracer_labels(tr, tx, rx, num_rays=50000, max_depth=2)
    n = x.shape[0]
    assert n == (n_train_tx + n_held_tx) * R
    has = t[:, 0] > 0.5
    assert 0.05 < has.float().mean().item() < 0.98
    n_train = n_train_tx * R
    lo = np.array([-75, -75, 0, -75, -75, 0], np.float32)
    hi = np.array([75, 75, 70, 75, 75, 3], np.float32)
    sur = rt.Surrogate(lo, hi, n_freq=32, width=256, n_hidden=8, sigma=1.0, seed=1)
    SG.set_fourier(sur, 0.25, 2.0, seed=1)   # smooth in the transmitter position
    losses = SG.train(sur, x[:n_train], t[:n_train], epochs=40, batch=2048, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    assert sur.status() == 0
    ev = SG.evaluate(sur, x[n_train:], t[n_train:])
    # the method without the network: free-space (Friis) gain for every pair
    # with a path, and the majority class for "has a path"
    d = torch.linalg.norm(x[n_train:, :3] - x[n_train:, 3:], dim=1)
    friis = 20 * torch.log10((3e8 / 3.5e9) / (4 * np.pi * d))
    hv = t[n_train:, 0] > 0.5
    rms_friis = torch.sqrt(((friis[hv] - t[n_train:, 1][hv]) ** 2).mean()).item()
    p_has = hv.float().mean().item()
    print(f"unseen sites: class accuracy {ev['class_accuracy']:.3f} (majority {max(p_has, 1 - p_has):.3f}), "
          f"rms {ev['rms_db_answered']:.2f} dB answered, {ev['rms_db_all_path_pairs']:.2f} dB all, Friis {rms_friis:.2f} dB")
    assert ev["class_accuracy"] > max(p_has, 1 - p_has) + 0.05
    assert ev["rms_db_answered"] < 0.8 * rms_friis
    # throughput: surrogate queries/s vs the tracer's (tx, rx) queries/s on this GPU
    q_sur, _ = SG.time_inference(sur, 1 << 20, lo, hi)
    q_tr, _ = SG.time_tracer_queries(tr, tx, rx, num_rays=50000, max_depth=2)
    assert q_sur > 100 * q_tr
    sur.close()
    tr.close()
