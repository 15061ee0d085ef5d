"""H(f) where the kernel is compute-bound (Sec. III-A: CIRs turned into OFDM
frequency responses): a dense seeded path list of about 64 paths per pair,
1000 pairs, 2 x 2 port pairs and 1024 subcarriers of 30 kHz, through
rt_freq_response_paths, against the oracle's direct FP64 sum element by
element. Ragged path counts (a pair spanning several path tiles, a pair
without paths) and a non-uniform subcarrier set are included."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import H_ABS, H_REL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_pp,uniform", [(4, True), (2, False), (1, True)])
def test_dense_freq_response_matches_oracle(n_pp, uniform):
    n_pairs = 1000 if n_pp == 4 else 257
    off, a, tau = S.dense_path_list(n_pairs, 64, n_pp, seed=6 + n_pp)
    if uniform:
        freqs = O.subcarrier_freqs(1024, 30e3)
    else:
        freqs = np.sort(np.random.default_rng(8).uniform(-15e6, 15e6, 777))
    K = len(freqs)
    tr = rt.Tracer(0, 3.5e9)
    dev = tr.device
    off_d = torch.as_tensor(off, device=dev)
    a_d = torch.view_as_real(torch.as_tensor(a, device=dev)).contiguous()
    tau_d = torch.as_tensor(tau, device=dev)
    f_d = torch.as_tensor(freqs, device=dev)
    H = torch.empty((n_pairs, n_pp, K, 2), dtype=torch.float32, device=dev)
    rt.rt_freq_response_paths(tr.ctx, off_d, n_pp, a_d, tau_d, f_d, H)
    Hg = torch.view_as_complex(H).cpu().numpy()
    tr.close()
    a64, tau64 = a.astype(np.complex128), tau.astype(np.float64)
    worst = 0.0
    for r in range(n_pairs):
        b, e = off[r], off[r + 1]
        if e == b:
            assert np.all(Hg[r] == 0)
            continue
        Ho = O.freq_response(a64[b:e], tau64[b:e], freqs)            # [n_pp, K]
        bound = H_REL * np.abs(Ho) + H_ABS * np.abs(a64[b:e]).sum(axis=0)[:, None]
        err = np.abs(Hg[r] - Ho)
        worst = max(worst, float((err / bound).max()))
        assert np.all(err <= bound), (r, float((err / bound).max()))
    print(f"dense H(f): worst error / tolerance = {worst:.3f}")
