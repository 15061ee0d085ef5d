"""Gradients of the replayed-path VJP kernels vs the oracle's dual-number
gradient and FP64 central finite differences (paper Sec. I/II:
differentiability w.r.t. materials and transmitter pose; Sec. III-A:
material learning from frequency responses).

Workload: seeded city with 8 materials (eps_r ~ U(2, 8), sigma ~
logU(1e-3, 1)), 1 transmitter, 16 receivers, max_depth 3. Both sides use the
same path list (the GPU's, checked to be the oracle's), so the comparison
isolates the field and its derivatives.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, GRAD_REL, compare_path_sets, gpu_paths, setup

pytestmark = pytest.mark.gpu


def _case():
    sc = S.city_scene(n_side=6, size=150.0, seed=5, n_materials=8)
    tx, rx = S.city_devices(sc, n_rx=16, half=70.0, tx_antenna=S.TR38901_VH)
    tx = S.Devices(tx.pos, np.array([[0.7, 0.12, 0.05]], np.float32), tx.antenna)
    return sc, tx, rx


@pytest.fixture(scope="module")
def prepared():
    sc, tx, rx = _case()
    tr = rt.Tracer(0, FC)
    setup(tr, sc, tx, rx)
    tr.compute_paths(3, 20000)
    gsets, p = gpu_paths(tr)
    osc = O.make_scene(sc)
    ora_paths, ora_c = O.compute_paths(osc, tx.pos[0], rx.pos, 3, 20000)
    compare_path_sets(osc, tx.pos[0], rx.pos, gsets, ora_paths, ora_c)
    # the oracle evaluates exactly the GPU's path list
    paths = [O.OPath(r, s, True, 1.0, None, 0.0) for r in range(len(rx.pos)) for s in gsets[r]]
    yield tr, sc, tx, rx, osc, paths
    tr.close()


def _theta(osc, tx):
    return np.concatenate([tx.pos[0].astype(np.float64), tx.ypr[0].astype(np.float64),
                           osc.mats[:, 0], osc.mats[:, 1]])


def _loss_rx_db(a, rx_of, n_rx):
    """Sum over receivers with paths of 10 log10(sum |a|^2)."""
    p = np.zeros(n_rx)
    np.add.at(p, rx_of, (np.abs(a) ** 2).sum(axis=(1, 2)))
    m = p > 0
    return float((10 * np.log10(p[m])).sum()), p


def test_received_power_gradient(prepared):
    tr, sc, tx, rx, osc, paths = prepared
    dev = tr.device
    eps = torch.tensor(sc.materials[:, 0], device=dev, requires_grad=True)
    sig = torch.tensor(sc.materials[:, 1], device=dev, requires_grad=True)
    pos = torch.tensor(tx.pos, device=dev, requires_grad=True)
    ypr = torch.tensor(tx.ypr, device=dev, requires_grad=True)
    a, tau = rt.CIR.apply(tr, eps, sig, pos, ypr)
    rx_of = torch.as_tensor(np.array([p.rx for p in paths]), device=dev)
    pw = torch.zeros(len(rx.pos), device=dev).index_add(0, rx_of, (a.abs() ** 2).sum(dim=(1, 2)))
    L = (10 * torch.log10(pw[pw > 0])).sum()
    L.backward()
    g_gpu = np.concatenate([pos.grad[0].cpu().numpy(), ypr.grad[0].cpu().numpy(), eps.grad.cpu().numpy(),
                            sig.grad.cpu().numpy()]).astype(np.float64)

    oa, otau, da, dtau = O.path_field(osc, FC, tx, rx, 0, paths, grad=True)
    rxo = np.array([p.rx for p in paths])
    L0, p = _loss_rx_db(oa, rxo, len(rx.pos))
    # dL/dtheta = sum_rx 10/(ln10 P_rx) sum 2 Re(conj(a) da/dtheta)
    w = 10.0 / (np.log(10.0) * p[rxo])
    g_ora = (w[:, None] * 2 * np.real(np.conj(oa)[..., None] * da).sum(axis=(1, 2))).sum(axis=0)
    assert abs(float(L.item()) - L0) < 1e-3 * abs(L0)

    # FP64 central differences of the oracle's loss (h = 1e-6 relative), paths frozen
    theta0 = _theta(osc, tx)
    g_fd = np.zeros_like(theta0)
    M = osc.M
    for k in range(len(theta0)):
        h = 1e-6 * max(abs(theta0[k]), 1.0)
        vals = []
        for sgn in (1, -1):
            t = theta0.copy()
            t[k] += sgn * h
            o2 = O.OScene(osc.V, osc.mat, np.stack([t[6:6 + M], t[6 + M:]], 1), osc.tmin, osc.eps)
            tx2 = S.Devices(t[None, :3], t[None, 3:6], tx.antenna)
            a2, _ = O.path_field(o2, FC, tx2, rx, 0, paths)
            vals.append(_loss_rx_db(a2, rxo, len(rx.pos))[0])
        g_fd[k] = (vals[0] - vals[1]) / (2 * h)
    scale = np.abs(g_ora).max()
    assert np.all(np.abs(g_fd - g_ora) <= 1e-6 * scale + 1e-6 * np.abs(g_ora))
    # 1e-3 relative per component; components below a tenth of their group's
    # largest are held to 1e-4 of that largest (FP32 tangents summed over paths)
    groups = [slice(0, 3), slice(3, 6), slice(6, 6 + M), slice(6 + M, 6 + 2 * M)]
    for gsl in groups:
        ref = g_ora[gsl]
        tol = GRAD_REL * np.maximum(np.abs(ref), 0.1 * np.abs(ref).max() + 1e-12)
        assert np.all(np.abs(g_gpu[gsl] - ref) <= tol), (gsl, g_gpu[gsl], ref)


def test_frequency_response_nmse_gradient(prepared):
    """Sec. III-A: NMSE between reference H and H with trainable materials."""
    tr, sc, tx, rx, osc, paths = prepared
    dev = tr.device
    freqs = O.subcarrier_freqs(128, 30e3)
    fr = torch.as_tensor(freqs, device=dev)
    # reference responses with the true materials
    a_ref, tau_ref = tr.cir()
    H_ref = tr.freq_response(a_ref, tau_ref, freqs).detach()
    # trainable materials at the paper's initial values (eps_r = 3, sigma = 0.1)
    eps = torch.full((osc.M,), 3.0, device=dev, requires_grad=True)
    sig = torch.full((osc.M,), 0.1, device=dev, requires_grad=True)
    pos = torch.tensor(tx.pos, device=dev, requires_grad=True)
    ypr = torch.tensor(tx.ypr, device=dev, requires_grad=True)
    a, tau = rt.CIR.apply(tr, eps, sig, pos, ypr)
    H = rt.FreqResponse.apply(tr, a, tau, fr)
    L = ((H - H_ref).abs() ** 2).sum() / (H_ref.abs() ** 2).sum()
    L.backward()
    g_gpu = np.concatenate([pos.grad[0].cpu().numpy(), ypr.grad[0].cpu().numpy(), eps.grad.cpu().numpy(),
                            sig.grad.cpu().numpy()]).astype(np.float64)
    tr.set_materials(sc.materials)

    # oracle: same loss and its gradient from dual-number tangents
    oa_ref, otau_ref = O.path_field(osc, FC, tx, rx, 0, paths)
    mats0 = np.stack([np.full(osc.M, 3.0), np.full(osc.M, 0.1)], 1)
    o2 = O.OScene(osc.V, osc.mat, mats0.astype(np.float32).astype(np.float64), osc.tmin, osc.eps)
    oa, otau, da, dtau = O.path_field(o2, FC, tx, rx, 0, paths, grad=True)
    rxo = np.array([p.rx for p in paths])
    num = 0.0
    den = 0.0
    g = np.zeros(da.shape[-1])
    for r in range(len(rx.pos)):
        idx = np.flatnonzero(rxo == r)
        if len(idx) == 0:
            continue
        Hr = O.freq_response(oa_ref[idx], otau_ref[idx], freqs)
        Hc = O.freq_response(oa[idx], otau[idx], freqs)
        ph = np.exp(-2j * np.pi * np.outer(otau[idx], freqs))              # [P, K]
        # dH/dtheta = sum_i (da_i - j 2 pi f tau'_i a_i) e^{-j 2 pi f tau_i}
        dH = (np.einsum("ipqg,ik->pqkg", da[idx], ph) +
              np.einsum("ipq,ik,ig,k->pqkg", oa[idx], ph, dtau[idx], -2j * np.pi * freqs))
        diff = Hc - Hr
        num += (np.abs(diff) ** 2).sum()
        den += (np.abs(Hr) ** 2).sum()
        g += 2 * np.real(np.conj(diff)[..., None] * dH).sum(axis=(0, 1, 2))
    g_ora = g / den
    assert abs(float(L.item()) - num / den) < 2e-3 * (num / den)
    M = osc.M
    for gsl in [slice(0, 3), slice(3, 6), slice(6, 6 + M), slice(6 + M, 6 + 2 * M)]:
        ref = g_ora[gsl]
        tol = GRAD_REL * np.maximum(np.abs(ref), 0.1 * np.abs(ref).max() + 1e-12)
        assert np.all(np.abs(g_gpu[gsl] - ref) <= tol), (gsl, g_gpu[gsl], ref)
