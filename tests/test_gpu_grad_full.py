"""Gradients at the differentiation workload's full size (Sec. III-A / III-B:
material learning and transmitter orientation by gradient descent): the
seeded 4802-triangle city with 8 materials (eps_r ~ U(2, 8), sigma ~
logU(1e-3, 1)), 1 TR 38.901 dual-polarized transmitter, 256 receivers,
1e6 rays, max_depth 3.

Every path the GPU found is re-validated by the oracle's image method. The
replayed-path VJP kernels (rt_cir_backward, rt_freq_response_backward,
through the torch.autograd.Functions CIR and FreqResponse) are compared with
the oracle's dual-number gradient over all of those paths, per component,
for the 8 eps_r, the 8 sigma, the transmitter xyz and its yaw/pitch/roll,
and the oracle's gradient with FP64 central finite differences
(h = 1e-6 relative) of its own loss, paths frozen.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, GRAD_REL, gpu_paths, setup

pytestmark = pytest.mark.gpu

N, D, N_RX = 1_000_000, 3, 256


@pytest.fixture(scope="module")
def full():
    sc = S.city_scene(20, n_materials=8)
    tx, rx = S.city_devices(sc, n_rx=N_RX, tx_antenna=S.TR38901_VH)
    tx = S.Devices(tx.pos, np.array([[tx.ypr[0, 0], 0.12, 0.05]], np.float32), tx.antenna)
    tr = rt.Tracer(0, FC)
    setup(tr, sc, tx, rx)
    P = tr.compute_paths(D, N)
    gsets, _ = gpu_paths(tr)
    osc = O.make_scene(sc)
    for r, seqs in enumerate(gsets):
        for s in seqs:
            ok, _, _, m = O.image_path(osc, tx.pos[0], rx.pos[r], s)
            assert ok or m < osc.eps, f"rx {r}: GPU path {s} is invalid in the oracle (margin {m})"
    paths = [O.OPath(r, s, True, 1.0, None, 0.0) for r in range(N_RX) for s in gsets[r]]
    assert P == len(paths) and P > 20
    yield tr, sc, tx, rx, osc, paths
    tr.close()


GROUPS = lambda M: [("tx xyz", slice(0, 3)), ("tx ypr", slice(3, 6)), ("eps_r", slice(6, 6 + M)),
                    ("sigma", slice(6 + M, 6 + 2 * M))]


def _check_groups(g_gpu, g_ora, M, floor):
    """GRAD_REL relative per component; a component below `floor` of its
    group's largest is held to GRAD_REL * floor * that largest."""
    worst = {}
    for name, gsl in GROUPS(M):
        ref = g_ora[gsl]
        tol = GRAD_REL * np.maximum(np.abs(ref), floor * np.abs(ref).max() + 1e-30)
        err = np.abs(g_gpu[gsl] - ref)
        worst[name] = float((err / tol).max())
        assert np.all(err <= tol), (name, g_gpu[gsl], ref)
    return worst


def _loss_db(a, rxo, n_rx):
    p = np.zeros(n_rx)
    np.add.at(p, rxo, (np.abs(a) ** 2).sum(axis=(1, 2)))
    m = p > 0
    return float((10 * np.log10(p[m])).sum()), p


def test_received_power_gradient_full_size(full):
    """L = sum over receivers with paths of 10 log10(sum |a|^2)."""
    tr, sc, tx, rx, osc, paths = full
    dev = tr.device
    M = osc.M
    eps = torch.tensor(sc.materials[:, 0], device=dev, requires_grad=True)
    sig = torch.tensor(sc.materials[:, 1], device=dev, requires_grad=True)
    pos = torch.tensor(tx.pos, device=dev, requires_grad=True)
    ypr = torch.tensor(tx.ypr, device=dev, requires_grad=True)
    a, _ = rt.CIR.apply(tr, eps, sig, pos, ypr)
    rx_of = torch.as_tensor(np.array([p.rx for p in paths]), device=dev)
    pw = torch.zeros(N_RX, device=dev).index_add(0, rx_of, (a.abs() ** 2).sum(dim=(1, 2)))
    L = (10 * torch.log10(pw[pw > 0])).sum()
    L.backward()
    g_gpu = np.concatenate([pos.grad[0].cpu().numpy(), ypr.grad[0].cpu().numpy(), eps.grad.cpu().numpy(),
                            sig.grad.cpu().numpy()]).astype(np.float64)

    oa, _, da, _ = O.path_field(osc, FC, tx, rx, 0, paths, grad=True)
    rxo = np.array([p.rx for p in paths])
    L0, p = _loss_db(oa, rxo, N_RX)
    w = 10.0 / (np.log(10.0) * p[rxo])
    g_ora = (w[:, None] * 2 * np.real(np.conj(oa)[..., None] * da).sum(axis=(1, 2))).sum(axis=0)
    assert abs(float(L.item()) - L0) < 1e-4 * abs(L0)

    # the oracle's dual-number gradient against FP64 central differences
    theta0 = np.concatenate([tx.pos[0].astype(np.float64), tx.ypr[0].astype(np.float64),
                             osc.mats[:, 0], osc.mats[:, 1]])
    g_fd = np.zeros_like(theta0)
    for k in range(len(theta0)):
        h = 1e-6 * max(abs(theta0[k]), 1.0)
        vals = []
        for sgn in (1, -1):
            t = theta0.copy()
            t[k] += sgn * h
            o2 = O.OScene(osc.V, osc.mat, np.stack([t[6:6 + M], t[6 + M:]], 1), osc.tmin, osc.eps)
            a2, _ = O.path_field(o2, FC, S.Devices(t[None, :3], t[None, 3:6], tx.antenna), rx, 0, paths)
            vals.append(_loss_db(a2, rxo, N_RX)[0])
        g_fd[k] = (vals[0] - vals[1]) / (2 * h)
    scale = np.abs(g_ora).max()
    assert np.all(np.abs(g_fd - g_ora) <= 1e-6 * scale + 1e-5 * np.abs(g_ora))
    worst = _check_groups(g_gpu, g_ora, M, 0.1)
    print("received-power gradient, worst error / tolerance per group:", worst)


def test_nmse_gradient_full_size(full):
    """Sec. III-A: NMSE of the frequency responses (128 subcarriers of 30 kHz)
    between the true materials and trainable ones at eps_r = 3, sigma = 0.1."""
    tr, sc, tx, rx, osc, paths = full
    dev = tr.device
    M = osc.M
    freqs = O.subcarrier_freqs(128, 30e3)
    fr = torch.as_tensor(freqs, device=dev)
    a_ref, tau_ref = tr.cir()
    H_ref = tr.freq_response(a_ref, tau_ref, freqs).detach()
    eps = torch.full((M,), 3.0, device=dev, requires_grad=True)
    sig = torch.full((M,), 0.1, device=dev, requires_grad=True)
    pos = torch.tensor(tx.pos, device=dev, requires_grad=True)
    ypr = torch.tensor(tx.ypr, device=dev, requires_grad=True)
    a, tau = rt.CIR.apply(tr, eps, sig, pos, ypr)
    H = rt.FreqResponse.apply(tr, a, tau, fr)
    L = ((H - H_ref).abs() ** 2).sum() / (H_ref.abs() ** 2).sum()
    L.backward()
    g_gpu = np.concatenate([pos.grad[0].cpu().numpy(), ypr.grad[0].cpu().numpy(), eps.grad.cpu().numpy(),
                            sig.grad.cpu().numpy()]).astype(np.float64)
    tr.set_materials(sc.materials)

    oa_ref, otau_ref = O.path_field(osc, FC, tx, rx, 0, paths)
    mats0 = np.stack([np.full(M, 3.0), np.full(M, 0.1)], 1).astype(np.float32).astype(np.float64)
    o2 = O.OScene(osc.V, osc.mat, mats0, osc.tmin, osc.eps)
    oa, otau, da, dtau = O.path_field(o2, FC, tx, rx, 0, paths, grad=True)
    rxo = np.array([p.rx for p in paths])
    num = den = 0.0
    g = np.zeros(da.shape[-1])
    for r in np.unique(rxo):
        idx = np.flatnonzero(rxo == r)
        Hr = O.freq_response(oa_ref[idx], otau_ref[idx], freqs)
        Hc = O.freq_response(oa[idx], otau[idx], freqs)
        ph = np.exp(-2j * np.pi * np.outer(otau[idx], freqs))
        dH = (np.einsum("ipqg,ik->pqkg", da[idx], ph) +
              np.einsum("ipq,ik,ig,k->pqkg", oa[idx], ph, dtau[idx], -2j * np.pi * freqs))
        diff = Hc - Hr
        num += (np.abs(diff) ** 2).sum()
        den += (np.abs(Hr) ** 2).sum()
        g += 2 * np.real(np.conj(diff)[..., None] * dH).sum(axis=(0, 1, 2))
    g_ora = g / den
    assert abs(float(L.item()) - num / den) < 1e-3 * (num / den)
    worst = _check_groups(g_gpu, g_ora, M, 0.1)
    print("NMSE gradient, worst error / tolerance per group:", worst)
