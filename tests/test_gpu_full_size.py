"""Full-size city workload (4802 triangles, 1 TR 38.901 dual-polarized Tx,
1000 receivers, 1e6 rays, max_depth 3, 1024 subcarriers) in the launch
configuration bench.py times, checked on outputs the oracle can compute
one by one: a sample of rays (per-ray hit lists), every receiver with paths
plus 20 without (image method of every GPU candidate, CIR, H(f)), and a
sampled ray range of the coverage map."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_ABS, A_REL, CM_DB, FC, H_ABS, H_REL, TAU_REL, gpu_candidates, gpu_paths, setup

pytestmark = pytest.mark.gpu

N, D = 1_000_000, 3


@pytest.fixture(scope="module")
def city():
    sc = S.city_scene(20)
    tx, rx = S.city_devices(sc, n_rx=1000)
    tr = rt.Tracer(0, FC)
    setup(tr, sc, tx, rx)
    P = tr.compute_paths(D, N, record_rays=True)
    yield tr, sc, tx, rx, O.make_scene(sc), P
    tr.close()


def test_full_size_ray_hits(city):
    tr, sc, tx, rx, osc, P = city
    assert sc.n_tris == 4802
    gh = tr.ray_hits()[0].cpu().numpy()
    rng = np.random.default_rng(0)
    ids = np.sort(rng.choice(N, 3000, replace=False))
    oh, om = O.trace_sbr(osc, tx.pos[0], N, D, ids)
    robust = om >= osc.eps
    assert robust.mean() > 0.97
    assert ((gh[ids] != oh) & robust).sum() == 0


def test_full_size_paths_cir_freq(city):
    tr, sc, tx, rx, osc, P = city
    assert P > 100   # dense city: most street receivers are fully shadowed
    gsets, p = gpu_paths(tr)
    off = p["offsets"].cpu().numpy()
    gc = gpu_candidates(tr, 0)
    seqs = sorted(gc.keys(), key=lambda s: (len(s), s))
    a, tau = tr.cir()
    a, tau = a.cpu().numpy(), tau.cpu().numpy()
    freqs = O.subcarrier_freqs(1024, 30e3)
    H = tr.freq_response(torch.as_tensor(a).cuda(), torch.as_tensor(tau).cuda(), freqs).cpu().numpy()
    rng = np.random.default_rng(1)
    # every receiver with GPU paths, and 20 receivers without
    with_paths = [r for r in range(len(rx.pos)) if gsets[r]]
    without = [r for r in range(len(rx.pos)) if not gsets[r]]
    sample = np.sort(np.concatenate([np.array(with_paths, np.int64),
                                     rng.choice(without, min(20, len(without)), replace=False)]))
    # the oracle's image method of every candidate against every sampled receiver, in one call
    c_all, r_all, v_all, m_all = O.validate(osc, tx.pos[0], rx.pos[sample], seqs, D)
    n_checked = 0
    for si, r in enumerate(sample):
        sel = r_all == si
        c, v, m = c_all[sel], v_all[sel], m_all[sel]
        valid = {seqs[ci] for ci, vi, mi in zip(c, v, m) if vi}
        near = {seqs[ci] for ci, vi, mi in zip(c, v, m) if mi < osc.eps}
        g = set(gsets[r])
        assert (valid - near) <= g, f"rx {r}: oracle-valid candidates missing on the GPU"
        assert g <= (valid | near), f"rx {r}: GPU paths the oracle rejects"
        robust = sorted(valid - near, key=lambda s: (len(s), s))
        paths = [O.OPath(int(r), s, True, 1.0, None, 0.0) for s in robust]
        rxd = S.Devices(rx.pos, rx.ypr, rx.antenna)
        oa, otau = O.path_field(osc, FC, tx, rxd, 0, paths)
        amax = np.abs(oa).max() if len(oa) else 0.0
        for j, s in enumerate(robust):
            i = off[r] + gsets[r].index(s)
            assert abs(tau[i] - otau[j]) <= TAU_REL * otau[j]
            assert np.all(np.abs(a[i] - oa[j]) <= A_REL * np.abs(oa[j]) + A_ABS * amax)
            n_checked += 1
        b, e = off[r], off[r + 1]
        Hk = O.freq_response(a[b:e].astype(np.complex128), tau[b:e].astype(np.float64), freqs)
        scale = np.abs(a[b:e]).sum(axis=0)[..., None] if e > b else 0.0
        assert np.all(np.abs(H[r] - Hk) <= H_REL * np.abs(Hk) + H_ABS * scale + 1e-30)
    assert n_checked > 0.9 * P, (n_checked, P)


def test_full_size_coverage_sample(city):
    tr, sc, tx, rx, osc, P = city
    grid = dict(x0=-250.0, y0=-250.0, cell=1.0, nx=500, ny=500, h=1.5)
    first, count = 600_000, 60_000          # a lattice sub-range of the 1e6-ray map (z < 0: downward)
    ids = np.arange(first, first + count)
    _, marg = O.trace_sbr(osc, tx.pos[0], N, D + 1, ids)
    bad = ids[marg[:, -1] < osc.eps]
    edges = np.concatenate([[first - 1], bad, [first + count]])
    ranges = [(int(a + 1), int(b - a - 1)) for a, b in zip(edges[:-1], edges[1:]) if b - a > 1]
    g, h = tr.coverage_map_ranges(grid, D, N, ranges, 0)
    g, h = g[0].cpu().numpy().astype(np.float64), h[0].cpu().numpy()
    og = np.zeros((500, 500))
    oh, om = og.copy(), og.copy()
    for f0, c0 in ranges:
        x, y, z = O.coverage(osc, FC, tx.pos[0], tx.ypr[0], tx.antenna, 0, rx.antenna, N, D, grid, f0, f0 + c0)
        og += x
        oh += y
        om += z
    clean = om == 0
    assert np.array_equal(h[clean], oh[clean].astype(np.int64))
    touched = clean & (oh > 0)
    assert touched.sum() > 300
    rel = np.abs(g[touched] - og[touched]) / og[touched]
    assert rel.max() < 1e-4
    assert np.all(np.abs(g - og) <= om + 1e-4 * og + 1e-30)
    sel = clean & (oh >= 16)
    if sel.any():
        assert (10 * np.abs(np.log10(g[sel] / og[sel]))).max() <= CM_DB
