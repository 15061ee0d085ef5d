"""CUDA path vs FP64 oracle, element by element on the same seeded inputs.

Sizes: tiny scenes and small seeded cities that the oracle finishes in
seconds, spanning several BVH levels, many warps of rays and ragged ray
counts; the full-size city (4802 triangles, 1000 receivers, 1e6 rays,
depth 3) in test_gpu_full_size.py on sampled outputs.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import (A_ABS, A_REL, CM_DB, FC, H_ABS, H_REL, TAU_REL, compare_candidates,
                         compare_path_sets, gpu_candidates, gpu_paths, setup)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    tr = rt.Tracer(0, FC)
    yield tr
    tr.close()


def _small_city(n_side=6, size=150.0, seed=5, n_materials=0):
    return S.city_scene(n_side=n_side, size=size, seed=seed, n_materials=n_materials)


# ------------------------------------------------------------------ launcher
def test_ray_directions_bitwise(tracer):
    N = 100003
    g = tracer.ray_directions(N).cpu().numpy()
    o = O.fibonacci(N).astype(np.float32)
    diff = np.abs(g.view(np.int32).astype(np.int64) - o.view(np.int32).astype(np.int64))
    assert diff.max() <= 1                 # at most one ulp (FP64 sin/cos of two libraries)
    assert (diff == 0).mean() > 0.9999
    sub = tracer.ray_directions(N, 777, 5).cpu().numpy()
    assert np.array_equal(sub, g[777:782])


# --------------------------------------------------------- traversal / SBR
@pytest.mark.parametrize("case", ["tiny_visible", "small_city"])
def test_ray_hits_match_oracle(tracer, case):
    if case == "tiny_visible":
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=True)
        N, D = 10000, 2
    else:
        sc = _small_city()
        tx, rx = S.city_devices(sc, n_rx=8, half=70.0)
        N, D = 30011, 3
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(D, N, record_rays=True)
    gh = tracer.ray_hits()[0].cpu().numpy()
    osc = O.make_scene(sc)
    oh, om = O.trace_sbr(osc, tx.pos[0], N, D)
    robust = om >= osc.eps
    assert robust.mean() > 0.98
    mism = (gh != oh) & robust
    assert mism.sum() == 0, f"{mism.sum()} non-degenerate ray hits differ"
    assert (gh[:, 0] >= 0).sum() > 100


# ------------------------------------------------------------- path sets
@pytest.mark.parametrize("case", ["tiny", "tiny_visible", "small_city", "small_city_multi_tx"])
def test_paths_match_oracle(tracer, case):
    if case.startswith("tiny"):
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=case == "tiny_visible")
        N, D = 10000, 2
    else:
        sc = _small_city()
        tx, rx = S.city_devices(sc, n_rx=24, half=70.0)
        N, D = 20000, 3
        if case == "small_city_multi_tx":
            tx = S.Devices(np.concatenate([tx.pos, tx.pos + np.float32([[6.0, -4.0, 5.0]])]),
                           np.concatenate([tx.ypr, tx.ypr + np.float32([[0.5, 0.0, 0.0]])]), tx.antenna)
    setup(tracer, sc, tx, rx)
    P = tracer.compute_paths(D, N)
    gsets, _ = gpu_paths(tracer)
    osc = O.make_scene(sc)
    n_rx = len(rx.pos)
    total_common = 0
    for t in range(len(tx.pos)):
        ora_paths, ora_c = O.compute_paths(osc, tx.pos[t], rx.pos, D, N)
        gc = gpu_candidates(tracer, t)
        compare_candidates(osc, tx.pos[t], N, D, gc, ora_c)
        common = compare_path_sets(osc, tx.pos[t], rx.pos, gsets[t * n_rx:(t + 1) * n_rx], ora_paths, ora_c)
        total_common += sum(len(v) for v in common.values())
    if case == "tiny":
        assert P == 0
    elif case == "tiny_visible":
        assert sorted(gsets[0]) == sorted([(), (1,), (12,), (12, 1)])
    else:
        assert total_common > 20


def test_uneven_rx_sets(tracer):
    sc = _small_city()
    tx, rx = S.city_devices(sc, n_rx=30, half=70.0)
    tx2 = S.Devices(np.concatenate([tx.pos, tx.pos + np.float32([[-5.0, 3.0, 2.0]]), tx.pos + np.float32([[4.0, 4.0, 0.0]])]),
                    np.zeros((3, 3), np.float32), tx.antenna)
    off = [0, 5, 5, 30]   # uneven, with an empty set
    setup(tracer, sc, tx2, rx, off)
    N, D = 12000, 2
    tracer.compute_paths(D, N)
    gsets, _ = gpu_paths(tracer)
    assert tracer.n_pairs == 30
    osc = O.make_scene(sc)
    for t in range(3):
        rxs = rx.pos[off[t]:off[t + 1]]
        if len(rxs) == 0:
            continue
        ora_paths, ora_c = O.compute_paths(osc, tx2.pos[t], rxs, D, N)
        compare_path_sets(osc, tx2.pos[t], rxs, gsets[off[t]:off[t + 1]], ora_paths, ora_c)


# ------------------------------------------------------------------ CIR
def _field_case(tracer, sc, tx, rx, N, D):
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(D, N)
    gsets, p = gpu_paths(tracer)
    a, tau = tracer.cir()
    a = a.cpu().numpy()
    tau = tau.cpu().numpy()
    osc = O.make_scene(sc)
    ora_paths, ora_c = O.compute_paths(osc, tx.pos[0], rx.pos, D, N)
    common = compare_path_sets(osc, tx.pos[0], rx.pos, gsets, ora_paths, ora_c)
    sel = [q for q in ora_paths if q.valid]
    oa, otau = O.path_field(osc, FC, tx, rx, 0, sel)
    off = p["offsets"].cpu().numpy()
    return gsets, a, tau, off, sel, oa, otau, common


@pytest.mark.parametrize("case", ["tiny_visible", "small_city_tr38901_vh"])
def test_cir_matches_oracle(tracer, case):
    if case == "tiny_visible":
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=True)
        N, D = 10000, 2
    else:
        sc = _small_city()
        tx, rx = S.city_devices(sc, n_rx=24, half=70.0)
        rx = S.Devices(rx.pos, rx.ypr + np.float32([0.3, 0.1, 0.0]), S.Antenna(S.ANT_DIPOLE, (np.pi / 4, -np.pi / 4)))
        N, D = 20000, 3
    gsets, a, tau, off, sel, oa, otau, common = _field_case(tracer, sc, tx, rx, N, D)
    idx = {(q.rx, q.seq): i for i, q in enumerate(sel)}
    n = 0
    for r in range(len(rx.pos)):
        amax = max([np.abs(oa[idx[(r, s)]]).max() for s in common[r]] + [0.0])
        for k, s in enumerate(gsets[r]):
            if s not in common[r]:
                continue
            i = off[r] + k
            j = idx[(r, s)]
            assert abs(tau[i] - otau[j]) <= TAU_REL * otau[j]
            err = np.abs(a[i] - oa[j])
            assert np.all(err <= A_REL * np.abs(oa[j]) + A_ABS * amax), (s, a[i], oa[j])
            n += 1
    assert n >= 4


def test_cir_flags(tracer):
    sc = S.tiny_scene()
    tx, rx = S.tiny_devices(visible=True)
    setup(tracer, sc, tx, rx)
    tracer.compute_paths(2, 10000)
    dep = tracer.paths()["depth"].cpu().numpy()
    a_all, _ = tracer.cir()
    a_los, _ = tracer.cir(los=True, reflection=False)
    a_ref, _ = tracer.cir(los=False, reflection=True)
    a_all, a_los, a_ref = (x.cpu().numpy() for x in (a_all, a_los, a_ref))
    assert np.all(a_los[dep > 0] == 0) and np.array_equal(a_los[dep == 0], a_all[dep == 0])
    assert np.all(a_ref[dep == 0] == 0) and np.array_equal(a_ref[dep > 0], a_all[dep > 0])
    # LOS only (max_depth 0)
    assert tracer.compute_paths(0, 0) == 1


# ---------------------------------------------------------------- H(f)
@pytest.mark.parametrize("uniform", [True, False])
def test_freq_response_matches_oracle(tracer, uniform):
    sc = _small_city()
    tx, rx = S.city_devices(sc, n_rx=24, half=70.0)
    gsets, a, tau, off, sel, oa, otau, common = _field_case(tracer, sc, tx, rx, 20000, 3)
    if uniform:
        freqs = O.subcarrier_freqs(1000, 30e3)     # ragged vs the 8-subcarrier runs
    else:
        freqs = np.sort(np.random.default_rng(3).uniform(-15e6, 15e6, 333))
    H = tracer.freq_response(torch.as_tensor(a).cuda(), torch.as_tensor(tau).cuda(), freqs).cpu().numpy()
    for r in range(len(rx.pos)):
        b, e = off[r], off[r + 1]
        # the kernel against the oracle's direct sum on the same (a, tau)
        Hk = O.freq_response(a[b:e].astype(np.complex128), tau[b:e].astype(np.float64), freqs)
        scale = np.abs(a[b:e]).sum(axis=0)[..., None] if e > b else 0.0
        assert np.all(np.abs(H[r] - Hk) <= H_REL * np.abs(Hk) + H_ABS * scale + 1e-30)
        # end to end against the oracle's paths when the path sets agree
        ora = [i for i, q in enumerate(sel) if q.rx == r]
        if sorted(q.seq for q in (sel[i] for i in ora)) == sorted(gsets[r]) and ora:
            Ho = O.freq_response(oa[ora], otau[ora], freqs)
            sc2 = np.abs(oa[ora]).sum(axis=0)[..., None]
            assert np.all(np.abs(H[r] - Ho) <= H_REL * np.abs(Ho) + H_ABS * sc2 + 1e-30)


# ------------------------------------------------------------ coverage map
@pytest.mark.parametrize("case", ["tiny_visible", "small_city"])
def test_coverage_matches_oracle(tracer, case):
    if case == "tiny_visible":
        sc = S.tiny_scene()
        tx, rx = S.tiny_devices(visible=True)
        grid = dict(x0=-100.0, y0=-100.0, cell=4.0, nx=50, ny=50, h=1.5)
        N, D = 100003, 2
    else:
        sc = _small_city()
        tx, _ = S.city_devices(sc, n_rx=1, half=70.0, tx_antenna=S.TR38901_VH)
        rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
        grid = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)
        N, D = 100003, 3
    setup(tracer, sc, tx, rx)
    osc = O.make_scene(sc)
    # Rays whose hit sequence is near-degenerate in the oracle may follow
    # another sequence in FP32: compare both sides over the other rays
    # (lattice sub-ranges between them).
    _, marg = O.trace_sbr(osc, tx.pos[0], N, D + 1)
    bad = np.flatnonzero(marg[:, -1] < osc.eps)
    assert len(bad) < 0.01 * N
    edges = np.concatenate([[-1], bad, [N]])
    ranges = [(int(a + 1), int(b - a - 1)) for a, b in zip(edges[:-1], edges[1:]) if b - a > 1]
    for port in range(tx.antenna.n_ports):
        g, h = tracer.coverage_map_ranges(grid, D, N, ranges, port)
        g, h = g[0].cpu().numpy().astype(np.float64), h[0].cpu().numpy()
        og = np.zeros((grid["ny"], grid["nx"]))
        oh, om = og.copy(), og.copy()
        for first, count in ranges:
            a, b, c = O.coverage(osc, FC, tx.pos[0], tx.ypr[0], tx.antenna, port, rx.antenna, N, D, grid,
                                 first, first + count)
            og += a
            oh += b
            om += c
        clean = om == 0
        assert clean.mean() > 0.6
        assert np.array_equal(h[clean], oh[clean].astype(np.int64))
        sel = clean & (oh >= 16)
        assert sel.sum() > 50
        db = 10 * np.abs(np.log10(g[sel] / og[sel]))
        assert db.max() <= CM_DB
        # every cell: the marginal mass (crossings near a cell edge) plus the
        # FP32 bound of the a_i rule applied to power (2e-3 relative, and a
        # floor relative to the strongest cell for cross-polarised residues
        # where the receive projection cancels)
        assert np.all(np.abs(g - og) <= om + 2 * A_REL * og + 1e-10 * og.max() + 1e-30)
    # the full map equals the sum over the partition of the lattice
    g_full, h_full = tracer.coverage_map(grid, D, N, 0)
    g_part, h_part = tracer.coverage_map_ranges(grid, D, N, [(0, N // 3), (N // 3, N - N // 3)], 0)
    assert torch.equal(h_full, h_part)
    assert torch.allclose(g_full, g_part, rtol=1e-5, atol=0)
