"""Batching (many transmitters, uneven receiver sets) in one persistent
launch, CUDA-graph capture and replay, and the launch-configuration
autotuner."""
import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, gpu_paths, setup

pytestmark = pytest.mark.gpu

GRID = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)


@pytest.fixture(scope="module")
def city():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    txs = S.rooftop_transmitters(sc, 5, half=70.0)
    rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    return sc, txs, rx


def test_multi_tx_coverage_matches_single_tx(city):
    sc, txs, rx = city
    tr = rt.Tracer(0, FC)
    setup(tr, sc, txs, rx)
    g_all, h_all = tr.coverage_map(GRID, 3, 50021, 0)
    for t in range(len(txs.pos)):
        one = S.Devices(txs.pos[t:t + 1], txs.ypr[t:t + 1], txs.antenna)
        tr.set_devices(one, rx)
        g, h = tr.coverage_map(GRID, 3, 50021, 0)
        assert torch.equal(h[0], h_all[t])
        assert torch.allclose(g[0], g_all[t], rtol=1e-5, atol=0)
    tr.close()


def test_multi_tx_paths_match_single_tx(city):
    sc, txs, _ = city
    _, rx = S.city_devices(sc, n_rx=12, half=70.0)
    tr = rt.Tracer(0, FC)
    off = [0, 3, 3, 10, 11, 12]          # uneven receiver sets, one empty
    setup(tr, sc, txs, rx, off)
    tr.compute_paths(3, 20000)
    gsets, _ = gpu_paths(tr)
    a_all, _ = tr.cir()
    for t in range(len(txs.pos)):
        if off[t] == off[t + 1]:
            continue
        one = S.Devices(txs.pos[t:t + 1], txs.ypr[t:t + 1], txs.antenna)
        sub = S.Devices(rx.pos[off[t]:off[t + 1]], rx.ypr[off[t]:off[t + 1]], rx.antenna)
        tr.set_devices(one, sub)
        tr.compute_paths(3, 20000)
        g1, _ = gpu_paths(tr)
        assert g1 == gsets[off[t]:off[t + 1]]
    tr.close()


def test_graph_capture_replay(city):
    sc, txs, rx = city
    tr = rt.Tracer(0, FC)
    setup(tr, sc, txs, rx)
    g_ref, h_ref = tr.coverage_map(GRID, 3, 40009, 0)       # also builds the ray order
    grid = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    gain = torch.zeros_like(g_ref)
    hits = torch.zeros_like(h_ref)
    rt.rt_graph_begin(tr.ctx)
    rt.rt_coverage_map(tr.ctx, grid, 3, 40009, 0, gain, hits)
    with pytest.raises(rt.RtError) as e:
        rt.rt_compute_paths(tr.ctx, 2, 100, rt.RT_LOS)
    assert e.value.code == -6
    rt.rt_graph_end(tr.ctx)
    assert int(hits.sum()) == 0            # recorded, not run
    for _ in range(2):
        rt.rt_graph_launch(tr.ctx)
        torch.cuda.synchronize()
        assert torch.equal(hits, h_ref)
        assert torch.allclose(gain, g_ref, rtol=1e-5, atol=0)
    # move the transmitters in place: the replay reads the new positions
    moved = S.Devices(txs.pos + np.float32([3.0, -2.0, 0.0]), txs.ypr, txs.antenna)
    tr.set_tx(moved.pos, moved.ypr, moved.antenna)
    rt.rt_graph_launch(tr.ctx)
    torch.cuda.synchronize()
    g2, h2 = tr.coverage_map(GRID, 3, 40009, 0)
    assert torch.equal(hits, h2)
    # a later call that reallocates a buffer the graph uses (a new ray count:
    # a larger ray order and direction table) invalidates the graph
    tr.coverage_map(GRID, 3, 2 * 40009, 0)
    with pytest.raises(rt.RtError) as e:
        rt.rt_graph_launch(tr.ctx)
    assert e.value.code == -6 and "capture the graph again" in str(e.value)
    tr.close()


def test_autotune_keeps_results(city, tmp_path):
    sc, txs, rx = city
    tr = rt.Tracer(0, FC)
    setup(tr, sc, txs, rx)
    g_ref, h_ref = tr.coverage_map(GRID, 3, 30011, 0)
    grid = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    cache = str(tmp_path / "tune.txt")
    rt.rt_autotune(tr.ctx, grid, 3, 30011, torch.empty_like(g_ref), torch.empty_like(h_ref), cache)
    b, c, s = rt.rt_get_tuning(tr.ctx)
    assert b in (128, 256) and s >= 0
    g, h = tr.coverage_map(GRID, 3, 30011, 0)
    assert torch.equal(h, h_ref)
    assert torch.allclose(g, g_ref, rtol=1e-5, atol=0)
    # a second context reuses the recorded choice
    tr2 = rt.Tracer(0, FC)
    setup(tr2, sc, txs, rx)
    rt.rt_autotune(tr2.ctx, grid, 3, 30011, torch.empty_like(g_ref), torch.empty_like(h_ref), cache)
    assert rt.rt_get_tuning(tr2.ctx) == (b, c, s)
    tr.close()
    tr2.close()
