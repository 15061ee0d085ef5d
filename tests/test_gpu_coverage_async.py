"""Coverage map on the context's second stream (rt_coverage_map_async): the
same map as rt_coverage_map, unchanged paths and responses when the map runs
beside rt_compute_paths / rt_cir / rt_freq_response, and the automatic joins
of the calls that change what the map reads."""
import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import FC, gpu_paths, setup

pytestmark = pytest.mark.gpu

GRID = dict(x0=-250.0, y0=-250.0, cell=2.0, nx=250, ny=250, h=1.5)
N_RAYS, D = 400_003, 3


@pytest.fixture(scope="module")
def city():
    sc = S.city_scene(n_side=20, size=500.0, seed=1)
    tx, rx = S.city_devices(sc, n_rx=64, half=240.0)
    tr = rt.Tracer(0, FC)
    setup(tr, sc, tx, rx)
    yield tr, sc, tx, rx
    tr.close()


def _same_map(a, b):
    ga, ha = (x.cpu().numpy() for x in a)
    gb, hb = (x.cpu().numpy() for x in b)
    assert np.array_equal(ha, hb)            # ray counts per cell: order-free integers
    assert ha.sum() > 0
    # float atomics in another order: equal up to rounding of the sums
    np.testing.assert_allclose(ga, gb, rtol=2e-5, atol=1e-30)


@pytest.mark.parametrize("blocks_per_sm,after_trace", [(0, False), (1, False), (2, False), (0, True)])
def test_async_map_equals_sync(city, blocks_per_sm, after_trace):
    """With no path trace to wait for, a deferred map starts at the join."""
    tr = city[0]
    ref = tr.coverage_map(GRID, D, N_RAYS)
    got = tr.coverage_map_async(GRID, D, N_RAYS, blocks_per_sm=blocks_per_sm, after_trace=after_trace)
    tr.join()
    _same_map(ref, got)


@pytest.mark.parametrize("after_trace", [False, True])
def test_async_map_beside_paths(city, after_trace):
    """Paths, CIR and H(f) computed while the map traces equal those of a
    run without the map, and the map equals the sequential one."""
    tr = city[0]
    freqs = torch.linspace(-15e6, 15e6, 64, dtype=torch.float64, device=tr.device)
    ref_map = tr.coverage_map(GRID, D, N_RAYS)
    tr.compute_paths(D, N_RAYS)
    ref_sets = gpu_paths(tr)[0]
    a0, t0 = tr.cir()
    h0 = tr.freq_response(a0, t0, freqs)
    a0, t0, h0 = a0.clone(), t0.clone(), h0.clone()
    for _ in range(3):
        m = tr.coverage_map_async(GRID, D, N_RAYS, blocks_per_sm=2, after_trace=after_trace)
        tr.compute_paths(D, N_RAYS)
        a, t = tr.cir()
        h = tr.freq_response(a, t, freqs)
        tr.join()
        assert gpu_paths(tr)[0] == ref_sets
        assert torch.equal(a, a0) and torch.equal(t, t0) and torch.equal(h, h0)
        _same_map(ref_map, m)


@pytest.mark.parametrize("after_trace", [False, True])
def test_yielding_map_beside_paths_on_a_high_priority_stream(city, after_trace):
    """The default async map (short-lived blocks) beside the path calls of a
    higher-priority stream, as the bench runs it: paths, CIR, H(f) and the map
    equal those of the calls in order."""
    tr = city[0]
    freqs = torch.linspace(-15e6, 15e6, 64, dtype=torch.float64, device=tr.device)
    ref_map = tr.coverage_map(GRID, D, N_RAYS)
    tr.compute_paths(D, N_RAYS)
    ref_sets = gpu_paths(tr)[0]
    a0, t0 = tr.cir()
    h0 = tr.freq_response(a0, t0, freqs)
    a0, t0, h0 = a0.clone(), t0.clone(), h0.clone()
    torch.cuda.synchronize()
    hi = torch.cuda.Stream(device=tr.device, priority=-1)
    with torch.cuda.stream(hi):
        for _ in range(2):
            m = tr.coverage_map_async(GRID, D, N_RAYS, after_trace=after_trace)
            tr.compute_paths(D, N_RAYS)
            a, t = tr.cir()
            h = tr.freq_response(a, t, freqs)
            tr.join()
            hi.synchronize()
            assert gpu_paths(tr)[0] == ref_sets
            assert torch.equal(a, a0) and torch.equal(t, t0) and torch.equal(h, h0)
            _same_map(ref_map, m)
    torch.cuda.synchronize()
    tr.sync_stream()


@pytest.mark.parametrize("after_trace", [False, True])
def test_mutators_join_first(city, after_trace):
    """A scene load, a transmitter move or a frequency change right after
    the async map waits for it (a deferred map is started first): the map is
    that of the scene, pose and frequency it was requested with."""
    tr, sc, tx, rx = city
    ref = tr.coverage_map(GRID, D, N_RAYS)
    m = tr.coverage_map_async(GRID, D, N_RAYS, after_trace=after_trace)
    rt.rt_set_frequency(tr.ctx, 2 * FC)
    rt.rt_set_frequency(tr.ctx, FC)
    tr.join()
    _same_map(ref, m)
    m = tr.coverage_map_async(GRID, D, N_RAYS, after_trace=after_trace)
    other = S.city_scene(n_side=8, size=300.0, seed=9)
    tr.load_scene(other)
    tr.join()
    _same_map(ref, m)
    setup(tr, sc, tx, rx)
    m = tr.coverage_map_async(GRID, D, N_RAYS, after_trace=after_trace)
    moved = S.Devices(tx.pos + np.float32([40.0, 0.0, 0.0]), tx.ypr, tx.antenna)
    tr.set_devices(moved, rx)
    tr.join()
    _same_map(ref, m)
    setup(tr, sc, tx, rx)
    # another ray count rebuilds the ray order only after the map is done
    m = tr.coverage_map_async(GRID, D, N_RAYS, after_trace=after_trace)
    tr.compute_paths(D, 100_000)
    tr.join()
    _same_map(ref, m)


def test_async_argument_errors(city):
    tr = city[0]
    with pytest.raises(rt.RtError):
        tr.coverage_map_async(GRID, D, N_RAYS, blocks_per_sm=-1)
    g = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    gain = torch.empty((1, GRID["ny"], GRID["nx"]), dtype=torch.float32, device=tr.device)
    hits = torch.empty((1, GRID["ny"], GRID["nx"]), dtype=torch.int32, device=tr.device)
    with pytest.raises(rt.RtError):
        rt.rt_coverage_map_async(tr.ctx, g, D, N_RAYS, 0, gain, hits, flags=4)
    tr.join()
    # not while capturing a graph
    tr.sync_stream()
    rt.rt_graph_begin(tr.ctx)
    with pytest.raises(rt.RtError):
        rt.rt_coverage_map_async(tr.ctx, g, D, N_RAYS, 0, gain, hits)
    rt.rt_graph_end(tr.ctx)
    torch.cuda.synchronize()
