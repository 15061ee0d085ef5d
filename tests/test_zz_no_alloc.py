"""rt_coverage_map_noalloc: the coverage map for callers that must not
allocate device memory at call time (a host whose device memory belongs to
another allocator, latency-critical loops, plug-ins barred from allocating).
It must give rt_coverage_map's result, through the C ABI, on consecutive
calls that share its static scratch, and reject sizes above its limit.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest
import torch

from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

pytestmark = pytest.mark.gpu

GRID = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)


def test_noalloc_matches_coverage_map():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    txs = S.rooftop_transmitters(sc, 3, half=70.0, antenna=S.TR38901_VH)
    rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    tr = rt.Tracer(0, 3.5e9)
    tr.load_scene(sc)
    tr.set_devices(txs, rx)
    grid = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    n_rays, depth = 200003, 3
    for port in (0, 1):
        g_ref, h_ref = tr.coverage_map(GRID, depth, n_rays, port)
        gain = torch.empty_like(g_ref)
        hits = torch.empty_like(h_ref)
        for call in range(2):                       # consecutive calls share the scratch
            gain.fill_(123.0)
            hits.fill_(7)
            rt.rt_coverage_map_noalloc(tr.ctx, grid, depth, n_rays, port, gain, hits)
            torch.cuda.synchronize()
            assert torch.equal(hits, h_ref), f"port {port} call {call}: hit counts differ"
            assert torch.allclose(gain, g_ref, rtol=1e-5, atol=0), f"port {port} call {call}"
    # the device memory in use does not change across a call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rt.rt_coverage_map_noalloc(tr.ctx, grid, depth, n_rays, 0, gain, hits)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1
    # max_depth 0 (line of sight only) on a stream other than the default one
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        rt.rt_set_stream(tr.ctx)
        g0, h0 = tr.coverage_map(GRID, 0, n_rays, 0)
        gain.fill_(123.0)
        hits.fill_(7)
        rt.rt_coverage_map_noalloc(tr.ctx, grid, 0, n_rays, 0, gain, hits)
    side.synchronize()
    assert int(h0.sum()) > 0 and torch.equal(hits, h0)
    assert torch.allclose(gain, g0, rtol=1e-5, atol=0)
    rt.rt_set_stream(tr.ctx)
    # captured in a CUDA graph after the warm-up calls above, then replayed
    # twice: every replay reuses the static array and must give the result
    gain.fill_(123.0)
    hits.fill_(7)
    rt.rt_graph_begin(tr.ctx)
    rt.rt_coverage_map_noalloc(tr.ctx, grid, depth, n_rays, 1, gain, hits)
    rt.rt_graph_end(tr.ctx)
    g_ref, h_ref = tr.coverage_map(GRID, depth, n_rays, 1)
    for replay in range(2):
        gain.fill_(123.0)
        hits.fill_(7)
        rt.rt_graph_launch(tr.ctx)
        torch.cuda.synchronize()
        assert torch.equal(hits, h_ref), f"replay {replay}: hit counts differ"
        assert torch.allclose(gain, g_ref, rtol=1e-5, atol=0), f"replay {replay}"
    # a size beyond the static scratch is rejected with a clear error
    with pytest.raises(rt.RtError) as e:
        rt.rt_coverage_map_noalloc(tr.ctx, grid, depth, (1 << 20) + 1, 0, gain, hits)
    assert e.value.code == -1 and "RT_NOALLOC_MAX_RAYS" in str(e.value)
    tr.close()
