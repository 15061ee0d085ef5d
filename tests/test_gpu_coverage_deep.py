"""Batched coverage maps at the batched workload's depth (Sec. II-A Listing 2,
coverage_map; max_depth 5): three rooftop transmitters (TR 38.901 pattern,
random azimuths, 25-60 m) traced in one persistent launch over a seeded
6 x 6 city, 100,003 Fibonacci rays each, 75 x 75 cells of 2 m at 1.5 m,
against the oracle's coverage estimator transmitter by transmitter.

Rays whose hit sequence (five reflections and the sixth segment) is
near-degenerate in the oracle for any of the transmitters may follow
another sequence in FP32; both sides are compared over the lattice
sub-ranges between them, which checks five-bounce reflection chains, the
FP32 field chain over five Fresnel/Jones steps and the per-transmitter map
offsets of the batched launch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2303_11103_gb300 import rt
from paper_2303_11103_gb300 import scenes as S

from gpu_helpers import A_REL, CM_DB, FC, setup

pytestmark = pytest.mark.gpu


def test_depth5_batched_coverage_matches_oracle():
    sc = S.city_scene(n_side=6, size=150.0, seed=5)
    txs = S.rooftop_transmitters(sc, 3, half=70.0)
    rx = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    grid = dict(x0=-75.0, y0=-75.0, cell=2.0, nx=75, ny=75, h=1.5)
    N, D = 100003, 5
    tr = rt.Tracer(0, FC)
    setup(tr, sc, txs, rx)
    osc = O.make_scene(sc)
    bad = []
    for t in range(3):
        _, marg = O.trace_sbr(osc, txs.pos[t], N, D + 1)
        bad.append(np.flatnonzero(marg[:, -1] < osc.eps))
    bad = np.unique(np.concatenate(bad))
    assert len(bad) < 0.03 * N
    edges = np.concatenate([[-1], bad, [N]])
    ranges = [(int(a + 1), int(b - a - 1)) for a, b in zip(edges[:-1], edges[1:]) if b - a > 1]
    g, h = tr.coverage_map_ranges(grid, D, N, ranges, 0)
    g, h = g.cpu().numpy().astype(np.float64), h.cpu().numpy()
    tr.close()
    for t in range(3):
        og = np.zeros((grid["ny"], grid["nx"]))
        oh, om = og.copy(), og.copy()
        for first, count in ranges:
            a, b, c = O.coverage(osc, FC, txs.pos[t], txs.ypr[t], txs.antenna, 0, rx.antenna, N, D, grid,
                                 first, first + count)
            og += a
            oh += b
            om += c
        clean = om == 0
        assert clean.mean() > 0.5
        assert np.array_equal(h[t][clean], oh[clean].astype(np.int64)), f"tx {t}: hit counts differ"
        sel = clean & (oh >= 16)
        assert sel.sum() > 50
        db = 10 * np.abs(np.log10(g[t][sel] / og[sel]))
        assert db.max() <= CM_DB, (t, db.max())
        # every cell: marginal mass plus the FP32 bound of the field chain
        assert np.all(np.abs(g[t] - og) <= om + 2 * A_REL * og + 1e-10 * og.max() + 1e-30)
        print(f"tx {t}: clean cells {clean.mean():.3f}, compared cells {int(sel.sum())}, "
              f"max |dB| {db.max():.2e}")
